"""Independent cross-check: the isomorphic complex 2m x 2n representation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. II A, Eq. TRG-in-C; Sec. III, the M+ and M- block forms and
Eq. mapping-formulas) identifies an m x n biquaternion matrix stored as
[M1..M8] = [E_R, E_I, F_R, F_I, G_I, -G_R, H_I, -H_R] with the complex
2m x 2n matrix

    M = M+ + M- ,  M+ = [[E, F], [-F*, E*]],  M- = [[G, H], [H*, -G*]]

and gives the inverse map E = (A + D*)/2, F = (B - C*)/2, G = (A - D*)/2,
H = (B + C*)/2 for M = [[A, B], [C, D]].  In this representation the product
of biquaternion matrices is the ordinary complex matrix product (Sec. II A,
the M1 M2 = Q1 Q2 equivalence), transposition is the plain transpose, complex
conjugation is the element-wise conjugate and Hermitian conjugation is the
conjugate transpose (Sec. III).  Quaternion conjugation maps the 2 x 2 block
pattern [[A, B], [C, D]] to [[D, -B], [-C, A]] (the adjugate of each 2 x 2
Pauli pattern, q1 I + q2 i sz + q3 i sy + q4 i sx -> q1 I - ...).

Nothing here uses the component-wise product of oracle.c; the matrix product
is numpy's complex matmul (a library primitive serving as one step).
"""
from __future__ import annotations

import numpy as np


def to_isomorph(M: np.ndarray) -> np.ndarray:
    """8 x m x n real components -> complex 2m x 2n matrix (M+ + M- blocks)."""
    M = np.asarray(M, dtype=np.float64)
    E = M[0] + 1j * M[1]
    F = M[2] + 1j * M[3]
    G = -M[5] + 1j * M[4]      # M5 = G_I, M6 = -G_R
    H = -M[7] + 1j * M[6]      # M7 = H_I, M8 = -H_R
    top = np.concatenate([E + G, F + H], axis=1)
    bot = np.concatenate([-np.conj(F) + np.conj(H), np.conj(E) - np.conj(G)], axis=1)
    return np.concatenate([top, bot], axis=0)


def from_isomorph(X: np.ndarray) -> np.ndarray:
    """complex 2m x 2n matrix -> 8 x m x n components via Eq. mapping-formulas."""
    X = np.asarray(X, dtype=np.complex128)
    m, n = X.shape[0] // 2, X.shape[1] // 2
    A, B = X[:m, :n], X[:m, n:]
    C, D = X[m:, :n], X[m:, n:]
    E = (A + np.conj(D)) / 2
    F = (B - np.conj(C)) / 2
    G = (A - np.conj(D)) / 2
    H = (B + np.conj(C)) / 2
    return np.stack([E.real, E.imag, F.real, F.imag, G.imag, -G.real, H.imag, -H.real])


def iso_op(op: str, X: np.ndarray) -> np.ndarray:
    """op on the complex representation: N, T, C (conjugate), H (dagger), QC."""
    if op == "N":
        return X
    if op == "T":
        return X.T.copy()
    if op == "C":
        return np.conj(X)
    if op == "H":
        return np.conj(X).T.copy()
    if op == "QC":
        m, n = X.shape[0] // 2, X.shape[1] // 2
        A, B = X[:m, :n], X[:m, n:]
        C, D = X[m:, :n], X[m:, n:]
        return np.block([[D, -B], [-C, A]])
    raise ValueError(op)


def iso_bq_gemm(A: np.ndarray, B: np.ndarray, opA="N", opB="N", alpha=1.0, beta=0.0,
                C: np.ndarray | None = None) -> np.ndarray:
    """alpha op(A) op(B) + beta C computed on the complex isomorph; returns 8 x m x n."""
    XA = iso_op(opA, to_isomorph(A))
    XB = iso_op(opB, to_isomorph(B))
    XC = complex(alpha) * (XA @ XB)
    if complex(beta) != 0:
        XC = XC + complex(beta) * to_isomorph(C)
    return from_isomorph(XC)


def iso_trace(M: np.ndarray) -> complex:
    """Trace of the complex representation of a square biquaternion matrix."""
    return complex(np.trace(to_isomorph(M)))
