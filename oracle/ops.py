"""CPU FP64 oracle for the element-wise HMAT operations and the diagonalisation
data movement (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the product path never
imports it.  Plain numpy, each function written from the passage it cites.

* :func:`scale`   - complex scaling alpha q, Sec. III (the alpha q formula:
  component e of the real part takes alpha_R M_e - alpha_I M_{e+4}, of the
  imaginary part alpha_R M_{e+4} + alpha_I M_e).
* :func:`add`     - component-wise addition, Sec. III (addition formula).
* :func:`trace`   - Tr[q] = 2 (Tr[M1] + i Tr[M5]) for square q, Sec. III.
* :func:`hermiticity_deviation` - largest |(q - q^dagger)_c| over the eight
  stored components, with q^dagger from the Hermitian-conjugation sign pattern
  of Sec. III; zero exactly when the complex image of Sec. III is Hermitian.
* :func:`hadamard_block` - Sec. III C (Hadamard transformation for
  diagonalisation): for a block anti-diagonal complex image
  M = [[0, A], [B, 0]] and a unit scalar alpha, M' = U_alpha^dagger M U_alpha
  with U_alpha = [[I, I], [alpha I, -alpha I]] / sqrt(2) (Eq.
  hadamard_general_transform); returns the upper-left block of M' and the
  largest magnitude in its lower-left block (zero when the reduction to
  Eq. reduced-hadamard-pure holds).

The op argument takes N, T, C, H and QC as in :func:`oracle.apply_op`.
"""
from __future__ import annotations

import numpy as np

from . import apply_op
from .isomorph import to_isomorph


def _op(op, X):
    return np.asarray(X, dtype=np.float64) if op == "N" else apply_op(op, X)


def scale(X: np.ndarray, alpha, op="N") -> np.ndarray:
    """alpha op(X) by the component formula of Sec. III."""
    M = _op(op, X)
    a = complex(alpha)
    out = np.empty_like(M)
    for e in range(4):
        out[e] = a.real * M[e] - a.imag * M[e + 4]
        out[e + 4] = a.real * M[e + 4] + a.imag * M[e]
    return out


def add(X: np.ndarray, Y: np.ndarray, alpha=1.0, beta=1.0, opX="N", opY="N") -> np.ndarray:
    """alpha op(X) + beta op(Y): the addition formula of Sec. III applied to two
    scaled operands (alpha = beta = 1 is the paper's plain sum)."""
    return scale(X, alpha, opX) + scale(Y, beta, opY)


def trace(X: np.ndarray, op="N") -> complex:
    """Tr[op(q)] = 2 (Tr[M1] + i Tr[M5]) of the (op-transformed) components."""
    M = _op(op, X)
    if M.shape[1] != M.shape[2]:
        raise ValueError("trace needs a square matrix")
    return 2.0 * complex(np.trace(M[0]), np.trace(M[4]))


def hermiticity_deviation(X: np.ndarray) -> float:
    """max over components and entries of |q - q^dagger| (0 for a Hermitian q)."""
    X = np.asarray(X, dtype=np.float64)
    if X.shape[1] != X.shape[2]:
        raise ValueError("Hermiticity needs a square matrix")
    return float(np.max(np.abs(X - apply_op("H", X)))) if X.size else 0.0


def hadamard_block(X: np.ndarray, alpha):
    """(M'_11, max |M'_21|) for the complex image M of X and the unit scalar alpha.

    Steps in the order of Sec. III C: form the complex image (M+ + M- blocks),
    form U_alpha, transform M' = U_alpha^dagger M U_alpha with numpy matmul,
    read the blocks."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[1]
    M = to_isomorph(X)
    a = complex(alpha)
    I = np.eye(n)
    U = np.block([[I, I], [a * I, -a * I]]) / np.sqrt(2.0)
    Mp = U.conj().T @ M @ U
    return Mp[:n, :n], (float(np.max(np.abs(Mp[n:, :n]))) if n else 0.0)


def antidiagonal_blocks(X: np.ndarray):
    """(A, B, max |diagonal blocks|) of the complex image [[P, A], [B, Q]] of X."""
    M = to_isomorph(np.asarray(X, dtype=np.float64))
    n = X.shape[1]
    diag = max(float(np.max(np.abs(M[:n, :n]))) if n else 0.0, float(np.max(np.abs(M[n:, n:]))) if n else 0.0)
    return M[:n, n:], M[n:, :n], diag
