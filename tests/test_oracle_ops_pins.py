"""Pins of the element-wise / mapping / Hadamard oracle (oracle/ops.py).

Each check computes the same quantity another way: on the complex 2n x 2n
image with numpy (the scalar, sum, trace and dagger of a complex matrix), by a
closed form the paper prints (Eq. reduced-hadamard-pure, Eq.
hadamard_general_transform), or by the spectrum (numpy eigvalsh).
"""
import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
from oracle import isomorph as iso
from oracle import ops

OPS = ["N", "T", "C", "H", "QC"]


def _rand(seed, r, c, flags=bi.BQ):
    return bi.uniform(seed, r, c, flags=flags).numpy().copy()


@pytest.mark.parametrize("op", OPS)
def test_scale_is_the_complex_scalar_of_the_image(op):
    """Sec. III alpha q formula == alpha times the complex image (Sec. III M+/M- blocks)."""
    X = _rand(200, 5, 7)
    alpha = 0.75 - 1.25j
    got = iso.to_isomorph(ops.scale(X, alpha, op))
    want = alpha * iso.iso_op(op, iso.to_isomorph(X))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def test_scale_by_i_twice_negates():
    X = _rand(201, 4, 4)
    np.testing.assert_array_equal(ops.scale(ops.scale(X, 1j), 1j), -X)


@pytest.mark.parametrize("opX,opY", [("N", "N"), ("T", "H"), ("C", "QC"), ("H", "N")])
def test_add_is_the_sum_of_images(opX, opY):
    X = _rand(202, 6, 3)
    tr = {"T", "H"}
    Y = _rand(203, 6, 3) if (opX in tr) == (opY in tr) else _rand(203, 3, 6)
    a, b = 2 - 1j, -0.5 + 3j
    got = iso.to_isomorph(ops.add(X, Y, a, b, opX, opY))
    want = a * iso.iso_op(opX, iso.to_isomorph(X)) + b * iso.iso_op(opY, iso.to_isomorph(Y))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_plain_add_is_componentwise():
    X = bi.small_int(204, 3, 4).numpy()
    Y = bi.small_int(205, 3, 4).numpy()
    np.testing.assert_array_equal(ops.add(X, Y), X + Y)


@pytest.mark.parametrize("op", OPS)
def test_trace_is_the_trace_of_the_image(op):
    """Tr[q] = 2(Tr M1 + i Tr M5) equals the trace of the complex image."""
    X = _rand(206, 9, 9)
    got = ops.trace(X, op)
    want = np.trace(iso.iso_op(op, iso.to_isomorph(X)))
    assert abs(got - want) < 1e-13


def test_trace_identity_and_cyclic():
    n = 6
    I = np.zeros((8, n, n))
    I[0] = np.eye(n)
    assert ops.trace(I) == 2 * n
    X = _rand(207, n, n)
    Y = _rand(208, n, n)
    t1 = ops.trace(oracle.bq_gemm(X, Y))
    t2 = ops.trace(oracle.bq_gemm(Y, X))
    assert abs(t1 - t2) < 1e-12


def test_hermiticity_matches_the_image():
    X = _rand(209, 7, 7)
    Hm = X + oracle.apply_op("H", X)
    assert ops.hermiticity_deviation(Hm) == 0.0
    Z = iso.to_isomorph(Hm)
    np.testing.assert_allclose(Z, Z.conj().T, rtol=0, atol=1e-14)
    # a non-Hermitian q has a non-Hermitian image
    assert ops.hermiticity_deviation(X) > 0.1
    Zx = iso.to_isomorph(X)
    assert np.max(np.abs(Zx - Zx.conj().T)) > 0.1
    # a planted asymmetry of size d in M1 shows up exactly
    P = Hm.copy()
    P[0, 1, 2] += 0.125
    assert ops.hermiticity_deviation(P) == 0.125


def _hermitian(seed, n, flags):
    X = _rand(seed, n, n, flags)
    return bi.apply_flags(torch.from_numpy(X + oracle.apply_op("H", X)), flags).numpy()


@pytest.mark.parametrize("sign", [1, -1])
def test_hadamard_pure_j(sign):
    """Pure j (F_R + i H_I; components M3, M7): alpha = +-i gives
    diag(alpha A, -alpha A) with A = F_R + i H_I (Eq. reduced-hadamard-pure)."""
    n = 8
    X = _hermitian(210, n, 0x44)
    alpha = sign * 1j
    blk, off = ops.hadamard_block(X, alpha)
    assert off < 1e-13
    A = X[2] + 1j * X[6]                            # F_R + i H_I
    np.testing.assert_allclose(blk, alpha * A, rtol=0, atol=1e-13)
    # spectrum of the image = spectrum of the two reduced blocks
    ev = np.linalg.eigvalsh(iso.to_isomorph(X))
    red = np.sort(np.concatenate([np.linalg.eigvalsh(blk), np.linalg.eigvalsh(-blk)]))
    np.testing.assert_allclose(ev, red, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sign", [1, -1])
def test_hadamard_pure_k(sign):
    """Pure k (F_I - i H_R; components M4, M8): alpha = +-1 gives the block
    +-(H_R + i F_I) (Eq. reduced-hadamard-pure)."""
    n = 8
    X = _hermitian(211, n, 0x88)
    alpha = float(sign)
    blk, off = ops.hadamard_block(X, alpha)
    assert off < 1e-13
    HR, FI = -X[7], X[3]
    np.testing.assert_allclose(blk, alpha * (HR + 1j * FI), rtol=0, atol=1e-13)
    ev = np.linalg.eigvalsh(iso.to_isomorph(X))
    red = np.sort(np.concatenate([np.linalg.eigvalsh(blk), np.linalg.eigvalsh(-blk)]))
    np.testing.assert_allclose(ev, red, rtol=0, atol=1e-12)


@pytest.mark.parametrize("alpha", [1j, -1.0, np.exp(0.3j)])
def test_hadamard_general_transform_closed_form(alpha):
    """M'_11 = (alpha A + alpha* B)/2 and M'_21 = (alpha A - alpha* B)/2 for any
    unit alpha (Eq. hadamard_general_transform); j and k together do not reduce."""
    n = 6
    X = _hermitian(212, n, 0xCC)
    A, B, diag = ops.antidiagonal_blocks(X)
    assert diag == 0.0
    blk, off = ops.hadamard_block(X, alpha)
    a = complex(alpha)
    np.testing.assert_allclose(blk, (a * A + a.conjugate() * B) / 2, rtol=0, atol=1e-13)
    assert abs(off - np.max(np.abs(a * A - a.conjugate() * B)) / 2) < 1e-13
    assert off > 0.1


@pytest.mark.parametrize("op", OPS)
def test_op_signs_match_the_image(op):
    """The sign patterns of Sec. III (transposition, complex and Hermitian
    conjugation, quaternion conjugation) are the matrix operations on the image."""
    X = bi.small_int(213, 5, 7).numpy()
    np.testing.assert_array_equal(iso.to_isomorph(oracle.apply_op(op, X)), iso.iso_op(op, iso.to_isomorph(X)))
