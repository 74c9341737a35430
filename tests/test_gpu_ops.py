"""GPU parity of the element-wise and mapping operations (through the C ABI)
against the CPU oracle (oracle/ops.py, oracle/isomorph.py).

Scaling, addition, the complex image, the inverse map and the Hermiticity
deviation are correctly rounded step by step on both sides, so they are
compared bit for bit; the trace (a sum in a different order) and the Hadamard
block (the oracle multiplies by U_alpha with matmul) within stated bounds.
Absent components hold NaN on the device and are checked never to be read.
"""
import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm
from oracle import isomorph as iso
from oracle import ops

pytestmark = pytest.mark.gpu
OPS = ["N", "T", "C", "H", "QC"]
FLAGS = [bi.REAL, bi.COMPLEX, bi.TRS, bi.TRA, bi.BQ, 0x5A]
DEV = "cuda"


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with hm.Handle() as h:
        yield h
        assert h.device_error() == 0


def stored(op, rows, cols):
    return (cols, rows) if op in ("T", "H") else (rows, cols)


def with_nan(X, flags):
    """Device copy of X with NaN in the absent components; host copy with zeros."""
    host = bi.apply_flags(X.clone(), flags)
    dev = host.clone()
    for c in range(8):
        if not (flags >> c) & 1:
            dev[c] = float("nan")
    return dev.to(DEV), host.numpy()


ALPHAS = [0.3 - 1.7j, 1.0, -1.0, 1j, -1j, 2.5, 0.0, -0.75j]   # every scalar kind


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("m,n", [(45, 70), (1, 1), (33, 1), (64, 96)])
def test_scale_bitexact(handle, op, m, n, alpha):
    X = bi.uniform(300, *stored(op, m, n))
    for flags in (bi.BQ, bi.TRA, bi.COMPLEX):
        dX, hX = with_nan(X, flags)
        Y = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=DEV)
        hm.hmat_bq_scale(handle, dX, Y, alpha, op, flags)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(Y.cpu().numpy(), ops.scale(hX, alpha, op))


@pytest.mark.parametrize("a,b", [(2 - 0.5j, -1.25 + 0.75j), (1.0, 1.0), (1.0, -1.0), (1j, -1j), (2.0, 1j),
                                 (-1.0, 0.5)])
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("T", "H"), ("C", "QC"), ("H", "N"), ("QC", "T")])
def test_add_bitexact(handle, opA, opB, a, b):
    m, n = 37, 83
    A = bi.uniform(301, *stored(opA, m, n))
    B = bi.uniform(302, *stored(opB, m, n))
    for fa, fb in [(bi.BQ, bi.BQ), (bi.TRS, bi.TRA), (bi.REAL, 0x5A)]:
        dA, hA = with_nan(A, fa)
        dB, hB = with_nan(B, fb)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=DEV)
        hm.hmat_bq_add(handle, dA, dB, C, a, b, opA, opB, fa, fb)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(C.cpu().numpy(), ops.add(hA, hB, a, b, opA, opB))
    # the paper's plain sum on integers
    Ai = bi.small_int(303, m, n)
    Bi = bi.small_int(304, m, n)
    C = torch.empty((8, m, n), dtype=torch.float64, device=DEV)
    hm.hmat_bq_add(handle, Ai.to(DEV), Bi.to(DEV), C)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.cpu().numpy(), (Ai + Bi).numpy())


def test_add_in_place_and_rejects_transposed_alias(handle):
    m = n = 50
    A = bi.uniform(305, m, n).to(DEV)
    B = bi.uniform(306, m, n).to(DEV)
    want = ops.add(A.cpu().numpy(), B.cpu().numpy(), 1j, 2.0, "C", "N")
    hm.hmat_bq_add(handle, A, B, A, 1j, 2.0, "C", "N")           # C aliases A, op C does not transpose
    torch.cuda.synchronize()
    np.testing.assert_array_equal(A.cpu().numpy(), want)
    with pytest.raises(hm.HmatError) as ei:
        hm.hmat_bq_add(handle, A, B, A, 1.0, 1.0, "T", "N")
    assert ei.value.status == 1


@pytest.mark.parametrize("op", OPS)
def test_trace(handle, op):
    n = 301
    Xi = bi.small_int(307, n, n)
    t = hm.hmat_bq_trace(handle, Xi.to(DEV), op).cpu().numpy()
    want = ops.trace(Xi.numpy(), op)
    assert complex(t[0], t[1]) == want                           # integers: exact
    X = bi.uniform(308, n, n)
    dX, hX = with_nan(X, bi.TRA)                                  # M1 absent: real part 0
    t = hm.hmat_bq_trace(handle, dX, op, bi.TRA).cpu().numpy()
    want = ops.trace(hX, op)
    bound = 4 * n * np.finfo(float).eps * 2 * np.abs(np.diagonal(hX[4])).sum()
    assert t[0] == 0.0 and abs(t[1] - want.imag) <= bound
    # repeatable bits
    t2 = hm.hmat_bq_trace(handle, dX, op, bi.TRA).cpu().numpy()
    assert t2[1] == t[1]


@pytest.mark.parametrize("op", OPS)
def test_to_complex_bitexact(handle, op):
    m, n = 45, 70
    X = bi.uniform(309, *stored(op, m, n))
    for flags in (bi.BQ, bi.TRS, 0xCC):
        dX, hX = with_nan(X, flags)
        Z = hm.hmat_bq_to_complex(handle, dX, op=op, flags=flags)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(Z.cpu().numpy(), iso.to_isomorph(oracle.apply_op(op, hX)))


def test_from_complex_bitexact_and_round_trip(handle):
    m, n = 40, 66
    g = torch.Generator().manual_seed(310)
    Z = torch.complex(torch.rand((2 * m, 2 * n), generator=g, dtype=torch.float64) * 2 - 1,
                      torch.rand((2 * m, 2 * n), generator=g, dtype=torch.float64) * 2 - 1)
    Y = hm.hmat_complex_to_bq(handle, Z.to(DEV))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Y.cpu().numpy(), iso.from_isomorph(Z.numpy()))
    X = bi.small_int(311, m, n).to(DEV)
    back = hm.hmat_complex_to_bq(handle, hm.hmat_bq_to_complex(handle, X))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(back.cpu().numpy(), X.cpu().numpy())


@pytest.mark.parametrize("n", [1, 31, 33, 100])
def test_hermiticity(handle, n):
    X = bi.uniform(312, n, n)
    for flags in (bi.BQ, bi.TRS, bi.COMPLEX):
        dX, hX = with_nan(X, flags)
        d = hm.hmat_bq_hermiticity(handle, dX, flags).cpu().numpy()[0]
        assert d == ops.hermiticity_deviation(hX)
        Hm = hX + oracle.apply_op("H", hX)
        dH, _ = with_nan(torch.from_numpy(Hm), flags)
        assert hm.hmat_bq_hermiticity(handle, dH, flags).cpu().numpy()[0] == 0.0
    if n > 1:
        P = torch.from_numpy(X.numpy() + oracle.apply_op("H", X.numpy())).to(DEV)
        P[3, n - 1, 0] = float("nan")
        assert np.isnan(hm.hmat_bq_hermiticity(handle, P).cpu().numpy()[0])


@pytest.mark.parametrize("n", [33, 65, 130])
def test_hermiticity_views_with_even_pitch(handle, n):
    """n x n views of an (n + 1) or (n + 2) wide buffer (row pitch and
    component stride larger than the view), ragged tiles, entries of the buffer
    outside the view NaN (never read), subalgebra flags and a planted
    deviation."""
    pitch = n + 1 if n % 2 else n + 2
    buf = torch.full((8, pitch, pitch), float("nan"), dtype=torch.float64)
    X = bi.uniform(316 + n, n, n).numpy()
    Hm = X + oracle.apply_op("H", X)
    buf[:, :n, :n] = torch.from_numpy(Hm)
    dbuf = buf.to(DEV)
    view = dbuf[:, :n, :n]
    assert view.stride(1) % 2 == 0 and view.stride(0) % 2 == 0
    for flags in (bi.BQ, bi.TRS, 0x66):
        assert hm.hmat_bq_hermiticity(handle, view, flags).cpu().numpy()[0] == 0.0
    dbuf[5, n - 1, 3] += 0.25                 # X[n-1][3] - conj(X[3][n-1]) = 0.25 in component 6
    got = hm.hmat_bq_hermiticity(handle, view).cpu().numpy()[0]
    want = ops.hermiticity_deviation(dbuf[:, :n, :n].cpu().numpy())
    assert got == want and abs(got - 0.25) < 1e-12


def _hermitian(seed, n, flags):
    X = bi.uniform(seed, n, n, flags=flags).numpy()
    return bi.apply_flags(torch.from_numpy(X + oracle.apply_op("H", X)), flags)


@pytest.mark.parametrize("flags,alpha,reduces", [(0x44, 1j, True), (0x44, -1j, True), (0x88, 1.0, True),
                                                 (0x88, -1.0, True), (0xCC, 1j, False),
                                                 (0xCC, np.exp(0.3j), False)])
@pytest.mark.parametrize("n", [7, 64, 129])
def test_hadamard_block(handle, flags, alpha, reduces, n):
    X = _hermitian(313 + n, n, flags)
    dX, hX = with_nan(X, flags)
    Z, off = hm.hmat_bq_hadamard_block(handle, dX, alpha, flags)
    torch.cuda.synchronize()
    blk, off_want = ops.hadamard_block(hX, alpha)
    scale = np.abs(hX).max()
    np.testing.assert_allclose(Z.cpu().numpy(), blk, rtol=0, atol=8 * np.finfo(float).eps * scale)
    got_off = off.cpu().numpy()[0]
    if reduces:
        assert got_off == 0.0 and off_want < 1e-13 * scale
    else:
        assert abs(got_off - off_want) <= 8 * np.finfo(float).eps * scale and got_off > 0


def test_hadamard_argument_errors(handle):
    X = _hermitian(320, 16, 0x44).to(DEV)
    with pytest.raises(hm.HmatError) as ei:
        hm.hmat_bq_hadamard_block(handle, X, 1j, flags=0x45)        # E present
    assert ei.value.status == 2
    with pytest.raises(hm.HmatError) as ei:
        hm.hmat_bq_hadamard_block(handle, X, 0.5j, flags=0x44)      # not a unit scalar
    assert ei.value.status == 1


def test_ops_at_n2048(handle):
    """Every operation once at n = 2048 (270 MB per operand), full comparison."""
    n = 2048
    A = bi.fock_like(330, n, n, device=DEV)
    B = bi.fock_like(331, n, n, device=DEV)
    hA, hB = A.cpu().numpy(), B.cpu().numpy()
    C = torch.empty_like(A)
    hm.hmat_bq_add(handle, A, B, C, 1 - 1j, 0.5, "H", "N")
    np.testing.assert_array_equal(C.cpu().numpy(), ops.add(hA, hB, 1 - 1j, 0.5, "H", "N"))
    Z = hm.hmat_bq_to_complex(handle, A, op="T")
    np.testing.assert_array_equal(Z.cpu().numpy(), iso.to_isomorph(oracle.apply_op("T", hA)))
    Y = hm.hmat_complex_to_bq(handle, Z)
    np.testing.assert_array_equal(Y.cpu().numpy(), iso.from_isomorph(Z.cpu().numpy()))
    d = hm.hmat_bq_hermiticity(handle, A).cpu().numpy()[0]
    assert d == ops.hermiticity_deviation(hA)
    t = hm.hmat_bq_trace(handle, A).cpu().numpy()
    tw = ops.trace(hA)
    assert abs(complex(t[0], t[1]) - tw) <= 8 * n * np.finfo(float).eps * 2 * np.abs(np.diagonal(hA[0])).sum() + 1e-300
    assert handle.device_error() == 0


def test_empty_and_degenerate_shapes(handle):
    """m or n = 0 returns at once; 1 x 1 and single rows / columns go through the ragged tails."""
    E = torch.empty((8, 0, 5), dtype=torch.float64, device=DEV)
    hm.hmat_bq_add(handle, E, E, torch.empty_like(E))
    hm.hmat_bq_scale(handle, E, torch.empty_like(E), 2.0)
    assert hm.hmat_bq_to_complex(handle, E).shape == (0, 10)
    t = hm.hmat_bq_trace(handle, torch.empty((8, 0, 0), dtype=torch.float64, device=DEV)).cpu().numpy()
    assert t[0] == 0.0 and t[1] == 0.0
    d = hm.hmat_bq_hermiticity(handle, torch.empty((8, 0, 0), dtype=torch.float64, device=DEV)).cpu().numpy()
    assert d[0] == 0.0
    for m, n in [(1, 1), (1, 257), (257, 1), (3, 2)]:
        X = bi.uniform(340 + m, m, n)
        Y = bi.uniform(350 + n, m, n)
        C = torch.empty((8, m, n), dtype=torch.float64, device=DEV)
        hm.hmat_bq_add(handle, X.to(DEV), Y.to(DEV), C, 1 - 2j, 3.0)
        np.testing.assert_array_equal(C.cpu().numpy(), ops.add(X.numpy(), Y.numpy(), 1 - 2j, 3.0))
        Z = hm.hmat_bq_to_complex(handle, X.to(DEV))
        np.testing.assert_array_equal(Z.cpu().numpy(), iso.to_isomorph(X.numpy()))
        np.testing.assert_array_equal(hm.hmat_complex_to_bq(handle, Z).cpu().numpy(), iso.from_isomorph(Z.cpu().numpy()))


def test_from_complex_edge_values(handle):
    """The inverse map halves in integer arithmetic: zeros, subnormals and the smallest normals come
    out exactly as numpy's correctly rounded halving.  (Infinities are left out: numpy's complex
    division by 2 turns an infinite imaginary part into a NaN real part.)"""
    m, n = 3, 70
    g = np.random.default_rng(360)
    special = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, -3e-320, 2.2250738585072014e-308,
                        4.450147717014403e-308, 1e307, 3.0])
    re = g.choice(special, size=(2 * m, 2 * n)) * g.choice([1.0, 0.5, -3.0], size=(2 * m, 2 * n))
    im = g.choice(special, size=(2 * m, 2 * n))
    Z = torch.complex(torch.from_numpy(re), torch.from_numpy(im))
    Y = hm.hmat_complex_to_bq(handle, Z.to(DEV))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Y.cpu().numpy(), iso.from_isomorph(Z.numpy()))
