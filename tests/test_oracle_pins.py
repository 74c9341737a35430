"""Pins of the CPU oracle to facts the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares the component-wise
64-product oracle with something computed another way (the quaternion
relations, the Pauli-matrix isomorphism, numpy matmul on the complex isomorph,
algebraic identities, subalgebra reductions, the zero patterns of Tables I-II).
"""
import itertools
import os

import numpy as np
import pytest

import bq_inputs as bi
import oracle
from oracle import isomorph as iso

OPS = ["N", "T", "C", "H", "QC"]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _np(t):
    return t.numpy().copy()


def basis(e, imag=False):
    """1x1 biquaternion with a single unit coefficient on basis element e (0=1, 1=i, 2=j, 3=k)."""
    M = np.zeros((8, 1, 1))
    M[e + (4 if imag else 0), 0, 0] = 1.0
    return M


def mul(a, b):
    return oracle.bq_gemm(a, b)


# ---------------------------------------------------------------- quaternion relations
def test_quaternion_defining_relations():
    """Sec. II A: i^2 = j^2 = k^2 = i j k = -1 and the complex unit is central."""
    one = basis(0)
    minus_one = -one
    qi, qj, qk = basis(1), basis(2), basis(3)
    for u in (qi, qj, qk):
        np.testing.assert_array_equal(mul(u, u), minus_one)
    np.testing.assert_array_equal(mul(mul(qi, qj), qk), minus_one)
    np.testing.assert_array_equal(mul(qi, mul(qj, qk)), minus_one)
    # the complex unit (basis element 1 with imaginary coefficient) commutes with everything
    ci = basis(0, imag=True)
    for e in range(4):
        for im in (False, True):
            u = basis(e, imag=im)
            np.testing.assert_array_equal(mul(ci, u), mul(u, ci))
    # i * i (complex) = -1
    np.testing.assert_array_equal(mul(ci, ci), minus_one)


def _pauli_2x2(M):
    """Sec. II A Eq. TRG-in-C / qmap1: q1 I + q2 (i sz) + q3 (i sy) + q4 (i sx)."""
    sx = np.array([[0, 1], [1, 0]], dtype=complex)
    sy = np.array([[0, -1j], [1j, 0]], dtype=complex)
    sz = np.array([[1, 0], [0, -1]], dtype=complex)
    q = [M[e, 0, 0] + 1j * M[e + 4, 0, 0] for e in range(4)]
    return q[0] * np.eye(2) + q[1] * 1j * sz + q[2] * 1j * sy + q[3] * 1j * sx


def test_product_matches_pauli_representation():
    """1x1 products equal 2x2 complex products under 1, i, j, k -> I, i sz, i sy, i sx."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        a = rng.uniform(-1, 1, (8, 1, 1))
        b = rng.uniform(-1, 1, (8, 1, 1))
        np.testing.assert_allclose(_pauli_2x2(mul(a, b)), _pauli_2x2(a) @ _pauli_2x2(b),
                                   rtol=0, atol=1e-15)
    # the Pauli route and the block route of the isomorph describe the same matrix
    a = rng.uniform(-1, 1, (8, 1, 1))
    X = iso.to_isomorph(a)
    np.testing.assert_allclose(X, _pauli_2x2(a), rtol=0, atol=0)


# ---------------------------------------------------------------- isomorph round trip
def test_isomorph_round_trip():
    """Eq. mapping-formulas inverts the M+ + M- block construction, and the map is onto."""
    rng = np.random.default_rng(3)
    M = rng.uniform(-1, 1, (8, 5, 7))
    np.testing.assert_array_equal(iso.from_isomorph(iso.to_isomorph(M)), M)
    X = rng.uniform(-1, 1, (10, 14)) + 1j * rng.uniform(-1, 1, (10, 14))
    np.testing.assert_allclose(iso.to_isomorph(iso.from_isomorph(X)), X, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- brute force on the isomorph
@pytest.mark.parametrize("opA,opB", list(itertools.product(OPS, OPS)))
def test_oracle_equals_isomorph_exact_integers(opA, opB):
    """Small integers: every operation is exact, so the two routes agree bit for bit."""
    m, n, k = 5, 6, 7
    A = _np(bi.small_int(11, *( (k, m) if opA in ("T", "H") else (m, k) )))
    B = _np(bi.small_int(12, *( (n, k) if opB in ("T", "H") else (k, n) )))
    C = _np(bi.small_int(13, m, n))
    got = oracle.bq_gemm(A, B, opA, opB, alpha=2 - 3j, beta=-1 + 2j, C=C)
    want = iso.iso_bq_gemm(A, B, opA, opB, alpha=2 - 3j, beta=-1 + 2j, C=C)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("opA,opB", [("N", "N"), ("H", "N"), ("T", "C"), ("QC", "H")])
def test_oracle_equals_isomorph_random(opA, opB):
    m, n, k = 17, 13, 29
    A = _np(bi.uniform(21, *((k, m) if opA in ("T", "H") else (m, k))))
    B = _np(bi.uniform(22, *((n, k) if opB in ("T", "H") else (k, n))))
    C = _np(bi.uniform(23, m, n))
    al, be = bi.complex_scalar(24), bi.complex_scalar(25)
    got = oracle.bq_gemm(A, B, opA, opB, alpha=al, beta=be, C=C)
    want = iso.iso_bq_gemm(A, B, opA, opB, alpha=al, beta=be, C=C)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 1e-14, err


def test_row_selection_matches_full_result():
    A = _np(bi.uniform(31, 9, 8))
    B = _np(bi.uniform(32, 8, 10))
    full = oracle.bq_gemm(A, B, threads=2)
    rows = [7, 0, 3]
    np.testing.assert_array_equal(oracle.bq_gemm(A, B, rows=rows, threads=3), full[:, rows, :])


def test_beta_zero_does_not_read_c():
    A = _np(bi.small_int(41, 4, 3))
    B = _np(bi.small_int(42, 3, 5))
    C = np.full((8, 4, 5), np.nan)
    got = oracle.bq_gemm(A, B, alpha=1.0, beta=0.0, C=C)
    assert np.isfinite(got).all()
    np.testing.assert_array_equal(got, oracle.bq_gemm(A, B))


# ---------------------------------------------------------------- algebraic identities
def test_associativity_exact():
    A = _np(bi.small_int(51, 4, 5))
    B = _np(bi.small_int(52, 5, 3))
    C = _np(bi.small_int(53, 3, 6))
    np.testing.assert_array_equal(mul(mul(A, B), C), mul(A, mul(B, C)))


@pytest.mark.parametrize("op", ["T", "H"])
def test_transposing_ops_reverse_products(op):
    """(AB)^T = B^T A^T and (AB)^dagger = B^dagger A^dagger (Sec. III)."""
    A = _np(bi.small_int(61, 4, 5))
    B = _np(bi.small_int(62, 5, 3))
    lhs = oracle.apply_op(op, mul(A, B))
    rhs = oracle.bq_gemm(B, A, op, op)
    np.testing.assert_array_equal(lhs, rhs)


def test_complex_conjugation_is_an_automorphism():
    """(AB)^* = A^* B^* (Sec. III complex conjugation: no reversal)."""
    A = _np(bi.small_int(71, 4, 5))
    B = _np(bi.small_int(72, 5, 3))
    np.testing.assert_array_equal(oracle.apply_op("C", mul(A, B)), oracle.bq_gemm(A, B, "C", "C"))


def test_quaternion_conjugation_reverses_scalar_products():
    """For 1x1 biquaternions conj(pq) = conj(q) conj(p); p conj(p) is a complex scalar."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        p = rng.integers(-5, 6, (8, 1, 1)).astype(float)
        q = rng.integers(-5, 6, (8, 1, 1)).astype(float)
        np.testing.assert_array_equal(oracle.apply_op("QC", mul(p, q)),
                                      oracle.bq_gemm(q, p, "QC", "QC"))
        n = oracle.bq_gemm(p, p, "N", "QC")
        assert np.all(n[[1, 2, 3, 5, 6, 7]] == 0)      # only the scalar part survives


def test_ops_are_involutions_and_dagger_composes():
    M = _np(bi.uniform(81, 6, 4))
    for op in OPS:
        np.testing.assert_array_equal(oracle.apply_op(op, oracle.apply_op(op, M)), M)
    np.testing.assert_array_equal(oracle.apply_op("H", M),
                                  oracle.apply_op("T", oracle.apply_op("C", M)))


# ---------------------------------------------------------------- subalgebras
def test_real_subalgebra_is_real_gemm():
    A = _np(bi.uniform(91, 6, 5, flags=bi.REAL))
    B = _np(bi.uniform(92, 5, 7, flags=bi.REAL))
    got = mul(A, B)
    np.testing.assert_allclose(got[0], A[0] @ B[0], rtol=0, atol=1e-14)
    assert np.all(got[1:] == 0)


def test_complex_subalgebra_is_complex_gemm():
    A = _np(bi.uniform(93, 6, 5, flags=bi.COMPLEX))
    B = _np(bi.uniform(94, 5, 7, flags=bi.COMPLEX))
    got = mul(A, B)
    want = (A[0] + 1j * A[4]) @ (B[0] + 1j * B[4])
    np.testing.assert_allclose(got[0] + 1j * got[4], want, rtol=0, atol=1e-14)
    assert np.all(got[[1, 2, 3, 5, 6, 7]] == 0)


def _left_regular_real(M):
    """4n x 4n real matrix of left multiplication by a real-quaternion matrix.

    Built from the quaternion relations only: the columns are the images of the
    basis 1, i, j, k; i j = k follows from i^2 = j^2 = k^2 = ijk = -1.
    """
    a, b, c, d = M[0], M[1], M[2], M[3]
    return np.block([[a, -b, -c, -d],
                     [b, a, -d, c],
                     [c, d, a, -b],
                     [d, -c, b, a]])


def test_real_quaternion_subalgebra_matches_left_regular_representation():
    A = _np(bi.small_int(95, 4, 3, flags=bi.TRS))
    B = _np(bi.small_int(96, 3, 5, flags=bi.TRS))
    got = mul(A, B)
    assert np.all(got[4:] == 0)
    LB = np.concatenate([B[0], B[1], B[2], B[3]], axis=0)          # 4k x n (columns = B's coefficients)
    prod = _left_regular_real(A) @ LB
    m = A.shape[1]
    for e in range(4):
        np.testing.assert_array_equal(got[e], prod[e * m:(e + 1) * m])


@pytest.mark.parametrize("fa,fb,want", [
    (bi.TRS, bi.TRS, bi.TRS), (bi.TRS, bi.TRA, bi.TRA), (bi.TRA, bi.TRS, bi.TRA), (bi.TRA, bi.TRA, bi.TRS)])
def test_trs_tra_closure(fa, fb, want):
    """TRS <-> H_R, TRA <-> i H_R (Sec. I): H_R H_R, (iH_R)(iH_R) in H_R; mixed in i H_R."""
    A = _np(bi.uniform(97, 5, 4, flags=fa))
    B = _np(bi.uniform(98, 4, 6, flags=fb))
    got = mul(A, B)
    for c in range(8):
        if (want >> c) & 1:
            assert np.linalg.norm(got[c]) > 0
        else:
            assert np.all(got[c] == 0)


def _pattern(s):
    bits = [int(x) for x in s.split(",")]
    return sum(b << i for i, b in enumerate(bits))


def test_table2_operator_patterns():
    """Tables I-II: zero patterns of (X^RKB)^dagger O X^RKB and of ... O X^{RMB,A} + h.c."""
    rows = []
    with open(os.path.join(GOLDEN, "table2_patterns.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([p.strip() for p in line.split("|")])
    assert len(rows) == 3
    rkb = _pattern("1,1,1,1,0,0,0,0")
    rmb_a = _pattern("0,0,0,0,0,1,1,1")
    nc, nb = 6, 4     # components x basis functions
    for i, (name, op_pat, want_rr, want_ra) in enumerate(rows):
        X = _np(bi.uniform(100 + i, nc, nb, flags=rkb))
        Y = _np(bi.uniform(200 + i, nc, nb, flags=rmb_a))
        O = _np(bi.uniform(300 + i, nc, nc, flags=_pattern(op_pat)))
        rr = oracle.bq_gemm(X, mul(O, X), "H", "N")
        xy = oracle.bq_gemm(X, mul(O, Y), "H", "N")
        ra = xy + oracle.apply_op("H", xy)
        for got, want in ((rr, _pattern(want_rr)), (ra, _pattern(want_ra))):
            for c in range(8):
                if (want >> c) & 1:
                    assert np.linalg.norm(got[c]) > 1e-12, (name, c)
                else:
                    assert np.max(np.abs(got[c])) < 1e-14, (name, c)


# ---------------------------------------------------------------- input recipe sanity
def test_fock_like_envelope_and_row_scales():
    X = bi.fock_like(5, 64, 64, decay=10.0, row_scale=True).numpy()
    assert X.shape == (8, 64, 64)
    far = np.abs(X[:, 0, 60]).max()
    near = np.abs(X[:, 0, :4]).max()
    assert far < near * 1e-1
    shapes = bi.batch_shapes(104, 512)
    assert len(shapes) == 512 and all(32 <= d <= 1024 for s in shapes for d in s)
