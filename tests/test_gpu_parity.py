"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact on small-integer inputs (every FP64 step and every residue step is
exact there); within the relative-Frobenius tolerance 1e-12 on random data.
"""
import itertools

import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm

pytestmark = pytest.mark.gpu
TOL = 1e-12
OPS = ["N", "T", "C", "H", "QC"]
MODES = ["fp64", "split"]


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with hm.Handle() as h:
        yield h
        assert h.device_error() == 0


def stored(op, rows, cols):
    return (cols, rows) if op in ("T", "H") else (rows, cols)


def run(handle, A, B, opA="N", opB="N", fa=bi.BQ, fb=bi.BQ, alpha=1.0, beta=0.0, C0=None, mode="fp64",
        m=None, n=None):
    dev = torch.device("cuda")
    if m is None:
        m = A.shape[2] if opA in ("T", "H") else A.shape[1]
    if n is None:
        n = B.shape[1] if opB in ("T", "H") else B.shape[2]
    C = (C0.clone() if C0 is not None else torch.full((8, m, n), float("nan"), dtype=torch.float64)).to(dev)
    hm.hmat_bq_gemm(handle, A.to(dev), B.to(dev), C, opA, opB, fa, fb, alpha, beta, mode=mode, tol=TOL)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def rel(got, want):
    return np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("opA,opB", list(itertools.product(OPS, OPS)))
def test_exact_integers_all_ops(handle, mode, opA, opB):
    m, n, k = 37, 45, 83
    A = bi.small_int(10, *stored(opA, m, k))
    B = bi.small_int(11, *stored(opB, k, n))
    C0 = bi.small_int(12, m, n)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), opA, opB, alpha=2 - 3j, beta=-1 + 2j, C=C0.numpy())
    got = run(handle, A, B, opA, opB, alpha=2 - 3j, beta=-1 + 2j, C0=C0, mode=mode)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 129, 257), (130, 33, 1025), (255, 300, 64), (128, 256, 2049)])
def test_exact_integers_ragged_shapes(handle, mode, m, n, k):
    A = bi.small_int(20, m, k)
    B = bi.small_int(21, k, n)
    want = oracle.bq_gemm(A.numpy(), B.numpy())
    np.testing.assert_array_equal(run(handle, A, B, mode=mode), want)


FLAGS = [bi.REAL, bi.COMPLEX, bi.TRS, bi.TRA, bi.BQ]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("fa,fb", list(itertools.product(FLAGS, FLAGS)))
def test_subalgebra_flags_exact(handle, mode, fa, fb):
    m, n, k = 40, 24, 70
    A = bi.small_int(30, m, k, flags=fa)
    B = bi.small_int(31, k, n, flags=fb)
    want = oracle.bq_gemm(A.numpy(), B.numpy())
    # absent components hold garbage: the library must not read them
    Ag, Bg = A.clone(), B.clone()
    for c in range(8):
        if not (fa >> c) & 1:
            Ag[c].fill_(float("nan"))
        if not (fb >> c) & 1:
            Bg[c].fill_(float("nan"))
    np.testing.assert_array_equal(run(handle, Ag, Bg, fa=fa, fb=fb, mode=mode), want)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("opA,opB", [("N", "N"), ("H", "N"), ("T", "QC"), ("C", "H")])
def test_random_within_tolerance(handle, mode, opA, opB):
    m, n, k = 200, 150, 700
    A = bi.uniform(40, *stored(opA, m, k))
    B = bi.uniform(41, *stored(opB, k, n))
    C0 = bi.uniform(42, m, n)
    al, be = bi.complex_scalar(43), bi.complex_scalar(44)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), opA, opB, alpha=al, beta=be, C=C0.numpy())
    got = run(handle, A, B, opA, opB, alpha=al, beta=be, C0=C0, mode=mode)
    err = rel(got, want)
    assert err <= (1e-14 if mode == "fp64" else TOL), err


@pytest.mark.parametrize("mode", MODES)
def test_fock_like_row_scaled(handle, mode):
    """The precision workload's structure (banded, rows scaled over 6 decades) at a small size."""
    m = n = k = 384
    A = bi.fock_like(50, m, k, row_scale=True)
    B = bi.fock_like(51, k, n, row_scale=True)
    want = oracle.bq_gemm(A.numpy(), B.numpy())
    err = rel(run(handle, A, B, mode=mode), want)
    assert err <= TOL, err


@pytest.mark.parametrize("mode", MODES)
def test_beta_zero_ignores_nan_and_k_zero_scales(handle, mode):
    m, n, k = 33, 17, 5
    A = bi.uniform(60, m, k)
    B = bi.uniform(61, k, n)
    got = run(handle, A, B, mode=mode)      # C pre-filled with NaN, beta = 0
    assert np.isfinite(got).all()
    C0 = bi.uniform(62, m, n)
    Aa = torch.empty((8, m, 0), dtype=torch.float64)
    Bb = torch.empty((8, 0, n), dtype=torch.float64)
    got = run(handle, Aa, Bb, beta=0.5 - 0.25j, C0=C0, mode=mode, m=m, n=n)
    want = oracle.bq_gemm(np.zeros((8, m, 1)), np.zeros((8, 1, n)), beta=0.5 - 0.25j, C=C0.numpy())
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("tol", [1e-3, 1e-6, 1e-9, 1e-13, 1e-14])
@pytest.mark.parametrize("fa,fb", [(bi.BQ, bi.BQ), (bi.TRS, bi.TRA), (bi.COMPLEX, bi.BQ)])
def test_split_tolerance_sweep(handle, tol, fa, fb):
    """Split mode meets each requested tolerance (relative Frobenius error over
    all eight components): 6 to 15 moduli, 2- and 3-limb encoding, 4- and
    5-limb CRT sums, the structured and the generic recombination, ragged
    shapes."""
    m, n, k = 150, 70, 333
    A = bi.uniform(70, m, k, flags=fa)
    B = bi.uniform(71, k, n, flags=fb)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), alpha=0.5 + 2j)
    dev = torch.device("cuda")
    C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
    hm.hmat_bq_gemm(handle, A.to(dev), B.to(dev), C, "N", "N", fa, fb, 0.5 + 2j, 0.0, mode="split", tol=tol)
    torch.cuda.synchronize()
    err = rel(C.cpu().numpy(), want)
    assert err <= tol, (err, hm.split_info(k, tol))


def _product_tensor():
    """T[e, c, d]: output component e of the product of storage basis elements c and d (oracle)."""
    T = np.zeros((8, 8, 8))
    for c in range(8):
        for d in range(8):
            a = np.zeros((8, 1, 1))
            b = np.zeros((8, 1, 1))
            a[c] = 1.0
            b[d] = 1.0
            T[:, c, d] = oracle.bq_gemm(a, b)[:, 0, 0]
    return T


@pytest.mark.parametrize("form", ["auto", "four_m"])
@pytest.mark.parametrize("tol,k", [(1e-12, 11776), (1e-13, 8900)])
def test_split_crt_worst_case_magnitude(handle, tol, k, form):
    """Outputs at the top of the integer range the modulus count allows.

    Every entry of op(A) is one biquaternion a and every entry of B one b, all
    eight storage values +-c with c = 2 - 2^-40 (scaled integer 2^b - 2^(b-41)),
    signs chosen so that all eight real products of one output component add
    up: |Q| = 8 k (2^b - 2^(b-41))^2.  Each k puts 8 k 2^(2b) just below
    P / 2^1.25 for the moduli it needs (b = 46 with 14 moduli, 4-limb CRT;
    b = 50 with 15 moduli, 5 limbs and 3-limb encoding), the least margin the
    modulus count leaves (|Q| / P = 0.418 and 0.419).  Every output is
    k N_e c^2 with an integer N_e, and split mode rounds the exact integer
    once: bit-exact against the rational value.  At these k the default takes
    Gauss's form; the four-multiplication form, forced, reaches the same
    outputs through two-term products over 2 k (many chunks).
    """
    from fractions import Fraction
    moduli, bits = hm.split_info(k, tol)
    P = 1
    for p in moduli:
        P *= p
    assert (len(moduli), bits) == ((14, 46) if tol == 1e-12 else (15, 50))
    assert 0.41 < 8 * k * (2 ** bits - 2 ** (bits - 41)) ** 2 / P < 0.42
    T = _product_tensor()
    signs = np.array([[1.0 if (v >> c) & 1 else -1.0 for c in range(8)] for v in range(256)])
    Q = np.einsum("sc,ecd,td->est", signs, T, signs)          # [e, sign pattern of a, of b]
    e_best, sa, sb = np.unravel_index(np.argmax(np.abs(Q)), Q.shape)
    N = Q[:, sa, sb]
    assert abs(N[e_best]) == 8.0
    c = 2.0 - 2.0 ** -40
    m, n = 3, 5
    dev = torch.device("cuda")
    A = torch.from_numpy(np.broadcast_to((signs[sa] * c)[:, None, None], (8, m, k)).copy()).to(dev)
    B = torch.from_numpy(np.broadcast_to((signs[sb] * c)[:, None, None], (8, k, n)).copy()).to(dev)
    want = np.array([float(Fraction(int(N[e]) * k) * Fraction(c) ** 2) for e in range(8)])
    handle.set_complex_form(form)
    try:
        for sign in (1.0, -1.0):            # both signs of the extreme component
            C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
            hm.hmat_bq_gemm(handle, sign * A, B, C, mode="split", tol=tol)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(C.cpu().numpy(), np.broadcast_to((sign * want)[:, None, None], (8, m, n)))
    finally:
        handle.set_complex_form("auto")


def test_strided_views(handle):
    """ld > columns and component strides larger than rows * ld."""
    dev = torch.device("cuda")
    m, n, k = 50, 40, 60
    Abig = bi.small_int(70, m + 5, k + 9).to(dev)
    Bbig = bi.small_int(71, k + 3, n + 11).to(dev)
    A = Abig[:, :m, :k]
    B = Bbig[:, :k, :n]
    Cbig = torch.zeros((8, m + 2, n + 7), dtype=torch.float64, device=dev)
    C = Cbig[:, :m, :n]
    for mode in MODES:
        hm.hmat_bq_gemm(handle, A, B, C, mode=mode)
        torch.cuda.synchronize()
        want = oracle.bq_gemm(A.cpu().numpy(), B.cpu().numpy())
        np.testing.assert_array_equal(C.cpu().numpy(), want)
        assert torch.all(Cbig[:, m:, :] == 0) and torch.all(Cbig[:, :, n:] == 0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("use_graph", [False, True])
def test_grouped_mixed_shapes(handle, mode, use_graph):
    dev = torch.device("cuda")
    shapes = [(33, 70, 129), (128, 64, 64), (5, 300, 17), (260, 100, 1100), (64, 64, 1)]
    flags = [(bi.BQ, bi.BQ), (bi.TRS, bi.TRA), (bi.BQ, bi.COMPLEX), (bi.TRS, bi.BQ), (bi.REAL, bi.BQ)]
    ops = [("N", "N"), ("H", "N"), ("T", "QC"), ("N", "C"), ("C", "T")]
    probs, descs = [], []
    for i, ((m, n, k), (fa, fb), (oa, ob)) in enumerate(zip(shapes, flags, ops)):
        A = bi.small_int(80 + i, *stored(oa, m, k), flags=fa)
        B = bi.small_int(90 + i, *stored(ob, k, n), flags=fb)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
        dA, dB = A.to(dev), B.to(dev)
        probs.append((A, B, C, oa, ob, dA, dB))
        descs.append(hm.make_desc(dA, dB, C, oa, ob, fa, fb))
    for _ in range(2):          # the second call replays the graph
        for p in probs:
            p[2].fill_(float("nan"))
        hm.hmat_bq_gemm_grouped(handle, descs, mode=mode, tol=TOL, use_graph=use_graph,
                                stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        for A, B, C, oa, ob, _, _ in probs:
            np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy(), oa, ob))


@pytest.mark.parametrize("use_graph", [False, True])
def test_grouped_full_plans_of_different_widths(handle, use_graph):
    """Several full-biquaternion products of different output widths (tile
    widths 32 to 256) in one grouped split-mode call: the residue GEMM's work
    items of different products interleave on every SM, so per-item state must
    not depend on a neighbouring item's shape.  Bit-exact on small integers."""
    dev = torch.device("cuda")
    shapes = [(100, 20, 90), (30, 250, 200), (200, 70, 64), (64, 160, 300), (140, 33, 17), (90, 300, 130),
              (257, 224, 40), (12, 96, 1000)]
    probs, descs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A = bi.small_int(140 + i, m, k)
        B = bi.small_int(150 + i, k, n)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
        dA, dB = A.to(dev), B.to(dev)          # kept alive: the descriptors hold their addresses
        probs.append((A, B, C, dA, dB))
        descs.append(hm.make_desc(dA, dB, C))
    for _ in range(2):
        for p in probs:
            p[2].fill_(float("nan"))
        hm.hmat_bq_gemm_grouped(handle, descs, mode="split", tol=TOL, use_graph=use_graph,
                                stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        for A, B, C, _, _ in probs:
            np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))


@pytest.mark.parametrize("use_graph", [False, True])
def test_grouped_modes_mixed(handle, use_graph):
    """One grouped call whose products run in different modes
    (hmat_bq_gemm_grouped_modes): split and FP64 products with mixed shapes,
    ops, flags and scalars.  On small integers every product equals the
    oracle bit for bit; on uniform inputs each split product equals the same
    product called alone in split mode bit for bit, each FP64 product the FP64
    call alone within 1e-14 (the built-in FP64 split-k rule counts the call's
    FP64 tiles, so the inner-dimension slicing may differ); the graph replays
    the same bits."""
    dev = torch.device("cuda")
    shapes = [(33, 70, 129), (128, 64, 64), (5, 300, 17), (260, 100, 1100), (64, 64, 1), (96, 40, 300)]
    flags = [(bi.BQ, bi.BQ), (bi.TRS, bi.TRA), (bi.BQ, bi.COMPLEX), (bi.TRS, bi.BQ), (bi.REAL, bi.BQ),
             (bi.BQ, bi.BQ)]
    ops = [("N", "N"), ("H", "N"), ("T", "QC"), ("N", "C"), ("C", "T"), ("N", "H")]
    modes = ["split", "fp64", "split", "fp64", "split", "fp64"]
    scal = [(1.0, 0.0), (2 - 3j, -1 + 2j), (1.0, 0.0), (0.5, 1.0), (-1j, 0.0), (1.0, 0.25)]
    for gen in ("small_int", "uniform"):
        probs, descs = [], []
        for i, ((m, n, k), (fa, fb), (oa, ob), (al, be)) in enumerate(zip(shapes, flags, ops, scal)):
            make = getattr(bi, gen)
            A = make(180 + i, *stored(oa, m, k), flags=fa)
            B = make(190 + i, *stored(ob, k, n), flags=fb)
            C0 = bi.small_int(200 + i, m, n)
            C = C0.to(dev)
            dA, dB = A.to(dev), B.to(dev)          # kept alive: the descriptors hold their addresses
            probs.append((A, B, C0, C, dA, dB, oa, ob, fa, fb, al, be))
            descs.append(hm.make_desc(dA, dB, C, oa, ob, fa, fb, al, be))
        results = []
        for _ in range(2):                          # the second call replays the graph
            for p in probs:
                p[3].copy_(p[2])
            hm.hmat_bq_gemm_grouped_modes(handle, descs, modes, tol=TOL, use_graph=use_graph,
                                          stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            results.append([p[3].cpu().numpy().copy() for p in probs])
        for a, b in zip(*results):
            np.testing.assert_array_equal(a, b)
        for (A, B, C0, C, dA, dB, oa, ob, fa, fb, al, be), md, got in zip(probs, modes, results[0]):
            if gen == "small_int":
                want = oracle.bq_gemm(A.numpy(), B.numpy(), oa, ob, alpha=al, beta=be, C=C0.numpy())
                np.testing.assert_array_equal(got, want)
            else:
                ref = C0.to(dev)
                hm.hmat_bq_gemm(handle, dA, dB, ref, oa, ob, fa, fb, alpha=al, beta=be, mode=md, tol=TOL)
                torch.cuda.synchronize()
                if md == "split":
                    np.testing.assert_array_equal(got, ref.cpu().numpy())
                else:
                    r = ref.cpu().numpy()
                    assert np.linalg.norm(got - r) <= 1e-14 * np.linalg.norm(r)


@pytest.mark.parametrize("algo", ["standard", "isomorph"])
def test_grouped_modes_mixed_comparison_algorithms(handle, algo):
    """A mode per product under the comparison algorithms: HMAT-standard (FP64
    products in several passes, the 64-product plan through the generic CRT)
    and CMAT (complex images mapped in and out around the products).  Small
    integers: every product equals the oracle bit for bit."""
    dev = torch.device("cuda")
    shapes = [(40, 70, 90), (64, 33, 130), (20, 100, 64)]
    flags = [(bi.BQ, bi.BQ), (bi.TRS, bi.BQ), (bi.COMPLEX, bi.TRA)]
    ops = [("N", "N"), ("H", "T"), ("C", "N")]
    modes = ["split", "fp64", "split"]
    handle.set_algorithm(algo)
    try:
        probs, descs = [], []
        for i, ((m, n, k), (fa, fb), (oa, ob)) in enumerate(zip(shapes, flags, ops)):
            A = bi.small_int(260 + i, *stored(oa, m, k), flags=fa)
            B = bi.small_int(270 + i, *stored(ob, k, n), flags=fb)
            C0 = bi.small_int(280 + i, m, n)
            C = C0.to(dev)
            dA, dB = A.to(dev), B.to(dev)
            probs.append((A, B, C0, C, dA, dB, oa, ob))
            descs.append(hm.make_desc(dA, dB, C, oa, ob, fa, fb, 2 - 1j, -1 + 0.5j))
        hm.hmat_bq_gemm_grouped_modes(handle, descs, modes, tol=TOL, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        for A, B, C0, C, _, _, oa, ob in probs:
            want = oracle.bq_gemm(A.numpy(), B.numpy(), oa, ob, alpha=2 - 1j, beta=-1 + 0.5j, C=C0.numpy())
            np.testing.assert_array_equal(C.cpu().numpy(), want)
    finally:
        handle.set_algorithm("bilinear")


def test_grouped_modes_rejects_an_unknown_mode(handle):
    dev = torch.device("cuda")
    A, B = bi.small_int(210, 8, 8).to(dev), bi.small_int(211, 8, 8).to(dev)
    C = torch.zeros((8, 8, 8), dtype=torch.float64, device=dev)
    descs = [hm.make_desc(A, B, C), hm.make_desc(A, B, C)]
    with pytest.raises(hm.HmatError):              # the size query refuses it too
        hm.hmat_workspace_size_modes(handle, descs, ["split", 7], tol=TOL)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    with pytest.raises(hm.HmatError) as e:
        hm.hmat_bq_gemm_grouped_modes(handle, descs, ["split", 7], tol=TOL, workspace=ws)
    assert "descriptor 1" in str(e.value)


def test_one_chunk_and_general_gemm_forms_agree(handle):
    """The residue GEMM has two forms: calls whose products all have k <= 1024
    launch one without the multi-chunk drain, others the general one.  The
    same products (k = 200 and 1024, ops and scalars) called alone (one-chunk
    form) and grouped with a product of k = 1100 (general form) give the same
    bits; the k = 1100 product matches the oracle on small integers."""
    dev = torch.device("cuda")
    cases = [((96, 130, 200), ("N", "H"), 2 - 1j, 0.5), ((70, 260, 1024), ("T", "N"), 1.0, 0.0)]
    big = (40, 50, 1100)
    probs = []
    for i, ((m, n, k), (oa, ob), al, be) in enumerate(cases):
        A = bi.uniform(220 + i, *stored(oa, m, k)).to(dev)
        B = bi.uniform(230 + i, *stored(ob, k, n)).to(dev)
        C0 = bi.uniform(240 + i, m, n).to(dev)
        alone = C0.clone()
        hm.hmat_bq_gemm(handle, A, B, alone, oa, ob, alpha=al, beta=be, mode="split", tol=TOL)
        probs.append((A, B, C0, alone, oa, ob, al, be))
    Ab, Bb = bi.small_int(250, big[0], big[2]), bi.small_int(251, big[2], big[1])
    dAb, dBb = Ab.to(dev), Bb.to(dev)
    Cb = torch.full((8, big[0], big[1]), float("nan"), dtype=torch.float64, device=dev)
    grouped = [p[2].clone() for p in probs]
    descs = [hm.make_desc(p[0], p[1], g, p[4], p[5], alpha=p[6], beta=p[7]) for p, g in zip(probs, grouped)]
    descs.append(hm.make_desc(dAb, dBb, Cb))
    hm.hmat_bq_gemm_grouped(handle, descs, mode="split", tol=TOL, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    for p, g in zip(probs, grouped):
        assert torch.equal(g, p[3])
    np.testing.assert_array_equal(Cb.cpu().numpy(), oracle.bq_gemm(Ab.numpy(), Bb.numpy()))


@pytest.fixture(scope="module")
def gauss_handle():
    h = hm.Handle()
    h.set_complex_form("gauss")
    yield h
    h.close()


@pytest.mark.parametrize("shape,ops,al,be", [((200, 300, 130), ("N", "N"), 1.0, 0.0),
                                             ((129, 257, 512), ("T", "H"), 2 - 1j, 0.5 + 0.25j),
                                             ((40, 33, 33), ("C", "QC"), -1.0, 1.0),
                                             ((300, 200, 700), ("H", "T"), 0.5j, -0.5)])
def test_four_multiplication_form_gives_gausss_bits(handle, gauss_handle, shape, ops, al, be):
    """Split mode forms each complex product of the full plan either with
    Gauss's three real products (24 residue GEMMs) or as two real products
    over twice the inner dimension (16 residue GEMMs, the subtracted term
    through the MMA's negate bit).  Every residue is exact, so both forms give
    the same bits: at k <= 512 (the default takes the four-multiplication
    form) and at k = 700 with the form forced (two 1024-deep chunks, the
    general GEMM form); the four-multiplication workspace is smaller."""
    dev = torch.device("cuda")
    (m, n, k), (oa, ob) = shape, ops
    A = bi.uniform(600 + k, *stored(oa, m, k)).to(dev)
    B = bi.uniform(610 + k, *stored(ob, k, n)).to(dev)
    C0 = bi.uniform(620 + k, m, n).to(dev)
    with hm.Handle() as four:
        four.set_complex_form("four_m")
        outs = []
        for h in (gauss_handle, four, handle):
            C = C0.clone()
            hm.hmat_bq_gemm(h, A, B, C, oa, ob, alpha=al, beta=be, mode="split", tol=TOL)
            outs.append(C)
        torch.cuda.synchronize()
        assert torch.equal(outs[1], outs[0])
        assert torch.equal(outs[2], outs[0])
        desc = [hm.make_desc(A, B, C0, oa, ob)]
        ws_g = hm.hmat_workspace_size(gauss_handle, desc, "split", TOL)
        ws_f = hm.hmat_workspace_size(four, desc, "split", TOL)
        ws_a = hm.hmat_workspace_size(handle, desc, "split", TOL)
        assert ws_f < ws_g
        assert ws_a == (ws_f if k <= 512 else ws_g)
        assert four.device_error() == 0
    want = oracle.bq_gemm(A.cpu().numpy(), B.cpu().numpy(), oa, ob, alpha=al, beta=be, C=C0.cpu().numpy())
    assert rel(outs[0].cpu().numpy(), want) < 1e-12


def test_four_multiplication_form_exact_integers(handle):
    """Four-multiplication form on small integers: the oracle's bits, through
    the one-chunk GEMM form (k = 512) and, forced, the general form (k = 1100,
    three chunks of the doubled depth), eager and grouped."""
    dev = torch.device("cuda")
    with hm.Handle() as four:
        four.set_complex_form("four_m")
        for i, (m, n, k) in enumerate([(96, 80, 512), (70, 130, 1100)]):
            A, B = bi.small_int(640 + i, m, k), bi.small_int(650 + i, k, n)
            for h in (handle, four):
                C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
                hm.hmat_bq_gemm(h, A.to(dev), B.to(dev), C, mode="split", tol=TOL)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))
        assert four.device_error() == 0


@pytest.mark.parametrize("use_graph,with_trs", [(False, False), (True, False), (False, True)])
def test_grouped_mixed_complex_forms(handle, gauss_handle, use_graph, with_trs):
    """One grouped call whose full-plan products take both forms under the
    default (k = 64 and 512: four multiplications; k = 513 and 1000: Gauss):
    the CRT's full-plan kernel picks each block's form; with a TRS x BQ
    product (its own plan) beside them the packed-weight CRT kernel serves all
    of them.  The outputs equal an all-Gauss handle's bit for bit."""
    dev = torch.device("cuda")
    shapes = [(130, 70, 64, bi.BQ), (64, 300, 512, bi.BQ), (200, 90, 513, bi.BQ), (33, 260, 1000, bi.BQ)]
    if with_trs:
        shapes.append((100, 100, 300, bi.TRS))
    mats = []
    for i, (m, n, k, fa) in enumerate(shapes):
        A = bi.uniform(660 + i, m, k, flags=fa).to(dev)
        B = bi.uniform(670 + i, k, n).to(dev)
        mats.append((A, B, fa, (m, n)))
    res = []
    for h in (handle, gauss_handle):
        Cs = [torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev) for _, _, _, (m, n) in mats]
        descs = [hm.make_desc(A, B, C, flagsA=fa) for (A, B, fa, _), C in zip(mats, Cs)]
        for _ in range(2 if use_graph else 1):
            hm.hmat_bq_gemm_grouped(h, descs, mode="split", tol=TOL, stream=torch.cuda.current_stream(),
                                    use_graph=use_graph)
        torch.cuda.synchronize()
        res.append(Cs)
    for a, b in zip(*res):
        assert torch.equal(a, b)
    for (A, B, fa, _), C in zip(mats, res[0]):
        want = oracle.bq_gemm(A.cpu().numpy(), B.cpu().numpy())
        assert rel(C.cpu().numpy(), want) < 1e-12
    assert handle.device_error() == 0


def test_complex_form_rejects_unknown_values(handle):
    with pytest.raises(hm.HmatError):
        handle.set_complex_form(3)
    with pytest.raises(hm.HmatError):
        handle.set_algorithm(3)


def _splitk_table(code):
    t = np.zeros((16, 16), dtype=np.int8)
    t[:, :] = code
    return t


@pytest.mark.parametrize("code", [1, 2, 3, 4])
@pytest.mark.parametrize("opA,opB,fa,fb", [("N", "N", bi.BQ, bi.BQ), ("H", "T", bi.TRS, bi.TRA),
                                           ("C", "QC", bi.COMPLEX, bi.BQ)])
def test_fp64_split_k(handle, code, opA, opB, fa, fb):
    """FP64 mode with the inner dimension in 1, 2, 4 or 8 slices (forced by the
    split-k table): within FP64 rounding of the oracle on random data with
    complex alpha, beta, and bit-exact on small integers; one slice is the
    unsplit computation bit for bit."""
    dev = torch.device("cuda")
    m, n, k = 96, 80, 700
    A = bi.uniform(160, *stored(opA, m, k), flags=fa)
    B = bi.uniform(161, *stored(opB, k, n), flags=fb)
    C0 = bi.uniform(162, m, n)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), opA, opB, alpha=0.5 + 1.5j, beta=-1 + 0.5j, C=C0.numpy())
    handle.set_fp64_splitk_table(_splitk_table(code))
    try:
        got = run(handle, A, B, opA, opB, fa, fb, alpha=0.5 + 1.5j, beta=-1 + 0.5j, C0=C0, mode="fp64")
        assert rel(got, want) <= 1e-14
        Ai = bi.small_int(163, *stored(opA, m, k), flags=fa)
        Bi = bi.small_int(164, *stored(opB, k, n), flags=fb)
        wi = oracle.bq_gemm(Ai.numpy(), Bi.numpy(), opA, opB)
        np.testing.assert_array_equal(run(handle, Ai, Bi, opA, opB, fa, fb, mode="fp64"), wi)
        if code == 1:                          # one slice: no workspace needed, same bits
            Cn = C0.clone().to(dev)
            hm.hmat_bq_gemm(handle, A.to(dev), B.to(dev), Cn, opA, opB, fa, fb, 0.5 + 1.5j, -1 + 0.5j,
                            mode="fp64", workspace=None)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(Cn.cpu().numpy(), got)
    finally:
        handle.set_fp64_splitk_table(None)


@pytest.mark.parametrize("use_graph", [False, True])
def test_fp64_split_k_builtin_rule_grouped(handle, use_graph):
    """Few-tile FP64 products in one grouped call take the built-in split-k
    rule (the workspace size query accounts for it); bit-exact on small
    integers, eager and replayed from a graph."""
    dev = torch.device("cuda")
    shapes = [(64, 64, 1024), (40, 100, 333), (128, 32, 65)]
    probs, descs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A = bi.small_int(170 + i, m, k)
        B = bi.small_int(180 + i, k, n)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
        dA, dB = A.to(dev), B.to(dev)
        probs.append((A, B, C, dA, dB))
        descs.append(hm.make_desc(dA, dB, C))
    assert hm.hmat_workspace_size(handle, descs, "fp64") > 0      # the partial outputs of the slices
    for _ in range(2):
        for p in probs:
            p[2].fill_(float("nan"))
        hm.hmat_bq_gemm_grouped(handle, descs, mode="fp64", use_graph=use_graph, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        for A, B, C, _, _ in probs:
            np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))
    h2 = hm.Handle()
    try:
        h2.set_profiling(True)
        probs[0][2].fill_(float("nan"))
        hm.hmat_bq_gemm(h2, probs[0][3], probs[0][4], probs[0][2], mode="fp64")
        torch.cuda.synchronize()
        assert h2.profile("fp64_splitk_reduce")[0] == 1               # n = 64: 4 tiles, k split
    finally:
        h2.close()


def test_argument_errors(handle):
    dev = torch.device("cuda")
    A = torch.zeros((8, 4, 4), dtype=torch.float64, device=dev)
    C = torch.zeros((8, 4, 4), dtype=torch.float64, device=dev)
    L = hm.lib()
    st = L.hmat_bq_gemm(handle.value, 9, 0, 0xFF, 0xFF, 4, 4, 4, 1.0, 0.0, A.data_ptr(), 4, 16, A.data_ptr(), 4, 16,
                        0.0, 0.0, C.data_ptr(), 4, 16, 0, 0.0, None, 0, None)
    assert st == 1                                        # bad op
    st = L.hmat_bq_gemm(handle.value, 0, 0, 0xFF, 0xFF, 4, 4, 4, 1.0, 0.0, A.data_ptr(), 3, 16, A.data_ptr(), 4, 16,
                        0.0, 0.0, C.data_ptr(), 4, 16, 0, 0.0, None, 0, None)
    assert st == 1                                        # lda < k
    st = L.hmat_bq_gemm(handle.value, 0, 0, 0xFF, 0xFF, 4, 4, 4, 1.0, 0.0, A.data_ptr() + 4, 4, 16, A.data_ptr(),
                        4, 16, 0.0, 0.0, C.data_ptr(), 4, 16, 0, 0.0, None, 0, None)
    assert st == 3                                        # misaligned
    st = L.hmat_bq_gemm(handle.value, 0, 0, 0xFF, 0xFF, 4, 4, 4, 1.0, 0.0, A.data_ptr(), 4, 16, A.data_ptr(), 4, 16,
                        0.0, 0.0, C.data_ptr(), 4, 16, 1, 0.0, None, 0, None)
    assert st == 4                                        # split mode without workspace
    st = L.hmat_bq_gemm(None, 0, 0, 0xFF, 0xFF, 4, 4, 4, 1.0, 0.0, A.data_ptr(), 4, 16, A.data_ptr(), 4, 16,
                        0.0, 0.0, C.data_ptr(), 4, 16, 0, 0.0, None, 0, None)
    assert st == 7                                        # no handle


@pytest.mark.parametrize("mode", MODES)
def test_grouped_batch_config_512(handle, mode):
    """The batching configuration at full size: 512 products, m,n,k log-uniform in [32,1024].

    16 sampled problems are compared with the oracle; every product is compared
    between the two modes (independent arithmetic: FP64 DFMA vs residue GEMMs)."""
    dev = torch.device("cuda")
    shapes = bi.batch_shapes(104, 512)
    mats, descs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A = bi.uniform(10_000 + i, m, k, device=dev)
        B = bi.uniform(20_000 + i, k, n, device=dev)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
        mats.append((A, B, C))
        descs.append(hm.make_desc(A, B, C))
    hm.hmat_bq_gemm_grouped(handle, descs, mode=mode, tol=TOL, use_graph=True, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    small = [i for i, (m, n, k) in enumerate(shapes) if m * n * k <= (1 << 25)]
    for i in rng.choice(small, size=16, replace=False):
        A, B, C = mats[i]
        want = oracle.bq_gemm(A.cpu().numpy(), B.cpu().numpy())
        assert rel(C.cpu().numpy(), want) <= (1e-14 if mode == "fp64" else TOL)
    other = "split" if mode == "fp64" else "fp64"
    outs = [C.clone() for _, _, C in mats]
    hm.hmat_bq_gemm_grouped(handle, descs, mode=other, tol=TOL, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    for (A, B, C), first in zip(mats, outs):
        e = float(torch.linalg.norm(C - first) / torch.linalg.norm(first))
        assert e <= TOL, e


@pytest.mark.parametrize("code", [1, 2, 3])
def test_tile_table_widths_give_identical_results(handle, code):
    """Every tuned tile width (64/128/256 columns) reproduces the oracle bit for bit."""
    m, n, k = 150, 300, 130
    A = bi.small_int(110, m, k)
    B = bi.small_int(111, k, n)
    t = np.zeros((16, 16), dtype=np.int8)
    t[:, :] = code
    handle.set_tile_table(t)
    try:
        got = run(handle, A, B, mode="split")
    finally:
        handle.set_tile_table(None)
    np.testing.assert_array_equal(got, oracle.bq_gemm(A.numpy(), B.numpy()))
    bad = np.full((16, 16), 7, dtype=np.int8)
    with pytest.raises(hm.HmatError):
        handle.set_tile_table(bad)


def test_bounded_wait_gives_up_with_an_error_status(handle):
    """A device wait that can never complete ends after its cycle limit with an
    error bit (no hang, no fault), and the context keeps working afterwards."""
    assert handle.device_error() == 0
    st = hm.lib().hmat_debug_wait_selftest(handle.value, 2_000_000, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert handle.device_error() == 0x20
    assert handle.device_error() == 0          # read-and-clear
    A = bi.small_int(120, 20, 30)
    B = bi.small_int(121, 30, 10)
    np.testing.assert_array_equal(run(handle, A, B, mode="split"), oracle.bq_gemm(A.numpy(), B.numpy()))


@pytest.mark.parametrize("algo", ["standard", "isomorph"])
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("opA,opB,fa,fb", [("N", "N", bi.BQ, bi.BQ), ("H", "T", bi.BQ, bi.BQ),
                                           ("C", "QC", bi.TRS, bi.TRA), ("T", "N", bi.COMPLEX, bi.BQ)])
def test_comparison_algorithms_exact(handle, algo, mode, opA, opB, fa, fb):
    """HMAT-standard and CMAT (complex isomorph) routes reproduce the oracle bit for bit."""
    m, n, k = 45, 70, 130
    A = bi.small_int(130, *stored(opA, m, k), flags=fa)
    B = bi.small_int(131, *stored(opB, k, n), flags=fb)
    C0 = bi.small_int(132, m, n)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), opA, opB, alpha=1 - 2j, beta=3 + 1j, C=C0.numpy())
    handle.set_algorithm(algo)
    try:
        got = run(handle, A, B, opA, opB, fa, fb, alpha=1 - 2j, beta=3 + 1j, C0=C0, mode=mode)
    finally:
        handle.set_algorithm("bilinear")
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("algo", ["standard", "isomorph"])
@pytest.mark.parametrize("mode", MODES)
def test_comparison_algorithms_random_and_grouped(handle, algo, mode):
    dev = torch.device("cuda")
    shapes = [(64, 96, 200), (130, 40, 33)]
    mats, descs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A = bi.uniform(140 + i, m, k, device=dev)
        B = bi.uniform(150 + i, k, n, device=dev)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
        mats.append((A, B, C))
        descs.append(hm.make_desc(A, B, C))
    handle.set_algorithm(algo)
    try:
        for use_graph in (False, True):
            hm.hmat_bq_gemm_grouped(handle, descs, mode=mode, tol=TOL, use_graph=use_graph,
                                    stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            for A, B, C in mats:
                want = oracle.bq_gemm(A.cpu().numpy(), B.cpu().numpy())
                assert rel(C.cpu().numpy(), want) <= (1e-14 if mode == "fp64" else TOL)
    finally:
        handle.set_algorithm("bilinear")


def test_two_threads_two_handles_concurrently():
    """Separate handles on separate streams from two host threads (ctypes releases the GIL)."""
    import threading
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda", 0)
    results, errors = {}, []
    cases = {t: (bi.small_int(700 + t, 150, 170), bi.small_int(710 + t, 170, 130)) for t in range(2)}

    def worker(t):
        try:
            torch.cuda.set_device(dev)
            stream = torch.cuda.Stream()
            A, B = (x.to(dev) for x in cases[t])
            C = torch.empty((8, 150, 130), dtype=torch.float64, device=dev)
            with hm.Handle() as h, torch.cuda.stream(stream):
                for _ in range(5):
                    hm.hmat_bq_gemm(h, A, B, C, mode="split" if t else "fp64", tol=TOL, stream=stream)
                stream.synchronize()
            results[t] = C.cpu().numpy()
        except Exception as e:          # reported below
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=120)
    assert not errors, errors
    for t in range(2):
        A, B = cases[t]
        np.testing.assert_array_equal(results[t], oracle.bq_gemm(A.numpy(), B.numpy()))


def _random_cases(seed, count):
    """Seeded random products: ragged m, n, k in [1, 300] (some k just above and
    below the four-multiplication limit 512), op pairs, subalgebra flags (full
    biquaternions twice as often), small-integer complex alpha and beta."""
    import random
    rng = random.Random(seed)
    flag_choices = FLAGS + [bi.BQ, bi.BQ]
    cases = []
    for i in range(count):
        m, n = rng.randint(1, 300), rng.randint(1, 300)
        k = rng.choice([rng.randint(1, 300), rng.randint(505, 520)])
        opA, opB = rng.choice(OPS), rng.choice(OPS)
        fa, fb = rng.choice(flag_choices), rng.choice(flag_choices)
        alpha = complex(rng.randint(-3, 3), rng.randint(-3, 3)) or 1.0
        beta = complex(rng.randint(-2, 2), rng.randint(-2, 2))
        cases.append((m, n, k, opA, opB, fa, fb, alpha, beta))
    return cases


@pytest.mark.parametrize("seed", [1, 2])
def test_random_products_exact_in_both_forms(handle, gauss_handle, seed):
    """24 seeded random products on small integers (every step exact): split
    mode in the default form (the four-multiplication form for full
    biquaternions with k <= 512) and in Gauss's form, and FP64 mode, each call
    alone, equal the oracle bit for bit; the same products in one grouped
    split-mode call, eager and replayed from a graph, give the same bits."""
    dev = torch.device("cuda")
    cases = _random_cases(seed, 24)
    prods = []
    for i, (m, n, k, opA, opB, fa, fb, alpha, beta) in enumerate(cases):
        A = bi.small_int(9000 + 10 * seed + 3 * i, *stored(opA, m, k), flags=fa)
        B = bi.small_int(9001 + 10 * seed + 3 * i, *stored(opB, k, n), flags=fb)
        C0 = bi.small_int(9002 + 10 * seed + 3 * i, m, n)
        want = oracle.bq_gemm(A.numpy(), B.numpy(), opA, opB, alpha=alpha, beta=beta, C=C0.numpy())
        for h, mode in ((handle, "split"), (gauss_handle, "split"), (handle, "fp64")):
            got = run(h, A, B, opA, opB, fa, fb, alpha=alpha, beta=beta, C0=C0, mode=mode)
            np.testing.assert_array_equal(got, want, err_msg=f"case {i} {cases[i]} {mode}")
        prods.append((A.to(dev), B.to(dev), C0.to(dev), want, cases[i]))
    for use_graph in (False, True):
        Cs = [p[2].clone() for p in prods]
        descs = [hm.make_desc(p[0], p[1], C, p[4][3], p[4][4], p[4][5], p[4][6], alpha=p[4][7], beta=p[4][8])
                 for p, C in zip(prods, Cs)]
        for _ in range(2 if use_graph else 1):
            for C, p in zip(Cs, prods):
                C.copy_(p[2])
            hm.hmat_bq_gemm_grouped(handle, descs, "split", TOL, stream=torch.cuda.current_stream(),
                                    use_graph=use_graph)
        torch.cuda.synchronize()
        for C, p in zip(Cs, prods):
            np.testing.assert_array_equal(C.cpu().numpy(), p[3], err_msg=f"grouped {p[4]}")
    assert handle.device_error() == 0 and gauss_handle.device_error() == 0
