"""Full-size configurations, checked on sampled output elements against the oracle
and over the whole matrix by a random-vector (Freivalds) check.

The oracle computes C[rows, cols] directly from A's rows and B's columns (the
plain definition restricted to those elements), so only a small sample has to
leave the GPU; the Freivalds check compares C x with op(A) (op(B) x).
"""
import os

import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with hm.Handle() as h:
        yield h
        assert h.device_error() == 0


def sampled_check(A, B, C, opA, opB, rows, cols):
    """Relative Frobenius error of C[:, rows, cols] against the oracle."""
    tA = opA in ("T", "H")
    tB = opB in ("T", "H")
    r = torch.as_tensor(rows, device=A.device)
    c = torch.as_tensor(cols, device=B.device)
    Asub = (A[:, :, r] if tA else A[:, r, :]).cpu().numpy()
    Bsub = (B[:, c, :] if tB else B[:, :, c]).cpu().numpy()
    want = oracle.bq_gemm(Asub, Bsub, opA, opB)
    got = C[:, r, :][:, :, c].cpu().numpy()
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def freivalds(A, B, C, opA, opB, seed):
    """Whole-matrix check of C = op(A) op(B) (Freivalds): for a random
    biquaternion vector x, ||C x - op(A) (op(B) x)|| / (||C||_F ||x||), with
    both sides computed by the oracle on the host.  ||C - C*||_F <= tol ||C*||_F
    bounds it by tol plus the rounding of the FP64 matrix-vector products."""
    k = C.shape[2]
    x = bi.uniform(seed, k, 1).numpy()
    An, Bn, Cn = A.cpu().numpy(), B.cpu().numpy(), C.cpu().numpy()
    y1 = oracle.bq_gemm(Cn, x)
    y2 = oracle.bq_gemm(An, oracle.bq_gemm(Bn, x, opB, "N"), opA, "N")
    return float(np.linalg.norm(y1 - y2) / (np.linalg.norm(Cn) * np.linalg.norm(x)))


def freivalds_gpu(handle, A, B, C, seed):
    """The same check with the matrix-vector products on the GPU through the
    library's FP64 mode (n = 1), for operands too large to copy to the host.
    Those products are compared with the oracle by the other tests, and a wrong
    tile of C cannot cancel out of both sides."""
    dev = C.device
    x = bi.uniform(seed, C.shape[2], 1, device=dev)
    y1 = torch.empty((8, C.shape[1], 1), dtype=torch.float64, device=dev)
    t = torch.empty((8, B.shape[1], 1), dtype=torch.float64, device=dev)
    y2 = torch.empty_like(y1)
    hm.hmat_bq_gemm(handle, C, x, y1, mode="fp64")
    hm.hmat_bq_gemm(handle, B, x, t, mode="fp64")
    hm.hmat_bq_gemm(handle, A, t, y2, mode="fp64")
    return float(torch.linalg.norm(y1 - y2) / (torch.linalg.norm(C) * torch.linalg.norm(x)))


CASES_4096 = [("BQ x BQ, op N,N", bi.BQ, bi.BQ, "N", "N"),
              ("TRS x TRA, op N,N", bi.TRS, bi.TRA, "N", "N"),
              ("BQ x BQ, op(A) = H", bi.BQ, bi.BQ, "H", "N")]


@pytest.mark.parametrize("mode", ["split", "fp64"])
@pytest.mark.parametrize("name,fa,fb,opA,opB", CASES_4096)
def test_config_n4096_fock_like(handle, mode, name, fa, fb, opA, opB):
    """m = n = k = 4096, N(0,1) exp(-|i-j|/200) entries; 96 x 96 sampled output block."""
    dev = torch.device("cuda")
    n = 4096
    A = bi.fock_like(201, n, n, flags=fa, device=dev)
    B = bi.fock_like(202, n, n, flags=fb, device=dev)
    C = torch.full((8, n, n), float("nan"), dtype=torch.float64, device=dev)
    hm.hmat_bq_gemm(handle, A, B, C, opA, opB, fa, fb, mode=mode, tol=TOL)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(n, 96, replace=False))
    cols = np.sort(rng.choice(n, 96, replace=False))
    err = sampled_check(A, B, C, opA, opB, rows, cols)
    assert err <= (1e-14 if mode == "fp64" else TOL), err
    assert torch.isfinite(C).all()
    fv = freivalds(A, B, C, opA, opB, 7)
    assert fv <= (1e-14 if mode == "fp64" else TOL + 1e-14), fv


# Mixed subalgebras at scale (the reduced plans of Sec. III B, last
# paragraph: absent terms omitted) and a rectangular product.
CASES_MIXED = [("R x BQ", bi.REAL, bi.BQ, 4096, 4096, 4096, "N", "N"),
               ("C x BQ", bi.COMPLEX, bi.BQ, 4096, 4096, 4096, "N", "N"),
               ("TRS x BQ", bi.TRS, bi.BQ, 4096, 4096, 4096, "N", "N"),
               ("BQ x TRA, op(B) = H", bi.BQ, bi.TRA, 4096, 4096, 4096, "N", "H"),
               ("C x C", bi.COMPLEX, bi.COMPLEX, 4096, 4096, 4096, "N", "N"),
               ("BQ x BQ rectangular 8192 x 2048 x 16384", bi.BQ, bi.BQ, 8192, 2048, 16384, "N", "N")]


@pytest.mark.parametrize("mode", ["split", "fp64"])
@pytest.mark.parametrize("name,fa,fb,m,n,k,opA,opB", CASES_MIXED)
def test_mixed_subalgebras_and_rectangular_at_scale(handle, mode, name, fa, fb, m, n, k, opA, opB):
    dev = torch.device("cuda")
    A = bi.fock_like(211, *((k, m) if opA in ("T", "H") else (m, k)), flags=fa, device=dev)
    B = bi.fock_like(212, *((n, k) if opB in ("T", "H") else (k, n)), flags=fb, device=dev)
    C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
    hm.hmat_bq_gemm(handle, A, B, C, opA, opB, fa, fb, mode=mode, tol=TOL)
    torch.cuda.synchronize()
    rng = np.random.default_rng(23)
    rows = np.sort(rng.choice(m, 64, replace=False))
    cols = np.sort(rng.choice(n, 64, replace=False))
    err = sampled_check(A, B, C, opA, opB, rows, cols)
    assert err <= (1e-14 if mode == "fp64" else TOL), err
    assert torch.isfinite(C).all()
    fv = freivalds(A, B, C, opA, opB, 29)
    assert fv <= (1e-14 if mode == "fp64" else TOL + 1e-14), fv


def test_config_n8192_split_whole_matrix(handle):
    """The n = 8192 precision workload (Fock-like, rows scaled over six
    decades) in split mode: every output element enters a Freivalds check
    against the oracle, and a 64 x 64 sampled block is compared directly."""
    dev = torch.device("cuda")
    n = 8192
    A = bi.fock_like(103, n, n, row_scale=True, device=dev)
    B = bi.fock_like(104, n, n, row_scale=True, device=dev)
    C = torch.full((8, n, n), float("nan"), dtype=torch.float64, device=dev)
    hm.hmat_bq_gemm(handle, A, B, C, mode="split", tol=TOL)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    rows = np.sort(rng.choice(n, 64, replace=False))
    cols = np.sort(rng.choice(n, 64, replace=False))
    err = sampled_check(A, B, C, "N", "N", rows, cols)
    assert err <= TOL, err
    fv = freivalds(A, B, C, "N", "N", 13)
    assert fv <= TOL + 1e-14, fv
    fg = freivalds_gpu(handle, A, B, C, 13)       # the form the n = 24576 check uses
    assert abs(fg - fv) <= 1e-14, (fg, fv)


# Component strides above 2^32 bytes (the n = 24576 configuration's 64-bit
# offsets) in seconds: one operand at 24576 x 24576 (4.8 GB per component),
# the others thin.  FP64 mode goes through hmat_bq_gemm; split mode's
# workspace for such a product (hundreds of GB of encoded factors and
# residues) exceeds HBM, so it runs through the streamed call with the
# operands left in device memory, whose blocks index the same 24576-row
# components with 64-bit offsets.
BIG = 24576
CASES_64BIT = [("C wide: m = n = 24576, k = 256", BIG, BIG, 256, "N"),
               ("A large: m = k = 24576, n = 256", BIG, 256, BIG, "N"),
               ("A large, op(A) = H: m = k = 24576, n = 256", BIG, 256, BIG, "H"),
               ("B large: n = k = 24576, m = 256", 256, BIG, BIG, "N")]


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("name,m,n,k,opA", CASES_64BIT)
def test_component_strides_beyond_4gb(handle, mode, name, m, n, k, opA):
    dev = torch.device("cuda")
    if opA in ("T", "H"):
        A = bi.fock_like(301, k, m, device=dev)
    else:
        A = bi.fock_like(301, m, k, device=dev)
    B = bi.fock_like(302, k, n, device=dev)
    C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
    assert max(A.stride(0), B.stride(0), C.stride(0)) * 8 > (1 << 32)
    if mode == "fp64":
        hm.hmat_bq_gemm(handle, A, B, C, opA, "N", mode="fp64")
    else:
        hm.hmat_bq_gemm_streamed(handle, A, B, C, opA, "N", mode="split", tol=TOL, budget=40 << 30)
    torch.cuda.synchronize()
    # The tolerance bounds the relative Frobenius error of the whole matrix, so
    # the sample must hold entries of the band (|C| ~ 1 near the diagonal of
    # these banded operands) as well as far ones (down to e^-60 of the band);
    # the last row and column sit at the largest offsets and are always in.
    rng = np.random.default_rng(17)
    rows = np.unique(np.concatenate([rng.choice(min(m, 2048), 12, replace=False),
                                     rng.choice(m, 12, replace=False), [m - 1]]))
    cols = np.unique(np.concatenate([rng.choice(min(n, 2048), 12, replace=False),
                                     rng.choice(n, 12, replace=False), [n - 1]]))
    err = sampled_check(A, B, C, opA, "N", rows, cols)
    assert err <= (1e-14 if mode == "fp64" else TOL), err
    assert torch.isfinite(C).all()
    if opA == "N":
        fv = freivalds_gpu(handle, A, B, C, 19)
        assert fv <= (1e-14 if mode == "fp64" else TOL + 1e-14), fv


@pytest.mark.skipif(os.environ.get("HMAT_RUN_LARGE") != "1",
                    reason="n = 24576 FP64 takes ~13 minutes on GB300 (set HMAT_RUN_LARGE=1)")
def test_config_n24576_fp64(handle):
    """m = n = k = 24576 FP64 (the complex isomorph would exceed 2^31 elements),
    Fock-like inputs, ~116 GB resident; 64 x 64 sampled output block."""
    dev = torch.device("cuda")
    n = 24576
    A = bi.fock_like(205, n, n, device=dev)
    B = bi.fock_like(206, n, n, device=dev)
    C = torch.empty((8, n, n), dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    hm.hmat_bq_gemm(handle, A, B, C, mode="fp64")
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(n, 64, replace=False))
    cols = np.sort(rng.choice(n, 64, replace=False))
    err = sampled_check(A, B, C, "N", "N", rows, cols)
    # whole matrix: C x against A (B x); three 39 GB operands stay on the GPU
    fv = freivalds_gpu(handle, A, B, C, 15)
    print(f"n=24576 fp64: {ms:.0f} ms, {64 * 2 * n**3 / (ms * 1e-3) / 1e12:.3f} TFLOP/s 64-equiv, "
          f"{24 * 2 * n**3 / (ms * 1e-3) / 1e12:.3f} executed, sampled error {err:.3e}, Freivalds {fv:.3e}")
    assert err <= 1e-14
    assert fv <= 1e-14


def test_streamed_n8192_from_host_equals_in_core(handle):
    """The n = 8192 precision workload with A, B, C in pinned host memory and a
    24 GB device budget: every block equals the in-core product bit for bit."""
    n = 8192
    dA = bi.fock_like(103, n, n, row_scale=True, device="cuda")
    dB = bi.fock_like(104, n, n, row_scale=True, device="cuda")
    dC = torch.empty((8, n, n), dtype=torch.float64, device="cuda")
    hm.hmat_bq_gemm(handle, dA, dB, dC, mode="split", tol=TOL)
    want = dC.cpu().numpy()
    A, B = dA.cpu().pin_memory(), dB.cpu().pin_memory()
    del dA, dB, dC
    torch.cuda.empty_cache()
    C = torch.empty((8, n, n), dtype=torch.float64).pin_memory()
    budget = 24 << 30
    mb, nb, kb, _ = hm.streamed_plan(n, n, n, mode="split", tol=TOL, budget=budget)
    assert kb == n and mb < n
    hm.hmat_bq_gemm_streamed(handle, A, B, C, mode="split", tol=TOL, budget=budget)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.numpy(), want)
