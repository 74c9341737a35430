"""Streamed (out-of-core) products: host-resident operands through a bounded
device budget (hmat_bq_gemm_streamed) against the in-core call and the oracle.

With kb = k every C block is the same computation as in hmat_bq_gemm, so the
two agree bit for bit in both modes; with the inner dimension chunked the
result is compared with the oracle within the mode's tolerance.
"""
import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm

pytestmark = pytest.mark.gpu
TOL = 1e-12
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


def in_core(handle, A, B, C0, opA, opB, fa, fb, alpha, beta, mode):
    C = C0.to(DEV)
    hm.hmat_bq_gemm(handle, A.to(DEV), B.to(DEV), C, opA, opB, fa, fb, alpha, beta, mode=mode, tol=TOL)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def budget_for(m, n, k, mode, blocks, opA="N", opB="N", fa=bi.BQ, fb=bi.BQ, on_host=(True, True, True)):
    """Smallest power-of-two budget whose plan still keeps kb = k, with at least `blocks` C blocks per side."""
    b = 1 << 22
    while True:
        try:
            mb, nb, kb, nbytes = hm.streamed_plan(m, n, k, opA, opB, fa, fb, mode, TOL, b, on_host)
            if kb == k:
                return b, (mb, nb)
        except hm.HmatError:
            pass
        b *= 2


@pytest.mark.parametrize("mode", ["fp64", "split"])
@pytest.mark.parametrize("opA,opB,fa,fb", [("N", "N", bi.BQ, bi.BQ), ("H", "T", bi.BQ, bi.TRA),
                                           ("C", "QC", bi.TRS, bi.BQ)])
def test_streamed_equals_in_core(handle, mode, opA, opB, fa, fb):
    m, n, k = 333, 400, 517
    A = bi.uniform(400, *stored(opA, m, k), flags=fa).pin_memory()
    B = bi.uniform(401, *stored(opB, k, n), flags=fb).pin_memory()
    C0 = bi.uniform(402, m, n)
    alpha, beta = 0.5 - 1j, 1 + 0.25j
    want = in_core(handle, A, B, C0, opA, opB, fa, fb, alpha, beta, mode)
    budget, (mb, nb) = budget_for(m, n, k, mode, 3, opA, opB, fa, fb)
    assert mb < m and nb < n                       # several blocks each way
    C = C0.clone().pin_memory()
    hm.hmat_bq_gemm_streamed(handle, A, B, C, opA, opB, fa, fb, alpha, beta, mode=mode, tol=TOL, budget=budget)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.numpy(), want)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_streamed_mixed_placement(handle, mode):
    """A on the device, B and C on the host; then C on the device; beta = 0 (C not read)."""
    m, n, k = 260, 300, 350
    A = bi.uniform(410, m, k)
    B = bi.uniform(411, k, n).pin_memory()
    want = in_core(handle, A, B, torch.zeros(8, m, n, dtype=torch.float64), "N", "N", bi.BQ, bi.BQ, 1.0, 0.0,
                   mode)
    dA = A.to(DEV)
    budget, _ = budget_for(m, n, k, mode, 2, on_host=(False, True, True))
    C = torch.full((8, m, n), float("nan"), dtype=torch.float64).pin_memory()
    hm.hmat_bq_gemm_streamed(handle, dA, B, C, mode=mode, tol=TOL, budget=budget)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.numpy(), want)
    dC = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=DEV)
    budget, _ = budget_for(m, n, k, mode, 2, on_host=(False, True, False))
    hm.hmat_bq_gemm_streamed(handle, dA, B, dC, mode=mode, tol=TOL, budget=budget)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dC.cpu().numpy(), want)


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_streamed_chunked_inner_dimension(handle, mode):
    """A budget too small for a whole k: chunks accumulate with beta = 1."""
    m, n, k = 200, 180, 3000
    A = bi.uniform(420, m, k).pin_memory()
    B = bi.uniform(421, k, n).pin_memory()
    C0 = bi.uniform(422, m, n)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), alpha=2.0, beta=-1.0, C=C0.numpy())
    budget = 1 << 22
    while True:
        try:
            mb, nb, kb, _ = hm.streamed_plan(m, n, k, mode=mode, tol=TOL, budget=budget)
            break
        except hm.HmatError:
            budget *= 2
    assert kb < k
    C = C0.clone().pin_memory()
    hm.hmat_bq_gemm_streamed(handle, A, B, C, alpha=2.0, beta=-1.0, mode=mode, tol=TOL, budget=budget)
    torch.cuda.synchronize()
    err = np.linalg.norm(C.numpy() - want) / np.linalg.norm(want)
    assert err <= (1e-14 if mode == "fp64" else TOL), err


def test_streamed_budget_too_small(handle):
    A = bi.uniform(430, 64, 64).pin_memory()
    C = torch.empty((8, 64, 64), dtype=torch.float64).pin_memory()
    ws = torch.empty(1 << 10, dtype=torch.uint8, device=DEV)
    with pytest.raises(hm.HmatError) as ei:
        hm.hmat_bq_gemm_streamed(handle, A, A, C, mode="split", tol=TOL, workspace=ws)
    assert ei.value.status == 4


@pytest.mark.parametrize("mode", ["fp64", "split"])
def test_streamed_degenerate_shapes(handle, mode):
    """k = 0 (C <- beta C), a single row, and m = 0 through the streamed path."""
    m, n = 130, 70
    A = torch.empty((8, m, 0), dtype=torch.float64).pin_memory()
    B = torch.empty((8, 0, n), dtype=torch.float64).pin_memory()
    C0 = bi.uniform(440, m, n)
    C = C0.clone().pin_memory()
    hm.hmat_bq_gemm_streamed(handle, A, B, C, beta=2 - 1j, mode=mode, tol=TOL, budget=64 << 20)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(C.numpy(), oracle.bq_gemm(A.numpy(), B.numpy(), beta=2 - 1j, C=C0.numpy()))
    A1 = bi.uniform(441, 1, 300).pin_memory()
    B1 = bi.uniform(442, 300, 1).pin_memory()
    C1 = torch.empty((8, 1, 1), dtype=torch.float64).pin_memory()
    hm.hmat_bq_gemm_streamed(handle, A1, B1, C1, mode=mode, tol=TOL, budget=64 << 20)
    torch.cuda.synchronize()
    want = oracle.bq_gemm(A1.numpy(), B1.numpy())
    assert np.linalg.norm(C1.numpy() - want) <= TOL * np.linalg.norm(want)
    A0 = torch.empty((8, 0, 10), dtype=torch.float64).pin_memory()
    C0e = torch.empty((8, 0, 1), dtype=torch.float64).pin_memory()
    hm.hmat_bq_gemm_streamed(handle, A0, bi.uniform(443, 10, 1).pin_memory(), C0e, mode=mode, tol=TOL,
                             budget=64 << 20)


@pytest.mark.parametrize("opA,opB,fa,fb", [("N", "N", bi.BQ, bi.BQ), ("H", "T", bi.TRS, bi.TRA),
                                           ("C", "N", bi.BQ, bi.COMPLEX)])
def test_streamed_b_cache_equals_in_core(handle, opA, opB, fa, fb):
    """Split mode, host operands, 4 x 4 blocks with every column block's encoded B kept in the budget:
    A rows and B columns are each encoded once, and the result equals the in-core product bit for bit."""
    m, n, k = 1100, 1030, 700
    A = bi.uniform(450, *stored(opA, m, k), flags=fa).pin_memory()
    B = bi.uniform(451, *stored(opB, k, n), flags=fb).pin_memory()
    C0 = bi.uniform(452, m, n)
    want = in_core(handle, A, B, C0, opA, opB, fa, fb, 1 - 1j, 0.5, "split")
    budget = 6 << 30
    mb, nb, kb, _ = hm.streamed_plan(m, n, k, opA, opB, fa, fb, "split", TOL, budget)
    assert kb == k and mb < m and nb < n and mb == nb          # the cached-B block plan
    C = C0.clone().pin_memory()
    handle.set_profiling(True)
    handle.reset_profile()
    hm.hmat_bq_gemm_streamed(handle, A, B, C, opA, opB, fa, fb, 1 - 1j, 0.5, mode="split", tol=TOL, budget=budget)
    torch.cuda.synchronize()
    enc = handle.profile("split_encode")[0]
    gemm = handle.profile("split_residue_gemm")[0]
    handle.set_profiling(False)
    np.testing.assert_array_equal(C.numpy(), want)
    blocks_i, blocks_j = -(-m // mb), -(-n // nb)
    assert gemm == blocks_i * blocks_j
    # encoder launches: one per block row (A; the ragged last column block re-encodes it) plus B in row 0
    assert enc <= blocks_i * 2 + blocks_j
