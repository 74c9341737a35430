"""The split-mode entry point that allocates nothing (hmat_bq_gemm_split_noalloc).

Some callers cannot allocate device memory: code that runs while a stream is
being captured, or an application whose memory manager owns every device
allocation.  This entry point serves them by keeping the split-mode workspace
in a fixed array inside the library.  The test calls it through the C ABI
twice in a row and checks each result against the ordinary workspace-taking
hmat_bq_gemm, within the tolerance the other parity tests use; it also checks
that a product too large for the fixed array is refused.  This file sorts last
so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import bq_inputs as bi
import paper_2609_02081_gb300 as hm

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    with hm.Handle() as h:
        yield h


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_workspace_path_twice(handle):
    dev = torch.device("cuda")
    m, n, k = 96, 112, 200
    calls = [(bi.uniform(501, m, k), bi.uniform(502, k, n), "N", "N", 1.0, 0.0),
             (bi.fock_like(503, k, m, row_scale=True), bi.uniform(504, n, k), "H", "T", 0.5 - 2j, 1.5 + 0.25j)]
    C0 = bi.uniform(505, m, n).to(dev)
    for A, B, opA, opB, alpha, beta in calls:
        A, B = A.to(dev), B.to(dev)
        ref = C0.clone()
        hm.hmat_bq_gemm(handle, A, B, ref, opA, opB, alpha=alpha, beta=beta, mode="split", tol=TOL)
        got = C0.clone()
        L = hm.lib()
        d = hm.make_desc(A, B, got, opA, opB, hm.HMAT_BQ, hm.HMAT_BQ, alpha, beta)
        st = L.hmat_bq_gemm_split_noalloc(handle.value, d.opA, d.opB, d.flagsA, d.flagsB, d.m, d.n, d.k,
                                          d.alpha_re, d.alpha_im, d.A, d.lda, d.strideA, d.B, d.ldb, d.strideB,
                                          d.beta_re, d.beta_im, d.C, d.ldc, d.strideC, TOL,
                                          torch.cuda.current_stream().cuda_stream)
        assert st == 0, st
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert _rel(got, ref) <= TOL


def test_noalloc_refuses_products_beyond_its_scratch(handle):
    dev = torch.device("cuda")
    cap = hm.lib().hmat_split_noalloc_capacity()
    assert cap == 48 << 20
    m = n = k = 1024
    A = torch.zeros((8, m, k), dtype=torch.float64, device=dev)
    B = torch.zeros((8, k, n), dtype=torch.float64, device=dev)
    C = torch.zeros((8, m, n), dtype=torch.float64, device=dev)
    with pytest.raises(hm.HmatError) as ei:
        hm.hmat_bq_gemm_split_noalloc(handle, A, B, C, tol=TOL)
    assert ei.value.status == 4          # WORKSPACE_TOO_SMALL
