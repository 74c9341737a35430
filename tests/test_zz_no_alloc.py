"""The split-mode entry point that allocates nothing (hmat_bq_gemm_split_noalloc).

Some callers cannot allocate device memory: an application whose own memory
manager owns every device allocation, or a plug-in whose host forbids
cudaMalloc because it synchronises the device.  This entry point serves them
by keeping the split-mode workspace in a fixed array inside the library.

The tests call it through the C ABI, twice in a row with different operands,
ops and scalars, and require the same bits as the ordinary workspace-taking
hmat_bq_gemm (both run the same deterministic kernels, in either complex
form, which the entry point takes from the handle); on small integers,
where every step is exact, the result must also equal the CPU oracle.  They
pin the size limit the header documents and check that a product too large
for the fixed array is refused.  This file sorts last so that a run stopping
at its first failure has already run every other test.
"""
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


def _noalloc(handle, A, B, C, opA, opB, fa, fb, alpha, beta):
    """One call through the raw C ABI on the current stream; returns the status."""
    L = hm.lib()
    d = hm.make_desc(A, B, C, opA, opB, fa, fb, alpha, beta)
    return L.hmat_bq_gemm_split_noalloc(handle.value, d.opA, d.opB, d.flagsA, d.flagsB, d.m, d.n, d.k,
                                        d.alpha_re, d.alpha_im, d.A, d.lda, d.strideA, d.B, d.ldb, d.strideB,
                                        d.beta_re, d.beta_im, d.C, d.ldc, d.strideC, TOL,
                                        torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("form", ["auto", "gauss"])
def test_noalloc_equals_workspace_path_bit_for_bit_twice(handle, form):
    """Both follow the handle's complex form (the default takes the four-
    multiplication form at this k, Gauss's form is the paper's)."""
    handle.set_complex_form(form)
    try:
        _bit_for_bit(handle)
    finally:
        handle.set_complex_form("auto")


def _bit_for_bit(handle):
    dev = torch.device("cuda")
    m, n, k = 96, 112, 200
    calls = [(bi.uniform(501, m, k), bi.uniform(502, k, n), "N", "N", bi.BQ, bi.BQ, 1.0, 0.0),
             (bi.fock_like(503, k, m, row_scale=True), bi.uniform(504, n, k), "H", "T", bi.BQ, bi.BQ,
              0.5 - 2j, 1.5 + 0.25j),
             (bi.uniform(505, m, k, flags=bi.TRS), bi.uniform(506, k, n, flags=bi.TRA), "C", "QC", bi.TRS, bi.TRA,
              -1.0 + 1j, 0.0)]
    C0 = bi.uniform(507, m, n).to(dev)
    for A, B, opA, opB, fa, fb, alpha, beta in calls:
        A, B = A.to(dev), B.to(dev)
        ref = C0.clone()
        hm.hmat_bq_gemm(handle, A, B, ref, opA, opB, fa, fb, alpha=alpha, beta=beta, mode="split", tol=TOL)
        got = C0.clone()
        assert _noalloc(handle, A, B, got, opA, opB, fa, fb, alpha, beta) == 0
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_noalloc_equals_the_oracle_on_small_integers(handle):
    dev = torch.device("cuda")
    m, n, k = 70, 90, 130
    A = bi.small_int(511, k, m)
    B = bi.small_int(512, k, n)
    C0 = bi.small_int(513, m, n)
    want = oracle.bq_gemm(A.numpy(), B.numpy(), "H", "N", alpha=2 - 3j, beta=-1 + 2j, C=C0.numpy())
    for _ in range(2):
        got = C0.to(dev)
        assert _noalloc(handle, A.to(dev), B.to(dev), got, "H", "N", bi.BQ, bi.BQ, 2 - 3j, -1 + 2j) == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), want)


def test_noalloc_size_limit_is_the_workspace_size(handle):
    """The documented boundary: with tol 1e-12, m = n = 96, k = 256 full
    biquaternions fit the fixed array and m = n = k = 1024 does not."""
    cap = hm.lib().hmat_split_noalloc_capacity()
    assert cap == 48 << 20

    def need(m, n, k):
        d = hm.hmat_gemm_desc()              # the size query reads only ops, flags and m, n, k
        d.opA = d.opB = hm.HMAT_OP_N
        d.flagsA = d.flagsB = hm.HMAT_BQ
        d.m, d.n, d.k = m, n, k
        return hm.hmat_workspace_size(handle, [d], "split", TOL)

    assert need(96, 96, 256) <= cap
    assert need(1024, 1024, 1024) > cap


def test_noalloc_size_limit_follows_the_complex_form(handle):
    """m = n = 128, k = 320 full biquaternions: the four-multiplication form's
    workspace fits the fixed array and Gauss's form's does not, so the call
    succeeds under the default form (with the workspace path's bits) and is
    refused, before any launch, under Gauss's form."""
    dev = torch.device("cuda")
    m = n = 128
    k = 320
    cap = hm.lib().hmat_split_noalloc_capacity()
    A, B = bi.uniform(520, m, k).to(dev), bi.uniform(521, k, n).to(dev)
    C0 = bi.uniform(522, m, n).to(dev)
    d = [hm.make_desc(A, B, C0)]
    need_auto = hm.hmat_workspace_size(handle, d, "split", TOL)
    with hm.Handle() as gauss:
        gauss.set_complex_form("gauss")
        need_gauss = hm.hmat_workspace_size(gauss, d, "split", TOL)
        assert need_auto <= cap < need_gauss
        got = C0.clone()
        assert _noalloc(gauss, A, B, got, "N", "N", bi.BQ, bi.BQ, 1.0, 0.0) == 4    # WORKSPACE_TOO_SMALL
        torch.cuda.synchronize()
        assert torch.equal(got, C0)                                                 # nothing launched
    ref = C0.clone()
    hm.hmat_bq_gemm(handle, A, B, ref, mode="split", tol=TOL)
    got = C0.clone()
    assert _noalloc(handle, A, B, got, "N", "N", bi.BQ, bi.BQ, 1.0, 0.0) == 0
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_noalloc_refuses_products_beyond_its_scratch(handle):
    dev = torch.device("cuda")
    m = n = k = 1024
    A = torch.zeros((8, m, k), dtype=torch.float64, device=dev)
    B = torch.zeros((8, k, n), dtype=torch.float64, device=dev)
    C = torch.zeros((8, m, n), dtype=torch.float64, device=dev)
    with pytest.raises(hm.HmatError) as ei:
        hm.hmat_bq_gemm_split_noalloc(handle, A, B, C, tol=TOL)
    assert ei.value.status == 4          # WORKSPACE_TOO_SMALL
