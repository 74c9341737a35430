"""A plain C program drives the library through include/hmat.h only
(tests/c_abi_client.c); its results match the oracle."""
import subprocess

import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
from oracle import ops
from test_abi_and_plan import _build_c_client

pytestmark = pytest.mark.gpu


def test_c_client_matches_oracle(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = _build_c_client(tmp_path)
    m, n, k = 37, 29, 53
    A = bi.small_int(600, m, k).numpy()
    B = bi.small_int(601, k, n).numpy()
    text = f"{m} {n} {k}\n" + "\n".join(repr(float(x)) for x in np.concatenate([A.ravel(), B.ravel()]))
    r = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    vals = np.array([float(x) for x in r.stdout.split()])
    nc, na = 8 * m * n, 8 * m * k
    assert vals.size == 2 * nc + na
    want = oracle.bq_gemm(A, B)
    np.testing.assert_array_equal(vals[:nc].reshape(8, m, n), want)            # FP64 mode
    np.testing.assert_array_equal(vals[nc:2 * nc].reshape(8, m, n), want)      # split mode (integers: exact)
    np.testing.assert_array_equal(vals[2 * nc:].reshape(8, m, k), ops.add(A, A, 1.0, 2 - 1j))
