"""Environment switches read at handle creation: HMAT_LOG and HMAT_TUNE_TABLE."""
import json

import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_hmat_log_prints_one_line_per_call(monkeypatch, capfd):
    monkeypatch.setenv("HMAT_LOG", "1")
    A = bi.small_int(500, 20, 30).cuda()
    B = bi.small_int(501, 30, 10).cuda()
    C = torch.empty((8, 20, 10), dtype=torch.float64, device="cuda")
    with hm.Handle() as h:
        hm.hmat_bq_gemm(h, A, B, C, mode="split", tol=1e-12)
        torch.cuda.synchronize()
    err = capfd.readouterr().err
    lines = [x for x in err.splitlines() if x.startswith("hmat: hmat_bq_gemm ")]
    assert len(lines) == 1 and "m=20 n=10 k=30 mode=split algo=bilinear -> success" in lines[0]
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.cpu().numpy(), B.cpu().numpy()))


def test_hmat_tune_table_file(monkeypatch, capfd, tmp_path):
    """A valid table is installed (results unchanged); a broken file warns and keeps the built-in rule."""
    A = bi.uniform(502, 300, 200).cuda()
    B = bi.uniform(503, 200, 260).cuda()
    want = None
    for content in [None, {"table": [[1] * 16] * 16}, {"table": [[3] * 16] * 16}, "not json"]:
        if content is None:
            monkeypatch.delenv("HMAT_TUNE_TABLE", raising=False)
        else:
            path = tmp_path / "table.json"
            path.write_text(content if isinstance(content, str) else json.dumps(content))
            monkeypatch.setenv("HMAT_TUNE_TABLE", str(path))
        C = torch.empty((8, 300, 260), dtype=torch.float64, device="cuda")
        with hm.Handle() as h:
            hm.hmat_bq_gemm(h, A, B, C, mode="split", tol=1e-12)
            torch.cuda.synchronize()
        got = C.cpu().numpy()
        if want is None:
            want = got
        np.testing.assert_array_equal(got, want)       # tile widths never change the exact result
    assert "HMAT_TUNE_TABLE" in capfd.readouterr().err  # the broken file was reported


def test_hmat_tune_table_flag_pair_entries(monkeypatch, tmp_path):
    """A "table_flags_AA_BB" entry of the file is installed for its flag pair:
    the workspace of a TRS x BQ product follows it (128-wide tiles: 384 padded
    columns of n = 300 instead of 320) while a BQ x BQ product keeps the
    general table; results are the oracle's bits."""
    dev = torch.device("cuda")
    m, n, k = 200, 300, 150
    zeros = [[0] * 16] * 16
    path = tmp_path / "flags.json"
    path.write_text(json.dumps({"table": zeros, "table_flags_0f_ff": [[2] * 16] * 16}))

    def sizes():
        A = torch.zeros((8, m, k), dtype=torch.float64, device=dev)
        B = torch.zeros((8, k, n), dtype=torch.float64, device=dev)
        C = torch.zeros((8, m, n), dtype=torch.float64, device=dev)
        with hm.Handle() as h:
            return [hm.hmat_workspace_size(h, [hm.make_desc(A, B, C, flagsA=fa, flagsB=bi.BQ)], "split", 1e-12)
                    for fa in (bi.TRS, bi.BQ)]
    monkeypatch.delenv("HMAT_TUNE_TABLE", raising=False)
    base = sizes()
    monkeypatch.setenv("HMAT_TUNE_TABLE", str(path))
    tuned = sizes()
    assert tuned[0] != base[0] and tuned[1] == base[1]
    A, B = bi.small_int(330, m, k, flags=bi.TRS), bi.small_int(331, k, n)
    C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
    with hm.Handle() as h:
        hm.hmat_bq_gemm(h, A.to(dev), B.to(dev), C, flagsA=bi.TRS, mode="split", tol=1e-12)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))
