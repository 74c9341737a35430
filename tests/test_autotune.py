"""The autotuner (paper_2609_02081_gb300.autotune): its tables are 16 x 16 codes
that the library installs (split-mode tile width: 0 = built-in rule, 1/2/3 =
64/128/256 columns; FP64 split-k: 1..4 = 1/2/4/8 slices), saved in the JSON
format HMAT_TUNE_TABLE and bench.py --tile-table read.  A tuned table only
chooses among layouts that compute the same exact integers, so a product on
small integers gives the oracle's bits with or without it."""
import json

import numpy as np
import pytest
import torch

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm
from paper_2609_02081_gb300 import autotune


def test_save_and_load_round_trip(tmp_path):
    t = np.zeros((16, 16), dtype=np.int8)
    t[3, 5], t[10, 10] = 2, 3
    f = np.zeros((16, 16), dtype=np.int8)
    f[6, 8] = 4
    path = tmp_path / "tuned.json"
    autotune.save(t, {"3,5": {"best": 128}}, str(path), f, {"6,8": {"best_slices": 8}})
    np.testing.assert_array_equal(autotune.load(str(path)), t)
    np.testing.assert_array_equal(autotune.load_fp64(str(path)), f)
    assert json.loads(path.read_text())["report"]["3,5"]["best"] == 128
    autotune.save(t, {}, str(path))
    assert autotune.load_fp64(str(path)) is None and autotune.load_flag_tables(str(path)) == {}
    g = np.zeros((16, 16), dtype=np.int8)
    g[8, 9] = 1
    autotune.save(t, {}, str(path), flag_tables={(0x0F, 0xFF): g, (0x11, 0x11): t})
    ft = autotune.load_flag_tables(str(path))
    assert set(ft) == {(0x0F, 0xFF), (0x11, 0x11)}
    np.testing.assert_array_equal(ft[(0x0F, 0xFF)], g)
    np.testing.assert_array_equal(ft[(0x11, 0x11)], t)
    assert "table_flags_0f_ff" in json.loads(path.read_text())


def test_bins_follow_ceil_log2():
    assert [autotune._bin(x) for x in (0, 1, 2, 3, 32, 33, 1024, 1 << 20)] == [0, 0, 1, 2, 5, 6, 10, 15]


def test_greedy_bins_keeps_only_clear_gains():
    """The grouped tuner's coordinate search: a bin takes the width whose
    whole-call time is lowest, only when that beats the bin's current code by
    more than the gain fraction; later bins are timed on top of the earlier
    choices."""
    base = 100.0
    # fake call time: bin (9, 9) is 5 % faster with 128 columns, bin (7, 8)
    # 0.2 % faster with 64 (noise-sized), bin (5, 5) 3 % faster with 256 but
    # only once (9, 9) has taken 128
    def timed(t):
        ms = base
        if t[9, 9] == 2:
            ms -= 5.0
        if t[7, 8] == 1:
            ms -= 0.2
        if t[5, 5] == 3 and t[9, 9] == 2:
            ms -= 3.0
        return ms
    calls = []

    def counted(t):
        calls.append(t.copy())
        return timed(t)
    table, report = autotune.greedy_bins([(9, 9), (7, 8), (5, 5)], counted, gain=0.01)
    assert table[9, 9] == 2 and table[7, 8] == 0 and table[5, 5] == 3
    assert int(np.count_nonzero(table)) == 2
    assert len(calls) == 3 * 4
    assert report["9,9"]["kept"] == 128 and report["7,8"]["kept"] == "rule" and report["5,5"]["kept"] == 256
    assert report["7,8"]["ms"][64] == pytest.approx(94.8)
    # a start table is taken as given, and a zero gain keeps any improvement
    start = np.zeros((16, 16), dtype=np.int8)
    start[9, 9] = 2
    table2, _ = autotune.greedy_bins([(7, 8)], timed, table=start, gain=0.0)
    assert table2[9, 9] == 2 and table2[7, 8] == 1
    assert start[7, 8] == 0                                   # the caller's table is not modified


@pytest.mark.gpu
def test_grouped_tuner_runs_and_keeps_the_bits():
    """tune_grouped times candidate tables on one grouped call and returns a
    table the library installs; products keep the oracle's bits under it."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    shapes = [(96, 200, 130), (300, 64, 70), (40, 40, 2000)]
    table, report = autotune.tune_grouped(shapes, reps=1, gain=0.0)
    assert table.shape == (16, 16) and set(np.unique(table)) <= {0, 1, 2, 3}
    assert report["grouped"]["problems"] == 3 and report["grouped"]["rule_ms"] > 0
    assert {k for k in report if k != "grouped"} == {"%d,%d" % (autotune._bin(m), autotune._bin(n))
                                                    for m, n, _ in shapes}
    dev = torch.device("cuda")
    with hm.Handle() as h:
        h.set_tile_table(table)
        descs, outs = [], []
        for i, (m, n, k) in enumerate(shapes):
            A, B = bi.small_int(340 + i, m, k), bi.small_int(350 + i, k, n)
            C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
            Ad, Bd = A.to(dev), B.to(dev)
            descs.append(hm.make_desc(Ad, Bd, C))
            outs.append((A, B, C, Ad, Bd))
        hm.hmat_bq_gemm_grouped(h, descs, "split", 1e-12)
        torch.cuda.synchronize()
        for A, B, C, _, _ in outs:
            np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))
        assert h.device_error() == 0


@pytest.mark.gpu
def test_tuned_tables_install_and_keep_the_bits():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    shapes = [(96, 200, 130), (300, 64, 70)]
    table, report = autotune.tune(shapes, reps=1)
    ftable, freport = autotune.tune_fp64([(256, 256, 256)], reps=1)
    assert table.shape == (16, 16) and set(np.unique(table)) <= {0, 1, 2, 3}
    assert len(report) == 2 and all(set(r["ms"]) == {"rule", 64, 128, 256} for r in report.values())
    assert set(np.unique(ftable)) <= {0, 1, 2, 3, 4} and len(freport) == 1
    dev = torch.device("cuda")
    with hm.Handle() as h:
        h.set_tile_table(table)
        h.set_fp64_splitk_table(ftable)
        for (m, n, k), mode in [(shapes[0], "split"), (shapes[1], "split"), ((256, 256, 256), "fp64")]:
            A, B = bi.small_int(300 + m, m, k), bi.small_int(301 + n, k, n)
            C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
            hm.hmat_bq_gemm(h, A.to(dev), B.to(dev), C, mode=mode, tol=1e-12)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))
        assert h.device_error() == 0


@pytest.mark.gpu
def test_flag_pair_table_applies_to_its_pair_only():
    """A tile table installed for one flag pair changes the layout (hence the
    workspace size) of products with exactly those flags, leaves others on the
    general rule, keeps the oracle's bits, and is removed again by None."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda")
    m, n, k = 200, 300, 150
    code1 = np.full((16, 16), 2, dtype=np.int8)       # 128-wide tiles: 384 padded columns of n = 300, not 320
    with hm.Handle() as h:
        def ws(fa, fb):
            A = torch.zeros((8, m, k), dtype=torch.float64, device=dev)
            B = torch.zeros((8, k, n), dtype=torch.float64, device=dev)
            C = torch.zeros((8, m, n), dtype=torch.float64, device=dev)
            return hm.hmat_workspace_size(h, [hm.make_desc(A, B, C, flagsA=fa, flagsB=fb)], "split", 1e-12)
        base_trs, base_bq = ws(bi.TRS, bi.BQ), ws(bi.BQ, bi.BQ)
        h.set_tile_table_flags(bi.TRS, bi.BQ, code1)
        assert ws(bi.TRS, bi.BQ) != base_trs and ws(bi.BQ, bi.BQ) == base_bq
        A, B = bi.small_int(320, m, k, flags=bi.TRS), bi.small_int(321, k, n)
        C = torch.full((8, m, n), float("nan"), dtype=torch.float64, device=dev)
        hm.hmat_bq_gemm(h, A.to(dev), B.to(dev), C, flagsA=bi.TRS, flagsB=bi.BQ, mode="split", tol=1e-12)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(C.cpu().numpy(), oracle.bq_gemm(A.numpy(), B.numpy()))
        h.set_tile_table_flags(bi.TRS, bi.BQ, None)
        assert ws(bi.TRS, bi.BQ) == base_trs
        with pytest.raises(hm.HmatError):
            h.set_tile_table_flags(0x100, bi.BQ, code1)
        assert h.device_error() == 0
