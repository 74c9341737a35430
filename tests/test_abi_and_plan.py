"""Host-side checks (no GPU): the C-ABI library, the product plans, split-mode parameters."""
import itertools
import math
import random
import os
import re

import numpy as np
import pytest

import bq_inputs as bi
import oracle
import paper_2609_02081_gb300 as hm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hmat.h")
FLAGS = [bi.REAL, bi.COMPLEX, bi.TRS, bi.TRA, bi.BQ]
FLAG_NAME = {bi.REAL: "R", bi.COMPLEX: "C", bi.TRS: "TRS", bi.TRA: "TRA", bi.BQ: "BQ"}
OPS = ["N", "T", "C", "H", "QC"]


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hmat_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = hm.lib()
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
        assert name in hm.SIGNATURES, f"binding lacks {name}"
    assert set(hm.SIGNATURES) == set(names)
    assert L.hmat_version() >= 100
    assert L.hmat_status_string(0) == b"success"
    assert L.hmat_status_string(4) == b"workspace too small"


def test_library_exports_only_the_c_abi():
    """The shared library's exported functions are exactly the header's entry
    points (internal symbols are hidden)."""
    import shutil
    import subprocess
    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm not available")
    hm.lib()
    out = subprocess.run([nm, "-D", "--defined-only", hm.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = sorted(line.split()[-1] for line in out.splitlines() if line.split()[1:2] == ["T"])
    assert exported == declared_functions()


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hm.HmatError) as ei:
        hm.Handle()
    assert ei.value.status == 5   # CUDA_ERROR


def structure_tensor(opA, opB):
    """T[e, c, d]: component e of op(a) op(b) for one-hot 1x1 a (component c), b (component d)."""
    T = np.zeros((8, 8, 8))
    for c in range(8):
        a = np.zeros((8, 1, 1)); a[c] = 1.0
        for d in range(8):
            b = np.zeros((8, 1, 1)); b[d] = 1.0
            T[:, c, d] = oracle.bq_gemm(a, b, opA, opB)[:, 0, 0]
    return T


@pytest.mark.parametrize("fa,fb", list(itertools.product(FLAGS, FLAGS)))
def test_plan_reproduces_structure_tensor(fa, fb):
    for opA, opB in [("N", "N"), ("T", "H"), ("C", "QC"), ("H", "N")]:
        P, U, V, W, _ = hm.plan_info(opA, opB, fa, fb)
        T = structure_tensor(opA, opB)
        got = np.einsum("ep,pc,pd->ecd", W, U.astype(float), V.astype(float))
        mask = np.zeros((8, 8, 8), bool)
        for c in range(8):
            for d in range(8):
                mask[:, c, d] = bool((fa >> c) & 1) and bool((fb >> d) & 1)
        np.testing.assert_array_equal(got[mask], T[mask])
        # absent components are never read
        for c in range(8):
            if not (fa >> c) & 1:
                assert np.all(U[:, c] == 0)
            if not (fb >> c) & 1:
                assert np.all(V[:, c] == 0)


def test_four_multiplication_form_reproduces_structure_tensor():
    """The split mode's four-multiplication form of the full plan (the eight
    complex products of Eq. bilinearH, each as Re = Re X Re Y - Im X Im Y and
    Im = Re X Im Y + Im X Re Y): 16 products of two terms each reproduce the
    product for every op pair, use only Re and Im factors (no Gauss sums), 16
    per side, and both terms of a product carry its weight (the second with
    its sign)."""
    for opA, opB in itertools.product(OPS, OPS):
        P, U, V, W, strategy = hm.plan_info(opA, opB, bi.BQ, bi.BQ, algo="four_m")
        assert P == 32 and strategy == 0
        T = structure_tensor(opA, opB)
        got = np.einsum("ep,pc,pd->ecd", W, U.astype(float), V.astype(float))
        np.testing.assert_array_equal(got, T)
        for side in (U, V):
            for row in side:
                assert not (np.any(row[:4]) and np.any(row[4:])), "a Gauss Re + Im factor"
            assert len({tuple(r) for r in side}) == 16
        for q in range(16):
            a, b = np.abs(W[:, 2 * q]), np.abs(W[:, 2 * q + 1])
            np.testing.assert_array_equal(a, b)
            assert np.count_nonzero(a) in (1, 4)
    # the same eight complex products as Gauss's plan: per output, the weights
    # of the products (not the terms) sum to at most 12 / 4 in magnitude
    _, _, _, W, _ = hm.plan_info("N", "N", bi.BQ, bi.BQ, algo="four_m")
    assert np.abs(W[:, 0::2]).sum(axis=1).max() == 3.0
    # other flag pairs keep the bilinear plan
    for fa, fb in [(bi.TRS, bi.BQ), (bi.COMPLEX, bi.COMPLEX), (bi.BQ, bi.TRA)]:
        four, gauss = hm.plan_info("N", "N", fa, fb, algo="four_m"), hm.plan_info("N", "N", fa, fb)
        assert four[0] == gauss[0]
        for x, y in zip(four[1:4], gauss[1:4]):
            np.testing.assert_array_equal(x, y)


def test_bilinear_24_and_reduced_counts():
    """Sec. III B: 64 -> 24 for full biquaternions, 16 -> 8 for real / imaginary quaternions."""
    counts = {(FLAG_NAME[a], FLAG_NAME[b]): hm.plan_info("N", "N", a, b)[0] for a in FLAGS for b in FLAGS}
    assert counts[("BQ", "BQ")] == 24
    assert hm.plan_info("N", "N", bi.BQ, bi.BQ)[4] == 0          # the paper's bilinear scheme
    for pair in [("TRS", "TRS"), ("TRA", "TRA"), ("TRS", "TRA"), ("TRA", "TRS")]:
        assert counts[pair] == 8
    want = {("R", "R"): 1, ("R", "C"): 2, ("R", "TRS"): 4, ("R", "TRA"): 4, ("R", "BQ"): 8,
            ("C", "C"): 3, ("C", "TRS"): 8, ("C", "TRA"): 8, ("C", "BQ"): 12,
            ("TRS", "BQ"): 16, ("TRA", "BQ"): 16}
    for (a, b), n in want.items():
        assert counts[(a, b)] == n, (a, b, counts[(a, b)])
        assert counts[(b, a)] == n, (b, a, counts[(b, a)])


def test_bq_plan_weights_are_the_papers():
    """Full plan: 8 complex products, weights 2 or 1/4 (Eq. bilinearH), Gauss triplets."""
    P, U, V, W, _ = hm.plan_info("N", "N", bi.BQ, bi.BQ)
    vals = set(np.round(np.abs(W[W != 0]), 6))
    assert vals <= {2.0, 0.25}
    # Gauss: every product is Re*Re, Im*Im or (Re+Im)*(Re+Im) of one complex factor
    kinds = []
    for p in range(P):
        re_l, im_l = U[p, :4] != 0, U[p, 4:] != 0
        re_r, im_r = V[p, :4] != 0, V[p, 4:] != 0
        kinds.append((re_l.any(), im_l.any(), re_r.any(), im_r.any()))
    assert kinds.count((True, False, True, False)) == 8
    assert kinds.count((False, True, False, True)) == 8
    assert kinds.count((True, True, True, True)) == 8


def _coprime(a, b):
    return math.gcd(a, b) == 1


@pytest.mark.parametrize("k,tol", [(1, 1e-12), (256, 1e-12), (4096, 1e-12), (8192, 1e-12), (24576, 1e-12),
                                   (1024, 1e-6), (8192, 1e-14)])
def test_split_parameters(k, tol):
    mods, bits = hm.split_info(k, tol)
    assert all(m % 2 == 1 and 129 < m <= 255 for m in mods)
    assert all(_coprime(a, b) for a, b in itertools.combinations(mods, 2))
    log2P = sum(math.log2(m) for m in mods)
    # CRT range covers the exact integer outputs: |Q| <= 8 k 2^(2b), P > 2|Q|
    assert log2P > 2 * bits + math.log2(max(k, 1)) + 4
    # the scaling error 2^-b sits below the target
    assert 2.0 ** (-bits) < tol / 16
    # residues in [-127, 127]: 1024-deep FP32 sums of products stay exact
    assert 1024 * 127 * 127 < 2 ** 24


def test_split_crt_margin_every_k():
    """The CRT takes its quotient as the nearest integer to a float estimate of
    S / P, which needs the exact outputs |Q| <= 8 k 2^(2b) to stay below
    P / 2^1.25 (|Q| < 0.42 P): every k the library accepts at tol 1e-12, and a
    spread of k at other tolerances, leaves that margin.  Integer check:
    (8 k 2^(2b))^4 * 2^5 < P^4."""
    def margin_ok(k, tol):
        try:
            mods, bits = hm.split_info(k, tol)
        except hm.HmatError:
            return True
        P = math.prod(mods)
        return (8 * k * 4 ** bits) ** 4 * 32 < P ** 4
    assert all(margin_ok(k, 1e-12) for k in range(1, 127 * 1024 + 1))
    ks = sorted({1, 3, 100, 127 * 1024} | {2 ** e + d for e in range(2, 17) for d in (-1, 0, 1)})
    for tol in (1e-3, 1e-6, 1e-9, 1e-13, 1e-14):
        assert all(margin_ok(k, tol) for k in ks), tol


def test_plan_weight_sums_within_the_crt_bound():
    """Every plan's output weights satisfy sum_p |4 w| <= 36, the bound behind
    the CRT's sums (|4Q| <= 36 * 127 with centred residues), which sizes their
    offset N P and the quotient estimate."""
    flags = [bi.REAL, bi.COMPLEX, bi.TRS, bi.TRA, bi.BQ, 0x03, 0x55, 0x81]
    worst = 0.0
    for algo in ("bilinear", "standard"):
        for fa, fb in itertools.product(flags, flags):
            for opA, opB in (("N", "N"), ("H", "N"), ("N", "T"), ("C", "QC")):
                P, U, V, W, _ = hm.plan_info(opA, opB, fa, fb, algo=algo)
                if P:
                    worst = max(worst, float(np.abs(4 * W).sum(axis=1).max()))
    assert worst <= 36.0, worst


def test_split_limits():
    with pytest.raises(hm.HmatError):
        hm.split_info(200000, 1e-12)           # beyond the int32 drained accumulators
    with pytest.raises(hm.HmatError):
        hm.split_info(8192, 1e-30)             # beyond the modulus table


def test_tile_table_codes_are_validated():
    import torch
    if torch.cuda.is_available():
        pytest.skip("handle creation is covered on the GPU")
    # host-only: the setter rejects codes outside 0..3 before touching the device
    L = hm.lib()
    assert L.hmat_set_tile_table(None, None) == 7     # no handle
    assert L.hmat_set_complex_form(None, 0) == 7
    assert L.hmat_set_algorithm(None, 0) == 7


def test_plan_info_four_m_is_host_only_and_validated():
    """hmat_plan_info's four-multiplication view needs no device, and the
    form's plan value is not an algorithm the handle accepts (host checks)."""
    P, U, V, W, _ = hm.plan_info("N", "N", bi.BQ, bi.BQ, algo="four_m")
    assert P == 32 and U.shape == (32, 8) and W.shape == (8, 32)
    L = hm.lib()
    n = hm.ctypes.c_int32()
    assert L.hmat_plan_info(4, 0, 0, 0xFF, 0xFF, hm.ctypes.byref(n), None, None, None, None) == 1   # INVALID_VALUE


@pytest.mark.parametrize("fa,fb", list(itertools.product(FLAGS, FLAGS)))
def test_standard_plan_reproduces_structure_tensor(fa, fb):
    """The component-wise (HMAT-standard) plan: same structure tensor, one real product per component pair."""
    for opA, opB in [("N", "N"), ("H", "T")]:
        P, U, V, W, strategy = hm.plan_info(opA, opB, fa, fb, algo="standard")
        assert strategy == 2
        T = structure_tensor(opA, opB)
        got = np.einsum("ep,pc,pd->ecd", W, U.astype(float), V.astype(float))
        mask = np.zeros((8, 8, 8), bool)
        for c in range(8):
            for d in range(8):
                mask[:, c, d] = bool((fa >> c) & 1) and bool((fb >> d) & 1)
        np.testing.assert_array_equal(got[mask], T[mask])
        assert np.all(np.count_nonzero(U, axis=1) == 1) and np.all(np.count_nonzero(V, axis=1) == 1)


def test_standard_counts():
    """Sec. III B: 64 real products for full biquaternions, 16 for real quaternions."""
    assert hm.plan_info("N", "N", bi.BQ, bi.BQ, algo="standard")[0] == 64
    assert hm.plan_info("N", "N", bi.TRS, bi.TRS, algo="standard")[0] == 16
    assert hm.plan_info("N", "N", bi.TRA, bi.TRA, algo="standard")[0] == 16
    assert hm.plan_info("N", "N", bi.REAL, bi.REAL, algo="standard")[0] == 1
    assert hm.plan_info("N", "N", bi.COMPLEX, bi.COMPLEX, algo="standard")[0] == 4


def test_streamed_plan_fits_budget_and_prefers_whole_k():
    """Out-of-core block plan (host-only): fits the budget, keeps kb = k while it can."""
    m = n = k = 4096
    prev = None
    for budget in [1 << 40, 64 << 30, 16 << 30, 4 << 30, 1 << 30]:
        mb, nb, kb, nbytes = hm.streamed_plan(m, n, k, mode="split", tol=1e-12, budget=budget,
                                              on_host=(False, True, True))
        assert nbytes <= budget
        assert mb % 128 == 0 or mb == m
        if prev is not None:
            assert mb * nb * kb <= prev
        prev = mb * nb * kb
    # host-resident operands, split mode: quarter blocks with the B sides cached (each operand block
    # copied and encoded once); FP64 mode: column panels; device-resident operands: one block
    assert hm.streamed_plan(m, n, k, mode="split", tol=1e-12, budget=1 << 40)[:3] == (m // 4, n // 4, k)
    assert hm.streamed_plan(m, n, k, mode="fp64", budget=1 << 40)[:3] == (m, n // 4, k)
    assert hm.streamed_plan(m, n, k, mode="split", tol=1e-12, budget=1 << 40,
                            on_host=(False, False, False))[:3] == (m, n, k)
    assert hm.streamed_plan(m, n, k, mode="fp64", budget=1 << 30)[2] == k     # FP64: only slots, k stays whole
    # device-resident operands need no slots
    full = hm.streamed_plan(m, n, k, mode="fp64", budget=1 << 40, on_host=(True, True, True))[3]
    none = hm.streamed_plan(m, n, k, mode="fp64", budget=1 << 40, on_host=(False, False, False))[3]
    nb = n // 4                                    # column panels: A whole, B and C in quarters
    assert none == 0 and full == 2 * 64 * (m * k + k * nb + m * nb)
    with pytest.raises(hm.HmatError) as ei:
        hm.streamed_plan(m, n, k, mode="split", tol=1e-12, budget=1 << 20)
    assert ei.value.status == 4


def test_streamed_traffic_counts_each_copy():
    """Bytes one streamed product copies (host-only), for each kind of plan."""
    m = n = k = 4096
    X = 64 * m * k                     # one full operand: 8 components of 8 bytes
    # split mode, quarter blocks with the column-block cache of encoded B: A and B once,
    # C out once and in once more when beta != 0
    assert hm.streamed_traffic(m, n, k, mode="split", tol=1e-12, budget=1 << 40) == (2 * X, X)
    assert hm.streamed_traffic(m, n, k, mode="split", tol=1e-12, budget=1 << 40, beta_nonzero=True) == (3 * X, X)
    # FP64 column panels (mb = m): one block row, so A and B once
    assert hm.streamed_traffic(m, n, k, mode="fp64", budget=1 << 40) == (2 * X, X)
    # present components only; device-resident operands are not copied
    assert hm.streamed_traffic(m, n, k, flagsA=bi.TRS, mode="fp64", budget=1 << 40)[0] == X // 2 + X
    assert hm.streamed_traffic(m, n, k, mode="fp64", budget=1 << 40, on_host=(False, False, True)) == (0, X)
    assert hm.streamed_traffic(m, n, k, mode="fp64", budget=1 << 40, on_host=(False, False, False)) == (0, 0)
    # whole k without the cache (small budget): B again for every block row
    mb, nb, kb, _ = hm.streamed_plan(m, n, k, mode="split", tol=1e-12, budget=1 << 30)
    assert kb == k and mb < m
    assert hm.streamed_traffic(m, n, k, mode="split", tol=1e-12, budget=1 << 30) == (X + X * (m // mb), X)
    # k in chunks: A again for every column block as well
    m = n = 1024
    k = 65536
    mb, nb, kb, _ = hm.streamed_plan(m, n, k, mode="split", tol=1e-12, budget=1 << 30)
    assert kb < k
    XA, XB = 64 * m * k, 64 * k * n
    assert hm.streamed_traffic(m, n, k, mode="split", tol=1e-12, budget=1 << 30) == (
        XA * (n // nb) + XB * (m // mb), 64 * m * n)


def test_bench_results_file_resume(tmp_path):
    """bench.py --results: a configuration already in the file is not run again."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = tmp_path / "results.jsonl"
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n", "24", "--steps", "1",
           "--warmup", "0", "--results", str(res)]
    first = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root)
    assert first.returncode == 0, first.stderr
    line1 = json.loads(first.stdout.strip().splitlines()[-1])
    assert len(res.read_text().strip().splitlines()) == 1
    second = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root)
    assert second.returncode == 0, second.stderr
    assert json.loads(second.stdout.strip().splitlines()[-1]) == line1
    assert len(res.read_text().strip().splitlines()) == 1          # not run again
    third = subprocess.run(cmd[:-2] + ["--seed", "7", "--results", str(res)], capture_output=True, text=True,
                           timeout=300, cwd=root)
    assert third.returncode == 0, third.stderr
    assert len(res.read_text().strip().splitlines()) == 2          # another key runs


def _build_c_client(out_dir):
    """Compile tests/c_abi_client.c against include/hmat.h and libhmat.so with the host C compiler."""
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = "/usr/local/cuda"
    libdir = os.path.dirname(hm.library_path())
    exe = os.path.join(str(out_dir), "c_abi_client")
    cmd = [cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-O2", "-I", os.path.join(root, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(root, "tests", "c_abi_client.c"), "-L", libdir,
           "-lhmat", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_client_compiles_against_the_header(tmp_path):
    """The header is valid C11 and a C program links against libhmat.so (run on the GPU in test_gpu_c_abi)."""
    hm.lib()
    assert os.path.exists(_build_c_client(tmp_path))


def test_crt_signed_digit_quotient_is_exact():
    """The CRT kernels' arithmetic, restated on the host: x_l (any integer in
    [-36 * 127, 36 * 127] congruent to 4 X modulo p_l) times the signed 32-bit
    digits of d_l = (P/p_l) ((P/p_l)^-1 4^-1 mod p_l), summed into L 64-bit limb
    sums started at N P (N = nmod * 36 * 127); signed carries; the quotient as
    the float32 round of the leading limbs (from the limb below P's top one)
    times fl(2^(32 pb) / P); X = S - q P.  Every modulus count the library uses,
    both limb counts that can run it, outputs at the margin |X| = P / 2^1.25 and
    the extreme representatives of every x_l give back X exactly."""
    W = 36 * 127
    lists = [hm.split_info(k, tol)[0] for k in (1, 64, 8192, 127 * 1024)
             for tol in (1e-3, 1e-6, 1e-9, 1e-12, 1e-14)]
    longest = max(lists, key=len)
    assert all(lst == longest[:len(lst)] for lst in lists)
    rng = random.Random(11)

    def digits(v, L):
        out, c = [], 0
        for q in range(L):
            w = ((v >> (32 * q)) & 0xFFFFFFFF) + c
            c = 1 if w >= 2 ** 31 else 0
            out.append(w - (c << 32))
        assert c == 0
        return out

    for nm in range(1, len(longest) + 1):
        mods = longest[:nm]
        P = math.prod(mods)
        top = (P.bit_length() - 1) // 32
        pb = max(top - 1, 0)
        for L in ((4, 5) if nm <= 14 else (5,)):
            f = 0.0
            for q in range(L - 1, pb - 1, -1):
                f = f * 2.0 ** 32 + float((P >> (32 * q)) & 0xFFFFFFFF)
            pinv = np.float32(1.0 / f)
            d = [digits((P // p) * (pow((P // p) % p, -1, p) * pow(4, -1, p) % p), L) for p in mods]
            off = nm * W * P
            lim = int(P / 2 ** 1.25)
            for trial in range(300):
                X = rng.choice([lim, -lim, rng.randrange(-lim, lim + 1), rng.randrange(-min(lim, 99), min(lim, 99) + 1)])
                acc = [(off >> (32 * q)) & 0xFFFFFFFF for q in range(L)]
                for p, dl in zip(mods, d):
                    r = (4 * X) % p
                    lo, hi = -W + (r + W) % p, W - (W - r) % p
                    xl = rng.choice([lo, hi, lo + p * rng.randrange(0, (hi - lo) // p + 1)])
                    for q in range(L):
                        acc[q] += xl * dl[q]
                x = [0] * L
                t = acc[0]
                x[0] = t & 0xFFFFFFFF
                for q in range(1, L):
                    t = acc[q] + (t >> 32)
                    x[q] = t & 0xFFFFFFFF
                sf = np.float32(np.float32(t >> 32) * np.float32(2.0 ** 32) + np.float32(x[L - 1]))
                for q in range(L - 2, pb - 1, -1):
                    sf = np.float32(sf * np.float32(2.0 ** 32) + np.float32(x[q]))
                qq = int(np.rint(np.float32(sf * pinv)))
                S = (t << (32 * (L - 1))) + sum(x[q] << (32 * q) for q in range(L - 1))
                assert 0 < S < 2 * nm * W * P
                assert S - qq * P == X, (nm, L, X)
