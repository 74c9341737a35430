"""bench.py's multi-rank host logic on CPU: two gloo ranks (no GPU needed).

Every rank of `bench.py --gpus N` runs an independent replica of the product
(the product does not shard: replicas only); ranks meet at barriers,
the step time is the maximum over ranks and only rank 0 prints.  Here the
helpers are driven by two real processes over gloo on 127.0.0.1.
"""
import io
import json
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    sys.path.insert(0, ROOT)
    import bench
    args = bench.parse(["--gpus", str(world), "--steps", "1", "--warmup", "1", "--impl", "reference", "--n", "24",
                        "--sample-rows", "2", "--no-fp64-compare", "--e2e-steps", "1"])
    r, w, _ = bench.dist_init(args)
    assert (r, w) == (rank, world)
    worst = bench.max_over_ranks(10.0 * (rank + 1), w)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args, r, w)
    bench.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((rank, worst, buf.getvalue()))


def test_two_gloo_ranks_max_time_and_rank0_output():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, worst, text = q.get(timeout=300)
        out[rank] = (worst, text)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 20.0          # max over ranks
    assert out[1][1] == ""                          # only rank 0 prints
    line = json.loads(out[0][1].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
