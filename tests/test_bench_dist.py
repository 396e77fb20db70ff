"""The benchmark's multi-process path on the host (gloo, world size 2): the
barrier, the max-over-ranks timing, and the reference arm, which only rank 0
runs (CPU only)."""
import importlib.util
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    b = _load_bench()
    world, r, _ = b.dist_setup()
    b.barrier(world)
    m = b.max_over_ranks(world, 1.5 + r)
    printed = ""
    if r == 1:  # rank 0 would run the full oracle sample: only rank 1's exit is checked
        sys.argv = ["bench.py", "--impl", "reference"]
        buf = io.StringIO()
        with redirect_stdout(buf):
            b.run_reference(b.parse())
        printed = buf.getvalue()
    b.barrier(world)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, world, m, printed))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[:3] for x in res] == [(0, 2, 2.5), (1, 2, 2.5)]
    assert res[1][3] == ""  # rank 1 of the reference arm prints nothing
