"""Host side of the multi-rank bench on CPU: two gloo ranks (one process each,
rendezvous on 127.0.0.1) go through the bench's rank set-up, barrier and
max-over-ranks reduction, and the reference arm leaves every rank but 0 without
work. The kernels themselves are replicas per GPU (no collective on the data
path), so these host steps are the whole multi-rank logic."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), IETI_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import io
    import contextlib
    import types
    import bench
    w, r, _ = bench.dist_init()
    bench.barrier(w)
    m = bench.allmax(w, 10.0 + r)
    buf = io.StringIO()
    if r != 0:
        with contextlib.redirect_stdout(buf):
            bench.reference(types.SimpleNamespace(steps=1, warmup=1))
    bench.barrier(w)
    torch.distributed.destroy_process_group()
    out.put((r, w, m, buf.getvalue()))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the time of the slowest rank, on every rank; the reference arm prints nothing on rank 1
    assert [(r, w, m) for r, w, m, _ in res] == [(0, 2, 11.0), (1, 2, 11.0)]
    assert res[1][3] == ""
