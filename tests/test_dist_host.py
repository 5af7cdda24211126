"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2).

The solver path shards by instance with no data-path collective, so what N > 1
adds is host logic: each rank builds its own instances (seeds offset by rank),
the timed region is reduced with MAX over ranks, and the reference arm runs on
rank 0 only.  No GPU is touched.
"""
import contextlib
import io
import os
import socket
import sys
import types

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out = {"rank": rank}
        out["max"] = bench.max_over_ranks(1.5 + 2.0 * rank, world)
        insts = bench.make_inputs(2, 17, 2, rank)
        out["F_sums"] = [float(np.abs(I["F"]).sum()) for I in insts]
        args = types.SimpleNamespace(n=17, k=2, batch=2, rtol=1e-10, precision="fp16", gpus=world, steps=1, warmup=0,
                                     ref_iters=1)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            out["ref_rc"] = bench.run_reference(args)
        out["ref_out"] = buf.getvalue()
        queue.put(out)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    res = [queue.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res = {r["rank"]: r for r in res}
    # MAX over ranks reaches every rank
    assert res[0]["max"] == res[1]["max"] == 3.5
    # instances differ between ranks (seed offset by rank), none repeated
    sums = res[0]["F_sums"] + res[1]["F_sums"]
    assert len(set(sums)) == 4
    # reference arm: rank 0 prints one JSON line, rank 1 exits 0 without output
    assert res[0]["ref_rc"] == 0 and res[1]["ref_rc"] == 0
    assert res[1]["ref_out"] == ""
    import json
    line = json.loads(res[0]["ref_out"].strip())
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["global_batch"] == 4
