"""The multi-process path of bench.py on CPU: two gloo ranks set up from the torchrun
environment, max-over-ranks timing, barriers, an independent batch of views per rank
(replicas, no data-path collective) and the reference arm run by rank 0 alone."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup("gloo")
    out = {"world": w, "rank": r, "max": bench.max_over_ranks(1.5 + r, w)}
    bench.barrier(w)
    sc, cams = bench.make_workload("drt8-1.5M", r, n_override=3000)
    out["views"] = [np.asarray(c.viewmat).tolist() for c in cams]
    out["sizes"] = [(c.width, c.height) for c in cams]
    out["scene"] = float(np.asarray(sc.pos_op, np.float64).sum())

    class A:
        workload, splats, steps, warmup, gpus = "drt8-1.5M", 3000, 1, 0, world
    if r != 0:
        out["reference"] = bench.run_reference(A, w, r)  # ranks other than 0 return without work
    bench.barrier(w)
    dist.destroy_process_group()
    q.put(out)


def test_two_gloo_ranks_run_independent_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    outs = sorted((q.get(timeout=300) for _ in procs), key=lambda o: o["rank"])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o["world"] for o in outs] == [2, 2]
    assert all(o["max"] == 2.5 for o in outs)  # max over ranks, seen by every rank
    assert outs[0]["sizes"] == outs[1]["sizes"]  # the same view sizes ...
    assert outs[0]["views"] != outs[1]["views"]  # ... of an independent batch of views per rank
    assert outs[0]["scene"] == outs[1]["scene"]  # every rank holds the same splats
    assert outs[1]["reference"] is None
