"""The multi-GPU path of bench.py on CPU: two gloo ranks run the host-side
rank logic (no GPU). Each rank keys its own context (the paper shuffles
independently per GPU), so the two ranks' tables differ and each is a valid
keyed layout; the ranks agree on the slowest rank's time; the reported
whole-job rate counts the work of every rank."""
import multiprocessing as mp
import os
import socket

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    import oracle as O
    from paper_2606_18400_gb300 import synth
    r, w, _ = bench.dist_setup(backend="gloo")
    om = O.OracleModel(synth.small_decoder(1, synth.DT_BF16))
    tb = O.keygen(om, bench.rank_key(r), 0)
    t_max = bench.max_over_ranks(10.0 + 5.0 * r, w)   # per-rank step time (ms)
    bench.barrier(w)
    rate = bench.job_rate(1000.0, t_max, w)
    out.put((r, w, t_max, rate, np.asarray(tb.tile_slot).tolist()))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, rate0, slots0), (r1, w1, t1, rate1, slots1) = res
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert t0 == t1 == 15.0                     # the slowest rank's time, on every rank
    assert rate0 == rate1 == 1000.0 * 2 / 0.015  # both ranks' units over that time
    assert slots0 != slots1                     # independent keys, independent layouts
    for s in (slots0, slots1):
        assert sorted(s) == sorted(set(s))      # each a valid (injective) gather table
