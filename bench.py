#!/usr/bin/env python3
"""Cloaked decode throughput of a 7B-class decoder layer on one GB300.

Workload: one LLaMA-7B-shaped decoder layer in BF16 (d_model 4096, 32 heads
of 128, gated MLP 11008; Wq, Wk, Wv, Wo, Wgate, Wup, Wdown = 12,352 tiles of
128x128, 404.75 MB), stored in the keyed, shuffled arena (2 MiB pages), random
N(0, 0.02) weights drawn on the device, N(0, 1) activations. A step is one
decode pass: the seven cloaked linears at batch M, replayed from a CUDA graph.
The metric is algorithmic bytes (weights + gather table + activations in and
out) per second. The uncloaked twin kernel (same code, arithmetic tile
addresses) runs beside it: the cloaking overhead is the ratio.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle (FP64 product on the logical weights,
read back through the tables) on a bounded sample of the same workload.
"""
from __future__ import annotations

import os

# the oracle leg is timed single-threaded (BLAS threads pinned before numpy loads)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cloaked decode GEMV GB/s (7B-class BF16 decoder layer)"
WORKLOAD = ("7B-class decoder layer, BF16, d_model 4096, 32x128 heads, gated MLP 11008, "
            "7 cloaked linears per decode step, 128x128 tiles over 2 MiB keyed pages")
KEY = 0x1234


def step_bytes(model, M):
    """Algorithmic bytes of one decode step: every weight tile once (2 B per
    element), its 4-byte gather-table entry, x in and y out (BF16)."""
    b = 0
    for t in model.tensors:
        nt, kt = model.tiles_of(t)
        b += t.n * t.k * 2 + 4 * nt * kt + M * (t.k + t.n) * 2
    return b


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "100",
                                       "-i", str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        busy = [s for s, p in zip(sm, power) if p > 0.3 * max(power)] if power else sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# ------------------------------------------------------------- distributed

def dist_setup(backend: str = "nccl"):
    """One process per GPU (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* from the
    launcher). The path shards by independent problems: every rank keys and
    runs its own context; the only collectives are the barrier and the max of
    the timings. backend "gloo" runs the same rank logic on CPU."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    if backend == "nccl":
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    else:
        dist.init_process_group(backend)
    return rank, ws, local


def rank_key(rank: int) -> int:
    """Each GPU shuffles its own copy under its own key (the paper shuffles
    independently per GPU)."""
    return KEY + rank


def job_rate(units_per_rank: float, ms_max: float, ws: int) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank does the same work)."""
    return units_per_rank * ws / (ms_max / 1e3)


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------ oracle (CPU)

def _oracle_worker(arena_path, M, seconds, steps, warmup, barrier):
    """One CPU worker of the oracle baseline (its own process, BLAS pinned to
    one thread): the oracle's cloaked linear (stored matrix read back through
    the tables in C, then the FP64 product in NumPy) over the 7B-class
    layer's tensors in turn: `warmup` untimed linears, then `seconds` (or
    `steps` linears) timed. Returns (bytes, seconds, linears timed)."""
    import oracle as O
    from paper_2606_18400_gb300 import synth
    model = synth.llama7b_layer(1)
    om = O.OracleModel(model)
    tb = O.keygen(om, KEY, 0)
    arena = np.load(arena_path, mmap_mode="r")
    xs = [synth.activations_host(M, t.k, seed=1 + i) for i, t in enumerate(model.tensors)]
    for w in range(max(1, warmup)):  # the first also pages the arena in
        O.cloaked_linear(om, tb, w % len(model.tensors), arena, xs[w % len(model.tensors)])
    barrier.wait()
    done_b, n, t0 = 0, 0, time.perf_counter()
    while True:
        i = (warmup + n) % len(model.tensors)
        tt = model.tensors[i]
        O.cloaked_linear(om, tb, i, arena, xs[i])
        done_b += tt.n * tt.k * 2 + 4 * (-(-tt.n // 128)) * (-(-tt.k // 128)) + M * (tt.n + tt.k) * 2
        n += 1
        el = time.perf_counter() - t0
        if (steps and n >= steps) or (not steps and el >= seconds and n >= len(model.tensors)):
            return done_b, el, n


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_cpu(model, M=1, seconds=8.0, steps=0, warmup=0, workers=(1, None)):
    """Time the CPU oracle on the 7B-class layer with 1 worker and with one
    worker per host core (processes started with spawn; each worker pinned to
    one BLAS thread, all reading one shared arena). Returns, per worker count,
    (GB/s of the layer's algorithmic bytes, seconds, linears, workers)."""
    import multiprocessing as mp
    import oracle as O
    from paper_2606_18400_gb300 import synth
    om = O.OracleModel(model)
    tb = O.keygen(om, KEY, 0)
    arena, _ = O.shuffle_model(om, tb, synth.weights_host(model, seed=0))
    out = {}
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "arena.npy")
        np.save(path, arena)
        del arena
        ctx = mp.get_context("spawn")
        for w in workers:
            n = w or host_cores()
            with ctx.Manager() as mgr:
                bar = mgr.Barrier(n)
                with ctx.Pool(n) as pool:
                    res = pool.starmap(_oracle_worker, [(path, M, seconds, steps, warmup, bar)] * n)
            b = sum(r[0] for r in res)
            el = max(r[1] for r in res)
            out[n] = (b / el / 1e9, el, sum(r[2] for r in res), n)
    return out


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on all host cores (one
    worker process per core, each single-threaded). A step is one
    single-tensor cloaked linear per worker, cycling over the layer's 7
    tensors."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2606_18400_gb300 import synth
    import oracle as O
    O.build()
    model = synth.llama7b_layer(1)
    M = args.M
    n = host_cores()
    r = oracle_cpu(model, M=M, steps=args.steps, warmup=args.warmup, workers=(None,))[n]
    value, el, linears, _ = r
    sample = (f"{args.steps} timed single-tensor linears per worker after {args.warmup} untimed, "
              f"{n} workers (one per host core), cycling over the layer's 7 tensors (M={M})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": M},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": n, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- GPU (cloak)

def traffic_record(kernel_src):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p))
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    return rec.get("dram_bytes_per_step") if rec.get("source_sha") == h else None


def tuned_shape(r):
    """The autotuner's choice, as reported in the JSON line."""
    return {"chunk": r["chunk"], "stages": r["stages"], "grid": r["grid"],
            "tuned_us": round(r["us"], 2), "default_us": round(r["default_us"], 2),
            "candidates": r["candidates"]}


def bench_extras(cloak, synth, torch, dev, stream, key, steps, tune=True, serve_rates=(2.0, 8.0, 32.0),
                 serve_seconds=10.0):
    """Other rows of the hot path, each on its own context: BF16 prefill of the
    7B-class layer (M = 512, 2048), the FP8 GQA layer (decode M = 1 and
    prefill M = 2048), and the in-place re-key of the 32-layer 12.95 GB stack."""
    out = {}

    def timed(fn, K, W=3):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(K):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / K

    def graph(fn, n=1):
        fn()
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(n):
                fn()
        return g

    def layer_run(cm, model, M, seed0):
        T = len(model.tensors)
        xs = [torch.from_numpy(synth.activations_host(M, t.k, seed=seed0 + i)).cuda().to(torch.bfloat16)
              for i, t in enumerate(model.tensors)]
        ys = [torch.empty((M, t.n), dtype=torch.bfloat16, device="cuda") for t in model.tensors]
        res = {}
        if tune:
            res["launch_shape"] = tuned_shape(cm.autotune(list(range(T)), xs, ys, out_dtype=cloak.OUT_BF16,
                                                          stream=stream.cuda_stream))
        # 10 consecutive chained steps per graph replay (the prefill GEMM
        # ignores the flag: its launches follow one another)
        for name, flags in (("cloaked", 0), ("uncloaked", cloak.LINEAR_UNCLOAKED)):
            def fn(flags=flags):
                cloak.cloak_linear_batch(cm.ctx, list(range(T)), [x.data_ptr() for x in xs],
                                         [y.data_ptr() for y in ys], M, cloak.OUT_BF16,
                                         flags | cloak.LINEAR_CHAINED, stream.cuda_stream)
            g = graph(fn, 10)
            res[name] = timed(g.replay, max(2, steps // 40)) / 10
            del g
        return res

    # BF16 prefill, 7B-class layer
    model = synth.llama7b_layer(1)
    cm = cloak.CloakModel(model, device=dev, twin=True)
    cm.keygen(key, 0)
    for t in range(len(model.tensors)):
        cm.shuffle(t, synth.weights_device(model, t, seed=0))
    flops1 = 2 * sum(t.n * t.k for t in model.tensors)
    pre = {}
    for M in (512, 2048):
        r = layer_run(cm, model, M, 300)
        pre[str(M)] = {"cloaked_tflops": round(flops1 * M / (r["cloaked"] / 1e3) / 1e12, 1),
                       "uncloaked_tflops": round(flops1 * M / (r["uncloaked"] / 1e3) / 1e12, 1),
                       "cloaked_ms": round(r["cloaked"], 4), "uncloaked_ms": round(r["uncloaked"], 4),
                       "launch_shape": r.get("launch_shape")}
    out["prefill_bf16_llama7b_layer"] = pre
    cm.close()
    torch.cuda.empty_cache()

    out["fp8_peak"] = fp8_peak(torch, dev)

    # FP8 GQA layer (d 3584, 28/4 heads, MLP 18944), E4M3 + FP32 row scales
    model = synth.gqa28_fp8(1)
    cm = cloak.CloakModel(model, device=dev, twin=True)
    cm.keygen(key, 0)
    for t in range(len(model.tensors)):
        cm.shuffle(t, synth.weights_device(model, t, seed=7))
    wbytes = sum(t.n * t.k for t in model.tensors)
    f8 = {}
    r = layer_run(cm, model, 1, 400)
    b1 = wbytes + 4 * cm.G + sum(2 * t.k + 2 * t.n + 4 * t.n for t in model.tensors)  # x, y, row scales
    f8["decode_M1"] = {"cloaked_gbs": round(b1 / (r["cloaked"] / 1e3) / 1e9, 1),
                       "uncloaked_gbs": round(b1 / (r["uncloaked"] / 1e3) / 1e9, 1),
                       "cloaked_us": round(r["cloaked"] * 1e3, 2), "weight_bytes": wbytes,
                       "launch_shape": r.get("launch_shape")}
    r = layer_run(cm, model, 2048, 500)
    f8["prefill_M2048"] = {"cloaked_tflops": round(2 * wbytes * 2048 / (r["cloaked"] / 1e3) / 1e12, 1),
                           "uncloaked_tflops": round(2 * wbytes * 2048 / (r["uncloaked"] / 1e3) / 1e12, 1),
                           "launch_shape": r.get("launch_shape")}
    pk = out["fp8_peak"].get("fp8_tflops")
    if pk:
        f8["prefill_M2048"]["frac_of_measured_fp8_peak"] = round(f8["prefill_M2048"]["cloaked_tflops"] / pk, 4)
    out["fp8_gqa3584_layer"] = f8
    cm.close()
    torch.cuda.empty_cache()

    # the 32-layer BF16 stack (12.95 GB): one persistent launch per decode
    # step (all 224 cloaked linears + glue, grid barriers between dependent
    # stages), replayed from a CUDA graph; then the in-place re-key of it.
    model = synth.llama7b_layer(32)
    cm = cloak.CloakModel(model, device=dev, twin=True)
    t0 = time.perf_counter()
    cm.keygen(key, 0)
    kg_ms = (time.perf_counter() - t0) * 1e3
    for t in range(len(model.tensors)):
        w = synth.weights_device(model, t, seed=0)
        cm.shuffle(t, w)
        del w
    torch.cuda.synchronize()
    desc = cm.stack_desc()
    wbytes = sum(t.n * t.k * 2 for t in model.tensors)
    stk = {}
    for M in (1, 8, 32, 64):
        h0 = torch.from_numpy(synth.activations_host(M, 4096, seed=M)).cuda()
        res = {}
        if tune:
            r = cm.autotune_stack(h0, desc=desc, stream=stream.cuda_stream)
            res["l2_prefetch"] = {"tiles_per_cta": r["l2_prefetch"], "tuned_ms": round(r["us"] / 1e3, 4),
                                  "default_ms": round(r["default_us"] / 1e3, 4)}
        for name, unc in (("cloaked", False), ("uncloaked", True)):
            hb = h0.clone()
            def fn(hb=hb, unc=unc):
                hb.copy_(h0)
                cm.stack_decode(hb, uncloaked=unc, desc=desc, stream=stream.cuda_stream)
            try:
                g2 = graph(fn)
                res[name] = timed(g2.replay, 10)
                del g2
            except Exception as e:  # graph capture refused: time eager launches
                res[name] = timed(fn, 10)
                res["graph_error"] = str(e)[:120]
        bytes_step = wbytes + 4 * cm.G + 32 * 2 * M * (4096 * 4 + 11008 * 2) * 2
        stk[str(M)] = {"cloaked_ms": round(res["cloaked"], 4), "uncloaked_ms": round(res["uncloaked"], 4),
                       "cloaked_gbs": round(bytes_step / (res["cloaked"] / 1e3) / 1e9, 1),
                       "uncloaked_gbs": round(bytes_step / (res["uncloaked"] / 1e3) / 1e9, 1),
                       "tokens_per_s": round(M / (res["cloaked"] / 1e3), 1),
                       "l2_prefetch": res.get("l2_prefetch")}
    assert cm.device_status() == 0
    out["stack_decode_llama7b_32L"] = stk
    ts = []
    for e in range(1, 5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record()
        cm.rekey(key, e)
        b.record()
        torch.cuda.synchronize()
        ts.append((a.elapsed_time(b), (time.perf_counter() - t0) * 1e3))
    moved = cm.NP * model.page_bytes
    med = statistics.median(x[0] for x in ts)
    out["rekey_llama7b_32L"] = {"ms": round(med, 3), "moved_bytes": moved,
                                "gbs_rw": round(2 * moved / (med / 1e3) / 1e9, 1),
                                "host_ms": round(statistics.median(x[1] for x in ts), 3),
                                "keygen_ms": round(kg_ms, 2), "pages": cm.NP, "spare": model.spare_pages,
                                "staging_pages": min(256, max(2, cm.NPS // 32))}
    assert cm.device_status() == 0
    cm.close()
    torch.cuda.empty_cache()
    out["vmm_page_remap"] = bench_vmm(cloak, synth, torch, dev, stream, key, timed, graph, layer_run)
    out["keyed_upload_llama7b_layer"] = bench_upload(cloak, synth, torch, dev, key)
    out["tile_rekey_llama7b_32L"] = bench_tile_rekey(cloak, synth, torch, dev, stream, key)
    out["moe_qwen3_30b_a3b_block"] = bench_moe(cloak, synth, torch, dev, stream, key)
    if serve_rates:
        from paper_2606_18400_gb300 import serve
        sw = serve_sweep(cloak, serve, synth, torch, serve_rates, serve_seconds, serve_seconds, 7000,
                         serve_seconds)
        out["serving_7b_32L_vocab32000"] = {
            "workload": f"Poisson arrivals for {serve_seconds:g} s per rate (+ up to {serve_seconds:g} s "
                        f"drain), prompts lognormal median 1024 clipped [128, 4096], outputs U[64, 1024], "
                        f"KV pool 7000 blocks of 16 tokens, re-key every {serve_seconds:g} s on the "
                        f"cloaked arm (concurrent)",
            "rates": sw}
    return out


def fp8_peak(torch, dev, n=8192, sustain_s=3.0):
    """Dense E4M3 tensor throughput of this GPU as cuBLAS gives it (the FP8
    denominator of the prefill roofline): torch._scaled_mm of two n x n E4M3
    matrices (per-tensor scales 1, BF16 out), 2 n^3 FLOP per call; the best of
    10 timed calls (burst) and the mean over back-to-back calls for
    `sustain_s` seconds (sustained), with the clocks sampled meanwhile."""
    try:
        clk = ClockSampler(dev)
        a = (torch.randn(n, n, device="cuda") * 0.5).to(torch.float8_e4m3fn)
        b = (torch.randn(n, n, device="cuda") * 0.5).to(torch.float8_e4m3fn).t()  # column-major
        one = torch.ones((), device="cuda", dtype=torch.float32)
        mm = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        for _ in range(3):
            mm()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mm()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        calls, e0, e1 = 0, torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < sustain_s:
            for _ in range(20):
                mm()
            calls += 20
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        flop = 2.0 * n ** 3
        res = {"fp8_tflops": round(flop / (best / 1e3) / 1e12, 1),
               "fp8_tflops_sustained": round(flop * calls / (e0.elapsed_time(e1) / 1e3) / 1e12, 1),
               "how": f"torch._scaled_mm E4M3 {n}^3, per-tensor scales, BF16 out: best of 10 calls "
                      f"(burst), {calls} back-to-back calls (sustained)",
               "clocks": clk.stop()}
        del a, b
        torch.cuda.empty_cache()
        return res
    except Exception as e:  # no FP8 GEMM in this torch build
        return {"error": str(e)[:200]}


def bench_moe(cloak, synth, torch, dev, stream, key, steps=64):
    """One MoE FFN block of the Qwen3-30B-A3B shape (128 experts of 768 x
    2048, top-8; 1.2 GB BF16) at decode batch 1 and 4: each step routes
    different tokens (64 seeded inputs in turn) and L2 is evicted (by reading) between
    steps, so the selected experts' tiles come from HBM. Graph-replayed
    steps, timed each with events on the launching stream. L2 is evicted by
    reading a 256 MB buffer between steps."""
    model = synth.moe_block()
    cm = cloak.CloakModel(model, device=dev, twin=True)
    cm.keygen(key, 0)
    for t in range(len(model.tensors)):
        cm.shuffle(t, synth.weights_device(model, t, seed=3))
    D, E, F, K = model.d_model, model.n_experts, model.d_ff, model.top_k
    desc = cm.moe_desc()
    flush = torch.ones(64 << 20, dtype=torch.int32, device="cuda")  # 256 MB
    flush_sink = torch.zeros((), dtype=torch.int32, device="cuda")
    res = {"experts": E, "top_k": K, "d_model": D, "d_ff": F}
    for M in (1, 4):
        xs = [torch.from_numpy(synth.activations_host(M, D, seed=900 + i)).cuda().to(torch.bfloat16)
              for i in range(steps)]
        xb = xs[0].clone()
        row = {}
        for name, unc in (("cloaked", False), ("uncloaked", True)):
            with torch.cuda.stream(stream):
                cm.moe_ffn(xb, desc=desc, uncloaked=unc, stream=stream.cuda_stream)  # uploads the table
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                yb = cm.moe_ffn(xb, desc=desc, uncloaked=unc, stream=stream.cuda_stream)
            ts = []
            with torch.cuda.stream(stream):
                for i in range(steps):
                    xb.copy_(xs[i])
                    # evict L2 by reading (a written flush leaves dirty lines
                    # whose write-back would land inside the timed step)
                    flush_sink.copy_(flush.max())
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    g.replay()
                    b.record(stream)
                    ts.append((a, b))
            torch.cuda.synchronize()
            us = statistics.median(a.elapsed_time(b) for a, b in ts[3:]) * 1e3
            del g
            row[name + "_us"] = round(us, 2)
        # algorithmic bytes: router, the selected experts (distinct per token),
        # their gather-table entries, x and y
        wb = E * D * 2 + M * K * 3 * F * D * 2
        tiles = (E // 128 or 1) * (D // 128) + M * K * 3 * (F // 128) * (D // 128)
        byts = wb + 4 * tiles + M * D * 2 + M * D * 4
        row["bytes_per_step"] = byts
        row["cloaked_gbs"] = round(byts / (row["cloaked_us"] / 1e6) / 1e9, 1)
        row["uncloaked_gbs"] = round(byts / (row["uncloaked_us"] / 1e6) / 1e9, 1)
        res[f"decode_M{M}"] = row
    assert cm.device_status() == 0
    cm.close()
    del flush
    torch.cuda.empty_cache()
    return res


def bench_tile_rekey(cloak, synth, torch, dev, stream, key):
    """Tile-level re-key of the 32-layer stack: a new tile permutation and
    page map, every 32 KiB tile moved to its new slot in place."""
    model = synth.llama7b_layer(32)
    model.tile_rekey = True
    cm = cloak.CloakModel(model, device=dev)
    cm.keygen(key, 0)
    for t in range(len(model.tensors)):
        w = synth.weights_device(model, t, seed=0)
        cm.shuffle(t, w)
        del w
    torch.cuda.synchronize()
    ts = []
    for e in range(1, 4):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        a.record(stream)
        cm.rekey(key, e, stream=stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        ts.append((a.elapsed_time(b), (time.perf_counter() - t0) * 1e3))
    moved = cm.G * cm.tile_bytes
    med = statistics.median(x[0] for x in ts)
    res = {"ms": round(med, 3), "host_ms": round(statistics.median(x[1] for x in ts), 3),
           "moved_bytes": moved, "gbs_rw": round(2 * moved / (med / 1e3) / 1e9, 1), "tiles": cm.G}
    assert cm.device_status() == 0
    cm.close()
    torch.cuda.empty_cache()
    return res


def bench_upload(cloak, synth, torch, dev, key):
    """Placing the 7B-class layer from host FP32 weights: the keyed upload
    (pages assembled on the host, sent whole in physical order) against the
    logical-order path (FP32 matrices copied to the device, then shuffled
    there). Rates count the arena bytes placed."""
    import numpy as np
    model = synth.llama7b_layer(1)
    Ws = synth.weights_host(model, seed=0)
    placed = sum(t.n * t.k * 2 for t in model.tensors)
    res = {"placed_bytes": placed, "host_threads": min(16, os.cpu_count() or 1)}
    cm = cloak.CloakModel(model, device=dev)
    cm.keygen(key, 0)
    cm.upload(Ws)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        cm.upload(Ws)
        ts.append(time.perf_counter() - t0)
    res["keyed_upload_s"] = round(min(ts), 4)
    res["keyed_upload_gbs"] = round(placed / min(ts) / 1e9, 2)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        for t, W in enumerate(Ws):
            w = torch.from_numpy(np.ascontiguousarray(W)).cuda(dev)
            cm.shuffle(t, w)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    res["logical_copy_and_shuffle_s"] = round(min(ts), 4)
    res["logical_copy_and_shuffle_gbs"] = round(placed / min(ts) / 1e9, 2)
    cm.close()
    torch.cuda.empty_cache()
    return res


def bench_vmm(cloak, synth, torch, dev, stream, key, timed, graph, layer_run):
    """Section 4.2's physical page remapping through CUDA VMM: the arena's
    2 MiB pages are separate physical chunks; the kernels read either the
    arena (the gather table does the page step) or the virtual view (the
    MMU does it). The same launches on both, and re-key + remap cost."""
    res = {}
    model = synth.llama7b_layer(1)
    T, M = len(model.tensors), 1
    xs = [torch.from_numpy(synth.activations_host(M, t.k, seed=600 + i)).cuda().to(torch.bfloat16)
          for i, t in enumerate(model.tensors)]
    ys = [torch.empty((M, t.n), dtype=torch.bfloat16, device="cuda") for t in model.tensors]
    b1 = step_bytes(model, M)
    lay = {}
    # the same launches, tuned alike, on one cudaMalloc block (malloc) and on
    # per-page chunks read through the arena (arena) or the view (view)
    for vmm, runs in ((False, (("malloc", 0),)), (True, (("arena", 0), ("view", cloak.LINEAR_VMM)))):
        cm = cloak.CloakModel(model, device=dev, vmm=vmm)
        cm.keygen(key, 0)
        for t in range(T):
            cm.shuffle(t, synth.weights_device(model, t, seed=0))
        cm.autotune(list(range(T)), xs, ys, out_dtype=cloak.OUT_BF16, stream=stream.cuda_stream)
        for name, flags in runs:
            def fn(flags=flags):
                cloak.cloak_linear_batch(cm.ctx, list(range(T)), [x.data_ptr() for x in xs],
                                         [y.data_ptr() for y in ys], M, cloak.OUT_BF16, flags,
                                         stream.cuda_stream)
            g = graph(fn)
            ms = timed(g.replay, 400)
            del g
            lay[name + "_us"] = round(ms * 1e3, 2)
            lay[name + "_gbs"] = round(b1 / (ms / 1e3) / 1e9, 1)
        cm.close()
        torch.cuda.empty_cache()
    res["decode_llama7b_layer_M1"] = lay

    model = synth.llama7b_layer(32)
    cm = cloak.CloakModel(model, device=dev, vmm=True)
    cm.keygen(key, 0)
    res["keygen_remap_ms"] = round(cm.vmm_stats()["remap_us"] / 1e3, 2)
    for t in range(len(model.tensors)):
        w = synth.weights_device(model, t, seed=0)
        cm.shuffle(t, w)
        del w
    torch.cuda.synchronize()
    desc = cm.stack_desc()
    stk = {}
    for M in (1, 8):
        h0 = torch.from_numpy(synth.activations_host(M, 4096, seed=M)).cuda()
        row = {}
        for name, vmm in (("arena", False), ("view", True)):
            hb = h0.clone()
            def fn(hb=hb, vmm=vmm):
                hb.copy_(h0)
                cm.stack_decode(hb, desc=desc, stream=stream.cuda_stream, vmm=vmm)
            g2 = graph(fn)
            row[name + "_ms"] = round(timed(g2.replay, 10), 4)
            del g2
        stk[str(M)] = row
    res["stack_decode_llama7b_32L"] = stk
    ts = []
    for e in range(1, 4):
        t0 = time.perf_counter()
        cm.rekey(key, e)
        torch.cuda.synchronize()
        st = cm.vmm_stats()
        ts.append(((time.perf_counter() - t0) * 1e3, st["remap_us"] / 1e3, st["pages_remapped"]))
    res["rekey_llama7b_32L"] = {"rekey_and_remap_ms": round(statistics.median(x[0] for x in ts), 2),
                                "remap_ms": round(statistics.median(x[1] for x in ts), 2),
                                "pages_remapped": int(statistics.median(x[2] for x in ts)),
                                "pages": cm.NP, "chunks": cm.vmm_stats()["chunks"]}
    assert cm.device_status() == 0
    cm.close()
    torch.cuda.empty_cache()
    return res


def run_cloak(args):
    import torch
    from paper_2606_18400_gb300 import cloak, synth

    rank, ws, local = dist_setup()
    dev = local
    torch.cuda.set_device(dev)
    cloak.load()
    model = synth.llama7b_layer(1)
    T = len(model.tensors)
    # all work runs on one non-default stream (CUDA graphs capture on it)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    cm = cloak.CloakModel(model, device=dev, twin=True)

    t0 = time.perf_counter()
    cm.keygen(rank_key(rank), 0)
    keygen_ms = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    shuffle_ms = 0.0
    for t in range(T):
        w = synth.weights_device(model, t, seed=0)
        ev0.record()
        cm.shuffle(t, w)
        ev1.record()
        torch.cuda.synchronize()
        shuffle_ms += ev0.elapsed_time(ev1)
        del w
    shuffle_gbs = sum(t.n * t.k * (4 + 2 * 2) for t in model.tensors) / (shuffle_ms / 1e3) / 1e9

    def make_io(M):
        xs = [torch.from_numpy(synth.activations_host(M, t.k, seed=1 + i)).cuda().to(torch.bfloat16)
              for i, t in enumerate(model.tensors)]
        ys = [torch.empty((M, t.n), dtype=torch.bfloat16, device="cuda") for t in model.tensors]
        return xs, ys

    tensors = list(range(T))

    def step_fn(xs, ys, M, unc, chained=False):
        # one launch: the seven linears' tiles split evenly over the SMs
        flags = (cloak.LINEAR_UNCLOAKED if unc else 0) | (cloak.LINEAR_CHAINED if chained else 0)
        cloak.cloak_linear_batch(cm.ctx, tensors, [x.data_ptr() for x in xs],
                                 [y.data_ptr() for y in ys], M, cloak.OUT_BF16, flags,
                                 stream.cuda_stream)

    def graph_of(xs, ys, M, unc, n=1, chained=False):
        for _ in range(2):
            step_fn(xs, ys, M, unc, chained)  # allocate workspaces outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        n0 = cm.launches()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(n):
                step_fn(xs, ys, M, unc, chained)
        return g, (cm.launches() - n0) // n

    def time_chain(xs, ys, M, unc, K, W):
        """K consecutive steps as chained launches (each launch streams its
        weights while the previous one finishes and reads x after it has
        completed), captured in one graph and replayed once after a W-step
        warm-up graph: the timed region is exactly K steps."""
        gw, _ = graph_of(xs, ys, M, unc, W, True)
        gk, lps = graph_of(xs, ys, M, unc, K, True)
        gw.replay()
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        gk.replay()
        b.record()
        torch.cuda.synchronize()
        barrier(ws)
        del gw, gk
        return max_over_ranks(a.elapsed_time(b) / K, ws), lps

    def time_graph(g, K, W):
        for _ in range(W):
            g.replay()
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(K):
            g.replay()
        b.record()
        torch.cuda.synchronize()
        barrier(ws)
        return max_over_ranks(a.elapsed_time(b) / K, ws)

    clocks = ClockSampler(dev)
    M = args.M
    xs, ys = make_io(M)
    shape = None
    if not args.no_tune:  # launch shape from the autotuner (measured here, on this GPU)
        shape = tuned_shape(cm.autotune(list(range(T)), xs, ys, out_dtype=cloak.OUT_BF16,
                                        stream=stream.cuda_stream))
    ms, launches_per_step = time_chain(xs, ys, M, False, args.steps, args.warmup)
    ms_un, _ = time_chain(xs, ys, M, True, args.steps, args.warmup)
    # the same steps unchained: one graph replay per step, each launch
    # starting after the previous one has completed
    g_cl, _ = graph_of(xs, ys, M, False)
    ms_plain = time_graph(g_cl, args.steps, args.warmup)
    del g_cl
    B = step_bytes(model, M)
    value = job_rate(B, ms, ws) / 1e9

    # kernel duration for the roofline: a GPU-side sleep lets the host queue
    # every launch and event first, so the launches run back to back
    reps = 50
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(reps)]
    torch.cuda.synchronize()
    torch.cuda._sleep(50_000_000)
    for r in range(reps):
        evs[r][0].record()
        step_fn(xs, ys, M, False)
        evs[r][1].record()
    torch.cuda.synchronize()
    kern_ms = statistics.median(a.elapsed_time(b) for a, b in evs)
    # per-tensor launches (one kernel per linear) for comparison
    evt = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(T)] for _ in range(20)]
    torch.cuda._sleep(50_000_000)
    for r in range(20):
        for t in range(T):
            evt[r][t][0].record()
            cloak.cloak_linear(cm.ctx, t, xs[t].data_ptr(), ys[t].data_ptr(), M, cloak.OUT_BF16, 0,
                               stream.cuda_stream)
            evt[r][t][1].record()
    torch.cuda.synchronize()
    per_tensor_us = [statistics.median(evt[r][t][0].elapsed_time(evt[r][t][1]) for r in range(20)) * 1e3
                     for t in range(T)]
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    hbm = peaks.get("hbm_gbs")
    peak_note = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    # a step of the timed region is one launch of the grouped kernel (graph
    # replay): its average duration there is the kernel's launch duration over
    # the timed region; the per-launch event brackets are kept beside it
    achieved = B / (ms / 1e3) / 1e9

    # batch sweep (cloaked / uncloaked), same method
    sweep = {}
    for Ms in (1, 8, 32, 64):
        xs2, ys2 = make_io(Ms)
        sh = None
        if not args.no_tune:
            sh = tuned_shape(cm.autotune(list(range(T)), xs2, ys2, out_dtype=cloak.OUT_BF16,
                                         stream=stream.cuda_stream))
        mc, _ = time_chain(xs2, ys2, Ms, False, max(20, args.steps), 3)
        mu, _ = time_chain(xs2, ys2, Ms, True, max(20, args.steps), 3)
        Bs = step_bytes(model, Ms)
        sweep[str(Ms)] = {"cloaked_gbs": round(Bs / (mc / 1e3) / 1e9, 1),
                          "uncloaked_gbs": round(Bs / (mu / 1e3) / 1e9, 1),
                          "cloaked_us": round(mc * 1e3, 2), "uncloaked_us": round(mu * 1e3, 2),
                          "launch_shape": sh}
        del xs2, ys2

    # end to end through the C ABI with host buffers (copies inside the timing):
    # the step's seven input vectors packed in one pinned buffer, its seven
    # outputs in another, one cloak_linear_batch_host call per step
    xpk = torch.cat([x.cpu().reshape(-1) for x in xs]).pin_memory()
    ypk = torch.empty(sum(M * t.n for t in model.tensors), dtype=torch.bfloat16).pin_memory()
    xh_ptr, yh_ptr, o, q = [], [], 0, 0
    for x, t in zip(xs, model.tensors):
        xh_ptr.append(xpk[o:].data_ptr())
        o += x.numel()
        yh_ptr.append(ypk[q:].data_ptr())
        q += M * t.n
    def e2e_step():
        cloak.cloak_linear_batch_host(cm.ctx, list(range(T)), xh_ptr, yh_ptr, M, cloak.OUT_BF16, 0,
                                      stream.cuda_stream)
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    ke = max(args.steps, 20)
    for _ in range(ke):
        e2e_step()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) / ke * 1e3, ws)
    h2d = sum(M * t.k * 2 for t in model.tensors)
    d2h = sum(M * t.n * 2 for t in model.tensors)

    # re-key of the placed layer (in place, all 193 pages)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rk = []
    for e in range(1, 4):
        a.record()
        cm.rekey(rank_key(rank), e)
        b.record()
        torch.cuda.synchronize()
        rk.append(a.elapsed_time(b))
    rekey_ms = statistics.median(rk)
    moved = cm.NP * model.page_bytes
    status = cm.device_status()
    cm.close()
    extras = None if args.no_extras else bench_extras(
        cloak, synth, torch, dev, stream, rank_key(rank), args.steps, tune=not args.no_tune,
        serve_rates=[float(r) for r in args.bench_serve_rates.split(",")] if args.bench_serve_rates else (),
        serve_seconds=args.bench_serve_seconds)
    clk = clocks.stop()

    if rank == 0:
        cpu = None
        if args.gpus == 1 and not args.no_cpu_baseline:
            r = oracle_cpu(model, M=M, seconds=args.cpu_seconds / 2)
            one = r[1]
            nc = max(r)
            allc = r[nc]
            cpu = {"value": allc[0], "unit": "GB/s", "cores": nc, "kind": "oracle",
                   "sample": f"{allc[2]} single-tensor oracle linears (M={M}) by {nc} worker processes "
                             f"(one per host core, one BLAS thread each) over {allc[1]:.1f} s, cycling "
                             f"over the layer's 7 tensors",
                   "host_cores": host_cores(),
                   "single_thread": {"value": one[0], "unit": "GB/s", "cores": 1,
                                     "sample": f"{one[2]} linears by one worker over {one[1]:.1f} s"}}
        traffic = traffic_record(os.path.join(ROOT, "paper_2606_18400_gb300", "csrc", "linear.cu"))
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "batch": M, "weight_bytes": sum(t.n * t.k * 2 for t in model.tensors),
                       "bytes_per_step": B, "tiles": cm.G, "pages": cm.NP, "spare_pages": model.spare_pages,
                       "launch": "one grouped launch (7 linears) per step; the K timed steps are K "
                                 "consecutive chained launches (CLOAK_LINEAR_CHAINED) in one CUDA graph: "
                                 "each launch streams its weight tiles while the previous one finishes "
                                 "and reads x after it has completed",
                       "launch_shape": shape,
                       "l2": "inputs larger than L2: 404.75 MB of weights per step vs 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(achieved / hbm, 4),
                         "traffic": traffic, "peak_source": peak_note,
                         "peak_kind": "copy bandwidth (read + write) measured on this GPU; the step is a "
                                      "read stream (2.4 MB written per 405 MB read)",
                         "kernel": "k_linear_tc<bf16, N=16>: one launch, 7 linears, swap-AB tcgen05, stream-K",
                         "kernel_us": round(ms * 1e3, 2),
                         "kernel_us_source": "CUDA events around the timed region (one replay of a graph "
                                             "of K chained launches, one per step), divided by the steps",
                         "kernel_us_unchained": round(ms_plain * 1e3, 2),
                         "kernel_us_unchained_source": "one graph replay per step (each launch starts "
                                                       "after the previous one completed)",
                         "kernel_us_bracketed": round(kern_ms * 1e3, 2)},
            "cpu_baseline": cpu,
            "e2e": {"value": round(job_rate(B, e2e_ms, ws) / 1e9, 2), "unit": "GB/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_ms, "api": "cloak_linear_batch_host (7 linears; inputs and outputs packed in pinned host buffers)"},
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "uncloaked": {"value": round(job_rate(B, ms_un, ws) / 1e9, 1), "ms_per_step": ms_un,
                          "overhead_pct": round((ms / ms_un - 1) * 100, 2)},
            "sweep_batch": sweep,
            "separate_launches_us": [round(v, 2) for v in per_tensor_us],
            "rekey": {"ms": round(rekey_ms, 3), "moved_bytes": moved,
                      "gbs_rw": round(2 * moved / (rekey_ms / 1e3) / 1e9, 1)},
            "keygen_ms": round(keygen_ms, 2), "shuffle_gbs": round(shuffle_gbs, 1),
            "device_status": status,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serve_sweep(cloak, serve, synth, torch, rates, seconds, drain, kv_blocks, rekey_period,
                rekey_between=False):
    """Serving workload on the 32-layer cloaked BF16 model with a 32,000-token
    lm_head: Poisson arrivals for `seconds` at each rate, lognormal prompts
    clipped to [128, 4096], outputs uniform in [64, 1024], continuous batching
    admitted by free KV blocks (up to `drain` more seconds to finish), a
    re-key every `rekey_period` s on the cloaked arm (concurrent: copies on a
    side stream, tables published between steps); cloaked and uncloaked arms
    on the same arrivals. Throughput counts every sampled token over the wall
    time; latencies are those of the requests that got their tokens."""
    model = synth.serving_model(32, 32000)
    sm = serve.ServedModel(model, kv_blocks=kv_blocks, max_blocks=(4096 + 1024) // 16 + 1, twin=True)
    results = {}
    for rate in rates:
        work = synth.requests_poisson(rate, seconds, 32000, seed=int(rate * 10))
        offered = sum(w[2] for w in work) / seconds
        row = {"requests_arrived": len(work), "offered_tokens_per_s": round(offered, 1)}
        for name, unc in (("cloaked", False), ("uncloaked", True)):
            # the plain model has nothing to re-key
            srv = serve.Server(sm, max_running=64, token_budget=2048, uncloaked=unc,
                               rekey_period=None if unc else rekey_period,
                               rekey_concurrent=not rekey_between)
            done, wall = srv.run(work, max_wall=seconds + drain)
            st = serve.latency_stats(done, wall)
            st["tokens_per_s"] = srv.tokens_out / wall
            st["tokens"] = srv.tokens_out
            st["steps"] = srv.steps
            st["mean_step_tokens"] = float(np.mean(srv.step_tokens)) if srv.step_tokens else 0.0
            st["rekeys"] = [{k: (round(v, 3) if isinstance(v, float) else v) for k, v in r.items()}
                            for r in srv.rekeys]
            row[name] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}
        c, u = row["cloaked"], row["uncloaked"]
        row["cloaked_vs_uncloaked_tokens_pct"] = round((c["tokens_per_s"] / u["tokens_per_s"] - 1) * 100, 2)
        # saturated: requests were still queued or running when the window
        # closed, or waited seconds for their first token
        row["saturated"] = bool(u["requests"] < len(work) or (u["ttft_p99_s"] or 0.0) > 1.0)
        results[str(rate)] = row
    assert sm.cm.device_status() == 0
    sm.close()
    torch.cuda.empty_cache()
    return results


def run_serve(args):
    """The serving sweep alone (one JSON line)."""
    import torch
    from paper_2606_18400_gb300 import cloak, serve, synth
    cloak.load()
    torch.cuda.set_device(0)
    rates = [float(r) for r in args.rates.split(",")]
    clocks = ClockSampler(0)
    results = serve_sweep(cloak, serve, synth, torch, rates, args.serve_seconds, args.drain_seconds,
                          args.kv_blocks, args.rekey_period, args.rekey_between_steps)
    clk = clocks.stop()
    tps = {r: results[r]["cloaked"]["tokens_per_s"] for r in results}
    line = {"metric": "serving tokens/s (cloaked 7B-class BF16 model, continuous batching)",
            "value": max(tps.values()), "unit": "tokens/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"Poisson {args.rates} req/s for {args.serve_seconds} s each (+ up to "
                                   f"{args.drain_seconds} s drain), prompts lognormal median 1024 clipped "
                                   f"[128, 4096], outputs U[64, 1024], 32 layers + vocab 32000, "
                                   f"KV pool {args.kv_blocks} blocks of 16 tokens, re-key every "
                                   f"{args.rekey_period:g} s "
                                   f"({'between steps' if args.rekey_between_steps else 'concurrent, side stream'})"
                                   f" on the cloaked arm"},
            "sweep": results, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Small cases of one kernel each, for ncu captures (a few GB at most):
    stack  -- a 4-layer 7B-class stack (1.6 GB), decode of --M tokens (default 1), 3 launches;
    fp8    -- one GQA E4M3 layer (233 MB), grouped decode M=1, 3 launches;
    fp8prefill -- the same layer, grouped prefill M=2048 (the prefill GEMM), 3 launches;
    prefill-- one 7B-class layer, grouped M=2048 (the prefill GEMM), 3 launches;
    decode -- one 7B-class layer, grouped M=1 (the headline step), 3 launches;
    moe    -- one MoE block of the Qwen3-30B-A3B shape (1.2 GB), decode M=1,
              3 steps (4 kernels each), a different token per step;
    serve  -- the 32-layer served model (13.4 GB) with --M requests of 1,000-token
              prompts prefilled, then one decode-only step (all kernels of the step;
              for launch lists: the KV cache makes it up to 35 GB at --M 64).
    serveprefill -- the same model, one step that prefills a prompt of --M tokens
              (one request; prefill GEMM, query-tiled attention).
    The linears' launch shape is tuned first (unless --no-tune); the profiled
    launches sit inside the NVTX range "profiled" (ncu --nvtx
    --nvtx-include "profiled/")."""
    import torch
    from paper_2606_18400_gb300 import cloak, synth
    cloak.load()
    torch.cuda.set_device(0)
    if args.profile == "serveprefill":
        from paper_2606_18400_gb300 import serve
        P = args.M
        sm = serve.ServedModel(synth.serving_model(32, 32000), kv_blocks=(P + 15) // 16 * 2 + 8,
                               max_blocks=(P + 15) // 16 + 2, twin=False)
        srv = serve.Server(sm, max_running=64, token_budget=max(2048, P), rekey_period=None)
        rng = np.random.default_rng(P)
        for rep in range(2):  # the first step warms up; the second is profiled
            r = serve.Request(rep, 0.0, rng.integers(0, 32000, P).astype(np.int32), 4)
            assert srv._admit(r, 0.0)
            torch.cuda.synchronize()
            if rep:
                torch.cuda.nvtx.range_push("profiled")
            srv.step_batch([r])
            torch.cuda.synchronize()
            if rep:
                torch.cuda.nvtx.range_pop()
            srv._release(r)
        assert sm.cm.device_status() == 0
        sm.close()
        print(json.dumps({"profile": args.profile, "prompt": P, "ok": True}))
        return
    if args.profile == "serve":
        from paper_2606_18400_gb300 import serve
        B = args.M
        sm = serve.ServedModel(synth.serving_model(32, 32000), kv_blocks=B * 66 + 8, max_blocks=66,
                               twin=False)
        srv = serve.Server(sm, max_running=64, token_budget=2048, rekey_period=None)
        rng = np.random.default_rng(B)
        reqs = [serve.Request(i, 0.0, rng.integers(0, 32000, 1000).astype(np.int32), 40) for i in range(B)]
        for r in reqs:
            assert srv._admit(r, 0.0)
        while any(r.prefilled < len(r.prompt) for r in reqs):
            owners, toks = srv.step_batch(reqs)
            for r, t in zip(owners, toks):
                r.out.append(int(t))
        for _ in range(3):  # decode steps before the profiled one
            owners, toks = srv.step_batch(reqs)
            for r, t in zip(owners, toks):
                r.out.append(int(t))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        srv.step_batch(reqs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        assert sm.cm.device_status() == 0
        sm.close()
        print(json.dumps({"profile": args.profile, "batch": B, "ok": True}))
        return
    if args.profile == "stack":
        model = synth.llama7b_layer(4)
    elif args.profile == "moe":
        model = synth.moe_block()
    elif args.profile in ("fp8", "fp8prefill"):
        model = synth.gqa28_fp8(1)
    else:
        model = synth.llama7b_layer(1)
    cm = cloak.CloakModel(model)
    cm.keygen(KEY, 0)
    for t in range(len(model.tensors)):
        cm.shuffle(t, synth.weights_device(model, t, seed=0))
    torch.cuda.synchronize()
    if args.profile == "moe":
        xs = [torch.from_numpy(synth.activations_host(1, model.d_model, seed=900 + i)).cuda().to(torch.bfloat16)
              for i in range(4)]
        desc = cm.moe_desc()
        cm.moe_ffn(xs[3], desc=desc)  # uploads the expert table
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        for i in range(3):
            cm.moe_ffn(xs[i], desc=desc)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    elif args.profile == "stack":
        h0 = torch.from_numpy(synth.activations_host(args.M, 4096, seed=1)).cuda()
        torch.cuda.nvtx.range_push("profiled")
        for _ in range(3):
            cm.stack_decode(h0.clone())
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    else:
        M = 2048 if args.profile in ("prefill", "fp8prefill") else 1
        xs = [torch.from_numpy(synth.activations_host(M, t.k, seed=i)).cuda().to(torch.bfloat16)
              for i, t in enumerate(model.tensors)]
        group = list(range(len(model.tensors)))
        shape = None if args.no_tune else cm.autotune(group, xs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled")
        for _ in range(3):
            cm.linear_batch(group, xs, chained=True)  # as the timed steps launch it
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"launch_shape": shape}))
    torch.cuda.synchronize()
    assert cm.device_status() == 0
    cm.close()
    print(json.dumps({"profile": args.profile, "ok": True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["cloak", "reference"], default="cloak")
    ap.add_argument("--M", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--serve", action="store_true", help="run the serving sweep instead")
    ap.add_argument("--profile", choices=["stack", "fp8", "fp8prefill", "prefill", "decode", "moe", "serve", "serveprefill"],
                    help="small case for ncu")
    ap.add_argument("--rates", default="2,8,32")
    ap.add_argument("--bench-serve-rates", default="2,8,32",
                    help="arrival rates of the serving sweep in the extras ('' to skip)")
    ap.add_argument("--bench-serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-seconds", type=float, default=30.0)
    ap.add_argument("--drain-seconds", type=float, default=30.0)
    ap.add_argument("--kv-blocks", type=int, default=7000)
    ap.add_argument("--rekey-period", type=float, default=30.0)
    ap.add_argument("--no-tune", action="store_true",
                    help="default launch shapes (skip the autotuner)")
    ap.add_argument("--rekey-between-steps", action="store_true",
                    help="serving: re-key between two steps instead of concurrently")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.profile:
        run_profile(args)
    elif args.serve:
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_cloak(args)


if __name__ == "__main__":
    main()
