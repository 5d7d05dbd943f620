"""Launch-shape autotuner of the tensor-core linear: tuned shapes, and
hand-written extreme ones (shallow rings, odd CTA counts, small chunks), keep
every linear within tolerance of the FP64 oracle, the cloaked kernel
bit-identical to the uncloaked one and BF16 outputs the rounded FP32 ones;
tuned shapes persist as JSON lines."""
import json

import numpy as np
import pytest
import torch

from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device
from test_gpu_linear import check_tensor

pytestmark = pytest.mark.gpu


def bucket(M):
    if M > 256:
        return -(-M // 256) * 256
    return next(c for c in (16, 32, 64, 128, 256) if M <= c)


def key(m, t, M):
    tt = m.tensors[t]
    return f"{'e4m3' if m.dtype == synth.DT_E4M3 else 'bf16'} m{bucket(M)} {tt.n}x{tt.k}"


SHAPES = [dict(chunk=0, stages=2, grid=7), dict(chunk=64, stages=3, grid=300),
          dict(chunk=128, stages=2, grid=1), dict(chunk=0, stages=4, grid=152)]


@pytest.mark.parametrize("dtype", [synth.DT_BF16, synth.DT_E4M3])
@pytest.mark.parametrize("shape", range(len(SHAPES)))
def test_hand_written_shapes_keep_parity(cloak_lib, tmp_path, dtype, shape):
    if dtype == synth.DT_BF16:
        m = synth.small_decoder(2, dtype, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200, spare_pages=5)
    else:
        m = synth.small_decoder(2, dtype, page_bytes=2 * 128 * 128, d_model=384, n_heads=6,
                                n_kv_heads=2, d_ff=256)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x77)
    Ms = [1, 17, 100, 300]
    f = tmp_path / "shapes.jsonl"
    with open(f, "w") as fh:
        for M in Ms:
            for t in range(len(m.tensors)):
                fh.write(json.dumps({**SHAPES[shape], "l2pf": -1, "us": 0.0, "key": key(m, t, M)}) + "\n")
    assert cm.tune_load(f) == len(Ms) * len(m.tensors)
    for M in Ms:
        for t in range(len(m.tensors)):
            check_tensor(cloak_lib, cm, om, tb, arena, scales, t, M, seed=M * 13 + t)
    assert cm.device_status() == 0
    cm.close()


def test_autotune_chooses_measures_and_persists(cloak_lib, tmp_path):
    m = synth.small_decoder(2, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=4, d_ff=1024,
                            head_dim=128, spare_pages=5)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x99)
    group = [0, 1, 2]                                  # q, k, v of layer 0
    outs = {}
    for M in (1, 100):
        xs = [x_device(m, synth.activations_host(M, m.tensors[t].k, seed=M + t)) for t in group]
        r = cm.autotune(group, xs, out_dtype=cloak_lib.OUT_F32)
        assert r["candidates"] >= 4 and r["us"] > 0 and r["default_us"] > 0
        assert r["us"] <= r["default_us"] * 1.0001      # never slower than the default it measured
        assert r["stages"] >= 0 and r["grid"] >= 0 and r["chunk"] in (0, 64, 128, 256)
        ys = cm.linear_batch(group, xs, out_dtype=cloak_lib.OUT_F32)
        yu = cm.linear_batch(group, xs, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
        torch.cuda.synchronize()
        for a, b in zip(ys, yu):
            assert torch.equal(a, b)
        outs[M] = (xs, [y.cpu() for y in ys])
        for t in range(len(m.tensors)):                # single-tensor keys are not tuned
            check_tensor(cloak_lib, cm, om, tb, arena, scales, t, M, seed=M * 5 + t)
    f = tmp_path / "tuned.jsonl"
    cm.tune_save(f)
    lines = [json.loads(l) for l in open(f)]
    assert len(lines) == 2 and all(set(l) == {"chunk", "stages", "grid", "l2pf", "us", "key"} for l in lines)
    cm.tune_clear()
    assert cm.tune_load(f) == 2
    for M, (xs, ref) in outs.items():                  # the same shapes again: the same bits
        ys = cm.linear_batch(group, xs, out_dtype=cloak_lib.OUT_F32)
        torch.cuda.synchronize()
        for a, b in zip(ys, ref):
            assert torch.equal(a.cpu(), b)
    bad = tmp_path / "bad.jsonl"
    bad.write_text('{"chunk": 64, "stages": 99, "grid": 1, "l2pf": -1, "us": 0, "key": "bf16 m16 512x512"}\n')
    with pytest.raises(cloak_lib.CloakError):
        cm.tune_load(bad)
    with pytest.raises(cloak_lib.CloakError):
        cm.tune_load(tmp_path / "missing.jsonl")
    cm.close()


@pytest.mark.parametrize("l2pf", [None, 0, 48])
def test_stack_l2_prefetch_depths_keep_parity(cloak_lib, tmp_path, l2pf):
    """The stack kernel's L2 prefetch depth (tuned, none, or more tiles than a
    CTA has) changes no bit of the result; the tuner leaves h untouched."""
    import oracle as O
    m = synth.small_decoder(3, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=320,
                            head_dim=128, spare_pages=3)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x5EED)
    M = 5
    h0 = synth.activations_host(M, m.d_model, seed=2)
    ref_dev = torch.from_numpy(h0).cuda()
    cm.stack_decode(ref_dev)                        # default depth
    torch.cuda.synchronize()
    if l2pf is None:
        h = torch.from_numpy(h0).cuda()
        r = cm.autotune_stack(h)
        torch.cuda.synchronize()
        assert torch.equal(h.cpu(), torch.from_numpy(h0))
        assert r["l2_prefetch"] in (0, 8, 16, 24, 32, 48) and r["us"] > 0
    else:
        f = tmp_path / "stack.jsonl"
        f.write_text(json.dumps({"chunk": 0, "stages": 0, "grid": 0, "l2pf": l2pf, "us": 0.0,
                                 "key": f"stack L3 d512 f320 m{bucket(M)}"}) + "\n")
        assert cm.tune_load(f) == 1
    h = torch.from_numpy(h0).cuda()
    cm.stack_decode(h)
    hu = torch.from_numpy(h0).cuda()
    cm.stack_decode(hu, uncloaked=True)
    torch.cuda.synchronize()
    assert cm.device_status() == 0
    assert torch.equal(h, ref_dev) and torch.equal(h, hu)
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    assert O.relative_error(h.cpu().numpy(), O.stack_decode_f64(m, W64, h0)) <= 1e-2
    cm.close()
