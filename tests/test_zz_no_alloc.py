"""cloak_linear_noalloc: the allocation-free cloaked linear.

Some callers cannot allocate device memory while they run: code inside CUDA
stream capture, serving loops whose memory pool owns every byte, real-time
paths that must not synchronise on cudaMalloc. For them the library keeps the
split-K scratch of the BF16 linear in a fixed device array instead of
context-owned buffers. These tests call that entry point through the C ABI
and compare it with cloak_linear on the same inputs, twice in a row (the
scratch array keeps the previous call's contents). The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu

BF16_TOL = 1e-2  # normwise relative error bound of the BF16 path


def _call(cloak, cm, t, x, M, uncloaked=False):
    y = torch.empty((M, cm.model.tensors[t].n), dtype=torch.float32, device="cuda")
    flags = cloak.LINEAR_UNCLOAKED if uncloaked else 0
    cloak.cloak_linear_noalloc(cm.ctx, t, x.data_ptr(), y.data_ptr(), M, cloak.OUT_F32, flags)
    return y


@pytest.mark.parametrize("M", [1, 8, 32])
def test_noalloc_matches_linear_two_calls(cloak_lib, M):
    m = synth.small_decoder(2, synth.DT_BF16, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200,
                            spare_pages=5)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x5151)
    for t in (0, 4, 6):
        xh = synth.activations_host(M, m.tensors[t].k, seed=70 + t)
        x = x_device(m, xh)
        ref = cm.linear(t, x, out_dtype=cloak_lib.OUT_F32)
        y1 = _call(cloak_lib, cm, t, x, M)
        y2 = _call(cloak_lib, cm, t, x, M)
        torch.cuda.synchronize()
        r = ref.cpu().numpy().astype(np.float64)
        for y in (y1, y2):
            assert O.relative_error(y.cpu().numpy(), r) <= BF16_TOL
        # same kernel, same split: identical to cloak_linear
        assert torch.equal(y1, ref) and torch.equal(y2, ref)
        # and within the BF16 bound of the FP64 oracle
        assert O.relative_error(y2.cpu().numpy(), O.cloaked_linear(om, tb, t, arena, xh)) <= BF16_TOL
    # the uncloaked twin through the same entry point: bit for bit cloak_linear's twin run
    xu = x_device(m, synth.activations_host(M, m.tensors[4].k, seed=1))
    yu1 = _call(cloak_lib, cm, 4, xu, M, uncloaked=True)
    yu2 = _call(cloak_lib, cm, 4, xu, M, uncloaked=True)
    refu = cm.linear(4, xu, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
    torch.cuda.synchronize()
    assert torch.equal(yu1, refu) and torch.equal(yu2, refu)
    # and the twin computes what the cloaked layout computes
    assert torch.equal(refu, cm.linear(4, xu, out_dtype=cloak_lib.OUT_F32))
    cm.close()


def _tune_line(cm, t, M, grid, stages=2, chunk=0):
    tt = cm.model.tensors[t]
    bucket = 16 if M <= 16 else 32
    return ('{"chunk": %d, "stages": %d, "grid": %d, "l2pf": -1, "us": 1.000, '
            '"key": "bf16 m%d %dx%d"}\n' % (chunk, stages, grid, bucket, tt.n, tt.k))


@pytest.mark.parametrize("M", [1, 8, 32])
def test_noalloc_follows_the_tuned_launch_shape(cloak_lib, M, tmp_path):
    """After the autotuner (or a loaded tune file) stores a launch shape, both
    entry points use it: the CTA count decides the split-K summation order, so
    a shape honoured by one and not the other would break bit equality. The
    7B-class layer's tensors have thousands of tiles, more than any grid."""
    m = synth.llama7b_layer(1)
    cm = cloak_lib.CloakModel(m, twin=True)
    cm.keygen(0x5152, 0)
    for t in (0, 4, 6):
        cm.shuffle(t, synth.weights_device(m, t, seed=0))
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    for t in (0, 4, 6):
        x = x_device(m, synth.activations_host(M, m.tensors[t].k, seed=80 + t))
        # the tuner's own choice
        cm.autotune([t], [x], out_dtype=cloak_lib.OUT_F32)
        ref = cm.linear(t, x, out_dtype=cloak_lib.OUT_F32)
        y1, y2 = _call(cloak_lib, cm, t, x, M), _call(cloak_lib, cm, t, x, M)
        torch.cuda.synchronize()
        assert torch.equal(y1, ref) and torch.equal(y2, ref)
        # stored shapes that differ from the default: 4 CTAs per SM, half the
        # SMs, a shallow ring, and a token chunk narrower than the batch
        for grid, stages, chunk in ((4 * sm, 2, 0), (sm // 2, 4, 0), (3 * sm, 2, max(1, M // 3))):
            f = tmp_path / f"tune_{t}_{grid}.jsonl"
            f.write_text(_tune_line(cm, t, M, grid, stages, chunk))
            cm.tune_clear()
            assert cm.tune_load(str(f)) == 1
            ref = cm.linear(t, x, out_dtype=cloak_lib.OUT_F32)
            y1, y2 = _call(cloak_lib, cm, t, x, M), _call(cloak_lib, cm, t, x, M)
            yu = _call(cloak_lib, cm, t, x, M, uncloaked=True)
            refu = cm.linear(t, x, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
            torch.cuda.synchronize()
            assert torch.equal(y1, ref) and torch.equal(y2, ref), (t, grid, stages, chunk)
            assert torch.equal(yu, refu) and torch.equal(yu, ref), (t, grid, stages, chunk)
        cm.tune_clear()
    cm.close()


def test_noalloc_rejects_a_stored_shape_beyond_the_scratch(cloak_lib, tmp_path):
    m = synth.llama7b_layer(1)
    cm = cloak_lib.CloakModel(m)
    cm.keygen(3, 0)
    x = torch.zeros((4, m.tensors[4].k), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((4, m.tensors[4].n), dtype=torch.float32, device="cuda")
    f = tmp_path / "wide.jsonl"
    f.write_text(_tune_line(cm, 4, 4, 5000))
    assert cm.tune_load(str(f)) == 1
    with pytest.raises(cloak_lib.CloakError) as e:
        cloak_lib.cloak_linear_noalloc(cm.ctx, 4, x.data_ptr(), y.data_ptr(), 4, cloak_lib.OUT_F32)
    assert e.value.status == cloak_lib.E_UNSUPPORTED and "scratch" in str(e.value)
    cm.tune_clear()
    cloak_lib.cloak_linear_noalloc(cm.ctx, 4, x.data_ptr(), y.data_ptr(), 4, cloak_lib.OUT_F32)
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(y)) == 0
    cm.close()


def test_noalloc_full_size_tensor(cloak_lib):
    """The 11008x4096 gate projection of a 7B-class layer (86 tile rows)."""
    m = synth.llama7b_layer(1)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234, twin=False)
    x = x_device(m, synth.activations_host(4, 4096, seed=9))
    ref = cm.linear(4, x, out_dtype=cloak_lib.OUT_F32)
    for _ in range(2):
        y = _call(cloak_lib, cm, 4, x, 4)
        torch.cuda.synchronize()
        assert O.relative_error(y.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= BF16_TOL
    cm.close()


def test_noalloc_rejects_sizes_beyond_its_limits(cloak_lib):
    m = synth.small_decoder(1, synth.DT_BF16)
    cm = cloak_lib.CloakModel(m)
    cm.keygen(3, 0)
    x = torch.zeros((33, m.tensors[0].k), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((33, m.tensors[0].n), dtype=torch.float32, device="cuda")
    with pytest.raises(cloak_lib.CloakError) as e:
        cloak_lib.cloak_linear_noalloc(cm.ctx, 0, x.data_ptr(), y.data_ptr(), 33, cloak_lib.OUT_F32)
    assert e.value.status == cloak_lib.E_INVAL and "M must be" in str(e.value)
    cm.close()
    f8 = cloak_lib.CloakModel(synth.small_decoder(1, synth.DT_E4M3, page_bytes=2 * 128 * 128))
    f8.keygen(3, 0)
    with pytest.raises(cloak_lib.CloakError) as e:
        cloak_lib.cloak_linear_noalloc(f8.ctx, 0, x.data_ptr(), y.data_ptr(), 4, cloak_lib.OUT_F32)
    assert e.value.status == cloak_lib.E_UNSUPPORTED
    f8.close()
