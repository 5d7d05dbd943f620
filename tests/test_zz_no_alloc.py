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
    yu = _call(cloak_lib, cm, 4, x_device(m, synth.activations_host(M, m.tensors[4].k, seed=1)), M,
               uncloaked=True)
    torch.cuda.synchronize()
    assert torch.isfinite(yu).all()
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
