"""Physical page remapping through CUDA virtual memory management (Section
4.2; Table 1b). A CLOAK_MODEL_VMM context backs every arena page with its own
physical chunk; the virtual view maps virtual page vp to chunk
page_alloc[vp]. Checked against the oracle: the physical view equals the
oracle's arena, the virtual view equals the oracle's pages taken in virtual
order (at every epoch, behind one unchanged pointer), and every kernel run on
the view gives the arena read's result bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu

MiB2 = 2 << 20


def vmm_model(dtype=synth.DT_BF16, layers=2):
    """Several 2 MiB pages (64 BF16 or 128 E4M3 tiles each) with ragged tile
    rows; a tensor's tiles straddle pages."""
    return synth.small_decoder(layers, dtype, d_model=1024, n_heads=8, n_kv_heads=2, d_ff=1424,
                               head_dim=128, spare_pages=4, page_bytes=MiB2)


def virtual_order(arena, tb, om):
    """The oracle's pages in virtual order: what the virtual view must hold."""
    P = om.model.page_bytes
    return np.concatenate([arena[p * P:(p + 1) * P] for p in tb.page_alloc[:om.NP].astype(np.int64)])


def view_ptr(cloak_lib, cm):
    return cloak_lib.cloak_arena(cm.ctx, 2)


@pytest.mark.parametrize("dtype", [synth.DT_BF16, synth.DT_E4M3])
def test_views_hold_the_oracle_layout(cloak_lib, dtype):
    m = vmm_model(dtype)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0xC0FFEE, twin=False, vmm=True)
    assert cm.NP >= 4
    st = cm.vmm_stats()
    assert st["chunks"] > cm.NPS and st["remaps"] == 1 and st["pages_remapped"] == cm.NP
    assert st["remap_us"] > 0
    phys = cm.arena_bytes(0).cpu().numpy()
    assert np.array_equal(phys, arena)
    view = cm.arena_bytes(2).cpu().numpy()
    assert view.size == cm.NP * m.page_bytes
    assert np.array_equal(view, virtual_order(arena, tb, om))
    cm.close()


@pytest.mark.parametrize("dtype,Ms", [(synth.DT_BF16, (1, 5, 16, 64, 300)),
                                      (synth.DT_E4M3, (1, 3, 40, 260))])
def test_linear_on_the_view_equals_the_arena_read(cloak_lib, dtype, Ms):
    """Same tiles, same summation order: bit for bit, and within the linear's
    oracle bound (1e-2 BF16, 5e-2 E4M3); M = 300 / 260 take the prefill GEMM."""
    m = vmm_model(dtype)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0xBEEF, twin=False, vmm=True)
    tol = 1e-2 if dtype == synth.DT_BF16 else 5e-2
    for M in Ms:
        for t in (0, 4, 6):
            x = synth.activations_host(M, m.tensors[t].k, seed=M + t)
            xd = x_device(m, x)
            ya = cm.linear(t, xd, out_dtype=cloak_lib.OUT_F32)
            yv = cm.linear(t, xd, out_dtype=cloak_lib.OUT_F32, vmm=True)
            torch.cuda.synchronize()
            assert torch.equal(ya, yv), (M, t)
            ref = O.cloaked_linear(om, tb, t, arena, x, scales[t] if scales else None)
            assert O.relative_error(yv.cpu().numpy(), ref) <= tol, (M, t)
        xs = [x_device(m, synth.activations_host(M, tt.k, seed=7 * i + M)) for i, tt in enumerate(m.tensors[:7])]
        ba = cm.linear_batch(list(range(7)), xs, out_dtype=cloak_lib.OUT_F32)
        bv = cm.linear_batch(list(range(7)), xs, out_dtype=cloak_lib.OUT_F32, vmm=True)
        torch.cuda.synchronize()
        for a, b in zip(ba, bv):
            assert torch.equal(a, b), M
    assert cm.device_status() == 0
    cm.close()


def test_rekey_moves_the_pages_behind_a_fixed_pointer(cloak_lib):
    """After each re-key the view, at the same address, holds the new epoch's
    oracle layout, and results on it do not change."""
    m = vmm_model()
    key = 0xFACE
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, twin=False, vmm=True)
    ptr0 = view_ptr(cloak_lib, cm)
    x = x_device(m, synth.activations_host(8, m.tensors[5].k, seed=1))
    y0 = cm.linear(5, x, out_dtype=cloak_lib.OUT_F32, vmm=True).cpu()
    for e in (1, 2):
        cm.rekey(key, e)
        tbe = O.keygen(om, key, e)
        O.rekey(om, tb0, tbe, arena0)
        tb0 = tbe
        assert view_ptr(cloak_lib, cm) == ptr0
        st = cm.vmm_stats()
        assert st["remaps"] == 1 + e and 0 < st["pages_remapped"] <= cm.NP
        view = cm.arena_bytes(2).cpu().numpy()
        assert np.array_equal(view, virtual_order(arena0, tbe, om)), e
        ye = cm.linear(5, x, out_dtype=cloak_lib.OUT_F32, vmm=True).cpu()
        assert torch.equal(ye, y0), e
    # a re-key to the same epoch moves no page and remaps none
    cm.rekey(key, 2)
    assert cm.vmm_stats()["pages_remapped"] == 0
    assert cm.device_status() == 0
    cm.close()


def test_concurrent_rekey_remaps_at_its_end(cloak_lib):
    """While a concurrent re-key moves pages the view is refused (its pages
    would be stale); the last advance remaps it to the new epoch."""
    m = vmm_model()
    key = 0xAB
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, twin=False, vmm=True)
    x = x_device(m, synth.activations_host(4, m.tensors[2].k, seed=2))
    y0 = cm.linear(2, x, out_dtype=cloak_lib.OUT_F32, vmm=True).cpu()
    serve, side = torch.cuda.Stream(), torch.cuda.Stream()
    cm.rekey_begin(key, 1, side)
    done = False
    while not done:
        with torch.cuda.stream(serve):
            ya = cm.linear(2, x, out_dtype=cloak_lib.OUT_F32)
            if not done:
                with pytest.raises(cloak_lib.CloakError):
                    cm.linear(2, x, out_dtype=cloak_lib.OUT_F32, vmm=True)
        done = cm.rekey_advance(serve, side)
        serve.synchronize()
        assert torch.equal(ya.cpu(), y0)
    tb1 = O.keygen(om, key, 1)
    O.rekey(om, tb0, tb1, arena0)
    assert np.array_equal(cm.arena_bytes(2).cpu().numpy(), virtual_order(arena0, tb1, om))
    assert torch.equal(cm.linear(2, x, out_dtype=cloak_lib.OUT_F32, vmm=True).cpu(), y0)
    assert cm.device_status() == 0
    cm.close()


@pytest.mark.parametrize("M", [1, 20])
def test_stack_decode_on_the_view(cloak_lib, M):
    """The persistent layer stack (its L2 prefetch included) on the view:
    bit for bit the arena read, within 1e-2 of the FP64 stack oracle."""
    m = synth.small_decoder(2, synth.DT_BF16, d_model=1024, n_heads=8, n_kv_heads=2, d_ff=1408,
                            head_dim=128, spare_pages=2, page_bytes=MiB2)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x5A, twin=False, vmm=True)
    h0 = synth.activations_host(M, m.d_model, seed=M)
    ha = cm.stack_decode(torch.from_numpy(h0).cuda())
    hv = cm.stack_decode(torch.from_numpy(h0).cuda(), vmm=True)
    torch.cuda.synchronize()
    assert torch.equal(ha, hv)
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    assert O.relative_error(hv.cpu().numpy(), O.stack_decode_f64(m, W64, h0)) <= 1e-2
    assert cm.device_status() == 0
    cm.close()


def test_vmm_context_rules(cloak_lib):
    """Pages smaller than the VMM granularity are refused at creation; the
    view flag is refused on a context without it and together with the twin
    flag."""
    small = synth.small_decoder(1, synth.DT_BF16)  # 4-tile (128 KiB) pages
    with pytest.raises(cloak_lib.CloakError):
        cloak_lib.CloakModel(small, vmm=True)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, small, key=1, twin=True)
    x = x_device(small, synth.activations_host(2, small.tensors[0].k, seed=0))
    with pytest.raises(cloak_lib.CloakError):
        cm.linear(0, x, vmm=True)
    with pytest.raises(cloak_lib.CloakError):
        cm.vmm_stats()
    cm.close()
    m = vmm_model()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=2, twin=True, vmm=True)
    x = x_device(m, synth.activations_host(2, m.tensors[0].k, seed=0))
    with pytest.raises(cloak_lib.CloakError):
        cm.linear(0, x, vmm=True, uncloaked=True)
    yt = cm.linear(0, x, out_dtype=cloak_lib.OUT_F32, uncloaked=True)
    yv = cm.linear(0, x, out_dtype=cloak_lib.OUT_F32, vmm=True)
    torch.cuda.synchronize()
    assert torch.equal(yt, yv)
    cm.close()
