"""Cloaked MoE FFN block (the paper's MoE model, Qwen3-30B-A3B shape)
against the FP64 oracle: router logits (FP32, normwise 1e-5), the routing
decided on the kernel's own logits (the same precision on both sides: the
oracle's selection must equal the kernel's exactly), and the output within
1e-2 (the intermediate activation is BF16); the cloaked read equals the
uncloaked twin's and the VMM view's bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu


def small_moe(page_bytes=4 * 32768):
    return synth.moe_block(n_layers=1, d_model=256, n_experts=16, top_k=4, d_ff=384, spare_pages=3,
                           page_bytes=page_bytes)


def run(cloak_lib, cm, x, **kw):
    m = cm.model
    M = x.shape[0]
    ex = torch.zeros((M, m.top_k), dtype=torch.int32, device="cuda")
    lg = torch.zeros((M, m.n_experts), dtype=torch.float32, device="cuda")
    y = cm.moe_ffn(x, experts_out=ex, logits_out=lg, **kw)
    torch.cuda.synchronize()
    return y.cpu().numpy(), ex.cpu().numpy(), lg.cpu().numpy()


def check_against_oracle(m, x_bf16, y, ex, lg, W64):
    """W64(t) -> FP64 logical weights of tensor t."""
    x64 = O.bf16_value(O.bf16_bits(x_bf16.float().cpu().numpy()))
    r = m.router_tensors[0]
    z = x64 @ W64(r).T
    assert O.relative_error(lg, z) <= 1e-5
    sel, w = O.moe_route_f64(lg, m.top_k)
    assert np.array_equal(sel, ex)

    class Experts:
        def __getitem__(self, e):
            g, u, d = m.expert_tensors[0][e]
            return W64(g), W64(u), W64(d)

    ref, _, _, _ = O.moe_ffn_f64(x64, W64(r), Experts(), m.top_k, select_logits=lg)
    err = O.relative_error(y, ref)
    assert err <= 1e-2, err
    return err


@pytest.mark.parametrize("M", [1, 3, 17])
def test_small_moe_block_matches_oracle(cloak_lib, M):
    m = small_moe()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x3E, twin=True)
    xh = synth.activations_host(M, m.d_model, seed=M)
    x = x_device(m, xh)
    y, ex, lg = run(cloak_lib, cm, x)
    W64 = lambda t: O.bf16_value(O.bf16_bits(Ws[t]))
    check_against_oracle(m, x, y, ex, lg, W64)
    assert len(set(ex[0])) == m.top_k
    yu, exu, lgu = run(cloak_lib, cm, x, uncloaked=True)
    assert np.array_equal(y.view(np.uint32), yu.view(np.uint32)) and np.array_equal(ex, exu)
    assert cm.device_status() == 0
    cm.close()


def test_moe_on_the_vmm_view_and_across_rekeys(cloak_lib):
    m = small_moe(page_bytes=2 << 20)
    key = 0x3F
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=key, twin=False, vmm=True)
    x = x_device(m, synth.activations_host(5, m.d_model, seed=9))
    y0, e0, _ = run(cloak_lib, cm, x)
    yv, ev, _ = run(cloak_lib, cm, x, vmm=True)
    assert np.array_equal(y0.view(np.uint32), yv.view(np.uint32)) and np.array_equal(e0, ev)
    cm.rekey(key, 1)
    y1, e1, _ = run(cloak_lib, cm, x, vmm=True)
    assert np.array_equal(y0.view(np.uint32), y1.view(np.uint32)) and np.array_equal(e0, e1)
    cm.close()


def test_moe_rejects_bad_descriptors(cloak_lib):
    m = small_moe()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=1, twin=False)
    x = x_device(m, synth.activations_host(1, m.d_model, seed=0))
    d = cm.moe_desc()
    d.top_k = 17
    with pytest.raises(cloak_lib.CloakError):
        cm.moe_ffn(x, desc=d)
    d = cm.moe_desc()
    d.expert_group = -1  # the router's rows are permuted: the group is required
    with pytest.raises(cloak_lib.CloakError):
        cm.moe_ffn(x, desc=d)
    cm.close()


@pytest.mark.parametrize("M", [1, 4])
def test_full_size_qwen3_moe_block(cloak_lib, M):
    """128 experts of 768 x 2048 (1.2 GB BF16), top-8: the oracle on the
    experts the kernel selected (weights redrawn on the device from their
    seeds, so only those experts come to the host)."""
    m = synth.moe_block()
    cm = cloak_lib.CloakModel(m)
    cm.keygen(0x1234, 0)
    for t in range(len(m.tensors)):
        cm.shuffle(t, synth.weights_device(m, t, seed=3))
    x = x_device(m, synth.activations_host(M, m.d_model, seed=M + 40))
    y, ex, lg = run(cloak_lib, cm, x)
    W64 = lambda t: O.bf16_value(O.bf16_bits(synth.weights_device(m, t, seed=3).cpu().numpy()))
    check_against_oracle(m, x, y, ex, lg, W64)
    assert cm.device_status() == 0
    cm.close()
