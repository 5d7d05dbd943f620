"""Cloaked MoE FFN block (the paper's MoE model, Qwen3-30B-A3B shape)
against the FP64 oracle: router logits (FP32, normwise 1e-5, and every logit
within the a priori bound of an FP32 sum of K products); the routing checked
against the oracle's own selection on its FP64 logits (every expert the
kernel picked is within twice the measured logit error of the oracle's k-th
best, and where the oracle's margin between its k-th and (k+1)-th expert is
wider than that, the two selections are the same set and the output is
compared with the oracle computed end to end on its own routing); the output
within 1e-2 normwise and per token (the intermediate activation is BF16); the
cloaked read equals the uncloaked twin's and the VMM view's bit for bit."""
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
    """W64(t) -> FP64 logical weights of tensor t. Returns (output error,
    tokens whose routing the oracle decided alone)."""
    x64 = O.bf16_value(O.bf16_bits(x_bf16.float().cpu().numpy()))
    r = m.router_tensors[0]
    Wr = W64(r)
    z = x64 @ Wr.T
    assert O.relative_error(lg, z) <= 1e-5
    # a priori: an FP32 sum of K products in any order is within
    # gamma_K * sum |x w| of the exact sum (gamma_K = K u / (1 - K u), u = 2^-24)
    K = x64.shape[1]
    u = 2.0 ** -24
    gamma = K * u / (1 - K * u)
    assert np.all(np.abs(lg - z) <= gamma * (np.abs(x64) @ np.abs(Wr).T) + 1e-30)
    eps = float(np.abs(lg - z).max())
    k = m.top_k
    sel_o, _ = O.moe_route_f64(z, k)

    class Experts:
        def __getitem__(self, e):
            g, u_, d = m.expert_tensors[0][e]
            return W64(g), W64(u_), W64(d)

    decided = 0
    for t in range(x64.shape[0]):
        zs = np.sort(z[t])[::-1]
        # every expert the kernel chose scores, in FP64, within 2 eps of the k-th best
        assert np.all(z[t, ex[t]] >= zs[k - 1] - 2 * eps), (t, ex[t], zs[k - 1], eps)
        assert len(set(ex[t].tolist())) == k
        if k < z.shape[1] and zs[k - 1] - zs[k] > 2 * eps:
            assert set(ex[t].tolist()) == set(sel_o[t].tolist()), (t, ex[t], sel_o[t])
            decided += 1
    # the output: the oracle on its own routing (FP64 logits) where it decided
    # alone, else on the kernel's selection (a near tie of the logits)
    ref_own, _, _, _ = O.moe_ffn_f64(x64, Wr, Experts(), k)
    ref_sel, _, _, _ = O.moe_ffn_f64(x64, Wr, Experts(), k, select_logits=lg)
    ref = ref_sel.copy()
    for t in range(x64.shape[0]):
        zs = np.sort(z[t])[::-1]
        if k < z.shape[1] and zs[k - 1] - zs[k] > 2 * eps:
            ref[t] = ref_own[t]
    err = O.relative_error(y, ref)
    assert err <= 1e-2, err
    for t in range(x64.shape[0]):  # no single bad token hidden by the norm over all
        assert O.relative_error(y[t:t + 1], ref[t:t + 1]) <= 1e-2, t
    return err, decided


@pytest.mark.parametrize("M", [1, 3, 17])
def test_small_moe_block_matches_oracle(cloak_lib, M):
    m = small_moe()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x3E, twin=True)
    xh = synth.activations_host(M, m.d_model, seed=M)
    x = x_device(m, xh)
    y, ex, lg = run(cloak_lib, cm, x)
    W64 = lambda t: O.bf16_value(O.bf16_bits(Ws[t]))
    _, decided = check_against_oracle(m, x, y, ex, lg, W64)
    assert decided >= (M + 1) // 2  # the oracle decided most routings on its own
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
    """128 experts of 768 x 2048 (1.2 GB BF16), top-8: the oracle's own
    routing on its FP64 logits (the kernel's where the logits nearly tie),
    weights redrawn on the device from their seeds, so only the router and
    the selected experts come to the host."""
    m = synth.moe_block()
    cm = cloak_lib.CloakModel(m)
    cm.keygen(0x1234, 0)
    for t in range(len(m.tensors)):
        cm.shuffle(t, synth.weights_device(m, t, seed=3))
    x = x_device(m, synth.activations_host(M, m.d_model, seed=M + 40))
    y, ex, lg = run(cloak_lib, cm, x)
    W64 = lambda t: O.bf16_value(O.bf16_bits(synth.weights_device(m, t, seed=3).cpu().numpy()))
    _, decided = check_against_oracle(m, x, y, ex, lg, W64)
    assert decided >= 1
    assert cm.device_status() == 0
    cm.close()


def test_tied_router_rows_route_to_the_lower_expert(cloak_lib):
    """Experts 2 and 9 get the same router row (scaled up so they are often
    selected): in one tile row their FP32 logits are computed alike and tie
    exactly, and the tie goes to the lower logical expert, so whenever 9 is
    selected 2 is too, ranked before it."""
    m = small_moe()
    r = m.router_tensors[0]
    Ws = synth.weights_host(m, seed=21)
    Ws[r][2] *= 4.0
    Ws[r][9] = Ws[r][2]
    cm, om, tb, arena, scales, _ = place_both(cloak_lib, m, key=0x40, twin=False, weights=Ws)
    x = x_device(m, synth.activations_host(64, m.d_model, seed=5))
    y, ex, lg = run(cloak_lib, cm, x)
    assert np.array_equal(lg[:, 2].view(np.uint32), lg[:, 9].view(np.uint32))
    both = 0
    for t in range(64):
        e = ex[t].tolist()
        if 9 in e:
            assert 2 in e
            both += 1
    assert both >= 8
    W64 = lambda t: O.bf16_value(O.bf16_bits(Ws[t]))
    check_against_oracle(m, x, y, ex, lg, W64)
    cm.close()
