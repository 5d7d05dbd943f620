"""Pins of the oracle's MoE FFN (§5's MoE model, Qwen3-30B-A3B shape):
properties of softmax top-k routing that hold whatever the weights, and the
stored router's relation to the expert-order permutation."""
import numpy as np
import pytest

import oracle as O
from paper_2606_18400_gb300 import synth


def rand_experts(rng, E, d, f):
    return [tuple(rng.standard_normal(s) * 0.1 for s in ((f, d), (f, d), (d, f))) for _ in range(E)]


def test_identical_experts_give_that_expert_whatever_the_routing():
    rng = np.random.default_rng(0)
    E, d, f = 8, 16, 12
    one = rand_experts(rng, 1, d, f)[0]
    x = rng.standard_normal((3, d))
    Wr = rng.standard_normal((E, d))
    y, z, sel, w = O.moe_ffn_f64(x, Wr, [one] * E, top_k=3)
    g, u, dn = one
    ref = np.stack([dn @ (O.silu(g @ xm) * (u @ xm)) for xm in x])
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)
    assert np.allclose(w.sum(1), 1.0)


def test_top1_is_the_argmax_expert_with_weight_one():
    rng = np.random.default_rng(1)
    E, d, f = 6, 10, 8
    ex = rand_experts(rng, E, d, f)
    x = rng.standard_normal((4, d))
    Wr = rng.standard_normal((E, d))
    y, z, sel, w = O.moe_ffn_f64(x, Wr, ex, top_k=1)
    for m in range(4):
        e = int(np.argmax(x[m] @ Wr.T))
        g, u, dn = ex[e]
        assert sel[m, 0] == e and w[m, 0] == 1.0
        assert np.allclose(y[m], dn @ (O.silu(g @ x[m]) * (u @ x[m])), rtol=1e-12)


def test_all_experts_selected_is_the_softmax_mixture():
    """top_k = E: the softmax-gated mixture of all experts (no selection)."""
    rng = np.random.default_rng(2)
    E, d, f = 5, 9, 7
    ex = rand_experts(rng, E, d, f)
    x = rng.standard_normal((2, d))
    Wr = rng.standard_normal((E, d))
    y, z, sel, w = O.moe_ffn_f64(x, Wr, ex, top_k=E)
    for m in range(2):
        zz = x[m] @ Wr.T
        p = np.exp(zz - zz.max()) / np.exp(zz - zz.max()).sum()
        outs = np.stack([dn @ (O.silu(g @ x[m]) * (u @ x[m])) for g, u, dn in ex])
        assert np.allclose(y[m], p @ outs, rtol=1e-12)


def test_relabelling_experts_changes_nothing():
    rng = np.random.default_rng(3)
    E, d, f = 8, 12, 6
    ex = rand_experts(rng, E, d, f)
    x = rng.standard_normal((3, d))
    Wr = rng.standard_normal((E, d))
    perm = rng.permutation(E)
    y0 = O.moe_ffn_f64(x, Wr, ex, top_k=3)[0]
    y1 = O.moe_ffn_f64(x, Wr[perm], [ex[p] for p in perm], top_k=3)[0]
    assert np.allclose(y0, y1, rtol=1e-12)


def test_ties_go_to_the_lower_expert_and_selection_follows_the_given_logits():
    z = np.array([[1.0, 3.0, 3.0, 0.5, 3.0]])
    sel, w = O.moe_route_f64(z, 2)
    assert list(sel[0]) == [1, 2] and np.allclose(w[0], [0.5, 0.5])
    rng = np.random.default_rng(4)
    ex = rand_experts(rng, 5, 4, 3)
    x = rng.standard_normal((1, 4))
    y, _, s2, _ = O.moe_ffn_f64(x, rng.standard_normal((5, 4)), ex, top_k=2, select_logits=z)
    assert list(s2[0]) == [1, 2]


def test_stored_router_rows_follow_the_expert_permutation():
    """The kernel maps the router's stored output e' to logical expert
    group_perm[e']: the stored router matrix is the logical one with rows in
    that order."""
    m = synth.moe_block(d_model=256, n_experts=16, top_k=4, d_ff=256, spare_pages=3, page_bytes=4 * 32768)
    om = O.OracleModel(m)
    tb = O.keygen(om, 0x5, 0)
    Ws = synth.weights_host(m, seed=1)
    arena, _ = O.shuffle_model(om, tb, Ws)
    r = m.router_tensors[0]
    stored = O.stored_f64(om, tb, r, arena)
    gp = O.group_perm(om, tb, m.expert_groups[0]).astype(np.int64)
    assert not np.array_equal(gp, np.arange(16))
    assert np.array_equal(stored, O.bf16_value(O.bf16_bits(Ws[r]))[gp])
