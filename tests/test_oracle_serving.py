"""Pins of the serving step's FP64 reference (the full forward: RoPE, causal
GQA attention, SwiGLU, unit-gain RMSNorm): properties that fix RoPE, and the
forward's agreement with the independently written stack reference and with
causality."""
import numpy as np

import oracle as O
from paper_2606_18400_gb300 import synth


def test_rope_is_the_identity_at_position_zero_and_keeps_pair_norms():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 3, 128))
    assert np.allclose(O.rope_f64(x[:1], [0]), x[:1], rtol=0, atol=0)
    y = O.rope_f64(x, np.arange(5) * 7)
    n0 = x[..., :64] ** 2 + x[..., 64:] ** 2
    n1 = y[..., :64] ** 2 + y[..., 64:] ** 2
    assert np.allclose(n0, n1, rtol=1e-12)


def test_rope_first_pair_turns_by_the_position():
    """Pair i = 0 has frequency theta^0 = 1: position p rotates it by p radians."""
    x = np.zeros((1, 1, 128))
    x[0, 0, 0] = 1.0                       # (a, b) = (1, 0) in pair 0
    for p in (1, 2, 5):
        y = O.rope_f64(x, [p])
        assert np.isclose(y[0, 0, 0], np.cos(p)) and np.isclose(y[0, 0, 64], np.sin(p))


def test_rope_scores_depend_only_on_the_distance():
    rng = np.random.default_rng(1)
    q = rng.standard_normal((1, 1, 128))
    k = rng.standard_normal((1, 1, 128))
    s = lambda pq, pk: float(np.sum(O.rope_f64(q, [pq]) * O.rope_f64(k, [pk])))
    assert np.isclose(s(10, 3), s(107, 100), rtol=1e-9)
    assert np.isclose(s(5, 5), float(np.sum(q * k)), rtol=1e-9)


def served(layers=2):
    m = synth.small_decoder(layers, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384,
                            head_dim=128)
    return synth.with_lm_head(m, 200)


def test_forward_is_causal():
    m = served()
    W = [w.astype(np.float64) for w in synth.weights_host(m, seed=2, std=0.05)]
    emb = synth.embedding_host(200, 512).astype(np.float64)
    a = O.transformer_logits_f64(m, W, emb, [3, 17, 42, 99, 5])
    b = O.transformer_logits_f64(m, W, emb, [3, 17, 42, 150, 151])
    assert np.allclose(a[:3], b[:3], rtol=0, atol=0)
    assert not np.allclose(a[3], b[3])


def test_one_token_forward_is_the_stack_step_then_the_output_projection():
    """For a single token at position 0 the attention is the token's own
    value (RoPE is the identity there): the forward equals the stack
    reference (written separately, one-token attention) followed by the final
    unit-gain RMSNorm and the lm_head."""
    m = served()
    dec = synth.small_decoder(2, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384,
                              head_dim=128)
    W = [w.astype(np.float64) for w in synth.weights_host(m, seed=3, std=0.05)]
    emb = synth.embedding_host(200, 512).astype(np.float64)
    tok = 77
    got = O.transformer_logits_f64(m, W, emb, [tok])[0]
    h = O.stack_decode_f64(dec, W[:len(dec.tensors)], emb[tok][None, :])[0]
    ref = (h / np.sqrt(np.mean(h * h) + 1e-5)) @ W[-1].T
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)
