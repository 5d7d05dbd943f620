"""Global residual-dimension permutation: one keyed group shared by the
columns of every matrix that reads the residual stream and the rows of
every matrix that writes it (the embedding and the lm_head included).
Against the oracle: the arena bit for bit (device shuffle and keyed upload),
the stack decode of the permuted stream equal to the logical result
permuted, and the served logits equal to the logical model's (unit-gain
RMSNorm does not see the order)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import cloak, serve, synth
from helpers import place_both

pytestmark = pytest.mark.gpu


def residual_model(dtype=synth.DT_BF16, vocab=1000, layers=2):
    m = synth.small_decoder(layers, dtype, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384, head_dim=128,
                            spare_pages=3)
    return synth.with_residual_permutation(synth.with_lm_head(m, vocab, cloaked_embedding=True))


@pytest.mark.parametrize("dtype", [synth.DT_BF16, synth.DT_E4M3])
def test_arena_equals_the_oracle_by_shuffle_and_by_upload(cloak_lib, dtype):
    m = residual_model(dtype)
    if dtype == synth.DT_E4M3:
        m.page_bytes = 2 * 128 * 128
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x6A, twin=False)
    got = cm.arena_bytes(0).cpu().numpy()
    P = m.page_bytes
    pages = tb.page_alloc[:om.NP].astype(np.int64)
    for p in pages:
        assert np.array_equal(got[p * P:(p + 1) * P], arena[p * P:(p + 1) * P])
    if dtype == synth.DT_E4M3:
        for t in range(len(m.tensors)):
            assert np.array_equal(cm.scales(t).cpu().numpy(), scales[t]), t
    up = cloak_lib.CloakModel(m)
    up.keygen(0x6A, 0)
    up.upload(Ws)
    gu = up.arena_bytes(0).cpu().numpy()
    for p in pages:
        assert np.array_equal(gu[p * P:(p + 1) * P], arena[p * P:(p + 1) * P])
    for t in range(len(m.tensors)):  # unshuffle undoes both axes
        u = cm.unshuffle(t).cpu().numpy()
        if dtype == synth.DT_BF16:
            assert np.array_equal(u.view(np.uint16), O.bf16_bits(Ws[t])), t
    up.close()
    cm.close()


@pytest.mark.parametrize("M", [1, 7])
def test_stack_decode_of_the_permuted_stream(cloak_lib, M):
    m = residual_model(layers=3)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x6B, twin=False)
    gp = O.group_perm(om, tb, m.residual_group).astype(np.int64)
    h0 = synth.activations_host(M, m.d_model, seed=M)
    h = torch.from_numpy(np.ascontiguousarray(h0[:, gp])).cuda()
    desc = cm.stack_desc()
    cm.stack_decode(h, desc=desc)
    torch.cuda.synchronize()
    dec = synth.small_decoder(3, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384, head_dim=128)
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws[:len(dec.tensors)]]
    ref = O.stack_decode_f64(dec, W64, h0)
    assert O.relative_error(h.cpu().numpy(), ref[:, gp]) <= 1e-2
    assert cm.device_status() == 0
    cm.close()


def test_served_logits_match_the_logical_model(cloak_lib):
    m = residual_model()
    Ws = synth.weights_host(m, seed=0, std=0.05)
    sm = serve.ServedModel(m, kv_blocks=256, max_blocks=32, weights=Ws)
    assert sm.embed_tensor >= 0
    dev = "cuda"
    toks = list(np.random.default_rng(8).integers(0, 1000, 21))
    T = lambda a: torch.tensor(a, dtype=torch.int32, device=dev)
    bt = torch.zeros((8, sm.max_blocks), dtype=torch.int32, device=dev)
    bt[0] = torch.arange(sm.max_blocks, dtype=torch.int32)
    out = torch.zeros(1, dtype=torch.int32, device=dev)
    lg = torch.zeros((1, 1000), dtype=torch.float32, device=dev)
    sm.step(T(toks), T(list(range(21))), T([0] * 21), bt, T([20]), out, lg)
    torch.cuda.synchronize()
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    emb64 = O.bf16_value(O.bf16_bits(synth.embedding_host(1000, 512)))
    ref = O.transformer_logits_f64(m, W64, emb64, toks)
    assert O.relative_error(lg.cpu().numpy()[0], ref[20]) <= 1e-2
    assert sm.cm.device_status() == 0
    sm.close()
