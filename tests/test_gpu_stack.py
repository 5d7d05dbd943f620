"""GPU persistent layer-stack decode against the FP64 oracle (normwise
relative error of the residual stream <= 1e-2), bit-identical between the
cloaked and uncloaked arenas and unchanged by a re-key."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both

pytestmark = pytest.mark.gpu


def small_stack(layers=3, d_ff=320):
    return synth.small_decoder(layers, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2,
                               d_ff=d_ff, head_dim=128, spare_pages=3)


def oracle_h(m, Ws, h0):
    W64 = [O.bf16_value(O.bf16_bits(w)) for w in Ws]
    return O.stack_decode_f64(m, W64, h0)


@pytest.mark.parametrize("M", [1, 5, 16, 40])
def test_small_stack_matches_oracle(cloak_lib, M):
    m = small_stack()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x51AC)
    h0 = synth.activations_host(M, m.d_model, seed=M)
    h = torch.from_numpy(h0).cuda()
    cm.stack_decode(h)
    hu = torch.from_numpy(h0).cuda()
    cm.stack_decode(hu, uncloaked=True)
    torch.cuda.synchronize()
    assert cm.device_status() == 0
    ref = oracle_h(m, Ws, h0)
    err = O.relative_error(h.cpu().numpy(), ref)
    delta = O.relative_error(ref, h0.astype(np.float64))  # the stack really changes h
    assert err <= 1e-2 and delta > 0.1, (err, delta)
    assert torch.equal(h, hu)
    cm.close()


def test_stack_survives_rekey_and_repeats(cloak_lib):
    m = small_stack(2, d_ff=384)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x77)
    h0 = synth.activations_host(3, m.d_model, seed=9)
    a = cm.stack_decode(torch.from_numpy(h0).cuda())
    b = cm.stack_decode(torch.from_numpy(h0).cuda())
    cm.rekey(0x77, 1)
    c = cm.stack_decode(torch.from_numpy(h0).cuda())
    torch.cuda.synchronize()
    assert torch.equal(a, b) and torch.equal(a, c)
    cm.close()


@pytest.mark.parametrize("M", [1, 8])
def test_full_size_two_layer_stack(cloak_lib, M):
    """Two 7B-class layers (d 4096, 32 heads, MLP 11008) against the oracle."""
    m = synth.llama7b_layer(2)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234, twin=False)
    h0 = synth.activations_host(M, 4096, seed=21)
    h = cm.stack_decode(torch.from_numpy(h0).cuda())
    torch.cuda.synchronize()
    err = O.relative_error(h.cpu().numpy(), oracle_h(m, Ws, h0))
    assert err <= 1e-2, err
    cm.close()


def test_full_stack_32_layers_cloaked_equals_uncloaked(cloak_lib):
    """The 12.95 GB 32-layer stack (weights drawn on the device): one decode
    step is finite and bit-identical between the cloaked arena and the twin."""
    m = synth.llama7b_layer(32)
    cm = cloak_lib.CloakModel(m, twin=True)
    cm.keygen(0x1234, 0)
    for t in range(len(m.tensors)):
        cm.shuffle(t, synth.weights_device(m, t, seed=0))
    h0 = torch.from_numpy(synth.activations_host(4, 4096, seed=3)).cuda()
    h1 = cm.stack_decode(h0.clone())
    h2 = cm.stack_decode(h0.clone(), uncloaked=True)
    torch.cuda.synchronize()
    assert torch.isfinite(h1).all()
    assert torch.equal(h1, h2)
    assert cm.device_status() == 0
    cm.close()
