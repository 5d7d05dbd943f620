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


def test_full_stack_32_layers_against_the_oracle(cloak_lib):
    """The 12.95 GB 32-layer stack (weights drawn on the device), decode at
    M = 1 and M = 8, checked layer by layer against the FP64 oracle: the
    launch runs the first l layers for every l = 1..32 (the same stage splits
    as the full stack, so the same intermediate states), and each layer's
    output must be within 1e-2 of the oracle's layer step applied to the
    launch's own input of that layer, normwise and per token. Each layer's
    weights are redrawn on the device from their seeds and brought to the
    host alone. The full 32-layer step is bit-identical between the cloaked
    arena and the twin. The drift of the whole step from the all-FP64 chain
    is printed: this random-weight model amplifies any per-layer difference
    (its residual stream grows about 15-fold over the 32 layers), so the
    chain is not a bound on the kernel."""
    import concurrent.futures as cf
    m = synth.llama7b_layer(32)
    one = synth.llama7b_layer(1)  # the structure of one layer for the oracle
    cm = cloak_lib.CloakModel(m, twin=True)
    cm.keygen(0x1234, 0)
    for t in range(len(m.tensors)):
        cm.shuffle(t, synth.weights_device(m, t, seed=0))
    desc = cm.stack_desc()
    lt = [desc.layer_tensors[i] for i in range(32 * 7)]
    h0 = {M: synth.activations_host(M, 4096, seed=30 + M) for M in (1, 8)}
    hs = {}
    for M in (1, 8):
        hs[M] = [h0[M].astype(np.float64)]
        for l in range(1, 33):
            desc.num_layers = l
            h = cm.stack_decode(torch.from_numpy(h0[M]).cuda(), desc=desc)
            torch.cuda.synchronize()
            hs[M].append(h.cpu().numpy().astype(np.float64))
        h2 = cm.stack_decode(torch.from_numpy(h0[M]).cuda(), uncloaked=True, desc=desc)
        torch.cuda.synchronize()
        assert np.array_equal(h2.cpu().numpy().astype(np.float64), hs[M][32])
    assert cm.device_status() == 0
    cm.close()
    exact = {M: h0[M].astype(np.float64) for M in (1, 8)}

    def w64(t):
        return O.bf16_value(O.bf16_bits(synth.weights_device(m, t, seed=0).cpu().numpy()))

    worst = {1: 0.0, 8: 0.0}
    worst_b = {1: 0.0, 8: 0.0}
    with cf.ThreadPoolExecutor(7) as ex:
        for l in range(32):
            W64 = list(ex.map(w64, lt[7 * l:7 * l + 7]))  # q, k, v, o, gate, up, down
            for M in (1, 8):
                ref = O.stack_decode_f64(one, W64, hs[M][l])
                err = O.relative_error(hs[M][l + 1], ref)
                assert err <= 1e-2, (M, l, err)
                for i in range(M):
                    assert O.relative_error(hs[M][l + 1][i:i + 1], ref[i:i + 1]) <= 1e-2, (M, l, i)
                worst[M] = max(worst[M], err)
                refb = O.stack_decode_f64(one, W64, hs[M][l], bf16_operands=True)
                worst_b[M] = max(worst_b[M], O.relative_error(hs[M][l + 1], refb))
                exact[M] = O.stack_decode_f64(one, W64, exact[M])
            del W64
    for M in (1, 8):
        drift = O.relative_error(hs[M][32], exact[M])
        grow = O.relative_error(exact[M], h0[M].astype(np.float64))
        print(f"32-layer stack M={M}: worst layer {worst[M]:.3e} vs the FP64 step, "
              f"{worst_b[M]:.3e} vs the BF16-operand step; whole step {drift:.3e} from the "
              f"all-FP64 chain (residual change {grow:.1f}x)")
        assert grow > 0.5
