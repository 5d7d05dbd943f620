"""Keyed upload (Section 5, "Implementation Details": the permutation and the
page allocation come before any weight transfer): every page is assembled on
the host and sent whole, in physical order. The arena it leaves equals the
oracle's (and the device shuffle's) bit for bit, E4M3 scales included."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mk,scope", [
    (lambda: synth.small_decoder(2, synth.DT_BF16, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200), 0),
    (lambda: synth.small_decoder(2, synth.DT_BF16, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200), 1),
    (lambda: synth.small_decoder(3, synth.DT_E4M3, page_bytes=2 * 128 * 128, spare_pages=7), 0),
    (lambda: synth.small_decoder(2, synth.DT_F32, spare_pages=0), 0),
    (synth.mlp2, 0),
])
@pytest.mark.parametrize("threads", [1, 0])
def test_upload_equals_the_oracle_arena(cloak_lib, mk, scope, threads):
    m = mk()
    m.tile_scope = scope
    key = 0x0B5C
    Ws = synth.weights_host(m, seed=3)
    cm = cloak_lib.CloakModel(m, twin=False)
    cm.keygen(key, 0)
    cm.upload(Ws, threads=threads)
    om = O.OracleModel(m)
    tb = O.keygen(om, key, 0)
    arena, scales = O.shuffle_model(om, tb, Ws)
    got = cm.arena_bytes(0).cpu().numpy()
    P = m.page_bytes
    for p in tb.page_alloc[:om.NP].astype(np.int64):  # every assigned page
        assert np.array_equal(got[p * P:(p + 1) * P], arena[p * P:(p + 1) * P]), p
    if m.dtype == synth.DT_E4M3:
        for t in range(len(m.tensors)):
            assert np.array_equal(cm.scales(t).cpu().numpy(), scales[t]), t
    cm.close()


def test_upload_equals_device_shuffle_full_size_layer(cloak_lib):
    """The 7B-class layer (193 pages of 2 MiB): upload and device shuffle give
    the same arena, and the same linear results."""
    m = synth.llama7b_layer(1)
    key = 0x1234
    Ws = synth.weights_host(m, seed=0)
    a = cloak_lib.CloakModel(m, twin=False)
    a.keygen(key, 0)
    for t, W in enumerate(Ws):
        a.shuffle(t, torch.from_numpy(np.ascontiguousarray(W)).cuda())
    b = cloak_lib.CloakModel(m, twin=False)
    b.keygen(key, 0)
    b.upload(Ws)
    pa = a.table(cloak_lib.TAB_PAGE_ALLOC)[:a.NP].astype(np.int64)
    ga, gb = a.arena_bytes(0), b.arena_bytes(0)
    P = m.page_bytes
    idx = torch.from_numpy(pa).cuda()
    va = ga.view(-1, P).index_select(0, idx)
    vb = gb.view(-1, P).index_select(0, idx)
    assert torch.equal(va, vb)
    x = x_device(m, synth.activations_host(4, m.tensors[0].k, seed=5))
    assert torch.equal(a.linear(0, x), b.linear(0, x))
    a.close()
    b.close()


def test_upload_rules(cloak_lib):
    m = synth.mlp2()
    Ws = synth.weights_host(m, seed=1)
    cm = cloak_lib.CloakModel(m, twin=False)
    with pytest.raises(cloak_lib.CloakError):
        cm.upload(Ws)                      # before keygen
    cm.close()
    cm = cloak_lib.CloakModel(m, twin=True)
    cm.keygen(1, 0)
    with pytest.raises(cloak_lib.CloakError):
        cm.upload(Ws)                      # a twin would need the logical layout on the bus
    cm.close()


@pytest.mark.parametrize("dtype", [synth.DT_BF16, synth.DT_E4M3])
def test_upload_equals_device_shuffle_on_every_bit_pattern(cloak_lib, dtype):
    """Weights drawn as random 32-bit patterns (NaNs, infinities, subnormals,
    values exactly halfway between two BF16 values) plus the largest finite
    floats: the host's rounding gives the device conversion's bytes (E4M3:
    finite patterns, scales compared bit for bit)."""
    m = (synth.small_decoder(2, dtype, d_model=384, n_heads=6, n_kv_heads=2, d_ff=200)
         if dtype == synth.DT_BF16 else
         synth.small_decoder(2, dtype, page_bytes=2 * 128 * 128, d_model=384, n_heads=6, n_kv_heads=2,
                             d_ff=256))
    rng = np.random.default_rng(11)
    Ws = []
    for t in m.tensors:
        bits = rng.integers(0, 2**32, size=(t.n, t.k), dtype=np.uint64).astype(np.uint32)
        ties = rng.random((t.n, t.k)) < 0.2          # low 16 bits exactly 0x8000
        bits[ties] = (bits[ties] & 0xFFFF0000) | 0x8000
        bits[0, :4] = [0x7F7FFFFF, 0xFF7FFFFF, 0x7F7F8000, 0x00008000]
        if dtype == synth.DT_E4M3:
            # a NaN's sign after the scale division is the host's or the
            # device's own choice: E4M3 takes finite weights only
            bad = (bits & 0x7F800000) == 0x7F800000
            bits[bad] = (bits[bad] & 0x80000000) | 0x7F7FFFFF
        Ws.append(bits.view(np.float32))
    key = 0x77
    a = cloak_lib.CloakModel(m, twin=False)
    a.keygen(key, 0)
    for t, W in enumerate(Ws):
        a.shuffle(t, torch.from_numpy(np.ascontiguousarray(W)).cuda())
    b = cloak_lib.CloakModel(m, twin=False)
    b.keygen(key, 0)
    b.upload(Ws)
    P = m.page_bytes
    ga, gb = a.arena_bytes(0).cpu().numpy(), b.arena_bytes(0).cpu().numpy()
    for p in a.table(cloak_lib.TAB_PAGE_ALLOC)[:a.NP].astype(np.int64):
        assert np.array_equal(ga[p * P:(p + 1) * P], gb[p * P:(p + 1) * P]), p
    if dtype == synth.DT_E4M3:
        for t in range(len(m.tensors)):
            sa, sb = a.scales(t).cpu().numpy(), b.scales(t).cpu().numpy()
            assert np.array_equal(sa.view(np.uint32), sb.view(np.uint32)), t
    a.close()
    b.close()
