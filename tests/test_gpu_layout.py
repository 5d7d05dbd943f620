"""GPU keygen, shuffle and unshuffle against the oracle: bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both

pytestmark = pytest.mark.gpu

TABLES = ["layer_perm", "group_perm", "tensor_base", "tile_perm", "page_alloc", "tile_slot"]


def small_models():
    return {
        "mlp2": synth.mlp2(),
        "bf16_2L": synth.small_decoder(2, synth.DT_BF16),
        "e4m3_2L": synth.small_decoder(2, synth.DT_E4M3, page_bytes=2 * 128 * 128),
        "bf16_gqa_ragged": synth.small_decoder(3, synth.DT_BF16, d_model=384, n_heads=6,
                                               n_kv_heads=2, d_ff=200, spare_pages=5),
    }


def compare_tables(cloak, cm, om, tb):
    for i, name in enumerate(TABLES):
        got = cm.table(i)
        ref = getattr(tb, name)
        n = {0: om.L, 1: om.U, 2: len(om.model.tensors), 3: om.G, 4: om.NPS, 5: om.G}[i]
        assert np.array_equal(got[:n], ref[:n]), name


@pytest.mark.parametrize("name", list(small_models()))
@pytest.mark.parametrize("key,epoch", [(0x1234, 0), (0xDEADBEEFCAFEF00D, 3), (2**64 - 1, 1)])
def test_keygen_tables_bit_exact(cloak_lib, name, key, epoch):
    m = small_models()[name]
    cm = cloak_lib.CloakModel(m)
    cm.keygen(key, epoch)
    om = O.OracleModel(m)
    compare_tables(cloak_lib, cm, om, O.keygen(om, key, epoch))
    cm.close()


def test_keygen_per_tensor_scope(cloak_lib):
    m = synth.small_decoder(2, synth.DT_BF16)
    m.tile_scope = 1
    cm = cloak_lib.CloakModel(m)
    om = O.OracleModel(m)
    for key in (1, 2, 3):
        cm.keygen(key, 0)
        compare_tables(cloak_lib, cm, om, O.keygen(om, key, 0))


def test_keygen_sequential_path_agrees(cloak_lib, monkeypatch):
    """The sequential Fisher-Yates kernel (taken when a bounded draw rejects)
    gives the same tables as the parallel one."""
    m = synth.small_decoder(2, synth.DT_BF16, d_ff=640)
    om = O.OracleModel(m)
    monkeypatch.setenv("CLOAK_FY_SEQUENTIAL", "1")
    cm = cloak_lib.CloakModel(m)
    cm.keygen(77, 2)
    compare_tables(cloak_lib, cm, om, O.keygen(om, 77, 2))


@pytest.mark.parametrize("mk", [lambda: synth.llama7b_layer(1), lambda: synth.gqa28_fp8(28),
                                lambda: synth.llama7b_layer(32)])
def test_keygen_full_size_bit_exact(cloak_lib, mk):
    m = mk()
    om = O.OracleModel(m)
    cm = cloak_lib.CloakModel(m)
    cm.keygen(0x1234, 0)
    compare_tables(cloak_lib, cm, om, O.keygen(om, 0x1234, 0))
    cm.close()


@pytest.mark.parametrize("name", list(small_models()))
def test_shuffle_arena_bit_exact(cloak_lib, name):
    m = small_models()[name]
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234)
    got = cm.arena_bytes(0).cpu().numpy()
    assert np.array_equal(got, arena)
    if m.dtype == synth.DT_E4M3:
        for t in range(len(m.tensors)):
            assert np.array_equal(cm.scales(t).cpu().numpy(), scales[t])
    # the twin is the identity layout: tile g at slot g
    twin = cm.arena_bytes(1).cpu().numpy()
    tbytes = om.tile_bytes
    slots = tb.tile_slot.astype(np.int64)
    for g in range(om.G):
        assert np.array_equal(twin[g * tbytes:(g + 1) * tbytes],
                              arena[slots[g] * tbytes:(slots[g] + 1) * tbytes])
    cm.close()


@pytest.mark.parametrize("name", list(small_models()))
def test_unshuffle_round_trip(cloak_lib, name):
    m = small_models()[name]
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=99)
    for t in range(len(m.tensors)):
        ref = O.unshuffle(om, tb, t, arena)
        for twin in (False, True):
            got = cm.unshuffle(t, from_twin=twin).cpu().numpy()
            assert np.array_equal(got.view(np.uint8), ref.view(np.uint8))
    cm.close()


def test_shuffle_full_size_layer(cloak_lib):
    """One 7B-class BF16 layer (12,352 tiles, 257 pages): arena bit-exact."""
    m = synth.llama7b_layer(1)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=0x1234, twin=False)
    got = cm.arena_bytes(0).cpu().numpy()
    assert np.array_equal(got, arena)
    cm.close()


@pytest.mark.parametrize("mk,seed", [(lambda: synth.gqa28_fp8(28), 7),
                                     (lambda: synth.llama7b_layer(32), 0)])
def test_shuffle_full_size_sampled(cloak_lib, mk, seed):
    """Full-size models (28-layer E4M3, 398,272 tiles; 32-layer BF16,
    395,264 tiles, 12.95 GB): every tensor placed from device-drawn weights; a
    keyed sample of tensors has 16 random tiles and all its FP8 scales compared
    bit for bit with the oracle's stored matrix."""
    import torch
    m = mk()
    om = O.OracleModel(m)
    tb = O.keygen(om, 7, 0)
    cm = cloak_lib.CloakModel(m)
    cm.keygen(7, 0)
    rng = np.random.default_rng(5)
    sample_t = set(int(t) for t in rng.choice(len(m.tensors), 5, replace=False))
    Wd = {}
    for t in range(len(m.tensors)):
        w = synth.weights_device(m, t, seed=seed)
        cm.shuffle(t, w)
        if t in sample_t:
            Wd[t] = w.cpu().numpy()
        del w
    torch.cuda.synchronize()
    arena_dev = cm.arena_bytes(0)
    tbytes = om.tile_bytes
    for t in sorted(sample_t):
        codes, sc = O.stored_codes(om, tb, t, Wd[t])
        nt, kt = m.tiles_of(m.tensors[t])
        base = int(tb.tensor_base[t])
        for u in rng.choice(nt * kt, 16, replace=False):
            s = int(tb.tile_slot[base + u])
            got = arena_dev[s * tbytes:(s + 1) * tbytes].cpu().numpy()
            assert np.array_equal(got, O.tile_of(om, codes, u // kt, u % kt))
        if sc is not None:
            assert np.array_equal(cm.scales(t).cpu().numpy(), sc)
    cm.close()
