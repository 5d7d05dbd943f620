"""Tile-level re-key (CLOAK_MODEL_TILE_REKEY): the tile permutation is
redrawn at every epoch too, and cloak_rekey moves every tile to its new slot
(Section 4.2 periodic re-randomisation, at tile granularity). Checked
against the oracle: the tables at every epoch bit for bit, the arena after a
re-key equal to a fresh shuffle at the new epoch (and to the oracle's own
tile re-key), linear and serving results unchanged."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import serve, synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu


def mapped(arena, tb, om):
    P = om.model.page_bytes
    return np.concatenate([arena[p * P:(p + 1) * P] for p in tb.page_alloc[:om.NP].astype(np.int64)])


def tiled(m, scope=0):
    m.tile_rekey = True
    m.tile_scope = scope
    return m


@pytest.mark.parametrize("scope", [0, 1])
def test_tables_at_every_epoch_equal_the_oracle(cloak_lib, scope):
    # (small tensors on 4-tile pages: per-tensor scope takes thousands of
    # draws to meet the no-succession invariant; this model stays under the cap)
    m = tiled(synth.small_decoder(2, synth.DT_BF16), scope)
    om = O.OracleModel(m)
    cm = cloak_lib.CloakModel(m)
    for e in (0, 1, 2, 7):
        cm.keygen(0x9E, e)
        tb = O.keygen(om, 0x9E, e)
        for which, ref in ((cloak_lib.TAB_TILE_PERM, tb.tile_perm), (cloak_lib.TAB_PAGE_ALLOC, tb.page_alloc),
                           (cloak_lib.TAB_TILE_SLOT, tb.tile_slot), (cloak_lib.TAB_LAYER_PERM, tb.layer_perm)):
            assert np.array_equal(cm.table(which), ref), (e, which)
    cm.close()


@pytest.mark.parametrize("in_place", [False, True])
@pytest.mark.parametrize("mk", [
    synth.mlp2,
    lambda: synth.small_decoder(2, synth.DT_BF16),
    lambda: synth.small_decoder(3, synth.DT_E4M3, page_bytes=2 * 128 * 128, spare_pages=7),
    lambda: synth.small_decoder(2, synth.DT_F32, spare_pages=0),
])
def test_tile_rekey_equals_fresh_shuffle(cloak_lib, mk, in_place, monkeypatch):
    """Out of place through a temporary buffer, and in place through the
    planner and the staging pages (CLOAK_TILE_REKEY_IN_PLACE=1)."""
    if in_place:
        monkeypatch.setenv("CLOAK_TILE_REKEY_IN_PLACE", "1")
    m = tiled(mk())
    key = 0xABCDEF
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, epoch=0, twin=False)
    runs = m.dtype != synth.DT_F32 or m.tile_r == 64
    xs = {t: x_device(m, synth.activations_host(3, tt.k, seed=50 + t)) for t, tt in enumerate(m.tensors) if runs}
    y0 = {t: cm.linear(t, xs[t], out_dtype=cloak_lib.OUT_F32).cpu() for t in xs}
    tb_prev, arena = tb0, arena0.copy()
    for e in (1, 2, 5):
        cm.rekey(key, e)
        torch.cuda.synchronize()
        tbe = O.keygen(om, key, e)
        assert np.array_equal(cm.table(cloak_lib.TAB_TILE_SLOT), tbe.tile_slot), e
        fresh, _ = O.shuffle_model(om, tbe, Ws)
        got = cm.arena_bytes(0).cpu().numpy()
        assert np.array_equal(mapped(got, tbe, om), mapped(fresh, tbe, om)), e
        O.rekey_tiles(om, tb_prev, tbe, arena)
        assert np.array_equal(mapped(got, tbe, om), mapped(arena, tbe, om)), e
        tb_prev = tbe
        for t in xs:
            assert torch.equal(cm.linear(t, xs[t], out_dtype=cloak_lib.OUT_F32).cpu(), y0[t]), (e, t)
    before = cm.arena_bytes(0).cpu().numpy()
    cm.rekey(key, 5)  # the same epoch: nothing moves
    torch.cuda.synchronize()
    assert np.array_equal(cm.arena_bytes(0).cpu().numpy(), before)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with pytest.raises(cloak_lib.CloakError):
        cm.rekey_begin(key, 6, s1)  # tile-level re-keys are synchronous
    assert cm.device_status() == 0
    cm.close()


@pytest.mark.parametrize("in_place", [False, True])
def test_tile_rekey_full_size_layer(cloak_lib, in_place, monkeypatch):
    """One 7B-class layer (12,352 tiles over 193 pages + 64 spare): every
    tile moved, bit for bit the oracle's tile re-key, by either path."""
    if in_place:
        monkeypatch.setenv("CLOAK_TILE_REKEY_IN_PLACE", "1")
    m = tiled(synth.llama7b_layer(1))
    key = 0x1234
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, twin=False)
    cm.rekey(key, 1)
    torch.cuda.synchronize()
    tb1 = O.keygen(om, key, 1)
    O.rekey_tiles(om, tb0, tb1, arena0)
    got = cm.arena_bytes(0).cpu().numpy()
    assert np.array_equal(mapped(got, tb1, om), mapped(arena0, tb1, om))
    moved = np.sum(tb0.tile_slot != tb1.tile_slot)
    assert moved > 0.9 * om.G
    assert cm.device_status() == 0
    cm.close()


def test_tile_rekey_with_the_vmm_view(cloak_lib):
    m = tiled(synth.small_decoder(2, synth.DT_BF16, d_model=1024, n_heads=8, n_kv_heads=2, d_ff=1424,
                                  head_dim=128, spare_pages=4, page_bytes=2 << 20))
    key = 0x44
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, twin=False, vmm=True)
    x = x_device(m, synth.activations_host(2, m.tensors[3].k, seed=8))
    y0 = cm.linear(3, x, out_dtype=cloak_lib.OUT_F32, vmm=True).cpu()
    cm.rekey(key, 1)
    tb1 = O.keygen(om, key, 1)
    fresh, _ = O.shuffle_model(om, tb1, Ws)
    assert np.array_equal(cm.arena_bytes(2).cpu().numpy(), mapped(fresh, tb1, om))
    assert torch.equal(cm.linear(3, x, out_dtype=cloak_lib.OUT_F32, vmm=True).cpu(), y0)
    cm.close()


def test_server_with_tile_rekeys(cloak_lib):
    """Serving with tile-level re-keys (between steps) gives the tokens of
    serving without re-keys."""
    def mk(tile):
        m = synth.small_decoder(2, synth.DT_BF16, d_model=512, n_heads=4, n_kv_heads=2, d_ff=384,
                                head_dim=128, spare_pages=3)
        m = synth.with_lm_head(m, 1000)
        m.tile_rekey = tile
        return m
    Ws = synth.weights_host(mk(False), seed=0, std=0.05)
    work = [(0.01 * i, np.random.default_rng(60 + i).integers(0, 1000, 20 + 5 * i).astype(np.int32), 3 + i % 3)
            for i in range(6)]
    outs = []
    for tile, period in ((False, None), (True, 0.02)):
        sm = serve.ServedModel(mk(tile), kv_blocks=128, max_blocks=16, weights=Ws)
        srv = serve.Server(sm, max_running=4, token_budget=64, rekey_period=period)
        done, wall = srv.run(work)
        outs.append({r.rid: r.out for r in done})
        if tile:
            assert len(srv.rekeys) >= 1 and all(r["mode"] == "between_steps" for r in srv.rekeys)
            tb = O.keygen(O.OracleModel(sm.model), sm.key, sm.epoch)
            assert np.array_equal(sm.cm.table(cloak_lib.TAB_TILE_SLOT), tb.tile_slot)
        assert sm.cm.device_status() == 0
        sm.close()
    assert outs[0] == outs[1]
