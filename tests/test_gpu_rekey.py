"""GPU re-key: after rekey(key, e+1) every mapped page of the arena equals a
fresh keygen(key, e+1) + shuffle, bit for bit; linear results are unchanged."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_18400_gb300 import synth
from helpers import place_both, x_device

pytestmark = pytest.mark.gpu


def mapped_pages(arena, tb, om):
    P = om.model.page_bytes
    return np.concatenate([arena[p * P:(p + 1) * P] for p in tb.page_alloc[:om.NP].astype(np.int64)])


@pytest.mark.parametrize("mk", [
    synth.mlp2,                                                # one tile per page, no spare pages
    lambda: synth.small_decoder(2, synth.DT_BF16),
    lambda: synth.small_decoder(3, synth.DT_E4M3, page_bytes=2 * 128 * 128, spare_pages=7),
    lambda: synth.small_decoder(2, synth.DT_F32, spare_pages=0),
])
def test_rekey_equals_fresh_shuffle(cloak_lib, mk):
    m = mk()
    key = 0xABCDEF
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, epoch=0, twin=False)
    for e in (1, 2, 5):
        cm.rekey(key, e)
        torch.cuda.synchronize()
        tbe = O.keygen(om, key, e)
        fresh, _ = O.shuffle_model(om, tbe, Ws)
        got = cm.arena_bytes(0).cpu().numpy()
        assert np.array_equal(mapped_pages(got, tbe, om), mapped_pages(fresh, tbe, om)), e
        assert np.array_equal(cm.table(cloak_lib.TAB_TILE_SLOT), tbe.tile_slot)
        assert np.array_equal(cm.table(cloak_lib.TAB_PAGE_ALLOC), tbe.page_alloc)
    # rekey to the same epoch moves nothing
    before = cm.arena_bytes(0).cpu().numpy()
    cm.rekey(key, 5)
    torch.cuda.synchronize()
    assert np.array_equal(cm.arena_bytes(0).cpu().numpy(), before)
    assert cm.device_status() == 0
    cm.close()


def test_rekey_keeps_linear_results(cloak_lib):
    m = synth.small_decoder(2, synth.DT_BF16)
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=11, twin=True)
    x = x_device(m, synth.activations_host(8, m.tensors[4].k, seed=3))
    y0 = cm.linear(4, x, out_dtype=cloak_lib.OUT_F32).cpu()
    cm.rekey(11, 1)
    y1 = cm.linear(4, x, out_dtype=cloak_lib.OUT_F32).cpu()
    assert torch.equal(y0, y1)
    with pytest.raises(cloak_lib.CloakError):
        cm.rekey(12, 2)  # another key is refused
    cm.close()


def test_rekey_full_size_layer(cloak_lib):
    """One 7B-class layer (193 pages of 2 MiB + 64 spare): bit-exact."""
    m = synth.llama7b_layer(1)
    key = 0x1234
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, twin=False)
    cm.rekey(key, 1)
    torch.cuda.synchronize()
    tb1 = O.keygen(om, key, 1)
    O.rekey(om, tb0, tb1, arena0)
    got = cm.arena_bytes(0).cpu().numpy()
    assert np.array_equal(mapped_pages(got, tb1, om), mapped_pages(arena0, tb1, om))
    cm.close()


def _concurrent_rekey(cloak_lib, cm, m, key, new_epoch, xs, y_ref):
    """Drive a concurrent re-key: at every step boundary enqueue a "step" (one
    linear per tensor) on the serving stream, then advance. Each step's
    outputs must equal the pre-re-key outputs bit for bit. Returns the number
    of steps the re-key spanned."""
    serve, side = torch.cuda.Stream(), torch.cuda.Stream()
    cm.rekey_begin(key, new_epoch, side)
    with pytest.raises(cloak_lib.CloakError):
        cm.rekey(key, new_epoch + 1)          # one re-key at a time
    with pytest.raises(cloak_lib.CloakError):
        cm.rekey_advance(serve, serve)        # the two streams must differ
    steps, done = 0, False
    while not done:
        with torch.cuda.stream(serve):
            ys = {t: cm.linear(t, xs[t], out_dtype=cloak_lib.OUT_F32) for t in xs}
        done = cm.rekey_advance(serve, side)
        serve.synchronize()
        for t in xs:
            assert torch.equal(ys[t].cpu(), y_ref[t]), (steps, t)
        steps += 1
        assert steps < 100000
    torch.cuda.synchronize()
    return steps


@pytest.mark.parametrize("mk", [
    synth.mlp2,
    lambda: synth.small_decoder(2, synth.DT_BF16),
    lambda: synth.small_decoder(3, synth.DT_E4M3, page_bytes=2 * 128 * 128, spare_pages=7),
    lambda: synth.small_decoder(2, synth.DT_F32, spare_pages=0),
    lambda: synth.llama7b_layer(1),
])
def test_concurrent_rekey_serves_throughout_and_ends_at_fresh_shuffle(cloak_lib, mk):
    """Every step between the waves computes exactly what it computed before
    the re-key; at the end arena and tables equal keygen(key, e+1) + shuffle."""
    m = mk()
    key = 0x5EED
    cm, om, tb0, arena0, scales, Ws = place_both(cloak_lib, m, key=key, epoch=0, twin=False)
    # (an FP32 model with 128x128 tiles has no linear kernel: layout only)
    runs = m.dtype != synth.DT_F32 or m.tile_r == 64
    xs = {t: x_device(m, synth.activations_host(4, tt.k, seed=40 + t))
          for t, tt in enumerate(m.tensors) if runs}
    y_ref = {t: cm.linear(t, xs[t], out_dtype=cloak_lib.OUT_F32).cpu() for t in xs}
    for e in (1, 2):
        steps = _concurrent_rekey(cloak_lib, cm, m, key, e, xs, y_ref)
        assert steps >= 1
        tbe = O.keygen(om, key, e)
        assert np.array_equal(cm.table(cloak_lib.TAB_TILE_SLOT), tbe.tile_slot), e
        assert np.array_equal(cm.table(cloak_lib.TAB_PAGE_ALLOC), tbe.page_alloc), e
        got = cm.arena_bytes(0).cpu().numpy()
        O.rekey(om, tb0, tbe, arena0)
        assert np.array_equal(mapped_pages(got, tbe, om), mapped_pages(arena0, tbe, om)), e
        tb0 = tbe
    # a synchronous re-key after a concurrent one continues from its state
    cm.rekey(key, 3)
    torch.cuda.synchronize()
    tb3 = O.keygen(om, key, 3)
    assert np.array_equal(cm.table(cloak_lib.TAB_TILE_SLOT), tb3.tile_slot)
    assert cm.device_status() == 0
    cm.close()


def test_rekey_advance_without_a_job_is_refused(cloak_lib):
    m = synth.mlp2()
    cm, om, tb, arena, scales, Ws = place_both(cloak_lib, m, key=3, twin=False)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with pytest.raises(cloak_lib.CloakError):
        cm.rekey_advance(s1, s2)
    cm.close()
