"""Property-based checks of the oracle's layout over random model shapes
(tensor sizes with ragged tiles, tile and page sizes, spare pages, scopes,
permutation groups on one or two axes): the tables are permutations, every
tile has its own slot on a mapped page, no physically adjacent slots hold
logically consecutive tiles, and unshuffle undoes shuffle bit for bit."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402
from paper_2606_18400_gb300 import synth  # noqa: E402


@st.composite
def models(draw):
    tile = draw(st.sampled_from([64, 128]))
    dtype = synth.DT_F32 if tile == 64 else synth.DT_BF16
    es = 4 if dtype == synth.DT_F32 else 2
    m = synth.Model(name="prop", dtype=dtype, tile_r=tile, tile_c=tile,
                    page_bytes=tile * tile * es * draw(st.sampled_from([1, 2, 4])),
                    spare_pages=draw(st.integers(0, 3)), tile_scope=draw(st.integers(0, 1)))
    layers = draw(st.integers(1, 3))
    unit = draw(st.sampled_from([1, 16]))
    for l in range(layers):
        n_units = draw(st.integers(2, 20))
        hid = n_units * unit                      # permuted hidden dimension
        d = draw(st.integers(1, 3)) * 16 + draw(st.sampled_from([0, tile]))  # ragged or whole tiles
        g = len(m.groups)
        m.groups.append(synth.Group(n_units, unit))
        m.tensors.append(synth.Tensor(hid, d, l, synth.K_W1, g, 0))   # producer: rows permuted
        m.tensors.append(synth.Tensor(d, hid, l, synth.K_W2, g, 1))   # consumer: columns permuted
    if draw(st.booleans()):                       # a second group on the other axis of every tensor
        d_all = {t.k if t.perm_axis == 0 else t.n for t in m.tensors}
        if len(d_all) == 1:
            g2 = len(m.groups)
            m.groups.append(synth.Group(d_all.pop(), 1))
            for t in m.tensors:
                t.perm_group2 = g2
    return m


@settings(max_examples=40, deadline=None)
@given(models(), st.integers(0, 2**64 - 1), st.integers(0, 3))
def test_layout_properties(m, key, epoch):
    om = O.OracleModel(m)
    try:
        tb = O.keygen(om, key, epoch)
    except RuntimeError:
        return  # the no-succession invariant unreachable within the draw cap (tiny pages)
    perm = lambda a, n: len(a) == n and np.array_equal(np.sort(np.asarray(a, np.int64)), np.arange(n))
    assert perm(tb.tile_perm, om.G) and perm(tb.page_alloc, om.NPS) and perm(tb.layer_perm[:om.L], om.L)
    for g, gr in enumerate(m.groups):
        assert perm(O.group_perm(om, tb, g), gr.n_units)
    slots = tb.tile_slot.astype(np.int64)
    assert len(np.unique(slots)) == om.G
    assert set(np.unique(slots // om.tpp)) <= set(tb.page_alloc[:om.NP].tolist())
    # no physically adjacent slots with logically consecutive tiles
    where = -np.ones(om.NPS * om.tpp, np.int64)
    where[slots] = np.arange(om.G)
    a, b = where[:-1], where[1:]
    assert not np.any((a >= 0) & (b == a + 1))
    Ws = synth.weights_host(m, seed=key % 1000)
    arena, _ = O.shuffle_model(om, tb, Ws)
    for t, W in enumerate(Ws):
        u = O.unshuffle(om, tb, t, arena)
        ref = W if m.dtype == synth.DT_F32 else O.bf16_bits(W)
        assert np.array_equal(u, ref), t
