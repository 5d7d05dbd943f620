"""Pins of oracle functions that the property tests leave open: the stream
seeds and the tables they drive, the RoPE frequency schedule and pairing,
and the multi-token forward of the serving reference. Each is compared with
a restatement written here from the reading it follows (pure Python integers
and floats, scalar loops), sharing no code with the oracle beyond the
SplitMix64 output function, which the published known answers pin."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle as O
from paper_2606_18400_gb300 import synth

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


# ------------------------------------------------------------ stream seeds

def _mix(z):
    """The SplitMix64 finaliser of z: the generator's next output from state
    z - gamma (the generator adds gamma, then finalises; its outputs are pinned
    by the known-answer file)."""
    s = C.c_uint64((z - GAMMA) & M64)
    return O.lib().orc_next(C.byref(s))


def _seed(key, tag, epoch, idx):
    """Stream separation (tags 1 layer order, 2 permutation group, 3 tile
    permutation, 4 page map): mix(key ^ mix(tag << 56 ^ epoch << 32 ^ idx))."""
    lane = ((tag << 56) ^ (epoch << 32) ^ idx) & M64
    return _mix((key ^ _mix(lane)) & M64)


def test_stream_seed_is_the_two_round_mix_of_key_and_lane():
    L = O.lib()
    keys = [0, 1, 0x1234, 0x5151, 0xDEADBEEFCAFEF00D, M64]
    for key in keys:
        for tag in (1, 2, 3, 4, 255):
            for epoch in (0, 1, 7, 0xFFFFFF, 0xFFFFFFFF):
                for idx in (0, 1, 3, 1000, 0xFFFFFFFF):
                    assert L.orc_stream_seed(key, tag, epoch, idx) == _seed(key, tag, epoch, idx), \
                        (key, tag, epoch, idx)


def test_stream_seed_restatement_tells_the_plausible_mistakes_apart():
    """The restatement is not symmetric in what a wrong seed would swap: the
    inner and outer rounds exchanged, or the tag and epoch fields exchanged,
    give other seeds."""
    key, tag, epoch, idx = 0x1234, 3, 5, 9
    good = _seed(key, tag, epoch, idx)
    lane = (tag << 56) ^ (epoch << 32) ^ idx
    assert good != _mix(_mix((key ^ lane) & M64))
    assert good != _seed(key, epoch, tag, idx)
    assert good != _mix((key ^ lane) & M64)


# --------------------------------------------- tables from a Python shuffle

class _Stream:
    def __init__(self, seed):
        self.s = C.c_uint64(seed)

    def next(self):
        return O.lib().orc_next(C.byref(self.s))

    def bounded(self, n):
        """Unbiased draw in [0, n): the high half of x*n, redrawn while the low
        half is below 2^64 mod n (Lemire 2019)."""
        x = self.next()
        m = x * n
        if (m & M64) < n:
            t = (1 << 64) % n
            while (m & M64) < t:
                x = self.next()
                m = x * n
        return m >> 64

    def fisher_yates(self, n):
        a = list(range(n))
        for i in range(n - 1, 0, -1):
            j = self.bounded(i + 1)
            a[i], a[j] = a[j], a[i]
        return a


def _three_tensor_model():
    """Three tensors over two layers (a producer/consumer pair sharing one
    group, and an unpermuted one), ragged edges, small pages."""
    m = synth.Model(name="three", dtype=synth.DT_BF16, tile_r=128, tile_c=128,
                    page_bytes=4 * 128 * 128 * 2, spare_pages=3)
    m.groups = [synth.Group(n_units=300, unit=1)]
    m.tensors = [synth.Tensor(300, 256, 0, synth.K_GATE, 0, 0),
                 synth.Tensor(256, 300, 1, synth.K_DOWN, 0, 1),
                 synth.Tensor(200, 384, 1, synth.K_Q)]
    return m


@pytest.mark.parametrize("key", [0x1234, 0x5151, 0xA5A5A5A5A5A5])
@pytest.mark.parametrize("epoch", [0, 3])
def test_tables_are_python_fisher_yates_on_the_keyed_streams(key, epoch):
    """Every table of a 3-tensor model equals Durstenfeld's shuffle driven by
    the pinned generator from its stream seed: the layer order (tag 1), the
    group (tag 2, index = group), the tile permutation (tag 3; its draw count
    taken from the oracle, the stream continued between draws) and the page
    map (tag 4, the epoch's stream); the gather table composes them as
    slot = page_map[v / tpp] * tpp + v % tpp with v the tile's virtual slot."""
    m = _three_tensor_model()
    om = O.OracleModel(m)
    tb = O.keygen(om, key, epoch)
    assert list(tb.layer_perm[:om.L]) == _Stream(_seed(key, 1, 0, 0)).fisher_yates(om.L)
    assert list(tb.group_perm[:300]) == _Stream(_seed(key, 2, 0, 0)).fisher_yates(300)
    s = _Stream(_seed(key, 3, 0, 0))
    for _ in range(tb.tile_draws):
        tp = s.fisher_yates(om.G)
    assert list(tb.tile_perm) == tp
    s = _Stream(_seed(key, 4, epoch, 0))
    for _ in range(tb.page_draws):
        pm = s.fisher_yates(om.NPS)
    assert list(tb.page_alloc[:om.NPS]) == pm
    inv = {g: v for v, g in enumerate(tp)}
    slots = [pm[inv[g] // om.tpp] * om.tpp + inv[g] % om.tpp for g in range(om.G)]
    assert list(tb.tile_slot) == slots


# --------------------------------------------------------------------- RoPE

THETA = 10000.0


def _angle(pos, i):
    """LLaMA rotary frequency of pair i of a 128-dim head: theta^(-2i/128)."""
    return pos * THETA ** (-(2.0 * i) / 128.0)


@pytest.mark.parametrize("pos", [1, 2, 17, 300, 4095])
def test_rope_rotates_every_pair_by_its_closed_form_angle(pos):
    """One-hot inputs, element by element against math.cos/math.sin of
    pos * 10000^(-i/64): the first half of a pair (index i) goes to
    (cos, sin) at (i, i + 64), the second half (index i + 64) to (-sin, cos)."""
    for i in range(64):
        a = _angle(pos, i)
        x = np.zeros((1, 2, 128))
        x[0, 0, i] = 1.0
        x[0, 1, i + 64] = 1.0
        y = O.rope_f64(x, [pos])
        want0 = np.zeros(128)
        want0[i], want0[i + 64] = math.cos(a), math.sin(a)
        want1 = np.zeros(128)
        want1[i], want1[i + 64] = -math.sin(a), math.cos(a)
        assert np.allclose(y[0, 0], want0, rtol=0, atol=1e-12), (pos, i)
        assert np.allclose(y[0, 1], want1, rtol=0, atol=1e-12), (pos, i)


def test_rope_known_frequencies():
    """Pair 32 turns by pos/100 (10000^(-1/2)); pair 16 by pos/10; pair 48
    by pos/1000: the base and the exponent of the schedule."""
    for i, f in ((16, 0.1), (32, 0.01), (48, 0.001)):
        x = np.zeros((1, 1, 128))
        x[0, 0, i] = 1.0
        y = O.rope_f64(x, [50])
        assert math.isclose(y[0, 0, i], math.cos(50 * f), abs_tol=1e-12)
        assert math.isclose(y[0, 0, i + 64], math.sin(50 * f), abs_tol=1e-12)


def test_rope_pairs_i_with_i_plus_64_not_neighbours():
    """A vector with its only entries in pair 5 keeps every other index at
    zero (an interleaved pairing would move mass into index 11)."""
    x = np.zeros((1, 1, 128))
    x[0, 0, 5], x[0, 0, 69] = 0.3, -1.7
    y = O.rope_f64(x, [9])[0, 0]
    others = np.delete(y, [5, 69])
    assert np.all(others == 0.0)
    a = _angle(9, 5)
    assert math.isclose(y[5], 0.3 * math.cos(a) + 1.7 * math.sin(a), abs_tol=1e-12)
    assert math.isclose(y[69], -1.7 * math.cos(a) + 0.3 * math.sin(a), abs_tol=1e-12)


# --------------------------------------------------- multi-token forward

def _forward_brute(model, W, emb, tokens, eps=1e-5):
    """The LLaMA-style forward written with scalar loops over positions,
    heads and keys: unit-gain RMSNorm, q/k/v, rotary pairs (i, i + 64) at
    angle pos * 10000^(-i/64), causal attention softmax(q.k / sqrt(128)) v
    with query head j reading KV head j // (H / H_kv), output projection and
    residual, RMSNorm, SwiGLU (silu(g) u) and residual; final RMSNorm and the
    output projection."""
    H, Hkv, hd = model.n_heads, model.n_kv_heads, 128
    grp = H // Hkv
    T = len(tokens)
    kinds = {}
    for i, t in enumerate(model.tensors):
        kinds.setdefault(t.layer, {})[t.kind] = i
    lm = [i for i, t in enumerate(model.tensors) if t.kind == synth.K_LMHEAD][0]

    def rms(v):
        return v / math.sqrt(sum(float(e) * float(e) for e in v) / len(v) + eps)

    def rot(v, pos):
        out = list(v)
        for i in range(64):
            a = _angle(pos, i)
            c, s = math.cos(a), math.sin(a)
            out[i] = v[i] * c - v[i + 64] * s
            out[i + 64] = v[i + 64] * c + v[i] * s
        return out

    h = [np.array(emb[tok], np.float64) for tok in tokens]
    for l in range(model.num_layers - 1):
        ts = kinds[l]
        x = [rms(v) for v in h]
        q = [[rot(list(W[ts[synth.K_Q]][j * hd:(j + 1) * hd] @ x[t]), t) for j in range(H)] for t in range(T)]
        k = [[rot(list(W[ts[synth.K_K]][j * hd:(j + 1) * hd] @ x[t]), t) for j in range(Hkv)] for t in range(T)]
        v = [[W[ts[synth.K_V]][j * hd:(j + 1) * hd] @ x[t] for j in range(Hkv)] for t in range(T)]
        for t in range(T):
            att = np.zeros(H * hd)
            for j in range(H):
                kv = j // grp
                sc = [sum(q[t][j][d] * k[u][kv][d] for d in range(hd)) / math.sqrt(hd) for u in range(t + 1)]
                mx = max(sc)
                e = [math.exp(z - mx) for z in sc]
                tot = sum(e)
                for u in range(t + 1):
                    att[j * hd:(j + 1) * hd] += (e[u] / tot) * v[u][kv]
            h[t] = h[t] + W[ts[synth.K_O]] @ att
        for t in range(T):
            xn = rms(h[t])
            g = W[ts[synth.K_GATE]] @ xn
            u = W[ts[synth.K_UP]] @ xn
            act = np.array([gi / (1.0 + math.exp(-gi)) * ui for gi, ui in zip(g, u)])
            h[t] = h[t] + W[ts[synth.K_DOWN]] @ act
    return np.stack([W[lm] @ rms(v) for v in h])


def _served(layers=2):
    m = synth.small_decoder(layers, synth.DT_BF16, d_model=256, n_heads=4, n_kv_heads=2, d_ff=192,
                            head_dim=128)
    return synth.with_lm_head(m, 64)


@pytest.mark.parametrize("T", [2, 7, 33])
def test_forward_equals_the_scalar_loop_forward(T):
    m = _served()
    W = [w.astype(np.float64) for w in synth.weights_host(m, seed=11, std=0.05)]
    emb = synth.embedding_host(64, 256, seed=3).astype(np.float64)
    toks = list(np.random.default_rng(T).integers(0, 64, T))
    got = O.transformer_logits_f64(m, W, emb, toks)
    ref = _forward_brute(m, W, emb, toks)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_forward_with_a_wide_score_spread():
    """Scores of tens of units: the softmax is far from uniform, so a scale
    other than 1/sqrt(128) (or none) changes the logits by far more than
    rounding."""
    m = _served(1)
    W = [w.astype(np.float64) for w in synth.weights_host(m, seed=12, std=0.05)]
    for t, tt in enumerate(m.tensors):
        if tt.kind in (synth.K_Q, synth.K_K):
            W[t] = W[t] * 12.0
    emb = synth.embedding_host(64, 256, seed=4).astype(np.float64)
    toks = [5, 9, 13, 2, 63, 40, 41, 7, 0, 22, 31]
    got = O.transformer_logits_f64(m, W, emb, toks)
    ref = _forward_brute(m, W, emb, toks)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    # the spread is real: scores without the 1/sqrt(d) scale give other logits
    Wn = [w.copy() for w in W]
    for t, tt in enumerate(m.tensors):
        if tt.kind == synth.K_Q:
            Wn[t] = Wn[t] * math.sqrt(128)
    far = O.transformer_logits_f64(m, Wn, emb, toks)
    assert np.abs(far - got).max() > 1e-3 * np.abs(got).max()


# ------------------------------------------- stack step with BF16 operands

def _bf16(x):
    """x rounded to FP32, then to BF16 by keeping the upper half of the FP32
    pattern with the lower half rounded to nearest, ties to an even upper
    half (finite inputs)."""
    import struct
    u = struct.unpack("<I", struct.pack("<f", float(x)))[0]
    lo, hi = u & 0xFFFF, u >> 16
    if lo > 0x8000 or (lo == 0x8000 and (hi & 1)):
        hi += 1
    return struct.unpack("<f", struct.pack("<I", (hi & 0xFFFF) << 16))[0]


def test_stack_step_with_bf16_operands_equals_a_scalar_restatement():
    """Two layers, two tokens: every linear input rounded to BF16 (R(h) into
    v, gate, up; v rounded after its row scale; the SwiGLU product rounded
    before the down projection), the residual kept in full precision."""
    m = synth.small_decoder(2, synth.DT_BF16, d_model=256, n_heads=4, n_kv_heads=2, d_ff=192,
                            head_dim=128)
    W = [w.astype(np.float64) for w in synth.weights_host(m, seed=4, std=0.05)]
    h0 = synth.activations_host(2, 256, seed=6).astype(np.float64)
    got = O.stack_decode_f64(m, W, h0, bf16_operands=True)
    R = np.vectorize(_bf16)
    h = h0.copy()
    for l in range(2):
        q, k, v, o, g, u, d = (W[7 * l + i] for i in range(7))
        for t in range(2):
            r = 1.0 / math.sqrt(sum(e * e for e in h[t]) / 256 + 1e-5)
            vv = R((v @ R(h[t])) * r)
            a = np.concatenate([vv[(j // 2) * 128:(j // 2 + 1) * 128] for j in range(4)])
            h[t] = h[t] + o @ a
            r = 1.0 / math.sqrt(sum(e * e for e in h[t]) / 256 + 1e-5)
            gg, uu = (g @ R(h[t])) * r, (u @ R(h[t])) * r
            act = R(np.array([x / (1.0 + math.exp(-x)) for x in gg]) * uu)
            h[t] = h[t] + d @ act
    assert np.allclose(got, h, rtol=0, atol=1e-12 * np.abs(h).max())
    plain = O.stack_decode_f64(m, W, h0)
    diff = O.relative_error(got, plain)
    assert 1e-5 < diff < 1e-2  # the roundings are there, and of BF16 size
