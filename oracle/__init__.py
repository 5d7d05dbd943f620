"""CPU oracle for the cloaked linear layer (CloakLM, arxiv 2606.18400).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA library under ``paper_2606_18400_gb300/``; the two meet only in
the seeded inputs of ``paper_2606_18400_gb300.synth``.

Layout (tables, shuffle, unshuffle, re-key, number formats) is plain C in
``cloak_oracle.c``, loaded through ctypes. The products are plain FP64 NumPy
matrix products on the logical, unshuffled weights: the method leaves the
function a network computes unchanged (Abstract: authorised execution sees a
valid view), so the reference result of a cloaked linear, MLP or layer is the
textbook product on the logical weights. The MoE FFN (the paper's MoE model,
Section 5) is written out the same way: softmax top-k routing over the
router's logits, renormalised weights, the selected experts' gated MLPs.

Pins (tests/test_oracle_*.py): the PRNG's published known answers, the
bounded draw's exact arithmetic, tables being permutations meeting the
layout invariants, shuffle/unshuffle round trips and independent NumPy
restatements of the stored matrices (one or two permuted axes), fresh
shuffles equal to re-keys (pages or tiles), compensated networks computing
the plain network's function (brute force on integer MLPs, a GQA layer, the
stack and full model under the residual permutation), the BF16/E4M3 codecs
against their format definitions, and the MoE routing's closed forms
(identical experts, top-1, the all-experts softmax mixture, relabelling,
ties).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cloak_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (no -ffast-math: FP32 division and
    comparisons must be IEEE)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Tensor(C.Structure):
    _fields_ = [(f, C.c_int32) for f in ("n", "k", "layer", "kind", "perm_group", "perm_axis", "perm_group2")]


class _Group(C.Structure):
    _fields_ = [(f, C.c_int32) for f in ("n_units", "unit", "parent", "ratio")]


class _Model(C.Structure):
    _fields_ = [("num_tensors", C.c_int32), ("num_groups", C.c_int32),
                ("tensors", C.POINTER(_Tensor)), ("groups", C.POINTER(_Group)),
                ("dtype", C.c_int32), ("tile_r", C.c_int32), ("tile_c", C.c_int32),
                ("spare_pages", C.c_int32), ("tile_scope", C.c_int32), ("tile_rekey", C.c_int32),
                ("page_bytes", C.c_int64)]


_u32p = C.POINTER(C.c_uint32)


class _Tables(C.Structure):
    _fields_ = [("layer_perm", _u32p), ("group_perm", _u32p), ("tensor_base", _u32p),
                ("tile_perm", _u32p), ("page_alloc", _u32p), ("tile_slot", _u32p),
                ("tile_draws", C.c_uint32), ("page_draws", C.c_uint32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp = C.c_void_p
        L.orc_mix.restype = C.c_uint64
        L.orc_mix.argtypes = [C.c_uint64]
        L.orc_next.restype = C.c_uint64
        L.orc_next.argtypes = [C.POINTER(C.c_uint64)]
        L.orc_bounded.restype = C.c_uint64
        L.orc_bounded.argtypes = [C.POINTER(C.c_uint64), C.c_uint64]
        L.orc_stream_seed.restype = C.c_uint64
        L.orc_stream_seed.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_fisher_yates.argtypes = [C.POINTER(C.c_uint64), C.c_uint32, vp]
        L.orc_geometry.argtypes = [C.POINTER(_Model), vp]
        L.orc_keygen.argtypes = [C.POINTER(_Model), C.c_uint64, C.c_uint32, C.POINTER(_Tables)]
        L.orc_shuffle_tensor.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.c_int, vp, vp, vp]
        L.orc_unshuffle_tensor.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.c_int, vp, vp]
        L.orc_stored_f64.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.c_int, vp, vp, vp]
        L.orc_stored_codes.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.c_int, vp, vp, vp]
        L.orc_axis_maps.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.c_int, vp, vp]
        L.orc_rekey.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.POINTER(_Tables), vp, vp]
        L.orc_rekey_tiles.argtypes = [C.POINTER(_Model), C.POINTER(_Tables), C.POINTER(_Tables), vp, vp]
        L.orc_bf16_encode.restype = C.c_uint16
        L.orc_bf16_encode.argtypes = [C.c_float]
        L.orc_bf16_decode.restype = C.c_float
        L.orc_bf16_decode.argtypes = [C.c_uint16]
        L.orc_e4m3_encode.restype = C.c_uint8
        L.orc_e4m3_encode.argtypes = [C.c_float]
        L.orc_e4m3_decode.restype = C.c_double
        L.orc_e4m3_decode.argtypes = [C.c_uint8]
        L.orc_bf16_encode_array.argtypes = [vp, vp, C.c_int64]
        L.orc_e4m3_encode_array.argtypes = [vp, vp, C.c_int64]
        L.orc_e4m3_decode_array.argtypes = [vp, vp, C.c_int64]
        L.orc_quant_rows_e4m3.argtypes = [vp, C.c_int64, C.c_int64, vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class OracleModel:
    """ctypes view of a ``synth.Model`` (kept alive with its arrays)."""

    def __init__(self, model):
        self.model = model
        T, Gn = len(model.tensors), len(model.groups)
        self._t = (_Tensor * T)(*[_Tensor(t.n, t.k, t.layer, t.kind, t.perm_group, t.perm_axis,
                                          getattr(t, "perm_group2", -1)) for t in model.tensors])
        self._g = (_Group * max(Gn, 1))(*[_Group(g.n_units, g.unit, g.parent, g.ratio)
                                          for g in model.groups])
        self.c = _Model(T, Gn, self._t, self._g, model.dtype, model.tile_r, model.tile_c,
                        model.spare_pages, model.tile_scope, int(getattr(model, "tile_rekey", False)),
                        model.page_bytes)
        geo = np.zeros(8, np.int64)
        rc = lib().orc_geometry(C.byref(self.c), _ptr(geo))
        if rc:
            raise ValueError(f"invalid model descriptor ({rc})")
        (self.L, self.G, self.tpp, self.NP, self.NPS, self.U, self.tile_bytes,
         self.esize) = (int(v) for v in geo)
        self.arena_bytes = self.NPS * model.page_bytes


@dataclass
class Tables:
    layer_perm: np.ndarray
    group_perm: np.ndarray
    tensor_base: np.ndarray
    tile_perm: np.ndarray
    page_alloc: np.ndarray
    tile_slot: np.ndarray
    tile_draws: int
    page_draws: int
    _c: object = None

    @property
    def page_map(self):
        return self.page_alloc


def _ctables(om: OracleModel, tb: Tables):
    u = lambda a: a.ctypes.data_as(_u32p)
    return _Tables(u(tb.layer_perm), u(tb.group_perm), u(tb.tensor_base), u(tb.tile_perm),
                   u(tb.page_alloc), u(tb.tile_slot), tb.tile_draws, tb.page_draws)


def keygen(om: OracleModel, key: int, epoch: int) -> Tables:
    """Keyed tables for (key, epoch)."""
    z = lambda n: np.zeros(max(n, 1), np.uint32)
    tb = Tables(z(om.L), z(om.U), z(len(om.model.tensors)), z(om.G), z(om.NPS), z(om.G), 0, 0)
    ct = _ctables(om, tb)
    rc = lib().orc_keygen(C.byref(om.c), C.c_uint64(key & (2**64 - 1)), epoch, C.byref(ct))
    if rc:
        raise RuntimeError(f"orc_keygen failed ({rc})")
    tb.tile_draws, tb.page_draws = ct.tile_draws, ct.page_draws
    tb.page_alloc = tb.page_alloc[:om.NPS]
    return tb


def group_perm(om: OracleModel, tb: Tables, g: int) -> np.ndarray:
    off = sum(gr.n_units for gr in om.model.groups[:g])
    return tb.group_perm[off:off + om.model.groups[g].n_units]


def new_arena(om: OracleModel) -> np.ndarray:
    return np.zeros(om.arena_bytes, np.uint8)


def shuffle(om: OracleModel, tb: Tables, t: int, W: np.ndarray, arena: np.ndarray):
    """Place tensor t's logical FP32 weights W into the arena. Returns the FP8
    per-stored-row scales (or None for FP32/BF16)."""
    W = np.ascontiguousarray(W, np.float32)
    tt = om.model.tensors[t]
    assert W.shape == (tt.n, tt.k)
    sc = np.zeros(tt.n, np.float32)
    ct = _ctables(om, tb)
    rc = lib().orc_shuffle_tensor(C.byref(om.c), C.byref(ct), t, _ptr(W), _ptr(arena), _ptr(sc))
    assert rc == 0
    return sc if om.model.dtype == 2 else None


def shuffle_model(om: OracleModel, tb: Tables, Ws):
    arena = new_arena(om)
    scales = [shuffle(om, tb, t, W, arena) for t, W in enumerate(Ws)]
    return arena, scales


_NP_DT = {0: np.float32, 1: np.uint16, 2: np.uint8}


def unshuffle(om: OracleModel, tb: Tables, t: int, arena: np.ndarray) -> np.ndarray:
    """Logical [n, k] array in the stored dtype (FP32 values, BF16 or E4M3
    bit patterns) read back from the arena."""
    tt = om.model.tensors[t]
    out = np.zeros((tt.n, tt.k), _NP_DT[om.model.dtype])
    ct = _ctables(om, tb)
    assert lib().orc_unshuffle_tensor(C.byref(om.c), C.byref(ct), t, _ptr(arena), _ptr(out)) == 0
    return out


def stored_f64(om: OracleModel, tb: Tables, t: int, arena: np.ndarray, scales=None) -> np.ndarray:
    """The stored (row/column-permuted) matrix as FP64 values."""
    tt = om.model.tensors[t]
    out = np.zeros((tt.n, tt.k), np.float64)
    sc = np.ascontiguousarray(scales if scales is not None else np.ones(tt.n), np.float32)
    ct = _ctables(om, tb)
    assert lib().orc_stored_f64(C.byref(om.c), C.byref(ct), t, _ptr(arena), _ptr(sc), _ptr(out)) == 0
    return out


def stored_codes(om: OracleModel, tb: Tables, t: int, W: np.ndarray):
    """(codes [n, k] in the storage type, in stored order; FP8 row scales or
    None) -- the content the arena holds for tensor t, before tiling."""
    W = np.ascontiguousarray(W, np.float32)
    tt = om.model.tensors[t]
    out = np.zeros((tt.n, tt.k), _NP_DT[om.model.dtype])
    sc = np.zeros(tt.n, np.float32)
    ct = _ctables(om, tb)
    assert lib().orc_stored_codes(C.byref(om.c), C.byref(ct), t, _ptr(W), _ptr(out), _ptr(sc)) == 0
    return out, (sc if om.model.dtype == 2 else None)


def tile_of(om: OracleModel, codes: np.ndarray, nt: int, kt: int) -> np.ndarray:
    """Bytes of tile (nt, kt) cut from a stored matrix (zero-padded)."""
    m = om.model
    blk = np.zeros((m.tile_r, m.tile_c), codes.dtype)
    part = codes[nt * m.tile_r:(nt + 1) * m.tile_r, kt * m.tile_c:(kt + 1) * m.tile_c]
    blk[:part.shape[0], :part.shape[1]] = part
    return blk.reshape(-1).view(np.uint8)


def axis_maps(om: OracleModel, tb: Tables, t: int):
    """(rmap, cmap): stored row r holds logical row rmap[r]; likewise columns."""
    tt = om.model.tensors[t]
    r = np.zeros(tt.n, np.int64)
    c = np.zeros(tt.k, np.int64)
    ct = _ctables(om, tb)
    lib().orc_axis_maps(C.byref(om.c), C.byref(ct), t, _ptr(r), _ptr(c))
    return r, c


def rekey(om: OracleModel, old: Tables, new: Tables, arena: np.ndarray):
    """Move every page from its old physical page to its new one (in place
    on the host buffer; the spare pages of the new map are don't-care)."""
    tmp = np.empty_like(arena)
    assert lib().orc_rekey(C.byref(om.c), C.byref(_ctables(om, old)), C.byref(_ctables(om, new)),
                           _ptr(arena), _ptr(tmp)) == 0


def rekey_tiles(om: OracleModel, old: Tables, new: Tables, arena: np.ndarray):
    """Tile-level re-key (models with tile_rekey): every tile from its old
    slot to its new one, the new map's empty slots zeroed (in place)."""
    tmp = np.empty_like(arena)
    assert lib().orc_rekey_tiles(C.byref(om.c), C.byref(_ctables(om, old)), C.byref(_ctables(om, new)),
                                 _ptr(arena), _ptr(tmp)) == 0


# ------------------------------------------------------------ number formats

def bf16_bits(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros(x.shape, np.uint16)
    lib().orc_bf16_encode_array(_ptr(x), _ptr(out), x.size)
    return out


def bf16_value(bits) -> np.ndarray:
    bits = np.ascontiguousarray(bits, np.uint16)
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def e4m3_bits(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros(x.shape, np.uint8)
    lib().orc_e4m3_encode_array(_ptr(x), _ptr(out), x.size)
    return out


def e4m3_value(codes) -> np.ndarray:
    codes = np.ascontiguousarray(codes, np.uint8)
    out = np.zeros(codes.shape, np.float64)
    lib().orc_e4m3_decode_array(_ptr(codes), _ptr(out), codes.size)
    return out


def quant_rows_e4m3(x):
    """Per-row (per-token) FP8 quantisation: (codes, fp32 scales)."""
    x = np.ascontiguousarray(x, np.float32)
    q = np.zeros(x.shape, np.uint8)
    s = np.zeros(x.shape[0], np.float32)
    lib().orc_quant_rows_e4m3(_ptr(x), x.shape[0], x.shape[1], _ptr(q), _ptr(s))
    return q, s


# ------------------------------------------------------------------ products

def linear_f64(x64: np.ndarray, W64: np.ndarray) -> np.ndarray:
    """y = x W^T in FP64 (the plain definition of a linear layer)."""
    return np.asarray(x64, np.float64) @ np.asarray(W64, np.float64).T


def x_operand(om: OracleModel, x: np.ndarray) -> np.ndarray:
    """The activation operand as the path consumes it, in FP64: FP32 as is,
    BF16 rounded (nearest even), or, for FP8 weights, BF16-rounded then
    quantised per token (scale amax/448) and dequantised."""
    if om.model.dtype == 0:
        return np.asarray(x, np.float32).astype(np.float64)
    xb = bf16_value(bf16_bits(x))
    if om.model.dtype == 1:
        return xb
    # FP8 models take BF16 activations and quantise them per token
    q, s = quant_rows_e4m3(xb.astype(np.float32))
    return e4m3_value(q) * s.astype(np.float64)[:, None]


def cloaked_linear(om: OracleModel, tb: Tables, t: int, arena: np.ndarray, x: np.ndarray,
                   scales=None) -> np.ndarray:
    """Reference output of the cloaked linear of tensor t: the FP64 product of
    the activation operand with the stored matrix read back from the arena."""
    return linear_f64(x_operand(om, x), stored_f64(om, tb, t, arena, scales))


def relative_error(y, ref) -> float:
    """Normwise relative error ||y - ref||_F / ||ref||_F."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(y - ref) / (den if den > 0 else 1.0))


def mlp2_f64(x64, W1, W2, relu=True):
    """y = W2 relu(W1 x): the plain two-layer MLP."""
    h = linear_f64(x64, W1)
    if relu:
        h = np.maximum(h, 0.0)
    return linear_f64(h, W2)


def contiguity(page_alloc: np.ndarray, NP: int) -> float:
    """Fraction of consecutive virtual page pairs backed by consecutive
    physical pages (the virtual-physical contiguity of Table 2)."""
    pm = np.asarray(page_alloc[:NP], np.int64)
    if NP < 2:
        return 1.0
    return float(np.mean(pm[1:] == pm[:-1] + 1))


# ------------------------------------------------------------- layer stack

def silu(g):
    return g / (1.0 + np.exp(-g))


def _bf16_round(x):
    """Each value rounded to BF16 (to FP32, then to nearest even BF16) and
    returned in FP64."""
    return bf16_value(bf16_bits(np.asarray(x, np.float64).astype(np.float32)))


def stack_decode_f64(model, W64, h0, eps=1e-5, bf16_operands=False):
    """One decode step of a LLaMA-style decoder stack in FP64 (the reference
    of the persistent stack launch). W64: per tensor, the weights as FP64 in
    descriptor order (q, k, v, o, gate, up, down per layer). Per layer, with
    r = 1/sqrt(mean(h^2) + eps) per token and unit norm gains:
      v = (h r) Wv^T; a = the value of the single token itself (softmax over
      one score is 1), query head j reading KV head j // (H / H_kv);
      h += a Wo^T; g, u = (h r') W^T; h += (silu(g) * u) Wd^T.
    q and k do not affect a one-token step.
    bf16_operands: every linear takes its activation operand in BF16, as the
    stack launch's linears do (R11: round to nearest even; the residual h
    stays in full precision): v = R((R(h) Wv^T) r), a from R-rounded v,
    g, u = (R(h) W^T) r', act = R(silu(g) u), where R rounds to BF16."""
    h = np.asarray(h0, np.float64).copy()
    M = h.shape[0]
    H, Hkv, hd = model.n_heads, model.n_kv_heads, model.head_dim
    R = _bf16_round if bf16_operands else (lambda z: z)
    for l in range(model.num_layers):
        ts = {t.kind: i for i, t in enumerate(model.tensors) if t.layer == l}
        r = 1.0 / np.sqrt(np.mean(h * h, axis=1, keepdims=True) + eps)
        v = R(linear_f64(R(h), W64[ts[4]]) * r)                  # kind 4 = v
        a = np.repeat(v.reshape(M, Hkv, hd), H // Hkv, axis=1).reshape(M, H * hd)
        h = h + linear_f64(a, W64[ts[5]])                         # o
        r = 1.0 / np.sqrt(np.mean(h * h, axis=1, keepdims=True) + eps)
        g = linear_f64(R(h), W64[ts[6]]) * r                      # gate
        u = linear_f64(R(h), W64[ts[7]]) * r                      # up
        h = h + linear_f64(R(silu(g) * u), W64[ts[8]])            # down
    return h


# ------------------------------------------------------------------ MoE FFN

def moe_route_f64(z, top_k):
    """Routing of the MoE model (§5, Qwen3-30B-A3B): per token the top_k
    experts by router logit (equal logits: the lower expert id first) and
    their weights, the softmax probabilities of the selected experts
    renormalised to sum to one. z: [M, E] logits (any precision; the choice
    is made on these values). Returns (selection [M, k], weights [M, k] FP64)."""
    z = np.asarray(z)
    M, E = z.shape
    sel = np.zeros((M, top_k), np.int64)
    w = np.zeros((M, top_k), np.float64)
    for m in range(M):
        order = sorted(range(E), key=lambda e: (-float(z[m, e]), e))
        sel[m] = order[:top_k]
        zz = np.asarray(z[m], np.float64)
        p = np.exp(zz - zz.max())
        p /= p.sum()
        w[m] = p[sel[m]] / p[sel[m]].sum()
    return sel, w


def moe_ffn_f64(x64, Wr64, experts64, top_k, select_logits=None):
    """MoE FFN in FP64 on logical weights: router logits z = x Wr^T, the
    routing of moe_route_f64 (decided on `select_logits` when given, e.g.
    the kernel's FP32 logits), and y = sum_j w_j down_j(silu(gate_j x) *
    up_j x). experts64[e] = (gate, up, down). Returns (y, z, sel, w)."""
    x = np.asarray(x64, np.float64)
    z = linear_f64(x, Wr64)
    sel, w = moe_route_f64(z if select_logits is None else select_logits, top_k)
    y = np.zeros((x.shape[0], experts64[0][2].shape[0]))
    for m in range(x.shape[0]):
        for j in range(top_k):
            g, u, d = experts64[sel[m, j]]
            h = silu(g @ x[m]) * (u @ x[m])
            y[m] += w[m, j] * (d @ h)
    return y, z, sel, w


# ------------------------------------------------------------- full forward

def rope_f64(x, pos, theta=10000.0):
    """Rotary embedding of 128-dim heads: pairs (i, i+64) rotated by
    pos * theta^(-i/64). x: [T, heads, 128], pos: [T]."""
    i = np.arange(64, dtype=np.float64)
    ang = np.asarray(pos, np.float64)[:, None] * theta ** (-i / 64.0)
    c, s = np.cos(ang)[:, None, :], np.sin(ang)[:, None, :]
    a, b = x[..., :64], x[..., 64:]
    return np.concatenate([a * c - b * s, b * c + a * s], axis=-1)


def transformer_logits_f64(model, W64, emb64, tokens, eps=1e-5, theta=10000.0):
    """Logits of every position of one sequence through the full model in
    FP64 (the reference of the serving step): embedding, per layer RMSNorm
    (unit gain), q/k/v, RoPE, causal softmax attention (GQA: query head j uses
    KV head j // (H/H_kv)), o + residual, RMSNorm, SwiGLU MLP + residual; final
    RMSNorm and the output projection."""
    T = len(tokens)
    H, Hkv, hd = model.n_heads, model.n_kv_heads, 128
    h = np.asarray(emb64, np.float64)[np.asarray(tokens)]
    pos = np.arange(T)
    ts_lm = [i for i, t in enumerate(model.tensors) if t.kind == 9][0]
    norm = lambda z: z / np.sqrt(np.mean(z * z, axis=1, keepdims=True) + eps)
    for l in range(model.tensors[ts_lm].layer):
        ts = {t.kind: i for i, t in enumerate(model.tensors) if t.layer == l}
        x = norm(h)
        q = rope_f64((x @ W64[ts[2]].T).reshape(T, H, hd), pos, theta)
        k = rope_f64((x @ W64[ts[3]].T).reshape(T, Hkv, hd), pos, theta)
        v = (x @ W64[ts[4]].T).reshape(T, Hkv, hd)
        a = np.zeros((T, H, hd))
        for j in range(H):
            kv = j // (H // Hkv)
            sc = q[:, j] @ k[:, kv].T / np.sqrt(hd) + np.triu(np.full((T, T), -np.inf), 1)
            p = np.exp(sc - sc.max(1, keepdims=True))
            a[:, j] = (p / p.sum(1, keepdims=True)) @ v[:, kv]
        h = h + a.reshape(T, H * hd) @ W64[ts[5]].T
        x = norm(h)
        g, u = x @ W64[ts[6]].T, x @ W64[ts[7]].T
        h = h + (silu(g) * u) @ W64[ts[8]].T
    return norm(h) @ W64[ts_lm].T
