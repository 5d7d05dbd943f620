"""Seeded synthetic workloads: model shapes and input tensors.

This module is the only thing the CUDA path and the CPU oracle share. It holds
shapes and seeded random numbers and none of the cloaking arithmetic: no
permutation, no table, no rounding, no quantisation. Weights are FP32
N(0, 0.02) and activations FP32 N(0, 1), drawn with NumPy's PCG64
(``default_rng``) on the host, or with a seeded ``torch.Generator`` on the
device for models too large to draw on the host.

The shapes stand in for the paper's workloads (Section 5, "Setup and
Hardware": Llama 3.1 8B / Qwen3 14B / Qwen3-30B under vLLM), whose trained
checkpoints are not available: a 7B-class dense decoder layer (d_model 4096,
32 heads of 128, gated MLP 11008), a 32-layer stack of it, and a 28-layer GQA
model (d_model 3584, 28 query / 4 KV heads of 128, gated MLP 18944).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

# storage dtypes of a model's weight tiles
DT_F32, DT_BF16, DT_E4M3 = 0, 1, 2
DTYPE_SIZE = {DT_F32: 4, DT_BF16: 2, DT_E4M3: 1}
DTYPE_NAME = {DT_F32: "f32", DT_BF16: "bf16", DT_E4M3: "e4m3"}

# tensor kinds (informational; the layer-stack launch uses them to wire stages)
(K_W1, K_W2, K_Q, K_K, K_V, K_O, K_GATE, K_UP, K_DOWN, K_LMHEAD, K_EMBED, K_ROUTER, K_EGATE, K_EUP,
 K_EDOWN) = range(15)


@dataclass
class Tensor:
    n: int            # output features (rows)
    k: int            # input features (columns)
    layer: int
    kind: int
    perm_group: int = -1   # -1: not permuted
    perm_axis: int = 0     # 0: rows permuted (producer), 1: columns (consumer)
    perm_group2: int = -1  # group of the other axis (the residual dimension), -1: none


@dataclass
class Group:
    n_units: int
    unit: int              # rows (or columns) per unit
    parent: int = -1       # derived group: follows parent's unit order
    ratio: int = 1         # units per parent unit when derived


@dataclass
class Model:
    name: str
    dtype: int
    tile_r: int
    tile_c: int
    page_bytes: int
    spare_pages: int
    tensors: List[Tensor] = field(default_factory=list)
    groups: List[Group] = field(default_factory=list)
    tile_scope: int = 0    # 0: one tile permutation over the whole model; 1: per tensor
    tile_rekey: bool = False  # redraw the tile permutation at every epoch (re-keys move tiles)
    # architecture constants used by the layer-stack/serving path
    d_model: int = 0
    n_heads: int = 0
    n_kv_heads: int = 0
    head_dim: int = 128
    d_ff: int = 0
    vocab: int = 0

    @property
    def tile_bytes(self) -> int:
        return self.tile_r * self.tile_c * DTYPE_SIZE[self.dtype]

    @property
    def num_layers(self) -> int:
        return 1 + max(t.layer for t in self.tensors)

    def tiles_of(self, t: Tensor):
        return (-(-t.n // self.tile_r), -(-t.k // self.tile_c))

    @property
    def num_tiles(self) -> int:
        return sum(a * b for a, b in (self.tiles_of(t) for t in self.tensors))

    @property
    def weight_bytes(self) -> int:
        return self.num_tiles * self.tile_bytes


def mlp2(d_model=256, d_ff=1024, name="mlp2_f32_256x1024") -> Model:
    """Two-layer MLP, FP32, 64x64 tiles, one tile per 16 KiB page.

    W1 [d_ff, d_model] is the producer (rows permuted), W2 [d_model, d_ff] the
    consumer (columns permuted with the same permutation)."""
    m = Model(name=name, dtype=DT_F32, tile_r=64, tile_c=64, page_bytes=16384,
              spare_pages=0, d_model=d_model, d_ff=d_ff)
    m.groups = [Group(n_units=d_ff, unit=1)]
    m.tensors = [Tensor(d_ff, d_model, 0, K_W1, 0, 0),
                 Tensor(d_model, d_ff, 1, K_W2, 0, 1)]
    return m


def decoder(n_layers: int, d_model: int, n_heads: int, n_kv_heads: int,
            d_ff: int, dtype: int, name: str, head_dim: int = 128,
            spare_pages: int = 64) -> Model:
    """Stack of LLaMA-style decoder layers (Wq, Wk, Wv, Wo, Wgate, Wup, Wdown).

    Per layer three permutation groups (intra-layer shuffling):
      * KV heads: rows of Wk and Wv in blocks of head_dim;
      * query heads: derived from the KV-head order, each query head moving
        with its KV head and the heads of one group permuted among themselves;
        rows of Wq and columns of Wo;
      * MLP hidden units: rows of Wgate and Wup, columns of Wdown.
    """
    tile = 128
    esz = DTYPE_SIZE[dtype]
    m = Model(name=name, dtype=dtype, tile_r=tile, tile_c=tile, page_bytes=2 << 20,
              spare_pages=spare_pages, d_model=d_model, n_heads=n_heads,
              n_kv_heads=n_kv_heads, head_dim=head_dim, d_ff=d_ff)
    assert (2 << 20) % (tile * tile * esz) == 0
    ratio = n_heads // n_kv_heads
    for l in range(n_layers):
        g_kv = len(m.groups)
        m.groups.append(Group(n_kv_heads, head_dim))
        g_q = len(m.groups)
        m.groups.append(Group(n_heads, head_dim, parent=g_kv, ratio=ratio))
        g_ff = len(m.groups)
        m.groups.append(Group(d_ff, 1))
        qd, kvd = n_heads * head_dim, n_kv_heads * head_dim
        m.tensors += [
            Tensor(qd, d_model, l, K_Q, g_q, 0),
            Tensor(kvd, d_model, l, K_K, g_kv, 0),
            Tensor(kvd, d_model, l, K_V, g_kv, 0),
            Tensor(d_model, qd, l, K_O, g_q, 1),
            Tensor(d_ff, d_model, l, K_GATE, g_ff, 0),
            Tensor(d_ff, d_model, l, K_UP, g_ff, 0),
            Tensor(d_model, d_ff, l, K_DOWN, g_ff, 1),
        ]
    return m


def moe_block(n_layers: int = 1, d_model: int = 2048, n_experts: int = 128, top_k: int = 8,
              d_ff: int = 768, spare_pages: int = 64, page_bytes: int = 2 << 20,
              name: str = "") -> Model:
    """MoE FFN blocks (the Qwen3-30B-A3B shape by default: d 2048, 128
    experts of gated MLP 768, top-8), BF16. Per layer a router [n_experts,
    d_model] whose rows follow the expert-order permutation group (unit 1:
    the router's stored output e' scores logical expert perm[e']), and per
    expert gate, up [d_ff, d_model] and down [d_model, d_ff] with their own
    hidden-unit group (rows of gate/up, columns of down). The tensors of
    logical expert e are expert_tensors[layer][e] = (gate, up, down)."""
    tile = 128
    m = Model(name=name or f"moe{n_experts}x{d_ff}_d{d_model}_{n_layers}L", dtype=DT_BF16, tile_r=tile,
              tile_c=tile, page_bytes=page_bytes, spare_pages=spare_pages, d_model=d_model, d_ff=d_ff)
    m.n_experts, m.top_k = n_experts, top_k
    m.router_tensors, m.expert_groups, m.expert_tensors = [], [], []
    for l in range(n_layers):
        g_e = len(m.groups)
        m.groups.append(Group(n_experts, 1))
        m.expert_groups.append(g_e)
        m.router_tensors.append(len(m.tensors))
        m.tensors.append(Tensor(n_experts, d_model, l, K_ROUTER, g_e, 0))
        ets = []
        for e in range(n_experts):
            g_h = len(m.groups)
            m.groups.append(Group(d_ff, 1))
            t0 = len(m.tensors)
            m.tensors += [Tensor(d_ff, d_model, l, K_EGATE, g_h, 0),
                          Tensor(d_ff, d_model, l, K_EUP, g_h, 0),
                          Tensor(d_model, d_ff, l, K_EDOWN, g_h, 1)]
            ets.append((t0, t0 + 1, t0 + 2))
        m.expert_tensors.append(ets)
    return m


def llama7b_layer(n_layers=1, dtype=DT_BF16) -> Model:
    """7B-class dense layer(s): d 4096, 32x128 heads (MHA), gated MLP 11008, BF16."""
    return decoder(n_layers, 4096, 32, 32, 11008, dtype,
                   name=f"llama7b_bf16_{n_layers}L")


def gqa28_fp8(n_layers=28) -> Model:
    """28-layer GQA shape: d 3584, 28 query / 4 KV heads of 128, MLP 18944, E4M3."""
    return decoder(n_layers, 3584, 28, 4, 18944, DT_E4M3,
                   name=f"gqa3584_e4m3_{n_layers}L", spare_pages=64)


def with_lm_head(model: Model, vocab: int, cloaked_embedding: bool = False) -> Model:
    """Append an output projection [vocab, d_model] (its own layer index,
    not permuted: the residual stream keeps its order); with
    `cloaked_embedding`, the embedding table [vocab, d_model] as a tensor of
    its own layer too, placed and looked up through the keyed layout."""
    L = model.num_layers
    model.tensors.append(Tensor(vocab, model.d_model, L, K_LMHEAD))
    if cloaked_embedding:
        model.tensors.append(Tensor(vocab, model.d_model, L + 1, K_EMBED))
    model.vocab = vocab
    return model


def with_residual_permutation(model: Model) -> Model:
    """One keyed permutation of the residual dimension (unit 1, its own
    group) shared by every matrix that reads the residual stream (columns of
    q, k, v, gate, up, the lm_head and the embedding table) or writes it
    (rows of o and down). The stream then lives in keyed order from the
    embedding to the output projection: RMSNorm with unit gains does not see
    the order, so the logits are unchanged. Call after with_lm_head."""
    g = len(model.groups)
    model.groups.append(Group(model.d_model, 1))
    for t in model.tensors:
        if t.kind in (K_Q, K_K, K_V, K_GATE, K_UP, K_LMHEAD, K_EMBED):
            assert t.perm_group < 0 or t.perm_axis == 0
            t.perm_axis = 0              # the other axis, columns, is the residual
        elif t.kind in (K_O, K_DOWN):
            assert t.perm_axis == 1      # rows are the residual
        else:
            continue
        t.perm_group2 = g
    model.residual_group = g
    return model


def serving_model(n_layers=32, vocab=32000) -> Model:
    """The served model: the 7B-class BF16 stack plus a 32,000-token lm_head."""
    return with_lm_head(llama7b_layer(n_layers), vocab)


def small_decoder(n_layers=2, dtype=DT_BF16, d_model=256, n_heads=4,
                  n_kv_heads=2, d_ff=384, head_dim=64, spare_pages=3,
                  page_bytes=None) -> Model:
    """A small decoder of the same structure, for tests the oracle finishes in
    seconds (several tiles per tensor, head_dim 64 so head blocks straddle
    nothing, d_ff not a multiple of the tile so the last tile row is ragged)."""
    m = decoder(n_layers, d_model, n_heads, n_kv_heads, d_ff, dtype,
                name=f"small_{DTYPE_NAME[dtype]}_{n_layers}L", head_dim=head_dim,
                spare_pages=spare_pages)
    m.page_bytes = page_bytes or 4 * m.tile_bytes
    return m


# --------------------------------------------------------------------------
# seeded data
# --------------------------------------------------------------------------

def weights_host(model: Model, seed: int = 0, std: float = 0.02):
    """FP32 logical weights, one [n, k] array per tensor, drawn in tensor order
    from a single PCG64 stream."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((t.n, t.k), dtype=np.float32) * np.float32(std)
            for t in model.tensors]


def activations_host(m: int, k: int, seed: int = 1) -> np.ndarray:
    """FP32 activations [m, k], N(0, 1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, k), dtype=np.float32)


def int_weights_host(model: Model, seed: int, lo=-2, hi=2):
    """Small-integer-valued FP32 weights (every FP32/FP64 sum stays exact)."""
    rng = np.random.default_rng(seed)
    return [rng.integers(lo, hi + 1, size=(t.n, t.k)).astype(np.float32)
            for t in model.tensors]


def embedding_host(vocab: int, d_model: int, seed: int = 5, std: float = 1.0):
    """Token embedding table [vocab, d_model], FP32 N(0, std)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((vocab, d_model), dtype=np.float32) * np.float32(std)


def requests_poisson(rate: float, duration: float, vocab: int, seed: int = 0,
                     prompt_median: int = 1024, prompt_sigma: float = 0.8,
                     prompt_min: int = 128, prompt_max: int = 4096,
                     out_min: int = 64, out_max: int = 1024):
    """Serving workload: Poisson arrivals at `rate` req/s over `duration` s,
    prompt lengths lognormal (median `prompt_median`) clipped to
    [prompt_min, prompt_max], output lengths uniform in [out_min, out_max],
    prompt tokens uniform over the vocabulary. Returns (arrival_s, prompt
    ndarray, max_new_tokens) tuples in arrival order."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(np.clip(np.exp(rng.normal(np.log(prompt_median), prompt_sigma)), prompt_min, prompt_max))
        out.append((t, rng.integers(0, vocab, n, dtype=np.int32), int(rng.integers(out_min, out_max + 1))))
    return out


def weights_device(model: Model, tensor_index: int, seed: int = 0,
                   std: float = 0.02, device="cuda"):
    """FP32 logical weights of one tensor drawn on the device (for models whose
    FP32 master weights are too large to draw on the host). The stream is
    keyed by (seed, tensor_index) so any tensor can be regenerated alone."""
    import torch
    t = model.tensors[tensor_index]
    g = torch.Generator(device=device)
    g.manual_seed(seed * 1000003 + tensor_index)
    w = torch.randn((t.n, t.k), generator=g, device=device, dtype=torch.float32)
    return w.mul_(std)
