// keygen.cu -- keyed tables drawn on the device.
//
// The paper seeds a PRNG, enumerates the weight allocations and computes a
// random permutation before any weight is transferred (Section 5,
// "Implementation Details"). Here every table is a Fisher-Yates shuffle of a
// SplitMix64 stream (Steele, Lea, Flood 2014) with Lemire's unbiased bounded
// draw (Lemire 2019):
//   stream(key, tag, epoch, idx) starts at mix(key ^ mix(tag<<56 ^ epoch<<32 ^ idx));
//   tag 1: layer order; tag 2: permutation group idx; tag 3: tile permutation
//   (idx 0, or the tensor in per-tensor scope); tag 4: page map (the only
//   table that depends on the epoch).
//
// Fisher-Yates is sequential as written (for i = n-1..1 swap a[i], a[j_i]),
// but its result has a closed form that parallelises:
//   * SplitMix64's k-th output is mix(state + k * gamma), so every draw j_i is
//     computed independently (a rejection in Lemire's method, probability
//     below n / 2^64 per draw, is detected and the whole batch is then redone
//     by the sequential kernel);
//   * step i moves v_i (the value at position i just before step i) to j_i
//     and finalises position i. With the writers of position q (steps w > q
//     with j_w = q) sorted ascending, w_1 < w_2 < ..., a step reads the value
//     its next larger co-writer wrote: final[w_k] = v[w_{k+1}] (or q for the
//     largest), v_q = v[w_1] (or q), final[0] = v[w_1 of position 0] (or 0),
//     and final[i] = v_i when j_i = i.
//   The v's form a forest (parent w_1(i) > i) resolved by pointer jumping.
// Both paths give the sequential algorithm's permutation bit for bit.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

namespace cloak {

int g_force_sequential_fy = 0;

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t stream_seed(uint64_t key, uint32_t tag, uint32_t epoch, uint32_t idx) {
    uint64_t lane = ((uint64_t)tag << 56) ^ ((uint64_t)epoch << 32) ^ (uint64_t)idx;
    return sm64_mix(key ^ sm64_mix(lane));
}

// A chain is `reps` consecutive Fisher-Yates shuffles of n elements drawn
// from one stream; outputs are contiguous from `off`.
struct FyChain {
    uint64_t state;
    uint32_t n, reps, off, sub_start;
};

__device__ __forceinline__ uint32_t seg_lookup(const uint32_t *seg_off, int nseg, uint32_t p) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return (uint32_t)lo;
}

// expand chains into one sub-segment per shuffle (states assume no rejection)
__global__ void k_fy_expand(const FyChain *ch, int nch, FySeg *sub, uint32_t *sub_off) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    FyChain q = ch[c];
    uint64_t adv = (uint64_t)(q.n > 0 ? q.n - 1 : 0) * SM64_GAMMA;
    for (uint32_t r = 0; r < q.reps; ++r) {
        FySeg s;
        s.state = q.state + (uint64_t)r * adv;
        s.n = q.n;
        s.off = q.off + r * q.n;
        sub[q.sub_start + r] = s;
        sub_off[q.sub_start + r] = s.off;
    }
}

struct FyArgs {
    const FySeg *seg;
    const uint32_t *seg_off;
    int nseg;
    uint32_t total;
    KeygenWork w;
};

__global__ void k_fy_draw(FyArgs a) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.total) return;
    FySeg s = a.seg[seg_lookup(a.seg_off, a.nseg, p)];
    uint32_t i = p - s.off;
    a.w.first[p] = NONE;
    a.w.cnt[p] = 0;
    a.w.cursor[p] = 0;
    if (i == 0) {
        a.w.j[p] = 0;
        return;
    }
    // step i is the (n - i)-th draw of the shuffle
    uint64_t x = sm64_mix(s.state + (uint64_t)(s.n - i) * SM64_GAMMA);
    uint64_t bound = (uint64_t)i + 1;
    uint64_t lo = x * bound;
    if (lo < bound) {
        uint64_t t = (0ull - bound) % bound;
        if (lo < t) atomicExch(&a.w.counters[1], 1u);  // rejection: redo sequentially
    }
    a.w.j[p] = (uint32_t)__umul64hi(x, bound);
}

__global__ void k_fy_count(FyArgs a) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.total) return;
    FySeg s = a.seg[seg_lookup(a.seg_off, a.nseg, p)];
    uint32_t i = p - s.off, jj = a.w.j[p];
    if (i == 0 || jj >= i) return;
    atomicAdd(&a.w.cnt[s.off + jj], 1u);
    atomicMin(&a.w.first[s.off + jj], i);
}

__global__ void k_fy_alloc(FyArgs a) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.total) return;
    uint32_t c = a.w.cnt[p];
    a.w.boff[p] = c ? atomicAdd(&a.w.counters[0], c) : 0u;
}

__global__ void k_fy_scatter(FyArgs a) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.total) return;
    FySeg s = a.seg[seg_lookup(a.seg_off, a.nseg, p)];
    uint32_t i = p - s.off, jj = a.w.j[p];
    if (i == 0 || jj >= i) return;
    uint32_t q = s.off + jj;
    uint32_t slot = atomicAdd(&a.w.cursor[q], 1u);
    a.w.bucket[a.w.boff[q] + slot] = i;
}

// sort each position's writers; link each writer to the next larger one
__global__ void k_fy_sort(FyArgs a) {
    uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.total) return;
    uint32_t c = a.w.cnt[q];
    if (c == 0) return;
    FySeg s = a.seg[seg_lookup(a.seg_off, a.nseg, q)];
    uint32_t *b = a.w.bucket + a.w.boff[q];
    for (uint32_t x = 1; x < c; ++x) {
        uint32_t v = b[x];
        int y = (int)x - 1;
        while (y >= 0 && b[y] > v) {
            b[y + 1] = b[y];
            --y;
        }
        b[y + 1] = v;
    }
    for (uint32_t x = 0; x < c; ++x) a.w.succ[s.off + b[x]] = (x + 1 < c) ? b[x + 1] : NONE;
}

__global__ void k_fy_ptr_init(FyArgs a) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.total) return;
    FySeg s = a.seg[seg_lookup(a.seg_off, a.nseg, p)];
    uint32_t i = p - s.off, f = a.w.first[p];
    if (i == 0 || f == NONE) {
        a.w.ptr0[p] = NONE;
        a.w.val0[p] = i;
    } else {
        a.w.ptr0[p] = s.off + f;
        a.w.val0[p] = 0;
    }
}

__global__ void k_fy_jump(const uint32_t *pin, const uint32_t *vin, uint32_t *pout, uint32_t *vout,
                          uint32_t total) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    uint32_t q = pin[p];
    if (q == NONE) {
        pout[p] = NONE;
        vout[p] = vin[p];
        return;
    }
    uint32_t qq = pin[q];
    if (qq == NONE) {
        pout[p] = NONE;
        vout[p] = vin[q];
    } else {
        pout[p] = qq;
        vout[p] = 0;
    }
}

__global__ void k_fy_final(FyArgs a, const uint32_t *v) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.total) return;
    FySeg s = a.seg[seg_lookup(a.seg_off, a.nseg, p)];
    uint32_t i = p - s.off;
    uint32_t r;
    if (i == 0) {
        uint32_t f = a.w.first[p];
        r = (f == NONE) ? 0u : v[s.off + f];
    } else {
        uint32_t jj = a.w.j[p];
        if (jj == i) {
            r = v[p];
        } else {
            uint32_t sc = a.w.succ[p];
            r = (sc == NONE) ? jj : v[s.off + sc];
        }
    }
    a.w.out[p] = r;
}

__device__ __forceinline__ uint64_t dev_next(uint64_t *st) {
    *st += SM64_GAMMA;
    return sm64_mix(*st);
}

// Advance chain states past the shuffles just drawn, or, if a rejection was
// seen (or the sequential path is forced), redo each chain sequentially.
__global__ void k_fy_fixup(FyChain *ch, int nch, uint32_t *out, const uint32_t *counters,
                           int force) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nch) return;
    FyChain q = ch[c];
    if (!force && counters[1] == 0) {
        ch[c].state = q.state + (uint64_t)q.reps * (uint64_t)(q.n > 0 ? q.n - 1 : 0) * SM64_GAMMA;
        return;
    }
    uint64_t st = q.state;
    for (uint32_t r = 0; r < q.reps; ++r) {
        uint32_t *a = out + q.off + r * q.n;
        for (uint32_t i = 0; i < q.n; ++i) a[i] = i;
        for (uint32_t i = q.n - 1; q.n > 1 && i >= 1; --i) {
            uint64_t bound = (uint64_t)i + 1;
            uint64_t x = dev_next(&st);
            uint64_t lo = x * bound;
            if (lo < bound) {
                uint64_t t = (0ull - bound) % bound;
                while (lo < t) {
                    x = dev_next(&st);
                    lo = x * bound;
                }
            }
            uint32_t j = (uint32_t)__umul64hi(x, bound);
            uint32_t tmp = a[i];
            a[i] = a[j];
            a[j] = tmp;
        }
    }
    ch[c].state = st;
}

static inline unsigned nblk(uint64_t n, unsigned b = 256) { return (unsigned)((n + b - 1) / b); }

// Device-side storage of a batch of chains (persistent across redraws)
struct FyBatch {
    FyChain *d_chains = nullptr;
    int nch = 0, nsub = 0;
    uint32_t total = 0, max_n = 0;
};

static cloak_status fy_batch_make(cloak_ctx *ctx, std::vector<FyChain> &chains, FyBatch &b,
                                  cudaStream_t s) {
    // chains must be given in increasing output offset, n > 0
    b.nch = (int)chains.size();
    b.nsub = 0;
    b.total = 0;
    b.max_n = 1;
    for (auto &c : chains) {
        c.sub_start = (uint32_t)b.nsub;
        b.nsub += (int)c.reps;
        b.total = std::max<uint32_t>(b.total, c.off + c.n * c.reps);
        b.max_n = std::max(b.max_n, c.n);
    }
    if (b.total > ctx->kw.cap || (uint32_t)b.nsub > ctx->kw.seg_cap) return CLOAK_E_INVAL;
    CLOAK_CUDA(ctx, cudaMallocAsync((void **)&b.d_chains, sizeof(FyChain) * chains.size(), s));
    CLOAK_CUDA(ctx, cudaMemcpyAsync(b.d_chains, chains.data(), sizeof(FyChain) * chains.size(),
                                    cudaMemcpyHostToDevice, s));
    return CLOAK_OK;
}

static void fy_batch_free(FyBatch &b, cudaStream_t s) {
    if (b.d_chains) cudaFreeAsync(b.d_chains, s);
    b.d_chains = nullptr;
}

// Draw one shuffle per sub-segment of the batch into ctx->kw.out.
static cloak_status fy_batch_run(cloak_ctx *ctx, FyBatch &b, cudaStream_t s) {
    KeygenWork &w = ctx->kw;
    CLOAK_CUDA(ctx, cudaMemsetAsync(w.counters, 0, 4 * sizeof(uint32_t), s));
    int force = g_force_sequential_fy;
    const char *env = getenv("CLOAK_FY_SEQUENTIAL");
    if (env && env[0] == '1') force = 1;
    if (!force) {
        k_fy_expand<<<nblk(b.nch), 256, 0, s>>>(b.d_chains, b.nch, w.segs, w.seg_off);
        CLOAK_LAUNCHED(ctx);
        FyArgs a{w.segs, w.seg_off, b.nsub, b.total, w};
        unsigned g = nblk(b.total);
        k_fy_draw<<<g, 256, 0, s>>>(a);
        CLOAK_LAUNCHED(ctx);
        k_fy_count<<<g, 256, 0, s>>>(a);
        CLOAK_LAUNCHED(ctx);
        k_fy_alloc<<<g, 256, 0, s>>>(a);
        CLOAK_LAUNCHED(ctx);
        k_fy_scatter<<<g, 256, 0, s>>>(a);
        CLOAK_LAUNCHED(ctx);
        k_fy_sort<<<g, 256, 0, s>>>(a);
        CLOAK_LAUNCHED(ctx);
        k_fy_ptr_init<<<g, 256, 0, s>>>(a);
        CLOAK_LAUNCHED(ctx);
        int rounds = 1;
        while ((1u << rounds) < b.max_n + 1) ++rounds;
        rounds += 1;
        uint32_t *pi = w.ptr0, *vi = w.val0, *po = w.ptr1, *vo = w.val1;
        for (int r = 0; r < rounds; ++r) {
            k_fy_jump<<<g, 256, 0, s>>>(pi, vi, po, vo, b.total);
            CLOAK_LAUNCHED(ctx);
            std::swap(pi, po);
            std::swap(vi, vo);
        }
        k_fy_final<<<g, 256, 0, s>>>(a, vi);
        CLOAK_LAUNCHED(ctx);
    }
    k_fy_fixup<<<nblk(b.nch, 64), 64, 0, s>>>(b.d_chains, b.nch, w.out, w.counters, force);
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

// ------------------------------------------------------------ table kernels

__global__ void k_copy_u32(uint32_t *dst, const uint32_t *src, uint32_t n, uint32_t add) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = src[p] + add;
}

// derived group: out[a*ratio + b] = parent[a]*ratio + inner[a*ratio + b]
__global__ void k_compose_group(uint32_t *dst, const uint32_t *parent, const uint32_t *inner,
                                uint32_t n_units, uint32_t ratio) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_units) return;
    dst[p] = parent[p / ratio] * ratio + inner[p];
}

// arena order of tensors: layers in layer_perm order, then descriptor order
__global__ void k_tensor_base(const uint32_t *layer_perm, int L, const TensorInfo *info, int T,
                              uint32_t *base) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    uint32_t b = 0;
    for (int p = 0; p < L; ++p)
        for (int t = 0; t < T; ++t)
            if (info[t].layer == (int)layer_perm[p]) {
                base[t] = b;
                b += (uint32_t)(info[t].nt * info[t].kt);
            }
}

// per-tensor scope: tile_perm[base + v] = base + local[base + v]
__global__ void k_tile_perm_local(uint32_t *tp, const uint32_t *local, const uint32_t *base,
                                  const TensorInfo *info, int T, uint32_t G) {
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G) return;
    // find tensor whose [base, base + tiles) holds v
    uint32_t b = 0;
    for (int t = 0; t < T; ++t) {
        uint32_t bt = base[t], nt = (uint32_t)(info[t].nt * info[t].kt);
        if (v >= bt && v < bt + nt) {
            b = bt;
            break;
        }
    }
    tp[v] = b + local[v];
}

__global__ void k_intra_check(const uint32_t *tp, uint32_t G, uint32_t tpp, uint32_t *viol) {
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v + 1 >= G) return;
    if ((v % tpp) != tpp - 1 && tp[v + 1] == tp[v] + 1) atomicAdd(viol, 1u);
}

__global__ void k_fill(uint32_t *a, uint32_t n, uint32_t v) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) a[p] = v;
}

__global__ void k_p2v(const uint32_t *pa, uint32_t NP, uint32_t *p2v) {
    uint32_t vp = blockIdx.x * blockDim.x + threadIdx.x;
    if (vp < NP) p2v[pa[vp]] = vp;
}

__global__ void k_cross_check(const uint32_t *tp, const uint32_t *p2v, uint32_t G, uint32_t tpp,
                              uint32_t NPS, uint32_t *viol) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p + 1 >= NPS) return;
    uint32_t a = p2v[p], b = p2v[p + 1];
    if (a == NONE || b == NONE) return;
    uint64_t vl = (uint64_t)a * tpp + tpp - 1, vf = (uint64_t)b * tpp;
    if (vl < G && vf < G && tp[vf] == tp[vl] + 1) atomicAdd(viol, 1u);
}

__global__ void k_inverse(const uint32_t *tp, uint32_t G, uint32_t *inv) {
    uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < G) inv[tp[v]] = v;
}

__global__ void k_tile_slot(const uint32_t *inv, const uint32_t *pa, uint32_t G, uint32_t tpp,
                            uint32_t *slot) {
    uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    uint32_t v = inv[g];
    slot[g] = pa[v / tpp] * tpp + v % tpp;
}

// ------------------------------------------------------------------ drivers

static constexpr uint32_t MAX_DRAWS = 100000;

static cloak_status read_u32(cloak_ctx *ctx, const uint32_t *d, uint32_t *h, cudaStream_t s) {
    CLOAK_CUDA(ctx, cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    return CLOAK_OK;
}

cloak_status keygen_alloc(cloak_ctx *ctx) {
    KeygenWork &w = ctx->kw;
    uint64_t cap = std::max<uint64_t>({(uint64_t)ctx->G, (uint64_t)ctx->NPS,
                                       (uint64_t)(ctx->L + ctx->U), 1});
    w.cap = (uint32_t)cap;
    uint32_t **arrs[] = {&w.j, &w.first, &w.cnt, &w.boff, &w.cursor, &w.bucket,
                         &w.succ, &w.ptr0, &w.ptr1, &w.val0, &w.val1, &w.out};
    for (auto a : arrs) CLOAK_CUDA(ctx, cudaMalloc((void **)a, cap * sizeof(uint32_t)));
    CLOAK_CUDA(ctx, cudaMalloc((void **)&w.counters, 4 * sizeof(uint32_t)));
    uint64_t segs = 1 + ctx->tensors.size() + 1;
    for (auto &g : ctx->groups) segs += (g.parent >= 0) ? (uint64_t)ctx->groups[g.parent].n_units : 1;
    w.seg_cap = (uint32_t)segs;
    CLOAK_CUDA(ctx, cudaMalloc((void **)&w.segs, segs * sizeof(FySeg)));
    CLOAK_CUDA(ctx, cudaMalloc((void **)&w.seg_off, segs * sizeof(uint32_t)));
    return CLOAK_OK;
}

// Page map of (key, epoch) for the current tile permutation, into d_out[NPS],
// redrawn until no two physically adjacent pages join consecutive tiles.
cloak_status keygen_page_map(cloak_ctx *ctx, uint64_t key, uint32_t epoch, uint32_t *d_out,
                             cudaStream_t s) {
    std::vector<FyChain> ch{{stream_seed(key, 4, epoch, 0), (uint32_t)ctx->NPS, 1, 0, 0}};
    FyBatch b;
    cloak_status rc = fy_batch_make(ctx, ch, b, s);
    if (rc) return rc;
    KeygenWork &w = ctx->kw;
    uint32_t draws = 0, viol = 1;
    while (viol) {
        if (++draws > MAX_DRAWS) { fy_batch_free(b, s); return CLOAK_E_DRAWS; }
        if ((rc = fy_batch_run(ctx, b, s))) return rc;
        k_copy_u32<<<nblk(ctx->NPS), 256, 0, s>>>(d_out, w.out, (uint32_t)ctx->NPS, 0);
        CLOAK_LAUNCHED(ctx);
        // p2v in w.j (free after the batch), violations in counters[2]
        k_fill<<<nblk(ctx->NPS), 256, 0, s>>>(w.j, (uint32_t)ctx->NPS, NONE);
        CLOAK_LAUNCHED(ctx);
        k_p2v<<<nblk(ctx->NP), 256, 0, s>>>(d_out, (uint32_t)ctx->NP, w.j);
        CLOAK_LAUNCHED(ctx);
        CLOAK_CUDA(ctx, cudaMemsetAsync(w.counters + 2, 0, sizeof(uint32_t), s));
        k_cross_check<<<nblk(ctx->NPS), 256, 0, s>>>(ctx->d_tile_perm, w.j, (uint32_t)ctx->G,
                                                     (uint32_t)ctx->tpp, (uint32_t)ctx->NPS,
                                                     w.counters + 2);
        CLOAK_LAUNCHED(ctx);
        if ((rc = read_u32(ctx, w.counters + 2, &viol, s))) return rc;
    }
    fy_batch_free(b, s);
    return CLOAK_OK;
}

cloak_status build_tile_slot(cloak_ctx *ctx, const uint32_t *d_page_alloc, cudaStream_t s) {
    uint32_t G = (uint32_t)ctx->G;
    k_inverse<<<nblk(G), 256, 0, s>>>(ctx->d_tile_perm, G, ctx->d_tile_inv);
    CLOAK_LAUNCHED(ctx);
    k_tile_slot<<<nblk(G), 256, 0, s>>>(ctx->d_tile_inv, d_page_alloc, G, (uint32_t)ctx->tpp,
                                        ctx->d_tile_slot);
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

cloak_status keygen_tables(cloak_ctx *ctx, uint64_t key, uint32_t epoch, cudaStream_t s) {
    KeygenWork &w = ctx->kw;
    cloak_status rc;
    const int T = (int)ctx->tensors.size();
    const int NG = (int)ctx->groups.size();

    // 1+2. layer order and permutation groups in one batch:
    //   [0, L) layer order; group g's units at L + goff[g] (root groups),
    //   derived groups' inner shuffles at the same place, composed after.
    std::vector<FyChain> ch;
    ch.push_back({stream_seed(key, 1, 0, 0), (uint32_t)ctx->L, 1, 0, 0});
    for (int g = 0; g < NG; ++g) {
        const cloak_group_desc &gr = ctx->groups[g];
        uint32_t off = (uint32_t)(ctx->L + ctx->goff[g]);
        if (gr.parent < 0)
            ch.push_back({stream_seed(key, 2, 0, (uint32_t)g), (uint32_t)gr.n_units, 1, off, 0});
        else
            ch.push_back({stream_seed(key, 2, 0, (uint32_t)g), (uint32_t)gr.ratio,
                          (uint32_t)ctx->groups[gr.parent].n_units, off, 0});
    }
    FyBatch b;
    if ((rc = fy_batch_make(ctx, ch, b, s))) return rc;
    if ((rc = fy_batch_run(ctx, b, s))) return rc;
    fy_batch_free(b, s);
    k_copy_u32<<<nblk(ctx->L), 256, 0, s>>>(ctx->d_layer_perm, w.out, (uint32_t)ctx->L, 0);
    CLOAK_LAUNCHED(ctx);
    for (int g = 0; g < NG; ++g) {
        const cloak_group_desc &gr = ctx->groups[g];
        uint32_t *dst = ctx->d_group_perm + ctx->goff[g];
        const uint32_t *src = w.out + ctx->L + ctx->goff[g];
        if (gr.parent < 0)
            k_copy_u32<<<nblk(gr.n_units), 256, 0, s>>>(dst, src, (uint32_t)gr.n_units, 0);
        else
            k_compose_group<<<nblk(gr.n_units), 256, 0, s>>>(
                dst, ctx->d_group_perm + ctx->goff[gr.parent], src, (uint32_t)gr.n_units,
                (uint32_t)gr.ratio);
        CLOAK_LAUNCHED(ctx);
    }

    // 3. arena order of tensors
    k_tensor_base<<<1, 32, 0, s>>>(ctx->d_layer_perm, (int)ctx->L, ctx->d_info, T,
                                   ctx->d_tensor_base);
    CLOAK_LAUNCHED(ctx);
    ctx->h_tensor_base.assign(T, 0);
    CLOAK_CUDA(ctx, cudaMemcpyAsync(ctx->h_tensor_base.data(), ctx->d_tensor_base,
                                    T * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CLOAK_CUDA(ctx, cudaStreamSynchronize(s));

    // 4. tile permutation, redrawn until no page holds a successor pair (its
    //    streams take the epoch when re-keys move tiles)
    ch.clear();
    const uint32_t tile_epoch = (ctx->flags & CLOAK_MODEL_TILE_REKEY) ? epoch : 0;
    if (ctx->scope == 0) {
        ch.push_back({stream_seed(key, 3, tile_epoch, 0), (uint32_t)ctx->G, 1, 0, 0});
    } else {
        std::vector<int> order(T);
        for (int t = 0; t < T; ++t) order[t] = t;
        std::sort(order.begin(), order.end(),
                  [&](int a, int c) { return ctx->h_tensor_base[a] < ctx->h_tensor_base[c]; });
        for (int t : order)
            ch.push_back({stream_seed(key, 3, tile_epoch, (uint32_t)t),
                          (uint32_t)(ctx->info[t].nt * ctx->info[t].kt), 1,
                          ctx->h_tensor_base[t], 0});
    }
    if ((rc = fy_batch_make(ctx, ch, b, s))) return rc;
    uint32_t draws = 0, viol = 1;
    while (viol) {
        if (++draws > MAX_DRAWS) { fy_batch_free(b, s); return CLOAK_E_DRAWS; }
        if ((rc = fy_batch_run(ctx, b, s))) return rc;
        if (ctx->scope == 0)
            k_copy_u32<<<nblk(ctx->G), 256, 0, s>>>(ctx->d_tile_perm, w.out, (uint32_t)ctx->G, 0);
        else
            k_tile_perm_local<<<nblk(ctx->G), 256, 0, s>>>(ctx->d_tile_perm, w.out,
                                                           ctx->d_tensor_base, ctx->d_info, T,
                                                           (uint32_t)ctx->G);
        CLOAK_LAUNCHED(ctx);
        CLOAK_CUDA(ctx, cudaMemsetAsync(w.counters + 2, 0, sizeof(uint32_t), s));
        k_intra_check<<<nblk(ctx->G), 256, 0, s>>>(ctx->d_tile_perm, (uint32_t)ctx->G,
                                                   (uint32_t)ctx->tpp, w.counters + 2);
        CLOAK_LAUNCHED(ctx);
        if ((rc = read_u32(ctx, w.counters + 2, &viol, s))) return rc;
    }
    fy_batch_free(b, s);

    // 5. page map of this epoch; 6. gather table
    if ((rc = keygen_page_map(ctx, key, epoch, ctx->d_page_alloc, s))) return rc;
    if ((rc = build_tile_slot(ctx, ctx->d_page_alloc, s))) return rc;
    CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    return CLOAK_OK;
}

}  // namespace cloak
