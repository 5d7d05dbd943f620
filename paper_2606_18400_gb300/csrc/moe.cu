// moe.cu -- cloaked MoE FFN block (the paper's MoE model, Qwen3-30B-A3B
// shape: Section 5 "Setup and Hardware"; Table 2), decode-sized batches.
//
// Every expert matrix is a cloaked tensor, tiles placed and found through
// the gather table like any weight; the router's rows follow a keyed
// expert-order permutation, so its stored output e' scores logical expert
// perm[e'] and no router column says which tensors it selects.
//
//   1. router logits z = x Wr^T          the cloaked linear (tensor cores)
//   2. routing                          top_k by logit (equal logits: the
//                                       lower logical expert), weights = the
//                                       selected softmax probabilities
//                                       renormalised (FP32)
//   3. gate, up of the selected experts  split-K GEMV over gathered tiles
//   4. act = bf16(silu(g) * u)
//   5. down of the selected experts      split-K GEMV over gathered tiles
//   6. y = sum_j w_j down_j               fixed order: deterministic
//
// Steps 3 and 5 read each selected tile once per token: HBM-bound GEMVs
// (two FLOPs per weight), so they run on the CUDA cores with 16-byte loads
// rather than being padded out to tensor-core tiles; a token's experts
// are not shared with other tokens of the batch.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "ptx.cuh"

namespace cloak {

namespace {

constexpr int MOE_MAX_K = 16;
constexpr int MOE_MAX_E = 1024;
constexpr int TILE_BYTES = 32768;  // 128 x 128 BF16

// Sum of n <= N partials in index order (the order a plain loop takes),
// with all n loads issued before the first add: one memory round trip.
template <int N>
__device__ __forceinline__ float sum_partials(const float *p, int n) {
    float v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = i < n ? __ldcg(p + i) : 0.0f;
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < n) s += v[i];
    return s;
}

// Routing of token blockIdx.x: the router logit of stored expert e' is the
// sum of its split-K partials (one thread per expert), then warp 0 takes K
// rounds of a warp argmax (largest logit, then smallest logical id gp[e']),
// lane l holding e' = l + 32 i.
template <int PER>  // logits per lane: E <= 32 * PER
__global__ void __launch_bounds__(256) k_moe_route(const float *rpart, int rkc, const uint32_t *gp, int E,
                                                   int K, int32_t *sel, float *w, float *logits_out,
                                                   int32_t *experts_out) {
    __shared__ float zs[MOE_MAX_E];
    __shared__ int ls[MOE_MAX_E];
    __shared__ float pz[MOE_MAX_K];
    __shared__ int pick[MOE_MAX_K];
    griddep_launch_dependents();  // the gate/up launch may be scheduled now
    griddep_wait();               // the router partials are the previous kernel's
    const int m = blockIdx.x;
    const size_t R = (size_t)((E + 127) / 128) * 128;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const float v = sum_partials<16>(rpart + ((size_t)m * R + e) * rkc, rkc);
        const int l = gp ? (int)gp[e] : e;
        zs[e] = v;
        ls[e] = l;
        if (logits_out) logits_out[(size_t)m * E + l] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    float z[PER];
    int lid[PER];
    uint32_t taken = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = lane + 32 * i;
        const bool ok = e < E;
        z[i] = ok ? zs[e] : -INFINITY;
        lid[i] = ok ? ls[e] : 0x7fffffff;
        if (!ok) taken |= 1u << i;
    }
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
        float v = 0.0f;
        int id = 0x7fffffff, at = -1;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (taken & (1u << i)) continue;
            if (at < 0 || z[i] > v || (z[i] == v && lid[i] < id)) { v = z[i]; id = lid[i]; at = i; }
        }
        int owner = at >= 0 ? lane : 32;
        for (int o = 16; o; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int id2 = __shfl_xor_sync(0xffffffffu, id, o);
            const int ow2 = __shfl_xor_sync(0xffffffffu, owner, o);
            if (ow2 < 32 && (owner == 32 || v2 > v || (v2 == v && id2 < id))) { v = v2; id = id2; owner = ow2; }
        }
        // every lane holds the winner; its owner marks it taken
        if (owner == lane && at >= 0) taken |= 1u << at;
        if (lane == 0) { pz[j] = v; pick[j] = id; }
    }
    __syncwarp();
    if (lane == 0) {
        const float mx = pz[0];
        float s = 0.0f, ex[MOE_MAX_K];
        for (int j = 0; j < K; ++j) { ex[j] = expf(pz[j] - mx); s += ex[j]; }
        for (int j = 0; j < K; ++j) {
            sel[m * K + j] = pick[j];
            w[m * K + j] = ex[j] / s;
            if (experts_out) experts_out[m * K + j] = pick[j];
        }
    }
    }
}

// Split-K GEMV over gathered 128x128 BF16 tiles: block b computes, for item
// p, matrix mi, tile row nt, the partial dot products of its 128 rows over
// tile columns [kc*ks, ...). Thread t reads 8 elements (16 bytes) of rows
// it*16 + t/16, it = 0..7, at columns (t%16)*8; the 16 threads of a row
// reduce with shuffles. The next tile's loads are issued before the current
// tile is multiplied. Epilogues (the last of a group's blocks to arrive,
// found with a self-resetting counter, sums the group's partials in a fixed
// order): ROUTER none; GATE_UP act = bf16(silu(g) * u) for the tile row;
// DOWN y = sum_j w_j down_j for the tile row.
// The step's launches after the router are chained (programmatic dependent
// launches): ROUTER and DOWN trigger their dependents at entry; the routing
// kernel too; GATE_UP waits for the routing first and triggers only then, so
// the routing is final before any DOWN block starts. DOWN looks up its tiles
// and loads the first one (the rest of its chunk pulled into L2) before it
// waits for GATE_UP's activations.
enum { EP_ROUTER = 0, EP_GATE_UP = 1, EP_DOWN = 2 };

struct GemvArgs {
    const uint8_t *wbase;
    const uint32_t *slot_of;
    const uint32_t *tab;      // [E][3] tensor bases (gate, up, down) of logical experts
    const int32_t *sel;       // [pairs] logical expert
    uint32_t base0;           // ROUTER: the router's first tile
    const __nv_bfloat16 *x;   // x row of item p: x + (x_per_token ? p / K : p) * xs
    int x_per_token, K, xs;
    int mat0, nmat;           // expert matrices mat0 .. mat0 + nmat - 1 (0 gate, 1 up, 2 down)
    int nt_n, kt_n, kc_n, ks; // tile rows, tile columns, K chunks, tiles per chunk
    float *part;              // [items][nmat][nt_n * 128][kc_n]
    uint32_t *cnt;            // arrival counters (zero between launches)
    __nv_bfloat16 *act;       // GATE_UP out: [pairs][nt_n * 128]
    const float *w;           // DOWN: routing weights [M][K]
    float *y;                 // DOWN out: [M][nt_n * 128]
    int rows;                 // valid rows (d_ff or d_model)
};

// MINB: CTAs per SM the registers allow (2: about 100 registers; 3: 80, a few
// spilled, the variant for batches of more than one token, whose experts
// fill one wave of three CTAs per SM where two would need two waves)
template <int EP, int MINB = 2>
__global__ void __launch_bounds__(256, MINB) k_moe_gemv(GemvArgs a) {
    int b = blockIdx.x;
    const int kc = b % a.kc_n; b /= a.kc_n;
    const int nt = b % a.nt_n; b /= a.nt_n;
    const int mi = b % a.nmat;
    const int p = b / a.nmat;
    if constexpr (EP == EP_GATE_UP) {
        griddep_wait();               // the routing
        griddep_launch_dependents();  // DOWN may start: the routing is final
    } else {
        griddep_launch_dependents();
    }
    const uint32_t base = EP == EP_ROUTER ? a.base0 : a.tab[__ldcg(a.sel + p) * 3 + a.mat0 + mi];
    const __nv_bfloat16 *x = a.x + (size_t)(a.x_per_token ? p / a.K : p) * a.xs;
    const int t = threadIdx.x, c = (t & 15) * 8;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int k0 = kc * a.ks, k1 = min(a.kt_n, k0 + a.ks);
    // the chunk's gather-table entries, looked up in parallel up front so
    // that no tile's loads wait on its own lookup
    __shared__ uint32_t slots[16];
    if (t < k1 - k0) {
        const uint32_t g = base + (uint32_t)(nt * a.kt_n + k0 + t);
        slots[t] = a.slot_of ? __ldg(a.slot_of + g) : g;
    }
    __syncthreads();
    auto tile_of = [&](int kt) {
        return reinterpret_cast<const uint4 *>(a.wbase + (int64_t)slots[kt - k0] * TILE_BYTES);
    };
    uint4 wv[8];
    if (k0 < k1) {
        const uint4 *tile = tile_of(k0);
#pragma unroll
        for (int it = 0; it < 8; ++it) wv[it] = __ldcs(tile + it * 256 + t);
    }
    if constexpr (EP == EP_DOWN) {
        // the chunk's other tiles into L2 (one 128-byte line per thread per tile)
        for (int kt = k0 + 1; kt < k1; ++kt)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const uint8_t *>(tile_of(kt)) + t * 128));
    }
    if constexpr (EP != EP_GATE_UP) griddep_wait();  // x / act: the previous kernel's
    for (int kt = k0; kt < k1; ++kt) {
        uint4 nv[8];
        if (kt + 1 < k1) {
            const uint4 *tile = tile_of(kt + 1);
#pragma unroll
            for (int it = 0; it < 8; ++it) nv[it] = __ldcs(tile + it * 256 + t);
        }
        const uint4 xv = *reinterpret_cast<const uint4 *>(x + kt * 128 + c);
        const __nv_bfloat162 *xp = reinterpret_cast<const __nv_bfloat162 *>(&xv);
        float2 xf[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) xf[q] = __bfloat1622float2(xp[q]);
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const __nv_bfloat162 *wp = reinterpret_cast<const __nv_bfloat162 *>(&wv[it]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 wf = __bfloat1622float2(wp[q]);
                acc[it] = fmaf(wf.x, xf[q].x, acc[it]);
                acc[it] = fmaf(wf.y, xf[q].y, acc[it]);
            }
        }
        if (kt + 1 < k1) {
#pragma unroll
            for (int it = 0; it < 8; ++it) wv[it] = nv[it];
        }
    }
    const int R = a.nt_n * 128;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        float v = acc[it];
        for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 15) == 0) {
            const int row = nt * 128 + it * 16 + (t >> 4);
            a.part[(((size_t)p * a.nmat + mi) * R + row) * a.kc_n + kc] = v;
        }
    }
    if constexpr (EP != EP_ROUTER) {
        // group: (pair, tile row) for GATE_UP, (token, tile row) for DOWN
        const int grp = EP == EP_GATE_UP ? p * a.nt_n + nt : (p / a.K) * a.nt_n + nt;
        const uint32_t expect = EP == EP_GATE_UP ? 2u * a.kc_n : (uint32_t)(a.K * a.kc_n);
        __shared__ int last;
        __threadfence();  // this block's partials before its arrival
        __syncthreads();  // (also: every thread is past its last use of slots)
        if (t == 0) last = atomicAdd(a.cnt + grp, 1u) == expect - 1;
        __syncthreads();
        if (!last) return;
        __threadfence();
        if (t < 128) {
            const int row = nt * 128 + t;
            if constexpr (EP == EP_GATE_UP) {
                const float g = sum_partials<16>(a.part + (((size_t)p * 2 + 0) * R + row) * a.kc_n, a.kc_n);
                const float u = sum_partials<16>(a.part + (((size_t)p * 2 + 1) * R + row) * a.kc_n, a.kc_n);
                a.act[(size_t)p * R + row] = __float2bfloat16_rn(g / (1.0f + expf(-g)) * u);
            } else {
                const int m = p / a.K;
                float d[MOE_MAX_K];
#pragma unroll
                for (int j = 0; j < MOE_MAX_K; ++j)
                    d[j] = j < a.K ? sum_partials<4>(a.part + ((size_t)(m * a.K + j) * R + row) * a.kc_n, a.kc_n)
                                   : 0.0f;
                float sacc = 0.0f;
#pragma unroll
                for (int j = 0; j < MOE_MAX_K; ++j)
                    if (j < a.K) sacc = fmaf(a.w[m * a.K + j], d[j], sacc);
                if (row < a.rows) a.y[(size_t)m * a.rows + row] = sacc;
            }
        }
        if (t == 0) a.cnt[grp] = 0;  // ready for the next launch
    }
}

// K chunks (at most `cap`: the epilogues' unrolled sums): the count whose
// waves of `per_sm` CTAs per SM take the least time, a block costing its
// tiles plus about three tiles' worth of fixed latency (table lookup, first
// load, arrival); fewer chunks on a tie
int chunks_for(int blocks_per_chunk, int kt_n, int sms, int cap, int per_sm) {
    int best = 1;
    long best_t = -1;
    for (int kc = 1; kc <= std::min(kt_n, cap); ++kc) {
        const int ks = (kt_n + kc - 1) / kc;
        if ((kt_n + ks - 1) / ks != kc) continue;  // the same split as a smaller count
        const long waves = ((long)blocks_per_chunk * kc + per_sm * sms - 1) / ((long)per_sm * sms);
        const long t = waves * (ks + 3);
        if (best_t < 0 || t < best_t) {
            best_t = t;
            best = kc;
        }
    }
    return best;
}

}  // namespace

cloak_status moe_run(cloak_ctx *ctx, const cloak_moe_desc *d, const void *x, float *y, int M, int flags,
                     int32_t *experts_out, float *logits_out, cudaStream_t s) {
    const int E = d->n_experts, K = d->top_k, D = d->d_model, F = d->d_ff;
    const int T = (int)ctx->tensors.size();
    if (ctx->dtype != CLOAK_BF16 || ctx->tile_r != 128 || ctx->tile_c != 128) return CLOAK_E_UNSUPPORTED;
    if (E < 1 || E > MOE_MAX_E || K < 1 || K > std::min(E, MOE_MAX_K) || D % 128 || F % 128 || D <= 0 ||
        F <= 0 || M < 1 || M > 64 || d->router < 0 || d->router >= T || !d->expert_tensors)
        return CLOAK_E_INVAL;
    const cloak_tensor_desc &rt = ctx->tensors[d->router];
    if (rt.n != E || rt.k != D) return CLOAK_E_INVAL;
    const uint32_t *gp = nullptr;
    if (d->expert_group >= 0) {
        if (d->expert_group >= (int)ctx->groups.size() || rt.perm_group != d->expert_group ||
            rt.perm_axis != 0 || ctx->groups[d->expert_group].n_units != E ||
            ctx->groups[d->expert_group].unit != 1)
            return CLOAK_E_INVAL;
        gp = ctx->d_group_perm + ctx->goff[d->expert_group];
    } else if (rt.perm_group >= 0) {
        return CLOAK_E_INVAL;  // permuted router rows need their group
    }
    // expert table: tensor bases of (gate, up, down) per logical expert,
    // uploaded when the descriptor or the layout changed
    std::vector<uint32_t> tab((size_t)E * 3);
    for (int e = 0; e < E; ++e)
        for (int q = 0; q < 3; ++q) {
            const int t = d->expert_tensors[e * 3 + q];
            if (t < 0 || t >= T) return CLOAK_E_INVAL;
            const cloak_tensor_desc &td = ctx->tensors[t];
            if (q < 2 ? (td.n != F || td.k != D) : (td.n != D || td.k != F)) return CLOAK_E_INVAL;
            tab[e * 3 + q] = ctx->h_tensor_base[t];
        }
    const int pairs = M * K, FT = F / 128, DT = D / 128, ET = (E + 127) / 128;
    // K chunks of at most 16 tiles (the gather-table entries a block looks
    // up front) and at most 16 (router, gate/up) or 4 (down) per row, the
    // epilogues' unrolled sums
    auto fit16 = [](int kc, int kt_n) { return std::max(kc, (kt_n + 15) / 16); };
    const int rkc = std::min(DT, 16);
    // one token: two CTAs per SM; more: three (measured: M = 1 37.4 vs 39.4 us,
    // M = 4 76 vs 81.7 us)
    const int per_sm = M == 1 ? 2 : 3;
    const int kc1 = fit16(chunks_for(pairs * 2 * FT, DT, ctx->sm_count, 16, per_sm), DT);
    const int kc2 = fit16(chunks_for(pairs * DT, FT, ctx->sm_count, 4, per_sm), FT);
    if (rkc < (DT + 15) / 16 || kc1 > 16 || kc2 > 4) return CLOAK_E_UNSUPPORTED;  // d_model > 32768 or d_ff > 8192
    auto r256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t b_tab = r256((size_t)E * 3 * 4), b_cnt = r256((size_t)64 * (FT * MOE_MAX_K + DT) * 4),
                 b_rp = r256((size_t)M * ET * 128 * rkc * 4), b_sel = r256((size_t)pairs * 4),
                 b_w = r256((size_t)pairs * 4), b_p1 = r256((size_t)pairs * 2 * F * kc1 * 4),
                 b_act = r256((size_t)pairs * F * 2), b_p2 = r256((size_t)pairs * D * kc2 * 4);
    const size_t need = b_tab + b_cnt + b_rp + b_sel + b_w + b_p1 + b_act + b_p2;
    if (need > ctx->moe_ws_cap) {
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
        if (ctx->d_moe_ws) CLOAK_CUDA(ctx, cudaFree(ctx->d_moe_ws));
        ctx->d_moe_ws = nullptr;
        CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_moe_ws, need));
        CLOAK_CUDA(ctx, cudaMemsetAsync(ctx->d_moe_ws, 0, b_tab + b_cnt, s));  // counters start at zero
        ctx->moe_ws_cap = need;
        ctx->moe_tab.clear();
    }
    uint8_t *ws = (uint8_t *)ctx->d_moe_ws;
    uint32_t *d_tab = (uint32_t *)ws; ws += b_tab;
    uint32_t *cnt = (uint32_t *)ws; ws += b_cnt;
    float *rp = (float *)ws; ws += b_rp;
    int32_t *sel = (int32_t *)ws; ws += b_sel;
    float *w = (float *)ws; ws += b_w;
    float *p1 = (float *)ws; ws += b_p1;
    __nv_bfloat16 *act = (__nv_bfloat16 *)ws; ws += b_act;
    float *p2 = (float *)ws;
    if (ctx->moe_tab != tab) {
        // a new descriptor may place the counters elsewhere: zero them
        CLOAK_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
        CLOAK_CUDA(ctx, cudaMemcpyAsync(d_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s));
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));  // the host copy may go away
        ctx->moe_tab = tab;
    }
    GemvArgs g{};
    g.wbase = weight_base(ctx, flags);
    g.slot_of = weight_slots(ctx, flags);
    g.tab = d_tab;
    g.sel = sel;
    g.K = K;
    // 1. router partials (stored expert order), one tile per block
    g.base0 = ctx->h_tensor_base[d->router];
    g.x = (const __nv_bfloat16 *)x;
    g.x_per_token = 0;
    g.xs = D;
    g.nmat = 1;
    g.nt_n = ET;
    g.kt_n = DT;
    g.kc_n = rkc;
    g.ks = (DT + rkc - 1) / rkc;
    g.part = rp;
    // (an ordinary launch: the kernel before it may have written the weights)
    k_moe_gemv<EP_ROUTER><<<M * ET * rkc, 256, 0, s>>>(g);
    CLOAK_LAUNCHED(ctx);
    // 2. routing (this and the later launches are chained)
    auto route = E <= 128 ? k_moe_route<4> : E <= 256 ? k_moe_route<8> : k_moe_route<32>;
    CLOAK_CUDA(ctx, launch_k(true, route, dim3(M), dim3(256), 0, s, (const float *)rp, rkc, gp, E, K, sel, w,
                             logits_out, experts_out));
    CLOAK_LAUNCHED(ctx);
    // 3-4. gate and up of the selected experts; the last block of a tile row writes act
    g.x_per_token = 1;
    g.mat0 = 0;
    g.nmat = 2;
    g.nt_n = FT;
    g.kt_n = DT;
    g.kc_n = kc1;
    g.ks = (DT + kc1 - 1) / kc1;
    g.part = p1;
    g.cnt = cnt;
    g.act = act;
    g.rows = F;
    CLOAK_CUDA(ctx, launch_k(true, per_sm == 2 ? k_moe_gemv<EP_GATE_UP, 2> : k_moe_gemv<EP_GATE_UP, 3>,
                             dim3(pairs * 2 * FT * kc1), dim3(256), 0, s, g));
    CLOAK_LAUNCHED(ctx);
    // 5-6. down; the last block of a token's tile row writes y
    g.x = act;
    g.x_per_token = 0;
    g.xs = F;
    g.mat0 = 2;
    g.nmat = 1;
    g.nt_n = DT;
    g.kt_n = FT;
    g.kc_n = kc2;
    g.ks = (FT + kc2 - 1) / kc2;
    g.part = p2;
    g.cnt = cnt + 64 * FT * MOE_MAX_K;
    g.w = w;
    g.y = y;
    g.rows = D;
    CLOAK_CUDA(ctx, launch_k(true, per_sm == 2 ? k_moe_gemv<EP_DOWN, 2> : k_moe_gemv<EP_DOWN, 3>,
                             dim3(pairs * DT * kc2), dim3(256), 0, s, g));
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

}  // namespace cloak
