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

namespace cloak {

namespace {

constexpr int MOE_MAX_K = 16;
constexpr int MOE_MAX_E = 1024;
constexpr int TILE_BYTES = 32768;  // 128 x 128 BF16

// top_k of one token's logits; stored index e' is logical expert gp[e']
__global__ void k_moe_route(const float *logits, const uint32_t *gp, int E, int K, int32_t *sel,
                            float *w, float *logits_out, int32_t *experts_out) {
    __shared__ float z[MOE_MAX_E];
    __shared__ int lid[MOE_MAX_E];
    __shared__ float bv[32];
    __shared__ int bi[32];
    __shared__ int pick[MOE_MAX_K];
    __shared__ float pz[MOE_MAX_K];
    const int m = blockIdx.x;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int l = gp ? (int)gp[e] : e;
        const float v = logits[(size_t)m * E + e];
        z[e] = v;
        lid[e] = l;
        if (logits_out) logits_out[(size_t)m * E + l] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = 0; j < K; ++j) {
        // best (largest logit, then smallest logical id) among unpicked
        float v = -INFINITY;
        int id = 0x7fffffff, at = -1;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            if (lid[e] < 0) continue;
            if (at < 0 || z[e] > v || (z[e] == v && lid[e] < id)) { v = z[e]; id = lid[e]; at = e; }
        }
        for (int o = 16; o; o >>= 1) {
            const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
            const int id2 = __shfl_xor_sync(0xffffffffu, id, o);
            const int at2 = __shfl_xor_sync(0xffffffffu, at, o);
            if (at2 >= 0 && (at < 0 || v2 > v || (v2 == v && id2 < id))) { v = v2; id = id2; at = at2; }
        }
        if (lane == 0) { bv[wid] = v; bi[wid] = at; }
        __syncthreads();
        if (threadIdx.x == 0) {
            int best = -1;
            for (int q = 0; q < nw; ++q) {
                const int a = bi[q];
                if (a < 0) continue;
                if (best < 0 || z[a] > z[best] || (z[a] == z[best] && lid[a] < lid[best])) best = a;
            }
            for (int e = 0; best < 0 && e < E; ++e)  // (only if every candidate compared false)
                if (lid[e] >= 0) best = e;
            pick[j] = lid[best];
            pz[j] = z[best];
            lid[best] = -1;  // taken
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
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

// Split-K GEMV over gathered 128x128 BF16 tiles: block b computes, for pair
// p (token m = p / K), matrix `mat` of the pair's expert, tile row nt, the
// partial dot products of its 128 rows over tile columns [kc*ks, ...).
// Thread t reads 8 elements (16 bytes) of rows it*16 + t/16, it = 0..7, at
// columns (t%16)*8; the 16 threads of a row reduce with shuffles.
struct GemvArgs {
    const uint8_t *wbase;
    const uint32_t *slot_of;
    const uint32_t *tab;      // [E][3] tensor bases (gate, up, down) of logical experts
    const int32_t *sel;       // [pairs] logical expert
    const __nv_bfloat16 *x;   // per pair row: x + (xrow_of_pair) * xs
    int x_per_token;          // 1: x row = token (p / K); 0: x row = pair p
    int K, xs;                // top_k; x row stride (elements)
    int mat0, nmat;           // which of gate/up/down: mat0 .. mat0 + nmat - 1
    int nt_n, kt_n, kc_n, ks; // tile rows, tile columns, K chunks, tiles per chunk
    float *part;              // [pairs][nmat][nt_n * 128][kc_n]
};

__global__ void __launch_bounds__(256) k_moe_gemv(GemvArgs a) {
    int b = blockIdx.x;
    const int kc = b % a.kc_n; b /= a.kc_n;
    const int nt = b % a.nt_n; b /= a.nt_n;
    const int mi = b % a.nmat;
    const int p = b / a.nmat;
    const int e = a.sel[p];
    const uint32_t base = a.tab[e * 3 + a.mat0 + mi];
    const __nv_bfloat16 *x = a.x + (size_t)(a.x_per_token ? p / a.K : p) * a.xs;
    const int t = threadIdx.x, c = (t & 15) * 8;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int k0 = kc * a.ks, k1 = min(a.kt_n, k0 + a.ks);
    for (int kt = k0; kt < k1; ++kt) {
        const uint32_t g = base + (uint32_t)(nt * a.kt_n + kt);
        const int64_t slot = a.slot_of ? (int64_t)__ldg(a.slot_of + g) : (int64_t)g;
        const uint4 *tile = reinterpret_cast<const uint4 *>(a.wbase + slot * TILE_BYTES);
        const uint4 xv = *reinterpret_cast<const uint4 *>(x + kt * 128 + c);
        uint4 wv[8];
#pragma unroll
        for (int it = 0; it < 8; ++it) wv[it] = __ldcs(tile + it * 256 + t);
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
    }
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        float v = acc[it];
        for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((t & 15) == 0) {
            const int row = nt * 128 + it * 16 + (t >> 4);
            a.part[(((size_t)p * a.nmat + mi) * a.nt_n * 128 + row) * a.kc_n + kc] = v;
        }
    }
}

// act[p][r] = bf16(silu(g) * u), g and u summed over the K chunks in order
__global__ void k_moe_act(const float *part, int F, int kc_n, int pairs, __nv_bfloat16 *act) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pairs * F) return;
    const int p = i / F, r = i % F;
    const float *pg = part + (((size_t)p * 2 + 0) * F + r) * kc_n;
    const float *pu = part + (((size_t)p * 2 + 1) * F + r) * kc_n;
    float g = 0.0f, u = 0.0f;
    for (int k = 0; k < kc_n; ++k) { g += pg[k]; u += pu[k]; }
    act[(size_t)p * F + r] = __float2bfloat16_rn(g / (1.0f + expf(-g)) * u);
}

// y[m][c] = sum_j w[m][j] * (sum_kc part[m*K + j][c][kc])
__global__ void k_moe_combine(const float *part, const float *w, int K, int D, int kc_n, int M, float *y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * D) return;
    const int m = i / D, c = i % D;
    float s = 0.0f;
    for (int j = 0; j < K; ++j) {
        const float *pp = part + ((size_t)(m * K + j) * D + c) * kc_n;
        float d = 0.0f;
        for (int k = 0; k < kc_n; ++k) d += pp[k];
        s = fmaf(w[m * K + j], d, s);
    }
    y[i] = s;
}

// K chunks so that the launch has about two CTAs per SM
int chunks_for(int blocks_per_chunk, int kt_n, int sms) {
    const int want = (2 * sms + blocks_per_chunk - 1) / blocks_per_chunk;
    return std::max(1, std::min(kt_n, want));
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
    const int pairs = M * K, FT = F / 128, DT = D / 128;
    const int kc1 = chunks_for(pairs * 2 * FT, DT, ctx->sm_count);
    const int kc2 = chunks_for(pairs * DT, FT, ctx->sm_count);
    auto r256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    const size_t b_tab = r256((size_t)E * 3 * 4), b_log = r256((size_t)M * E * 4), b_sel = r256((size_t)pairs * 4),
                 b_w = r256((size_t)pairs * 4), b_p1 = r256((size_t)pairs * 2 * F * kc1 * 4),
                 b_act = r256((size_t)pairs * F * 2), b_p2 = r256((size_t)pairs * D * kc2 * 4);
    const size_t need = b_tab + b_log + b_sel + b_w + b_p1 + b_act + b_p2;
    if (need > ctx->moe_ws_cap) {
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
        if (ctx->d_moe_ws) CLOAK_CUDA(ctx, cudaFree(ctx->d_moe_ws));
        ctx->d_moe_ws = nullptr;
        CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_moe_ws, need));
        ctx->moe_ws_cap = need;
        ctx->moe_tab.clear();
    }
    uint8_t *ws = (uint8_t *)ctx->d_moe_ws;
    uint32_t *d_tab = (uint32_t *)ws; ws += b_tab;
    float *logits = (float *)ws; ws += b_log;
    int32_t *sel = (int32_t *)ws; ws += b_sel;
    float *w = (float *)ws; ws += b_w;
    float *p1 = (float *)ws; ws += b_p1;
    __nv_bfloat16 *act = (__nv_bfloat16 *)ws; ws += b_act;
    float *p2 = (float *)ws;
    if (ctx->moe_tab != tab) {
        CLOAK_CUDA(ctx, cudaMemcpyAsync(d_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s));
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));  // the host copy may go away
        ctx->moe_tab = tab;
    }
    // 1. router logits (stored expert order)
    const int32_t rt_t[1] = {d->router};
    const void *xs[1] = {x};
    void *ys[1] = {logits};
    cloak_status rc = linear_batch_run(ctx, 1, rt_t, xs, ys, M, CLOAK_OUT_F32,
                                       flags & (CLOAK_LINEAR_UNCLOAKED | CLOAK_LINEAR_VMM), s);
    if (rc) return rc;
    // 2. routing
    k_moe_route<<<M, 256, 0, s>>>(logits, gp, E, K, sel, w, logits_out, experts_out);
    CLOAK_LAUNCHED(ctx);
    // 3-4. gate and up, act
    GemvArgs g{};
    g.wbase = weight_base(ctx, flags);
    g.slot_of = weight_slots(ctx, flags);
    g.tab = d_tab;
    g.sel = sel;
    g.x = (const __nv_bfloat16 *)x;
    g.x_per_token = 1;
    g.K = K;
    g.xs = D;
    g.mat0 = 0;
    g.nmat = 2;
    g.nt_n = FT;
    g.kt_n = DT;
    g.kc_n = kc1;
    g.ks = (DT + kc1 - 1) / kc1;
    g.part = p1;
    k_moe_gemv<<<pairs * 2 * FT * kc1, 256, 0, s>>>(g);
    CLOAK_LAUNCHED(ctx);
    k_moe_act<<<(pairs * F + 255) / 256, 256, 0, s>>>(p1, F, kc1, pairs, act);
    CLOAK_LAUNCHED(ctx);
    // 5. down
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
    k_moe_gemv<<<pairs * DT * kc2, 256, 0, s>>>(g);
    CLOAK_LAUNCHED(ctx);
    // 6. weighted sum
    k_moe_combine<<<(M * D + 255) / 256, 256, 0, s>>>(p2, w, K, D, kc2, M, y);
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

}  // namespace cloak
