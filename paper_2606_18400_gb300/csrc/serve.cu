// serve.cu -- one forward step of a continuously batched LLaMA-style model
// over the cloaked arena: a mixed batch of prefill-chunk and decode tokens of
// many requests, with a paged KV cache (the serving loop of the host decides
// the batch; this file runs it on the device).
//
// Per layer, tokens independent except through their own request's KV cache:
//   x = rmsnorm(h); q, k, v = cloaked linears of x; RoPE(q, k); k, v -> cache;
//   a = causal attention of q over its request's cached keys/values (GQA);
//   h += cloaked o(a); x = rmsnorm(h); g, u = cloaked gate/up of x;
//   h += cloaked down(silu(g) * u)
// then logits = cloaked lm_head(rmsnorm(h)) at the sampled rows, greedy argmax.
// Every token's result depends only on its own inputs and its request's cache
// (the linears' split does not depend on the batch size), so a request gets
// the same numbers alone and in a mix.
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cmath>

#include "internal.cuh"
#include "ptx.cuh"

namespace cloak {

// Every kernel of a step: the next kernel may be scheduled at once (it waits
// for this one's completion before it reads this one's outputs), and this one
// waits for the previous kernel's completion before it reads anything.
// Without a programmatic dependent launch both are no-ops.
__device__ __forceinline__ void chain_enter() {
    griddep_launch_dependents();
    griddep_wait();
}

static inline unsigned nb(size_t n, unsigned b = 256) { return (unsigned)((n + b - 1) / b); }

// The step's linears over rows [0, M): decode rows [0, m_dec) through the
// split-K decode kernel, prompt rows [m_dec, M) through the whole-tile
// prefill GEMM. Each kernel's summation order depends on the weights only, so
// a row's result does not depend on the rest of the batch.
static cloak_status step_linears(cloak_ctx *ctx, int n, const int32_t *ts, const void *const *xs,
                                 void *const *ys, int M, int m_dec, int out_dtype, int flags, cudaStream_t s) {
    cloak_status rc = CLOAK_OK;
    if (m_dec > 0 && (rc = linear_batch_run(ctx, n, ts, xs, ys, m_dec, out_dtype, flags, s))) return rc;
    if (M > m_dec) {
        const int oes = out_dtype == CLOAK_OUT_F32 ? 4 : 2;
        const void *xp[8];
        void *yp[8];
        for (int i = 0; i < n; ++i) {
            const TensorInfo &ti = ctx->info[ts[i]];
            xp[i] = (const uint8_t *)xs[i] + (size_t)m_dec * ti.k * 2;
            yp[i] = (uint8_t *)ys[i] + (size_t)m_dec * ti.n * oes;
        }
        rc = gemm_run(ctx, n, ts, xp, nullptr, yp, M - m_dec, out_dtype == CLOAK_OUT_F32, 0,
                      weight_slots(ctx, flags), weight_map(ctx, flags), s);
    }
    return rc;
}

// token ids outside [0, V) give a zero row
__global__ void k_embed(const __nv_bfloat16 *emb, const int32_t *ids, int D, int V, float *h) {
    chain_enter();
    const int m = blockIdx.x;
    const int id = ids[m];
    if ((unsigned)id >= (unsigned)V) {
        for (int c = threadIdx.x; c < D; c += blockDim.x) h[(size_t)m * D + c] = 0.0f;
        return;
    }
    const __nv_bfloat16 *e = emb + (size_t)id * D;
    for (int c = threadIdx.x; c < D; c += blockDim.x) h[(size_t)m * D + c] = __bfloat162float(e[c]);
}

// Cloaked embedding: token id's row is row id % 128 of tile row id / 128 of
// the embedding tensor; column c sits in tile column c / 128. Each tile is
// found through the gather table (nullptr: the uncloaked twin, tile g at
// slot g); 16-byte loads of 8 BF16 columns.
__global__ void k_embed_tiled(const uint8_t *wbase, const uint32_t *slot_of, uint32_t base, int kt,
                              const int32_t *ids, int D, int V, float *h) {
    chain_enter();
    const int m = blockIdx.x;
    const int id = ids[m];
    if ((unsigned)id >= (unsigned)V) {
        for (int c = threadIdx.x; c < D; c += blockDim.x) h[(size_t)m * D + c] = 0.0f;
        return;
    }
    const int64_t tr = id / 128, r = id % 128;
    for (int c8 = threadIdx.x; c8 * 8 < D; c8 += blockDim.x) {
        const int c = c8 * 8;
        const uint32_t g = base + (uint32_t)(tr * kt + c / 128);
        const int64_t slot = slot_of ? (int64_t)__ldg(slot_of + g) : (int64_t)g;
        const uint4 v = *reinterpret_cast<const uint4 *>(wbase + slot * 32768 + (r * 128 + c % 128) * 2);
        const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(&v);
        float *o = h + (size_t)m * D + c;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float2 f = __bfloat1622float2(p[j]);
            o[2 * j] = f.x;
            o[2 * j + 1] = f.y;
        }
    }
}

// x = bf16(h * r), r = 1/sqrt(mean(h^2) + eps); optional row subset
__global__ void k_rmsnorm(const float *h, const int32_t *rows, int D, float eps, __nv_bfloat16 *x) {
    chain_enter();
    const int m = blockIdx.x;
    const int src = rows ? rows[m] : m;
    const float *hr = h + (size_t)src * D;
    float ss = 0.0f;
    for (int c = threadIdx.x; c < D; c += blockDim.x) ss += hr[c] * hr[c];
    __shared__ float red[32];
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x < 32) {
        ss = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (threadIdx.x == 0) red[0] = rsqrtf(ss / (float)D + eps);
    }
    __syncthreads();
    const float r = red[0];
    for (int c = threadIdx.x; c < D; c += blockDim.x) x[(size_t)m * D + c] = __float2bfloat16_rn(hr[c] * r);
}

// Residual add and RMSNorm in one pass over a token's row: h += y (y may be
// null), then x = bf16(h * r), r = 1/sqrt(mean(h^2) + eps). Block i takes
// token rows[i] (rows null: token i) and writes x row i. 16-byte loads; the
// row (d_model a multiple of 4, at most 256 * 4 * VR) stays in registers.
// The sum of squares: each thread's own values in column order, then a
// fixed tree over the lanes and the warps, so a token's result does not
// depend on the batch.
template <int VR>
__global__ void __launch_bounds__(256) k_add_rmsnorm(float *h, const float *y, const int32_t *rows, int D,
                                                     float eps, __nv_bfloat16 *x) {
    chain_enter();
    const int i = blockIdx.x, t = threadIdx.x;
    const int src = rows ? rows[i] : i;
    float4 *hr = reinterpret_cast<float4 *>(h + (size_t)src * D);
    const float4 *yr = y ? reinterpret_cast<const float4 *>(y + (size_t)src * D) : nullptr;
    const int D4 = D / 4;
    float4 v[VR];
#pragma unroll
    for (int k = 0; k < VR; ++k) {
        const int c = k * 256 + t;
        v[k] = c < D4 ? hr[c] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (yr) {
#pragma unroll
        for (int k = 0; k < VR; ++k) {
            const int c = k * 256 + t;
            if (c < D4) {
                const float4 a = yr[c];
                v[k].x += a.x;
                v[k].y += a.y;
                v[k].z += a.z;
                v[k].w += a.w;
                hr[c] = v[k];
            }
        }
    }
    float ss = 0.0f;
#pragma unroll
    for (int k = 0; k < VR; ++k)
        ss = fmaf(v[k].w, v[k].w, fmaf(v[k].z, v[k].z, fmaf(v[k].y, v[k].y, fmaf(v[k].x, v[k].x, ss))));
    __shared__ float red[8];
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((t & 31) == 0) red[t >> 5] = ss;
    __syncthreads();
    ss = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
    const float r = rsqrtf(ss / (float)D + eps);
    uint2 *xr = reinterpret_cast<uint2 *>(x + (size_t)i * D);
#pragma unroll
    for (int k = 0; k < VR; ++k) {
        const int c = k * 256 + t;
        if (c < D4) {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(v[k].x * r, v[k].y * r);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(v[k].z * r, v[k].w * r);
            xr[c] = make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
        }
    }
}
constexpr int NORM_VR = 8;  // d_model up to 8192 in registers

// RoPE (rotate-half pairs (i, i+64) of a 128-dim head, angle pos * theta^(-i/64))
// on q and k; k and v written to the paged cache [block][16][n_kv][128].
// One block per token: the 64 angles of its position are computed once and
// shared by all its heads; a thread rotates 8 pairs of one head (16-byte
// loads and stores of each half).
__device__ __forceinline__ void rope8(uint4 &lo, uint4 &hi, const float *cs, const float *sn) {
    __nv_bfloat162 *l2 = reinterpret_cast<__nv_bfloat162 *>(&lo);
    __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(&hi);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 a = __bfloat1622float2(l2[j]), b = __bfloat1622float2(h2[j]);
        const float c0 = cs[2 * j], s0 = sn[2 * j], c1 = cs[2 * j + 1], s1 = sn[2 * j + 1];
        l2[j] = __floats2bfloat162_rn(a.x * c0 - b.x * s0, a.y * c1 - b.y * s1);
        h2[j] = __floats2bfloat162_rn(b.x * c0 + a.x * s0, b.y * c1 + a.y * s1);
    }
}

__global__ void __launch_bounds__(256) k_rope_cache(__nv_bfloat16 *q, const __nv_bfloat16 *k,
                                                    const __nv_bfloat16 *v, const int32_t *pos,
                                                    const int32_t *req, const int32_t *btab, int max_blocks,
                                                    int HQ, int HKV, float theta, __nv_bfloat16 *kc,
                                                    __nv_bfloat16 *vc) {
    chain_enter();
    __shared__ float cs_s[64], sn_s[64];
    const int m = blockIdx.x;
    const int p = pos[m];
    if (threadIdx.x < 64) {
        const int i = threadIdx.x;
        const float freq = powf(theta, -(float)i / 64.0f);
        sincosf((float)p * freq, &sn_s[i], &cs_s[i]);
    }
    __syncthreads();
    const int blk = HKV > 0 ? btab[(size_t)req[m] * max_blocks + p / 16] : 0;
    for (int w = threadIdx.x; w < (HQ + HKV) * 8; w += blockDim.x) {
        const int head = w >> 3, i0 = (w & 7) * 8;  // pairs i0 .. i0 + 7
        if (head < HQ) {
            uint4 *qh = reinterpret_cast<uint4 *>(q + ((size_t)m * HQ + head) * 128);
            uint4 lo = qh[i0 / 8], hi = qh[8 + i0 / 8];
            rope8(lo, hi, cs_s + i0, sn_s + i0);
            qh[i0 / 8] = lo;
            qh[8 + i0 / 8] = hi;
        } else {
            const int kh = head - HQ;  // < HKV
            const uint4 *kr = reinterpret_cast<const uint4 *>(k + ((size_t)m * HKV + kh) * 128);
            const uint4 *vr = reinterpret_cast<const uint4 *>(v + ((size_t)m * HKV + kh) * 128);
            const size_t off = (((size_t)blk * 16 + p % 16) * HKV + kh) * 128;
            uint4 lo = kr[i0 / 8], hi = kr[8 + i0 / 8];
            rope8(lo, hi, cs_s + i0, sn_s + i0);
            uint4 *kd = reinterpret_cast<uint4 *>(kc + off);
            uint4 *vd = reinterpret_cast<uint4 *>(vc + off);
            kd[i0 / 8] = lo;
            kd[8 + i0 / 8] = hi;
            vd[i0 / 8] = vr[i0 / 8];
            vd[8 + i0 / 8] = vr[8 + i0 / 8];
        }
    }
}

// Causal attention of single queries (decode tokens), split over the keys:
// block (split, row, head) takes keys [128 split, 128 split + 128) of token
// m = rows[row]; each of its 4 warps 32 of them, 8 at a time (8 keys lie in
// one 16-key block of the cache: one table entry per batch). A lane holds 4
// of the 128 dimensions: K and V rows are read as 256-byte coalesced warp
// loads, 16 of them in flight per lane; scores are warp sums. Online softmax
// in FP32 per warp, merged across the warps in shared memory. A token with
// one split writes its output; otherwise the block writes (max, sum,
// acc[128]) and the last of the token's blocks to finish (an arrival count
// per token and head) merges the splits in order. The split depends only on
// the token's own position, so the result does not depend on the batch.
constexpr int ATT_SPLIT = 128;
constexpr int ATT_PART = 132;  // floats per partial: max, sum, pad, acc[128]
constexpr int ATT_GRID_X = 16;  // blocks per (token, head); longer contexts loop

__global__ void __launch_bounds__(128) k_attn_decode(const __nv_bfloat16 *q, const __nv_bfloat16 *kc,
                                                     const __nv_bfloat16 *vc, const int32_t *pos,
                                                     const int32_t *req, const int32_t *btab,
                                                     const int32_t *rows, int max_blocks, int HQ,
                                                     int HKV, int max_splits, float *part,
                                                     uint32_t *cnt, __nv_bfloat16 *out) {
    chain_enter();
    const int r = blockIdx.y, j = blockIdx.z;
    const int m = rows ? rows[r] : r;
    const int n = pos[m] + 1;
    const int nsplit = (n + ATT_SPLIT - 1) / ATT_SPLIT;
    if ((int)blockIdx.x >= nsplit) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
    const int kvh = j / (HQ / HKV);
    const int32_t *bt = btab + (size_t)req[m] * max_blocks;
    float qd[4];
    {
        const uint2 raw = *reinterpret_cast<const uint2 *>(q + ((size_t)m * HQ + j) * 128 + 4 * lane);
        const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&raw);
        const float2 a = __bfloat1622float2(h2[0]), b = __bfloat1622float2(h2[1]);
        const float sc = 0.08838834764831845f;  // 1/sqrt(128)
        qd[0] = a.x * sc; qd[1] = a.y * sc; qd[2] = b.x * sc; qd[3] = b.y * sc;
    }
    __shared__ float wm[4], wl[4];
    __shared__ float wa[4][128];
    __shared__ int last;
    float *pb = part + ((size_t)r * HQ + j) * max_splits * ATT_PART;
    // a block takes splits blockIdx.x, blockIdx.x + gridDim.x, ...; each
    // split's arithmetic is the same whichever block takes it
    for (int sp = blockIdx.x; sp < nsplit; sp += gridDim.x) {
        const int k_begin = sp * ATT_SPLIT + w * (ATT_SPLIT / 4);
        const int k_end = min(n, k_begin + ATT_SPLIT / 4);
        float mx = -FLT_MAX, sum = 0.0f, acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        const bool hi = (lane >> 4) & 1;
        const size_t kstr = (size_t)HKV * 128;  // elements between consecutive keys of a cache block
        for (int kb = k_begin; kb < k_end; kb += 8) {
            // kb is a multiple of 8: the 8 keys lie in one 16-key block of the cache
            const size_t base = (((size_t)bt[kb >> 4] * 16 + (kb & 15)) * HKV + kvh) * 128 + 4 * lane;
            uint2 kr[8], vr[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const size_t off = base + (size_t)(min(kb + i, k_end - 1) - kb) * kstr;
                kr[i] = *reinterpret_cast<const uint2 *>(kc + off);
                vr[i] = *reinterpret_cast<const uint2 *>(vc + off);
            }
            float s[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&kr[i]);
                const float2 a = __bfloat1622float2(h2[0]), b = __bfloat1622float2(h2[1]);
                s[i] = fmaf(qd[0], a.x, fmaf(qd[1], a.y, fmaf(qd[2], b.x, qd[3] * b.y)));
            }
            // sums over the 32 lanes: lane bit 4 splits the keys 4/4 (each half
            // keeps its four and adds the partner's copy of them), bits 3..0
            // finish the sums, and one exchange gives every lane all eight
            {
                float t4[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float mine = hi ? s[i + 4] : s[i], give = hi ? s[i] : s[i + 4];
                    t4[i] = mine + __shfl_xor_sync(0xffffffffu, give, 16);
                }
#pragma unroll
                for (int o = 8; o; o >>= 1) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) t4[i] += __shfl_xor_sync(0xffffffffu, t4[i], o);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float other = __shfl_xor_sync(0xffffffffu, t4[i], 16);
                    s[i] = hi ? other : t4[i];
                    s[i + 4] = hi ? t4[i] : other;
                }
            }
            float cm = mx;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (kb + i >= k_end) s[i] = -FLT_MAX;
                cm = fmaxf(cm, s[i]);
            }
            const float scale = expf(mx - cm);
            sum *= scale;
#pragma unroll
            for (int d = 0; d < 4; ++d) acc[d] *= scale;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float p = kb + i < k_end ? expf(s[i] - cm) : 0.0f;
                sum += p;
                const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&vr[i]);
                const float2 a = __bfloat1622float2(h2[0]), b = __bfloat1622float2(h2[1]);
                acc[0] = fmaf(p, a.x, acc[0]);
                acc[1] = fmaf(p, a.y, acc[1]);
                acc[2] = fmaf(p, b.x, acc[2]);
                acc[3] = fmaf(p, b.y, acc[3]);
            }
            mx = cm;
        }
        // merge the four warps
        if (lane == 0) { wm[w] = mx; wl[w] = sum; }
#pragma unroll
        for (int d = 0; d < 4; ++d) wa[w][4 * lane + d] = acc[d];
        __syncthreads();
        float M = -FLT_MAX;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (wl[v] > 0.0f) M = fmaxf(M, wm[v]);
        float L = 0.0f, A = 0.0f;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (wl[v] > 0.0f) {
                const float e = expf(wm[v] - M);
                L = fmaf(wl[v], e, L);
                A = fmaf(wa[v][t], e, A);
            }
        }
        if (nsplit == 1) {
            out[((size_t)m * HQ + j) * 128 + t] = __float2bfloat16_rn(A / L);
            return;
        }
        float *pp = pb + sp * ATT_PART;
        if (t == 0) { pp[0] = M; pp[1] = L; }
        pp[4 + t] = A;
        // the last split of (token, head) to finish merges all of them, in
        // split order (the same arithmetic whichever block it is), and resets
        // the count; its arrival is the block's last (every split has arrived)
        // (the block's stores are ordered before thread 0's fence by the
        // barrier; the fence makes them visible before the arrival)
        __syncthreads();  // also: wm, wl, wa are free for the next split
        if (t == 0) {
            __threadfence();
            last = atomicAdd(cnt + (size_t)r * HQ + j, 1u) == (uint32_t)nsplit - 1;
            if (last) __threadfence();
        }
        __syncthreads();
        if (last) break;
    }
    if (nsplit == 1 || !last) return;
    float Mx = -FLT_MAX;
    for (int q = 0; q < nsplit; ++q) Mx = fmaxf(Mx, __ldcg(pb + q * ATT_PART));
    float Ls = 0.0f, As = 0.0f;
    for (int q = 0; q < nsplit; ++q) {
        const float e = expf(__ldcg(pb + q * ATT_PART) - Mx);
        Ls = fmaf(__ldcg(pb + q * ATT_PART + 1), e, Ls);
        As = fmaf(__ldcg(pb + q * ATT_PART + 4 + t), e, As);
    }
    out[((size_t)m * HQ + j) * 128 + t] = __float2bfloat16_rn(As / Ls);
    if (t == 0) cnt[(size_t)r * HQ + j] = 0u;
}

// Query-tiled causal attention for runs of consecutive tokens of one request
// (prefill chunks), on the tensor cores: a block takes up to 64 queries of
// one head, 16 per warp. Per 64-key tile (starting at absolute multiples of
// 64, so a query's result does not depend on the batch it is in): K and V
// land in shared memory through cp.async (two buffers, the next tile in
// flight while this one is used; 16-byte chunks XOR-swizzled by row), S =
// Q K^T with warp-level BF16 MMAs (m16n8k16, FP32 accumulate), causal mask,
// online softmax in FP32 (exp2 with the 1/sqrt(128) scale folded in), then
// O += P V with P taken from the S registers as BF16 and V fragments read
// transposed from shared memory. tiles: [n][3] = (first batch token, query
// count, -); query i of a tile is batch token first + i, positions
// consecutive.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// byte offset of 16-byte chunk c of row r in a [64][256-byte] tile
__device__ __forceinline__ uint32_t att_sw(int r, int c) { return (uint32_t)(r * 256 + ((c ^ (r & 7)) << 4)); }

constexpr int ATT_TILE_BYTES = 64 * 256;  // 64 keys x 128 BF16 dims

__global__ void __launch_bounds__(128) k_attention_tiled(const __nv_bfloat16 *q, const __nv_bfloat16 *kc,
                                                         const __nv_bfloat16 *vc, const int32_t *pos,
                                                         const int32_t *req, const int32_t *btab,
                                                         const int32_t *tiles, int max_blocks, int HQ,
                                                         int HKV, __nv_bfloat16 *out) {
    chain_enter();
    extern __shared__ __align__(128) uint8_t att_smem[];  // [2 buffers][K tile, V tile]
    // blocks start in list order, all heads of a tile together: a list with
    // the latest positions (the most keys) first leaves the light tiles last
    const int tile = blockIdx.y, j = blockIdx.x, t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int first = tiles[3 * tile], nq = tiles[3 * tile + 1];
    const int kvh = j / (HQ / HKV);
    const int r = req[first];
    const int p0 = pos[first];
    const int p_last = pos[first + nq - 1];
    const int32_t *bt = btab + (size_t)r * max_blocks;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(att_smem);
    // this thread's two query rows (fragment rows lane/4 and lane/4 + 8)
    const int qa = warp * 16 + (lane >> 2), qb = qa + 8;
    const int pa = p0 + qa, pb = p0 + qb;  // positions (beyond the tile: masked, not written)
    // Q fragments for the 8 k16 steps over the 128 dims
    uint32_t qf[8][4];
    {
        const __nv_bfloat16 *ra = q + ((size_t)(first + min(qa, nq - 1)) * HQ + j) * 128;
        const __nv_bfloat16 *rb = q + ((size_t)(first + min(qb, nq - 1)) * HQ + j) * 128;
        const int c = 2 * (lane & 3);
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            qf[s][0] = *reinterpret_cast<const uint32_t *>(ra + 16 * s + c);
            qf[s][1] = *reinterpret_cast<const uint32_t *>(rb + 16 * s + c);
            qf[s][2] = *reinterpret_cast<const uint32_t *>(ra + 16 * s + 8 + c);
            qf[s][3] = *reinterpret_cast<const uint32_t *>(rb + 16 * s + 8 + c);
        }
    }
    float o[16][4];
#pragma unroll
    for (int n = 0; n < 16; ++n) o[n][0] = o[n][1] = o[n][2] = o[n][3] = 0.0f;
    float ma = -FLT_MAX, mb = -FLT_MAX, la = 0.0f, lb = 0.0f;
    const float sl2 = 0.08838834764831845f * 1.4426950408889634f;  // 1/sqrt(128) * log2(e)

    // stage key tile kt (64 keys from kt*64) into buffer b: 128 threads x
    // 8 chunks of K and 8 of V; keys past the last query's position are zero
    auto stage = [&](int kt, int b) {
        const uint32_t kd = sbase + b * 2 * ATT_TILE_BYTES, vd = kd + ATT_TILE_BYTES;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = i * 128 + t;          // 1024 chunks of 16 bytes per tile
            const int row = e >> 4, c = e & 15;
            const int key = kt * 64 + row;
            const bool ok = key <= p_last;
            const size_t off = ok ? (((size_t)bt[key / 16] * 16 + key % 16) * HKV + kvh) * 128 + c * 8 : 0;
            cp_async16(kd + att_sw(row, c), kc + off, ok);
            cp_async16(vd + att_sw(row, c), vc + off, ok);
        }
        cp_async_commit();
    };
    const int ntile = p_last / 64 + 1;
    stage(0, 0);
    for (int kt = 0; kt < ntile; ++kt) {
        const int b = kt & 1;
        if (kt + 1 < ntile) {
            stage(kt + 1, b ^ 1);  // the other buffer was released at the end of the last tile
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const uint32_t kd = sbase + b * 2 * ATT_TILE_BYTES, vd = kd + ATT_TILE_BYTES;
        // S = Q K^T for this warp's 16 queries x 64 keys (8 blocks of 8 keys)
        float sc[8][4];
#pragma unroll
        for (int n = 0; n < 8; ++n) sc[n][0] = sc[n][1] = sc[n][2] = sc[n][3] = 0.0f;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
#pragma unroll
            for (int n = 0; n < 8; n += 2) {
                // matrices: keys n*8.. (dims 16s, 16s+8), keys (n+1)*8.. (same)
                const int mi = lane >> 3, rr = lane & 7;
                const int key = (n + (mi >> 1)) * 8 + rr;
                const int chunk = 2 * s + (mi & 1);
                uint32_t b0, b1, b2, b3;
                ldsm_x4(kd + att_sw(key, chunk), b0, b1, b2, b3);
                mma_bf16(sc[n], qf[s], b0, b1);
                mma_bf16(sc[n + 1], qf[s], b2, b3);
            }
        }
        // causal mask, online softmax (rows a and b of this thread)
        float ca = ma, cb = mb;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const int k0 = kt * 64 + n * 8 + 2 * (lane & 3);
            sc[n][0] = (k0 <= pa) ? sc[n][0] * sl2 : -FLT_MAX;
            sc[n][1] = (k0 + 1 <= pa) ? sc[n][1] * sl2 : -FLT_MAX;
            sc[n][2] = (k0 <= pb) ? sc[n][2] * sl2 : -FLT_MAX;
            sc[n][3] = (k0 + 1 <= pb) ? sc[n][3] * sl2 : -FLT_MAX;
            ca = fmaxf(ca, fmaxf(sc[n][0], sc[n][1]));
            cb = fmaxf(cb, fmaxf(sc[n][2], sc[n][3]));
        }
        ca = fmaxf(ca, __shfl_xor_sync(0xffffffffu, ca, 1));
        ca = fmaxf(ca, __shfl_xor_sync(0xffffffffu, ca, 2));
        cb = fmaxf(cb, __shfl_xor_sync(0xffffffffu, cb, 1));
        cb = fmaxf(cb, __shfl_xor_sync(0xffffffffu, cb, 2));
        const float fa = (ma == -FLT_MAX) ? 0.0f : exp2f(ma - ca);
        const float fb = (mb == -FLT_MAX) ? 0.0f : exp2f(mb - cb);
        ma = ca;
        mb = cb;
        float sa = 0.0f, sb = 0.0f;
        uint32_t pf[4][4];  // P as A fragments for the 4 k16 steps over the 64 keys
#pragma unroll
        for (int n = 0; n < 8; ++n) {
            const float e0 = sc[n][0] == -FLT_MAX ? 0.0f : exp2f(sc[n][0] - ca);
            const float e1 = sc[n][1] == -FLT_MAX ? 0.0f : exp2f(sc[n][1] - ca);
            const float e2 = sc[n][2] == -FLT_MAX ? 0.0f : exp2f(sc[n][2] - cb);
            const float e3 = sc[n][3] == -FLT_MAX ? 0.0f : exp2f(sc[n][3] - cb);
            sa += e0 + e1;
            sb += e2 + e3;
            pf[n >> 1][(n & 1) * 2 + 0] = pack_bf16(e0, e1);
            pf[n >> 1][(n & 1) * 2 + 1] = pack_bf16(e2, e3);
        }
        la = la * fa + sa;
        lb = lb * fb + sb;
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            o[n][0] *= fa;
            o[n][1] *= fa;
            o[n][2] *= fb;
            o[n][3] *= fb;
        }
        // O += P V: 4 k16 steps (keys) x 16 blocks of 8 dims
#pragma unroll
        for (int s = 0; s < 4; ++s) {
#pragma unroll
            for (int n = 0; n < 16; n += 2) {
                // transposed matrices: keys 16s.. / 16s+8.. x dims n*8.., (n+1)*8..
                const int mi = lane >> 3, rr = lane & 7;
                const int key = 16 * s + (mi & 1) * 8 + rr;
                const int chunk = n + (mi >> 1);
                uint32_t b0, b1, b2, b3;
                ldsm_x4_t(vd + att_sw(key, chunk), b0, b1, b2, b3);
                mma_bf16(o[n], pf[s], b0, b1);
                mma_bf16(o[n + 1], pf[s], b2, b3);
            }
        }
        __syncthreads();  // buffer b is free for the tile after next
    }
    // quad sums of the denominators, then the outputs of valid queries
    la += __shfl_xor_sync(0xffffffffu, la, 1);
    la += __shfl_xor_sync(0xffffffffu, la, 2);
    lb += __shfl_xor_sync(0xffffffffu, lb, 1);
    lb += __shfl_xor_sync(0xffffffffu, lb, 2);
    const float ia = 1.0f / la, ib = 1.0f / lb;
    const int c = 2 * (lane & 3);
    if (qa < nq) {
        __nv_bfloat16 *oa = out + ((size_t)(first + qa) * HQ + j) * 128;
#pragma unroll
        for (int n = 0; n < 16; ++n)
            *reinterpret_cast<__nv_bfloat162 *>(oa + n * 8 + c) = __floats2bfloat162_rn(o[n][0] * ia, o[n][1] * ia);
    }
    if (qb < nq) {
        __nv_bfloat16 *ob = out + ((size_t)(first + qb) * HQ + j) * 128;
#pragma unroll
        for (int n = 0; n < 16; ++n)
            *reinterpret_cast<__nv_bfloat162 *>(ob + n * 8 + c) = __floats2bfloat162_rn(o[n][2] * ib, o[n][3] * ib);
    }
}

__global__ void k_add(float *h, const float *y, size_t n) {
    chain_enter();
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) h[i] += y[i];
}

// act = bf16(silu(g) * u), four elements per thread (16-byte loads; the
// buffers are 256-byte aligned), a scalar tail
__global__ void k_silu_mul(const float *g, const float *u, __nv_bfloat16 *act, size_t n) {
    chain_enter();
    const size_t i = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) * 4;
    if (i + 4 > n) {
        for (size_t e = i; e < n; ++e) act[e] = __float2bfloat16_rn(g[e] / (1.0f + expf(-g[e])) * u[e]);
        return;
    }
    {
        const float4 a = *reinterpret_cast<const float4 *>(g + i);
        const float4 b = *reinterpret_cast<const float4 *>(u + i);
        const __nv_bfloat162 lo = __floats2bfloat162_rn(a.x / (1.0f + expf(-a.x)) * b.x,
                                                        a.y / (1.0f + expf(-a.y)) * b.y);
        const __nv_bfloat162 hi = __floats2bfloat162_rn(a.z / (1.0f + expf(-a.z)) * b.z,
                                                        a.w / (1.0f + expf(-a.w)) * b.w);
        *reinterpret_cast<uint2 *>(act + i) =
            make_uint2(*reinterpret_cast<const uint32_t *>(&lo), *reinterpret_cast<const uint32_t *>(&hi));
    }
}

// greedy sampling: first index of the maximum logit (NaN never wins; all
// -inf gives 0). 1024 threads; 16-byte loads when the vocabulary is a
// multiple of 4.
__global__ void __launch_bounds__(1024) k_argmax(const float *logits, int V, int32_t *out) {
    chain_enter();
    const int m = blockIdx.x;
    const float *l = logits + (size_t)m * V;
    float best = -FLT_MAX;
    int bi = 0;
    if ((V & 3) == 0) {
        const float4 *l4 = reinterpret_cast<const float4 *>(l);
        for (int c = threadIdx.x; c < V / 4; c += blockDim.x) {
            const float4 a = l4[c];
            if (a.x > best) { best = a.x; bi = 4 * c; }
            if (a.y > best) { best = a.y; bi = 4 * c + 1; }
            if (a.z > best) { best = a.z; bi = 4 * c + 2; }
            if (a.w > best) { best = a.w; bi = 4 * c + 3; }
        }
    } else {
        for (int c = threadIdx.x; c < V; c += blockDim.x)
            if (l[c] > best) { best = l[c]; bi = c; }
    }
    __shared__ float bv[32];
    __shared__ int bidx[32];
    for (int o = 16; o; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = best; bidx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (bv[w] > best || (bv[w] == best && bidx[w] < bi)) { best = bv[w]; bi = bidx[w]; }
        out[m] = bi;
    }
}

static cloak_status serve_step_body(cloak_ctx *ctx, const cloak_serve_desc *d,
                                    const cloak_serve_batch *b, cudaStream_t s);

// The linears keep the default CTA split here (tuned chunk and ring depth do
// not change a sum's order): a token computes the same in any batch.
cloak_status serve_step_run(cloak_ctx *ctx, const cloak_serve_desc *d, const cloak_serve_batch *b,
                            cudaStream_t s) {
    const bool was = ctx->tune_invariant;
    ctx->tune_invariant = true;
    ctx->chained = false;
    const cloak_status rc = serve_step_body(ctx, d, b, s);
    ctx->tune_invariant = was;
    ctx->chained = false;
    return rc;
}

static cloak_status serve_step_body(cloak_ctx *ctx, const cloak_serve_desc *d,
                                    const cloak_serve_batch *b, cudaStream_t s) {
    const cloak_stack_desc &sd = d->stack;
    if (ctx->dtype != CLOAK_BF16 || sd.head_dim != 128) return CLOAK_E_UNSUPPORTED;
    const int M = b->num_tokens, S = b->num_sample;
    if (M < 1 || S < 0 || S > M || !b->token_ids || !b->positions || !b->req_slots || !b->block_tables)
        return CLOAK_E_INVAL;
    const int D = sd.d_model, F = sd.d_ff, HQ = sd.n_heads, HKV = sd.n_kv_heads, V = d->vocab;
    const int QD = HQ * 128, KD = HKV * 128;
    if (d->lm_head < 0 || d->lm_head >= (int)ctx->tensors.size() || ctx->tensors[d->lm_head].n != V ||
        ctx->tensors[d->lm_head].k != D)
        return CLOAK_E_INVAL;
    if (d->embed_tensor >= 0) {
        const cloak_tensor_desc &et = ctx->tensors[d->embed_tensor];
        // rows in token order (columns may follow a residual permutation)
        if (et.n != V || et.k != D || ctx->info[d->embed_tensor].r_unit || D % 8) return CLOAK_E_INVAL;
    }
    const int flags = (b->flags & (CLOAK_LINEAR_UNCLOAKED | CLOAK_LINEAR_VMM));
    const int m_dec = (b->flags & CLOAK_SERVE_DECODE_FIRST) ? b->num_single : b->num_tokens;
    // workspace: h, y (fp32 [M, max(D, F)]), g, u (fp32 [M, F]), x, attn, q, k, v, act (bf16), logits
    const size_t Mz = (size_t)M;
    auto r256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    // single-query attention: every token without a work split, split over the keys
    const int n_single = b->qtiles ? b->num_single : M;
    const int32_t *single = b->qtiles ? b->single_rows : nullptr;
    if (n_single < 0 || n_single > M ||
        (b->qtiles && (b->num_qtiles < 0 || b->num_qtiles > 65535 || (n_single && !single))))
        return CLOAK_E_INVAL;
    const int max_splits = (d->max_blocks * 16 + ATT_SPLIT - 1) / ATT_SPLIT;
    const size_t part_bytes = (size_t)std::max(n_single, 1) * HQ * max_splits * ATT_PART * 4;
    const size_t need = r256(Mz * D * 4) + r256(Mz * D * 4) + 2 * r256(Mz * F * 4) + r256(Mz * D * 2) +
                        r256(Mz * QD * 2) * 2 + 2 * r256(Mz * KD * 2) + r256(Mz * F * 2) +
                        r256((size_t)std::max(S, 1) * V * 4) + r256((size_t)std::max(S, 1) * D * 2) +
                        r256(part_bytes);
    if (need > ctx->serve_ws_cap) {
        if (ctx->d_serve_ws) CLOAK_CUDA(ctx, cudaFree(ctx->d_serve_ws));
        ctx->d_serve_ws = nullptr;
        CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_serve_ws, need));
        ctx->serve_ws_cap = need;
    }
    uint8_t *w = (uint8_t *)ctx->d_serve_ws;
    auto take = [&](size_t n) { uint8_t *p = w; w += r256(n); return p; };
    float *h = (float *)take(Mz * D * 4);
    float *y = (float *)take(Mz * D * 4);
    float *g = (float *)take(Mz * F * 4);
    float *u = (float *)take(Mz * F * 4);
    __nv_bfloat16 *x = (__nv_bfloat16 *)take(Mz * D * 2);
    __nv_bfloat16 *q = (__nv_bfloat16 *)take(Mz * QD * 2);
    __nv_bfloat16 *attn = (__nv_bfloat16 *)take(Mz * QD * 2);
    __nv_bfloat16 *k = (__nv_bfloat16 *)take(Mz * KD * 2);
    __nv_bfloat16 *v = (__nv_bfloat16 *)take(Mz * KD * 2);
    __nv_bfloat16 *act = (__nv_bfloat16 *)take(Mz * F * 2);
    float *logits = b->out_logits ? b->out_logits : (float *)take((size_t)std::max(S, 1) * V * 4);
    __nv_bfloat16 *xs = (__nv_bfloat16 *)take((size_t)std::max(S, 1) * D * 2);
    float *apart = (float *)take(part_bytes);
    const size_t cnt_need = (size_t)std::max(n_single, 1) * HQ;
    if (cnt_need > ctx->att_cnt_cap) {
        if (ctx->d_att_cnt) CLOAK_CUDA(ctx, cudaFree(ctx->d_att_cnt));
        ctx->d_att_cnt = nullptr;
        CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_att_cnt, cnt_need * 4));
        CLOAK_CUDA(ctx, cudaMemsetAsync(ctx->d_att_cnt, 0, cnt_need * 4, s));
        ctx->att_cnt_cap = cnt_need;
    }
    cloak_status rc;
    if (b->qtiles) {
        static std::atomic<uint64_t> attr_devs{0};  // devices set up
        if (attr_needed(attr_devs, ctx->device)) {
            CLOAK_CUDA(ctx, cudaFuncSetAttribute(k_attention_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 4 * ATT_TILE_BYTES));
            attr_set_on(attr_devs, ctx->device);
        }
    }
    if (d->embed_tensor >= 0) {
        k_embed_tiled<<<M, 128, 0, s>>>(weight_base(ctx, flags), weight_slots(ctx, flags),
                                        ctx->h_tensor_base[d->embed_tensor],
                                        ctx->info[d->embed_tensor].kt, b->token_ids, D, V, h);
    } else {
        k_embed<<<M, 256, 0, s>>>((const __nv_bfloat16 *)d->embedding, b->token_ids, D, V, h);
    }
    CLOAK_LAUNCHED(ctx);
    // The step's first kernel follows whatever ran before it on the stream (a
    // table update of a concurrent re-key, the caller's copies); every later
    // kernel follows one of the step's own, none of which writes the weights or
    // the tables, so each may start -- a linear fetching its weight tiles --
    // while its predecessor finishes, and waits for it before reading its output.
    ctx->chained = true;
    // h += yy (yy null: no add), then the RMSNorm of n rows (rows null: all)
    // into xo; one fused kernel where the row fits its registers
    auto add_norm = [&](const float *yy, const int32_t *rows, int n, __nv_bfloat16 *xo) -> cloak_status {
        if (D % 4 == 0 && D <= 256 * 4 * NORM_VR) {
            CLOAK_CUDA(ctx, launch_k(ctx->chained, k_add_rmsnorm<NORM_VR>, dim3(n), dim3(256), 0, s, h, yy, rows,
                                     D, sd.rms_eps, xo));
            CLOAK_LAUNCHED(ctx);
            return CLOAK_OK;
        }
        if (yy) {
            CLOAK_CUDA(ctx, launch_k(ctx->chained, k_add, dim3(nb(Mz * D)), dim3(256), 0, s, h, yy, Mz * D));
            CLOAK_LAUNCHED(ctx);
        }
        CLOAK_CUDA(ctx, launch_k(ctx->chained, k_rmsnorm, dim3(n), dim3(256), 0, s, h, rows, D, sd.rms_eps, xo));
        CLOAK_LAUNCHED(ctx);
        return CLOAK_OK;
    };
    if (sd.num_layers > 0 && (rc = add_norm(nullptr, nullptr, M, x))) return rc;
    for (int l = 0; l < sd.num_layers; ++l) {
        const int32_t *lt = sd.layer_tensors + 7 * l;
        __nv_bfloat16 *kc = (__nv_bfloat16 *)d->k_cache + (size_t)l * d->num_blocks * 16 * KD;
        __nv_bfloat16 *vc = (__nv_bfloat16 *)d->v_cache + (size_t)l * d->num_blocks * 16 * KD;
        {
            const int32_t ts[3] = {lt[0], lt[1], lt[2]};
            const void *xs3[3] = {x, x, x};
            void *ys3[3] = {q, k, v};
            if ((rc = step_linears(ctx, 3, ts, xs3, ys3, M, m_dec, CLOAK_OUT_BF16, flags, s))) return rc;
        }
        CLOAK_CUDA(ctx, launch_k(ctx->chained, k_rope_cache, dim3(M), dim3(256), 0, s, q, k, v,
                                 b->positions, b->req_slots, b->block_tables, d->max_blocks, HQ, HKV,
                                 d->rope_theta, kc, vc));
        CLOAK_LAUNCHED(ctx);
        if (b->qtiles && b->num_qtiles > 0) {
            // prefill runs: query tiles sharing staged K/V tiles
            CLOAK_CUDA(ctx, launch_k(ctx->chained, k_attention_tiled, dim3(HQ, b->num_qtiles), dim3(128),
                                     4 * ATT_TILE_BYTES, s, q, kc, vc, b->positions, b->req_slots,
                                     b->block_tables, b->qtiles, d->max_blocks, HQ, HKV, attn));
            CLOAK_LAUNCHED(ctx);
        }
        if (n_single > 0) {
            // single queries (all tokens without a work split): split over the keys
            CLOAK_CUDA(ctx, launch_k(ctx->chained, k_attn_decode, dim3(std::min(max_splits, ATT_GRID_X), n_single, HQ),
                                     dim3(128), 0, s, q, kc, vc, b->positions, b->req_slots, b->block_tables,
                                     single, d->max_blocks, HQ, HKV, max_splits, apart, ctx->d_att_cnt, attn));
            CLOAK_LAUNCHED(ctx);
        }
        {
            const int32_t t1[1] = {lt[3]};
            const void *x1[1] = {attn};
            void *y1[1] = {y};
            if ((rc = step_linears(ctx, 1, t1, x1, y1, M, m_dec, CLOAK_OUT_F32, flags, s))) return rc;
        }
        if ((rc = add_norm(y, nullptr, M, x))) return rc;
        {
            const int32_t ts[2] = {lt[4], lt[5]};
            const void *xs2[2] = {x, x};
            void *ys2[2] = {g, u};
            if ((rc = step_linears(ctx, 2, ts, xs2, ys2, M, m_dec, CLOAK_OUT_F32, flags, s))) return rc;
        }
        CLOAK_CUDA(ctx, launch_k(ctx->chained, k_silu_mul, dim3(nb((Mz * F + 3) / 4)), dim3(256), 0, s, g, u, act,
                                 Mz * F));
        CLOAK_LAUNCHED(ctx);
        {
            const int32_t t1[1] = {lt[6]};
            const void *x1[1] = {act};
            void *y1[1] = {y};
            if ((rc = step_linears(ctx, 1, t1, x1, y1, M, m_dec, CLOAK_OUT_F32, flags, s))) return rc;
        }
        // the next layer's input norm, or after the last layer the final norm
        // of the sampled rows (nothing reads the other rows of h after it)
        if (l + 1 < sd.num_layers) {
            if ((rc = add_norm(y, nullptr, M, x))) return rc;
        } else if (S > 0) {
            if ((rc = add_norm(y, b->sample_rows, S, xs))) return rc;
        }
    }
    if (S > 0) {
        if (sd.num_layers == 0 && (rc = add_norm(nullptr, b->sample_rows, S, xs))) return rc;
        if ((rc = linear_run(ctx, d->lm_head, xs, logits, S, CLOAK_OUT_F32, flags, s))) return rc;
        CLOAK_CUDA(ctx, launch_k(ctx->chained, k_argmax, dim3(S), dim3(1024), 0, s, logits, V, b->out_tokens));
        CLOAK_LAUNCHED(ctx);
    }
    return CLOAK_OK;
}

}  // namespace cloak
