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

namespace cloak {

static inline unsigned nb(size_t n, unsigned b = 256) { return (unsigned)((n + b - 1) / b); }

__global__ void k_embed(const __nv_bfloat16 *emb, const int32_t *ids, int D, float *h) {
    const int m = blockIdx.x;
    const __nv_bfloat16 *e = emb + (size_t)ids[m] * D;
    for (int c = threadIdx.x; c < D; c += blockDim.x) h[(size_t)m * D + c] = __bfloat162float(e[c]);
}

// x = bf16(h * r), r = 1/sqrt(mean(h^2) + eps); optional row subset
__global__ void k_rmsnorm(const float *h, const int32_t *rows, int D, float eps, __nv_bfloat16 *x) {
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

// RoPE (rotate-half pairs (i, i+64) of a 128-dim head, angle pos * theta^(-i/64))
// on q and k; k and v written to the paged cache [block][16][n_kv][128].
__global__ void k_rope_cache(__nv_bfloat16 *q, const __nv_bfloat16 *k, const __nv_bfloat16 *v,
                             const int32_t *pos, const int32_t *req, const int32_t *btab,
                             int max_blocks, int HQ, int HKV, float theta, __nv_bfloat16 *kc,
                             __nv_bfloat16 *vc) {
    const int m = blockIdx.x, head = blockIdx.y, i = threadIdx.x;  // i < 64
    const int p = pos[m];
    const float freq = powf(theta, -(float)i / 64.0f);
    float sn, cs;
    sincosf((float)p * freq, &sn, &cs);
    if (head < HQ) {
        __nv_bfloat16 *qh = q + ((size_t)m * HQ + head) * 128;
        const float a = __bfloat162float(qh[i]), b = __bfloat162float(qh[i + 64]);
        qh[i] = __float2bfloat16_rn(a * cs - b * sn);
        qh[i + 64] = __float2bfloat16_rn(b * cs + a * sn);
    } else {
        const int kh = head - HQ;  // < HKV
        const __nv_bfloat16 *kr = k + ((size_t)m * HKV + kh) * 128;
        const __nv_bfloat16 *vr = v + ((size_t)m * HKV + kh) * 128;
        const int blk = btab[(size_t)req[m] * max_blocks + p / 16];
        const size_t off = (((size_t)blk * 16 + p % 16) * HKV + kh) * 128;
        const float a = __bfloat162float(kr[i]), b = __bfloat162float(kr[i + 64]);
        kc[off + i] = __float2bfloat16_rn(a * cs - b * sn);
        kc[off + i + 64] = __float2bfloat16_rn(b * cs + a * sn);
        vc[off + i] = vr[i];
        vc[off + i + 64] = vr[i + 64];
    }
}

// Causal attention of single queries (decode tokens), split over the keys:
// block (split, row, head) takes keys [256 split, 256 split + 256) of token
// m = rows[row]; each of its 4 warps 64 of them, 8 at a time. A lane holds 4
// of the 128 dimensions: K and V rows are read as 256-byte coalesced warp
// loads, 16 of them in flight per lane; scores are warp sums. Online softmax
// in FP32 per warp, merged across the warps in shared memory. A token with
// one split writes its output; otherwise the block writes (max, sum,
// acc[128]) and k_attn_combine merges the splits in order. The split depends
// only on the token's own position, so the result does not depend on the
// batch.
constexpr int ATT_SPLIT = 256;
constexpr int ATT_PART = 132;  // floats per partial: max, sum, pad, acc[128]

__global__ void __launch_bounds__(128) k_attn_decode(const __nv_bfloat16 *q, const __nv_bfloat16 *kc,
                                                     const __nv_bfloat16 *vc, const int32_t *pos,
                                                     const int32_t *req, const int32_t *btab,
                                                     const int32_t *rows, int max_blocks, int HQ,
                                                     int HKV, int max_splits, float *part,
                                                     __nv_bfloat16 *out) {
    const int sp = blockIdx.x, r = blockIdx.y, j = blockIdx.z;
    const int m = rows ? rows[r] : r;
    const int n = pos[m] + 1;
    const int nsplit = (n + ATT_SPLIT - 1) / ATT_SPLIT;
    if (sp >= nsplit) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    const int k_begin = sp * ATT_SPLIT + w * (ATT_SPLIT / 4);
    const int k_end = min(n, k_begin + ATT_SPLIT / 4);
    float mx = -FLT_MAX, sum = 0.0f, acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int kb = k_begin; kb < k_end; kb += 8) {
        uint2 kr[8], vr[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int key = min(kb + i, k_end - 1);
            const size_t off = (((size_t)bt[key >> 4] * 16 + (key & 15)) * HKV + kvh) * 128 + 4 * lane;
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
#pragma unroll
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
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
    __shared__ float wm[4], wl[4];
    __shared__ float wa[4][128];
    if (lane == 0) { wm[w] = mx; wl[w] = sum; }
#pragma unroll
    for (int d = 0; d < 4; ++d) wa[w][4 * lane + d] = acc[d];
    __syncthreads();
    const int t = threadIdx.x;
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
    float *pp = part + (((size_t)r * HQ + j) * max_splits + sp) * ATT_PART;
    if (t == 0) { pp[0] = M; pp[1] = L; }
    pp[4 + t] = A;
}

// Merge the splits of tokens with more than one, in split order.
__global__ void __launch_bounds__(128) k_attn_combine(const int32_t *pos, const int32_t *rows, int HQ,
                                                      int max_splits, const float *part,
                                                      __nv_bfloat16 *out) {
    const int r = blockIdx.x, j = blockIdx.y, t = threadIdx.x;
    const int m = rows ? rows[r] : r;
    const int nsplit = (pos[m] + ATT_SPLIT) / ATT_SPLIT;
    if (nsplit == 1) return;
    const float *pp = part + ((size_t)r * HQ + j) * max_splits * ATT_PART;
    float M = -FLT_MAX;
    for (int sp = 0; sp < nsplit; ++sp) M = fmaxf(M, pp[sp * ATT_PART]);
    float L = 0.0f, A = 0.0f;
    for (int sp = 0; sp < nsplit; ++sp) {
        const float e = expf(pp[sp * ATT_PART] - M);
        L = fmaf(pp[sp * ATT_PART + 1], e, L);
        A = fmaf(pp[sp * ATT_PART + 4 + t], e, A);
    }
    out[((size_t)m * HQ + j) * 128 + t] = __float2bfloat16_rn(A / L);
}

// Query-tiled causal attention for runs of consecutive tokens of one request
// (prefill chunks): a block takes up to 64 queries of one head; each 64-key
// tile of K and V is staged once in shared memory (FP32) and used by all of
// them. Thread t: query t/2, dimension half t%2 (64 dims); a score is the
// sum of the two halves. Online softmax in FP32 over key chunks of 16.
// tiles: [n][3] = (first batch token, query count, -) ; query i of a tile is
// batch token first + i, positions consecutive.
__global__ void __launch_bounds__(128) k_attention_tiled(const __nv_bfloat16 *q, const __nv_bfloat16 *kc,
                                                         const __nv_bfloat16 *vc, const int32_t *pos,
                                                         const int32_t *req, const int32_t *btab,
                                                         const int32_t *tiles, int max_blocks, int HQ,
                                                         int HKV, __nv_bfloat16 *out) {
    extern __shared__ float sm[];
    float *Ks = sm, *Vs = sm + 64 * 128;
    const int tile = blockIdx.x, j = blockIdx.y, t = threadIdx.x;
    const int first = tiles[3 * tile], nq = tiles[3 * tile + 1];
    const int qi = t >> 1, half = t & 1;
    const int kvh = j / (HQ / HKV);
    const int m = first + min(qi, nq - 1);
    const int r = req[first];
    const int p = pos[m];
    const int p_last = pos[first + nq - 1];
    const int32_t *bt = btab + (size_t)r * max_blocks;
    float qv[64];
    const __nv_bfloat16 *qr = q + ((size_t)m * HQ + j) * 128 + half * 64;
#pragma unroll
    for (int d = 0; d < 64; ++d) qv[d] = __bfloat162float(qr[d]) * 0.08838834764831845f;
    float acc[64];
#pragma unroll
    for (int d = 0; d < 64; ++d) acc[d] = 0.0f;
    float mx = -FLT_MAX, sum = 0.0f;
    for (int k0 = 0; k0 <= p_last; k0 += 64) {
        __syncthreads();
        // stage 64 keys: 128 threads, each 64 of the 8192 values of K and of V
        for (int e = t; e < 64 * 16; e += 128) {
            const int kk = e >> 4, part = e & 15;  // 16 parts of 8 dims
            const int key = k0 + kk;
            float4 a0 = make_float4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
            if (key <= p_last) {
                const size_t off = (((size_t)bt[key / 16] * 16 + key % 16) * HKV + kvh) * 128 + part * 8;
                const uint4 rk = *reinterpret_cast<const uint4 *>(kc + off);
                const uint4 rv = *reinterpret_cast<const uint4 *>(vc + off);
                const __nv_bfloat162 *hk = reinterpret_cast<const __nv_bfloat162 *>(&rk);
                const __nv_bfloat162 *hv = reinterpret_cast<const __nv_bfloat162 *>(&rv);
                float2 f;
                f = __bfloat1622float2(hk[0]); a0.x = f.x; a0.y = f.y;
                f = __bfloat1622float2(hk[1]); a0.z = f.x; a0.w = f.y;
                f = __bfloat1622float2(hk[2]); a1.x = f.x; a1.y = f.y;
                f = __bfloat1622float2(hk[3]); a1.z = f.x; a1.w = f.y;
                f = __bfloat1622float2(hv[0]); b0.x = f.x; b0.y = f.y;
                f = __bfloat1622float2(hv[1]); b0.z = f.x; b0.w = f.y;
                f = __bfloat1622float2(hv[2]); b1.x = f.x; b1.y = f.y;
                f = __bfloat1622float2(hv[3]); b1.z = f.x; b1.w = f.y;
            }
            float4 *kd = reinterpret_cast<float4 *>(Ks + kk * 128 + part * 8);
            float4 *vd = reinterpret_cast<float4 *>(Vs + kk * 128 + part * 8);
            kd[0] = a0; kd[1] = a1;
            vd[0] = b0; vd[1] = b1;
        }
        __syncthreads();
        const int kn = min(64, p_last + 1 - k0);
        for (int c = 0; c < kn; c += 16) {
            float sc[16];
#pragma unroll
            for (int z = 0; z < 16; ++z) {
                const float *kr = Ks + (c + z) * 128 + half * 64;
                float d0 = 0.0f;
#pragma unroll
                for (int d = 0; d < 64; d += 4) {
                    const float4 kv = *reinterpret_cast<const float4 *>(kr + d);
                    d0 = fmaf(qv[d], kv.x, d0);
                    d0 = fmaf(qv[d + 1], kv.y, d0);
                    d0 = fmaf(qv[d + 2], kv.z, d0);
                    d0 = fmaf(qv[d + 3], kv.w, d0);
                }
                d0 += __shfl_xor_sync(0xffffffffu, d0, 1);
                const int key = k0 + c + z;
                sc[z] = (c + z < kn && key <= p) ? d0 : -FLT_MAX;
            }
            float cm = mx;
#pragma unroll
            for (int z = 0; z < 16; ++z) cm = fmaxf(cm, sc[z]);
            const float scale = expf(mx - cm);
            sum *= scale;
#pragma unroll
            for (int d = 0; d < 64; ++d) acc[d] *= scale;
#pragma unroll
            for (int z = 0; z < 16; ++z) {
                const float pz = sc[z] == -FLT_MAX ? 0.0f : expf(sc[z] - cm);
                sum += pz;
                const float *vr = Vs + (c + z) * 128 + half * 64;
#pragma unroll
                for (int d = 0; d < 64; d += 4) {
                    const float4 vv = *reinterpret_cast<const float4 *>(vr + d);
                    acc[d] = fmaf(pz, vv.x, acc[d]);
                    acc[d + 1] = fmaf(pz, vv.y, acc[d + 1]);
                    acc[d + 2] = fmaf(pz, vv.z, acc[d + 2]);
                    acc[d + 3] = fmaf(pz, vv.w, acc[d + 3]);
                }
            }
            mx = cm;
        }
    }
    if (qi < nq) {
        __nv_bfloat16 *o = out + ((size_t)m * HQ + j) * 128 + half * 64;
        const float inv = 1.0f / sum;
#pragma unroll
        for (int d = 0; d < 64; ++d) o[d] = __float2bfloat16_rn(acc[d] * inv);
    }
}

__global__ void k_add(float *h, const float *y, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) h[i] += y[i];
}

__global__ void k_silu_mul(const float *g, const float *u, __nv_bfloat16 *act, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float a = g[i];
        act[i] = __float2bfloat16_rn(a / (1.0f + expf(-a)) * u[i]);
    }
}

// greedy sampling: first index of the maximum logit
__global__ void k_argmax(const float *logits, int V, int32_t *out) {
    const int m = blockIdx.x;
    const float *l = logits + (size_t)m * V;
    float best = -FLT_MAX;
    int bi = 0;
    for (int c = threadIdx.x; c < V; c += blockDim.x)
        if (l[c] > best) { best = l[c]; bi = c; }
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
    const cloak_status rc = serve_step_body(ctx, d, b, s);
    ctx->tune_invariant = was;
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
    const int flags = (b->flags & CLOAK_LINEAR_UNCLOAKED);
    // workspace: h, y (fp32 [M, max(D, F)]), g, u (fp32 [M, F]), x, attn, q, k, v, act (bf16), logits
    const size_t Mz = (size_t)M;
    auto r256 = [](size_t n) { return (n + 255) & ~(size_t)255; };
    // single-query attention: every token without a work split, split over the keys
    const int n_single = b->qtiles ? b->num_single : M;
    const int32_t *single = b->qtiles ? b->single_rows : nullptr;
    if (n_single < 0 || n_single > M || (b->qtiles && (b->num_qtiles < 0 || (n_single && !single))))
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
    cloak_status rc;
    if (b->qtiles) {
        static bool attr = false;
        if (!attr) {
            CLOAK_CUDA(ctx, cudaFuncSetAttribute(k_attention_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 2 * 64 * 128 * (int)sizeof(float)));
            attr = true;
        }
    }
    k_embed<<<M, 256, 0, s>>>((const __nv_bfloat16 *)d->embedding, b->token_ids, D, h);
    CLOAK_LAUNCHED(ctx);
    for (int l = 0; l < sd.num_layers; ++l) {
        const int32_t *lt = sd.layer_tensors + 7 * l;
        __nv_bfloat16 *kc = (__nv_bfloat16 *)d->k_cache + (size_t)l * d->num_blocks * 16 * KD;
        __nv_bfloat16 *vc = (__nv_bfloat16 *)d->v_cache + (size_t)l * d->num_blocks * 16 * KD;
        k_rmsnorm<<<M, 256, 0, s>>>(h, nullptr, D, sd.rms_eps, x);
        CLOAK_LAUNCHED(ctx);
        {
            const int32_t ts[3] = {lt[0], lt[1], lt[2]};
            const void *xs3[3] = {x, x, x};
            void *ys3[3] = {q, k, v};
            if ((rc = linear_batch_run(ctx, 3, ts, xs3, ys3, M, CLOAK_OUT_BF16, flags, s))) return rc;
        }
        k_rope_cache<<<dim3(M, HQ + HKV), 64, 0, s>>>(q, k, v, b->positions, b->req_slots, b->block_tables,
                                                      d->max_blocks, HQ, HKV, d->rope_theta, kc, vc);
        CLOAK_LAUNCHED(ctx);
        if (b->qtiles && b->num_qtiles > 0) {
            // prefill runs: query tiles sharing staged K/V tiles
            k_attention_tiled<<<dim3(b->num_qtiles, HQ), 128, 2 * 64 * 128 * sizeof(float), s>>>(
                q, kc, vc, b->positions, b->req_slots, b->block_tables, b->qtiles, d->max_blocks, HQ,
                HKV, attn);
            CLOAK_LAUNCHED(ctx);
        }
        if (n_single > 0) {
            // single queries (all tokens without a work split): split over the keys
            k_attn_decode<<<dim3(max_splits, n_single, HQ), 128, 0, s>>>(
                q, kc, vc, b->positions, b->req_slots, b->block_tables, single, d->max_blocks, HQ, HKV,
                max_splits, apart, attn);
            CLOAK_LAUNCHED(ctx);
            k_attn_combine<<<dim3(n_single, HQ), 128, 0, s>>>(b->positions, single, HQ, max_splits, apart,
                                                              attn);
            CLOAK_LAUNCHED(ctx);
        }
        if ((rc = linear_run(ctx, lt[3], attn, y, M, CLOAK_OUT_F32, flags, s))) return rc;
        k_add<<<nb(Mz * D), 256, 0, s>>>(h, y, Mz * D);
        CLOAK_LAUNCHED(ctx);
        k_rmsnorm<<<M, 256, 0, s>>>(h, nullptr, D, sd.rms_eps, x);
        CLOAK_LAUNCHED(ctx);
        {
            const int32_t ts[2] = {lt[4], lt[5]};
            const void *xs2[2] = {x, x};
            void *ys2[2] = {g, u};
            if ((rc = linear_batch_run(ctx, 2, ts, xs2, ys2, M, CLOAK_OUT_F32, flags, s))) return rc;
        }
        k_silu_mul<<<nb(Mz * F), 256, 0, s>>>(g, u, act, Mz * F);
        CLOAK_LAUNCHED(ctx);
        if ((rc = linear_run(ctx, lt[6], act, y, M, CLOAK_OUT_F32, flags, s))) return rc;
        k_add<<<nb(Mz * D), 256, 0, s>>>(h, y, Mz * D);
        CLOAK_LAUNCHED(ctx);
    }
    if (S > 0) {
        k_rmsnorm<<<S, 256, 0, s>>>(h, b->sample_rows, D, sd.rms_eps, xs);
        CLOAK_LAUNCHED(ctx);
        if ((rc = linear_run(ctx, d->lm_head, xs, logits, S, CLOAK_OUT_F32, flags, s))) return rc;
        k_argmax<<<S, 256, 0, s>>>(logits, V, b->out_tokens);
        CLOAK_LAUNCHED(ctx);
    }
    return CLOAK_OK;
}

}  // namespace cloak
