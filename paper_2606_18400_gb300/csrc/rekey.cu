// rekey.cu -- periodic re-randomisation of the physical page placement
// (Section 4.2, "Physical page remapping"; the shuffle period trade-off of
// Figure 7), done in place at HBM copy bandwidth.
//
// The new page map (same key, next epoch) sends the content of physical page
// old[vp] to new[vp]. As a graph on physical pages every node has at most one
// outgoing and one incoming move, so the moves form chains (ending at a page
// that was free) and cycles. A component x_0 -> x_1 -> ... executes back to
// front: e_1 writes the free end (or, for a cycle, x_0), e_2 writes the page
// e_1 just read, and so on. Components are cut into segments of L moves run
// side by side: wave w executes the w-th move of every segment. The last move
// of a segment reads the page the next segment overwrites in its first wave,
// so that page (and x_0 of a cycle) is first copied to a staging page in
// wave 0 and read from there. L is the smallest length whose staging need
// fits the pool; components that do not fit run in a later pass.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace cloak {

static inline unsigned nblk(uint64_t n, unsigned b = 256) { return (unsigned)((n + b - 1) / b); }

// plan (u32): [0] waves, [1] ops, [2] status (0 ok), [3] passes, [4..7] 0;
// wave_start[0 .. waves] at PLAN_HDR; ops (src, dst) at ops_offset(NP).
// A location below STAGE_BIT is an arena page, else a staging page.
constexpr uint32_t PLAN_HDR = 8;
constexpr uint32_t STAGE_BIT = 0x80000000u;
__host__ __device__ inline uint64_t ops_offset(uint64_t NP) { return PLAN_HDR + 2 * NP + 4; }
uint64_t rekey_plan_words(uint64_t NP) { return ops_offset(NP) + 4 * NP + 8; }

struct PlanArgs {
    const uint32_t *old_pa, *new_pa;
    uint32_t NP, NPS, cap_stage;
    uint32_t *plan;
    uint32_t *scratch;  // 5 * NPS + 8 words (used when the arrays do not fit in smem)
    int use_smem;
};

__global__ void k_rekey_plan(PlanArgs a) {
    extern __shared__ uint32_t sm[];
    uint32_t *base = a.use_smem ? sm : a.scratch;
    uint32_t *dst_of = base, *src_of = base + a.NPS, *cstart = base + 2 * a.NPS,
             *clen = base + 3 * a.NPS, *cursor = base + 4 * a.NPS;
    for (uint32_t p = threadIdx.x; p < a.NPS; p += blockDim.x) {
        dst_of[p] = NONE;
        src_of[p] = NONE;
    }
    __syncthreads();
    for (uint32_t vp = threadIdx.x; vp < a.NP; vp += blockDim.x) {
        uint32_t o = a.old_pa[vp], n = a.new_pa[vp];
        if (o != n) {
            dst_of[o] = n;
            src_of[n] = o;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    uint32_t *plan = a.plan;
    for (int i = 0; i < (int)PLAN_HDR; ++i) plan[i] = 0;
    const uint32_t VIS = NONE - 1;
    // components: chains start where nothing moves in; the rest are cycles
    uint32_t nc = 0, maxm = 0;
    for (uint32_t p = 0; p < a.NPS; ++p) {
        if (dst_of[p] == NONE || src_of[p] != NONE) continue;
        uint32_t m = 0, x = p;
        while (dst_of[x] != NONE) {
            src_of[x] = VIS;
            ++m;
            x = dst_of[x];
            if (m > a.NPS) {  // not a valid map pair: refuse instead of looping
                plan[2] = 3;
                return;
            }
        }
        cstart[nc] = p;
        clen[nc++] = m;
        maxm = max(maxm, m);
    }
    for (uint32_t p = 0; p < a.NPS; ++p) {
        if (dst_of[p] == NONE || src_of[p] == VIS) continue;
        uint32_t m = 0, x = p;
        do {
            src_of[x] = VIS;
            ++m;
            x = dst_of[x];
            if (m > a.NPS || x == NONE) {
                plan[2] = 3;
                return;
            }
        } while (x != p);
        cstart[nc] = p;
        clen[nc++] = m | STAGE_BIT;
        maxm = max(maxm, m);
    }
    if (nc == 0) return;  // nothing moves
    auto need_of = [&](uint32_t c, uint32_t L) {
        uint32_t m = clen[c] & ~STAGE_BIT, segs = (m + L - 1) / L;
        return (clen[c] & STAGE_BIT) ? segs : segs - 1;
    };
    auto staged = [&](uint32_t L) {
        uint64_t s = 0;
        for (uint32_t c = 0; c < nc; ++c) s += need_of(c, L);
        return s;
    };
    uint32_t L = maxm;
    if (staged(maxm) <= a.cap_stage) {
        uint32_t lo = 1, hi = maxm;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (staged(mid) <= a.cap_stage) hi = mid;
            else lo = mid + 1;
        }
        L = lo;
    }
    uint32_t *ws = plan + PLAN_HDR;
    uint32_t *ops = plan + ops_offset(a.NP);
    uint32_t nops = 0, wave = 0, passes = 0, c0 = 0;
    while (c0 < nc) {
        uint32_t c1 = c0, used = 0, plen = 0;
        while (c1 < nc) {
            uint32_t need = need_of(c1, L);
            if (c1 > c0 && used + need > a.cap_stage) break;
            used += need;
            plen = max(plen, min(clen[c1] & ~STAGE_BIT, L));
            ++c1;
        }
        if (used > a.cap_stage) {  // a single component needs more than the pool
            plan[2] = 1;
            return;
        }
        const uint32_t nw = 1 + plen;  // staging wave + move waves
        for (uint32_t w = 0; w < nw; ++w) cursor[w] = 0;
        // count: a component of m moves puts move k (1..m, execution order)
        // in wave 1 + (k-1) % L; staged reads add one op to wave 0
        for (uint32_t c = c0; c < c1; ++c) {
            uint32_t m = clen[c] & ~STAGE_BIT;
            cursor[0] += need_of(c, L);
            for (uint32_t k = 1; k <= m; ++k) cursor[1 + (k - 1) % L] += 1;
        }
        for (uint32_t w = 0; w < nw; ++w) {
            uint32_t cnt = cursor[w];
            ws[wave + w] = nops;
            cursor[w] = nops;
            nops += cnt;
        }
        ws[wave + nw] = nops;
        // fill: walk each component forward; move x_i -> x_{i+1} is e_k with
        // k = m - i. It reads staging when it ends a segment that is not the
        // component's last move, or when it is a cycle's last move.
        uint32_t sidx = 0;
        for (uint32_t c = c0; c < c1; ++c) {
            uint32_t m = clen[c] & ~STAGE_BIT;
            bool cyc = (clen[c] & STAGE_BIT) != 0;
            uint32_t x = cstart[c];
            for (uint32_t i = 0; i < m; ++i) {
                uint32_t y = dst_of[x];
                uint32_t k = m - i;
                uint32_t w = 1 + (k - 1) % L;
                bool st = (k % L == 0 && k < m) || (cyc && k == m);
                uint32_t src = x;
                if (st) {
                    uint32_t o = cursor[0]++;
                    ops[2 * o] = x;
                    ops[2 * o + 1] = STAGE_BIT | sidx;
                    src = STAGE_BIT | sidx;
                    ++sidx;
                }
                uint32_t o = cursor[w]++;
                ops[2 * o] = src;
                ops[2 * o + 1] = y;
                x = y;
            }
        }
        wave += nw;
        ++passes;
        c0 = c1;
    }
    plan[0] = wave;
    plan[1] = nops;
    plan[3] = passes;
}

// One wave: grid.x = ops of the wave, grid.y = chunks of a page. Each block
// copies one chunk with 16-byte streaming loads and stores.
__global__ void __launch_bounds__(256) k_rekey_wave(const uint32_t *ops, uint32_t op0,
                                                    uint8_t *arena, uint8_t *stage,
                                                    int64_t page_bytes, int64_t chunk) {
    const uint32_t o = op0 + blockIdx.x;
    const uint32_t s = ops[2 * o], d = ops[2 * o + 1];
    const uint8_t *src = (s & STAGE_BIT) ? stage + (int64_t)(s & ~STAGE_BIT) * page_bytes
                                         : arena + (int64_t)s * page_bytes;
    uint8_t *dst = (d & STAGE_BIT) ? stage + (int64_t)(d & ~STAGE_BIT) * page_bytes
                                   : arena + (int64_t)d * page_bytes;
    const int64_t lo = (int64_t)blockIdx.y * chunk;
    const int64_t hi = min(lo + chunk, page_bytes);
    const uint4 *S = reinterpret_cast<const uint4 *>(src + lo);
    uint4 *D = reinterpret_cast<uint4 *>(dst + lo);
    const int64_t n = (hi - lo) / 16;
    constexpr int U = 4;
    int64_t i = threadIdx.x;
    for (; i + (U - 1) * 256 < n; i += U * 256) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = __ldcs(S + i + u * 256);
#pragma unroll
        for (int u = 0; u < U; ++u) __stcs(D + i + u * 256, v[u]);
    }
    for (; i < n; i += 256) __stcs(D + i, __ldcs(S + i));
}

__global__ void k_copy_words(uint32_t *dst, const uint32_t *src, uint32_t n) {
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) dst[p] = src[p];
}

cloak_status rekey_run(cloak_ctx *ctx, uint64_t key, uint32_t new_epoch, cudaStream_t s) {
    cloak_status rc;
    if ((rc = keygen_page_map(ctx, key, new_epoch, ctx->d_page_new, s))) return rc;
    const uint64_t words = rekey_plan_words(ctx->NP);
    if (ctx->plan_cap < words) {
        if (ctx->d_plan) CLOAK_CUDA(ctx, cudaFree(ctx->d_plan));
        ctx->d_plan = nullptr;
        // plan + 5*NPS+8 scratch words for the planner's arrays
        CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_plan, (words + 5 * (uint64_t)ctx->NPS + 8) * 4));
        ctx->plan_cap = words;
    }
    PlanArgs pa;
    pa.old_pa = ctx->d_page_alloc;
    pa.new_pa = ctx->d_page_new;
    pa.NP = (uint32_t)ctx->NP;
    pa.NPS = (uint32_t)ctx->NPS;
    pa.cap_stage = (uint32_t)ctx->stage_pages;
    pa.plan = ctx->d_plan;
    pa.scratch = ctx->d_plan + words;
    size_t smem = (5 * (size_t)ctx->NPS + 8) * 4;
    pa.use_smem = smem <= 200 * 1024;
    if (pa.use_smem) {
        CLOAK_CUDA(ctx, cudaFuncSetAttribute(k_rekey_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
    } else {
        smem = 0;
    }
    k_rekey_plan<<<1, 1024, smem, s>>>(pa);
    CLOAK_LAUNCHED(ctx);
    uint32_t hdr[PLAN_HDR];
    CLOAK_CUDA(ctx, cudaMemcpyAsync(hdr, ctx->d_plan, sizeof hdr, cudaMemcpyDeviceToHost, s));
    CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    if (hdr[2] != 0) {
        ctx->last_err = "re-key plan does not fit the staging pool";
        return CLOAK_E_UNSUPPORTED;
    }
    const uint32_t waves = hdr[0];
    std::vector<uint32_t> ws(waves + 1);
    if (waves) {
        CLOAK_CUDA(ctx, cudaMemcpyAsync(ws.data(), ctx->d_plan + PLAN_HDR, (waves + 1) * 4,
                                        cudaMemcpyDeviceToHost, s));
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    }
    const int64_t chunk = std::min<int64_t>(ctx->page_bytes, 64 * 1024);
    const unsigned chunks = (unsigned)((ctx->page_bytes + chunk - 1) / chunk);
    const uint32_t *ops = ctx->d_plan + ops_offset(ctx->NP);
    for (uint32_t w = 0; w < waves; ++w) {
        uint32_t n = ws[w + 1] - ws[w];
        if (!n) continue;
        k_rekey_wave<<<dim3(n, chunks), 256, 0, s>>>(ops, ws[w], ctx->arena, ctx->d_stage,
                                                     ctx->page_bytes, chunk);
        CLOAK_LAUNCHED(ctx);
    }
    k_copy_words<<<nblk(ctx->NPS), 256, 0, s>>>(ctx->d_page_alloc, ctx->d_page_new,
                                                (uint32_t)ctx->NPS);
    CLOAK_LAUNCHED(ctx);
    if ((rc = build_tile_slot(ctx, ctx->d_page_alloc, s))) return rc;
    ctx->epoch = new_epoch;
    return CLOAK_OK;
}

}  // namespace cloak
