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
#include <cstdlib>
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

// Parallel planner (one CTA of 1024 threads, arrays in global scratch).
// Each move source x gets its component (its chain's start, or the smallest
// page of its cycle) and its position i from that start by pointer jumping
// backwards along the moves: a node's record covers up to 2^r nodes behind
// it (count, last node, smallest page and the distance to it). With m moves
// in the component, x's move is e_k, k = m - i: wave 1 + (k-1) % L, segment
// (k-1) / L. A pass is [staging ops][wave 1: one slot per segment]...[wave
// plen]; every op's slot is a closed form, and short segments leave holes
// that the copy kernel skips.
constexpr uint32_t PAR_SCRATCH_ARRAYS = 21;  // words of scratch = 21 * NPS + 64

struct ParPlan {
    const uint32_t *old_pa, *new_pa;
    uint32_t NP, NPS, cap_stage, max_ops;
    uint32_t *plan;
    uint32_t *w;
};

__global__ void __launch_bounds__(1024) k_rekey_plan_par(ParPlan a) {
    const uint32_t N = a.NPS, tid = threadIdx.x, nth = blockDim.x;
    uint32_t *dst_of = a.w, *src_of = a.w + N;
    uint32_t *jp[2] = {a.w + 2 * N, a.w + 3 * N}, *jl[2] = {a.w + 4 * N, a.w + 5 * N},
             *jm[2] = {a.w + 6 * N, a.w + 7 * N}, *jd[2] = {a.w + 8 * N, a.w + 9 * N},
             *ja[2] = {a.w + 10 * N, a.w + 11 * N};
    uint32_t *msize = a.w + 12 * N, *head = a.w + 13 * N, *cinfo = a.w + 14 * N,
             *c_pass = a.w + 15 * N, *c_seg = a.w + 16 * N, *c_stg = a.w + 17 * N,
             *pass_rec = a.w + 18 * N, *misc = a.w + 21 * N;
    uint32_t *plan = a.plan;
    __shared__ uint32_t s_scan[1024];
    __shared__ uint64_t s_red[32];
    for (uint32_t p = tid; p < N; p += nth) {
        dst_of[p] = NONE;
        src_of[p] = NONE;
        msize[p] = 0;
        head[p] = 0;
    }
    if (tid < PLAN_HDR) plan[tid] = 0;
    __syncthreads();
    for (uint32_t vp = tid; vp < a.NP; vp += nth) {
        const uint32_t o = a.old_pa[vp], n = a.new_pa[vp];
        if (o != n) {
            dst_of[o] = n;
            src_of[n] = o;
        }
    }
    __syncthreads();
    for (uint32_t x = tid; x < N; x += nth) {
        jp[0][x] = src_of[x];
        jl[0][x] = 1;
        jm[0][x] = x;
        jd[0][x] = 0;
        ja[0][x] = x;
    }
    __syncthreads();
    int cur = 0;
    for (uint32_t span = 1; span < 2 * N; span <<= 1) {
        const int nx = cur ^ 1;
        for (uint32_t x = tid; x < N; x += nth) {
            const uint32_t y = jp[cur][x];
            if (y == NONE) {
                jp[nx][x] = NONE;
                jl[nx][x] = jl[cur][x];
                jm[nx][x] = jm[cur][x];
                jd[nx][x] = jd[cur][x];
                ja[nx][x] = ja[cur][x];
            } else {
                jp[nx][x] = jp[cur][y];
                jl[nx][x] = min(jl[cur][x] + jl[cur][y], 2 * N);
                if (jm[cur][y] < jm[cur][x]) {
                    jm[nx][x] = jm[cur][y];
                    jd[nx][x] = jl[cur][x] + jd[cur][y];
                } else {
                    jm[nx][x] = jm[cur][x];
                    jd[nx][x] = jd[cur][x];
                }
                ja[nx][x] = ja[cur][y];
            }
        }
        __syncthreads();
        cur = nx;
    }
    uint32_t *P = jp[cur], *Ln = jl[cur], *Mn = jm[cur], *Md = jd[cur], *La = ja[cur];
    // component (La) and position from its start (Md) of every move source
    for (uint32_t x = tid; x < N; x += nth) {
        if (dst_of[x] == NONE) continue;
        const bool chain = P[x] == NONE;
        const uint32_t comp = chain ? La[x] : Mn[x];
        Md[x] = chain ? Ln[x] - 1 : Md[x];
        La[x] = comp;
        atomicAdd(&msize[comp], 1u);
        head[comp] = chain ? 1u : 2u;
    }
    __syncthreads();
    // dense component indices in page order (block scan of the head flags)
    const uint32_t per = (N + nth - 1) / nth;
    const uint32_t lo = min(N, tid * per), hi = min(N, (tid + 1) * per);
    uint32_t cnt = 0;
    for (uint32_t x = lo; x < hi; ++x) cnt += head[x] ? 1u : 0u;
    s_scan[tid] = cnt;
    __syncthreads();
    for (uint32_t off = 1; off < nth; off <<= 1) {
        const uint32_t v = tid >= off ? s_scan[tid - off] : 0u;
        __syncthreads();
        s_scan[tid] += v;
        __syncthreads();
    }
    uint32_t idx = s_scan[tid] - cnt;
    for (uint32_t x = lo; x < hi; ++x)
        if (head[x]) {
            cinfo[idx] = msize[x] | (head[x] == 2 ? STAGE_BIT : 0u);
            head[x] = idx;  // page -> dense component index
            ++idx;
        }
    const uint32_t nc = s_scan[nth - 1];
    __syncthreads();
    if (nc == 0) return;  // nothing moves
    uint32_t maxm = 0;
    for (uint32_t c = tid; c < nc; c += nth) maxm = max(maxm, cinfo[c] & ~STAGE_BIT);
    for (int o = 16; o; o >>= 1) maxm = max(maxm, __shfl_xor_sync(0xffffffffu, maxm, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = maxm;
    __syncthreads();
    maxm = 0;
    for (uint32_t i = 0; i < (nth >> 5); ++i) maxm = max(maxm, (uint32_t)s_red[i]);
    __syncthreads();
    auto need = [](uint32_t mc, uint32_t L) {
        const uint32_t m = mc & ~STAGE_BIT, segs = (m + L - 1) / L;
        return (mc & STAGE_BIT) ? segs : segs - 1;
    };
    auto total_need = [&](uint32_t L) -> uint64_t {
        uint64_t sum = 0;
        for (uint32_t c = tid; c < nc; c += nth) sum += need(cinfo[c], L);
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if ((tid & 31) == 0) s_red[tid >> 5] = sum;
        __syncthreads();
        uint64_t t = 0;
        for (uint32_t i = 0; i < (nth >> 5); ++i) t += s_red[i];
        __syncthreads();
        return t;
    };
    // segment length: the smallest L whose total staging fits the pool; if
    // none does, the smallest with which each component fits a pass alone
    uint32_t L;
    if (total_need(maxm) <= a.cap_stage) {
        uint32_t l0 = 1, h0 = maxm;
        while (l0 < h0) {
            const uint32_t mid = (l0 + h0) >> 1;
            if (total_need(mid) <= a.cap_stage) h0 = mid;
            else l0 = mid + 1;
        }
        L = l0;
    } else {
        L = 1;
        while (L < maxm && need(maxm | STAGE_BIT, L) > a.cap_stage) L = max(L + 1, L * 2);
        L = min(L, maxm);
    }
    // passes: components in order while their staging fits (thread 0; the
    // number of components of a random page map is small)
    if (tid == 0) {
        uint32_t *ws = plan + PLAN_HDR;
        uint32_t wave = 0, opbase = 0, pass = 0, c = 0, status = 0;
        while (c < nc) {
            uint32_t c1 = c, used = 0, nseg = 0, plen = 0;
            while (c1 < nc) {
                const uint32_t nd = need(cinfo[c1], L);
                if (c1 > c && used + nd > a.cap_stage) break;
                const uint32_t m = cinfo[c1] & ~STAGE_BIT;
                c_pass[c1] = pass;
                c_seg[c1] = nseg;
                c_stg[c1] = used;
                used += nd;
                nseg += (m + L - 1) / L;
                plen = max(plen, min(m, L));
                ++c1;
            }
            const uint64_t pass_ops = used + (uint64_t)plen * nseg;
            if (used > a.cap_stage || opbase + pass_ops > a.max_ops ||
                PLAN_HDR + wave + plen + 2 > ops_offset(a.NP)) {
                status = 2;
                break;
            }
            pass_rec[3 * pass] = opbase;
            pass_rec[3 * pass + 1] = used;
            pass_rec[3 * pass + 2] = nseg;
            ws[wave] = opbase;
            for (uint32_t w = 1; w <= plen; ++w) ws[wave + w] = opbase + used + (w - 1) * nseg;
            opbase += (uint32_t)pass_ops;
            wave += 1 + plen;
            ws[wave] = opbase;
            c = c1;
            ++pass;
        }
        misc[0] = L;
        misc[1] = status;
        misc[2] = opbase;
        plan[0] = status ? 0 : wave;
        plan[1] = opbase;
        plan[2] = status;
        plan[3] = pass;
    }
    __syncthreads();
    if (misc[1]) return;
    L = misc[0];
    const uint32_t nops = misc[2];
    uint32_t *ops = plan + ops_offset(a.NP);
    for (uint32_t o = tid; o < nops; o += nth) {
        ops[2 * o] = NONE;
        ops[2 * o + 1] = NONE;
    }
    __syncthreads();
    for (uint32_t x = tid; x < N; x += nth) {
        if (dst_of[x] == NONE) continue;
        const uint32_t c = head[La[x]];
        const uint32_t mc = cinfo[c], m = mc & ~STAGE_BIT;
        const bool cyc = (mc & STAGE_BIT) != 0;
        const uint32_t segs = (m + L - 1) / L;
        const uint32_t k = m - Md[x];
        const uint32_t sg = (k - 1) / L, w = 1 + (k - 1) % L;
        const uint32_t pass = c_pass[c];
        const uint32_t opbase = pass_rec[3 * pass], used = pass_rec[3 * pass + 1],
                       nseg = pass_rec[3 * pass + 2];
        const bool st = (k % L == 0 && k < m) || (cyc && k == m);
        uint32_t src = x;
        if (st) {
            const uint32_t sidx = c_stg[c] + ((k == m) ? segs - 1 : k / L - 1);
            ops[2 * (opbase + sidx)] = x;
            ops[2 * (opbase + sidx) + 1] = STAGE_BIT | sidx;
            src = STAGE_BIT | sidx;
        }
        const uint32_t slot = opbase + used + (w - 1) * nseg + c_seg[c] + sg;
        ops[2 * slot] = src;
        ops[2 * slot + 1] = dst_of[x];
    }
}

// One wave: grid.x = ops of the wave, grid.y = chunks of a page. Each block
// copies one chunk with 16-byte streaming loads and stores.
__global__ void __launch_bounds__(256) k_rekey_wave(const uint32_t *ops, uint32_t op0,
                                                    uint8_t *arena, uint8_t *stage,
                                                    int64_t page_bytes, int64_t chunk) {
    const uint32_t o = op0 + blockIdx.x;
    const uint32_t s = ops[2 * o], d = ops[2 * o + 1];
    if (s == NONE) return;  // hole left by a segment shorter than the wave count
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

// What a re-key moves: n_virt units (pages, or tiles at tile granularity),
// unit v from location old_map[v] to new_map[v] among n_phys locations of
// unit_bytes each, with cap_stage staging units after them.
struct MoveSet {
    const uint32_t *old_map, *new_map;
    uint32_t n_virt, n_phys, cap_stage;
    int64_t unit_bytes;
};

static MoveSet page_moves(const cloak_ctx *ctx) {
    return {ctx->d_page_alloc, ctx->d_page_new, (uint32_t)ctx->NP, (uint32_t)ctx->NPS,
            (uint32_t)ctx->stage_pages, ctx->page_bytes};
}

// Plan the moves of `m`; on return ws holds the wave starts (waves + 1).
// Blocks the calling thread on `s` (the planners' header is read back).
static cloak_status plan_moves(cloak_ctx *ctx, const MoveSet &m, cudaStream_t s, std::vector<uint32_t> &ws) {
    // plan: header + wave table + ops (up to 8 * n_phys + 1024 ops) and the
    // planners' scratch arrays
    const uint64_t max_ops = 8 * (uint64_t)m.n_phys + 1024;
    const uint64_t words = ops_offset(m.n_virt) + 2 * max_ops;
    const uint64_t scratch = PAR_SCRATCH_ARRAYS * (uint64_t)m.n_phys + 64;
    if (ctx->plan_cap < words + scratch) {
        if (ctx->d_plan) CLOAK_CUDA(ctx, cudaFree(ctx->d_plan));
        ctx->d_plan = nullptr;
        CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_plan, (words + scratch) * 4));
        ctx->plan_cap = words + scratch;
    }
    ParPlan pp;
    pp.old_pa = m.old_map;
    pp.new_pa = m.new_map;
    pp.NP = m.n_virt;
    pp.NPS = m.n_phys;
    pp.cap_stage = m.cap_stage;
    pp.max_ops = (uint32_t)max_ops;
    pp.plan = ctx->d_plan;
    pp.w = ctx->d_plan + words;
    k_rekey_plan_par<<<1, 1024, 0, s>>>(pp);
    CLOAK_LAUNCHED(ctx);
    uint32_t hdr[PLAN_HDR];
    CLOAK_CUDA(ctx, cudaMemcpyAsync(hdr, ctx->d_plan, sizeof hdr, cudaMemcpyDeviceToHost, s));
    CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    if (hdr[2] != 0) {
        // the compact layout did not fit: the sequential planner packs ops densely
        PlanArgs pa;
        pa.old_pa = m.old_map;
        pa.new_pa = m.new_map;
        pa.NP = m.n_virt;
        pa.NPS = m.n_phys;
        pa.cap_stage = m.cap_stage;
        pa.plan = ctx->d_plan;
        pa.scratch = ctx->d_plan + words;
        size_t smem = (5 * (size_t)m.n_phys + 8) * 4;
        pa.use_smem = smem <= 200 * 1024;
        if (pa.use_smem)
            CLOAK_CUDA(ctx, cudaFuncSetAttribute(k_rekey_plan,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        else
            smem = 0;
        k_rekey_plan<<<1, 1024, smem, s>>>(pa);
        CLOAK_LAUNCHED(ctx);
        CLOAK_CUDA(ctx, cudaMemcpyAsync(hdr, ctx->d_plan, sizeof hdr, cudaMemcpyDeviceToHost, s));
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    }
    if (hdr[2] != 0) {
        ctx->last_err = "re-key plan does not fit the staging pool";
        return CLOAK_E_UNSUPPORTED;
    }
    const uint32_t waves = hdr[0];
    ws.assign(waves + 1, 0);
    if (waves) {
        CLOAK_CUDA(ctx, cudaMemcpyAsync(ws.data(), ctx->d_plan + PLAN_HDR, (waves + 1) * 4,
                                        cudaMemcpyDeviceToHost, s));
        CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    }
    return CLOAK_OK;
}

static cloak_status launch_wave(cloak_ctx *ctx, const MoveSet &m, const std::vector<uint32_t> &ws,
                                uint32_t w, cudaStream_t s) {
    const uint32_t n = ws[w + 1] - ws[w];
    if (!n) return CLOAK_OK;
    const int64_t chunk = std::min<int64_t>(m.unit_bytes, 64 * 1024);
    const unsigned chunks = (unsigned)((m.unit_bytes + chunk - 1) / chunk);
    const uint32_t *ops = ctx->d_plan + ops_offset(m.n_virt);
    k_rekey_wave<<<dim3(n, chunks), 256, 0, s>>>(ops, ws[w], ctx->arena, ctx->d_stage, m.unit_bytes,
                                                 chunk);
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

cloak_status rekey_run(cloak_ctx *ctx, uint64_t key, uint32_t new_epoch, cudaStream_t s) {
    cloak_status rc;
    std::vector<uint32_t> ws;
    if ((rc = keygen_page_map(ctx, key, new_epoch, ctx->d_page_new, s))) return rc;
    const MoveSet m = page_moves(ctx);
    if ((rc = plan_moves(ctx, m, s, ws))) return rc;
    for (uint32_t w = 0; w + 1 < ws.size(); ++w)
        if ((rc = launch_wave(ctx, m, ws, w, s))) return rc;
    k_copy_words<<<nblk(ctx->NPS), 256, 0, s>>>(ctx->d_page_alloc, ctx->d_page_new,
                                                (uint32_t)ctx->NPS);
    CLOAK_LAUNCHED(ctx);
    if ((rc = build_tile_slot(ctx, ctx->d_page_alloc, s))) return rc;
    ctx->epoch = new_epoch;
    return CLOAK_OK;
}

// Zero the slots of the last virtual page that hold no tile (past tile G-1),
// where a tile-level re-key may have left another tile's old bytes.
__global__ void k_zero_tail_slots(const uint32_t *page_alloc, uint32_t G, uint32_t tpp, uint32_t NP,
                                  uint8_t *arena, int64_t tile_bytes) {
    const uint32_t v = G + blockIdx.x;
    if (v >= NP * tpp) return;
    uint4 *t = reinterpret_cast<uint4 *>(arena + ((int64_t)page_alloc[v / tpp] * tpp + v % tpp) * tile_bytes);
    for (int64_t i = threadIdx.x; i < tile_bytes / 16; i += blockDim.x) t[i] = make_uint4(0, 0, 0, 0);
}

// Out-of-place tile moves: tile g from its old slot in the arena to its new
// slot in `tmp` (an arena-sized buffer); one tile per block iteration, each
// thread's 16-byte loads of the tile all in flight before its stores.
// new slot -> tile (the inverse of the new gather table; inv starts all NONE)
__global__ void k_slot_inverse(const uint32_t *__restrict__ new_slot, uint32_t G, uint32_t *__restrict__ inv) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) inv[new_slot[g]] = g;
}

// Every tile from its old slot in the arena to its new slot in tmp, taken in
// new-slot order: the blocks running at one time write one run of tmp (the
// reads are scattered either way).
__global__ void __launch_bounds__(256) k_tile_gather(const uint32_t *__restrict__ old_slot,
                                                     const uint32_t *__restrict__ inv, uint32_t nslots,
                                                     const uint8_t *__restrict__ arena, uint8_t *__restrict__ tmp,
                                                     int64_t tile_bytes) {
    constexpr int PT = 8;  // 16-byte pieces per thread and round: 32 KiB per block round
    const int64_t n16 = tile_bytes / 16;
    for (uint32_t d = blockIdx.x; d < nslots; d += gridDim.x) {
        const uint32_t g = inv[d];
        if (g == NONE) continue;
        const uint4 *src = reinterpret_cast<const uint4 *>(arena + (int64_t)old_slot[g] * tile_bytes);
        uint4 *dst = reinterpret_cast<uint4 *>(tmp + (int64_t)d * tile_bytes);
        for (int64_t i0 = 0; i0 < n16; i0 += (int64_t)PT * blockDim.x) {
            uint4 v[PT];
#pragma unroll
            for (int j = 0; j < PT; ++j) {
                const int64_t i = i0 + (int64_t)j * blockDim.x + threadIdx.x;
                if (i < n16) v[j] = __ldcs(src + i);
            }
#pragma unroll
            for (int j = 0; j < PT; ++j) {
                const int64_t i = i0 + (int64_t)j * blockDim.x + threadIdx.x;
                if (i < n16) __stcs(dst + i, v[j]);
            }
        }
    }
}

// Tile-level re-key (CLOAK_MODEL_TILE_REKEY): the tables of (key, new_epoch)
// -- a new tile permutation as well as a new page map -- and every tile moved
// from its old slot to its new one: out of place through a temporary buffer
// of the arena's size when the device has room, else in place with the same
// planner and copy waves as the page re-key, at tile granularity (the
// staging pages hold tpp tiles each). Layer order, group permutations and
// tensor bases depend on the key only, so they do not change.
cloak_status tile_rekey_run(cloak_ctx *ctx, uint64_t key, uint32_t new_epoch, cudaStream_t s) {
    cloak_status rc;
    if (!ctx->d_slot_old) CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_slot_old, (size_t)ctx->G * 4));
    CLOAK_CUDA(ctx, cudaMemcpyAsync(ctx->d_slot_old, ctx->d_tile_slot, (size_t)ctx->G * 4,
                                    cudaMemcpyDeviceToDevice, s));
    const uint32_t old_epoch = ctx->epoch;
    if ((rc = keygen_tables(ctx, key, new_epoch, s))) {
        keygen_tables(ctx, key, old_epoch, s);  // the tiles have not moved: keep their tables
        return rc;
    }
    // Out of place when an arena-sized buffer can be had (HBM is large next
    // to most models; the first such re-key allocates it and the context
    // keeps it): every tile to its new slot in the buffer, then one device
    // copy back (the arena keeps its address, so tensor maps and captured
    // graphs stay valid). Else in place, through the planner and the staging
    // pages, like the page re-key.
    const size_t bytes = (size_t)ctx->NPS * (size_t)ctx->page_bytes;
    const char *ip = getenv("CLOAK_TILE_REKEY_IN_PLACE");  // no temporary buffer wanted
    const bool in_place = ip && ip[0] == '1';
    if (!in_place && !ctx->d_tile_tmp && cudaMalloc((void **)&ctx->d_tile_tmp, bytes) != cudaSuccess) {
        ctx->d_tile_tmp = nullptr;
        cudaGetLastError();  // the failed allocation is not a sticky error
    }
    if (!in_place && ctx->d_tile_tmp) {
        const uint32_t nslots = (uint32_t)(ctx->NPS * ctx->tpp);
        if (!ctx->d_slot_inv) CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_slot_inv, (size_t)nslots * 4));
        CLOAK_CUDA(ctx, cudaMemsetAsync(ctx->d_slot_inv, 0xFF, (size_t)nslots * 4, s));
        k_slot_inverse<<<(unsigned)((ctx->G + 255) / 256), 256, 0, s>>>(ctx->d_tile_slot, (uint32_t)ctx->G,
                                                                         ctx->d_slot_inv);
        CLOAK_LAUNCHED(ctx);
        k_tile_gather<<<ctx->sm_count * 8, 256, 0, s>>>(ctx->d_slot_old, ctx->d_slot_inv, nslots, ctx->arena,
                                                        ctx->d_tile_tmp, ctx->tile_bytes);
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->arena, ctx->d_tile_tmp, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "tile re-key (out of place)");
    } else {
        const MoveSet m{ctx->d_slot_old, ctx->d_tile_slot, (uint32_t)ctx->G, (uint32_t)(ctx->NPS * ctx->tpp),
                        (uint32_t)(ctx->stage_pages * ctx->tpp), ctx->tile_bytes};
        std::vector<uint32_t> ws;
        if ((rc = plan_moves(ctx, m, s, ws))) {
            keygen_tables(ctx, key, old_epoch, s);
            return rc;
        }
        for (uint32_t w = 0; w + 1 < ws.size(); ++w)
            if ((rc = launch_wave(ctx, m, ws, w, s))) return rc;
    }
    const uint32_t tail = (uint32_t)(ctx->NP * ctx->tpp - ctx->G);
    if (tail) {
        k_zero_tail_slots<<<tail, 256, 0, s>>>(ctx->d_page_alloc, (uint32_t)ctx->G, (uint32_t)ctx->tpp,
                                               (uint32_t)ctx->NP, ctx->arena, ctx->tile_bytes);
        CLOAK_LAUNCHED(ctx);
    }
    ctx->epoch = new_epoch;
    return CLOAK_OK;
}

// ------------------------------------------------------ concurrent re-key
//
// The same plan, executed while the model keeps serving. Every wave's
// destinations are pages no published gather-table entry points at (the
// free end of a chain, a staging page, or a page whose content an earlier,
// already published wave moved away), so a wave can copy on a side stream
// while a step reads the model. After a wave has landed, a publish on the
// serving stream repoints the moved pages' tiles at their new slots; being
// stream-ordered, it runs after every step that could still read the old
// slots, so the next wave may overwrite them. Staging pages sit after the
// arena's own pages, inside the arena's tensor map, so a tile can be read
// from its staged copy in between.

__global__ void k_owner_init(uint32_t total, uint32_t *owner) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < total) owner[p] = NONE;
}

__global__ void k_owner_set(const uint32_t *pa, uint32_t NP, uint32_t *owner) {
    const uint32_t vp = blockIdx.x * blockDim.x + threadIdx.x;
    if (vp < NP) owner[pa[vp]] = vp;
}

// One block per op of the wave: the virtual page held at the source now lives
// at the destination; its tiles' gather-table entries follow it.
__global__ void k_rekey_publish(const uint32_t *ops, uint32_t op0, uint32_t *owner,
                                const uint32_t *tile_perm, uint32_t *tile_slot, uint32_t G,
                                uint32_t NPS, uint32_t tpp, int *status) {
    const uint32_t o = op0 + blockIdx.x;
    const uint32_t s = ops[2 * o], d = ops[2 * o + 1];
    if (s == NONE) return;
    const uint32_t ps = (s & STAGE_BIT) ? NPS + (s & ~STAGE_BIT) : s;
    const uint32_t pd = (d & STAGE_BIT) ? NPS + (d & ~STAGE_BIT) : d;
    // within a wave no destination is also a source, so owner[ps] is stable
    const uint32_t vp = owner[ps];
    if (vp == NONE) {
        if (threadIdx.x == 0) atomicExch(status, 3);
        return;
    }
    for (uint32_t j = threadIdx.x; j < tpp; j += blockDim.x) {
        const uint64_t v = (uint64_t)vp * tpp + j;
        if (v < G) tile_slot[tile_perm[v]] = pd * tpp + j;
    }
    if (threadIdx.x == 0) owner[pd] = vp;
}

cloak_status rekey_begin(cloak_ctx *ctx, uint64_t key, uint32_t new_epoch, cudaStream_t side) {
    cloak_status rc;
    auto &rk = ctx->rk;
    const uint32_t total = (uint32_t)(ctx->NPS + ctx->stage_pages);
    if (!rk.d_owner) CLOAK_CUDA(ctx, cudaMalloc(&rk.d_owner, (size_t)total * 4));
    if (!rk.copied) CLOAK_CUDA(ctx, cudaEventCreateWithFlags(&rk.copied, cudaEventDisableTiming));
    if (!rk.published)
        CLOAK_CUDA(ctx, cudaEventCreateWithFlags(&rk.published, cudaEventDisableTiming));
    if ((rc = keygen_page_map(ctx, key, new_epoch, ctx->d_page_new, side))) return rc;
    if ((rc = plan_moves(ctx, page_moves(ctx), side, rk.ws))) return rc;
    k_owner_init<<<nblk(total), 256, 0, side>>>(total, rk.d_owner);
    CLOAK_LAUNCHED(ctx);
    k_owner_set<<<nblk(ctx->NP), 256, 0, side>>>(ctx->d_page_alloc, (uint32_t)ctx->NP, rk.d_owner);
    CLOAK_LAUNCHED(ctx);
    rk.wave = 0;
    rk.epoch = new_epoch;
    if (rk.ws.size() > 1 && (rc = launch_wave(ctx, page_moves(ctx), rk.ws, 0, side))) return rc;
    CLOAK_CUDA(ctx, cudaEventRecord(rk.copied, side));
    rk.active = true;
    return CLOAK_OK;
}

cloak_status rekey_advance(cloak_ctx *ctx, cudaStream_t serve, cudaStream_t side, int32_t *done) {
    auto &rk = ctx->rk;
    *done = 0;
    const cudaError_t q = cudaEventQuery(rk.copied);
    if (q == cudaErrorNotReady) return CLOAK_OK;
    CLOAK_CUDA(ctx, q);
    CLOAK_CUDA(ctx, cudaStreamWaitEvent(serve, rk.copied, 0));  // already complete: orders only
    const uint32_t waves = (uint32_t)rk.ws.size() - 1;
    if (rk.wave < waves) {
        const uint32_t n = rk.ws[rk.wave + 1] - rk.ws[rk.wave];
        if (n) {
            k_rekey_publish<<<n, 128, 0, serve>>>(ctx->d_plan + ops_offset(ctx->NP), rk.ws[rk.wave],
                                                  rk.d_owner, ctx->d_tile_perm, ctx->d_tile_slot,
                                                  (uint32_t)ctx->G, (uint32_t)ctx->NPS,
                                                  (uint32_t)ctx->tpp, ctx->d_status);
            CLOAK_LAUNCHED(ctx);
        }
        ++rk.wave;
    }
    // the next non-empty wave copies once the publish has run on the serving stream
    while (rk.wave < waves && rk.ws[rk.wave + 1] == rk.ws[rk.wave]) ++rk.wave;
    if (rk.wave < waves) {
        CLOAK_CUDA(ctx, cudaEventRecord(rk.published, serve));
        CLOAK_CUDA(ctx, cudaStreamWaitEvent(side, rk.published, 0));
        cloak_status rc;
        if ((rc = launch_wave(ctx, page_moves(ctx), rk.ws, rk.wave, side))) return rc;
        CLOAK_CUDA(ctx, cudaEventRecord(rk.copied, side));
        return CLOAK_OK;
    }
    // every page is at its new place and every tile's entry points there
    k_copy_words<<<nblk(ctx->NPS), 256, 0, serve>>>(ctx->d_page_alloc, ctx->d_page_new,
                                                    (uint32_t)ctx->NPS);
    CLOAK_LAUNCHED(ctx);
    ctx->epoch = rk.epoch;
    rk.active = false;
    *done = 1;
    return CLOAK_OK;
}

}  // namespace cloak
