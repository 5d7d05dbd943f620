// gemm.cu -- prefill-shaped cloaked linears (M >= 256 tokens): y = x W^T
// with W read tile by tile through the keyed gather table, like linear.cu,
// but scheduled for reuse rather than for a weight stream.
//
// Each CTA of a persistent launch computes whole output tiles of 256 weight
// rows x 256 tokens over all of K (no split-K, no partial sums): two
// M = 128 UMMAs per K step (one per 128-row tile of the pair) share the
// activation slab, so a 64 KiB pipeline stage (two 16 KiB weight halves +
// 32 KiB of activations) feeds 2 x 128 x 256 x K-step of work. The FP32
// accumulators of both halves fill TMEM (2 x 256 columns). Tiles are taken
// row-pair-major, token-chunk-minor, so the CTAs working at one time share a
// few row pairs: each weight tile is fetched from HBM once and then hit in L2
// by the other token chunks, and the activations (a few MB) stay in L2.
// Problems are ordered longest rows first and tiles are handed out by an
// atomic counter (each CTA's first tile is its own index), so the last tiles
// to start are short ones and no CTA is left with two long ones.
//
// A K "slab" is 128 bytes wide: half of a 128x128 BF16 tile (64 columns) or a
// whole 128x128 E4M3 tile. The same code serves both types; E4M3 applies the
// per-row weight scale and per-token activation scale in the epilogue.
//
// Warp roles (320 threads): warp 0 TMA (gather-table entries fetched 32 k-tiles
// ahead by the whole warp), warp 1 TMEM owner + MMA issue, warps 2-9 epilogue:
// two warps per TMEM lane quarter, each draining half of every 32 tokens (the
// drain is instruction-bound: one warp per scheduler left the tensor cores
// idle for a third of the launch while it ran).
#include <cuda_bf16.h>

#include <algorithm>
#include <numeric>

#include "internal.cuh"
#include "ptx.cuh"

namespace cloak {

constexpr int GMAXP = 8;
constexpr int GEPI = 256;  // epilogue threads (warps 2-9)

struct GemmProblem {
    uint32_t base;         // first logical tile of the tensor
    int N, K, NT, KT;      // rows, columns, tile rows, tile columns
    int RP, TC, SL;        // row pairs, 256-token chunks, 128-byte K slabs per tile row
    uint32_t item_begin;   // first output tile of the problem in the launch
    void *y;
    const float *w_scale, *x_scale;  // E4M3 only
};

struct GemmArgs {
    const uint32_t *slot_of;  // gather table; nullptr: uncloaked (slot = tile index)
    int np, M, out_f32, relu;
    uint32_t items;
    uint32_t *next;           // tiles handed out after each CTA's first (zeroed per launch)
    int *status;
    GemmProblem p[GMAXP];
};

struct GemmMaps {
    CUtensorMap x[GMAXP];  // activations of each problem: [M, K], box 128 bytes x 256 rows
};

template <bool FP8>
struct GemmCfg {
    static constexpr int A_HALF = 16384;          // 128 weight rows x 128 bytes
    static constexpr int B_BYTES = 256 * 128;     // 256 tokens x 128 bytes
    static constexpr int STAGE = 2 * A_HALF + B_BYTES;
    static constexpr int STAGES = 3;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 1024 + 2048;  // + two tiles' activation scales
    static constexpr int QD = 4;                  // depth of the tile-index queue
    static constexpr uint32_t IDESC = idesc_make(FP8 ? 0u : 1u, 128, 256);
};

struct GItem {
    int p;
    int rp, tc;
    bool two;  // the pair's second tile row exists
};

__device__ __forceinline__ GItem gitem(const GemmArgs &g, uint32_t it) {
    int p = 0;
    while (p + 1 < g.np && it >= g.p[p + 1].item_begin) ++p;
    const GemmProblem &P = g.p[p];
    const uint32_t local = it - P.item_begin;
    GItem r;
    r.p = p;
    r.rp = (int)(local / (uint32_t)P.TC);
    r.tc = (int)(local % (uint32_t)P.TC);
    r.two = 2 * r.rp + 1 < P.NT;
    return r;
}

// arena slot of tile (row, kt) of problem P (0 past the row's end)
__device__ __forceinline__ uint32_t gslot(const GemmArgs &g, const GemmProblem &P, int row, int kt) {
    if (row >= P.NT || kt >= P.KT) return 0;
    const uint32_t t = P.base + (uint32_t)row * (uint32_t)P.KT + (uint32_t)kt;
    return g.slot_of ? __ldg(g.slot_of + t) : t;
}

template <bool FP8>
__global__ void __launch_bounds__(64 + GEPI, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tw, const __grid_constant__ GemmMaps xm,
              const __grid_constant__ GemmArgs g) {
    using C = GemmCfg<FP8>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::STAGES * C::STAGE);
    uint64_t *empty = full + C::STAGES;
    uint64_t *tfull = empty + C::STAGES;
    uint64_t *tempty = tfull + 1;
    uint64_t *id_full = tempty + 1;     // [QD] a tile index is published
    uint64_t *id_empty = id_full + C::QD;  // [QD] the MMA thread and all epilogue threads read it
    uint32_t *ids = reinterpret_cast<uint32_t *>(id_empty + C::QD);
    uint32_t *tmem_slot = ids + C::QD;
    float *xs_smem = reinterpret_cast<float *>(smem + C::STAGES * C::STAGE + 1024);  // [2][256]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, GEPI);
        for (int q = 0; q < C::QD; ++q) {
            mbar_init(&id_full[q], 1);
            mbar_init(&id_empty[q], 1 + GEPI);
        }
        fence_mbar_init();
        prefetch_tmap(&tw);
        for (int p = 0; p < g.np; ++p) prefetch_tmap(&xm.x[p]);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        const uint64_t pol_w = policy_evict_last(), pol_x = policy_evict_last();
        uint32_t it = 0;  // slab counter over all items (ring position)
        bool ok = true;
        for (uint32_t n = 0; ok; ++n) {
            // next tile: publish its index to the MMA and epilogue warps
            uint32_t item = 0;
            if (lane == 0) {
                const int q = n % C::QD;
                if (n >= (uint32_t)C::QD) ok = mbar_wait(&id_empty[q], ((n / C::QD) & 1) ^ 1, g.status);
                item = n == 0 ? blockIdx.x : gridDim.x + atomicAdd(g.next, 1u);
                if (item >= g.items || !ok) item = NONE;
                ids[q] = item;
                mbar_arrive(&id_full[q]);
            }
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item == NONE) break;
            const GItem w = gitem(g, item);
            const GemmProblem &P = g.p[w.p];
            const int r0 = 2 * w.rp, r1 = r0 + 1;
            // gather-table entries of the pair's two tile rows, 32 k-tiles per
            // fetch, one fetch ahead
            uint32_t c0 = gslot(g, P, r0, lane), c1 = w.two ? gslot(g, P, r1, lane) : 0;
            uint32_t n0 = gslot(g, P, r0, 32 + lane), n1 = w.two ? gslot(g, P, r1, 32 + lane) : 0;
            for (int sl = 0; sl < P.SL; ++sl, ++it) {
                const int kt = FP8 ? sl : (sl >> 1);
                const int col = FP8 ? 0 : (sl & 1) * 64;
                if ((kt & 31) == 0 && kt > 0 && (FP8 || (sl & 1) == 0)) {
                    c0 = n0;
                    c1 = n1;
                    n0 = gslot(g, P, r0, kt + 32 + lane);
                    n1 = w.two ? gslot(g, P, r1, kt + 32 + lane) : 0;
                }
                const uint32_t s0 = __shfl_sync(0xffffffffu, c0, kt & 31);
                const uint32_t s1 = __shfl_sync(0xffffffffu, c1, kt & 31);
                const int s = it % C::STAGES;
                if (lane == 0) {
                    if (it >= (uint32_t)C::STAGES) ok = mbar_wait(&empty[s], ((it / C::STAGES) & 1) ^ 1, g.status);
                    if (ok) {
                        uint8_t *sa = smem + s * C::STAGE;
                        mbar_expect_tx(&full[s], (w.two ? 2 : 1) * C::A_HALF + C::B_BYTES);
                        tma_load_2d_hint(sa, &tw, &full[s], col, (int32_t)(s0 * 128u), pol_w);
                        if (w.two) tma_load_2d_hint(sa + C::A_HALF, &tw, &full[s], col, (int32_t)(s1 * 128u), pol_w);
                        tma_load_2d_hint(sa + 2 * C::A_HALF, &xm.x[w.p], &full[s], sl * (FP8 ? 128 : 64),
                                         w.tc * 256, pol_x);
                    }
                }
                ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------------------- MMA
        if (lane == 0) {
            uint32_t it = 0, n = 0;
            bool ok = true;
            for (;; ++n) {
                const int q = n % C::QD;
                if (!mbar_wait(&id_full[q], (n / C::QD) & 1, g.status)) break;
                const uint32_t item = ids[q];
                mbar_arrive(&id_empty[q]);
                if (item == NONE) break;
                const GItem w = gitem(g, item);
                const GemmProblem &P = g.p[w.p];
                // the epilogue has drained the previous tile's accumulators
                if (n > 0 && !mbar_wait(tempty, (n - 1) & 1, g.status)) break;
                tc_fence_after();
                for (int sl = 0; sl < P.SL; ++sl, ++it) {
                    const int s = it % C::STAGES;
                    if (!mbar_wait(&full[s], (it / C::STAGES) & 1, g.status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * C::STAGE), sb = sa + 2 * C::A_HALF;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (h == 1 && !w.two) break;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = sdesc_sw128(sa + h * C::A_HALF + kk * 32);
                            const uint64_t bd = sdesc_sw128(sb + kk * 32);
                            if (FP8) umma_f8(tmem + h * 256, ad, bd, C::IDESC, (sl > 0 || kk > 0) ? 1u : 0u);
                            else umma_f16(tmem + h * 256, ad, bd, C::IDESC, (sl > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(tfull);
            }
            (void)ok;
        }
    } else {
        // ---------------------------------------------------------- epilogue
        const int qd = warp & 3;               // TMEM lane quarter of this warp
        const int r_in = qd * 32 + lane;
        const int th = (warp >= 6) ? 16 : 0;   // which 16 of every 32 tokens
        const int et = threadIdx.x - 64;
        for (uint32_t n = 0;; ++n) {
            const int q = n % C::QD;
            if (!mbar_wait(&id_full[q], (n / C::QD) & 1, g.status)) break;
            const uint32_t item = ids[q];
            mbar_arrive(&id_empty[q]);
            if (item == NONE) break;
            const GItem w = gitem(g, item);
            const GemmProblem &P = g.p[w.p];
            float wsc[2] = {1.0f, 1.0f};
            float *xs = xs_smem + (n & 1) * 256;  // the tile's activation scales (E4M3)
            if (FP8) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int row = w.rp * 256 + h * 128 + r_in;
                    wsc[h] = row < P.N ? P.w_scale[row] : 0.0f;
                }
                // two buffers by tile parity: the one written here was last read
                // two tiles ago, before the barrier below of the previous tile
                if (et < 256) {
                    const int m = w.tc * 256 + et;
                    xs[et] = m < g.M ? P.x_scale[m] : 0.0f;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(GEPI) : "memory");
            }
            const int N = P.N;
            const int nh = w.two ? 2 : 1;
            if (!mbar_wait(tfull, n & 1, g.status)) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16);
            // per round, this warp's 16 tokens of both row halves: two TMEM
            // loads, one wait; then 16 outputs per row along a running pointer
#pragma unroll 1
            for (int c0 = th; c0 < 256; c0 += 32) {
                const int m0 = w.tc * 256 + c0;
                if (m0 >= g.M) break;
                const int nt = min(16, g.M - m0);
                uint32_t v[2][16];
                tmem_ld16_nw(taddr + c0, v[0]);
                if (nh == 2) tmem_ld16_nw(taddr + 256 + c0, v[1]);
                tmem_wait_ld(v[0]);
                if (nh == 2) tmem_hold(v[1]);
                float sx[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) sx[j] = FP8 ? xs[c0 + j] : 1.0f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (h >= nh) break;
                    const int row = w.rp * 256 + h * 128 + r_in;
                    if (row >= N) continue;
                    float o[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        o[j] = __uint_as_float(v[h][j]);
                        if (FP8) o[j] *= wsc[h] * sx[j];
                        if (g.relu) o[j] = fmaxf(o[j], 0.0f);
                    }
                    if (g.out_f32) {
                        float *py = reinterpret_cast<float *>(P.y) + (int64_t)m0 * N + row;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (j < nt) *py = o[j];
                            py += N;
                        }
                    } else {
                        __nv_bfloat16 *py = reinterpret_cast<__nv_bfloat16 *>(P.y) + (int64_t)m0 * N + row;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (j < nt) *py = __float2bfloat16_rn(o[j]);
                            py += N;
                        }
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(tempty);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

template <bool FP8>
static cloak_status gemm_launch(cloak_ctx *ctx, const CUtensorMap &tw, const GemmMaps &mp, const GemmArgs &g,
                                int grid, cudaStream_t s) {
    using C = GemmCfg<FP8>;
    static std::atomic<uint64_t> attr_devs{0};  // per instantiation: devices set up
    if (attr_needed(attr_devs, ctx->device)) {
        CLOAK_CUDA(ctx, cudaFuncSetAttribute(k_gemm_tc<FP8>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        attr_set_on(attr_devs, ctx->device);
    }
    k_gemm_tc<FP8><<<grid, 64 + GEPI, C::SMEM, s>>>(tw, mp, g);
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

cloak_status gemm_run(cloak_ctx *ctx, int n, const int32_t *tensors, const void *const *xs,
                      const float *const *x_scales, void *const *ys, int M, int out_f32, int relu,
                      const uint32_t *slot_of, const CUtensorMap &tw, cudaStream_t s) {
    if (n < 1 || n > GMAXP || M < 1) return CLOAK_E_INVAL;
    const bool fp8 = ctx->dtype == CLOAK_E4M3;
    if (!fp8 && ctx->dtype != CLOAK_BF16) return CLOAK_E_UNSUPPORTED;
    // problems with the longest rows first, so the last wave holds short tiles
    int order[GMAXP];
    std::iota(order, order + n, 0);
    std::stable_sort(order, order + n, [&](int a, int b) {
        return ctx->info[tensors[a]].kt > ctx->info[tensors[b]].kt;
    });
    GemmArgs g{};
    GemmMaps mp;
    g.slot_of = slot_of;
    g.np = n;
    g.M = M;
    g.out_f32 = out_f32;
    g.relu = relu;
    g.status = ctx->d_status;
    const int es = fp8 ? 1 : 2;
    uint32_t items = 0;
    for (int i = 0; i < n; ++i) {
        const int q = order[i];
        const TensorInfo &ti = ctx->info[tensors[q]];
        GemmProblem &P = g.p[i];
        P.base = ctx->h_tensor_base[tensors[q]];
        P.N = ti.n;
        P.K = ti.k;
        P.NT = ti.nt;
        P.KT = ti.kt;
        P.RP = (ti.nt + 1) / 2;
        P.TC = (M + 255) / 256;
        P.SL = fp8 ? ti.kt : 2 * ti.kt;
        P.item_begin = items;
        items += (uint32_t)P.RP * (uint32_t)P.TC;
        P.y = ys[q];
        P.w_scale = fp8 ? ctx->d_scales + ti.scale_off : nullptr;
        P.x_scale = fp8 ? x_scales[q] : nullptr;
        if (!encode_tmap_2d(&mp.x[i], fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                            xs[q], (uint64_t)ti.k, (uint64_t)M, (uint64_t)ti.k * es, 128 / es, 256)) {
            ctx->last_err = "cuTensorMapEncodeTiled failed for x";
            return CLOAK_E_CUDA;
        }
    }
    g.items = items;
    if (!ctx->d_gemm_next) CLOAK_CUDA(ctx, cudaMalloc(&ctx->d_gemm_next, 256));
    CLOAK_CUDA(ctx, cudaMemsetAsync(ctx->d_gemm_next, 0, sizeof(uint32_t), s));
    g.next = (uint32_t *)ctx->d_gemm_next;
    const int grid = (int)std::min<uint32_t>(items, (uint32_t)ctx->sm_count);
    return fp8 ? gemm_launch<true>(ctx, tw, mp, g, grid, s) : gemm_launch<false>(ctx, tw, mp, g, grid, s);
}

}  // namespace cloak
