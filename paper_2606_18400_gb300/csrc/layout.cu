// layout.cu -- placing weights into the cloaked arena and moving them.
//
//   shuffle    logical FP32 weights -> permuted rows/columns (intra-layer
//              shuffling), converted (BF16 RNE / E4M3 with per-row scale),
//              cut into tiles, each tile written to its keyed slot
//              (inter-layer shuffling + page remapping, Section 4.2);
//   unshuffle  the exact inverse, in the storage type;
//   rekey      periodic re-randomisation (Section 4.2, "Physical page
//              remapping"; Figure 7): every page moves from its physical page
//              under the old map to its physical page under the new one, in
//              place. The moves form chains and cycles over physical pages;
//              each is cut into segments executed in parallel waves, and the
//              page a segment's last move reads (the one the next segment
//              overwrites first) is staged in a small pool beforehand.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace cloak {

static inline unsigned nblk(uint64_t n, unsigned b = 256) { return (unsigned)((n + b - 1) / b); }

// stored index -> logical index on the tensor's permuted axis
__device__ __forceinline__ int64_t perm_map(const uint32_t *gp, int32_t unit, int64_t i) {
    return (int64_t)gp[i / unit] * unit + i % unit;
}

// stored row / column -> logical row / column (gp: all group permutations)
__device__ __forceinline__ int64_t row_map(const uint32_t *gp, const TensorInfo &ti, int64_t r) {
    return ti.r_unit ? perm_map(gp + ti.r_goff, ti.r_unit, r) : r;
}
__device__ __forceinline__ int64_t col_map(const uint32_t *gp, const TensorInfo &ti, int64_t c) {
    return ti.c_unit ? perm_map(gp + ti.c_goff, ti.c_unit, c) : c;
}

// per stored row: scale = amax(|row|) / 448 (1 if the row is zero), FP32
// (the row's column order does not change its maximum)
__global__ void k_row_scales(const float *W, TensorInfo ti, const uint32_t *gp, float *scales) {
    int64_t r = blockIdx.x;
    int64_t lr = row_map(gp, ti, r);
    const float *row = W + lr * ti.k;
    float m = 0.0f;
    for (int c = threadIdx.x; c < ti.k; c += blockDim.x) m = fmaxf(m, fabsf(row[c]));
    __shared__ float red[32];
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) scales[r] = m > 0.0f ? __fdiv_rn(m, 448.0f) : 1.0f;
    }
}

template <int ES>
struct Elem;
template <>
struct Elem<4> { using T = float; };
template <>
struct Elem<2> { using T = uint16_t; };
template <>
struct Elem<1> { using T = uint8_t; };

template <int ES>
__device__ __forceinline__ typename Elem<ES>::T encode(float v, float s) {
    if constexpr (ES == 4) {
        return v;
    } else if constexpr (ES == 2) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    } else {
        return (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(v, s), __NV_SATFINITE, __NV_E4M3);
    }
}

// One block per tile of the tensor; writes the whole tile (zeros outside
// the matrix) to the arena slot and, if present, to the twin's slot g.
template <int ES>
__global__ void k_shuffle(const float *W, TensorInfo ti, int tile_r, int tile_c, uint32_t base,
                          const uint32_t *slot_of, const uint32_t *gp, const float *scales,
                          uint8_t *arena, uint8_t *twin, int64_t tile_bytes) {
    using T = typename Elem<ES>::T;
    const int64_t u = blockIdx.x;
    const int64_t nt = u / ti.kt, kt = u % ti.kt;
    const uint32_t g = base + (uint32_t)u;
    T *dst = reinterpret_cast<T *>(arena + (int64_t)slot_of[g] * tile_bytes);
    T *dst2 = twin ? reinterpret_cast<T *>(twin + (int64_t)g * tile_bytes) : nullptr;
    const int elems = tile_r * tile_c;
    for (int e = threadIdx.x; e < elems; e += blockDim.x) {
        int i = e / tile_c, j = e % tile_c;
        int64_t r = nt * tile_r + i, c = kt * tile_c + j;
        float v = 0.0f, s = 1.0f;
        if (r < ti.n && c < ti.k) {
            int64_t lr = row_map(gp, ti, r);
            int64_t lc = col_map(gp, ti, c);
            v = W[lr * ti.k + lc];
            if (ES == 1) s = scales[r];
        }
        T q = encode<ES>(v, s);
        dst[e] = q;
        if (dst2) dst2[e] = q;
    }
}

template <int ES>
__global__ void k_unshuffle(const uint8_t *arena, TensorInfo ti, int tile_r, int tile_c,
                            uint32_t base, const uint32_t *slot_of, const uint32_t *gp,
                            uint8_t *out, int64_t tile_bytes, int from_twin) {
    using T = typename Elem<ES>::T;
    const int64_t u = blockIdx.x;
    const int64_t nt = u / ti.kt, kt = u % ti.kt;
    const uint32_t g = base + (uint32_t)u;
    const int64_t slot = from_twin ? (int64_t)g : (int64_t)slot_of[g];
    const T *src = reinterpret_cast<const T *>(arena + slot * tile_bytes);
    T *o = reinterpret_cast<T *>(out);
    const int elems = tile_r * tile_c;
    for (int e = threadIdx.x; e < elems; e += blockDim.x) {
        int i = e / tile_c, j = e % tile_c;
        int64_t r = nt * tile_r + i, c = kt * tile_c + j;
        if (r >= ti.n || c >= ti.k) continue;
        int64_t lr = row_map(gp, ti, r);
        int64_t lc = col_map(gp, ti, c);
        o[lr * ti.k + lc] = src[e];
    }
}

cloak_status launch_shuffle(cloak_ctx *ctx, int t, const float *src, cudaStream_t s) {
    const TensorInfo &ti = ctx->info[t];
    const uint32_t *gp = ctx->d_group_perm;
    float *sc = ctx->d_scales + ti.scale_off;
    unsigned tiles = (unsigned)(ti.nt * ti.kt);
    uint32_t base = ctx->h_tensor_base[t];
    if (ctx->dtype == CLOAK_E4M3) {
        k_row_scales<<<ti.n, 256, 0, s>>>(src, ti, gp, sc);
        CLOAK_LAUNCHED(ctx);
    }
#define SHUF(ES)                                                                         \
    k_shuffle<ES><<<tiles, 256, 0, s>>>(src, ti, ctx->tile_r, ctx->tile_c, base,          \
                                        ctx->d_tile_slot, gp, sc, ctx->arena, ctx->twin, \
                                        ctx->tile_bytes)
    if (ctx->esize == 4) SHUF(4);
    else if (ctx->esize == 2) SHUF(2);
    else SHUF(1);
#undef SHUF
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}

cloak_status launch_unshuffle(const cloak_ctx *cctx, int t, void *dst, int from_twin,
                              cudaStream_t s) {
    cloak_ctx *ctx = const_cast<cloak_ctx *>(cctx);
    const TensorInfo &ti = ctx->info[t];
    const uint32_t *gp = ctx->d_group_perm;
    unsigned tiles = (unsigned)(ti.nt * ti.kt);
    const uint8_t *a = from_twin ? ctx->twin : ctx->arena;
#define UNSHUF(ES)                                                                          \
    k_unshuffle<ES><<<tiles, 256, 0, s>>>(a, ti, ctx->tile_r, ctx->tile_c,                  \
                                          ctx->h_tensor_base[t], ctx->d_tile_slot, gp,      \
                                          (uint8_t *)dst, ctx->tile_bytes, from_twin)
    if (ctx->esize == 4) UNSHUF(4);
    else if (ctx->esize == 2) UNSHUF(2);
    else UNSHUF(1);
#undef UNSHUF
    CLOAK_LAUNCHED(ctx);
    return CLOAK_OK;
}


}  // namespace cloak
