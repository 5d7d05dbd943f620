// noalloc.cu -- cloak_linear_noalloc: the BF16 cloaked linear for callers
// that must not allocate device memory while they run (see include/cloak.h).
//
// The split-K partial sums and the tile-row arrival counters that
// cloak_linear keeps in context-owned buffers (grown on demand with
// cudaMalloc) live here in one fixed file-scope device array instead. Every
// GPU that loads the library holds this array until the process exits.
#include <mutex>

#include "internal.cuh"

namespace cloak {
namespace {

// Limits of the allocation-free path. The array holds the partial sums of
// the largest launch cloak_linear can make for these batches: the autotuner
// tries up to 4 CTAs per SM, and devices of up to 160 SMs are supported.
constexpr int NOALLOC_MAX_M = 32;                        // rows of x (MMA N padded to 16 or 32)
constexpr uint32_t NOALLOC_MAX_SMS = 160;                // SMs of the device (GB300: 152)
constexpr uint32_t NOALLOC_MAX_GRID = 4 * NOALLOC_MAX_SMS;  // CTAs of one launch
constexpr uint32_t NOALLOC_MAX_ROWS = 4096;              // tile rows of one tensor (n <= 524,288)
constexpr size_t NOALLOC_PART_FLOATS = (size_t)NOALLOC_MAX_GRID * 2 * 128 * NOALLOC_MAX_M;
constexpr size_t NOALLOC_PART_BYTES = NOALLOC_PART_FLOATS * sizeof(float);      // 20 MiB
constexpr size_t NOALLOC_BYTES = NOALLOC_PART_BYTES + NOALLOC_MAX_ROWS * sizeof(uint32_t);

// partial sums at offset 0, row counters after them
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
struct DeviceScratch {
    std::mutex mu;
    unsigned char *ptr = nullptr;  // device address of g_noalloc_scratch on this device; set on success only
};
DeviceScratch g_dev[MAX_DEVICES];

}  // namespace
}  // namespace cloak

using namespace cloak;

extern "C" cloak_status cloak_linear_noalloc(cloak_ctx *ctx, int32_t tensor, const void *x_dev,
                                             void *y_dev, int32_t M, int32_t out_dtype,
                                             int32_t flags, void *stream) {
    if (!ctx || !x_dev || !y_dev || tensor < 0 || tensor >= (int32_t)ctx->tensors.size() ||
        (out_dtype != CLOAK_OUT_F32 && out_dtype != CLOAK_OUT_BF16) || (flags & ~3) ||
        ((uintptr_t)x_dev & 15))
        return CLOAK_E_INVAL;
    if (M < 1 || M > NOALLOC_MAX_M) {
        ctx->last_err = "cloak_linear_noalloc: M must be in [1, 32]";
        return CLOAK_E_INVAL;
    }
    if (ctx->dtype != CLOAK_BF16) {
        ctx->last_err = "cloak_linear_noalloc: BF16 models only";
        return CLOAK_E_UNSUPPORTED;
    }
    if ((uint32_t)ctx->info[tensor].nt > NOALLOC_MAX_ROWS) {
        ctx->last_err = "cloak_linear_noalloc: tensor has more than 4096 tile rows";
        return CLOAK_E_INVAL;
    }
    if ((uint32_t)ctx->sm_count > NOALLOC_MAX_SMS) {
        ctx->last_err = "cloak_linear_noalloc: devices of more than 160 SMs are not supported";
        return CLOAK_E_UNSUPPORTED;
    }
    if (!ctx->keyed) return CLOAK_E_STATE;
    if ((flags & CLOAK_LINEAR_UNCLOAKED) && !ctx->twin) return CLOAK_E_STATE;
    if (ctx->device < 0 || ctx->device >= MAX_DEVICES) return CLOAK_E_UNSUPPORTED;
    CLOAK_CUDA(ctx, cudaSetDevice(ctx->device));
    // once per device, with that device current: the array's device address
    // (host code cannot use the symbol itself). A failed look-up is not kept:
    // the next call tries again.
    DeviceScratch &d = g_dev[ctx->device];
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(d.mu);
        if (!d.ptr) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return cuda_fail(ctx, e, "noalloc scratch set-up");
            d.ptr = (unsigned char *)p;
        }
        base = d.ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *rowcnt = reinterpret_cast<uint32_t *>(base + NOALLOC_PART_BYTES);
    // counters must start at zero; a completed call leaves them zero, an
    // aborted one or another tensor's may not, so clear the ones this tensor uses
    CLOAK_CUDA(ctx, cudaMemsetAsync(rowcnt, 0, (size_t)ctx->info[tensor].nt * sizeof(uint32_t), s));
    return linear_run_given_scratch(ctx, tensor, x_dev, y_dev, M, out_dtype, flags,
                                    reinterpret_cast<float *>(base), NOALLOC_PART_FLOATS, rowcnt, s);
}
