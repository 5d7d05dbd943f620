// selftest.cu -- failure detection checked without a fault: waits that
// nothing satisfies must give up after their limit, record a timeout in the
// device status word the host reads, and leave the context usable.
#include "internal.cuh"
#include "ptx.cuh"

namespace cloak {

namespace {

// Thread 0 waits on an mbarrier whose one arrival never comes (the helper
// every pipelined kernel waits with); thread 32 spins on a flag that
// nothing sets, with the same time limit. seen[i] = 1 when wait i gave up.
__global__ void k_check_waits(const volatile int *flag, int *status, int *seen) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        seen[0] = mbar_wait(&bar, 0, status) ? 0 : 1;
    } else if (threadIdx.x == 32) {
        const unsigned long long t0 = globaltimer();
        int gave_up = 0;
        for (uint32_t it = 0;; ++it) {
            if (*flag) break;
            if ((it & 255u) == 0 && globaltimer() - t0 > WAIT_LIMIT_NS) {
                atomicExch(status, DEV_E_TIMEOUT);
                gave_up = 1;
                break;
            }
        }
        seen[1] = gave_up;
    }
}

}  // namespace

cloak_status check_waits_run(cloak_ctx *ctx, cudaStream_t s) {
    int *d = nullptr;  // [0] flag (never set), [1..2] seen
    CLOAK_CUDA(ctx, cudaMalloc(&d, 3 * sizeof(int)));
    cloak_status rc = CLOAK_OK;
    int h[3] = {0, 0, 0}, st = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(int), s);
    if (e == cudaSuccess) {
        k_check_waits<<<1, 64, 0, s>>>(d, ctx->d_status, d + 1);
        ctx->launches++;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "wait self-test");
    if (h[1] != 1 || h[2] != 1 || st != DEV_E_TIMEOUT) {
        ctx->last_err = "a bounded wait did not report its timeout";
        rc = CLOAK_E_CUDA;
    }
    return rc;
}

}  // namespace cloak
