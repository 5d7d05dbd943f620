// vmm.cu -- physical page remapping through CUDA virtual memory management
// (Section 4.2, "Physical page remapping"; Table 1b).
//
// With CLOAK_MODEL_VMM the arena is not one cudaMalloc block but one
// physical chunk (cuMemCreate) per arena page, including the re-key staging
// pages. Each chunk is mapped twice:
//   * the physical view (ctx->arena): chunk p at page p. Every kernel that
//     gathers through the tile-slot table, the shuffle and the re-key copies
//     run on it unchanged.
//   * the virtual view (ctx->vview): virtual page vp is backed by chunk
//     page_alloc[vp] (vp < NP). A kernel reading a tile at its virtual
//     position v (tile permutation only) finds it at vview + v * tile_bytes:
//     the page step of the gather is done by the MMU, as in the paper, where
//     tensor pointers stay fixed while the pages behind them move.
// The two views alias the same memory, so the mode adds no footprint. The
// virtual view is remapped after every keygen and re-key, at a sync point:
// the device is synchronised before any page is unmapped, so no kernel of
// this process reads a page while its mapping changes.
#include <cudaTypedefs.h>

#include <chrono>
#include <mutex>

#include "internal.cuh"

namespace cloak {

namespace {

struct VmmApi {
    PFN_cuMemCreate_v10020 create = nullptr;
    PFN_cuMemRelease_v10020 release = nullptr;
    PFN_cuMemAddressReserve_v10020 reserve = nullptr;
    PFN_cuMemAddressFree_v10020 addr_free = nullptr;
    PFN_cuMemMap_v10020 map = nullptr;
    PFN_cuMemUnmap_v10020 unmap = nullptr;
    PFN_cuMemSetAccess_v10020 set_access = nullptr;
    PFN_cuMemGetAllocationGranularity_v10020 granularity = nullptr;
    bool ok = false;
};

VmmApi g_vmm;
std::once_flag g_vmm_once;

template <class F>
bool entry(const char *name, F &out) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &fn, 10020, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return false;
    out = reinterpret_cast<F>(fn);
    return true;
}

const VmmApi &api() {
    std::call_once(g_vmm_once, [] {
        VmmApi a;
        a.ok = entry("cuMemCreate", a.create) && entry("cuMemRelease", a.release) &&
               entry("cuMemAddressReserve", a.reserve) && entry("cuMemAddressFree", a.addr_free) &&
               entry("cuMemMap", a.map) && entry("cuMemUnmap", a.unmap) &&
               entry("cuMemSetAccess", a.set_access) &&
               entry("cuMemGetAllocationGranularity", a.granularity);
        g_vmm = a;
    });
    return g_vmm;
}

CUmemAllocationProp chunk_prop(int device) {
    CUmemAllocationProp p{};
    p.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    p.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    p.location.id = device;
    return p;
}

cloak_status drv_fail(cloak_ctx *ctx, CUresult r, const char *where) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s failed (CUresult %d)", where, (int)r);
    ctx->last_err = buf;
    return r == CUDA_ERROR_OUT_OF_MEMORY ? CLOAK_E_NOMEM : CLOAK_E_CUDA;
}

#define VMM_DRV(ctx, call, where)                          \
    do {                                                   \
        CUresult r_ = (call);                              \
        if (r_ != CUDA_SUCCESS) return drv_fail(ctx, r_, where); \
    } while (0)

cloak_status set_rw(cloak_ctx *ctx, CUdeviceptr va, size_t bytes) {
    CUmemAccessDesc acc{};
    acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    acc.location.id = ctx->device;
    acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    VMM_DRV(ctx, api().set_access(va, bytes, &acc, 1), "cuMemSetAccess");
    return CLOAK_OK;
}

}  // namespace

cloak_status vmm_create(cloak_ctx *ctx, int64_t chunks) {
    const VmmApi &a = api();
    if (!a.ok) {
        ctx->last_err = "CUDA virtual memory management entry points not found";
        return CLOAK_E_UNSUPPORTED;
    }
    CUmemAllocationProp prop = chunk_prop(ctx->device);
    size_t gran = 0;
    VMM_DRV(ctx, a.granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_MINIMUM),
            "cuMemGetAllocationGranularity");
    if (gran == 0 || ctx->page_bytes % (int64_t)gran) {
        ctx->last_err = "page_bytes must be a multiple of the VMM allocation granularity (" +
                        std::to_string(gran) + " bytes)";
        return CLOAK_E_UNSUPPORTED;
    }
    const size_t P = (size_t)ctx->page_bytes;
    ctx->vmm_chunks.reserve((size_t)chunks);
    for (int64_t i = 0; i < chunks; ++i) {
        CUmemGenericAllocationHandle h;
        VMM_DRV(ctx, a.create(&h, P, &prop, 0), "cuMemCreate");
        ctx->vmm_chunks.push_back(h);
    }
    CUdeviceptr pv = 0, vv = 0;
    VMM_DRV(ctx, a.reserve(&pv, P * (size_t)chunks, P, 0, 0), "cuMemAddressReserve");
    ctx->vmm_phys_bytes = P * (size_t)chunks;
    ctx->arena = reinterpret_cast<uint8_t *>(pv);
    for (int64_t i = 0; i < chunks; ++i) {
        VMM_DRV(ctx, a.map(pv + (CUdeviceptr)(i * P), P, 0, ctx->vmm_chunks[i], 0), "cuMemMap");
        ctx->vmm_phys_mapped = i + 1;
    }
    if (cloak_status rc = set_rw(ctx, pv, P * (size_t)chunks)) return rc;
    VMM_DRV(ctx, a.reserve(&vv, P * (size_t)ctx->NP, P, 0, 0), "cuMemAddressReserve");
    ctx->vview = reinterpret_cast<uint8_t *>(vv);
    ctx->vmm_map.assign((size_t)ctx->NP, NONE);
    return CLOAK_OK;
}

cloak_status vmm_remap(cloak_ctx *ctx) {
    const VmmApi &a = api();
    const auto t0 = std::chrono::steady_clock::now();
    ctx->vmm_ready = false;  // until every page is mapped again
    // the sync point: nothing of this process may read the view while its
    // pages are unmapped
    CLOAK_CUDA(ctx, cudaDeviceSynchronize());
    std::vector<uint32_t> pa((size_t)ctx->NP);
    CLOAK_CUDA(ctx, cudaMemcpy(pa.data(), ctx->d_page_alloc, pa.size() * 4, cudaMemcpyDeviceToHost));
    const size_t P = (size_t)ctx->page_bytes;
    const CUdeviceptr vv = reinterpret_cast<CUdeviceptr>(ctx->vview);
    const uint32_t nch = (uint32_t)ctx->vmm_chunks.size();
    for (int64_t vp = 0; vp < ctx->NP; ++vp)
        if (pa[vp] >= nch) {
            ctx->last_err = "page map entry out of range";
            return CLOAK_E_CUDA;
        }
    // runs of consecutive virtual pages whose chunk changes: one unmap per
    // run of mapped pages, one map per page, one access grant per run. A
    // page's entry in vmm_map is written only once its run is accessible, so
    // after a failure the view stays refused (vmm_ready false) and no entry
    // claims a page that a kernel could not read.
    int64_t changed = 0;
    for (int64_t v0 = 0; v0 < ctx->NP;) {
        if (ctx->vmm_map[v0] == pa[v0]) { ++v0; continue; }
        int64_t v1 = v0;
        while (v1 < ctx->NP && ctx->vmm_map[v1] != pa[v1]) ++v1;
        for (int64_t u0 = v0; u0 < v1;) {
            if (ctx->vmm_map[u0] == NONE) { ++u0; continue; }
            int64_t u1 = u0;
            while (u1 < v1 && ctx->vmm_map[u1] != NONE) ++u1;
            VMM_DRV(ctx, a.unmap(vv + (CUdeviceptr)(u0 * P), (size_t)(u1 - u0) * P), "cuMemUnmap");
            for (int64_t u = u0; u < u1; ++u) ctx->vmm_map[u] = NONE;
            u0 = u1;
        }
        for (int64_t v = v0; v < v1; ++v)
            VMM_DRV(ctx, a.map(vv + (CUdeviceptr)(v * P), P, 0, ctx->vmm_chunks[pa[v]], 0), "cuMemMap");
        if (cloak_status rc = set_rw(ctx, vv + (CUdeviceptr)(v0 * P), (size_t)(v1 - v0) * P)) return rc;
        for (int64_t v = v0; v < v1; ++v) ctx->vmm_map[v] = pa[v];
        changed += v1 - v0;
        v0 = v1;
    }
    ctx->vmm_remapped = changed;
    ctx->vmm_remaps++;
    ctx->vmm_remap_us = std::chrono::duration_cast<std::chrono::microseconds>(
                            std::chrono::steady_clock::now() - t0).count();
    ctx->vmm_ready = true;
    return CLOAK_OK;
}

void vmm_release(cloak_ctx *ctx) {
    const VmmApi &a = api();
    if (!a.ok) return;
    const size_t P = (size_t)ctx->page_bytes;
    if (ctx->vview) {
        const CUdeviceptr vv = reinterpret_cast<CUdeviceptr>(ctx->vview);
        for (size_t vp = 0; vp < ctx->vmm_map.size(); ++vp)
            if (ctx->vmm_map[vp] != NONE) a.unmap(vv + (CUdeviceptr)(vp * P), P);
        a.addr_free(vv, P * (size_t)ctx->NP);
        ctx->vview = nullptr;
    }
    if (ctx->arena && ctx->vmm_phys_bytes) {
        const CUdeviceptr pv = reinterpret_cast<CUdeviceptr>(ctx->arena);
        for (int64_t i = 0; i < ctx->vmm_phys_mapped; ++i) a.unmap(pv + (CUdeviceptr)(i * P), P);
        a.addr_free(pv, ctx->vmm_phys_bytes);
        ctx->arena = nullptr;
    }
    for (auto h : ctx->vmm_chunks) a.release(h);
    ctx->vmm_chunks.clear();
}

}  // namespace cloak
