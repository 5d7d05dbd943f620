// upload.cu -- keyed upload (Section 5, "Implementation Details": the
// permutation is computed and the physical pages allocated before any weight
// transfer, so that the bus never carries a structured layout).
//
// The host assembles every assigned arena page from the logical FP32 weights
// -- rows/columns permuted (intra-layer shuffling), converted (BF16 round to
// nearest even; E4M3 with a per-stored-row scale amax/448, satfinite), cut
// into tiles, each tile at its keyed slot -- and sends the pages to the
// device whole, in physical page order. The bytes of a physical page are a
// keyed set of tiles of keyed tensors, so neither the order of the
// transfers nor their destinations say which layer or tensor they carry.
// The result is the arena cloak_shuffle writes, bit for bit: BF16 rounds half
// to even as the device conversion does (a branch-free form below, checked
// against it), E4M3 calls the same host-callable CUDA conversion, and the
// scale is the same IEEE single-precision quotient.
//
// Two passes, each with sequential reads: (1) host threads convert the
// source rows, read whole and in order, into the tiles in logical order (a
// host buffer of the model's tile bytes); (2) they copy whole tiles into
// physical pages, one pinned staging buffer of `batch` pages while the copies
// of the previous one are in flight; runs of consecutive physical pages go in
// one copy. (Filling pages straight from the source reads each tile row from
// a different source row: a memory latency per 512 bytes, several times
// slower.)
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace cloak {

namespace {

struct HostTables {
    std::vector<uint32_t> tile_perm, page_alloc, group_perm;
    std::vector<int64_t> p2v;             // physical page -> virtual page (-1: unassigned)
    std::vector<int32_t> by_base;         // tensor indices ordered by first tile
};

inline int64_t perm_map_h(const uint32_t *gp, int32_t unit, int64_t i) {
    return (int64_t)gp[i / unit] * unit + i % unit;
}
// stored row / column -> logical (gp: all group permutations)
inline int64_t row_map_h(const uint32_t *gp, const TensorInfo &ti, int64_t r) {
    return ti.r_unit ? perm_map_h(gp + ti.r_goff, ti.r_unit, r) : r;
}
inline int64_t col_map_h(const uint32_t *gp, const TensorInfo &ti, int64_t c) {
    return ti.c_unit ? perm_map_h(gp + ti.c_goff, ti.c_unit, c) : c;
}

// FP32 -> BF16, round half to even, for a row of n values. For a non-NaN x
// the 16 discarded bits d of its pattern round the kept half k up exactly
// when d > 2^15, or d = 2^15 and k is odd: adding 2^15 - 1 + (k & 1) and
// truncating does that, carries into the exponent included (so the largest
// finite values round to infinity, as IEEE requires). The loop is branch
// free, so the compiler vectorises it; a row holding a NaN is redone with the
// CUDA conversion, which defines the NaN's encoding.
void bf16_row(const float *x, uint16_t *o, int n) {
    uint32_t nan = 0;
    for (int j = 0; j < n; ++j) {
        uint32_t b;
        std::memcpy(&b, x + j, 4);
        nan |= (uint32_t)((b & 0x7FFFFFFFu) > 0x7F800000u);
        o[j] = (uint16_t)((b + 0x7FFFu + ((b >> 16) & 1u)) >> 16);
    }
    if (nan)
        for (int j = 0; j < n; ++j) o[j] = __bfloat16_as_ushort(__float2bfloat16_rn(x[j]));
}

// scale of every stored row of every E4M3 tensor (the tensor's scale_off
// layout); the same quotient as the device shuffle
void row_scales(const cloak_ctx *ctx, const HostTables &h, const float *const *w, std::vector<float> &sc,
                int threads) {
    const int T = (int)ctx->info.size();
    std::vector<std::pair<int, int64_t>> jobs;  // (tensor, first row) in blocks of 64 rows
    for (int t = 0; t < T; ++t)
        for (int64_t r = 0; r < ctx->info[t].n; r += 64) jobs.push_back({t, r});
    std::atomic<size_t> next{0};
    auto work = [&] {
        for (size_t j; (j = next.fetch_add(1)) < jobs.size();) {
            const int t = jobs[j].first;
            const TensorInfo &ti = ctx->info[t];
            const uint32_t *gp = h.group_perm.data();
            const int64_t r1 = std::min<int64_t>(ti.n, jobs[j].second + 64);
            for (int64_t r = jobs[j].second; r < r1; ++r) {
                const int64_t lr = row_map_h(gp, ti, r);
                const float *row = w[t] + lr * ti.k;
                float m = 0.0f;
                for (int64_t c = 0; c < ti.k; ++c) m = std::fmax(m, std::fabs(row[c]));
                sc[ti.scale_off + r] = m > 0.0f ? m / 448.0f : 1.0f;
            }
        }
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < threads; ++i) pool.emplace_back(work);
    work();
    for (auto &th : pool) th.join();
}

// Pass 1: the tiles of row block nt of tensor t (tile_r stored rows, all
// kt tiles), converted into `tiles` in logical tile order. Source rows are
// read whole and in order, so the reads stream.
template <int ES>
void fill_row_block(const cloak_ctx *ctx, const HostTables &h, const float *const *w, const float *sc,
                    int t, int64_t nt, uint8_t *tiles, float *buf) {
    const TensorInfo &ti = ctx->info[t];
    const uint32_t *gp = h.group_perm.data();
    const uint32_t *cgp = gp + ti.c_goff;  // the column map's group
    const int TR = ctx->tile_r, TC = ctx->tile_c;
    const int64_t KP = ti.kt * (int64_t)TC;  // row length padded to whole tiles
    uint8_t *blk = tiles + ((int64_t)ctx->h_tensor_base[t] + nt * ti.kt) * ctx->tile_bytes;
    for (int i = 0; i < TR; ++i) {
        const int64_t r = nt * TR + i;
        if (r >= ti.n) {
            for (int64_t kt = 0; kt < ti.kt; ++kt)
                std::memset(blk + kt * ctx->tile_bytes + (size_t)i * TC * ES, 0, (size_t)TC * ES);
            continue;
        }
        const float *row = w[t] + row_map_h(gp, ti, r) * ti.k;
        // the stored row, zero-padded to whole tiles: read in place when its
        // columns keep their order (only a ragged last tile goes through buf)
        const float *src = buf;
        if (!ti.c_unit) {
            if (KP == ti.k) src = row;
            else std::memcpy(buf, row, (size_t)ti.k * 4);
        } else if (ti.c_unit == 1) {
            for (int64_t c = 0; c < ti.k; ++c) buf[c] = row[cgp[c]];
        } else {
            for (int64_t c = 0; c < ti.k; ++c) buf[c] = row[perm_map_h(cgp, ti.c_unit, c)];
        }
        if (src == buf)
            for (int64_t c = ti.k; c < KP; ++c) buf[c] = 0.0f;
        const float s = ES == 1 ? sc[ti.scale_off + r] : 1.0f;
        for (int64_t kt = 0; kt < ti.kt; ++kt) {
            uint8_t *out = blk + kt * ctx->tile_bytes + (size_t)i * TC * ES;
            const float *x = src + kt * TC;
            if constexpr (ES == 4) {
                std::memcpy(out, x, (size_t)TC * 4);
            } else if constexpr (ES == 2) {
                bf16_row(x, reinterpret_cast<uint16_t *>(out), TC);
            } else {
                // zero padding encodes as the device's 0 / 1: +0 either way
                for (int j = 0; j < TC; ++j)
                    out[j] = (uint8_t)__nv_cvt_float_to_fp8(x[j] / s, __NV_SATFINITE, __NV_E4M3);
            }
        }
    }
}

// Pass 2: physical page assembled from whole tiles (virtual page vp)
void fill_page(const cloak_ctx *ctx, const HostTables &h, const uint8_t *tiles, int64_t vp, uint8_t *dst) {
    for (int64_t j = 0; j < ctx->tpp; ++j) {
        const int64_t v = vp * ctx->tpp + j;
        uint8_t *tile = dst + j * ctx->tile_bytes;
        if (v >= ctx->G) std::memset(tile, 0, (size_t)ctx->tile_bytes);
        else std::memcpy(tile, tiles + (int64_t)h.tile_perm[v] * ctx->tile_bytes, (size_t)ctx->tile_bytes);
    }
}

// f(item, worker) over items 0..n-1 on up to `threads` workers (the caller
// is worker 0)
template <class F>
void parallel_for(int64_t n, int threads, F &&f) {
    std::atomic<int64_t> next{0};
    auto work = [&](int worker) {
        for (int64_t i; (i = next.fetch_add(1)) < n;) f(i, worker);
    };
    std::vector<std::thread> pool;
    const int nt = (int)std::min<int64_t>(threads, n);
    for (int k = 1; k < nt; ++k) pool.emplace_back(work, k);
    work(0);
    for (auto &th : pool) th.join();
}

}  // namespace

cloak_status upload_run(cloak_ctx *ctx, const float *const *w, int threads, cudaStream_t s) {
    const int T = (int)ctx->info.size();
    HostTables h;
    h.tile_perm.resize((size_t)ctx->G);
    h.page_alloc.resize((size_t)ctx->NPS);
    h.group_perm.resize((size_t)std::max<int64_t>(ctx->U, 1));
    CLOAK_CUDA(ctx, cudaStreamSynchronize(s));
    CLOAK_CUDA(ctx, cudaMemcpy(h.tile_perm.data(), ctx->d_tile_perm, ctx->G * 4, cudaMemcpyDeviceToHost));
    CLOAK_CUDA(ctx, cudaMemcpy(h.page_alloc.data(), ctx->d_page_alloc, ctx->NPS * 4, cudaMemcpyDeviceToHost));
    if (ctx->U)
        CLOAK_CUDA(ctx, cudaMemcpy(h.group_perm.data(), ctx->d_group_perm, ctx->U * 4, cudaMemcpyDeviceToHost));
    h.p2v.assign((size_t)ctx->NPS, -1);
    for (int64_t vp = 0; vp < ctx->NP; ++vp) {
        if (h.page_alloc[vp] >= (uint64_t)ctx->NPS) {
            ctx->last_err = "page map entry out of range";
            return CLOAK_E_STATE;
        }
        h.p2v[h.page_alloc[vp]] = vp;
    }
    for (int64_t v = 0; v < ctx->G; ++v)
        if (h.tile_perm[v] >= (uint64_t)ctx->G) {
            ctx->last_err = "tile permutation entry out of range";
            return CLOAK_E_STATE;
        }
    h.by_base.resize(T);
    for (int t = 0; t < T; ++t) h.by_base[t] = t;
    std::sort(h.by_base.begin(), h.by_base.end(),
              [&](int a, int b) { return ctx->h_tensor_base[a] < ctx->h_tensor_base[b]; });
    if (threads <= 0) threads = (int)std::min(16u, std::max(1u, std::thread::hardware_concurrency()));

    std::vector<float> sc;
    if (ctx->dtype == CLOAK_E4M3) {
        sc.assign((size_t)ctx->scales_total, 1.0f);
        row_scales(ctx, h, w, sc, threads);
    }
    // pass 1: every tile in logical order, in host memory of the arena's size
    // (not zeroed: pass 1 writes every byte, and its threads take the first
    // touch of the memory in parallel)
    std::unique_ptr<uint8_t[]> tiles(new (std::nothrow) uint8_t[(size_t)ctx->G * (size_t)ctx->tile_bytes]);
    if (!tiles) {
        ctx->last_err = "keyed upload: no host memory for the tile buffer";
        return CLOAK_E_NOMEM;
    }
    {
        std::vector<std::pair<int, int64_t>> blocks;  // (tensor, tile row)
        for (int t = 0; t < T; ++t)
            for (int64_t nt = 0; nt < ctx->info[t].nt; ++nt) blocks.push_back({t, nt});
        int64_t kmax = 0;
        for (int t = 0; t < T; ++t) kmax = std::max<int64_t>(kmax, ctx->info[t].kt * (int64_t)ctx->tile_c);
        std::vector<std::vector<float>> bufs(threads, std::vector<float>((size_t)kmax));
        parallel_for((int64_t)blocks.size(), threads, [&](int64_t i, int worker) {
            float *b = bufs[worker].data();
            const int t = blocks[i].first;
            if (ctx->esize == 4) fill_row_block<4>(ctx, h, w, sc.data(), t, blocks[i].second, tiles.get(), b);
            else if (ctx->esize == 2) fill_row_block<2>(ctx, h, w, sc.data(), t, blocks[i].second, tiles.get(), b);
            else fill_row_block<1>(ctx, h, w, sc.data(), t, blocks[i].second, tiles.get(), b);
        });
    }
    // assigned physical pages in ascending order
    std::vector<int64_t> pages;
    pages.reserve((size_t)ctx->NP);
    for (int64_t p = 0; p < ctx->NPS; ++p)
        if (h.p2v[p] >= 0) pages.push_back(p);

    const size_t P = (size_t)ctx->page_bytes;
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>((int64_t)pages.size(), (64ll << 20) / (int64_t)P));
    cudaEvent_t done[2] = {nullptr, nullptr};
    cloak_status rc = CLOAK_OK;
    auto cleanup = [&] {
        for (int i = 0; i < 2; ++i)
            if (done[i]) { cudaEventSynchronize(done[i]); cudaEventDestroy(done[i]); }
    };
    // pinned staging, kept by the context for later uploads
    if ((size_t)batch * P > ctx->upload_stage_bytes) {
        for (int i = 0; i < 2; ++i)
            if (ctx->h_upload_stage[i]) { cudaFreeHost(ctx->h_upload_stage[i]); ctx->h_upload_stage[i] = nullptr; }
        ctx->upload_stage_bytes = 0;
        for (int i = 0; i < 2 && !rc; ++i) {
            cudaError_t e = cudaHostAlloc((void **)&ctx->h_upload_stage[i], (size_t)batch * P, cudaHostAllocDefault);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "upload staging");
        }
        if (!rc) ctx->upload_stage_bytes = (size_t)batch * P;
    }
    uint8_t *stage[2] = {ctx->h_upload_stage[0], ctx->h_upload_stage[1]};
    for (int i = 0; i < 2 && !rc; ++i) {
        cudaError_t e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "upload event");
    }
    bool recorded[2] = {false, false};
    for (int64_t b0 = 0, it = 0; b0 < (int64_t)pages.size() && !rc; b0 += batch, ++it) {
        const int buf = (int)(it & 1);
        const int64_t nb = std::min<int64_t>(batch, (int64_t)pages.size() - b0);
        if (recorded[buf]) {
            cudaError_t e = cudaEventSynchronize(done[buf]);  // its previous copies have left
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "upload staging reuse"); break; }
        }
        uint8_t *st = stage[buf];
        parallel_for(nb, threads, [&](int64_t i, int) {
            fill_page(ctx, h, tiles.get(), h.p2v[pages[b0 + i]], st + (size_t)i * P);
        });
        // one copy per run of consecutive physical pages
        for (int64_t i = 0; i < nb && !rc;) {
            int64_t j = i + 1;
            while (j < nb && pages[b0 + j] == pages[b0 + j - 1] + 1) ++j;
            cudaError_t e = cudaMemcpyAsync(ctx->arena + (size_t)pages[b0 + i] * P, st + (size_t)i * P,
                                            (size_t)(j - i) * P, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "upload copy");
            i = j;
        }
        if (!rc) {
            cudaError_t e = cudaEventRecord(done[buf], s);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "upload event");
            recorded[buf] = true;
        }
    }
    if (!rc && ctx->dtype == CLOAK_E4M3) {
        cudaError_t e = cudaMemcpyAsync(ctx->d_scales, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "upload scales");
    }
    cleanup();
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "upload");
    }
    if (!rc) ctx->placed_any = true;
    return rc;
}

}  // namespace cloak
