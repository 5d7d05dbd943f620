// tune.cu -- autotuner of the tensor-core cloaked linear's launch shape.
//
// Three knobs change how a launch maps onto the machine but not what it
// computes: the activation chunk (the UMMA N of one launch: a batch of M
// tokens runs as ceil(M / chunk) launches), the depth of the TMA ring (how
// many gathered tiles are in flight per CTA; a shallower ring lets two CTAs
// share an SM) and the CTA count of the stream-K split (which decides how the
// tiles of a row are split into partial sums). For one (weight dtype, set of
// weight shapes, M bucket) the tuner times every candidate with
// CUDA events on the caller's stream and keeps the fastest. Entries depend
// neither on the cloaked/uncloaked flag nor on the output type, so all of
// them keep the same summation order; the serving step uses the tuned chunk and ring depth but
// the default CTA count, so that a token's result does not depend on its
// batch. Entries persist as JSON lines.
//
// The layer-stack kernel has one more depth to choose: how many of the next
// stage's weight tiles each CTA pulls into L2 while the current stage drains
// and the grid barrier is pending (beyond the tiles its smem ring takes).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace cloak {

static int m_bucket(int M) { return M <= 256 ? tc_npad(M) : ((M + 255) / 256) * 256; }

std::string tune_key(const cloak_ctx *ctx, int n, const int32_t *tensors, int M, int out_dtype) {
    (void)out_dtype;  // one shape for both output types: BF16 y stays the rounded FP32 y
    std::string k = ctx->dtype == CLOAK_E4M3 ? "e4m3" : "bf16";
    k += " m" + std::to_string(m_bucket(M));
    for (int p = 0; p < n; ++p) {
        const TensorInfo &ti = ctx->info[tensors[p]];
        k += " " + std::to_string(ti.n) + "x" + std::to_string(ti.k);
    }
    return k;
}

TuneCfg tune_lookup(const cloak_ctx *ctx, int n, const int32_t *tensors, int M, int out_dtype) {
    if (ctx->tune_force) return *ctx->tune_force;
    if (ctx->tune.empty()) return TuneCfg{};
    auto it = ctx->tune.find(tune_key(ctx, n, tensors, M, out_dtype));
    return it == ctx->tune.end() ? TuneCfg{} : it->second;
}

static int tmem_cols(int npad) {
    const int c = 2 * npad;
    return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

// the candidate launch shapes for a batch of M tokens
static std::vector<TuneCfg> candidates(const cloak_ctx *ctx, int n, const int32_t *tensors, int M) {
    const bool fp8 = ctx->dtype == CLOAK_E4M3;
    const int sm = ctx->sm_count;
    std::vector<int> chunks = {M <= 256 ? M : 256};
    if (M > 128) chunks.push_back(128);
    if (M > 64) chunks.push_back(64);
    int rows = 0;
    for (int p = 0; p < n; ++p) rows += ctx->info[tensors[p]].nt;
    std::vector<TuneCfg> out;
    for (int c : chunks) {
        const int np = tc_npad(std::min(c, M));
        const int maxs = tc_max_stages(fp8, np), sb = tc_stage_bytes(fp8, np);
        std::vector<int> depths = {maxs, maxs / 2, 4, 2};
        std::sort(depths.begin(), depths.end());
        depths.erase(std::unique(depths.begin(), depths.end()), depths.end());
        for (int st : depths) {
            if (st < 2 || st > maxs) continue;
            const int smem = st * sb + 2048;
            const int per_sm = std::min((228 * 1024) / (smem + 1024), 512 / tmem_cols(np));
            std::vector<int> grids = {sm, sm / 2};
            // several CTAs per SM: independent producers and MMA issuers hide the
            // per-tile issue latency of small (E4M3) tiles
            for (int k = 2; k <= 4; ++k)
                if (per_sm >= k) grids.push_back(k * sm);
            if (rows < sm * std::max(per_sm, 1)) grids.push_back(rows);
            std::sort(grids.begin(), grids.end());
            grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
            for (int g : grids) {
                TuneCfg t;
                t.chunk = c == M && M <= 256 ? 0 : c;  // 0: the whole batch in one launch
                t.stages = st;
                t.grid = g;
                out.push_back(t);
            }
        }
    }
    return out;
}

// mean time of `reps` runs of the batch with launch shape `c`, after one warm-up
static cloak_status time_cfg(cloak_ctx *ctx, const TuneCfg &c, int n, const int32_t *tensors,
                             const void *const *xs, void *const *ys, int M, int out_dtype,
                             cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps, float *us) {
    ctx->tune_force = &c;
    cloak_status rc = linear_batch_run(ctx, n, tensors, xs, ys, M, out_dtype, 0, s);
    if (!rc) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !rc; ++r) rc = linear_batch_run(ctx, n, tensors, xs, ys, M, out_dtype, 0, s);
        cudaEventRecord(e1, s);
    }
    ctx->tune_force = nullptr;
    if (rc) return rc;
    CLOAK_CUDA(ctx, cudaEventSynchronize(e1));
    float ms = 0.0f;
    CLOAK_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
    *us = 1e3f * ms / (float)reps;
    return CLOAK_OK;
}

cloak_status autotune_run(cloak_ctx *ctx, int n, const int32_t *tensors, const void *const *xs,
                          void *const *ys, int M, int out_dtype, cudaStream_t s, cloak_tune_result *res) {
    if (ctx->dtype == CLOAK_F32) return CLOAK_E_UNSUPPORTED;
    std::vector<TuneCfg> cand = candidates(ctx, n, tensors, M);
    cudaEvent_t e0, e1;
    CLOAK_CUDA(ctx, cudaEventCreate(&e0));
    CLOAK_CUDA(ctx, cudaEventCreate(&e1));
    cloak_status rc = CLOAK_OK;
    // the default shape first, then every candidate; the best three again, longer
    TuneCfg dflt;
    float t_default = 0.0f;
    rc = time_cfg(ctx, dflt, n, tensors, xs, ys, M, out_dtype, s, e0, e1, 10, &t_default);
    for (size_t i = 0; i < cand.size() && !rc; ++i)
        rc = time_cfg(ctx, cand[i], n, tensors, xs, ys, M, out_dtype, s, e0, e1, 5, &cand[i].us);
    if (!rc) {
        std::sort(cand.begin(), cand.end(), [](const TuneCfg &a, const TuneCfg &b) { return a.us < b.us; });
        const size_t top = std::min<size_t>(3, cand.size());
        for (size_t i = 0; i < top && !rc; ++i)
            rc = time_cfg(ctx, cand[i], n, tensors, xs, ys, M, out_dtype, s, e0, e1, 20, &cand[i].us);
        if (!rc) rc = time_cfg(ctx, dflt, n, tensors, xs, ys, M, out_dtype, s, e0, e1, 20, &t_default);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    std::sort(cand.begin(), cand.begin() + std::min<size_t>(3, cand.size()),
              [](const TuneCfg &a, const TuneCfg &b) { return a.us < b.us; });
    TuneCfg best = cand.empty() ? dflt : cand[0];
    if (cand.empty() || t_default <= best.us) {  // keep the default unless beaten
        best = dflt;
        best.us = t_default;
    }
    ctx->tune[tune_key(ctx, n, tensors, M, out_dtype)] = best;
    if (res) {
        res->chunk = best.chunk;
        res->stages = best.stages;
        res->grid = best.grid;
        res->us = best.us;
        res->default_us = t_default;
        res->candidates = (int32_t)cand.size();
        res->l2_prefetch = -1;
    }
    return CLOAK_OK;
}

static std::string stack_key(const cloak_stack_desc *d, int M) {
    return "stack L" + std::to_string(d->num_layers) + " d" + std::to_string(d->d_model) + " f" +
           std::to_string(d->d_ff) + " m" + std::to_string(m_bucket(M));
}

constexpr int STACK_L2PF_DEFAULT = 0;

int stack_l2_prefetch(const cloak_ctx *ctx, const cloak_stack_desc *d, int M) {
    if (ctx->stack_l2_pf_force >= 0) return ctx->stack_l2_pf_force;
    if (!ctx->tune.empty()) {
        auto it = ctx->tune.find(stack_key(d, M));
        if (it != ctx->tune.end() && it->second.l2pf >= 0) return it->second.l2pf;
    }
    return STACK_L2PF_DEFAULT;
}

cloak_status autotune_stack_run(cloak_ctx *ctx, const cloak_stack_desc *d, const float *h, int M,
                                cudaStream_t s, cloak_tune_result *res) {
    if (M < 1 || M > 64 || d->d_model <= 0) return CLOAK_E_INVAL;
    const size_t hb = (size_t)M * d->d_model * sizeof(float);
    float *hs = nullptr;
    CLOAK_CUDA(ctx, cudaMalloc(&hs, hb));  // the kernel updates h in place: run on a copy
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cloak_status rc = CLOAK_OK;
    const int cand[] = {0, 8, 16, 24, 32, 48};
    const int nc = (int)(sizeof cand / sizeof cand[0]);
    float us[sizeof cand / sizeof cand[0]] = {};
    auto run = [&](int reps) -> cloak_status {
        for (int r = 0; r < reps; ++r) {
            if (cudaMemcpyAsync(hs, h, hb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "stack tuner copy");
            cloak_status q = stack_decode_run(ctx, d, hs, M, 0, s);
            if (q) return q;
        }
        return CLOAK_OK;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = CLOAK_E_CUDA;
    for (int pass = 0; pass < 2 && !rc; ++pass) {  // two passes, keep each candidate's best
        for (int i = 0; i < nc && !rc; ++i) {
            ctx->stack_l2_pf_force = cand[i];
            rc = run(1);
            if (!rc) {
                cudaEventRecord(e0, s);
                rc = run(5);
                cudaEventRecord(e1, s);
            }
            if (!rc && cudaEventSynchronize(e1) == cudaSuccess) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                const float t = 1e3f * ms / 5.0f;
                us[i] = pass == 0 ? t : std::min(us[i], t);
            }
        }
    }
    ctx->stack_l2_pf_force = -1;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(hs);
    if (rc) return rc;
    int best = 0, dflt = 0;
    for (int i = 0; i < nc; ++i) {
        if (us[i] < us[best]) best = i;
        if (cand[i] == STACK_L2PF_DEFAULT) dflt = i;
    }
    TuneCfg c;
    c.l2pf = cand[best];
    c.us = us[best];
    ctx->tune[stack_key(d, M)] = c;
    if (res) {
        res->chunk = 0;
        res->stages = 0;
        res->grid = ctx->sm_count;
        res->us = us[best];
        res->default_us = us[dflt];
        res->candidates = nc;
        res->l2_prefetch = cand[best];
    }
    return CLOAK_OK;
}

cloak_status tune_save(const cloak_ctx *ctx, const char *path) {
    FILE *f = std::fopen(path, "w");
    if (!f) return CLOAK_E_INVAL;
    std::vector<std::string> keys;
    for (const auto &kv : ctx->tune) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end());
    for (const auto &k : keys) {
        const TuneCfg &c = ctx->tune.at(k);
        std::fprintf(f,
                     "{\"chunk\": %d, \"stages\": %d, \"grid\": %d, \"l2pf\": %d, \"us\": %.3f, "
                     "\"key\": \"%s\"}\n",
                     c.chunk, c.stages, c.grid, c.l2pf, c.us, k.c_str());
    }
    return std::fclose(f) == 0 ? CLOAK_OK : CLOAK_E_INVAL;
}

cloak_status tune_load(cloak_ctx *ctx, const char *path, int32_t *entries) {
    FILE *f = std::fopen(path, "r");
    if (!f) return CLOAK_E_INVAL;
    char line[1024];
    int count = 0;
    cloak_status rc = CLOAK_OK;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] != '{') continue;
        TuneCfg c;
        char key[900];
        if (std::sscanf(line,
                        "{\"chunk\": %d, \"stages\": %d, \"grid\": %d, \"l2pf\": %d, \"us\": %f, "
                        "\"key\": \"%899[^\"]\"}",
                        &c.chunk, &c.stages, &c.grid, &c.l2pf, &c.us, key) != 6 ||
            c.chunk < 0 || c.chunk > 65536 || c.stages < 0 || c.stages > 16 || c.grid < 0 ||
            c.grid > 65535 || c.l2pf < -1 || c.l2pf > 1024) {
            rc = CLOAK_E_INVAL;
            break;
        }
        ctx->tune[key] = c;
        ++count;
    }
    std::fclose(f);
    if (entries) *entries = count;
    return rc;
}

}  // namespace cloak
