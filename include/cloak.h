/*
 * cloak.h -- C ABI of libcloak: a cloaked linear layer for one GB300 (sm_103a).
 *
 * CloakLM (arxiv 2606.18400) hides where model weights sit in GPU memory: the
 * authorised execution keeps a valid logical view of the weights while raw
 * memory shows fragmented, shuffled state (Abstract; Section 4.2). This
 * library keeps every weight matrix as fixed-size tiles placed in HBM in a
 * keyed order and computes y = x W^T by gathering the tiles through a table:
 *
 *   inter-layer shuffling   layers take a keyed order in the arena
 *                           (Section 4.2, "Inter-layer randomization");
 *   intra-layer shuffling   a producer's output rows and its consumer's input
 *                           columns are permuted by the same keyed permutation,
 *                           so the network computes the same function (named in
 *                           the Abstract and the Contributions);
 *   page remapping          tiles sit at keyed slots of keyed physical pages,
 *                           re-randomised by re-keying (Section 4.2, "Physical
 *                           page remapping"; Table 1b; Figure 7).
 *
 * Tables are drawn from a caller-supplied 64-bit key before any weight is
 * placed (Section 5, "Implementation Details"): SplitMix64 streams, Lemire's
 * unbiased bounded draw and Fisher-Yates shuffles, redrawn until no two
 * physically adjacent slots hold logically consecutive tiles.
 *
 * Conventions
 *   - Every pointer named *_dev is CUDA device memory owned by the caller;
 *     *_host is host memory owned by the caller (pinned memory makes the
 *     copies asynchronous). The context owns the arena, its uncloaked twin,
 *     the tables, the FP8 scales and its workspaces.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls enqueue work on it and return; the exceptions say so.
 *   - Every call returns a cloak_status; no exception crosses the ABI. A CUDA
 *     error is reported as CLOAK_E_CUDA and its message is kept for
 *     cloak_last_error().
 *   - A context is not thread-safe; use one context per host thread.
 *   - Weight matrices are [n, k] (out, in), row-major; y = x W^T with x [M, k]
 *     and y [M, n], row-major.
 */
#ifndef CLOAK_H
#define CLOAK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CLOAK_API __attribute__((visibility("default")))
#else
#define CLOAK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t cloak_status;
enum {
    CLOAK_OK = 0,
    CLOAK_E_INVAL = -1,        /* bad argument or descriptor                    */
    CLOAK_E_NOMEM = -2,        /* device or host allocation failed              */
    CLOAK_E_CUDA = -3,         /* a CUDA call failed (see cloak_last_error)     */
    CLOAK_E_TIMEOUT = -4,      /* a bounded device wait gave up                 */
    CLOAK_E_STATE = -5,        /* call out of order (e.g. linear before keygen) */
    CLOAK_E_UNSUPPORTED = -6,  /* shape/dtype not supported by any kernel       */
    CLOAK_E_DRAWS = -7         /* layout invariant not met within the draw cap  */
};

/* weight storage types (all tensors of a model share one) */
enum { CLOAK_F32 = 0, CLOAK_BF16 = 1, CLOAK_E4M3 = 2 };

/* One weight matrix. perm_group >= 0 links it to an intra-layer permutation:
 * perm_axis 0 permutes its rows (a producer), 1 its columns (a consumer).
 * perm_group2 >= 0 permutes the other axis (1 - perm_axis) as well: e.g. one
 * residual-dimension group shared by the columns of every matrix that reads
 * the residual stream and the rows of every matrix that writes it. Each
 * permuted dimension must equal its group's n_units * unit. */
typedef struct {
    int32_t n, k;            /* rows (out features), columns (in features)  */
    int32_t layer;           /* layer index, 0..L-1                          */
    int32_t kind;            /* free tag (q, k, v, o, gate, up, down, ...)   */
    int32_t perm_group;      /* -1: not permuted                             */
    int32_t perm_axis;       /* 0 rows, 1 columns                            */
    int32_t perm_group2;     /* group of the other axis, -1: none            */
} cloak_tensor_desc;

/* A keyed permutation of n_units blocks of `unit` rows/columns. A derived
 * group (parent >= 0, declared after its parent) has parent.n_units * ratio
 * units: block a*ratio+b holds parent_perm[a]*ratio + inner_a[b], so grouped
 * query heads move with their KV head. */
typedef struct {
    int32_t n_units, unit, parent, ratio;
} cloak_group_desc;

enum {
    CLOAK_MODEL_TWIN = 1,  /* also keep an uncloaked tile-major copy          */
    CLOAK_MODEL_VMM = 2,   /* Section 4.2 physical page remapping through CUDA
                              virtual memory management: every arena page is
                              its own physical chunk (cuMemCreate), mapped at
                              its physical position in the arena and, in a
                              second address range (the virtual view), at
                              virtual page vp -> chunk page_alloc[vp]. The two
                              views alias: no extra memory. page_bytes must be
                              a multiple of the VMM allocation granularity
                              (2 MiB), else cloak_create fails with
                              CLOAK_E_UNSUPPORTED. See CLOAK_LINEAR_VMM.     */
    CLOAK_MODEL_TILE_REKEY = 4  /* the tile permutation is redrawn at every
                              epoch too (its streams seeded with the epoch;
                              epoch 0 draws what a model without the flag
                              draws): cloak_rekey then moves every tile
                              (32 KiB BF16, 16 KiB E4M3) to its slot under the
                              new tables, so tiles also change pages and
                              neighbours: through a device buffer of the
                              arena's size, allocated by the first such
                              re-key and kept by the context until
                              cloak_destroy (in place through the staging
                              pages if it cannot be allocated, or if the
                              environment sets CLOAK_TILE_REKEY_IN_PLACE=1);
                              the arena keeps its address. Synchronous
                              re-keys only:
                              cloak_rekey_begin returns CLOAK_E_UNSUPPORTED. */
};

typedef struct {
    int32_t num_tensors, num_groups;
    const cloak_tensor_desc *tensors;
    const cloak_group_desc *groups;
    int32_t dtype;           /* CLOAK_F32 / CLOAK_BF16 / CLOAK_E4M3           */
    int32_t tile_r, tile_c;  /* tile shape in elements (128x128 for the
                                tensor-core kernels, 64x64 for FP32)          */
    int32_t spare_pages;     /* extra physical pages left free in the arena   */
    int32_t tile_scope;      /* 0: one tile permutation over the model;
                                1: one per tensor (layers still shuffled)     */
    int32_t flags;           /* CLOAK_MODEL_TWIN | _VMM | _TILE_REKEY         */
    int64_t page_bytes;      /* page size, a multiple of the tile bytes       */
} cloak_model_desc;

typedef struct cloak_ctx cloak_ctx;

/* Create a context on `device`: validates the descriptor, allocates the
 * zeroed arena of (ceil(tiles / tiles_per_page) + spare_pages) pages, the twin
 * if requested, tables and workspaces. Synchronous. Paper: Section 4.2
 * ("Physical page remapping", Table 1b) places weights on non-contiguous
 * physical pages of a fixed size; the arena is that page pool, allocated
 * whole before anything is placed (Section 5, "Implementation Details"). The
 * context owns every buffer it allocates; errors: CLOAK_E_INVAL (descriptor),
 * CLOAK_E_NOMEM, CLOAK_E_CUDA. */
CLOAK_API cloak_status cloak_create(const cloak_model_desc *desc, int32_t device, cloak_ctx **out);

/* Release everything the context owns. Synchronises the device first. */
CLOAK_API cloak_status cloak_destroy(cloak_ctx *ctx);

/* Geometry: out[0..7] = layers, tiles, tiles per page, pages, pages incl.
 * spare, permutation units, tile bytes, element bytes. */
CLOAK_API cloak_status cloak_geometry(const cloak_ctx *ctx, int64_t out[8]);

/* Draw every table for (key, epoch) on the device (Section 5: the random
 * permutation is computed before any weight is placed): layer order, group
 * permutations, tile permutation, page map, gather table. Blocks until done
 * (the redraw loop reads a flag back). Any placed weights become stale:
 * shuffle again after a keygen (use cloak_rekey to move placed weights). */
CLOAK_API cloak_status cloak_keygen(cloak_ctx *ctx, uint64_t key, uint32_t epoch, void *stream);

enum {
    CLOAK_TAB_LAYER_PERM = 0,  /* [L]   arena position -> layer               */
    CLOAK_TAB_GROUP_PERM = 1,  /* [U]   per group: stored unit -> logical unit */
    CLOAK_TAB_TENSOR_BASE = 2, /* [T]   first logical tile of each tensor      */
    CLOAK_TAB_TILE_PERM = 3,   /* [G]   virtual position -> logical tile       */
    CLOAK_TAB_PAGE_ALLOC = 4,  /* [NP+S] virtual page -> physical page, then
                                          the free physical pages            */
    CLOAK_TAB_TILE_SLOT = 5    /* [G]   logical tile -> arena slot             */
};
/* Copy one table to host memory (count entries). Synchronous. For tests and
 * audits; the tables are secret in deployment. */
CLOAK_API cloak_status cloak_export_table(const cloak_ctx *ctx, int32_t which, uint32_t *host_out,
                                size_t count);

/* Place tensor `tensor` from its logical FP32 weights [n, k] (device):
 * permute rows or columns, convert to the storage type (BF16: round to
 * nearest even; E4M3: per-stored-row scale amax/448 then round to nearest
 * even, saturating), cut into tiles, write each tile to its keyed slot, and to
 * the twin if present. Ragged tile edges are written as zeros. Paper: the
 * keyed placement of Section 5 ("Implementation Details": permutation before
 * any weight is placed) combining inter- and intra-layer weight shuffling
 * (Abstract; Contributions) with the page placement of Section 4.2. The caller
 * keeps ownership of logical_dev (read only, asynchronous on `stream`: keep it
 * alive until the stream reaches this point). Errors: CLOAK_E_INVAL (tensor
 * index, null pointer), CLOAK_E_STATE before a keygen or during a concurrent
 * re-key. */
CLOAK_API cloak_status cloak_shuffle(cloak_ctx *ctx, int32_t tensor, const float *logical_dev, void *stream);

/* Inverse of cloak_shuffle: read the tiles back and write the logical
 * [n, k] matrix in the storage type (FP32 values, BF16 or E4M3 bit patterns)
 * with the permutation undone. from_twin = 1 reads the uncloaked twin. Paper:
 * the authorised execution keeps a valid logical view of the weights
 * (Abstract; Section 4.2, pointers and access semantics unchanged); this is
 * that view materialised. logical_dev is caller-owned, [n, k] elements of the
 * storage type, row-major. Errors: CLOAK_E_INVAL, CLOAK_E_STATE (not keyed,
 * no twin for from_twin = 1). */
CLOAK_API cloak_status cloak_unshuffle(const cloak_ctx *ctx, int32_t tensor, void *logical_dev,
                             int32_t from_twin, void *stream);

/* Keyed upload (Section 5, "Implementation Details": the permutation is
 * drawn and the physical pages allocated before any weight is transferred,
 * so the bus never carries a structured layout). w_host[t] is tensor t's
 * logical FP32 matrix [n, k], row-major, in host memory (pageable or pinned),
 * for every tensor of the model. The host assembles each assigned arena page
 * (permuted, converted, tiled and placed exactly as cloak_shuffle does) and
 * copies it to the device whole; pages go in ascending physical order, runs
 * of consecutive pages in one copy, through two pinned staging buffers of at
 * most 64 MiB (kept by the context). The call also holds host memory of the
 * model's tile bytes (the tiles in logical order, assembled first). E4M3 scales are computed on the host and uploaded after the
 * pages. The arena afterwards equals cloak_shuffle of every tensor, bit for
 * bit. threads: host threads assembling pages (0: the hardware's, at most
 * 16). Synchronous (returns when the copies have landed). Errors:
 * CLOAK_E_STATE before a keygen, during a concurrent re-key, or on a context
 * with a twin (the twin is in logical order: filling it would put the
 * logical layout on the bus). */
CLOAK_API cloak_status cloak_upload(cloak_ctx *ctx, const float *const *w_host, int32_t threads,
                                    void *stream);

/* Device pointer to tensor `tensor`'s FP32 scales [n] in stored-row order
 * (E4M3 models only; owned by the context). */
CLOAK_API cloak_status cloak_scales(const cloak_ctx *ctx, int32_t tensor, const float **dev_out);

/* Device pointer to the arena and its size in bytes (for audits and tests;
 * owned by the context). which = 0 arena, 1 twin, 2 the virtual view of a
 * CLOAK_MODEL_VMM context (NP pages; valid once keyed, and its pointer does
 * not change across re-keys; the pages behind it do). */
CLOAK_API cloak_status cloak_arena(const cloak_ctx *ctx, int32_t which, void **dev_out, int64_t *bytes);

enum {
    CLOAK_LINEAR_UNCLOAKED = 1,  /* run the same kernel on the twin, tiles
                                    addressed arithmetically (tile-major)    */
    CLOAK_LINEAR_RELU = 2,       /* y = max(y, 0)                             */
    CLOAK_LINEAR_VMM = 8,        /* CLOAK_MODEL_VMM contexts: run the same
                                    kernel on the virtual view, each tile
                                    found at its virtual position (the tile
                                    permutation); the MMU supplies the page
                                    map. Same tiles, same summation order:
                                    bit for bit the result of the arena
                                    read. Not with CLOAK_LINEAR_UNCLOAKED, and
                                    CLOAK_E_STATE while a concurrent re-key
                                    is in progress.                          */
    CLOAK_LINEAR_CHAINED = 16    /* cloak_linear / cloak_linear_batch on a
                                    BF16 or E4M3 model: a programmatic
                                    dependent launch. Its CTAs may start
                                    while the kernel enqueued before it on
                                    the stream is still running and fetch
                                    weight tiles at once; they read x, the
                                    scratch and y only after that kernel has
                                    completed (griddepcontrol.wait). The
                                    caller asserts that the kernel before it
                                    on the stream writes none of this
                                    context's weights, tables or scales
                                    (another linear call, or the caller's
                                    own kernels producing x, qualify;
                                    shuffle, upload, re-key and a concurrent
                                    re-key's table update do not). Results
                                    are bit for bit those without the flag.
                                    E4M3 decode batches then quantise x in a
                                    separate kernel, chained the same way.
                                    Prefill-shaped batches (whole-tile GEMM)
                                    and FP32 models ignore it.               */
};
enum { CLOAK_OUT_F32 = 0, CLOAK_OUT_BF16 = 1 };

/* y[M, n] = x[M, k] W^T for tensor `tensor`, reading W's tiles through the
 * gather table. W is the stored (permuted) matrix, so a producer's output
 * comes out permuted and its consumer takes it as is. x is FP32 for FP32
 * models and BF16 otherwise (E4M3 models quantise x per row inside the call:
 * scale amax/448, round to nearest even). Accumulation is FP32; with the same
 * M, the cloaked and uncloaked kernels sum in the same order and agree bit for
 * bit. x and y must not alias; x must be 16-byte aligned. 1 <= M <= 65536.
 * Paper: the authorised execution's valid logical view (Abstract; Section 4.2:
 * the engine computes on the weights as if they were contiguous, with no
 * measurable overhead, Figure 5). x [M, k] and y [M, n] are row-major,
 * caller-owned device buffers; asynchronous on `stream`; workspaces are
 * context-owned and may grow (cudaMalloc). Errors: CLOAK_E_INVAL (arguments),
 * CLOAK_E_STATE (not keyed; uncloaked without a twin), CLOAK_E_CUDA. */
CLOAK_API cloak_status cloak_linear(cloak_ctx *ctx, int32_t tensor, const void *x_dev, void *y_dev,
                          int32_t M, int32_t out_dtype, int32_t flags, void *stream);

/* Up to 8 independent cloaked linears in one launch (e.g. the seven
 * projections of a decoder layer): y_i = x_i W_{t_i}^T for i < n, all with M
 * rows. Their tiles are concatenated and split evenly over the SMs, so the
 * launch and pipeline fill are paid once. The summation order depends on the
 * whole batch; cloaked and uncloaked batches agree bit for bit. Same rules as
 * cloak_linear for each x_i / y_i. */
CLOAK_API cloak_status cloak_linear_batch(cloak_ctx *ctx, int32_t n, const int32_t *tensors,
                                          const void *const *x_dev, void *const *y_dev, int32_t M,
                                          int32_t out_dtype, int32_t flags, void *stream);

/* cloak_linear from host buffers: copies x in, computes, copies y out and
 * waits for the stream (synchronous). Uses a context-owned staging buffer. */
CLOAK_API cloak_status cloak_linear_host(cloak_ctx *ctx, int32_t tensor, const void *x_host, void *y_host,
                               int32_t M, int32_t out_dtype, int32_t flags, void *stream);

/* cloak_linear_batch from host buffers: the n inputs are copied in, the
 * grouped launch runs, the n outputs are copied back and the stream is waited
 * for (synchronous). Inputs that lie back to back in host memory (x_host[i+1]
 * == x_host[i] + its size) move in one copy, and so do such outputs, so a
 * caller that packs a step's vectors pays one copy each way. Pinned host
 * memory gives asynchronous DMA; pageable memory works but is staged by the
 * driver. Staging on the device is context-owned (grown with cudaMalloc).
 * Same rules as cloak_linear_batch otherwise. Paper: the authorised view of
 * Section 4.2 driven from the host, the way a serving engine hands the layer
 * one step's activations. */
CLOAK_API cloak_status cloak_linear_batch_host(cloak_ctx *ctx, int32_t n, const int32_t *tensors,
                                               const void *const *x_host, void *const *y_host, int32_t M,
                                               int32_t out_dtype, int32_t flags, void *stream);

/* cloak_linear for callers that cannot allocate device memory while they
 * run: code inside CUDA stream capture (an allocation there breaks the
 * capture), serving loops under a memory pool that owns every byte, or
 * real-time paths where cudaMalloc's synchronisation is not allowed.
 * cloak_linear itself may grow its context-owned scratch with cudaMalloc; this
 * call never calls cudaMalloc, cudaFree or any allocating routine. Its scratch
 * (split-K partial sums and tile-row counters) is one fixed 20 MiB + 16 KiB
 * device array inside the library, held on every GPU that loads it until the
 * process exits. The paper has no counterpart: this is a deployment aid.
 *   Limits: BF16 models only, devices of at most 160 SMs (else
 *   CLOAK_E_UNSUPPORTED); 1 <= M <= 32 and at most 4096 tile rows per tensor
 *   (else CLOAK_E_INVAL); a launch shape stored for the tensor (tuner or
 *   cloak_tune_load) of more than 4 CTAs per SM of a 160-SM device
 *   (CLOAK_E_UNSUPPORTED). Messages in cloak_last_error.
 *   The first call on a device looks up the array's device address; make that
 *   first call before any stream capture. A failed look-up is reported and
 *   retried by the next call. Every call shares the one array and clears the
 *   counters it uses on `stream` (an asynchronous memset); calls that overlap
 *   on the GPU (other streams, other contexts) race on it and must be ordered
 *   by the caller.
 * It launches the kernel cloak_linear launches, in the launch shape cloak_linear
 * takes for the same tensor and M (the stored tuned shape, else the default),
 * so results equal cloak_linear's for the same arguments, bit for bit. */
CLOAK_API cloak_status cloak_linear_noalloc(cloak_ctx *ctx, int32_t tensor, const void *x_dev,
                                            void *y_dev, int32_t M, int32_t out_dtype,
                                            int32_t flags, void *stream);

/* A LLaMA-style decoder stack whose seven linears per layer are cloaked
 * tensors of this context (BF16, head_dim 128). */
typedef struct {
    int32_t num_layers;
    const int32_t *layer_tensors;  /* [num_layers * 7]: q, k, v, o, gate, up, down */
    int32_t d_model, n_heads, n_kv_heads, head_dim, d_ff;
    float rms_eps;
} cloak_stack_desc;

/* One decode step of the whole stack in a single persistent launch (all
 * layers' cloaked linears plus the glue, grid barriers between dependent
 * stages; CUDA-graph capturable after a first call has sized the workspace).
 * h_dev is the FP32 residual stream [M, d_model], updated in place. Per
 * layer, with r = 1/sqrt(mean(h^2) + eps) per token and unit norm gains:
 * q,k,v = (h W^T) r; the attention of a single token is its own value, each
 * query head taking its group's v; h += a Wo^T; g,u = (h W^T) r';
 * h += (silu(g) * u) Wd^T. Intra-layer permutations cancel inside the layer
 * (the stored head order is consistent across q, k, v, o and the MLP order
 * across gate, up, down). 1 <= M <= 64. flags: CLOAK_LINEAR_UNCLOAKED runs on
 * the twin. Device waits are bounded; a timeout sets cloak_device_status. */
CLOAK_API cloak_status cloak_stack_decode(cloak_ctx *ctx, const cloak_stack_desc *desc, float *h_dev,
                                          int32_t M, int32_t flags, void *stream);

/* A served model: the decoder stack, a cloaked lm_head tensor [vocab,
 * d_model], the embedding [vocab, d_model] -- either a cloaked tensor of the
 * context (embed_tensor >= 0: its rows are looked up through the gather
 * table, so the table is as hidden as the weights) or a plain BF16 table
 * (embed_tensor = -1; device, caller's) -- and the paged KV cache (device,
 * caller's): per layer, num_blocks blocks of 16 tokens x n_kv_heads x 128,
 * BF16, for keys and for values. */
typedef struct {
    cloak_stack_desc stack;
    int32_t lm_head;          /* tensor index of the output projection        */
    int32_t vocab;
    const void *embedding;    /* BF16 [vocab, d_model]; NULL with embed_tensor  */
    void *k_cache, *v_cache;  /* BF16 [layers][num_blocks][16][n_kv][128]       */
    int32_t num_blocks;
    int32_t max_blocks;       /* block-table row length (blocks per request)    */
    float rope_theta;
    int32_t embed_tensor;     /* cloaked embedding tensor [vocab, d_model], not
                                 permuted (a BF16 model), or -1                  */
} cloak_serve_desc;

/* One step's batch: num_tokens tokens of any requests (prefill chunks and
 * decode tokens mixed). All arrays are device int32. Token m of request
 * req_slots[m] sits at position positions[m] and attends to that request's
 * positions 0..positions[m] through block_tables[req][pos / 16] (a request's
 * earlier positions must be in the cache or in this batch). sample_rows lists
 * the tokens whose next token is sampled (greedy) into out_tokens;
 * out_logits (FP32 [num_sample, vocab], may be NULL) receives their logits.
 * A token id outside [0, vocab) embeds as a zero row. */
/* cloak_serve_batch.flags, besides CLOAK_LINEAR_UNCLOAKED: the first
 * num_single tokens are the batch's decode tokens and the others prompt
 * tokens. The linears then run the decode rows through the split-K decode
 * kernel and the prompt rows through the whole-tile prefill kernel; either
 * kernel's summation order depends on the weights only, so a token's result
 * still depends only on its own request (and on being a decode or a prompt
 * token). Without the flag every row takes the decode kernel. */
enum { CLOAK_SERVE_DECODE_FIRST = 4 };

typedef struct {
    int32_t num_tokens, num_sample, flags;  /* CLOAK_LINEAR_UNCLOAKED, CLOAK_SERVE_DECODE_FIRST */
    const int32_t *token_ids, *positions, *req_slots, *block_tables, *sample_rows;
    int32_t *out_tokens;
    float *out_logits;
    /* Optional attention work split (device int32; NULL qtiles: one block
     * per token). qtiles[num_qtiles][3] = (first token, count <= 64, 0): runs
     * of consecutive tokens of one request at consecutive positions, whose
     * queries share staged K/V tiles; single_rows[num_single]: the other
     * tokens, one block each. Together they must cover every token once. A
     * token's result depends only on which of the two lists holds it; the
     * qtiles order is the order their blocks start (latest positions first
     * balances the work). */
    int32_t num_qtiles, num_single;
    const int32_t *qtiles, *single_rows;
} cloak_serve_batch;

/* One forward step of the served model over a mixed batch: per layer
 * RMSNorm, cloaked q/k/v, RoPE (theta, rotate-half pairs), KV-cache write,
 * causal paged attention (GQA), cloaked o + residual, RMSNorm, cloaked
 * gate/up, SiLU-gated product, cloaked down + residual; then RMSNorm, the
 * cloaked lm_head at the sampled rows and greedy argmax. Enqueued on `stream`;
 * the context-owned workspace grows with the batch. A token's results depend
 * only on its own request, so a request computes the same alone or batched.
 * The step's first kernel is an ordinary launch (it follows whatever the
 * caller enqueued, e.g. a concurrent re-key's table update); the later ones
 * are programmatic dependent launches of one another, each waiting for its
 * predecessor before it reads that kernel's outputs. */
CLOAK_API cloak_status cloak_serve_step(cloak_ctx *ctx, const cloak_serve_desc *desc,
                                        const cloak_serve_batch *batch, void *stream);

/* Launch-shape autotuner of the tensor-core linear (BF16 / E4M3 models).
 * Times, with CUDA events on `stream`, the candidate launch shapes of
 * cloak_linear_batch(ctx, n, tensors, x_dev, y_dev, M, out_dtype, 0): the
 * activation chunk (UMMA N of one launch), the depth of the TMA gather ring
 * and the CTA count of the stream-K split; keeps the fastest (or the
 * default, if none beats it) for (weight dtype, the n weight shapes, the M
 * bucket), and reports it in `out`. Later linear calls with that key use it,
 * cloaked or uncloaked and for either output type alike (the same summation
 * order); the serving step keeps the default CTA count. Runs the real computation: the y
 * buffers are overwritten. Blocks until the measurements are done.
 * CLOAK_E_UNSUPPORTED for FP32 models. */
typedef struct {
    int32_t chunk;        /* tokens per launch; 0: the whole batch (up to 256)  */
    int32_t stages;       /* TMA ring depth                                     */
    int32_t grid;         /* CTAs of the stream-K split; 0: one per SM          */
    float us;             /* time of the chosen shape, microseconds             */
    float default_us;     /* time of the default shape                          */
    int32_t candidates;   /* shapes measured                                    */
    int32_t l2_prefetch;  /* layer stack: next-stage tiles per CTA pulled into
                             L2 during a stage's tail (-1 for linears)         */
} cloak_tune_result;
CLOAK_API cloak_status cloak_autotune(cloak_ctx *ctx, int32_t n, const int32_t *tensors,
                                      const void *const *x_dev, void *const *y_dev, int32_t M,
                                      int32_t out_dtype, void *stream, cloak_tune_result *out);
/* Tune the layer-stack launch (cloak_stack_decode) for `desc` and M: times
 * its L2 prefetch depths (0 to 48 tiles per CTA) on a copy of h_dev (h_dev is
 * not changed) and keeps the fastest for (layers, d_model, d_ff, M bucket).
 * Key: "stack L<layers> d<d_model> f<d_ff> m<bucket>". */
CLOAK_API cloak_status cloak_autotune_stack(cloak_ctx *ctx, const cloak_stack_desc *desc,
                                            const float *h_dev, int32_t M, void *stream,
                                            cloak_tune_result *out);
/* Write the tuned shapes as JSON lines ({"chunk", "stages", "grid", "l2pf",
 * "us", "key"}) / read such a file, adding its entries (count in *entries). A key
 * reads "<bf16|e4m3> m<bucket> <N>x<K> ..." (the bucket is the UMMA N for
 * M <= 256: 16, 32, 64, 128 or 256; above, M rounded up to 256; then each
 * weight's shape in call order).
 * CLOAK_E_INVAL if the file cannot be opened or a line does not parse. */
CLOAK_API cloak_status cloak_tune_save(const cloak_ctx *ctx, const char *path);
CLOAK_API cloak_status cloak_tune_load(cloak_ctx *ctx, const char *path, int32_t *entries);
/* Forget every tuned shape (back to the defaults). */
CLOAK_API cloak_status cloak_tune_clear(cloak_ctx *ctx);

/* Re-key (periodic re-randomisation, Section 4.2 and Figure 7): draw the page
 * map of (key, new_epoch) and move every placed page to its new physical page
 * in place, through a small staging pool, so the arena ends bit-identical to
 * keygen(key, new_epoch) + shuffle. The key must be the one of the last
 * keygen. Blocks until the move plan is built, then enqueues the moves and
 * returns. Linear calls must not run concurrently with the moves: order them
 * on the same stream or with events. */
/* A cloaked MoE FFN block (the paper's MoE model, Qwen3-30B-A3B shape:
 * Section 5). Every expert matrix is a tensor of the context; the router
 * [n_experts, d_model] has its rows in the order of a keyed expert-order
 * permutation group (unit 1, n_units = n_experts): its stored output e'
 * scores logical expert perm[e'] (expert_group = -1: rows not permuted). */
typedef struct {
    int32_t n_experts, top_k;   /* 1 <= top_k <= min(n_experts, 16), n_experts <= 1024 */
    int32_t d_model, d_ff;      /* multiples of 128                                    */
    int32_t router;             /* tensor [n_experts, d_model]                         */
    int32_t expert_group;       /* the router rows' group, or -1                       */
    const int32_t *expert_tensors;  /* host [n_experts][3]: gate [d_ff, d_model], up
                                   [d_ff, d_model], down [d_model, d_ff] of logical
                                   expert e (gate/up rows and down columns in one
                                   hidden order, e.g. one permutation group)        */
} cloak_moe_desc;

/* y[M, d_model] (FP32) = the MoE FFN of x[M, d_model] (BF16, 16-byte
 * aligned), 1 <= M <= 64: router logits z = x Wr^T (cloaked linear, FP32);
 * per token the top_k experts by logit (equal logits: the lower logical
 * expert), weights = their softmax probabilities renormalised to sum to 1
 * (FP32); y = sum_j w_j Wdown_j bf16(silu(Wgate_j x) * (Wup_j x)), FP32
 * accumulation in a fixed order (deterministic). Expert tiles are gathered
 * through the gather table like every weight (flags: CLOAK_LINEAR_UNCLOAKED
 * reads the twin, CLOAK_LINEAR_VMM the virtual view). Optional device
 * outputs: experts_out [M, top_k] the selected logical experts, logits_out
 * [M, n_experts] the router logits in logical expert order. BF16 models with
 * 128x128 tiles only. The first call for a descriptor (and the first after a
 * keygen) uploads the expert table and synchronises the stream; later calls
 * are asynchronous and capturable. */
CLOAK_API cloak_status cloak_moe_ffn(cloak_ctx *ctx, const cloak_moe_desc *desc, const void *x_dev,
                                     float *y_dev, int32_t M, int32_t flags, int32_t *experts_out,
                                     float *logits_out, void *stream);

CLOAK_API cloak_status cloak_rekey(cloak_ctx *ctx, uint64_t key, uint32_t new_epoch, void *stream);

/* CLOAK_MODEL_VMM contexts: cloak_keygen, cloak_rekey and the last
 * cloak_rekey_advance (the one that sets *done = 1) end with the remap of the
 * virtual view to the new page map. The remap is a sync point: it
 * synchronises the device (nothing may read the view while a page is
 * unmapped), then unmaps and maps each virtual page whose chunk changed
 * (cuMemUnmap, cuMemMap, cuMemSetAccess). out[0] = pages changed by the last
 * remap, out[1] = remaps so far, out[2] = chunks (arena pages incl. staging),
 * out[3] = host time of the last remap in microseconds, the device
 * synchronisation included. CLOAK_E_STATE for a context without
 * CLOAK_MODEL_VMM. */
CLOAK_API cloak_status cloak_vmm_stats(const cloak_ctx *ctx, int64_t out[4]);

/* Concurrent re-key: the same moves as cloak_rekey, made while the model
 * keeps serving. The remap of Section 4.2 pauses execution at a sync point;
 * here no step waits for the copy. cloak_rekey_begin draws the page map of (key,
 * new_epoch), plans the moves (blocking the calling thread on `side_stream`
 * only) and starts the first wave of page copies on `side_stream`. Every wave
 * writes only pages that no published gather-table entry points at. Then, at
 * each step boundary of the serving stream, cloak_rekey_advance checks
 * (without blocking) whether the wave in flight has landed; if so it enqueues
 * on `serve_stream` the table update that points the moved tiles at their
 * new slots, and starts the next wave on `side_stream` after that update.
 * Until *done = 1 all calls that read the model (linear, stack, serve step,
 * unshuffle) must be ordered on `serve_stream`, and keygen, shuffle and
 * cloak_rekey return CLOAK_E_STATE. At *done = 1 (the last update enqueued)
 * the arena and tables are those of keygen(key, new_epoch) + shuffle.
 * Errors: CLOAK_E_STATE (no job / a job already running), CLOAK_E_INVAL
 * (wrong key, the two streams equal, null `done`). */
CLOAK_API cloak_status cloak_rekey_begin(cloak_ctx *ctx, uint64_t key, uint32_t new_epoch,
                                         void *side_stream);
CLOAK_API cloak_status cloak_rekey_advance(cloak_ctx *ctx, void *serve_stream, void *side_stream,
                                           int32_t *done);

/* Status recorded by device code (bounded waits, bounds checks) since the
 * last call; reading it synchronises the device and clears it. */
CLOAK_API cloak_status cloak_device_status(cloak_ctx *ctx);

/* Failure-detection self-test, with no fault: one block runs two waits that
 * nothing satisfies -- the bounded mbarrier wait every pipelined kernel uses,
 * on a barrier nothing arrives at, and a bounded spin on a device flag
 * nothing sets. Each must give up after its limit (2 s) and record
 * CLOAK_E_TIMEOUT in the status word cloak_device_status reads. Blocks about
 * 2 s; clears the status afterwards; the context stays usable. CLOAK_OK when
 * both waits reported their timeout, CLOAK_E_CUDA (with a message) if not. */
CLOAK_API cloak_status cloak_check_waits(cloak_ctx *ctx, void *stream);

/* Text of the last CUDA error recorded in this context (or ""). */
CLOAK_API const char *cloak_last_error(const cloak_ctx *ctx);

/* Number of kernels this context has launched (a running count). */
CLOAK_API int64_t cloak_launch_count(const cloak_ctx *ctx);

/* Library build identification string. */
CLOAK_API const char *cloak_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CLOAK_H */
