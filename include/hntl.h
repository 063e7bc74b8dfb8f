/*
 * hntl.h - C ABI of the B300 (sm_103a) HNTL batched query path.
 *
 * HNTL (Hierarchical No-pointer Tangent-Local search) splits the corpus into
 * grains, stores each row as r tangent coordinates in its grain's local PCA
 * basis plus a residual norm, and answers a query in five steps:
 *   1. routing to the nprobe nearest grain centres      (sec. 2.1 step 1, sec. 2.3)
 *   2. projection into each probed grain's basis        (Eq. 1-4)
 *   3. Block-SoA scan with D = ||z_q - z_i||^2 + rho_q + rho_i   (Eq. 6, sec. 2.4)
 *   4. pool of the C smallest D                          (Table 1, "Pool C")
 *   5. exact L2 rerank of the pool to the top k          (sec. 2.1 step 4, Mode B)
 *
 * Conventions for every call:
 *   - Return value: HNTL_OK (0) or a negative HNTL_E* code; no exception or
 *     abort crosses the ABI. hntl_last_error() gives a thread-local message.
 *   - "device" pointers are CUDA global-memory addresses on the index's
 *     device; "host" pointers are ordinary CPU memory. The caller owns every
 *     buffer it passes; the library owns the index and frees it in
 *     hntl_index_free().
 *   - Asynchronous calls take a cudaStream_t passed as void* (NULL = legacy
 *     default stream). They enqueue work and return; argument errors are
 *     reported before anything is enqueued, launch errors from the enqueue.
 *   - Distances are squared L2. Ordering everywhere is (distance, id)
 *     ascending; routing is (distance, grain) ascending.
 *   - Limits: 1 <= r <= 64, r <= d, 1 <= nprobe <= G, 1 <= k <= C <= 1024
 *     (C below k is raised to k), G <= 8192. Violations return HNTL_EINVAL.
 */
#ifndef HNTL_H_
#define HNTL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HNTL_OK 0
#define HNTL_EINVAL (-1)   /* bad argument, size or limit */
#define HNTL_ENOMEM (-2)   /* device or host allocation failed */
#define HNTL_ECUDA (-3)    /* a CUDA call or kernel launch failed */
#define HNTL_EIO (-4)      /* file could not be opened, read or written */
#define HNTL_EFORMAT (-5)  /* index file malformed, truncated or checksum mismatch */
#define HNTL_ETIMEOUT (-6) /* a bounded device wait gave up */
#define HNTL_EBUSY (-7)    /* admission refused: memory budget or slots exhausted */

/* Index precision. FP32: FP32 raw rows and coordinates (the plain method).
 * BF16_FP8: BF16 raw rows, FP8-E4M3 coordinates with a per-grain FP32 scale.
 * INT16: the paper's 16-bit form (Eq. 5), built at load from an FP32 file:
 * per grain the steps delta_g = fl32(max |z| / 16383) and
 * dres_g = fl32(max(max rho, fl32(max|z|^2) 2^-20) / 32767) (rows use at most
 * half of each 16-bit range),
 * int16 coordinates rint(fl32(z / delta_g)) and uint16 residual norms
 * rint(fl32(rho / dres_g)), all in IEEE single precision; queries are
 * quantised with the same steps, coordinates saturating at +-32767 and the
 * residual code clipped at 65535, and a grain is left out of a query's scan
 * when more than a quarter of the query's coordinates saturate (the
 * Quantization Envelope Filter, sec. 2.3). The scan evaluates Eq. 6 on the
 * codes: the exact integer S = sum_j (q_j - c_j)^2 (on the integer dot-product
 * units), then D = fl32(fl32(delta_g^2) * fl32(S)) + fl32(rho_q + rho_i) with
 * the residuals on their grid. FP32 raw rows for the rerank. Mode A is not
 * available for this form. */
#define HNTL_PREC_FP32 0
#define HNTL_PREC_BF16_FP8 1
#define HNTL_PREC_INT16 2
/* OR-ed into the 16-bit form's precision (hntl_index_load, or the precision
 * of hntl_build_params): also leave a grain out of a query's scan when the
 * query's residual code would exceed 65535, instead of clipping it. The
 * paper's filter counts saturated coordinates only; this option is the
 * library's own rule for queries far outside a grain's subspace, whose clipped
 * residual would make that grain's rows look close. HNTL_EINVAL with the
 * other forms. */
#define HNTL_INT16_RESID_PRUNE 0x200u
/* OR-ed into the precision of hntl_build_params with HNTL_PREC_BF16_FP8: the
 * index also keeps the second BF16 part of every raw row, bf16(x - bf16(x))
 * (N x d BF16 more; with the first part it carries 16 significant bits of x
 * exactly), and the rerank (Mode B) takes two stages: the pool by distance to
 * the BF16 rows, then its min(C, 2k) smallest (distance, id) by distance to
 * the sum of both parts, of which the k smallest are returned. The library's
 * own option (the paper's rerank is on the raw rows): it wins back the
 * ranking the BF16 rows lose at about 2k more row reads per query.
 * HNTL_EINVAL with the other forms and at load (index files hold one BF16
 * part). */
#define HNTL_RERANK_REFINE 0x400u

/* The 16-bit form's quantisation of stored rows (Eq. 5, the steps above) as
 * the loader and the builder apply it, on host arrays: Z [N][r] FP32
 * coordinates and rho [N] FP32 residual norms of rows stored grain by grain,
 * goff [G + 1] grain offsets (goff[0] = 0, non-decreasing, goff[G] = N).
 * Writes delta [G] and dres [G] (1 for a grain whose values are all zero),
 * codes [N][r] int16 and rho_grid [N] = fl32(residual code * dres_g), the
 * residual norms the scan uses. All buffers are the caller's; host only, no
 * device is touched. Errors: EINVAL (null pointer, G = 0, r = 0, bad offsets),
 * ENOMEM (host allocation). */
int hntl_int16_quantize_host(const float* Z, const float* rho, const uint64_t* goff, uint32_t G, uint32_t r,
                             float* delta, float* dres, int16_t* codes, float* rho_grid);

typedef struct hntl_index hntl_index; /* opaque; owned by the library */

typedef struct {
  uint64_t n;              /* rows */
  uint32_t d;              /* ambient dimension */
  uint32_t G;              /* grains */
  uint32_t r;              /* tangent dimension */
  uint32_t precision;      /* HNTL_PREC_* */
  uint32_t has_attr;       /* 1 if an int64 attribute column is loaded */
  uint32_t block_rows;     /* rows per Block-SoA block (128) */
  uint64_t n_blocks;       /* Block-SoA blocks over all grains */
  uint64_t max_grain_rows; /* rows of the largest grain */
  uint64_t device_bytes;   /* device memory held by the index */
  int device;              /* CUDA device ordinal */
} hntl_index_desc;

/* Library version string. */
const char* hntl_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* hntl_last_error(void);

/* Load an index file (format: header "HNTLIDX\0", version 1, sections for
 * centres, bases, optional eigenvalues, grain offsets, grain-ordered ids,
 * coordinates and residual norms, optional FP8 coordinates + scales, raw rows
 * in id order (FP32 or BF16), optional int64 attributes, and a trailing
 * position-weighted 64-bit word checksum) onto `device`, laid out as 128-row
 * Block-SoA blocks (dimension-major inside a block, grains padded to whole
 * blocks). precision selects which coordinate/raw-row sections the search
 * uses (HNTL_PREC_BF16_FP8 needs them in the file); OR-ing HNTL_LOAD_NO_RAW
 * into it leaves the raw rows on the host: such an index serves Mode A
 * (hntl_search_mode_a, which reads no raw row, as sec. 1 describes Mode A) and
 * routing, and hntl_search (Mode B) returns HNTL_EINVAL. Blocking; on success
 * *out owns device memory. Errors: EIO (open/read), EFORMAT (magic, version,
 * sizes, offsets, ids, truncation, checksum), EINVAL, ENOMEM, ECUDA. */
#define HNTL_LOAD_NO_RAW 0x100u
int hntl_index_load(const char* path, int device, uint32_t precision, hntl_index** out);

/* Parameters of hntl_index_build (zero-initialise, then set what you need). */
typedef struct {
  uint32_t precision;     /* HNTL_PREC_*: FP32, or BF16 rows + FP8 coordinates */
  uint32_t max_iter;      /* Lloyd iterations on the training rows (0 = 10) */
  uint64_t n_train;       /* k-means training rows, strided over the data (0 = min(N, 256 G)) */
  uint64_t n_seed;        /* k-means++ seeding rows, strided over the training rows (0 = min(n_train, 32 G)) */
  uint32_t pca_iters;     /* orthogonal iterations for each grain's basis (0 = 12) */
  uint32_t max_grain_rows; /* 0: every row joins its nearest centre; else grains of at most this many rows
                              (>= ceil(N / G)) by deferred acceptance, see hntl_index_build */
  uint64_t seed;          /* initial bases, and the k-means++ draws when u is NULL */
  const double* u;        /* host, G uniform draws in [0, 1) consumed by k-means++, or NULL */
  const int64_t* d_attr;  /* device, N int64 attributes in id order (for filtered search), or NULL */
} hntl_build_params;

/* Build an index on the GPU from raw rows d_X (device, N x d FP32 row-major;
 * the index keeps its own copy, BF16 in the precision form) and return it in
 * *out. Grains: k-means++ seeding and Lloyd iterations (the paper leaves the
 * partitioning open, sec. 2.2), then every row goes to its nearest centre and
 * each centre becomes the mean of its members. With max_grain_rows = cap > 0
 * the final assignment instead bounds every grain at cap rows: deferred
 * acceptance with rows proposing (Gale and Shapley, 1962), rows ranking
 * centres by (distance, grain) and centres ranking rows by (distance, row),
 * which gives the row-optimal stable assignment (balanced work per grain; the
 * grains are then no longer the centres' Voronoi cells). Basis of each grain (sec. 2.2):
 * the dominant r-dimensional subspace of the grain covariance by orthogonal
 * iteration; coordinates and residual norms by Eq. 1-4. Precision form: FP8
 * E4M3 coordinates with scale s_g = max|z| / 448 per grain, BF16 rows.
 * Blocking (synchronises `stream`). Temporary device memory: about
 * 4 (256 G + 32 G) d + 12 N + min(8 GiB, 4 G d^2) bytes plus the index.
 * Errors: EINVAL (sizes, 1 <= r <= min(d, 64), G <= min(N, 8192)), ENOMEM, ECUDA. */
int hntl_index_build(const float* d_X, uint64_t N, uint32_t d, uint32_t G, uint32_t r, const hntl_build_params* params,
                     int device, void* stream, hntl_index** out);

/* Describe an index. */
int hntl_index_info(const hntl_index* idx, hntl_index_desc* out);

/* Free an index and its device memory (NULL is a no-op). Blocking. */
void hntl_index_free(hntl_index* idx);

/* ---- grain shards (the query path of sec. 2.1 split by grains) ----------
 * Steps 1-4 run grain by grain, so an index splits into S shards by grains:
 * every shard keeps all G centres and bases (it routes each query as the
 * whole index does) and the rows, coordinates and raw rows of its own grains
 * (the others are empty). A search of a shard returns that shard's top k of
 * its own pool of C; hntl_merge_topk takes the k best by (distance, id) over
 * the shards. The shards' pools together contain the whole index's pool, so
 * the merged top k is the exact-distance top k over a superset of it (equal
 * to the single-index result whenever that pool's top k is also each
 * owning shard's). */

/* Assign grains to S shards by rows (host only): grains in order of
 * (rows descending, grain ascending), each to the shard with the fewest rows
 * so far (lowest shard on ties). h_grain_rows: G row counts (as from
 * hntl_index_grain_rows); h_shard_of_grain: G outputs in [0, S).
 * Errors: EINVAL (null, G = 0, S = 0 or S > G). */
int hntl_shard_assign(const uint32_t* h_grain_rows, uint32_t G, uint32_t S, uint32_t* h_shard_of_grain);

/* Make shard `shard` of idx on `device` (any device; copied through host
 * memory): the grains g with h_shard_of_grain[g] == shard keep their rows,
 * the others are empty. The shard numbers its rows 0..n_s-1 in ascending
 * original id (ties break as in idx) and reports local ids from its searches;
 * hntl_shard_global_ids maps them back. *out is an ordinary index (search,
 * Mode A, filters, server) owned by the caller (hntl_index_free). Blocking.
 * Errors: EINVAL (null, idx itself a shard, no grain owned, bad device),
 * ENOMEM, ECUDA. */
int hntl_index_shard(const hntl_index* idx, const uint32_t* h_shard_of_grain, uint32_t shard, int device,
                     hntl_index** out);

/* In place on the shard's device: each local id in d_ids (count int64) is
 * replaced by its original id; -1 (padding) and out-of-range values become -1.
 * Asynchronous on `stream`. Errors: EINVAL (null, not a shard), ECUDA. */
int hntl_shard_global_ids(const hntl_index* shard, int64_t* d_ids, uint64_t count, void* stream);

/* Merge S result lists per query (device): d_ids/d_dist are S x nq x k
 * (shard-major; ids distinct across shards, -1 = padding with any distance),
 * d_out_ids/d_out_dist nq x k: the k best by (distance, id), padded with -1
 * and +inf. Asynchronous on `stream` (the current device's). Errors: EINVAL
 * (null with nq > 0, S = 0, k = 0, S k > 2^24), ECUDA. */
int hntl_merge_topk(const int64_t* d_ids, const float* d_dist, uint32_t S, uint32_t nq, uint32_t k,
                    int64_t* d_out_ids, float* d_out_dist, void* stream);

/* The same merge on host arrays (for results gathered to host memory, e.g.
 * across processes). Errors: EINVAL. */
int hntl_merge_topk_host(const int64_t* h_ids, const float* h_dist, uint32_t S, uint32_t nq, uint32_t k,
                         int64_t* h_out_ids, float* h_out_dist);

/* Bytes of device workspace hntl_search needs for these parameters (0 if
 * the parameters are invalid; see hntl_last_error). */
size_t hntl_search_workspace_bytes(const hntl_index* idx, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe);

/* Batched Mode B search (the five steps above), asynchronous on `stream`.
 *   d_queries  device, nq x d FP32 row-major
 *   d_filter   device, nq x 2 int64 inclusive [lo, hi] attribute range per
 *              query, or NULL for no filtering (needs an index with attributes)
 *   d_ws       device workspace of ws_bytes >= hntl_search_workspace_bytes(),
 *              256-byte aligned; contents need not be initialised
 *   d_out_ids  device, nq x k int64 ids, (distance, id) ascending; -1 pads
 *   d_out_dist device, nq x k FP32 exact squared distances; +inf pads
 *   d_cand_ids device, nq x C uint32 pool ids (0xFFFFFFFF pads), or NULL
 *   d_cand_dist device, nq x C FP32 approximate distances D of the pool
 *              (+inf pads), or NULL (both or neither)
 *   d_probe    device, nq x nprobe int32 probed grains, or NULL
 * The call is reentrant across streams when each call has its own workspace. */
int hntl_search(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
                const int64_t* d_filter, void* d_ws, size_t ws_bytes, int64_t* d_out_ids, float* d_out_dist,
                uint32_t* d_cand_ids, float* d_cand_dist, int32_t* d_probe, void* stream);

/* Batched Mode A search (sec. 2.1 step 4 "Mode A"; sec. 1, the dual-mode
 * planner): steps 1-4 as hntl_search, then the pool is reranked by the
 * squared distance from the query, as routed and projected, to each member's
 * reconstruction mu_g + W_g z_i (the subspace reconstruction of Eq. 3) from
 * its grain's centre and basis and its stored coordinates; no raw row is
 * read. Computed as ||v'||^2 - 2 z_i . z_q + z_i^T (U_g U_g^T) z_i with
 * v' = q - mu_g (q, mu_g, U_g BF16 and z_i the decoded FP8 coordinates in the
 * precision form), which equals the reconstruction distance for any basis.
 * Arguments, layout, workspace (hntl_search_workspace_bytes), ownership and
 * errors as hntl_search; d_out_dist holds the reconstruction distances, and
 * there is no probe output. */
int hntl_search_mode_a(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C,
                       uint32_t nprobe, const int64_t* d_filter, void* d_ws, size_t ws_bytes, int64_t* d_out_ids,
                       float* d_out_dist, uint32_t* d_cand_ids, float* d_cand_dist, void* stream);

/* Device workspace hntl_search_host needs: the search workspace followed by
 * device staging for the queries, the filters (if with_filter) and results. */
size_t hntl_search_host_workspace_bytes(const hntl_index* idx, uint32_t nq, uint32_t k, uint32_t C, uint32_t nprobe,
                                        int with_filter);

/* Blocking convenience form with HOST buffers (pinned memory makes the
 * copies asynchronous): copies the queries (and filters) to device staging
 * inside d_ws, runs hntl_search on `stream`, copies ids and distances back
 * and synchronises the stream. h_filter may be NULL. h_out_ids/h_out_dist
 * are nq x k. */
int hntl_search_host(const hntl_index* idx, const float* h_queries, uint32_t nq, uint32_t k, uint32_t C,
                     uint32_t nprobe, const int64_t* h_filter, void* d_ws, size_t ws_bytes, int64_t* h_out_ids,
                     float* h_out_dist, void* stream);

/* Per-grain row counts (host array of G entries). */
int hntl_index_grain_rows(const hntl_index* idx, uint32_t* h_rows);

/* Copy the index's arrays to HOST memory in grain order (any pointer may be
 * NULL to skip it): centres G x d, bases G x r x d, grain offsets G+1, ids N
 * (original id of each grain-ordered row), coordinates N x r (FP8 indices:
 * codes decoded and multiplied by the grain scale) and residual norms N.
 * Blocking. */
int hntl_index_export(const hntl_index* idx, float* h_M, float* h_U, uint64_t* h_grain_off, uint32_t* h_ids,
                      float* h_Z, float* h_rho);

/* Stage timing. While enabled, every hntl_search records CUDA events on its
 * own stream between its stages: 0 routing, 1 bucketing, 2 projection,
 * 3 pool threshold (pilot), 4 scan, 5 pool selection, 6 rerank.
 * hntl_profile_read waits for the recorded events, adds their elapsed
 * milliseconds per stage into ms[0..6], returns the number of searches
 * covered in *calls and clears the record. */
#define HNTL_NSTAGES 7
int hntl_profile_enable(int on);
int hntl_profile_read(double* ms, uint64_t* calls);

/* Centroid routing alone (step 1), asynchronous: the nprobe nearest grain
 * centres of each query by (||q - mu_g||^2, g), with their FP32 distances.
 * d_ws/ws_bytes as for hntl_search_workspace_bytes(idx, nq, 1, 1, nprobe). */
int hntl_route(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t nprobe, void* d_ws,
               size_t ws_bytes, int32_t* d_probe, float* d_probe_dist, void* stream);

/* Allocation-free centroid routing (the paper has no counterpart; this is a
 * service to callers). Some callers cannot allocate device memory at query
 * time, for example a host application that reserves the whole GPU at start-up
 * and gives its plug-ins no allocator, or a latency-critical loop in which a
 * cudaMalloc would synchronise the device. This call makes the selection
 * hntl_route makes (the nprobe nearest centres of each query by (distance,
 * grain), with their FP32 squared distances, into d_probe / d_probe_dist,
 * nq x nprobe, device) without any caller workspace and without allocating:
 * its scratch is one fixed device array inside the library of 2^21 floats
 * (8 MiB), held by every GPU that loads the library until the process exits.
 * It always forms each distance in the direct SIMT form (one FP32 sum of
 * (q_t - mu_t)^2 per centre), while hntl_route may take tensor-core
 * approximations refined in another summation order; the distances then agree
 * to FP32 rounding, and where two centres are closer than that rounding the
 * two calls can order them, or pick the nprobe-th, differently.
 *   - nq * G must not exceed 2^21 (2,097,152); larger batches return
 *     HNTL_EINVAL with a message. Route them in slices.
 *   - FP32 indices only (HNTL_EINVAL for the precision form).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins.
 *   - All calls share the array, so calls whose kernels may overlap on the GPU
 *     (different streams or host threads) race; serialise them.
 * Asynchronous on `stream`; errors as for hntl_route. */
int hntl_route_noalloc(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t nprobe, int32_t* d_probe,
                       float* d_probe_dist, void* stream);

/* Search with caller-supplied probes (e.g. from hntl_router_route): as
 * hntl_search, but step 1 is replaced by d_probe_in (device, nq x nprobe
 * int32 grain ids, distinct within a query; an id outside [0, G) is replaced
 * by 0 and sets bit 2 of the device status). The routing distances the
 * projection needs are recomputed for the given probes. Workspace as for
 * hntl_search_workspace_bytes. */
int hntl_search_probes(const hntl_index* idx, const float* d_queries, uint32_t nq, uint32_t k, uint32_t C,
                       uint32_t nprobe, const int32_t* d_probe_in, const int64_t* d_filter, void* d_ws,
                       size_t ws_bytes, int64_t* d_out_ids, float* d_out_dist, uint32_t* d_cand_ids,
                       float* d_cand_dist, void* stream);

/* Diagnostic: the number of pool survivors of each query (rows whose scan
 * distance passed the query's pilot bound, before the exact C-smallest
 * selection) of the last hntl_search that used this workspace with the same
 * nq, C and nprobe; copied to d_counts (device, nq uint32) on `stream`. A
 * count above max(16384, 32 C) means the survivor list overflowed and the pool
 * was recomputed from every probed row. */
int hntl_search_survivors(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                          uint32_t nprobe, uint32_t* d_counts, void* stream);

/* Diagnostic: the scan's work-item counters of the last hntl_search of the
 * precision form that used this workspace with the same nq, C and nprobe,
 * copied to d_stats (device, 5 uint32) on `stream`: [0] dense items claimed
 * by the tensor-core scan (at least [1]), [1] dense items (at least kSTDense =
 * 8 live pairs), [2] sparse items with few live pairs, [3] sparse items
 * claimed by the direct-form scan (at least [2] + [4]), [4] costly sparse
 * items (taken first). All zero for the FP32 and 16-bit forms, which scan
 * every probed block in one kernel. */
int hntl_search_scan_stats(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                           uint32_t nprobe, uint32_t* d_stats, void* stream);

/* Diagnostic of the 16-bit form: the query codes of the last hntl_search that
 * used this workspace with the same nq, C and nprobe (Eq. 5 applied to each
 * (query, probe) pair's z_q and rho_q), in query order: d_codes (device,
 * nq x nprobe x r int16) and d_rcodes (device, nq x nprobe int32 residual
 * codes, -1 for a pair the envelope filter left out), on `stream`. With them
 * an oracle can evaluate the integer scan on exactly the GPU's integer inputs.
 * HNTL_EINVAL for the other forms. */
int hntl_search_pair_codes(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                           uint32_t nprobe, int16_t* d_codes, int32_t* d_rcodes, void* stream);

/* Diagnostic: the projection step's output (Eq. 1-4) of the last hntl_search
 * that used this workspace with the same nq, C and nprobe, in query order:
 * d_zq (device, nq x nprobe x r FP32 z_q) and d_rhoq (device, nq x nprobe FP32
 * rho_q), on `stream`. In the 16-bit form these are the values on the grain's
 * grids, and rho_q is +inf for a pair the envelope filter left out. */
int hntl_search_pair_proj(const hntl_index* idx, const void* d_ws, size_t ws_bytes, uint32_t nq, uint32_t C,
                          uint32_t nprobe, float* d_zq, float* d_rhoq, void* stream);

/* Test hook (the paper has no counterpart): caps the grid of every persistent
 * kernel of the search (tensor-core routing, the tensor-core projection and
 * explicit residual of either form, both scans of the precision form) at
 * `ctas` CTAs, 0 restoring the default of about one
 * per SM. A capped kernel still processes every work item, each CTA looping
 * over many of them, so a small test case exercises the multi-item paths
 * (accumulator ping-pong, mbarrier phases carried across items, prefetch of
 * the next item) that full-size batches take. Process-wide; set it only
 * while no search runs. Always HNTL_OK. */
int hntl_debug_set_persistent_cap(uint32_t ctas);

/* Device status word of an index (blocking read): bit 0 = a bounded
 * device-side wait gave up (kernels then skip their results), bit 1 = an
 * invalid probe id was supplied. Returns HNTL_ETIMEOUT if bit 0 is set,
 * else HNTL_OK; `clear` resets the word. */
int hntl_device_status(const hntl_index* idx, int* status, int clear);

/* Test hook for the bounded device waits: launches one kernel that polls, at
 * most `polls` times (1 .. 2^20), an mbarrier phase that nothing completes,
 * then gives up and sets bit 0 of the index's device status, as a stalled
 * tensor-core pipeline would. hntl_device_status then returns HNTL_ETIMEOUT.
 * The GPU context stays usable. */
int hntl_selftest_wait_timeout(const hntl_index* idx, uint32_t polls, void* stream);

/* ---- learned grain router (the paper lists learned grain partitioning as
 * future work, sec. 4; this router is the library's own addition) ----
 * An MLP d -> h1 -> h2 -> G with exact GELU after each hidden layer and a
 * softmax over the G grains. Training: soft-label cross-entropy against
 * targets T (per row, the share of the query's brute-force top-10 neighbours
 * stored in each grain) with AdamW (decoupled weight decay, FP32 master
 * weights). Matrix products are tcgen05 BF16 GEMMs with FP32 accumulation;
 * the tensors rounded to BF16 are the input, the weights, both hidden
 * activations and the three back-propagated output/hidden gradients, and
 * nothing else. d, h1, h2, G and training batches must be multiples of 8. */
typedef struct hntl_router hntl_router;

/* Create a router on `device` with the given initial FP32 parameters (host;
 * W1 h1 x d, b1 h1, W2 h2 x h1, b2 h2, W3 G x h2, b3 G, row-major). Device
 * buffers are sized for batches of at most max_batch rows. */
int hntl_router_create(int device, uint32_t d, uint32_t h1, uint32_t h2, uint32_t G, uint32_t max_batch,
                       const float* h_W1, const float* h_b1, const float* h_W2, const float* h_b2, const float* h_W3,
                       const float* h_b3, hntl_router** out);
void hntl_router_free(hntl_router* router);

/* Copy the FP32 master parameters / the gradients of the last step to host (NULL skips). Blocking. */
int hntl_router_params(const hntl_router* router, float* h_W1, float* h_b1, float* h_W2, float* h_b2, float* h_W3,
                       float* h_b3);
int hntl_router_grads(const hntl_router* router, float* h_dW1, float* h_db1, float* h_dW2, float* h_db2,
                      float* h_dW3, float* h_db3);

/* One training step on a batch (device X: B x d FP32, T: B x G FP32 soft
 * targets): forward, loss (added to *d_loss, device FP32, if not NULL),
 * backward, and with update != 0 one AdamW step (lr, weight decay wd on the
 * weight matrices, betas 0.9 / 0.999, eps 1e-8; the step count lives on the
 * device). Asynchronous on `stream`. By default the step's launches are
 * captured once into a CUDA graph on a private stream and the graph is
 * launched on `stream`; a call whose arguments (pointers, B, lr, wd, update)
 * differ from the captured ones captures again first. Not for concurrent
 * calls on one router from several threads. */
int hntl_router_step(hntl_router* router, const float* d_X, const float* d_T, uint32_t B, float lr, float wd,
                     int update, float* d_loss, void* stream);

/* enable = 0: hntl_router_step launches its kernels directly instead of
 * through the captured graph (the same kernels and arguments, so the same
 * parameters and gradients bit for bit; the loss is a sum of per-row atomic
 * adds on both paths, so its last bits follow the order the rows finish in);
 * enable != 0 (the default) restores the graph. */
int hntl_router_set_graphs(hntl_router* router, int enable);

/* HNTL_ETIMEOUT if a tensor-core pipeline wait of one of the router's GEMMs
 * gave up (the kernel then skipped its output), else HNTL_OK. Blocking: reads
 * the router's device error flag after the work queued so far on the legacy
 * default stream. */
int hntl_router_status(const hntl_router* router);

/* Logits (device, B x G FP32) of a batch of rows. Asynchronous. */
int hntl_router_logits(hntl_router* router, const float* d_X, uint32_t B, float* d_logits, void* stream);

/* Router routing: each query's nprobe largest-logit grains (ties to the
 * lower grain); where their softmax mass is below tau the query takes its
 * centroid routing instead (tau <= 0 never falls back, tau > 1 always does).
 * For nprobe <= 64 and G <= 8192 one fused kernel per query selects the
 * probes and decides the fallback from the logits, and with tau <= 0 the
 * centroid routing is not computed at all. *d_nfallback (device, optional)
 * counts the queries that fell back. Workspace:
 * hntl_router_route_workspace_bytes. */
size_t hntl_router_route_workspace_bytes(const hntl_router* router, const hntl_index* idx, uint32_t nq,
                                         uint32_t nprobe);
int hntl_router_route(hntl_router* router, const hntl_index* idx, const float* d_queries, uint32_t nq,
                      uint32_t nprobe, float tau, void* d_ws, size_t ws_bytes, int32_t* d_probe,
                      uint32_t* d_nfallback, void* stream);

/* ---- continuous-batching server (the library's addition; the paper serves
 * one query at a time on a CPU) ----
 * A worker thread batches admitted requests as they arrive and runs each batch
 * as one captured CUDA graph (gather of its rows from the slot table, the
 * whole Mode B search with each query's own k and C, result copy to pinned
 * memory). The slot table is mapped pinned host memory: a submission stores
 * its rows there with no CUDA call, and the gather reads them over the host
 * link, so admitting a request never waits behind a running batch. Batches run
 * on one of three lanes, so one forms while others run. A
 * request's result is the same as hntl_search of that query alone with its k
 * and C (every stage is per query). */
typedef struct hntl_server hntl_server;

typedef struct {
  uint64_t completed;  /* requests finished since creation or the last reset */
  uint64_t batches;    /* batches launched */
  double mean_batch;   /* requests per batch */
  double p50_us, p99_us, max_us; /* latency from arrival (or submission) to completion */
  uint32_t slots;      /* requests admitted at once (max_slots) */
  /* the latency in four parts: arrival stamp to the submission call (the
   * caller's lag), the call to admission (the row's copy into its slot),
   * admission to the launch of the request's batch, launch to completion */
  double lag_p50_us, lag_p99_us, queue_p50_us, queue_p99_us, service_p50_us, service_p99_us;
  double upload_p50_us, upload_p99_us;
} hntl_server_stats;

/* Create a server over `idx` (which must outlive it). mem_budget (bytes of
 * device memory) must hold three lanes (each a search workspace for `batch`
 * queries with k_max, C_max and nprobe, plus batch buffers): ENOMEM if it
 * cannot. max_slots requests can be admitted at once; their slot table takes
 * max_slots x (4 d + 24) bytes of pinned host memory (ENOMEM if that cannot
 * be pinned). Blocking (captures the graphs). */
int hntl_server_create(const hntl_index* idx, size_t mem_budget, uint32_t max_slots, uint32_t batch, uint32_t nprobe,
                       uint32_t k_max, uint32_t C_max, hntl_server** out);
void hntl_server_free(hntl_server* server);

/* Admit up to n requests (host queries n x d FP32, k and C per request, optional
 * inclusive int64 ranges n x 2 for an index with attributes, optional arrival
 * times in steady-clock nanoseconds for latency accounting). Requests are
 * admitted in order while slots are free: *n_admitted tells how many; the
 * call returns HNTL_EBUSY if fewer than n were admitted. tickets[i] identifies
 * admitted request i. Makes no CUDA call: the rows are copied into their
 * slots with host stores. Safe to call from several threads. */
int hntl_server_submit(hntl_server* server, const float* h_queries, uint32_t n, const uint32_t* h_k,
                       const uint32_t* h_C, const int64_t* h_ranges, const int64_t* h_arrival_ns, uint64_t* tickets,
                       uint32_t* n_admitted);

/* Collects many results at once. For each i < n with done[i] == 0 whose
 * request has completed, copies its k ids and distances to row i of h_ids /
 * h_dist (row stride `stride` >= k_max elements; either may be NULL to
 * discard), releases the ticket and sets done[i] = 1 (entries already 1 are
 * skipped). Waits up to timeout_ms for the rest; *n_done = results copied by
 * this call. Returns HNTL_OK when every entry is done, HNTL_ETIMEOUT if some
 * are still pending, HNTL_EINVAL for an unknown ticket. */
int hntl_server_poll_many(hntl_server* server, const uint64_t* tickets, uint32_t n, int64_t* h_ids,
                          float* h_dist, uint32_t stride, uint8_t* done, uint32_t timeout_ms, uint32_t* n_done);

/* Open-loop replay of a request stream (for measuring the server): request
 * i (query row i of h_queries, n x d; h_k, h_C, optional ranges n x 2) is
 * submitted at or right after its arrival time h_arrival_ns[i] (nanoseconds
 * after the start of the call, non-decreasing), together with the requests
 * that have arrived by then, from the calling thread, which also releases
 * finished requests every millisecond and whenever the slots run out. The
 * arrival stamps are the latency record's start points. For each i with h_want[i] != 0 (h_want may be NULL) the
 * request's k ids are copied to row i of h_ids (n x k_max). Returns HNTL_OK
 * once every request finished (*n_done = n), HNTL_ETIMEOUT after timeout_ms,
 * or the first error of a submission. The server's latency record covers
 * the replayed requests. */
int hntl_server_replay(hntl_server* server, const float* h_queries, uint32_t n, const uint32_t* h_k,
                       const uint32_t* h_C, const int64_t* h_ranges, const int64_t* h_arrival_ns,
                       const uint8_t* h_want, int64_t* h_ids, uint32_t timeout_ms, uint32_t* n_done);

/* Wait up to timeout_ms for a request; on success copy its k ids and
 * distances to host buffers (each must hold the request's k entries; k_max
 * always suffices) and release the ticket. HNTL_ETIMEOUT if it is not done in
 * time (the ticket stays valid), HNTL_EINVAL for an unknown ticket, HNTL_ECUDA
 * once the serving worker has stopped on a CUDA error (its unfinished
 * requests never complete; the call returns as soon as the worker stops). */
int hntl_server_poll(hntl_server* server, uint64_t ticket, int64_t* h_ids, float* h_dist, uint32_t timeout_ms);

/* Latency record since creation or the last reset: completed requests,
 * batches launched and their mean size, p50 / p99 / max latency from each
 * request's arrival stamp to its completion and p50 / p99 of its four parts,
 * and the request slots. Quantiles come from log-linear histograms (64
 * buckets per power of two nanoseconds), so each is within 1/64 of the
 * sample it stands for; the maximum is exact. hntl_server_reset_stats clears
 * the record (not the slots). */
int hntl_server_get_stats(hntl_server* server, hntl_server_stats* out);
int hntl_server_reset_stats(hntl_server* server);

#ifdef __cplusplus
}
#endif

#endif /* HNTL_H_ */
