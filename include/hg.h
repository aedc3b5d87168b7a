/*
 * hg.h -- C ABI of the GB300-native HashGraph library (libhg.so).
 *
 * HashGraph (Green, "HashGraph - Scalable Hash Tables Using A Sparse Graph
 * Data Structure", 2019) stores a static hash table as a CSR graph: bucket v
 * (a "vertex", Section 3.1) owns the edges [offsets[v], offsets[v+1]) of the
 * edge arrays (keys, ids).  The table always holds exactly n edges whatever
 * the number of buckets V (Section 3.2, "HashGraph Collision Management").
 *
 * Conventions for every entry point
 *   - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *     never allocates, frees or retains them.  Host pointers (configs, table
 *     views) are only read during the call.
 *   - d_keys / d_ids / d_queries must be aligned to 16 bytes (tensors from a
 *     CUDA caching allocator are); other device arrays to their element size.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  Argument errors are returned synchronously and launch
 *     nothing.  A failed launch returns HG_ERR_CUDA; a build or binned probe
 *     whose partition launch failed returns before any kernel that would read
 *     the partition's output is launched.
 *   - Calls that take a workspace write a device status word into it (bounded
 *     waits that gave up, capacity overflow).  Read it after the stream has
 *     finished with hg_workspace_status().
 *   - Keys are uint32 or uint64.  Key value 0 and the maximum key are ordinary
 *     keys: there is no empty-slot sentinel because there is no open
 *     addressing (Section 3.2).
 *   - Canonical table order: inside a bucket, edges appear in ascending input
 *     position.  Every algorithm variant (V1, V2, any bin size, batched)
 *     produces the same bytes.
 */
#ifndef HG_H
#define HG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HG_OK = 0,
  HG_ERR_INVALID_ARG = 1,         /* bad pointer, size, alignment or enum value */
  HG_ERR_WORKSPACE_TOO_SMALL = 2, /* ws_bytes below the *_workspace_size() result */
  HG_ERR_OVERFLOW = 3,            /* output capacity exceeded (device status) */
  HG_ERR_CUDA = 4,                /* a CUDA launch or runtime call failed */
  HG_ERR_TIMEOUT = 5,             /* a bounded device-side wait gave up (device status) */
  HG_ERR_MODEL = 6,               /* malformed learned-map model blob */
  HG_ERR_UNSUPPORTED = 7          /* valid request outside what this build supports */
} hg_status;

typedef enum { HG_KEY_U32 = 0, HG_KEY_U64 = 1 } hg_key_type;

/* Bucket map.  MURMUR3: bucket = MurmurHash3_x86_32(key bytes, little-endian,
 * 4 or 8 bytes, seed) mod V -- Eq. 1 of Section 2 ("hash(a) mod N/C_V").
 * LEARNED: an order-preserving fp32 piecewise-linear CDF model (not in the
 * paper; see hg_learned_train). */
typedef enum { HG_MAP_MURMUR3 = 0, HG_MAP_LEARNED = 1 } hg_map_kind;

/* Build algorithm.  V1 = Alg. 1 (one level: global histogram, prefix sum,
 * scatter).  V2 = Alg. 2 (two levels: partition by hash range into bins, then
 * build every bin in on-chip shared memory).  AUTO picks V2 when it applies. */
typedef enum { HG_ALGO_AUTO = 0, HG_ALGO_V1 = 1, HG_ALGO_V2 = 2 } hg_algo;

typedef struct {
  int32_t key_type;          /* hg_key_type */
  int32_t map;               /* hg_map_kind */
  uint64_t num_buckets;      /* V = N / C_V (Eq. 1); 1 <= V <= 2^32 (V2: <= 2^30) */
  uint32_t seed;             /* Murmur3 seed */
  int32_t algo;              /* hg_algo */
  const void* d_model;       /* learned map: device pointer to the model blob */
  uint32_t bin_shift;        /* V2: log2(buckets per bin); 0 = automatic */
  uint32_t threads_per_bin;  /* V2: threads of the bin-build kernel (512|1024); 0 = auto */
} hg_config;

/* A built table (read-only view).  offsets: uint32[V+1]; keys: n keys of
 * cfg.key_type; ids: uint32[n] (the build input position, or the caller's id). */
typedef struct {
  uint64_t n;
  const uint32_t* d_offsets;
  const void* d_keys;
  const uint32_t* d_ids;
} hg_table;

/* ---------------------------------------------------------------- build --
 * HashGraph build (Alg. 1 / Alg. 2, Section 3.2-3.3).
 *   d_keys     [n] keys (cfg->key_type)
 *   d_ids      [n] uint32 ids, or NULL for ids = 0..n-1 (the input position,
 *              "E[pos] <- (A[i], i)" in Alg. 1)
 *   d_offsets  out [V+1] uint32: exclusive prefix sum of the bucket sizes,
 *              offsets[0] = 0, offsets[V] = n
 *   d_csr_keys out [n] keys grouped by bucket
 *   d_csr_ids  out [n] ids in the same order
 *   d_ws/ws_bytes  workspace of at least hg_build_workspace_size(cfg, n) bytes
 * Requires n < 2^32.  Output buffers must not overlap the inputs.  The
 * result is one canonical table whatever the configuration: inside every
 * bucket the edges follow their input order (with d_ids NULL the build may
 * partition in any order and restore it from the ids, which are then the
 * positions). */
size_t hg_build_workspace_size(const hg_config* cfg, uint64_t n);
hg_status hg_build(const hg_config* cfg, const void* d_keys, const uint32_t* d_ids, uint64_t n,
                   uint32_t* d_offsets, void* d_csr_keys, uint32_t* d_csr_ids, void* d_ws,
                   size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------- probe --
 * HashGraph-Probe-Standard (Section 3.4): for each query, map it to its
 * bucket and count every edge of that bucket whose key equals the query
 * ("finds all instances", Section 5.2).
 *   table      a table built with the same cfg (key type, V, map, seed)
 *   d_queries  [q] keys;  d_counts out [q] uint32 match counts
 * Needs no workspace. */
hg_status hg_probe(const hg_config* cfg, const hg_table* table, const void* d_queries, uint64_t q,
                   uint32_t* d_counts, void* stream);

/* Binned probe: the same result as hg_probe (per-query match counts), for
 * large query batches.  The queries are first partitioned by bucket range
 * into at most 256 groups (128 by default; the V2 build's histogram and
 * partition kernels applied to the queries), each group is probed while its
 * slice of the table stays in L2, and the counts are merged back into query
 * order.  Trades random DRAM reads (one burst per 4-byte read) for
 * sequential passes.
 *   d_queries must be 16-byte aligned; q < 2^32.
 *   d_ws/ws_bytes: at least hg_probe_workspace_size(cfg, table->n, q) bytes. */
size_t hg_probe_workspace_size(const hg_config* cfg, uint64_t table_n, uint64_t q);
hg_status hg_probe_binned(const hg_config* cfg, const hg_table* table, const void* d_queries,
                          uint64_t q, uint32_t* d_counts, void* d_ws, size_t ws_bytes,
                          void* stream);

/* -------------------------------------------------------- host buffers --
 * Build and probe with inputs and results in host memory, one call: keys
 * and queries are copied host -> device into the caller's staging buffers
 * (d_keys [n], d_queries [q]), the table is built into `table` (device
 * buffers of n keys, table->n must equal n) with implicit ids, the queries
 * are probed (binned when d_probe_ws is given, else direct) into d_counts
 * [q], and the counts are copied back to h_counts [q].  Everything is
 * asynchronous with respect to the host (host buffers should be pinned for
 * the copies to overlap other work); h_counts is valid after `stream` is
 * synchronised.  The two host -> device copies run on a copy stream the
 * library keeps per device, ordered after the work already queued on
 * `stream` and joined back to `stream` by events, and the kernels of a call
 * start after those of the previous call on the same device (on whatever
 * stream).  Calls made on several streams (batches in flight) therefore
 * queue their uploads one after another, run their kernels back to back,
 * and overlap one call's copies with another's kernels.  Calls from several
 * host threads are serialised while they enqueue.  Not meant for stream
 * capture (the ordering events live outside any graph).  Workspaces as for
 * hg_build and hg_probe_binned.  No counterpart in the paper: it is the
 * whole hot path behind one call. */
hg_status hg_build_probe_host(const hg_config* cfg, const void* h_keys, uint64_t n, const void* h_queries,
                              uint64_t q, uint32_t* h_counts, void* d_keys, void* d_queries, uint32_t* d_counts,
                              const hg_table* table, void* d_build_ws, size_t build_ws_bytes, void* d_probe_ws,
                              size_t probe_ws_bytes, void* stream);

/* ----------------------------------------------------------- self-test --
 * Every wait inside the kernels (TMA copy completion on an mbarrier) is
 * bounded: after 2 s it records HG_ERR_TIMEOUT in the workspace status and
 * the kernel returns, so the context stays usable.  This call exercises that
 * path on purpose: one CTA waits on a barrier that is never completed (it
 * expects two arrivals and gets one) with a limit of limit_ms (1..5000); the
 * workspace status (first 256 bytes of d_ws) then reads HG_ERR_TIMEOUT.  No
 * counterpart in the paper. */
hg_status hg_selftest_wait_timeout(void* d_ws, uint32_t limit_ms, void* stream);

/* ----------------------------------------------------------------- join --
 * HashGraph-Probe-New (Alg. 3, Section 3.4): both inputs are built into
 * tables with the same V and map; bucket v of A is intersected with bucket v
 * of B.  The inner-join size is the number of (a, b) edge pairs with equal
 * keys.  Both CSRs are walked side by side in bucket order (merge-style); the
 * bucket map is not evaluated, so the tables must be as hg_build wrote them
 * (offsets starting at 0, bucket v's edges at [offsets[v], offsets[v+1])).
 * hg_join_count:
 *   d_total          out [1] int64 join size
 *   d_bucket_counts  out [V] int64 pairs per bucket, or NULL
 * hg_join_materialize: writes every pair (A id, B id) in canonical order
 * (bucket ascending, then A's CSR position, then B's CSR position).
 *   d_build_ids, d_probe_ids  out [capacity] int64
 *   d_total          out [1] int64 join size (also when it exceeds capacity;
 *                    then only the first `capacity` pairs are written and the
 *                    device status is HG_ERR_OVERFLOW)
 * Both need hg_join_workspace_size(cfg, A->n, B->n) bytes of workspace. */
size_t hg_join_workspace_size(const hg_config* cfg, uint64_t nA, uint64_t nB);
/* hg_join_materialize_after_count: hg_join_materialize for a pair of tables
 * that hg_join_count has just counted with the same workspace.  The count
 * leaves every A edge's match count in the workspace; this call scans those
 * into output positions and writes the pairs, so a count followed by the
 * materialisation intersects the buckets once, not twice.  Neither table
 * nor the workspace may change in between.  The device checks that the
 * workspace holds the count of these tables (A and B sizes, offsets and keys
 * pointers, V): on a mismatch it writes no pair, *d_total = 0 and the
 * workspace status reads HG_ERR_INVALID_ARG.  The counts are consumed: a
 * second call without a new count is a mismatch. */
hg_status hg_join_count(const hg_config* cfg, const hg_table* A, const hg_table* B,
                        int64_t* d_total, int64_t* d_bucket_counts, void* d_ws, size_t ws_bytes,
                        void* stream);
hg_status hg_join_materialize(const hg_config* cfg, const hg_table* A, const hg_table* B,
                              int64_t* d_build_ids, int64_t* d_probe_ids, uint64_t capacity,
                              int64_t* d_total, void* d_ws, size_t ws_bytes, void* stream);
hg_status hg_join_materialize_after_count(const hg_config* cfg, const hg_table* A, const hg_table* B,
                                          int64_t* d_build_ids, int64_t* d_probe_ids, uint64_t capacity,
                                          int64_t* d_total, void* d_ws, size_t ws_bytes, void* stream);

/* -------------------------------------------------------------- learned --
 * Learned bucket map: an order-preserving stand-in for "hash(a) mod V".  It
 * is not in the paper (Section 2 hashes with Murmur); the murmur map remains
 * the default and the reference it is judged against.  Model (blob of
 * hg_learned_model_bytes(L) bytes, 8-byte aligned):
 *   header 32 B: u32 magic 'HGLM', u32 L, u64 V, f32 a, f32 b, u32 key_type, u32 flags
 *   leaf   24 B: u64 xmin, f32 slope, f32 icpt, u32 base, u32 width
 *   root:  leaf = clamp(floor(a * f(key) + b), 0, L-1), f(key) = fp32 of the
 *          IEEE bits of fp32(key) (monotone, roughly 2^23 log2 key)
 *   leaf j: bucket = base + clamp(floor(slope * fp32(key - xmin) + icpt), 0, width-1)
 *   (fp32 round-to-nearest, no fused multiply-add; bucket < V; monotone in key)
 * hg_learned_train draws a sample of sample_size keys (SplitMix64 indices,
 * stream 'LEARN', seed), sorts it, fits the root, finds the knots
 * (xmin_j = smallest key the root sends to leaf j or beyond), and fits the
 * knot values of the continuous piecewise-linear CDF.  The prior Y0 is the
 * interpolant, linear in the key, of the sample's rank targets
 * (0, 0), (x_i, V(2i+1)/(2S)), (key max + 1, V) at the knots.  Then `iters`
 * rounds of a Jacobi-preconditioned gradient step (step 0.9) on
 *   loss(Y) = (1/S) [ sum_i (P(x_i) - V(2i+1)/(2S))^2 + rho sum_{j=1..J} (Y_j - Y0_j)^2 ]
 * each followed by the projection onto
 *   Y_j - Y_{j-1} >= gamma (Y0_j - Y0_{j-1})   (running max of Y - gamma Y0)
 * with J the last leaf the root can reach, rho = 1 and gamma = 0.5: the
 * ridge keeps the minimiser unique where knots see few samples, the floor
 * keeps every leaf at least half as wide in buckets as the prior makes it.
 * Deterministic.
 *   d_diag (optional, L+5 doubles): [loss before, loss after, root loss,
 *   unused, knot values Y_0..Y_L]
 * hg_learned_sorted_sample / _root_grad / _leaf_grad expose the sampling and
 * the gradients (root: loss, dL/da, dL/db in double; leaves: dL/dY_j and
 * d2L/dY_j^2 in fp32 at knot values d_Y, Y0 taken from d_sorted) for
 * checking.
 * hg_bucket_stats: bucket-length max, mean, variance and non-empty count of a
 * map over a key set (d_counts: V uint32 scratch). */
size_t hg_learned_model_bytes(uint32_t num_leaves);
size_t hg_learned_workspace_size(int32_t key_type, uint64_t n, uint64_t sample_size, uint32_t num_leaves);
hg_status hg_learned_train(int32_t key_type, const void* d_keys, uint64_t n, uint64_t num_buckets,
                           uint32_t num_leaves, uint64_t sample_size, uint64_t seed, uint32_t iters,
                           void* d_model, double* d_diag, void* d_ws, size_t ws_bytes, void* stream);
hg_status hg_learned_sorted_sample(int32_t key_type, const void* d_keys, uint64_t n,
                                   uint64_t sample_size, uint64_t seed, uint64_t* d_out, void* d_ws,
                                   size_t ws_bytes, void* stream);
hg_status hg_learned_root_grad(int32_t key_type, const uint64_t* d_sorted, uint64_t S,
                               uint32_t num_leaves, double a, double b, double* d_out3, void* d_ws,
                               size_t ws_bytes, void* stream);
hg_status hg_learned_leaf_grad(int32_t key_type, const uint64_t* d_sorted, uint64_t S,
                               uint64_t num_buckets, float a, float b, uint32_t num_leaves,
                               const double* d_Y, float* d_grad, float* d_diag, double* d_loss,
                               void* d_ws, size_t ws_bytes, void* stream);
hg_status hg_bucket_stats(const hg_config* cfg, const void* d_keys, uint64_t n, uint32_t* d_counts,
                          double* d_out4, void* d_ws, size_t ws_bytes, void* stream);

/* Fallback rule of the learned map (not in the paper): Murmur is its judge.
 * Both maps are applied to the same n keys (hg_bucket_stats with cfg's
 * learned model, then with Murmur and cfg->seed); the learned map is kept
 * (*h_keep = 1) while its bucket-length variance is at most var_tolerance
 * times Murmur's and its longest bucket at most max_factor times Murmur's,
 * else *h_keep = 0 and the caller builds with Murmur.  A strict "no worse
 * than Murmur" rule would never keep it: Murmur's balls-into-bins variance
 * equals the load factor, and a CDF fitted to a sample cannot beat that on
 * fresh keys.  Tolerances <= 0 select the defaults below.
 *   cfg        map = HG_MAP_LEARNED, d_model, num_buckets V, seed (for Murmur)
 *   d_counts   V uint32 scratch;  d_ws/ws_bytes >= hg_learned_judge_workspace_size()
 *   h_stats8   optional host out: learned {max, mean, variance, non-empty
 *              buckets}, then Murmur's
 * Synchronous: returns after `stream` has finished both statistics. */
#define HG_LEARNED_VAR_TOLERANCE 1.25
#define HG_LEARNED_MAX_FACTOR 4.0
size_t hg_learned_judge_workspace_size(void);
hg_status hg_learned_judge(const hg_config* cfg, const void* d_keys, uint64_t n, double var_tolerance,
                           double max_factor, uint32_t* d_counts, void* d_ws, size_t ws_bytes, double* h_stats8,
                           int32_t* h_keep, void* stream);

/* -------------------------------------------------------------- batched --
 * Many independent tables of uneven sizes built and probed together.  The
 * paper builds one table per call; batching is not in it.  Table t has n_t
 * uint32 keys (ids 0..n_t-1, their positions), V_t >= 1 buckets (Eq. 1 with
 * its own V_t and the common seed) and q_t queries.  Device arrays are the
 * concatenation over t = 0..T-1 at the positions hg_batch_layout returns
 * (each table's keys and queries start on a 16-byte boundary; up to 3
 * padding slots follow a table and are ignored):
 *   keys      [totals[0]] uint32, table t at key_begin[t]
 *   queries   [totals[1]] uint32, table t at query_begin[t]
 *   offsets   [totals[2]] uint32; table t's V_t + 1 offsets start at
 *             offset_begin[t] and are positions in the concatenated CSR
 *             arrays: bucket v of table t is [offsets[ob+v], offsets[ob+v+1])
 *   csr_keys, csr_ids  [totals[0]]; ids are table-local
 *   counts    [totals[1]] uint32: matches of each query in its own table
 * Table t equals the table hg_build makes from its keys alone, every offset
 * raised by key_begin[t]; counts equal hg_probe's.  The caller owns every
 * buffer; the plan (host memory) owns a CUDA stream, two events and the
 * cached graph.  Arguments are checked synchronously; device errors
 * (timeouts) are read with hg_workspace_status(d_ws).
 * hg_batch_plan_create: host only.  h_num_buckets NULL means V_t =
 *   max(1, n_t).  Totals below 2^32.  Key type uint32 only (uint64:
 *   HG_ERR_UNSUPPORTED).
 * hg_batch_run: enqueues the batch on `stream`.  Tables are grouped into
 *   waves whose buckets fit 2^15 bins of the bin size; per wave one
 *   two-level build (Alg. 2) and one binned probe over the wave's slice of
 *   the common bucket space.  The launch sequence is captured into a CUDA
 *   graph on the first call with a given set of buffers and configuration
 *   and replayed by later calls with the same ones.
 * hg_batch_run_eager: the same launch sequence enqueued directly, without
 *   a graph (per-kernel tracing and profiling see each launch).
 * hg_batch_autotune: synchronous; times `reps` runs of every candidate (bin
 *   shift near the automatic one x 512 / 1024 threads per bin) on the given
 *   buffers, keeps the fastest and returns its time.  Results do not depend
 *   on the configuration.
 * hg_batch_run_plain: the same work as a host loop of hg_build + hg_probe,
 *   one table at a time (offsets then table-local), for comparison.
 * Workspace: hg_batch_workspace_size(plan) bytes, 256-byte aligned, for all
 * three calls. */
typedef struct hg_batch_plan hg_batch_plan;
hg_status hg_batch_plan_create(int32_t key_type, uint32_t seed, uint32_t num_tables,
                               const uint64_t* h_table_sizes, const uint64_t* h_query_sizes,
                               const uint64_t* h_num_buckets, hg_batch_plan** out);
void hg_batch_plan_destroy(hg_batch_plan* plan);
/* h_totals4: keys, queries, offset entries, tables; each *_begin (T+1
 * entries) may be NULL */
hg_status hg_batch_layout(const hg_batch_plan* plan, uint64_t* h_totals4, uint64_t* h_key_begin,
                          uint64_t* h_query_begin, uint64_t* h_offset_begin);
size_t hg_batch_workspace_size(const hg_batch_plan* plan);
/* bin_shift 0 / threads_per_bin 0 = automatic */
hg_status hg_batch_set_config(hg_batch_plan* plan, uint32_t bin_shift, uint32_t threads_per_bin);
hg_status hg_batch_get_config(const hg_batch_plan* plan, uint32_t* bin_shift, uint32_t* threads_per_bin,
                              uint32_t* waves);
hg_status hg_batch_run(hg_batch_plan* plan, const void* d_keys, const void* d_queries, uint32_t* d_offsets,
                       void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts, void* d_ws,
                       size_t ws_bytes, void* stream);
hg_status hg_batch_run_eager(hg_batch_plan* plan, const void* d_keys, const void* d_queries,
                             uint32_t* d_offsets, void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts,
                             void* d_ws, size_t ws_bytes, void* stream);
hg_status hg_batch_autotune(hg_batch_plan* plan, const void* d_keys, const void* d_queries,
                            uint32_t* d_offsets, void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts,
                            void* d_ws, size_t ws_bytes, void* stream, uint32_t reps, float* h_best_ms);
hg_status hg_batch_run_plain(hg_batch_plan* plan, const void* d_keys, const void* d_queries,
                             uint32_t* d_offsets, void* d_csr_keys, uint32_t* d_csr_ids, uint32_t* d_counts,
                             void* d_ws, size_t ws_bytes, void* stream);

/* ------------------------------------------------ build, no allocation --
 * The paper has no counterpart of this entry point.  It is hg_build (V2)
 * for callers that cannot allocate device memory -- code running inside a
 * host runtime that owns all device memory and offers no allocator, or a
 * serving loop that bans cudaMalloc/cudaFree because they can synchronise
 * the device.  Inputs and outputs are still the caller's; the scratch space
 * is a fixed device array inside the library, hg_static_scratch_bytes()
 * bytes (8 MiB) per GPU that loads the library, held until the process exits.
 *   Same arguments and results as hg_build, without the workspace.
 *   Requests whose V2 plan needs more scratch than the array holds (more
 *   than hg_static_scratch_bytes() from hg_build_workspace_size; with the
 *   automatic bin size, cfg->bin_shift = 0, up to 2^18 keys always fit for
 *   V <= 2^29 with uint32 keys and V <= 2^28 with uint64 keys) return
 *   HG_ERR_WORKSPACE_TOO_SMALL;
 *   cfg->algo == HG_ALGO_V1 returns HG_ERR_UNSUPPORTED.
 *   The first call on a device looks up the array's device address; make it
 *   before any stream capture (a first call inside a capture returns
 *   HG_ERR_UNSUPPORTED).  Calls on a stream that is not capturing look the
 *   address up again, so a device reset between calls is harmless.  All
 *   calls share the one array and it keeps the last call's contents: calls
 *   whose GPU work overlaps race, so serialise them (one stream, or
 *   host-side ordering).
 * hg_static_scratch_status: the device status word the last build left in
 *   the array (HG_OK, or HG_ERR_TIMEOUT / HG_ERR_OVERFLOW when the table is
 *   not valid).  Synchronises `stream` first; allocates nothing.  The next
 *   build clears it. */
size_t hg_static_scratch_bytes(void);
hg_status hg_build_static_scratch(const hg_config* cfg, const void* d_keys, const uint32_t* d_ids,
                                  uint64_t n, uint32_t* d_offsets, void* d_csr_keys,
                                  uint32_t* d_csr_ids, void* stream);
hg_status hg_static_scratch_status(void* stream);

/* --------------------------------------------------------------- status --
 * Device status word of a workspace (HG_OK when no device-side error was
 * recorded).  Synchronises `stream` first.  hg_workspace_clear resets it. */
hg_status hg_workspace_status(const void* d_ws, void* stream);
hg_status hg_workspace_clear(void* d_ws, void* stream);
const char* hg_status_string(hg_status s);
const char* hg_version(void);

/* ---------------------------------------------------------------- trace --
 * Per-kernel timing.  While enabled, every kernel the library launches is
 * bracketed by two CUDA events recorded on the launch stream.
 * hg_profile_read synchronises on the recorded events and returns the number
 * of distinct kernels; for the first max_entries of them it fills
 * names[i] (static strings owned by the library), total_ms[i] (summed
 * event-to-event time) and launches[i].  Any output pointer may be NULL.
 * Returns -1 if an event query failed.  hg_profile_reset drops the records. */
void hg_profile_enable(int on);
void hg_profile_reset(void);
int hg_profile_read(int max_entries, const char** names, double* total_ms, uint64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* HG_H */
