/*
 * aot.h - C ABI of the GB300 AOT triangle engine (libaot.so).
 *
 * AOT (adaptive orientation triangle listing) lists every triangle of an
 * undirected simple graph exactly once (problem statement of Sec. 2.1) with
 * the edge iterator of Algorithm 3: the graph is oriented along a global
 * order eta (Sec. 1, Sec. 2.2), and each oriented edge <u,v> is charged to
 * the endpoint with the larger out-degree, whose out-neighbour index H is
 * probed by the out-list of the other endpoint (Sec. 3.1, Sec. 3.2), for
 * Theta(sum over <u,v> of min{deg+(u), deg+(v)}) work (Sec. 3.2).
 *
 * Conventions shared by every entry point
 *  - Pointers named d_* are DEVICE pointers (the current CUDA device); h_*
 *    are HOST pointers.  Vertex ids are int32 in [0, n).
 *  - Ownership: the caller owns every buffer.  The library never calls
 *    cudaMalloc or cudaFree; sizes of the device workspaces it needs are
 *    reported by the *_workspace_size queries, and the workspace must stay
 *    alive and untouched while a graph handle that points into it is used.
 *    The only host allocation is the small aot_graph handle.
 *  - Streams: every call is ordered on the given stream (NULL = legacy
 *    default stream).  A call that returns a host value (h_*) synchronises
 *    that stream before it returns.
 *  - Errors: every entry point returns an aot_status and never aborts or
 *    traps.  Bad input found on the device (a vertex id outside [0, n))
 *    raises a device error word that the call reads back before returning.
 *    After AOT_ERR_CUDA the CUDA context may be unusable.
 *  - Thread safety: a graph handle must not be used by two host threads at
 *    once; distinct handles are independent.
 */
#ifndef AOT_H
#define AOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so that this header does not need
 * the CUDA runtime headers. */
typedef struct CUstream_st* aot_stream_t;

typedef enum {
  AOT_OK = 0,
  AOT_ERR_INVALID_ARG = 1,  /* NULL pointer, negative size, unknown flag   */
  AOT_ERR_VERTEX_RANGE = 2, /* an input id lies outside [0, n)             */
  AOT_ERR_OVERFLOW = 3,     /* a size exceeds the index types (see below)  */
  AOT_ERR_WORKSPACE = 4,    /* workspace too small or not 256-byte aligned */
  AOT_ERR_CUDA = 5,         /* a CUDA runtime call failed                  */
  AOT_ERR_TIMEOUT = 6,      /* a bounded device wait ran out               */
  AOT_ERR_DEVICE_CHECK = 7, /* a device-side consistency check failed      */
  AOT_ERR_NOT_READY = 8     /* e.g. learned routing without router weights */
} aot_status;

/* How oriented edges are assigned to intersection variants.  The output never
 * depends on the route: every variant finds the same triangles. */
typedef enum {
  AOT_ROUTE_PLAIN = 0,   /* Algorithm 3: every edge probes its pivot's index */
  AOT_ROUTE_LEARNED = 1, /* the MLP router chooses a variant per edge        */
  AOT_ROUTE_PROBE = 2,   /* fixed: pivot index probe (same as PLAIN)         */
  AOT_ROUTE_MERGE = 3,   /* fixed: warp merge of the two sorted lists        */
  AOT_ROUTE_BSEARCH = 4, /* fixed: binary search of each walked entry        */
  AOT_ROUTE_RANDOM = 5   /* test only: seeded random variant per edge        */
} aot_route;

/* Orientation flags (aot_orient).  The global order eta of Sec. 1: */
#define AOT_ETA_DEG_DESC 0x0u /* degree non-increasing, ties by smaller id (default) */
#define AOT_ETA_DEG_ASC 0x1u  /* degree non-decreasing, ties by smaller id           */
/* The degeneracy order that kClist orients by (Sec. 2.3, Algorithm 2), by
 * peeling level by level: at level k every round removes all remaining
 * vertices of current degree <= k at once, and k rises to the smallest
 * remaining degree when none is left; eta = (removal round, id).  Every
 * vertex then has at most its core number of later neighbours.  Not
 * combinable with AOT_ETA_DEG_ASC. */
#define AOT_ETA_DEGENERACY 0x20u
#define AOT_FLAG_NO_LIST 0x2u /* size the workspace without the listing arrays      */
/* Ablations of Sec. 4.2 ("More on AOT") and the charging of the baselines
 * (Sec. 2.2, Sec. 2.3); counts and per-vertex counts never change:
 *  AOT_FLAG_NO_CLIP      a negative item walks all of N+(u), as Algorithm 3
 *                        prints it, instead of only the part after v.
 *  AOT_FLAG_LOCAL_RANDOM AOT-randomOrder: every out-list in one fixed
 *                        pseudo-random order (a bijection of the head rank)
 *                        instead of the eta order; implies AOT_FLAG_NO_CLIP.
 *                        Hubs then run on the global-bitmap path (hub_mode 1)
 *                        whatever the tuning; only AOT_ROUTE_PLAIN and
 *                        AOT_ROUTE_PROBE are accepted, and aot_list,
 *                        aot_graph_features and the merge / binary-search
 *                        cost recording return AOT_ERR_INVALID_ARG.
 *  AOT_FLAG_TAIL_PIVOT   no adaptive orientation: every edge <u,v> is an item
 *                        of its tail u walking all of N+(v).  With the probe
 *                        route this is the work of kClist (Algorithm 2,
 *                        sum of deg+(v)); with AOT_ROUTE_MERGE that of CF
 *                        (Algorithm 1, sum of deg+(u) + deg+(v)). */
#define AOT_FLAG_NO_CLIP 0x4u
#define AOT_FLAG_LOCAL_RANDOM 0x8u
#define AOT_FLAG_TAIL_PIVOT 0x10u

/* Size limits: n < 2^31, num_edges < 2^40, oriented edges m < 2^32.  Larger
 * inputs return AOT_ERR_OVERFLOW. */

typedef struct aot_graph aot_graph; /* opaque host handle */

/* Human-readable name of a status code (static string, never NULL). */
const char* aot_status_string(aot_status status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int aot_version(void);

/* Device workspace bytes that aot_orient needs for an input of num_edges
 * pairs over num_vertices ids with the given flags (an upper bound: it does
 * not depend on the edge values). */
aot_status aot_orient_workspace_size(int64_t num_edges, int32_t num_vertices, uint32_t flags,
                                     size_t* bytes);

/* Orientation (Algorithm 3, first step; local order of Sec. 3.2):
 *  1. cleanup: drop self-loops, merge duplicate and reversed pairs (the input
 *     is treated as an undirected simple graph, Sec. 2.1);
 *  2. eta: rank vertices by degree (flags), ties by smaller id (footnote of
 *     the correctness argument in Sec. 3.2);
 *  3. oriented out-CSR in rank space, every out-list sorted by eta;
 *  4. the work items of Algorithm 3: an edge <u,v> becomes a positive item of
 *     pivot u walking N+(v) when key(v) < key(u), else a negative item of
 *     pivot v walking the part of N+(u) after v (key = (deg+, rank));
 *  5. degree bins of the pivots for the intersection kernels.
 * d_src, d_dst: num_edges int32 endpoint pairs (any direction).
 * d_workspace: >= aot_orient_workspace_size bytes, 256-byte aligned.
 * On success *out receives a new handle (free it with aot_graph_destroy).
 * Synchronises s.  Errors: AOT_ERR_VERTEX_RANGE if an id is outside [0, n). */
aot_status aot_orient(const int32_t* d_src, const int32_t* d_dst, int64_t num_edges,
                      int32_t num_vertices, uint32_t flags, void* d_workspace, size_t ws_bytes,
                      aot_stream_t s, aot_graph** out);

/* Host-side facts of an oriented graph: n, m (= undirected simple edges =
 * oriented edges), W = summed walk length of Algorithm 3 (the work counter
 * of the Sec. 3.2 analysis, with negative walks clipped after the pivot),
 * S = summed deg+ of the pivots that own at least one item (index staging),
 * max_outdeg = max deg+.  Any pointer may be NULL. */
aot_status aot_graph_info(const aot_graph* g, int32_t* n, int64_t* m, uint64_t* work_w,
                          uint64_t* staged_s, int32_t* max_outdeg);

/* Work counters of an oriented graph (cost model of Sec. 2.2, Sec. 2.3 and
 * Sec. 3.2, for the graph's orientation flags):
 *  walk        W, the summed walk length of the work items (probe route);
 *  merge       W + sum over pivots of items(p) x deg+(p): the entries a
 *              merge of every item's walk with N+(p) reads (merge route);
 *  staged      S, as in aot_graph_info;
 *  positive    items whose pivot is the tail of their edge;
 *  items       all items (= m). */
typedef struct {
  uint64_t walk;
  uint64_t merge;
  uint64_t staged;
  uint64_t positive;
  uint64_t items;
} aot_costs;
aot_status aot_graph_costs(const aot_graph* g, aot_costs* out);

/* Copy the orientation into caller buffers (any pointer may be NULL):
 * d_perm[n] (eta position -> original id), d_rank[n] (original id -> eta
 * position), d_out_off[n+1] (uint32 offsets of the out-CSR, rank space),
 * d_out_adj[m] (uint32 heads, ascending inside each list; in the fixed
 * pseudo-random order with AOT_FLAG_LOCAL_RANDOM),
 * d_items[n] (uint32 number of work items per pivot), d_walk[n] (uint64
 * summed walk length per pivot).  Ordered on s (no sync). */
aot_status aot_graph_export(const aot_graph* g, int32_t* d_perm, int32_t* d_rank,
                            uint32_t* d_out_off, uint32_t* d_out_adj, uint32_t* d_items,
                            uint64_t* d_walk, aot_stream_t s);

/* Triangle count T (Sec. 5: listing solves counting).  Synchronises s. */
aot_status aot_count(aot_graph* g, aot_route route, uint64_t* h_total, aot_stream_t s);

/* Per-vertex counts t(v) = triangles containing v, written to d_counts[n]
 * (uint64, ORIGINAL ids; overwritten).  sum t(v) = 3T.  h_total may be NULL
 * (then the call does not synchronise). */
aot_status aot_count_per_vertex(aot_graph* g, aot_route route, uint64_t* d_counts,
                                uint64_t* h_total, aot_stream_t s);

/* Listing by count, exclusive scan, write.  Triangles are numbered in the
 * canonical order: (x,y,z) with eta(x) < eta(y) < eta(z), sorted by
 * (eta(x), eta(y), eta(z)).  This call writes triangles [cursor, cursor+k)
 * with k = min(cap, T - cursor) to d_out (3*cap int32, ORIGINAL ids, x y z
 * per triangle), and returns k in *h_written and cursor + k in *h_next (== T
 * when done).  The first call on a graph runs the count and scan passes; the
 * per-edge offsets are kept in the workspace for later chunks.  Needs a
 * workspace sized without AOT_FLAG_NO_LIST.  Synchronises s. */
aot_status aot_list(aot_graph* g, aot_route route, uint64_t cursor, int32_t* d_out,
                    uint64_t cap, uint64_t* h_written, uint64_t* h_next, aot_stream_t s);

/* Launch tuning of the intersection kernels.  Pivots are binned by deg+:
 * deg+ <= warp_max_outdeg -> one warp per pivot (hash table in the warp's
 * shared memory; warp_max_outdeg <= 64), deg+ <= cta_max_outdeg -> the CTA
 * bin (shared-memory hash table; cta_max_outdeg <= 8192; a CTA of
 * cta_threads threads per pivot, or a warp per pivot when cta_threads is
 * 32), larger -> hub path.  hub_mode 0: a shared-memory bitmap over eta ranks, swept one
 * segment of seg_bits ranks at a time (a multiple of 32 in [1024, 1572864])
 * by a CTA per (pivot, block of 1536 items), items with at least seg_long
 * entries walked by a warp (in rounds of 256 entries while at least seg_wide
 * entries remain, else of 128), shorter ones by a thread each; hub_mode 1:
 * global bitmaps of n bits, hub_bitmaps (1..32) hubs at a time, all CTAs
 * sharing their items.  cta_threads is a multiple of 32 in [32, 1024].
 * tile_bits (hub_mode 0): 0, or in [16, 31]: the hub tasks are handed out
 * tile by tile of the walked out-lists, a tile being the lists that fill
 * 2^tile_bits consecutive adjacency entries, so that the lists walked at the
 * same time stay in L2; 0 hands them out pivot by pivot.
 * seg_tail (hub_mode 0): in every segment after the first, a long item with
 * fewer than seg_tail entries left is walked by one thread instead of a warp
 * (its later visits are short); 0 keeps every long item warp-wide.
 * seg_threads (hub_mode 0): threads per CTA of the segmented bitmap kernel, a
 * multiple of 32 in [256, 1024]; with 512 and seg_bits <= 589824 two CTAs fit
 * one SM.
 * seg_hash (hub_mode 0): after the first segment, a pivot with at most
 * seg_hash entries of N+(p) left takes all its later segments in one pass:
 * those entries go to a two-choice cuckoo hash table of S slots in the
 * bitmap's shared memory (S the largest power of two <= seg_bits / 32), and
 * every item walks the rest of its list once; 0 sweeps every segment.  A
 * table that cannot be built (likely above S / 2 entries, certain above S)
 * falls back to the segments; the default fills at most 3/8 of S = 32768.
 * Built-in defaults: warp_max_outdeg 64, cta_max_outdeg 512, cta_threads 32,
 * hub_bitmaps 32, hub_mode 0, seg_bits 1310720, seg_long 128, seg_wide 512,
 * tile_bits 0, seg_tail 128, seg_threads 1024, seg_hash 12288.
 * Tuning never changes results, only speed. */
typedef struct {
  uint32_t warp_max_outdeg;
  uint32_t cta_max_outdeg;
  int32_t cta_threads;
  int32_t hub_bitmaps;
  int32_t hub_mode;
  uint32_t seg_bits;
  uint32_t seg_long;
  uint32_t seg_wide;
  uint32_t tile_bits;
  uint32_t seg_tail;
  int32_t seg_threads;
  uint32_t seg_hash;
} aot_tuning;

/* Work statistics of one pivot bin under the current tuning. */
typedef struct {
  uint64_t pivots; /* pivots with at least one item in this bin         */
  uint64_t items;  /* their work items (oriented edges)                 */
  uint64_t walk;   /* summed walk length of those items (part of W)     */
  uint64_t staged; /* summed deg+ of those pivots (index entries built) */
} aot_bin_stats;

/* Statistics of the three bins (warp, CTA, hub), in that order. */
aot_status aot_graph_bins(const aot_graph* g, aot_bin_stats out[3]);

/* Current tuning of a graph (defaults after aot_orient). */
aot_status aot_graph_get_tuning(const aot_graph* g, aot_tuning* t);

/* Set the tuning and re-bin the pivots (synchronises s).  Out-of-range values
 * return AOT_ERR_INVALID_ARG and leave the graph unchanged.  hub_bitmaps may
 * not exceed the value the workspace was sized for (32). */
aot_status aot_graph_set_tuning(aot_graph* g, const aot_tuning* t, aot_stream_t s);

/* ---- learned router (the build's addition; the paper has no learned part) ----
 * An 8 -> 64 -> 64 -> 3 perceptron (ReLU hidden layers) predicts, per work
 * item, the standardised log cost of the three variants (probe, merge, binary
 * search) from eight features of its oriented edge <u,v> (rank space, u < v):
 * log1p deg+(u), log1p deg+(v), log1p |{w in N+(u): w > v}|, log1p deg-(u),
 * log1p deg-(v), log1p deg(u), log1p deg(v), (v - u) / n.  AOT_ROUTE_LEARNED
 * keeps the probe of Algorithm 3 unless another variant's predicted cost is
 * lower by more than the model's margin.  Routing never changes results.
 *
 * Model buffer (AOT_MLP_MODEL_BYTES, device memory, 16-byte aligned):
 *   float in_mean[8], in_std[8]    feature standardisation  (bytes   0.. 63)
 *   float out_mean[4], out_std[4]  output de-standardisation (bytes 64.. 95)
 *   float margin, reserved[7]                                (bytes 96..127)
 *   bfloat16 params[4931] from byte 128: W1[64][8], b1[64], W2[64][64],
 *   b2[64], W3[3][64], b3[3] (row-major [out][in]).
 * Numerics: bf16 inputs, parameters and hidden activations (round to nearest
 * even), fp32 accumulation, fp32 outputs. */
#define AOT_MLP_PARAMS 4931
#define AOT_MLP_MODEL_BYTES 10240

/* Attach (or detach with NULL) router parameters used by AOT_ROUTE_LEARNED.
 * The buffer stays owned by the caller and must outlive its use. */
aot_status aot_graph_set_router(aot_graph* g, const void* d_model);

/* Router that aot_orient attaches to every new graph (process-wide; NULL:
 * none, the initial state).  Batches use it for AOT_ROUTE_LEARNED. */
aot_status aot_set_default_router(const void* d_model);

/* The eight raw (unstandardised) features of every oriented edge, written to
 * d_feat[m][8] (float, rows in out-CSR edge order).  Ordered on s. */
aot_status aot_graph_features(aot_graph* g, float* d_feat, aot_stream_t s);

/* Timing capture: run the work items through one variant (0 probe, 1 merge,
 * 2 binary search) with per-item clock64 timing and write the cycles of each
 * oriented edge (its walk plus its share of index staging) to d_cycles[m]
 * (CSR edge order; 0 for items not run).  The probe variant runs every item;
 * the other two only the items whose hash has its low sample_log2 bits zero
 * (sample_log2 = 0: all).  These are the router's training labels.
 * Synchronises s. */
aot_status aot_graph_record_costs(aot_graph* g, int32_t variant, int32_t sample_log2,
                                  uint32_t* d_cycles, aot_stream_t s);

/* Network output y[n][3] (standardised log costs) for raw features x[n][8]
 * (the kernel standardises them with the model's in_mean / in_std).  Uses the
 * tensor-core inference kernel.  Ordered on s. */
aot_status aot_mlp_forward(const void* d_model, const float* d_x, int64_t n, float* d_y, aot_stream_t s);

/* Workspace of aot_mlp_train_step for a batch size. */
aot_status aot_mlp_train_workspace_size(int32_t batch, size_t* bytes);

/* One training step on a batch: forward, loss sum (y - t)^2 / batch with
 * standardised targets d_t[batch][3], backward; if lr > 0 one Adam step
 * (beta 0.9 / 0.999, eps 1e-8; step counts from 1) of the fp32 master copy
 * d_master[4931] with moments d_m1, d_m2, whose bf16 rounding is written back
 * into the model.  d_grad_out (optional, 4931 floats) receives the gradient
 * in parameter order; h_loss (optional) the loss (then s is synchronised). */
aot_status aot_mlp_train_step(void* d_model, float* d_master, float* d_m1, float* d_m2, int32_t step,
                              float lr, const float* d_x, const float* d_t, int32_t batch, void* d_ws,
                              size_t ws_bytes, float* d_grad_out, float* h_loss, aot_stream_t s);

/* ---- launch accounting and profiling (no effect on results) ---- */

/* Number of kernels this library has launched in this process. */
unsigned long long aot_kernel_launches(void);

/* One profiled kernel: its name, launches and summed device time. */
typedef struct {
  char name[64];
  uint64_t launches;
  double total_ms;
} aot_profile_entry;

/* Start recording: every later launch is bracketed by a pair of CUDA events
 * on its stream (a previous recording is discarded). */
aot_status aot_profile_begin(void);

/* Stop recording, wait for the recorded events, and aggregate by kernel name:
 * up to cap entries are written to out, *count receives the number of
 * distinct kernels. */
aot_status aot_profile_end(aot_profile_entry* out, int32_t cap, int32_t* count);

/* ---- counting without device allocation ----
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory (no cudaMalloc allowed where they run,
 * or a memory budget owned by a host framework that only hands out its input
 * and output buffers) and therefore cannot supply the workspace the other
 * entry points need.  Its scratch memory is a fixed __device__ array of
 * AOT_STATIC_SCRATCH_BYTES inside libaot.so, held by every GPU that loads the
 * library until the process exits.
 *
 * Same result as aot_orient(..., AOT_FLAG_NO_LIST, ...) followed by
 * aot_count_per_vertex (or aot_count when d_counts is NULL) with the plain
 * route: *h_total = T and, if d_counts != NULL, d_counts[n] = t(v) (uint64,
 * original ids).  Synchronises s.  The call makes no cudaMalloc / cudaFree
 * and uses no allocating library routine.
 * Limit: the workspace that aot_orient_workspace_size reports for
 * (num_edges, num_vertices, AOT_FLAG_NO_LIST) must fit the array, else the
 * call returns AOT_ERR_OVERFLOW and does nothing (e.g. 262,144 pairs over
 * 16,384 vertices fit in 9.4 MB; 1,200,000 pairs over 65,536 vertices need
 * 42.0 MB and are rejected).
 * The first call on a device (run with that device current) looks up the
 * array's device address and caches it: make that first call before any
 * stream capture.  The cached address does not survive cudaDeviceReset: do
 * not call this entry point on a device after resetting it.  All calls share
 * the array, which keeps the last call's contents (each call re-initialises
 * what must start at zero): calls that overlap on the GPU race, so serialise
 * them.  A call that fails after queuing kernels synchronises s before it
 * returns. */
#define AOT_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)
aot_status aot_count_per_vertex_static(const int32_t* d_src, const int32_t* d_dst,
                                       int64_t num_edges, int32_t num_vertices,
                                       uint64_t* d_counts, uint64_t* h_total, aot_stream_t s);

/* Tuning that aot_orient gives every new graph (process-wide; the built-in
 * defaults until set).  Invalid values return AOT_ERR_INVALID_ARG. */
aot_status aot_set_default_tuning(const aot_tuning* t);
aot_status aot_get_default_tuning(aot_tuning* t);

/* Autotuner: coordinate search over the bin thresholds (CTA-hash cutoff,
 * warp cutoff), CTA size, the segmented walk's short/long and 128/256-entry
 * thresholds, the bitmap segment width and the walked-list tile size, timing each candidate on this
 * graph with CUDA events (best of reps) in mode 0 (count) or 1 (per-vertex
 * count); a candidate replaces the current tuning only when it is at least
 * 1 % faster.  The chosen tuning is set on the graph and returned in
 * *best_out (may be NULL) with its time in *h_best_ms (may be NULL).
 * Synchronises s.  Results never change, only speed. */
aot_status aot_tune(aot_graph* g, int32_t mode, int32_t reps, aot_tuning* best_out,
                    float* h_best_ms, aot_stream_t s);

/* ---- batches of independent graphs ---- */

/* Device workspace for aot_batch (an upper bound for these totals). */
aot_status aot_batch_workspace_size(int64_t total_edges, int32_t num_graphs, int64_t total_vertices,
                                    size_t* bytes);

/* Per-graph triangle counts and per-vertex counts of num_graphs independent
 * graphs in one pass.  Graph g owns the pairs [d_edge_ofs[g], d_edge_ofs[g+1])
 * of d_src / d_dst, with LOCAL ids in [0, d_nv[g]) (int64 offsets, G+1 of
 * them, d_edge_ofs[0] = 0, d_edge_ofs[G] = total_edges; total_vertices =
 * sum of d_nv).  Output: d_tri[g] (uint64) and d_vcount[voff[g] + v] = t(v)
 * (uint64) with voff the exclusive prefix of d_nv.  The batch is processed as
 * the disjoint union of its graphs (one orientation, one set of persistent
 * bin kernels, the process default tuning); the counting phase is captured
 * into a CUDA graph and launched when s is a created stream that is not
 * already capturing (else its kernels are launched on s directly).  Each
 * host thread keeps its last instantiated graph per device and updates it in
 * place for the next call whose captured kernels match (the orientation, with
 * its host synchronisations, always runs outside the graph).  Synchronises s.
 * Errors: AOT_ERR_INVALID_ARG for inconsistent offsets or counts,
 * AOT_ERR_VERTEX_RANGE if an id lies outside its own graph. */
aot_status aot_batch(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_edge_ofs,
                     const int32_t* d_nv, int32_t num_graphs, int64_t total_edges,
                     int64_t total_vertices, aot_route route, uint64_t* d_tri, uint64_t* d_vcount,
                     void* d_ws, size_t ws_bytes, aot_stream_t s);

/* Autotuner for batches: builds the union graph of the batch exactly as
 * aot_batch does and runs aot_tune on it in per-vertex mode (reps timings
 * per candidate); the best tuning is returned in *best_out (hub_mode 0) and
 * its time in *h_best_ms (may be NULL).  Install it with
 * aot_set_default_tuning before aot_batch, which takes the default tuning.
 * Arguments as for aot_batch; the same workspace size.  Synchronises s. */
aot_status aot_batch_tune(const int32_t* d_src, const int32_t* d_dst, const int64_t* d_edge_ofs,
                          const int32_t* d_nv, int32_t num_graphs, int64_t total_edges,
                          int64_t total_vertices, int32_t reps, aot_tuning* best_out,
                          float* h_best_ms, void* d_ws, size_t ws_bytes, aot_stream_t s);

/* Free the host handle (the workspace stays with the caller). */
aot_status aot_graph_destroy(aot_graph* g);

#ifdef __cplusplus
}
#endif
#endif /* AOT_H */
