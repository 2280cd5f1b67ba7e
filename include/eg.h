/*
 * eg.h -- C ABI of the GB300 extremum-graph library.
 *
 * The library computes the extremum graph (maximum graph by default) of a
 * scalar field (float32 by default; 8- to 64-bit integers and float64 through
 * eg_compute_typed, Sec. 5) sampled on a d-dimensional regular grid, 1 <= d <= 5,
 * under the Freudenthal triangulation of the grid (Sec. 3.2, Algorithm 1), as
 * defined in Sec. 2 of Ande, Subhash & Natarajan, "Tachyon: efficient shared
 * memory parallel computation of extremum graphs":
 *
 *   nodes   the maxima (upper link empty) and the (n-1)-saddles (upper link
 *           with two or more connected components), Table 1;
 *   arcs    (s, m) iff a gradient path that leaves saddle s through one of its
 *           upper-link components ends at maximum m (Sec. 3.4, Algorithm 2:
 *           UpperLinkRep, then follow the gradient = the highest upper-link
 *           vertex, Sec. 3.3);
 *   labels  for every vertex, the maximum its gradient path reaches (the
 *           descending manifold of that maximum, i.e. the Morse decomposition).
 *
 * Ties are broken by simulation of simplicity (Sec. 3.3): vertex w is higher
 * than v iff f[w] > f[v], or f[w] == f[v] and w > v (linear index).  Values are
 * compared exactly in the field's own element type.  -0.0 equals +0.0;
 * infinities are ordinary values; NaN is rejected.
 *
 * Grid layout: axis 0 is fastest; vertex index v = x0 + n0*(x1 + n1*(x2 + ..)).
 * Every vertex id in and out of the library is this linear index (uint32), so a
 * field holds at most 2^32 - 1 vertices.
 *
 * Conventions for every call:
 *   - Status codes, never exceptions; the library never aborts the process.
 *   - "device" pointers are CUDA device pointers on the handle's device;
 *     "host" pointers are ordinary host memory (pinned or pageable).
 *   - Streams are passed as void* (a cudaStream_t; NULL = the legacy default
 *     stream).  Calls enqueue work on the stream and return; the results of a
 *     computation are ready once eg_get_graph returns EG_OK.
 *   - The library owns every intermediate and result device buffer until
 *     eg_release; the caller owns its inputs and its host output buffers.
 *   - A handle may be used from several host threads; calls on one handle are
 *     serialised internally.
 */
#ifndef EG_H
#define EG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define EG_API __attribute__((visibility("default")))
#else
#define EG_API
#endif

#define EG_MAX_DIM 5

typedef enum eg_status {
    EG_OK = 0,
    EG_ERR_ARG = 1,            /* bad dimension, extent, pointer, size or id      */
    EG_ERR_NAN = 2,            /* the field holds a NaN                           */
    EG_ERR_OOM = 3,            /* device or pinned host memory exhausted          */
    EG_ERR_CUDA = 4,           /* a CUDA runtime call failed                      */
    EG_ERR_NOT_CONVERGED = 5,  /* gradient-path resolution exceeded its bound     */
    EG_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up              */
    EG_ERR_BUSY = 7,           /* admission refused: not enough free device memory */
    EG_ERR_INTERNAL = 8        /* a device-side consistency check failed          */
} eg_status;

/* Element types of a field (Sec. 5: 8-, 16-, 32- and 64-bit signed and
 * unsigned integers, 32- and 64-bit floats). */
typedef enum eg_dtype {
    EG_DTYPE_F32 = 0,
    EG_DTYPE_F64 = 1,
    EG_DTYPE_I8 = 2,
    EG_DTYPE_U8 = 3,
    EG_DTYPE_I16 = 4,
    EG_DTYPE_U16 = 5,
    EG_DTYPE_I32 = 6,
    EG_DTYPE_U32 = 7,
    EG_DTYPE_I64 = 8,
    EG_DTYPE_U64 = 9
} eg_dtype;
#define EG_DTYPE_COUNT 10

/* eg_field_desc.flags bits 16..19: the field's element type (an eg_dtype;
 * 0 = float32), e.g. flags = EG_FLAG_DTYPE(EG_DTYPE_U8). */
#define EG_FLAG_DTYPE(t) ((uint32_t)(t) << 16)
#define EG_FLAG_DTYPE_MASK 0xf0000u

/* eg_config.flags */
#define EG_FLAG_MINIMUM_GRAPH 0x1u  /* minimum graph: the same order reversed (Sec. 2) */
#define EG_FLAG_NO_LABELS     0x2u  /* do not keep per-vertex labels in the result    */
#define EG_FLAG_NO_GRAPH      0x4u  /* eg_batch_submit: launch the steps directly
                                       instead of replaying captured CUDA graphs    */
#define EG_FLAG_PATHS         0x8u  /* also keep the arc geometry (eg_get_paths)    */
#define EG_FLAG_NO_FUSED      0x10u /* eg_compute(_typed): small fields take the
                                       general launches, not the fused kernel       */

/* Tuning knobs.  Zero in any field means "library default" (or the value a
 * previous eg_autotune chose for this handle).  The neighbourhood halo is one
 * vertex wide by construction (Algorithm 1 offsets are in {-1,0,1}^d) and is
 * not a knob. */
typedef struct eg_config {
    uint32_t flags;
    int32_t classify_rows;    /* 2D/3D classification tile: grid rows per tile (brick)   */
    int32_t classify_planes;  /* planes one work item of the classifier marches over     */
    int32_t resolve_walks;    /* gradient walks each resolver thread keeps in flight:
                                 2, 4 or 8                                               */
    int32_t persistent_ctas;  /* CTAs per SM of the persistent classifier work queue     */
    int32_t reserved[3];
} eg_config;

typedef struct eg_ctx *eg_handle;
typedef uint64_t eg_result_id;

/* One field of a batch.  field: device array of the element type named in
 * flags (float32 unless EG_FLAG_DTYPE says otherwise), caller-owned, valid
 * until the batch's results are read; extents[k] >= 1 for k < d. */
typedef struct eg_field_desc {
    const void *field;
    int32_t d;
    int32_t flags;           /* per-field EG_FLAG_* (ORed with the handle's)        */
    int64_t extents[EG_MAX_DIM];
} eg_field_desc;

/* Result description.  eg_get_graph always fills the counts; every array
 * pointer that is non-NULL receives a copy (host memory, caller-allocated with
 * at least the counted size).  Call once with NULL arrays to learn the sizes. */
typedef struct eg_graph {
    int32_t d;
    int32_t dtype;           /* element type of the field and of max_val, sad_val */
    int64_t extents[EG_MAX_DIM];
    int64_t n_vertices;
    int64_t n_maxima;        /* M                                                   */
    int64_t n_saddles;       /* S                                                   */
    int64_t n_paths;         /* P = sum of beta0+ over saddles (gradient paths)     */
    int64_t n_arcs;          /* A = number of unique (saddle, maximum) pairs        */
    uint32_t *maxima;        /* [M]   ascending vertex ids                          */
    void *max_val;           /* [M]   f at each maximum (exact copy, element type
                                      dtype: eg_dtype_size(dtype) bytes each)        */
    uint32_t *saddles;       /* [S]   ascending vertex ids                          */
    uint8_t *sad_beta0;      /* [S]   upper-link components of each saddle          */
    void *sad_val;           /* [S]   f at each saddle (exact copy, element type dtype) */
    uint64_t *row_ptr;       /* [S+1] CSR row offsets into col                      */
    uint32_t *col;           /* [A]   maxima of each saddle, ascending, unique      */
    uint32_t *labels;        /* [N]   maximum reached from every vertex             */
} eg_graph;

/* Create a handle on CUDA device `device`.  cfg may be NULL (defaults).
 * Errors: EG_ERR_ARG (bad device or out == NULL), EG_ERR_CUDA. */
EG_API eg_status eg_create(eg_handle *out, int device, const eg_config *cfg);

/* Wait for all work of the handle, free every buffer it owns (results
 * included) and the handle itself.  NULL is accepted. */
EG_API eg_status eg_destroy(eg_handle h);

/* Extremum graph of one field (Sec. 3.3 classification, Sec. 3.4 arcs).
 * field: device float32[N], caller-owned, must stay valid until the result is
 * read; d in 1..5; extents[0..d-1] >= 1, product < 2^32; stream: cudaStream_t.
 * Enqueues classification, path resolution and graph assembly on `stream`; the
 * call itself waits only for the node counts (to size the result buffers).
 * A field of at most 65,536 vertices (eg_compute and eg_compute_typed,
 * without EG_FLAG_PATHS) does not wait at all: its result buffers are sized
 * by bounds (maxima and saddles at most N, arc ends at most N times the most
 * components an upper link can have), and a device-side error (EG_ERR_NAN,
 * EG_ERR_TIMEOUT) is then returned by the first call that reads the result.
 * On success *out names the result.
 * Errors: EG_ERR_ARG, EG_ERR_NAN (field holds NaN), EG_ERR_OOM, EG_ERR_CUDA. */
EG_API eg_status eg_compute(eg_handle h, const float *field, int d, const int64_t *extents,
                            void *stream, eg_result_id *out);

/* As eg_compute, for a field of element type `dtype` (an eg_dtype): device
 * array of N elements of eg_dtype_size(dtype) bytes, naturally aligned.
 * Values are compared exactly in that type (Sec. 3.3's order; Sec. 5's list
 * of types); the value copies of the result (eg_graph.max_val, sad_val) have
 * that type too.  Integers of at most 16 bits are exact in float32 with their
 * order and ties kept: they are widened to float32 on the device and take the
 * float32 kernels.  32- and 64-bit integers and float64 take a classifier
 * that compares them in their own type.
 * Errors: as eg_compute, plus EG_ERR_ARG for an unknown dtype or a misaligned
 * field; EG_ERR_NAN for a float64 NaN. */
EG_API eg_status eg_compute_typed(eg_handle h, const void *field, int dtype, int d, const int64_t *extents,
                                  void *stream, eg_result_id *out);

/* Size in bytes of one element of type `dtype`, 0 if dtype is unknown. */
EG_API size_t eg_dtype_size(int dtype);

/* As eg_compute, for a field in HOST memory: the host-to-device copy of the
 * field is enqueued on `stream` first (through the handle's pinned staging
 * buffer when the field is pageable).  field must stay valid until the call
 * returns. */
EG_API eg_status eg_compute_host(eg_handle h, const float *field, int d,
                                 const int64_t *extents, void *stream, eg_result_id *out);

/* Many fields of uneven sizes and dimensions in one launch per step: the
 * persistent classifier drains a device work queue of (field, tile) items and
 * every other step covers all fields' bricks in one grid.  The steps are
 * captured once per batch layout (shapes, flags, configuration) into CUDA
 * graphs and replayed for every later batch with the same layout; the
 * per-field pointers reach the kernels through a descriptor table uploaded by
 * the graph itself.  out_ids[n] receives one
 * result per field, in order.  Field pointers must stay valid until their
 * results are read.  Errors as eg_compute; on error no result is created. */
EG_API eg_status eg_batch_submit(eg_handle h, const eg_field_desc *fields, int n, void *stream,
                                 eg_result_id *out_ids);

/* Wait for the result and copy it into the caller's host buffers (see
 * eg_graph).  Device-side failures detected during the computation (NaN,
 * unbounded path, queue timeout) are reported here.
 * Errors: EG_ERR_ARG (unknown id), plus any deferred device status. */
EG_API eg_status eg_get_graph(eg_handle h, eg_result_id id, eg_graph *out);

/* Same as eg_get_graph but fills the array pointers with the library-owned
 * DEVICE buffers instead of copying (valid until eg_release). */
EG_API eg_status eg_get_graph_device(eg_handle h, eg_result_id id, eg_graph *out);

/* eg_get_graph_device for n results in one call (one lock, one pass): out[i]
 * for ids[i]; status[i] (may be NULL) receives each result's status.  Returns
 * EG_OK, or the first failing result's status (the others are still filled).
 * Errors: EG_ERR_ARG (n < 0, or NULL arrays with n > 0). */
EG_API eg_status eg_get_graphs_device(eg_handle h, const eg_result_id *ids, int n, eg_graph *out,
                                      int32_t *status);

/* Arc geometry (Algorithm 2, Sec. 3.4): for every saddle, in the order of
 * eg_graph.saddles, and every component of its upper link, in ascending order
 * of its highest vertex (UpperLinkRep), the path of vertex ids
 *   s, rep, gradient(rep), gradient(gradient(rep)), ..., m
 * where m is the maximum reached (the arc end) and gradient(v) is v's highest
 * neighbour.  There are n_paths paths (eg_graph.n_paths); path p is
 * path_vtx[path_ptr[p] .. path_ptr[p + 1]).  Only results computed with
 * EG_FLAG_PATHS (handle configuration or eg_field_desc.flags) carry it; the
 * geometry is gathered between classification and resolution and adds two
 * host round trips to that computation (fields with paths never replay a
 * captured graph).
 * Call with path_ptr == path_vtx == NULL to get *n_path_vertices; then
 * path_ptr must hold n_paths + 1 entries and path_vtx *n_path_vertices, both
 * caller-owned host memory.
 * Errors: EG_ERR_ARG (unknown id, no geometry kept, NULL n_path_vertices),
 * plus any deferred device status as eg_get_graph. */
EG_API eg_status eg_get_paths(eg_handle h, eg_result_id id, uint64_t *path_ptr, uint32_t *path_vtx,
                              uint64_t *n_path_vertices);

/* Arc bundling (Sec. 3.5) on a finished result: when several saddles connect
 * the same two maxima, only the highest of them (value in the field's own
 * element type, then index; the lowest for a minimum graph) stands for that
 * pair.  keep[i] (caller-owned
 * host memory, n_saddles bytes, in the order of eg_graph.saddles) is set to
 * 1 when saddle i stands for at least one pair of its arc ends, or connects
 * no pair (all its arcs end at one maximum), else 0; the bundled graph is the
 * kept saddles with their arcs.  Runs on the device (a hash table over the
 * pairs of maxima) on the handle's own stream and waits for it.
 * Errors: EG_ERR_ARG (unknown id, NULL keep with saddles present),
 * EG_ERR_OOM, EG_ERR_INTERNAL (table overflow; cannot happen), plus any
 * deferred device status as eg_get_graph. */
EG_API eg_status eg_get_bundled(eg_handle h, eg_result_id id, uint8_t *keep);

/* Persistence-directed cancellation (Sec. 3.5) on a finished float32 result,
 * with persistence threshold tau.  The cost of a saddle is the difference in
 * value between it and the second highest maximum its arcs currently reach
 * (for a simple saddle: the lower of its two maxima; the lowest for a minimum
 * graph), computed in float32 (0 for equal values).  Saddles are cancelled in
 * increasing order of (current cost, vertex id) while that cost is at most
 * tau; cancelling a saddle merges every maximum it reaches except the highest
 * (the survivor) into the survivor, so arcs that ended at a merged maximum
 * end at the survivor afterwards.  A saddle whose arcs all reach one maximum
 * is never cancelled.  Where a merge lowers the cost of a multi-saddle (two of
 * its maxima merge), the lower cost counts at once: the paper assumes costs
 * never fall and leaves that case open.  The order of cancellations is the
 * paper's serial queue; it runs on the device in data-parallel rounds that
 * cancel, at once, every saddle that no neighbouring saddle could precede.
 * alive: caller-owned host uint8[n_saddles], in the order of eg_graph.saddles,
 *        1 = the saddle stays in the simplified graph, 0 = cancelled;
 * survivor: caller-owned host uint32[n_maxima], in the order of
 *        eg_graph.maxima: the vertex id of the maximum it was merged into
 *        (itself when it survives);
 * n_cancelled, n_rounds (may be NULL): cancelled saddles, device rounds run.
 * The simplified graph is the kept saddles with the survivors of their arc
 * ends.  Runs on the handle's own stream and waits for it.
 * The rounds run in one cooperative launch whose grid barriers wait at most
 * about a second each (EG_ERR_TIMEOUT if one gives up).
 * Errors: EG_ERR_ARG (unknown id, NaN tau, a result that is not float32,
 * NULL outputs with saddles or maxima present), EG_ERR_OOM, EG_ERR_TIMEOUT,
 * EG_ERR_INTERNAL, plus any deferred device status as eg_get_graph. */
EG_API eg_status eg_get_cancelled(eg_handle h, eg_result_id id, float tau, uint8_t *alive, uint32_t *survivor,
                                  int64_t *n_cancelled, int32_t *n_rounds);

/* Autotuner: time candidate values/* Autotuner: time candidate values of every eg_config knob on this batch of
 * fields (coordinate descent over the knobs, each candidate a full run of the
 * pipeline timed with CUDA events on `stream`), keep the fastest in the
 * handle's configuration for later calls, and return it in *best (may be
 * NULL).  Results of the trial runs are discarded.  Errors as eg_batch_submit. */
EG_API eg_status eg_autotune(eg_handle h, const eg_field_desc *fields, int n, void *stream, eg_config *best);

/* Free a result's buffers (they return to the handle's pool). */
EG_API eg_status eg_release(eg_handle h, eg_result_id id);

/* Device memory the library would need to compute a field of this shape
 * (result buffers excluded), for admission control.  Returns 0 on bad input. */
EG_API uint64_t eg_workspace_bytes(int d, const int64_t *extents);

/* Free and total device memory seen by the handle's device, plus the bytes the
 * handle currently holds (pool + live results). */
EG_API eg_status eg_mem_info(eg_handle h, uint64_t *free_bytes, uint64_t *total_bytes,
                             uint64_t *held_bytes);

/* Step timing.  With timing enabled, every computation records CUDA events on
 * its own stream around each step; eg_step_times then returns, once the
 * result is complete, the device time in milliseconds of
 *   ms[0] classification (steps a+c), ms[1] path resolution (step b),
 *   ms[2] graph assembly (steps d+e), ms[3] the whole computation.
 * For a batch every field of the submission reports the batch's times.  A
 * small field computed by the fused kernel (every step in one launch)
 * reports that launch as ms[0] and ms[3], with ms[1] = ms[2] = 0.
 * Errors: EG_ERR_ARG (unknown id, or timing was off for that computation). */
EG_API eg_status eg_set_timing(eg_handle h, int enable);
EG_API eg_status eg_step_times(eg_handle h, eg_result_id id, float ms[4]);

/* Largest field (in vertices) that eg_labels_static accepts. */
#define EG_STATIC_MAX_VERTICES (1u << 20)

/* Per-vertex labels (the maximum each vertex's gradient path reaches, or the
 * minimum with EG_FLAG_MINIMUM_GRAPH in flags) WITHOUT allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library call cudaMalloc or cudaFree -- for example when another
 * allocator owns all device memory, under a fixed memory budget, or in a
 * latency-critical loop where those calls may synchronise the whole device.
 *
 * field: device float32[N]; labels: device uint32[N] (written); d in 1..4;
 * extents as for eg_compute, with N <= EG_STATIC_MAX_VERTICES.  Larger fields
 * are rejected with EG_ERR_ARG before any work is enqueued.
 * Work runs on `stream`; the call returns after it has finished (it reads back
 * a status word and synchronises the stream), so labels are ready on return.
 * A stream that is being captured into a CUDA graph is therefore refused
 * (EG_ERR_ARG, checked before any work is enqueued).
 * Scratch: a fixed array compiled into the library (about 16 bytes per vertex
 * of EG_STATIC_MAX_VERTICES, ~17 MB) that every GPU loading the library holds
 * until the process exits.  Every call looks up its device address with the
 * caller's current device (no address is cached, so a device reset leaves
 * nothing stale); the first call on a device loads the library's device code
 * there, so make it before any capture begins on that device.  All calls on a
 * device share the one array, and it keeps the last call's contents (the call
 * clears what must start at zero): calls that overlap on the GPU -- from
 * several host threads or on several streams -- race on it and must be
 * serialised by the caller.
 * Needs no handle.  Errors: EG_ERR_ARG, EG_ERR_NAN, EG_ERR_NOT_CONVERGED,
 * EG_ERR_CUDA. */
EG_API eg_status eg_labels_static(const float *field, int d, const int64_t *extents, uint32_t flags,
                                  uint32_t *labels, void *stream);

/* Kernel launches issued by the handle since its creation (for accounting). */
EG_API uint64_t eg_launch_count(eg_handle h);

/* Test hook: make the k-th next device allocation of the handle fail with
 * EG_ERR_OOM (k = 0 disables).  Host-side fault injection only. */
EG_API eg_status eg_debug_fail_alloc(eg_handle h, int k);

/* Test hook: run one bounded device-side wait (the look-back used by the
 * scans) on a predecessor that never publishes.  The wait gives up after its
 * spin budget (about a second) and the call returns EG_ERR_TIMEOUT; the CUDA
 * context stays usable.  Blocks until done. */
EG_API eg_status eg_debug_wait_timeout(eg_handle h, void *stream);

/* Human-readable name of a status code (static string). */
EG_API const char *eg_status_str(eg_status s);

#ifdef __cplusplus
}
#endif
#endif /* EG_H */
