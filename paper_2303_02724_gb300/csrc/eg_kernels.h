// Host-callable launchers of the library's kernels (internal).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "eg_internal.cuh"

namespace eg {

// Steps (a)+(c), general kernel: one CTA per flat brick (any d, any extents).
// fields: the slice of descriptors using this kernel dimension and
// classification type (float32 for narrow integer fields, whose float32
// image it reads; else the element type); the grid covers their bricks,
// global ids from fields[0].brick0.
cudaError_t launch_classify_flat(int kd, uint32_t dtype, const FieldDev *fields, int nf, uint64_t bricks,
                                 cudaStream_t st);

// Steps (a)+(c), row classifier for 4D float32 fields with rows of at most
// 1024 vertices (row layout: ty whole rows of one (z, w) plane per brick);
// one CTA per brick, global ids from fields[0].brick0.
cudaError_t launch_classify_r4(bool minimum, const FieldDev *fields, int nf, uint64_t bricks, cudaStream_t st);
// 5D row classifier: float32 fields whose rows hold at most kR5MaxRow
// vertices; one thread per vertex, bricks of whole rows of one (z, w, u) plane.
constexpr int kR5CtaThreads = 256;
constexpr uint32_t kR5MaxRow = 256;
constexpr uint32_t kR5Passes = 4;  // bricks of up to 4 x 256 vertices
cudaError_t launch_classify_r5(bool minimum, const FieldDev *fields, int nf, uint64_t bricks, cudaStream_t st);
constexpr int kR4Vertices = 4;    // vertices per thread along axis 0
constexpr int kR4CtaThreads = 256;

// Element types (Sec. 5): widening of a narrow integer field (field->fraw,
// 8/16-bit, n elements) to its float32 image field->f.  Reads the descriptor
// on the device (so it can be captured in graphs).
cudaError_t launch_widen(uint32_t dtype, const FieldDev *field, uint64_t n, int sm_count, cudaStream_t st);

// Steps (a)+(c), plane-marching kernel for 2D/3D fields with rows of at most
// kZmMaxRow vertices.
// lut: the 2-bit class of every 14-bit upper mask (1024 words), then, as
// 16-bit words, the component holding each mask's lowest set bit.
constexpr uint32_t kZmMaxRow = 2048;
size_t zm_smem_bytes(uint32_t n0, uint32_t ty);
// Persistent: grid = min(total_items, sm_count * ctas_per_sm) CTAs take work
// items from *ticket (zeroed before the launch).
cudaError_t launch_classify_zm(bool minimum, const FieldDev *fields, int nf, uint64_t total_items, size_t smem,
                               const uint32_t *lut, unsigned long long *ticket, int sm_count, int ctas_per_sm,
                               cudaStream_t st);

// Zero the totals and status word of every field of a launch.
cudaError_t launch_init_fields(const FieldDev *fields, int nf, cudaStream_t st);
// Set the classifier's shared-memory attribute on the current device (also
// done lazily by launch_classify_zm; call it before capturing a graph).
cudaError_t prepare_classify_zm();

// Test hook: a look-back wait whose predecessor never publishes.
cudaError_t launch_lookback_orphan(uint64_t *st, uint32_t *err, cudaStream_t s);

// Scan A (arcs = false) / scan B (arcs = true) over all bricks of all fields.
uint64_t scan_tiles(uint32_t nbricks);
size_t scan_workspace_bytes(uint64_t total_tiles);
cudaError_t launch_scan(bool arcs, const FieldDev *fields, int nf, uint64_t total_tiles, void *ws, cudaStream_t st);

// Single-field, descriptor-by-value variants of the flat classifier and of the
// resolver (flat brick layout).
cudaError_t launch_classify_one(int kd, const FieldDev &F, cudaStream_t st);
cudaError_t launch_resolve_one(const FieldDev &F, cudaStream_t st);

// Step (b): labels = fixed points of the gradient pointers (all fields).
cudaError_t launch_resolve(const FieldDev *fields, int nf, uint64_t total_bricks, int walks, cudaStream_t st);

// Step (b), tiled pass for fields with few maxima (long gradient paths), run
// before launch_resolve: tiles numbered by FieldDev::rtile0 over all fields.
cudaError_t launch_resolve_tiles(const FieldDev *fields, int nf, uint64_t tiles, cudaStream_t st);
// Resolution tile extents (log2) of a field of extents n0 x n1 x n2, and the
// number of its tiles (alone: the field is the launch's only one).
void resolve_tile_shape(uint32_t n0, uint32_t n1, uint32_t n2, bool alone, uint32_t rt[3], uint64_t *tiles);

// Steps (d)+(e): nodes and arc ends per brick (one kernel dimension), then CSR.
cudaError_t launch_nodes_d(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks, cudaStream_t st);
cudaError_t launch_csr(const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st);

// Arc geometry (fields with path_ptr set; between classification and
// resolution): path lengths per brick, their scan (one CTA per field of the
// table), then offsets and vertices.
cudaError_t launch_path_len(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks, cudaStream_t st);
cudaError_t launch_path_scan(const FieldDev *fields, int nf, cudaStream_t st);
cudaError_t launch_path_write(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks,
                              cudaStream_t st);

// Arc bundling on a finished graph: pair count (added to *count), then the
// hash-table passes (keys preset to all ones, best to zero, 2^lg slots).
cudaError_t launch_bundle_pairs(const uint64_t *row_ptr, uint64_t S, unsigned long long *count, cudaStream_t st);
cudaError_t launch_bundle(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles,
                          const float *sad_val, uint64_t S, bool minimum, unsigned long long *keys,
                          unsigned long long *best, uint32_t lg, uint8_t *keep, uint32_t *err, cudaStream_t st);
// The same for a field of another element type: saddle values sad_raw in
// that type; the highest saddle of a pair is found in two rounds (its value
// key in best, then its vertex id among the saddles with that value in
// best_id; both tables zeroed).
cudaError_t launch_bundle_typed(uint32_t dtype, const uint64_t *row_ptr, const uint32_t *col,
                                const uint32_t *saddles, const void *sad_raw, uint64_t S, bool minimum,
                                unsigned long long *keys, unsigned long long *best, unsigned int *best_id,
                                uint32_t lg, uint8_t *keep, uint32_t *err, cudaStream_t st);

// Persistence-directed cancellation on a finished float32 graph, in rounds
// (see eg_cancel.cu).  Every array is device memory sized as noted.
struct CancelDev {
    const uint32_t *maxima;      // [M] vertex ids, ascending
    const float *max_val;        // [M]
    const float *sad_val;        // [S]
    const uint64_t *row_ptr;     // [S+1] arcs of every saddle
    uint32_t *end;               // [A] arc end as an index into maxima
    uint32_t *aroot[2];          // [A] each: survivor of every arc end, snapshot of the rounds of one parity
    uint32_t *parent;            // [M] merge target of a merged maximum, else itself
    unsigned long long *minlb[2]; // [M] each: smallest lb key of the saddles reaching it (by round parity)
    unsigned long long *min2[2];  // [M] each: smallest lb key but the smallest one's holder
    unsigned long long *costkey; // [S]
    unsigned long long *lbkey;   // [S]
    uint32_t *high;              // [S] highest current maximum of the saddle
    uint8_t *state;              // [S] 0 waiting, 1 cancelled, 2 never cancelled
    uint32_t *list[2];           // [S] each: saddles walked by this / the next round
    unsigned long long *ctrl;    // [3 r .. 3 r + 2] round slot r (cheapest key, cancellations,
                                 // length of the list kept), [9] rounds, [10] grid barrier
    uint32_t *err;               // status word
    uint32_t M, S;
    float tau;
    int minimum;
};
// Fused path for one small 1D-3D float32 field: every step in one
// cooperative launch over a flat layout of small_bricks(N) bricks of 256
// vertices (bcap 256, at most 256 bricks); bar: the barrier's count, zero at
// the start (the launch leaves it at 4 times the grid size); next_err,
// next_count: the status word and barrier count of the next launch's block,
// zeroed by this one; htotals[4] and herr:
// page-locked host memory (device-accessible under unified addressing) that
// receives F's totals and status word when the launch finishes, and is left
// as it was if a barrier timed out.  F.err must be zero at the start.
constexpr uint64_t kSmallMaxVertices = 1u << 16;
constexpr uint32_t kSmallBrick = 256;
uint32_t small_bricks(uint64_t n);
cudaError_t launch_small(const FieldDev &F, unsigned *bar, uint32_t *next_err, unsigned *next_count,
                         unsigned long long *htotals, uint32_t *herr, int sm_count, cudaStream_t st);

// Set-up (every saddle waits, in list[0], ctrl zeroed but slot 0's key, which
// is all ones); all rounds in one cooperative launch; the results.
cudaError_t launch_cancel_setup(const CancelDev &C, const uint32_t *col, uint64_t A, cudaStream_t st);
cudaError_t launch_cancel_rounds(const CancelDev &C, int sm_count, cudaStream_t st);
cudaError_t launch_cancel_out(const CancelDev &C, uint8_t *alive, uint32_t *survivor, cudaStream_t st);

}  // namespace eg
