// C ABI of the extremum-graph library: handles, memory pools, orchestration.
//
// One computation (eg_compute, or one eg_batch_submit for many fields) runs
//   classify (steps a+c) -> resolve (step b) -> emit (steps d+e)
// on the caller's stream.  The only host wait is for the node counts written
// by classify (a few bytes copied on a side stream that waits for classify
// alone, so resolve keeps the GPU busy meanwhile); they size the result
// buffers that emit fills.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "eg.h"
#include "eg_internal.cuh"
#include "eg_kernels.h"

using namespace eg;

static_assert(kF32 == EG_DTYPE_F32 && kF64 == EG_DTYPE_F64 && kI8 == EG_DTYPE_I8 && kU8 == EG_DTYPE_U8 &&
                  kI16 == EG_DTYPE_I16 && kU16 == EG_DTYPE_U16 && kI32 == EG_DTYPE_I32 && kU32 == EG_DTYPE_U32 &&
                  kI64 == EG_DTYPE_I64 && kU64 == EG_DTYPE_U64 && kNumTypes == EG_DTYPE_COUNT,
              "internal element-type codes follow eg_dtype");
static_assert(kFlagMinimum == EG_FLAG_MINIMUM_GRAPH && kFlagNoLabels == EG_FLAG_NO_LABELS && kFlagPaths == EG_FLAG_PATHS &&
                  kFlagNoFused == EG_FLAG_NO_FUSED,
              "flag bits of the ABI and the kernels differ");

namespace {

eg_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return EG_OK;
    if (e == cudaErrorMemoryAllocation) return EG_ERR_OOM;
    return EG_ERR_CUDA;
}

// Caching device allocator: exact size classes, reused across calls so the
// steady state performs no cudaMalloc.
struct DevPool {
    std::unordered_map<size_t, std::vector<void *>> free_;
    std::unordered_map<void *, size_t> size_of_;
    uint64_t held = 0;
    int fail_in = 0;  // fault injection: the fail_in-th next fresh allocation fails

    static size_t round(size_t b)
    {
        if (b < 256) return 256;
        if (b <= (1u << 20)) {
            size_t r = 256;
            while (r < b) r <<= 1;
            return r;
        }
        return (b + (1u << 20) - 1) & ~size_t((1u << 20) - 1);
    }
    cudaError_t alloc(void **p, size_t bytes)
    {
        *p = nullptr;
        if (fail_in > 0 && --fail_in == 0) return cudaErrorMemoryAllocation;
        const size_t sz = round(bytes);
        auto it = free_.find(sz);
        if (it != free_.end() && !it->second.empty()) {
            *p = it->second.back();
            it->second.pop_back();
            return cudaSuccess;
        }
        cudaError_t e = cudaMalloc(p, sz);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            trim();
            e = cudaMalloc(p, sz);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return e;
        }
        size_of_[*p] = sz;
        held += sz;
        return cudaSuccess;
    }
    void release(void *p)
    {
        if (!p) return;
        auto it = size_of_.find(p);
        if (it == size_of_.end()) return;
        free_[it->second].push_back(p);
    }
    void trim()
    {
        for (auto &kv : free_) {
            for (void *p : kv.second) {
                cudaFree(p);
                held -= kv.first;
                size_of_.erase(p);
            }
            kv.second.clear();
        }
    }
    void destroy()
    {
        for (auto &kv : size_of_) cudaFree(kv.first);
        size_of_.clear();
        free_.clear();
        held = 0;
    }
};

struct HostPool {
    std::unordered_map<size_t, std::vector<void *>> free_;
    std::unordered_map<void *, size_t> size_of_;
    cudaError_t alloc(void **p, size_t bytes)
    {
        size_t sz = DevPool::round(bytes);
        auto it = free_.find(sz);
        if (it != free_.end() && !it->second.empty()) {
            *p = it->second.back();
            it->second.pop_back();
            return cudaSuccess;
        }
        cudaError_t e = cudaHostAlloc(p, sz, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return e;
        }
        size_of_[*p] = sz;
        return cudaSuccess;
    }
    void release(void *p)
    {
        if (!p) return;
        auto it = size_of_.find(p);
        if (it != size_of_.end()) free_[it->second].push_back(p);
    }
    void destroy()
    {
        for (auto &kv : size_of_) cudaFreeHost(kv.first);
        size_of_.clear();
        free_.clear();
    }
};

// Fields of at most this many vertices, computed alone, get result buffers
// sized by bounds instead of waiting for their node counts.
constexpr uint64_t kBoundedVertices = 1u << 16;

// Per-field small device block: totals[4] (M, S, P, A) + status word.
struct alignas(16) SmallBlock {
    unsigned long long totals[4];
    uint32_t err;
    uint32_t bar[2];   // grid-barrier words of the fused small-field kernel
    uint32_t pad[5];
};

struct Result {
    int d = 0;
    uint32_t dtype = 0;     // element type of the field and of the value copies
    void *wide = nullptr;   // float32 image of a narrow integer field (while classifying)
    int64_t ext[kMaxDim] = {};
    uint64_t N = 0;
    uint32_t flags = 0;
    void *lab = nullptr;
    void *small = nullptr;  // its SmallBlock on the device (in the launch's array)
    int slot = 0;           // index of that SmallBlock in the launch's array
    void *maxima = nullptr, *max_val = nullptr, *saddles = nullptr, *sad_b0 = nullptr, *sad_val = nullptr,
         *row_ptr = nullptr, *col = nullptr, *ends = nullptr, *ucnt = nullptr;
    void *path_ptr = nullptr, *path_vtx = nullptr, *pbrick = nullptr;  // arc geometry (EG_FLAG_PATHS)
    uint64_t M = 0, S = 0, P = 0, A = 0, V = 0;
    bool have_A = false;
    bool bounded = false;   // buffers sized by bounds; counts read when the result is collected
    uint32_t err = 0;
    cudaEvent_t done = nullptr;  // the launch's completion event (owned by the launch)
    std::shared_ptr<struct Launch> launch;  // keeps the descriptor table alive
};

// Descriptor tables of one launch (shared by the results of a batch), and
// the results' SmallBlocks, one array read back once for all of them.
struct Launch {
    void *desc_dev = nullptr;
    void *desc_host = nullptr;
    size_t bytes = 0;
    void *smalls = nullptr;           // SmallBlock[nsmall] on the device
    int nsmall = 0;
    std::vector<SmallBlock> hsmall;   // host copy once the launch finished
    void *hsmall_pin = nullptr;       // page-locked copy, written by the launch's last step
    cudaEvent_t done = nullptr;       // recorded after the launch's last step
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // step timing (optional)
    bool fused = false;               // one fused kernel: only ev[0] and ev[1] are recorded
    struct eg_ctx *owner = nullptr;   // the handle whose event pool the events return to
    ~Launch();
};

}  // namespace

struct eg_ctx {
    std::mutex mu;
    int device = 0;
    int sm_count = 0;
    eg_config cfg{};
    DevPool pool;
    HostPool hpool;
    cudaStream_t side = nullptr;
    cudaEvent_t ws_free = nullptr;  // recorded after the last kernel that used the workspace
    // workspace (reused by every computation)
    void *ws_rec_sid = nullptr, *ws_rec_info = nullptr, *ws_rec_val = nullptr;
    uint64_t ws_rec_cap = 0;
    void *ws_bcnt = nullptr, *ws_boff = nullptr, *ws_acnt = nullptr, *ws_aoff = nullptr;
    uint64_t ws_bricks = 0;
    void *ws_scan = nullptr;
    uint64_t ws_tiles = 0;
    void *lut3 = nullptr;  // saddle class table of the 3D link graph + two-component table
    // the fused small-field kernel's totals, status and barrier words: two
    // blocks used in turn; launch k works in block k % 2 and zeroes the
    // status and barrier count of the other for launch k + 1 (the launches
    // of a handle are ordered on the GPU by ws_free, so no memset is needed)
    void *fused_pair = nullptr;
    uint64_t fused_seq = 0;
    void *stage = nullptr;  // device staging for eg_compute_host
    size_t stage_bytes = 0;
    void *hstage = nullptr;  // pinned staging for pageable host fields
    size_t hstage_bytes = 0;
    std::unordered_map<uint64_t, std::unique_ptr<Result>> results;
    uint64_t next_id = 1;
    std::atomic<uint64_t> launches{0};
    bool timing = false;
    cudaStream_t cap = nullptr;  // private stream for graph capture
    std::unique_ptr<struct eg_graph_cache> graphs;
    uint64_t ws_gen = 0;  // bumped whenever the workspace is reallocated
    std::vector<cudaEvent_t> ev_pool[2];  // idle events: [0] without timing, [1] with
};

namespace {

// Events are reused: creating them costs more host time than a small field's
// whole computation.  An event returns to its handle's pool only when its
// launch is gone, i.e. after every result of the launch was released (which
// waits for the launch's last event), or after a failed call synchronised
// its stream.
cudaError_t get_event(eg_ctx *h, cudaEvent_t *e, bool timed)
{
    auto &pool = h->ev_pool[timed ? 1 : 0];
    if (!pool.empty()) {
        *e = pool.back();
        pool.pop_back();
        return cudaSuccess;
    }
    return timed ? cudaEventCreate(e) : cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}

}  // namespace

Launch::~Launch()
{
    for (auto &e : ev)
        if (e) owner->ev_pool[1].push_back(e);
    if (done) owner->ev_pool[0].push_back(done);
}

namespace {

struct Shape {
    int d;
    uint32_t n[kMaxDim];
    uint32_t s[kMaxDim];
    uint64_t N;
};

bool make_shape(int d, const int64_t *ext, Shape &sh)
{
    if (d < 1 || d > kMaxDim || !ext) return false;
    uint64_t N = 1;
    for (int i = 0; i < kMaxDim; i++) {
        sh.n[i] = 1;
        sh.s[i] = 0;
    }
    for (int i = 0; i < d; i++) {
        if (ext[i] < 1 || ext[i] > 0xffffffffll) return false;
        sh.s[i] = uint32_t(N);
        N *= uint64_t(ext[i]);
        if (N > 0xffffffffull) return false;
        sh.n[i] = uint32_t(ext[i]);
    }
    // fields of 1..3 dimensions run as 3D: unused axes have extent 1
    for (int i = d; i < kMaxDim; i++) sh.s[i] = uint32_t(N);
    sh.d = d;
    sh.N = N;
    return true;
}

// Brick layout of one field (see eg_internal.cuh): row layout for the
// plane-marching classifier when the rows are short enough, else flat.
struct Layout {
    int kd;
    bool zm;
    bool r4;  // 4D row classifier (row layout over (z, w) planes)
    bool r5;  // 5D row classifier (row layout over (z, w, u) planes)
    uint32_t ty, nyb, nbricks, bcap, zc, nzc;
    size_t smem;
};

Layout make_layout(const Shape &sh, int sm_count, const eg_config &cfg, uint32_t dtype = kF32)
{
    Layout L{};
    L.kd = sh.d == 5 ? 5 : (sh.d == 4 ? 4 : 3);
    const uint32_t n0 = sh.n[0], n1 = sh.n[1], n2 = sh.n[2];
    // the plane-marching classifier reads float32 (the field, or the float32
    // image of a narrow integer field); other types take the flat classifier
    const bool f32_values = dtype == kF32 || dtype_narrow(dtype);
    if (L.kd == 3 && n0 <= kZmMaxRow && f32_values) {
        // one thread per 8 consecutive vertices of a row, 256 threads per CTA
        // (rows of more than 1024 vertices: one row per brick)
        const uint32_t txn = (n0 + 7) / 8;
        uint32_t ty = 256 / txn;
        if (cfg.classify_rows >= 1) {
            ty = std::min<uint32_t>(ty, uint32_t(cfg.classify_rows));
        } else if (uint64_t((n1 + ty - 1) / ty) * n2 < uint64_t(std::max(sm_count, 1))) {
            // a small field: thinner row blocks, so that its bricks (and the
            // CTAs of every step) cover the GPU
            ty = std::max<uint32_t>(1, std::min<uint32_t>(ty, uint32_t(uint64_t(n1) * n2 / uint64_t(std::max(sm_count, 1)))));
        }
        // rows per brick: the saddle queue of the classifier stores ring rows in 7 bits
        ty = std::max<uint32_t>(1, std::min(std::min(ty, 126u), n1));
        L.zm = true;
        L.ty = ty;
        L.nyb = (n1 + ty - 1) / ty;
        L.nbricks = L.nyb * n2;
        L.bcap = ty * n0;
        if (cfg.classify_planes > 0) {
            L.zc = std::min<uint32_t>(n2, uint32_t(cfg.classify_planes));
        } else {
            // enough work items to fill the GPU a few times over
            const uint64_t want = uint64_t(std::max(sm_count, 1)) * 8;
            const uint32_t nzc = uint32_t(std::min<uint64_t>(n2, std::max<uint64_t>(1, (want + L.nyb - 1) / L.nyb)));
            L.zc = (n2 + nzc - 1) / nzc;
        }
        L.nzc = (n2 + L.zc - 1) / L.zc;
        L.smem = zm_smem_bytes(n0, ty);
    } else if (L.kd == 4 && n0 <= 1024 && f32_values) {
        // 4D row classifier: one thread per kR4Vertices consecutive vertices of
        // a row, ty whole rows of one (z, w) plane per brick
        const uint32_t txn = (n0 + kR4Vertices - 1) / kR4Vertices;
        const uint32_t ty = std::max<uint32_t>(1, std::min<uint32_t>(uint32_t(kR4CtaThreads) / txn, n1));
        L.zm = false;
        L.r4 = true;
        L.ty = ty;
        L.nyb = (n1 + ty - 1) / ty;
        L.nbricks = L.nyb * n2 * sh.n[3];
        L.bcap = ty * n0;
        L.zc = L.nzc = 0;
        L.smem = 0;
    } else if (L.kd == 5 && n0 <= kR5MaxRow && f32_values) {
        // 5D row classifier: ty whole rows of one (z, w, u) plane per brick,
        // classified in up to kR5Passes passes of one vertex per thread
        const uint32_t ty = std::max<uint32_t>(1, std::min<uint32_t>(uint32_t(kR5CtaThreads) / n0 * kR5Passes, n1));
        L.zm = false;
        L.r5 = true;
        L.ty = ty;
        L.nyb = (n1 + ty - 1) / ty;
        L.nbricks = L.nyb * n2 * sh.n[3] * sh.n[4];
        L.bcap = ty * n0;
        L.zc = L.nzc = 0;
        L.smem = 0;
    } else {
        L.zm = false;
        L.ty = 0;
        L.nyb = 0;
        L.nbricks = uint32_t((sh.N + kFlatBrick - 1) / kFlatBrick);
        L.bcap = kFlatBrick;
        L.zc = L.nzc = 0;
        L.smem = 0;
    }
    return L;
}

template <typename T>
eg_status grow(eg_ctx *h, void **p, uint64_t &cap, uint64_t want, size_t elem)
{
    if (want <= cap && *p) return EG_OK;
    h->pool.release(*p);
    *p = nullptr;
    cap = 0;
    const uint64_t c = std::max<uint64_t>(want, 64);
    cudaError_t e = h->pool.alloc(p, c * elem);
    if (e != cudaSuccess) return from_cuda(e);
    cap = c;
    return EG_OK;
}

eg_status ensure_workspace(eg_ctx *h, uint64_t recs, uint64_t bricks, uint64_t tiles)
{
    if (recs <= h->ws_rec_cap && bricks <= h->ws_bricks && tiles <= h->ws_tiles) return EG_OK;
    // earlier computations may still use the old workspace
    cudaEventSynchronize(h->ws_free);
    h->ws_gen++;
    eg_status s;
    uint64_t cap = h->ws_rec_cap;
    if (recs > h->ws_rec_cap) {
        uint64_t c1 = h->ws_rec_cap, c2 = h->ws_rec_cap;
        if ((s = grow<uint32_t>(h, &h->ws_rec_sid, cap, recs, 4)) != EG_OK) return s;
        if ((s = grow<uint64_t>(h, &h->ws_rec_info, c1, recs, 8)) != EG_OK) return s;
        if ((s = grow<float>(h, &h->ws_rec_val, c2, recs, 4)) != EG_OK) return s;
        h->ws_rec_cap = std::min(cap, std::min(c1, c2));
    }
    if (bricks > h->ws_bricks) {
        uint64_t a = h->ws_bricks, b = h->ws_bricks, c = h->ws_bricks, d = h->ws_bricks;
        if ((s = grow<uint4>(h, &h->ws_bcnt, a, bricks, sizeof(uint4))) != EG_OK) return s;
        if ((s = grow<uint4>(h, &h->ws_boff, b, bricks, sizeof(uint4))) != EG_OK) return s;
        if ((s = grow<uint32_t>(h, &h->ws_acnt, c, bricks, 4)) != EG_OK) return s;
        if ((s = grow<uint64_t>(h, &h->ws_aoff, d, bricks, 8)) != EG_OK) return s;
        h->ws_bricks = std::min(std::min(a, b), std::min(c, d));
    }
    if (tiles > h->ws_tiles) {
        uint64_t t = h->ws_tiles;
        h->pool.release(h->ws_scan);
        h->ws_scan = nullptr;
        const uint64_t c = std::max<uint64_t>(tiles, 64);
        cudaError_t e = h->pool.alloc(&h->ws_scan, scan_workspace_bytes(c));
        if (e != cudaSuccess) {
            h->ws_tiles = 0;
            return from_cuda(e);
        }
        (void)t;
        h->ws_tiles = c;
    }
    return EG_OK;
}

void free_result_buffers(eg_ctx *h, Result *r)
{
    void **bufs[] = {&r->lab, &r->maxima,   &r->max_val,  &r->saddles, &r->sad_b0, &r->sad_val, &r->row_ptr,
                     &r->col, &r->ends,     &r->ucnt,     &r->path_ptr, &r->path_vtx, &r->pbrick, &r->wide};
    for (void **b : bufs) {
        h->pool.release(*b);
        *b = nullptr;
    }
}

void release_launch(eg_ctx *h, Launch *L)
{
    if (!L) return;
    h->pool.release(L->desc_dev);
    h->hpool.release(L->desc_host);
    h->pool.release(L->smalls);
    h->hpool.release(L->hsmall_pin);
    L->desc_dev = L->desc_host = L->smalls = L->hsmall_pin = nullptr;
}

struct Job {
    const void *field;
    Shape sh;
    uint32_t flags;
    uint32_t dtype = kF32;
};

// One launch slice: fields of one classifier kind, contiguous in the table.
struct Group {
    int key, first, count;
    uint64_t brick0, bricks, items;
    size_t smem;
    bool zm, minimum;
    int kd;
    uint32_t cdt;  // type the classifier compares in (float32 for narrow integers)
    bool r4;
    bool r5;
};

// A field (table position) whose element type needs extra work.
struct TypedField {
    int pos;
    uint32_t dtype;
    uint64_t n;
};

// Everything the enqueue phases of one call need besides the table contents.
struct Plan {
    int nf = 0;
    std::vector<Group> groups;
    uint64_t total_bricks = 0, total_tiles = 0;
    uint64_t total_rtiles = 0;  // tiled resolution pass (3D kernels)
    size_t desc_bytes = 0;
    int walks = 4, ctas = 3;
    int sm_count = 0;
    std::vector<TypedField> widen;   // narrow integer fields: float32 image before classification
    std::string signature;  // identical for calls that can share a captured graph
};

// Enqueue one phase of the pipeline on st, reading descriptors from Dd:
//   0: descriptor upload, scan state reset, counters reset, classification
//      (steps a+c), scan A;   1: resolution (step b);
//   2: descriptor upload, nodes and arc ends, scan B, CSR (steps d+e).
// Only stream-ordered operations: the same calls are captured into graphs.
eg_status enqueue_part(eg_ctx *h, int part, const Plan &P, const FieldDev *Dd, const void *desc_host,
                       cudaStream_t st, int *launches)
{
    cudaError_t e = cudaSuccess;
    int nl = 0;
    if (part == 0) {
        if ((e = cudaMemcpyAsync(const_cast<FieldDev *>(Dd), desc_host, P.desc_bytes, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return from_cuda(e);
        if ((e = cudaMemsetAsync(h->ws_scan, 0, scan_workspace_bytes(P.total_tiles), st)) != cudaSuccess)
            return from_cuda(e);
        if ((e = launch_init_fields(Dd, P.nf, st)) != cudaSuccess) return from_cuda(e);
        nl++;
        for (const TypedField &t : P.widen) {
            if ((e = launch_widen(t.dtype, Dd + t.pos, t.n, P.sm_count, st)) != cudaSuccess) return from_cuda(e);
            nl++;
        }
        for (size_t gi = 0; gi < P.groups.size(); gi++) {
            const Group &G = P.groups[gi];
            if (G.zm)
                e = launch_classify_zm(G.minimum, Dd + G.first, G.count, G.items, G.smem,
                                       static_cast<const uint32_t *>(h->lut3),
                                       reinterpret_cast<unsigned long long *>(h->ws_scan) + 2 + gi, h->sm_count,
                                       P.ctas, st);
            else if (G.r4)
                e = launch_classify_r4(G.minimum, Dd + G.first, G.count, G.bricks, st);
            else if (G.r5)
                e = launch_classify_r5(G.minimum, Dd + G.first, G.count, G.bricks, st);
            else
                e = launch_classify_flat(G.kd, G.cdt, Dd + G.first, G.count, G.bricks, st);
            if (e != cudaSuccess) return from_cuda(e);
            nl++;
        }
        if ((e = launch_scan(false, Dd, P.nf, P.total_tiles, h->ws_scan, st)) != cudaSuccess) return from_cuda(e);
        nl++;
    } else if (part == 1) {
        if (P.total_rtiles) {
            if ((e = launch_resolve_tiles(Dd, P.nf, P.total_rtiles, st)) != cudaSuccess) return from_cuda(e);
            nl++;
        }
        if ((e = launch_resolve(Dd, P.nf, P.total_bricks, P.walks, st)) != cudaSuccess) return from_cuda(e);
        nl++;
    } else {
        if ((e = cudaMemcpyAsync(const_cast<FieldDev *>(Dd), desc_host, P.desc_bytes, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return from_cuda(e);
        for (const Group &G : P.groups) {
            if ((e = launch_nodes_d(G.kd, Dd + G.first, G.count, G.brick0, G.bricks, st)) != cudaSuccess)
                return from_cuda(e);
            nl++;
        }
        if ((e = launch_scan(true, Dd, P.nf, P.total_tiles, h->ws_scan, st)) != cudaSuccess) return from_cuda(e);
        if ((e = launch_csr(Dd, P.nf, P.total_bricks, st)) != cudaSuccess) return from_cuda(e);
        nl += 2;
    }
    if (launches) *launches = nl;
    return EG_OK;
}

// Captured graphs of the three phases for one plan signature.
struct GraphEntry {
    cudaGraph_t g[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t x[3] = {nullptr, nullptr, nullptr};
    cudaGraphNode_t upload[3] = {nullptr, nullptr, nullptr};  // descriptor memcpy of phases 0 and 2
    int launches[3] = {0, 0, 0};
    void *desc_dev = nullptr;
    uint64_t ws_gen = 0, last_use = 0;
};

void destroy_graph(eg_ctx *h, GraphEntry &E);

}  // namespace

// (graph cache lives in the handle)
struct eg_graph_cache {
    std::map<std::string, GraphEntry> entries;
    uint64_t clock = 0;
};

namespace {

eg_graph_cache &graph_cache(eg_ctx *h)
{
    if (!h->graphs) h->graphs.reset(new eg_graph_cache());
    return *h->graphs;
}

uint64_t &ws_generation(eg_ctx *h) { return h->ws_gen; }

void destroy_graph(eg_ctx *h, GraphEntry &E)
{
    for (int p = 0; p < 3; p++) {
        if (E.x[p]) cudaGraphExecDestroy(E.x[p]);
        if (E.g[p]) cudaGraphDestroy(E.g[p]);
        E.x[p] = nullptr;
        E.g[p] = nullptr;
    }
    h->pool.release(E.desc_dev);
    E.desc_dev = nullptr;
}

// Capture the three phases of plan P (descriptor upload source: desc_host).
eg_status capture_graphs(eg_ctx *h, const Plan &P, const void *desc_host, GraphEntry &E, cudaStream_t cap)
{
    cudaError_t e = h->pool.alloc(&E.desc_dev, P.desc_bytes);
    if (e != cudaSuccess) return from_cuda(e);
    if ((e = prepare_classify_zm()) != cudaSuccess) return from_cuda(e);
    for (int p = 0; p < 3; p++) {
        if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return from_cuda(e);
        eg_status s = enqueue_part(h, p, P, static_cast<const FieldDev *>(E.desc_dev), desc_host, cap, &E.launches[p]);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        if (s != EG_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return from_cuda(e);
        E.g[p] = g;
        if (p != 1) {
            size_t nn = 0;
            cudaGraphGetNodes(g, nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            cudaGraphGetNodes(g, nodes.data(), &nn);
            for (auto n : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeMemcpy) E.upload[p] = n;
            }
            if (!E.upload[p]) return EG_ERR_INTERNAL;
        }
        if ((e = cudaGraphInstantiate(&E.x[p], g, 0)) != cudaSuccess) return from_cuda(e);
    }
    return EG_OK;
}

// Run a set of fields (all of one call) through the pipeline.  use_graph:
// replay (capturing on first use) the graphs of this call's layout.
// Arc geometry of the fields that asked for it (EG_FLAG_PATHS), enqueued after
// the counts are known and before resolution (lab[] still holds the gradient
// pointers): path lengths, their scan, a read-back of each field's total, the
// vertex buffers, then the paths.  The descriptor table is uploaded before
// each kernel group (the host copy changes in between).
eg_status enqueue_paths(eg_ctx *h, const Plan &P, Launch *L, FieldDev *Dh,
                        std::vector<std::unique_ptr<Result>> &res, const std::vector<int> &order, cudaStream_t st)
{
    FieldDev *Dd = static_cast<FieldDev *>(L->desc_dev);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(Dd, L->desc_host, P.desc_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return from_cuda(e);
    for (const Group &G : P.groups)
        if ((e = launch_path_len(G.kd, Dd + G.first, G.count, G.brick0, G.bricks, st)) != cudaSuccess)
            return from_cuda(e);
    if ((e = launch_path_scan(Dd, P.nf, st)) != cudaSuccess) return from_cuda(e);
    h->launches += uint64_t(P.groups.size() + 1);
    cudaEvent_t k2;
    if ((e = cudaEventCreateWithFlags(&k2, cudaEventDisableTiming)) != cudaSuccess) return from_cuda(e);
    cudaEventRecord(k2, st);
    cudaStreamWaitEvent(h->side, k2, 0);
    void *hv = nullptr;
    if ((e = h->hpool.alloc(&hv, sizeof(uint64_t) * size_t(P.nf))) != cudaSuccess) {
        cudaEventDestroy(k2);
        return from_cuda(e);
    }
    uint64_t *V = static_cast<uint64_t *>(hv);
    for (int oi = 0; oi < P.nf; oi++) {
        V[oi] = 0;
        if (Dh[oi].path_ptr)
            cudaMemcpyAsync(V + oi, Dh[oi].pbrick + Dh[oi].nbricks, 8, cudaMemcpyDeviceToHost, h->side);
    }
    e = cudaStreamSynchronize(h->side);
    cudaEventDestroy(k2);
    eg_status s = EG_OK;
    for (int oi = 0; oi < P.nf && e == cudaSuccess && s == EG_OK; oi++) {
        if (!Dh[oi].path_ptr) continue;
        Result &r = *res[order[oi]];
        r.V = V[oi];
        cudaError_t a = h->pool.alloc(&r.path_vtx, std::max<uint64_t>(r.V, 1) * 4);
        if (a != cudaSuccess) s = from_cuda(a);
        else Dh[oi].path_vtx = static_cast<uint32_t *>(r.path_vtx);
    }
    h->hpool.release(hv);
    if (e != cudaSuccess) return from_cuda(e);
    if (s != EG_OK) return s;
    if ((e = cudaMemcpyAsync(Dd, L->desc_host, P.desc_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return from_cuda(e);
    for (const Group &G : P.groups)
        if ((e = launch_path_write(G.kd, Dd + G.first, G.count, G.brick0, G.bricks, st)) != cudaSuccess)
            return from_cuda(e);
    h->launches += uint64_t(P.groups.size());
    return EG_OK;
}

eg_status run_jobs(eg_ctx *h, const std::vector<Job> &jobs, cudaStream_t st, std::vector<uint64_t> &ids,
                   const eg_config &cfg, bool use_graph = false, bool single_call = false)
{
    const int nf = int(jobs.size());
    std::vector<Layout> lay(nf);
    for (int i = 0; i < nf; i++) lay[i] = make_layout(jobs[i].sh, h->sm_count, cfg, jobs[i].dtype);
    // the arc geometry needs the gradient pointers after the counts are known
    // and before resolution: such calls run step by step, without graphs
    bool any_paths = false;
    for (int i = 0; i < nf; i++) any_paths = any_paths || (jobs[i].flags & kFlagPaths);
    if (any_paths) use_graph = false;
    // a small field alone: result buffers sized by bounds, so the call never
    // waits for the node counts (they arrive with the launch's last copy)
    // (single-field calls only: batches and served streams keep exact buffers)
    const bool bounded = single_call && nf == 1 && !any_paths && !use_graph && jobs[0].sh.N <= kBoundedVertices;
    // ... and a 1D-3D float32 one takes every step in one cooperative launch
    // over a flat layout of 256-vertex bricks (eg_small.cu)
    const bool fused = bounded && !(cfg.flags & kFlagNoFused) && jobs[0].sh.d <= 3 && jobs[0].dtype == kF32 &&
                       jobs[0].sh.N <= kSmallMaxVertices;
    if (fused) {
        Layout &ly = lay[0];
        ly = Layout{};
        ly.kd = 3;
        ly.nbricks = small_bricks(jobs[0].sh.N);
        ly.bcap = kSmallBrick;
    }
    // group fields by classifier kind so every launch covers a contiguous slice
    auto cdt = [&](int i) { return dtype_narrow(jobs[i].dtype) ? uint32_t(kF32) : jobs[i].dtype; };
    auto key = [&](int i) {
        // (the plane-marching kernel's rows longer than 1024 vertices launch
        // on their own: their ring needs more shared memory per CTA)
        const int kind = lay[i].zm ? (jobs[i].sh.n[0] > 1024 ? 3 : 0) : (lay[i].r4 ? 1 : (lay[i].r5 ? 4 : 2));
        return int(cdt(i)) * 64 + kind * 16 + lay[i].kd * 2 + ((jobs[i].flags & kFlagMinimum) ? 1 : 0);
    };
    std::vector<int> order(nf);
    for (int i = 0; i < nf; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });

    Plan P;
    P.nf = nf;
    P.walks = cfg.resolve_walks > 0 ? cfg.resolve_walks : 4;
    P.ctas = cfg.persistent_ctas > 0 ? cfg.persistent_ctas : 3;
    P.sm_count = h->sm_count;
    uint64_t total_recs = 0;
    for (int i = 0; i < nf; i++) {
        P.total_bricks += lay[i].nbricks;
        total_recs += uint64_t(lay[i].nbricks) * lay[i].bcap;
        P.total_tiles += scan_tiles(lay[i].nbricks);
    }
    P.desc_bytes = sizeof(FieldDev) * size_t(nf);
    eg_status es = ensure_workspace(h, total_recs, P.total_bricks, P.total_tiles);
    if (es != EG_OK) return es;

    auto L = std::make_shared<Launch>();
    L->owner = h;
    L->bytes = P.desc_bytes;
    cudaError_t e;
    std::vector<std::unique_ptr<Result>> res(nf);
    auto fail = [&](eg_status s) {
        cudaStreamSynchronize(st);
        for (auto &r : res)
            if (r) {
                free_result_buffers(h, r.get());
            }
        release_launch(h, L.get());
        return s;
    };
    if (!use_graph && (e = h->pool.alloc(&L->desc_dev, L->bytes)) != cudaSuccess) return fail(from_cuda(e));
    if ((e = h->hpool.alloc(&L->desc_host, L->bytes)) != cudaSuccess) return fail(from_cuda(e));
    if ((e = h->pool.alloc(&L->smalls, sizeof(SmallBlock) * size_t(nf))) != cudaSuccess) return fail(from_cuda(e));
    if ((e = h->hpool.alloc(&L->hsmall_pin, sizeof(SmallBlock) * size_t(nf))) != cudaSuccess) return fail(from_cuda(e));
    L->nsmall = nf;
    FieldDev *Dh = reinterpret_cast<FieldDev *>(L->desc_host);
    std::memset(Dh, 0, L->bytes);

    uint64_t brick0 = 0, rec0 = 0, tile0 = 0;
    if (use_graph) {  // (the key of the captured graphs)
        char sig[128];
        std::snprintf(sig, sizeof sig, "c%d/%d/%d/%d/%u|", cfg.classify_rows, cfg.classify_planes, P.walks, P.ctas,
                      cfg.flags);
        P.signature = sig;
    }
    for (int oi = 0; oi < nf; oi++) {
        const int i = order[oi];
        const Job &j = jobs[i];
        const Layout &ly = lay[i];
        if (P.groups.empty() || P.groups.back().key != key(i))
            P.groups.push_back(
                {key(i), oi, 0, brick0, 0, 0, 0, ly.zm, (j.flags & kFlagMinimum) != 0, ly.kd, cdt(i), ly.r4,
                 ly.r5});
        Group &G = P.groups.back();
        auto r = std::make_unique<Result>();
        r->d = j.sh.d;
        for (int q = 0; q < kMaxDim; q++) r->ext[q] = q < j.sh.d ? j.sh.n[q] : 0;
        r->N = j.sh.N;
        r->flags = j.flags;
        r->dtype = j.dtype;
        r->launch = L;
        e = h->pool.alloc(&r->lab, j.sh.N * sizeof(uint32_t));
        if (e == cudaSuccess && dtype_narrow(j.dtype)) e = h->pool.alloc(&r->wide, j.sh.N * sizeof(float));
        r->small = static_cast<SmallBlock *>(L->smalls) + i;
        r->slot = i;
        res[i] = std::move(r);
        if (e != cudaSuccess) return fail(from_cuda(e));
        Result &R = *res[i];
        FieldDev &F = Dh[oi];
        // the float32 kernels read the field itself, or the float32 image of
        // a narrow integer field; the 32/64-bit types are read through fraw
        F.f = j.dtype == kF32 ? static_cast<const float *>(j.field)
                              : (dtype_narrow(j.dtype) ? static_cast<const float *>(R.wide) : nullptr);
        F.fraw = j.field;
        F.dtype = j.dtype;
        if (dtype_narrow(j.dtype)) P.widen.push_back({oi, j.dtype, j.sh.N});
        F.lab = static_cast<uint32_t *>(R.lab);
        F.rec_sid = static_cast<uint32_t *>(h->ws_rec_sid) + rec0;
        F.rec_info = static_cast<uint64_t *>(h->ws_rec_info) + rec0;
        F.rec_val = static_cast<float *>(h->ws_rec_val) + rec0;
        F.bcnt = static_cast<uint4 *>(h->ws_bcnt) + brick0;
        F.boff = static_cast<uint4 *>(h->ws_boff) + brick0;
        F.acnt = static_cast<uint32_t *>(h->ws_acnt) + brick0;
        F.aoff = static_cast<uint64_t *>(h->ws_aoff) + brick0;
        F.totals = reinterpret_cast<SmallBlock *>(R.small)->totals;
        F.err = &reinterpret_cast<SmallBlock *>(R.small)->err;
        for (int q = 0; q < kMaxDim; q++) {
            F.n[q] = j.sh.n[q];
            F.s[q] = j.sh.s[q];
        }
        F.N = uint32_t(j.sh.N);
        F.nbricks = ly.nbricks;
        F.bcap = ly.bcap;
        F.ty = ly.ty;
        F.nyb = ly.nyb;
        F.zc = ly.zc;
        F.nzc = ly.nzc;
        F.vec = (j.sh.n[0] % 4 == 0 && (reinterpret_cast<uintptr_t>(F.f) & 15) == 0) ? 1u : 0u;
        F.brick0 = brick0;
        F.item0 = G.items;
        F.stile0 = tile0;
        F.kd = ly.kd;
        F.flags = j.flags;
        F.rtile0 = P.total_rtiles;
        if (ly.kd == 3) {
            uint64_t nt = 0;
            resolve_tile_shape(F.n[0], F.n[1], F.n[2], nf == 1, F.rt, &nt);
            P.total_rtiles += nt;
        }
        G.count++;
        G.bricks += ly.nbricks;
        G.items += ly.zm ? uint64_t(ly.nyb) * ly.nzc : ly.nbricks;
        G.smem = std::max(G.smem, ly.smem);
        brick0 += ly.nbricks;
        rec0 += uint64_t(ly.nbricks) * ly.bcap;
        tile0 += scan_tiles(ly.nbricks);
        if (use_graph) {  // (the key of the captured graphs)
            char fs[192];
            std::snprintf(fs, sizeof fs, "%d,%d,%u,%u,%u,%u,%u,%u,%u,%u,%u,%u,%u,%u;", key(i), ly.kd, F.N, ly.ty,
                          ly.nyb, ly.nbricks, ly.zc, ly.nzc, F.vec, F.n[0], F.n[1], F.n[2], F.n[3], j.dtype);
            P.signature += fs;
        }
    }

    // graphs for this layout (captured on first use; the workspace generation
    // is part of their validity because scan-state pointers are baked in)
    GraphEntry *GE = nullptr;
    if (use_graph) {
        eg_graph_cache &C = graph_cache(h);
        auto it = C.entries.find(P.signature);
        if (it != C.entries.end() && it->second.ws_gen != ws_generation(h)) {
            cudaEventSynchronize(h->ws_free);
            destroy_graph(h, it->second);
            C.entries.erase(it);
            it = C.entries.end();
        }
        if (it == C.entries.end()) {
            if (C.entries.size() >= 16) {  // evict the least recently used
                auto lru = C.entries.begin();
                for (auto jt = C.entries.begin(); jt != C.entries.end(); ++jt)
                    if (jt->second.last_use < lru->second.last_use) lru = jt;
                cudaEventSynchronize(h->ws_free);
                destroy_graph(h, lru->second);
                C.entries.erase(lru);
            }
            GraphEntry E;
            E.ws_gen = ws_generation(h);
            eg_status cs = capture_graphs(h, P, L->desc_host, E, h->cap);
            if (cs != EG_OK) {
                destroy_graph(h, E);
                return fail(cs);
            }
            it = C.entries.emplace(P.signature, E).first;
        }
        GE = &it->second;
        GE->last_use = ++C.clock;
    }
    const FieldDev *Dd = static_cast<const FieldDev *>(GE ? GE->desc_dev : L->desc_dev);
    auto run_part = [&](int p) -> eg_status {
        if (!GE) {
            int nl = 0;
            eg_status s = enqueue_part(h, p, P, Dd, L->desc_host, st, &nl);
            h->launches += uint64_t(nl);
            return s;
        }
        if (p != 1) {
            cudaError_t x = cudaGraphExecMemcpyNodeSetParams1D(GE->x[p], GE->upload[p], GE->desc_dev, L->desc_host,
                                                               P.desc_bytes, cudaMemcpyHostToDevice);
            if (x != cudaSuccess) return from_cuda(x);
        }
        cudaError_t x = cudaGraphLaunch(GE->x[p], st);
        if (x != cudaSuccess) return from_cuda(x);
        h->launches += uint64_t(GE->launches[p]);
        return EG_OK;
    };

    // the workspace is free once earlier computations' last kernels finished
    if ((e = cudaStreamWaitEvent(st, h->ws_free, 0)) != cudaSuccess) return fail(from_cuda(e));
    if (h->timing) {
        for (int q = 0; q < (fused ? 2 : 5); q++)
            if ((e = get_event(h, &L->ev[q], true)) != cudaSuccess) return fail(from_cuda(e));
        cudaEventRecord(L->ev[0], st);
    }
    // steps (a)+(c) and the node counts (the fused path runs every step
    // further down, once its result buffers exist)
    if (!fused && (es = run_part(0)) != EG_OK) return fail(es);
    if (h->timing && !fused) cudaEventRecord(L->ev[1], st);
    cudaEvent_t k1 = nullptr;
    if (!bounded) {
        if ((e = cudaEventCreateWithFlags(&k1, cudaEventDisableTiming)) != cudaSuccess) return fail(from_cuda(e));
        cudaEventRecord(k1, st);
    }
    // step (b) runs while the host reads the counts back (after the geometry
    // when that is wanted)
    if (!any_paths && !fused) {
        if ((es = run_part(1)) != EG_OK) {
            if (k1) cudaEventDestroy(k1);
            return fail(es);
        }
        if (h->timing) cudaEventRecord(L->ev[2], st);
    }
    if (bounded) {
        // M + S <= N (a vertex gives at most one record), P <= S times the
        // most components of an upper link
        Result &r = *res[0];
        const int d = jobs[0].sh.d;
        const uint64_t N = jobs[0].sh.N;
        r.M = N;
        r.S = N;
        r.P = N * uint64_t(d == 1 ? 2 : (d == 2 ? 3 : (d == 5 ? 20 : 10)));
        r.bounded = true;
    }
    void *hcounts = nullptr;
    if (!bounded && (e = h->hpool.alloc(&hcounts, sizeof(SmallBlock) * size_t(nf))) != cudaSuccess) {
        if (k1) cudaEventDestroy(k1);
        return fail(from_cuda(e));
    }
    if (!bounded) {
        cudaStreamWaitEvent(h->side, k1, 0);
        cudaMemcpyAsync(hcounts, L->smalls, sizeof(SmallBlock) * size_t(nf), cudaMemcpyDeviceToHost, h->side);
        e = cudaStreamSynchronize(h->side);
    }
    if (k1) cudaEventDestroy(k1);
    if (e != cudaSuccess) {
        h->hpool.release(hcounts);
        return fail(from_cuda(e));
    }
    eg_status first_err = EG_OK;
    for (int i = 0; i < nf && !bounded; i++) {
        const SmallBlock &sb = static_cast<SmallBlock *>(hcounts)[i];
        Result &r = *res[i];
        r.M = sb.totals[0];
        r.S = sb.totals[1];
        r.P = sb.totals[2];
        r.err = sb.err;
        if (sb.err & kErrNaN) first_err = EG_ERR_NAN;
        else if (sb.err & kErrTimeout) first_err = EG_ERR_TIMEOUT;
    }
    h->hpool.release(hcounts);
    if (first_err != EG_OK) return fail(first_err);

    // exact result buffers (and the per-result arc staging)
    for (int oi = 0; oi < nf; oi++) {
        Result &r = *res[order[oi]];
        FieldDev &F = Dh[oi];
        const size_t es = dtype_size(r.dtype);
        struct { void **p; size_t b; } want[] = {
            {&r.maxima, r.M * 4}, {&r.max_val, r.M * es}, {&r.saddles, r.S * 4}, {&r.sad_b0, r.S},
            {&r.sad_val, r.S * es}, {&r.row_ptr, (r.S + 1) * 8}, {&r.col, r.P * 4},
            {&r.ends, r.P * 4}, {&r.ucnt, r.S}};
        for (auto &w : want)
            if ((e = h->pool.alloc(w.p, std::max<size_t>(w.b, 8))) != cudaSuccess) return fail(from_cuda(e));
        F.maxima = static_cast<uint32_t *>(r.maxima);
        F.saddles = static_cast<uint32_t *>(r.saddles);
        F.sad_b0 = static_cast<uint8_t *>(r.sad_b0);
        // float32 value copies come with the records; other types are copied
        // from the field by the node kernel
        const bool f32 = r.dtype == kF32;
        F.max_val = f32 ? static_cast<float *>(r.max_val) : nullptr;
        F.sad_val = f32 ? static_cast<float *>(r.sad_val) : nullptr;
        F.max_raw = f32 ? nullptr : r.max_val;
        F.sad_raw = f32 ? nullptr : r.sad_val;
        F.row_ptr = static_cast<uint64_t *>(r.row_ptr);
        F.col = static_cast<uint32_t *>(r.col);
        F.ends = static_cast<uint32_t *>(r.ends);
        F.ucnt = static_cast<uint8_t *>(r.ucnt);
        if (r.flags & kFlagPaths) {
            if ((e = h->pool.alloc(&r.path_ptr, (r.P + 1) * 8)) != cudaSuccess) return fail(from_cuda(e));
            if ((e = h->pool.alloc(&r.pbrick, (uint64_t(F.nbricks) + 1) * 8)) != cudaSuccess)
                return fail(from_cuda(e));
            F.path_ptr = static_cast<uint64_t *>(r.path_ptr);
            F.pbrick = static_cast<uint64_t *>(r.pbrick);
        }
    }
    if (any_paths && (es = enqueue_paths(h, P, L.get(), Dh, res, order, st)) != EG_OK) return fail(es);
    if (any_paths) {
        if ((es = run_part(1)) != EG_OK) return fail(es);
        if (h->timing) cudaEventRecord(L->ev[2], st);
    }
    // phase 0 has finished (we waited for it), so the host table may change;
    // phase 2 uploads it again, ordered after resolution on the stream
    if (fused) {
        // every step in one launch, in the handle's current fused block
        // (status and barrier count zeroed by the launch before); the kernel
        // writes the counts and the status into the page-locked block itself
        // (which reads as a timeout until it does); the step timing reports
        // the whole kernel as classification, with one event after it
        SmallBlock *pair = static_cast<SmallBlock *>(h->fused_pair);
        SmallBlock *cur = pair + (h->fused_seq & 1u), *nxt = pair + ((h->fused_seq + 1u) & 1u);
        FieldDev &F = Dh[0];
        F.totals = cur->totals;
        F.err = &cur->err;
        SmallBlock *hb = static_cast<SmallBlock *>(L->hsmall_pin);
        std::memset(hb, 0, sizeof(SmallBlock));
        hb->err = kErrTimeout;
        if ((e = launch_small(F, cur->bar, &nxt->err, nxt->bar, hb->totals, &hb->err, h->sm_count, st)) !=
            cudaSuccess)
            return fail(from_cuda(e));
        h->fused_seq++;
        h->launches += 1;
        L->fused = true;
        if (h->timing) cudaEventRecord(L->ev[1], st);
    } else {
        if (h->timing) cudaEventRecord(L->ev[3], st);
        if ((es = run_part(2)) != EG_OK) return fail(es);
        if (h->timing) cudaEventRecord(L->ev[4], st);
    }
    cudaEventRecord(h->ws_free, st);
    // every result's counts and status word, read by collect() once `done`
    // fired (the fused kernel wrote them already)
    if (!fused && (e = cudaMemcpyAsync(L->hsmall_pin, L->smalls, sizeof(SmallBlock) * size_t(nf),
                                       cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return fail(from_cuda(e));
    ids.resize(nf);
    if ((e = get_event(h, &L->done, false)) != cudaSuccess) return fail(from_cuda(e));
    cudaEventRecord(L->done, st);
    for (int i = 0; i < nf; i++) res[i]->done = L->done;
    for (int i = 0; i < nf; i++) {
        uint64_t id = h->next_id++;
        ids[i] = id;
        h->results[id] = std::move(res[i]);
    }
    return EG_OK;
}

eg_status collect(eg_ctx *h, Result &r)
{
    cudaError_t e = cudaEventSynchronize(r.done);
    if (e != cudaSuccess) return from_cuda(e);
    if (!r.have_A) {
        // every result of the launch has finished with this one: read all
        // their SmallBlocks at once, the first time any of them is collected
        Launch &L = *r.launch;
        if (L.hsmall.empty()) {
            L.hsmall.resize(size_t(L.nsmall));
            std::memcpy(L.hsmall.data(), L.hsmall_pin, sizeof(SmallBlock) * size_t(L.nsmall));
        }
        const SmallBlock &sb = L.hsmall[size_t(r.slot)];
        if (r.bounded) {
            r.M = sb.totals[0];
            r.S = sb.totals[1];
            r.P = sb.totals[2];
        }
        r.A = sb.totals[3];
        r.err |= sb.err;
        r.have_A = true;
        h->pool.release(r.ends);
        h->pool.release(r.ucnt);
        h->pool.release(r.pbrick);
        h->pool.release(r.wide);
        r.ends = r.ucnt = r.pbrick = r.wide = nullptr;
        if (r.launch && r.launch.use_count() == 1) release_launch(h, r.launch.get());
    }
    if (r.err & kErrNaN) return EG_ERR_NAN;
    if (r.err & kErrNotConverged) return EG_ERR_NOT_CONVERGED;
    if (r.err & kErrTimeout) return EG_ERR_TIMEOUT;
    if (r.err & (kErrInternal | kErrBounds)) return EG_ERR_INTERNAL;
    return EG_OK;
}

void fill_counts(const Result &r, eg_graph *out)
{
    out->d = r.d;
    out->dtype = int32_t(r.dtype);
    for (int i = 0; i < kMaxDim; i++) out->extents[i] = r.ext[i];
    out->n_vertices = int64_t(r.N);
    out->n_maxima = int64_t(r.M);
    out->n_saddles = int64_t(r.S);
    out->n_paths = int64_t(r.P);
    out->n_arcs = int64_t(r.A);
}

}  // namespace

extern "C" {

const char *eg_status_str(eg_status s)
{
    switch (s) {
    case EG_OK: return "ok";
    case EG_ERR_ARG: return "invalid argument";
    case EG_ERR_NAN: return "field contains NaN";
    case EG_ERR_OOM: return "out of memory";
    case EG_ERR_CUDA: return "CUDA error";
    case EG_ERR_NOT_CONVERGED: return "gradient path resolution did not converge";
    case EG_ERR_TIMEOUT: return "device-side wait timed out";
    case EG_ERR_BUSY: return "not enough free device memory";
    case EG_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

eg_status eg_create(eg_handle *out, int device, const eg_config *cfg)
{
    if (!out) return EG_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return EG_ERR_CUDA;
    }
    if (device < 0 || device >= n) return EG_ERR_ARG;
    auto h = std::make_unique<eg_ctx>();
    h->device = device;
    if (cfg) h->cfg = *cfg;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return from_cuda(e);
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    if ((e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking)) != cudaSuccess) return from_cuda(e);
    if ((e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking)) != cudaSuccess) return from_cuda(e);
    if ((e = cudaEventCreateWithFlags(&h->ws_free, cudaEventDisableTiming)) != cudaSuccess) return from_cuda(e);
    cudaEventRecord(h->ws_free, h->side);
    {
        // saddle table of the 3D neighbourhood, 2 bits per upper-link mask m (14
        // neighbour slots): 0 fewer than two connected components, 1 exactly
        // two, 2 three or more; then, as 16-bit words, the component holding
        // the lowest set bit of every non-empty mask
        std::vector<uint32_t> lut(1024 + 8192, 0u);
        uint16_t *lowc = reinterpret_cast<uint16_t *>(lut.data() + 1024);
        for (uint32_t m = 0; m < (1u << 14); m++) {
            uint32_t left = m, comps = 0, first_comp = 0;
            while (left) {
                uint32_t comp = left & (~left + 1u), grow = comp;
                while (grow) {
                    const int k = __builtin_ctz(grow);
                    grow &= grow - 1;
                    const uint32_t nb = Nbr<3>::adj_mask(k) & m & ~comp;
                    comp |= nb;
                    grow |= nb;
                }
                left &= ~comp;
                if (comps == 0) first_comp = comp;
                comps++;
            }
            const uint32_t cls = comps < 2 ? 0u : (comps == 2 ? 1u : 2u);
            lut[m >> 4] |= cls << ((m & 15) * 2);
            lowc[m] = uint16_t(first_comp);
        }
        if ((e = h->pool.alloc(&h->lut3, lut.size() * 4)) != cudaSuccess) return from_cuda(e);
        if ((e = cudaMemcpy(h->lut3, lut.data(), lut.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
            return from_cuda(e);
    }
    if ((e = h->pool.alloc(&h->fused_pair, 2 * sizeof(SmallBlock))) != cudaSuccess) return from_cuda(e);
    if ((e = cudaMemset(h->fused_pair, 0, 2 * sizeof(SmallBlock))) != cudaSuccess) return from_cuda(e);
    *out = h.release();
    return EG_OK;
}

eg_status eg_destroy(eg_handle h)
{
    if (!h) return EG_OK;
    {
        std::lock_guard<std::mutex> g(h->mu);
        cudaSetDevice(h->device);
        cudaDeviceSynchronize();
        h->results.clear();  // (their launches return their events to the pools)
        for (auto &pool : h->ev_pool)
            for (cudaEvent_t e : pool) cudaEventDestroy(e);
        if (h->graphs) {
            for (auto &kv : h->graphs->entries) destroy_graph(h, kv.second);
            h->graphs.reset();
        }
        if (h->cap) cudaStreamDestroy(h->cap);
        h->pool.destroy();
        h->hpool.destroy();
        if (h->stage) cudaFree(h->stage);
        if (h->hstage) cudaFreeHost(h->hstage);
        if (h->side) cudaStreamDestroy(h->side);
        if (h->ws_free) cudaEventDestroy(h->ws_free);
    }
    delete h;
    return EG_OK;
}

eg_status eg_compute(eg_handle h, const float *field, int d, const int64_t *extents, void *stream,
                     eg_result_id *out)
{
    if (!h || !field || !out) return EG_ERR_ARG;
    Shape sh;
    if (!make_shape(d, extents, sh)) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    std::vector<Job> jobs{{field, sh, h->cfg.flags & (kFlagMinimum | kFlagNoLabels | kFlagPaths)}};
    std::vector<uint64_t> ids;
    eg_status s = run_jobs(h, jobs, static_cast<cudaStream_t>(stream), ids, h->cfg, false, true);
    if (s == EG_OK) *out = ids[0];
    return s;
}

size_t eg_dtype_size(int dtype)
{
    return dtype >= 0 && dtype < int(kNumTypes) ? dtype_size(uint32_t(dtype)) : 0;
}

eg_status eg_compute_typed(eg_handle h, const void *field, int dtype, int d, const int64_t *extents,
                           void *stream, eg_result_id *out)
{
    if (!h || !field || !out || dtype < 0 || dtype >= int(kNumTypes)) return EG_ERR_ARG;
    if (reinterpret_cast<uintptr_t>(field) % dtype_size(uint32_t(dtype)) != 0) return EG_ERR_ARG;
    Shape sh;
    if (!make_shape(d, extents, sh)) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    std::vector<Job> jobs{{field, sh, h->cfg.flags & (kFlagMinimum | kFlagNoLabels | kFlagPaths), uint32_t(dtype)}};
    std::vector<uint64_t> ids;
    eg_status s = run_jobs(h, jobs, static_cast<cudaStream_t>(stream), ids, h->cfg, false, true);
    if (s == EG_OK) *out = ids[0];
    return s;
}

eg_status eg_compute_host(eg_handle h, const float *field, int d, const int64_t *extents, void *stream,
                          eg_result_id *out)
{
    if (!h || !field || !out) return EG_ERR_ARG;
    Shape sh;
    if (!make_shape(d, extents, sh)) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sh.N * sizeof(float);
    // the staging buffer may still feed an earlier computation
    cudaEventSynchronize(h->ws_free);
    if (h->stage_bytes < bytes) {
        if (h->stage) cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        cudaError_t e = cudaMalloc(&h->stage, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return from_cuda(e);
        }
        h->stage_bytes = bytes;
    }
    cudaPointerAttributes pa{};
    bool pinned = cudaPointerGetAttributes(&pa, field) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();
    const void *src = field;
    if (!pinned) {
        if (h->hstage_bytes < bytes) {
            if (h->hstage) cudaFreeHost(h->hstage);
            h->hstage = nullptr;
            h->hstage_bytes = 0;
            cudaError_t e = cudaHostAlloc(&h->hstage, bytes, cudaHostAllocDefault);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return from_cuda(e);
            }
            h->hstage_bytes = bytes;
        }
        std::memcpy(h->hstage, field, bytes);
        src = h->hstage;
    }
    cudaError_t e = cudaMemcpyAsync(h->stage, src, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    std::vector<Job> jobs{{static_cast<const float *>(h->stage), sh, h->cfg.flags & (kFlagMinimum | kFlagNoLabels | kFlagPaths)}};
    std::vector<uint64_t> ids;
    // (not bounded: the staging buffer is reused by the next call, so the
    // call returns only after classification has read it)
    eg_status s = run_jobs(h, jobs, st, ids, h->cfg);
    if (s == EG_OK) *out = ids[0];
    return s;
}

}  // extern "C"

namespace {

// A batch descriptor as a job; false on a bad field.
bool job_of(eg_ctx *h, const eg_field_desc &fd, Job &j)
{
    if (!fd.field || !make_shape(fd.d, fd.extents, j.sh)) return false;
    const uint32_t dt = (uint32_t(fd.flags) & EG_FLAG_DTYPE_MASK) >> 16;
    if (dt >= kNumTypes || reinterpret_cast<uintptr_t>(fd.field) % dtype_size(dt) != 0) return false;
    j.field = fd.field;
    j.dtype = dt;
    j.flags = (h->cfg.flags | uint32_t(fd.flags)) & (kFlagMinimum | kFlagNoLabels | kFlagPaths);
    return true;
}

// Counts and library-owned device pointers of result `id` (waits for it).
eg_status device_view(eg_ctx *h, eg_result_id id, eg_graph *out)
{
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    eg_status s = collect(h, r);
    fill_counts(r, out);
    if (s != EG_OK) return s;
    out->maxima = static_cast<uint32_t *>(r.maxima);
    out->max_val = r.max_val;
    out->saddles = static_cast<uint32_t *>(r.saddles);
    out->sad_beta0 = static_cast<uint8_t *>(r.sad_b0);
    out->sad_val = r.sad_val;
    out->row_ptr = static_cast<uint64_t *>(r.row_ptr);
    out->col = static_cast<uint32_t *>(r.col);
    out->labels = static_cast<uint32_t *>(r.lab);
    return EG_OK;
}

}  // namespace

extern "C" {

eg_status eg_batch_submit(eg_handle h, const eg_field_desc *fields, int n, void *stream, eg_result_id *out_ids)
{
    if (!h || (n > 0 && (!fields || !out_ids)) || n < 0) return EG_ERR_ARG;
    if (n == 0) return EG_OK;
    std::vector<Job> jobs(n);
    for (int i = 0; i < n; i++)
        if (!job_of(h, fields[i], jobs[i])) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    std::vector<uint64_t> ids;
    const bool graph = !(h->cfg.flags & EG_FLAG_NO_GRAPH);
    eg_status s = run_jobs(h, jobs, static_cast<cudaStream_t>(stream), ids, h->cfg, graph);
    if (s == EG_OK)
        for (int i = 0; i < n; i++) out_ids[i] = ids[i];
    return s;
}

namespace {

// ev: start | classify | resolve | (count read-back, buffer set-up) | emit;
// a fused launch records start | whole kernel, reported as classification.
eg_status event_times(const Launch &L, float ms[4])
{
    const cudaEvent_t last = L.fused ? L.ev[1] : L.ev[4];
    cudaError_t e = cudaEventSynchronize(last);
    if (e != cudaSuccess) return from_cuda(e);
    float a = 0, b = 0, c = 0, t = 0;
    cudaEventElapsedTime(&a, L.ev[0], L.ev[1]);
    if (!L.fused) {
        cudaEventElapsedTime(&b, L.ev[1], L.ev[2]);
        cudaEventElapsedTime(&c, L.ev[3], L.ev[4]);
    }
    cudaEventElapsedTime(&t, L.ev[0], last);
    ms[0] = a;
    ms[1] = b;
    ms[2] = c;
    ms[3] = t;
    return EG_OK;
}

// Device milliseconds of the steps of one launch (timing must have been on).
eg_status launch_times(const Launch &L, float ms[4])
{
    if (!L.ev[0]) return EG_ERR_ARG;
    return event_times(L, ms);
}

// One timed run of the whole pipeline on `jobs` with configuration c; the
// results are released.  *ms receives the step times of the fastest of `reps`
// repetitions (by total).
eg_status timed_trial(eg_ctx *h, const std::vector<Job> &jobs, cudaStream_t st, const eg_config &c, int reps,
                      float ms[4])
{
    ms[0] = ms[1] = ms[2] = ms[3] = 1e30f;
    for (int r = 0; r < reps; r++) {
        std::vector<uint64_t> ids;
        eg_status s = run_jobs(h, jobs, st, ids, c);
        if (s != EG_OK) return s;
        float t[4] = {0, 0, 0, 0};
        eg_status ts = launch_times(*h->results[ids[0]]->launch, t);
        for (uint64_t id : ids) {
            Result &R = *h->results[id];
            eg_status cs = collect(h, R);
            free_result_buffers(h, &R);
            if (R.launch && R.launch.use_count() == 1) release_launch(h, R.launch.get());
            h->results.erase(id);
            if (cs != EG_OK) return cs;
        }
        if (ts != EG_OK) return ts;
        if (t[3] < ms[3])
            for (int k = 0; k < 4; k++) ms[k] = t[k];
    }
    return EG_OK;
}

}  // namespace

eg_status eg_autotune(eg_handle h, const eg_field_desc *fields, int n, void *stream, eg_config *best)
{
    if (!h || n <= 0 || !fields) return EG_ERR_ARG;
    std::vector<Job> jobs(n);
    for (int i = 0; i < n; i++)
        if (!job_of(h, fields[i], jobs[i])) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool saved_timing = h->timing;
    h->timing = true;
    eg_config cur = h->cfg;
    if (cur.resolve_walks <= 0) cur.resolve_walks = 4;
    if (cur.persistent_ctas <= 0) cur.persistent_ctas = 3;
    float ms[4];
    eg_status s = timed_trial(h, jobs, st, cur, 2, ms);  // also warms the workspace
    float cur_total = ms[3];
    // coordinate descent: one knob at a time, the others at their current best
    struct Knob { int32_t eg_config::*field; std::vector<int32_t> values; };
    const std::vector<Knob> knobs = {
        {&eg_config::classify_planes, {0, 16, 32, 64, 128}},
        {&eg_config::classify_rows, {0, 8, 4, 2}},
        {&eg_config::persistent_ctas, {2, 3}},
        {&eg_config::resolve_walks, {2, 4, 8}},
    };
    for (const Knob &k : knobs) {
        if (s != EG_OK) break;
        for (int32_t v : k.values) {
            if (cur.*(k.field) == v) continue;
            eg_config c = cur;
            c.*(k.field) = v;
            s = timed_trial(h, jobs, st, c, 2, ms);
            if (s != EG_OK) break;
            if (ms[3] < cur_total) {
                cur = c;
                cur_total = ms[3];
            }
        }
    }
    h->timing = saved_timing;
    if (s != EG_OK) return s;
    h->cfg = cur;
    if (best) *best = cur;
    return EG_OK;
}

eg_status eg_get_graph(eg_handle h, eg_result_id id, eg_graph *out)
{
    if (!h || !out) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    eg_status s = collect(h, r);
    fill_counts(r, out);
    if (s != EG_OK) return s;
    const size_t es = dtype_size(r.dtype);
    struct { void *dst; const void *src; size_t b; } cp[] = {
        {out->maxima, r.maxima, r.M * 4}, {out->max_val, r.max_val, r.M * es},
        {out->saddles, r.saddles, r.S * 4}, {out->sad_beta0, r.sad_b0, r.S},
        {out->sad_val, r.sad_val, r.S * es}, {out->row_ptr, r.row_ptr, (r.S + 1) * 8},
        {out->col, r.col, r.A * 4}, {out->labels, r.lab, r.N * 4}};
    // all copies in flight at once on the side stream (they overlap when the
    // destinations are pinned), then one wait
    for (auto &c : cp)
        if (c.dst && c.b) {
            cudaError_t e = cudaMemcpyAsync(c.dst, c.src, c.b, cudaMemcpyDeviceToHost, h->side);
            if (e != cudaSuccess) {
                cudaStreamSynchronize(h->side);
                return from_cuda(e);
            }
        }
    cudaError_t e = cudaStreamSynchronize(h->side);
    return e == cudaSuccess ? EG_OK : from_cuda(e);
}

eg_status eg_get_paths(eg_handle h, eg_result_id id, uint64_t *path_ptr, uint32_t *path_vtx,
                       uint64_t *n_path_vertices)
{
    if (!h || !n_path_vertices) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    if (!r.path_ptr) return EG_ERR_ARG;
    eg_status s = collect(h, r);
    *n_path_vertices = r.V;
    if (s != EG_OK) return s;
    if (path_ptr) {
        cudaError_t e = cudaMemcpyAsync(path_ptr, r.path_ptr, (r.P + 1) * 8, cudaMemcpyDeviceToHost, h->side);
        if (e != cudaSuccess) return from_cuda(e);
    }
    if (path_vtx && r.V) {
        cudaError_t e = cudaMemcpyAsync(path_vtx, r.path_vtx, r.V * 4, cudaMemcpyDeviceToHost, h->side);
        if (e != cudaSuccess) return from_cuda(e);
    }
    cudaError_t e = cudaStreamSynchronize(h->side);
    return e == cudaSuccess ? EG_OK : from_cuda(e);
}

eg_status eg_get_bundled(eg_handle h, eg_result_id id, uint8_t *keep)
{
    if (!h) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    eg_status s = collect(h, r);
    if (s != EG_OK) return s;
    if (r.S == 0) return EG_OK;
    if (!keep) return EG_ERR_ARG;
    cudaStream_t st = h->side;
    void *small = nullptr, *keys = nullptr, *best = nullptr, *dkeep = nullptr, *best_id = nullptr;
    auto done = [&](eg_status x) {
        cudaStreamSynchronize(st);
        for (void *p : {small, keys, best, dkeep, best_id}) h->pool.release(p);
        return x;
    };
    cudaError_t e;
    // [0] pair count, [1] status word
    if ((e = h->pool.alloc(&small, 16)) != cudaSuccess) return done(from_cuda(e));
    unsigned long long *cnt = static_cast<unsigned long long *>(small);
    uint32_t *err = reinterpret_cast<uint32_t *>(cnt + 1);
    if ((e = cudaMemsetAsync(small, 0, 16, st)) != cudaSuccess) return done(from_cuda(e));
    const uint64_t *row_ptr = static_cast<const uint64_t *>(r.row_ptr);
    if ((e = launch_bundle_pairs(row_ptr, r.S, cnt, st)) != cudaSuccess) return done(from_cuda(e));
    unsigned long long pairs = 0;
    if ((e = cudaMemcpyAsync(&pairs, cnt, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return done(from_cuda(e));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(from_cuda(e));
    uint32_t lg = 10;
    while ((1ull << lg) < 2 * pairs) lg++;
    const size_t tb = size_t(8) << lg;
    if ((e = h->pool.alloc(&keys, tb)) != cudaSuccess) return done(from_cuda(e));
    if ((e = h->pool.alloc(&best, tb)) != cudaSuccess) return done(from_cuda(e));
    if ((e = h->pool.alloc(&dkeep, r.S)) != cudaSuccess) return done(from_cuda(e));
    if ((e = cudaMemsetAsync(keys, 0xff, tb, st)) != cudaSuccess) return done(from_cuda(e));
    if ((e = cudaMemsetAsync(best, 0, tb, st)) != cudaSuccess) return done(from_cuda(e));
    if (r.dtype == kF32) {
        if ((e = launch_bundle(row_ptr, static_cast<const uint32_t *>(r.col),
                               static_cast<const uint32_t *>(r.saddles), static_cast<const float *>(r.sad_val), r.S,
                               (r.flags & kFlagMinimum) != 0, static_cast<unsigned long long *>(keys),
                               static_cast<unsigned long long *>(best), lg, static_cast<uint8_t *>(dkeep), err,
                               st)) != cudaSuccess)
            return done(from_cuda(e));
        h->launches += 3;
    } else {
        if ((e = h->pool.alloc(&best_id, size_t(4) << lg)) != cudaSuccess) return done(from_cuda(e));
        if ((e = cudaMemsetAsync(best_id, 0, size_t(4) << lg, st)) != cudaSuccess) return done(from_cuda(e));
        if ((e = launch_bundle_typed(r.dtype, row_ptr, static_cast<const uint32_t *>(r.col),
                                     static_cast<const uint32_t *>(r.saddles), r.sad_val, r.S,
                                     (r.flags & kFlagMinimum) != 0, static_cast<unsigned long long *>(keys),
                                     static_cast<unsigned long long *>(best), static_cast<unsigned int *>(best_id),
                                     lg, static_cast<uint8_t *>(dkeep), err, st)) != cudaSuccess)
            return done(from_cuda(e));
        h->launches += 4;
    }
    uint32_t herr = 0;
    if ((e = cudaMemcpyAsync(keep, dkeep, r.S, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return done(from_cuda(e));
    if ((e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return done(from_cuda(e));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(from_cuda(e));
    return done(herr ? EG_ERR_INTERNAL : EG_OK);
}

eg_status eg_get_cancelled(eg_handle h, eg_result_id id, float tau, uint8_t *alive, uint32_t *survivor,
                           int64_t *n_cancelled, int32_t *n_rounds)
{
    if (!h || tau != tau) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    eg_status s = collect(h, r);
    if (s != EG_OK) return s;
    if (r.dtype != kF32 || (r.S && !alive) || (r.M && !survivor)) return EG_ERR_ARG;
    cudaStream_t st = h->side;
    constexpr int kBufs = 17;
    void *buf[kBufs] = {};
    auto done = [&](eg_status x) {
        cudaStreamSynchronize(st);
        for (void *p : buf) h->pool.release(p);
        return x;
    };
    const uint64_t M = r.M, S = r.S, A = r.A;
    const size_t sizes[kBufs] = {4 * A, 4 * A, 4 * M, 8 * M, 8 * M, 8 * S, 8 * S, 4 * S, S,
                                 4 * S, 4 * S, 128, S, 4 * M, 4 * A, 8 * M, 8 * M};
    cudaError_t e;
    for (int i = 0; i < kBufs; i++)
        if ((e = h->pool.alloc(&buf[i], std::max<size_t>(sizes[i], 16))) != cudaSuccess) return done(from_cuda(e));
    CancelDev C{};
    C.maxima = static_cast<const uint32_t *>(r.maxima);
    C.max_val = static_cast<const float *>(r.max_val);
    C.sad_val = static_cast<const float *>(r.sad_val);
    C.row_ptr = static_cast<const uint64_t *>(r.row_ptr);
    C.end = static_cast<uint32_t *>(buf[0]);
    C.aroot[0] = static_cast<uint32_t *>(buf[1]);
    C.aroot[1] = static_cast<uint32_t *>(buf[14]);
    C.parent = static_cast<uint32_t *>(buf[2]);
    C.minlb[0] = static_cast<unsigned long long *>(buf[3]);
    C.minlb[1] = static_cast<unsigned long long *>(buf[15]);
    C.min2[0] = static_cast<unsigned long long *>(buf[4]);
    C.min2[1] = static_cast<unsigned long long *>(buf[16]);
    C.costkey = static_cast<unsigned long long *>(buf[5]);
    C.lbkey = static_cast<unsigned long long *>(buf[6]);
    C.high = static_cast<uint32_t *>(buf[7]);
    C.state = static_cast<uint8_t *>(buf[8]);
    C.list[0] = static_cast<uint32_t *>(buf[9]);
    C.list[1] = static_cast<uint32_t *>(buf[10]);
    C.ctrl = static_cast<unsigned long long *>(buf[11]);
    C.err = reinterpret_cast<uint32_t *>(C.ctrl + 12);
    C.M = uint32_t(M);
    C.S = uint32_t(S);
    C.tau = tau;
    C.minimum = (r.flags & kFlagMinimum) ? 1 : 0;
    // round slot 0 = {no key, 0, 0}, the rest (rounds, barrier, status) zero
    unsigned long long ctrl0[13] = {};
    ctrl0[0] = ~0ull;
    if ((e = cudaMemcpyAsync(C.ctrl, ctrl0, sizeof ctrl0, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return done(from_cuda(e));
    if ((e = launch_cancel_setup(C, static_cast<const uint32_t *>(r.col), A, st)) != cudaSuccess)
        return done(from_cuda(e));
    if ((e = launch_cancel_rounds(C, h->sm_count, st)) != cudaSuccess) return done(from_cuda(e));
    h->launches += 3;
    uint8_t *dalive = static_cast<uint8_t *>(buf[12]);
    uint32_t *dsurv = static_cast<uint32_t *>(buf[13]);
    if ((e = launch_cancel_out(C, dalive, dsurv, st)) != cudaSuccess) return done(from_cuda(e));
    h->launches += 1;
    uint32_t herr = 0;
    if (S && (e = cudaMemcpyAsync(alive, dalive, S, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return done(from_cuda(e));
    if (M && (e = cudaMemcpyAsync(survivor, dsurv, 4 * M, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return done(from_cuda(e));
    if ((e = cudaMemcpyAsync(&herr, C.err, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return done(from_cuda(e));
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return done(from_cuda(e));
    if (herr & kErrTimeout) return done(EG_ERR_TIMEOUT);
    if (herr) return done(EG_ERR_INTERNAL);
    if (n_cancelled) {
        int64_t c = 0;
        for (uint64_t i = 0; i < S; i++) c += alive[i] ? 0 : 1;
        *n_cancelled = c;
    }
    if (n_rounds) {
        unsigned long long rounds = 0;
        if ((e = cudaMemcpy(&rounds, C.ctrl + 9, 8, cudaMemcpyDeviceToHost)) != cudaSuccess) return done(from_cuda(e));
        *n_rounds = int32_t(rounds);
    }
    return done(EG_OK);
}

eg_status eg_get_graph_device(eg_handle h, eg_result_id id, eg_graph *out)
{
    if (!h || !out) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    return device_view(h, id, out);
}

eg_status eg_get_graphs_device(eg_handle h, const eg_result_id *ids, int n, eg_graph *out, int32_t *status)
{
    if (!h || n < 0 || (n > 0 && (!ids || !out))) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    eg_status first = EG_OK;
    for (int i = 0; i < n; i++) {
        const eg_status s = device_view(h, ids[i], out + i);
        if (status) status[i] = int32_t(s);
        if (s != EG_OK && first == EG_OK) first = s;
    }
    return first;
}

eg_status eg_release(eg_handle h, eg_result_id id)
{
    if (!h) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    if (r.done) cudaEventSynchronize(r.done);
    free_result_buffers(h, &r);
    if (r.launch && r.launch.use_count() == 1) release_launch(h, r.launch.get());
    h->results.erase(it);
    return EG_OK;
}

uint64_t eg_workspace_bytes(int d, const int64_t *extents)
{
    Shape sh;
    if (!make_shape(d, extents, sh)) return 0;
    eg_config cfg{};
    const Layout ly = make_layout(sh, 152, cfg);
    const uint64_t recs = uint64_t(ly.nbricks) * ly.bcap;
    // records (id, info, value) + per-brick counts/offsets + scan state + labels
    return recs * (4 + 8 + 4) + uint64_t(ly.nbricks) * (16 + 16 + 4 + 8) +
           scan_workspace_bytes(scan_tiles(ly.nbricks)) + sh.N * 4;
}

eg_status eg_mem_info(eg_handle h, uint64_t *free_bytes, uint64_t *total_bytes, uint64_t *held_bytes)
{
    if (!h) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    size_t fr = 0, to = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &to);
    if (e != cudaSuccess) return from_cuda(e);
    if (free_bytes) *free_bytes = fr;
    if (total_bytes) *total_bytes = to;
    if (held_bytes) *held_bytes = h->pool.held;
    return EG_OK;
}

eg_status eg_set_timing(eg_handle h, int enable)
{
    if (!h) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    h->timing = enable != 0;
    return EG_OK;
}

eg_status eg_step_times(eg_handle h, eg_result_id id, float ms[4])
{
    if (!h || !ms) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end() || !it->second->launch || !it->second->launch->ev[0]) return EG_ERR_ARG;
    return event_times(*it->second->launch, ms);
}

uint64_t eg_launch_count(eg_handle h) { return h ? h->launches.load() : 0; }

eg_status eg_debug_wait_timeout(eg_handle h, void *stream)
{
    if (!h) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *buf = nullptr;
    cudaError_t e = h->pool.alloc(&buf, 256);
    if (e != cudaSuccess) return from_cuda(e);
    uint64_t *status = static_cast<uint64_t *>(buf);   // two look-back words, both empty
    uint32_t *err = reinterpret_cast<uint32_t *>(static_cast<char *>(buf) + 64);
    uint32_t herr = 0;
    e = cudaMemsetAsync(buf, 0, 256, st);
    if (e == cudaSuccess) e = launch_lookback_orphan(status, err, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    h->pool.release(buf);
    if (e != cudaSuccess) return from_cuda(e);
    return (herr & kErrTimeout) ? EG_ERR_TIMEOUT : EG_OK;
}

eg_status eg_debug_fail_alloc(eg_handle h, int k)
{
    if (!h || k < 0) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    h->pool.fail_in = k;
    return EG_OK;
}

}  // extern "C"
