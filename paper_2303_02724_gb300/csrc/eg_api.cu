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
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/eg.h"
#include "eg_internal.cuh"
#include "eg_kernels.h"

using namespace eg;

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

// Per-field small device block: totals[4] (M, S, P, A) + status word.
struct alignas(16) SmallBlock {
    unsigned long long totals[4];
    uint32_t err;
    uint32_t pad[7];
};

struct Result {
    int d = 0;
    int64_t ext[kMaxDim] = {0, 0, 0, 0};
    uint64_t N = 0;
    uint32_t flags = 0;
    void *lab = nullptr;
    void *small = nullptr;  // SmallBlock on device
    void *maxima = nullptr, *max_val = nullptr, *saddles = nullptr, *sad_b0 = nullptr, *sad_val = nullptr,
         *row_ptr = nullptr, *col = nullptr;
    uint64_t M = 0, S = 0, P = 0, A = 0;
    bool have_A = false;
    uint32_t err = 0;
    cudaEvent_t done = nullptr;
    std::shared_ptr<struct Launch> launch;  // keeps the descriptor table alive
};

// Descriptor tables of one launch (shared by the results of a batch).
struct Launch {
    void *desc_dev = nullptr;
    void *desc_host = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // step timing (optional)
    ~Launch()
    {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
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
    void *ws_rec_sid = nullptr, *ws_rec_info = nullptr, *ws_bcnt = nullptr, *ws_emit = nullptr;
    uint64_t ws_bricks = 0;
    void *stage = nullptr;  // device staging for eg_compute_host
    size_t stage_bytes = 0;
    void *hstage = nullptr;  // pinned staging for pageable host fields
    size_t hstage_bytes = 0;
    std::unordered_map<uint64_t, std::unique_ptr<Result>> results;
    uint64_t next_id = 1;
    std::atomic<uint64_t> launches{0};
    bool timing = false;
};

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
    sh.d = d;
    sh.N = N;
    return true;
}

uint64_t bricks_of(uint64_t N) { return (N + kBrick - 1) / kBrick; }

eg_status ensure_workspace(eg_ctx *h, uint64_t bricks, cudaStream_t st)
{
    if (bricks <= h->ws_bricks) return EG_OK;
    // previous computations may still read the old workspace
    cudaEventSynchronize(h->ws_free);
    h->pool.release(h->ws_rec_sid);
    h->pool.release(h->ws_rec_info);
    h->pool.release(h->ws_bcnt);
    h->pool.release(h->ws_emit);
    h->ws_rec_sid = h->ws_rec_info = h->ws_bcnt = h->ws_emit = nullptr;
    h->ws_bricks = 0;
    uint64_t cap = std::max<uint64_t>(bricks, 16);
    cudaError_t e;
    if ((e = h->pool.alloc(&h->ws_rec_sid, cap * kBrick * sizeof(uint32_t))) != cudaSuccess) return from_cuda(e);
    if ((e = h->pool.alloc(&h->ws_rec_info, cap * kBrick * sizeof(uint64_t))) != cudaSuccess) return from_cuda(e);
    if ((e = h->pool.alloc(&h->ws_bcnt, cap * sizeof(uint4))) != cudaSuccess) return from_cuda(e);
    if ((e = h->pool.alloc(&h->ws_emit, emit_workspace_bytes(cap) + 256 * kMaxDim)) != cudaSuccess)
        return from_cuda(e);
    h->ws_bricks = cap;
    (void)st;
    return EG_OK;
}

void free_result_buffers(eg_ctx *h, Result *r)
{
    void **bufs[] = {&r->lab, &r->small, &r->maxima, &r->max_val, &r->saddles,
                     &r->sad_b0, &r->sad_val, &r->row_ptr, &r->col};
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
    L->desc_dev = L->desc_host = nullptr;
}

struct Job {
    const float *field;
    Shape sh;
    uint32_t flags;
};

// Run a set of fields (all of one call) through the three steps.
eg_status run_jobs(eg_ctx *h, const std::vector<Job> &jobs, cudaStream_t st, std::vector<uint64_t> &ids)
{
    const int nf = int(jobs.size());
    // order fields by dimension so every launch covers a contiguous slice
    std::vector<int> order(nf);
    for (int i = 0; i < nf; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].sh.d < jobs[b].sh.d; });

    uint64_t total_bricks = 0;
    for (auto &j : jobs) total_bricks += bricks_of(j.sh.N);
    eg_status es = ensure_workspace(h, total_bricks, st);
    if (es != EG_OK) return es;

    auto L = std::make_shared<Launch>();
    L->bytes = sizeof(FieldDev) * size_t(nf);
    cudaError_t e;
    std::vector<std::unique_ptr<Result>> res(nf);
    auto fail = [&](eg_status s) {
        cudaStreamSynchronize(st);
        for (auto &r : res)
            if (r) {
                free_result_buffers(h, r.get());
                if (r->done) cudaEventDestroy(r->done);
            }
        release_launch(h, L.get());
        return s;
    };
    if ((e = h->pool.alloc(&L->desc_dev, L->bytes)) != cudaSuccess) return fail(from_cuda(e));
    if ((e = h->hpool.alloc(&L->desc_host, L->bytes)) != cudaSuccess) return fail(from_cuda(e));
    FieldDev *D = reinterpret_cast<FieldDev *>(L->desc_host);
    std::memset(D, 0, L->bytes);

    // per-dimension groups: brick0 is relative to the group's first field
    uint64_t ws_off = 0;  // brick offset into the shared workspace
    struct Group { int d, first, count; uint64_t bricks, ws0; };
    std::vector<Group> groups;
    for (int oi = 0; oi < nf; oi++) {
        const Job &j = jobs[order[oi]];
        if (groups.empty() || groups.back().d != j.sh.d) groups.push_back({j.sh.d, oi, 0, 0, ws_off});
        Group &G = groups.back();
        auto r = std::make_unique<Result>();
        r->d = j.sh.d;
        for (int i = 0; i < kMaxDim; i++) r->ext[i] = i < j.sh.d ? j.sh.n[i] : 0;
        r->N = j.sh.N;
        r->flags = j.flags;
        r->launch = L;
        if ((e = h->pool.alloc(&r->lab, j.sh.N * sizeof(uint32_t))) != cudaSuccess) {
            res[order[oi]] = std::move(r);
            return fail(from_cuda(e));
        }
        if ((e = h->pool.alloc(&r->small, sizeof(SmallBlock))) != cudaSuccess) {
            res[order[oi]] = std::move(r);
            return fail(from_cuda(e));
        }
        FieldDev &F = D[oi];
        F.f = j.field;
        F.lab = static_cast<uint32_t *>(r->lab);
        F.rec_sid = static_cast<uint32_t *>(h->ws_rec_sid) + ws_off * kBrick;
        F.rec_info = static_cast<uint64_t *>(h->ws_rec_info) + ws_off * kBrick;
        F.bcnt = static_cast<uint4 *>(h->ws_bcnt) + ws_off;
        F.totals = reinterpret_cast<SmallBlock *>(r->small)->totals;
        F.err = &reinterpret_cast<SmallBlock *>(r->small)->err;
        for (int i = 0; i < kMaxDim; i++) {
            F.n[i] = j.sh.n[i];
            F.s[i] = j.sh.s[i];
        }
        F.N = uint32_t(j.sh.N);
        F.nbricks = uint32_t(bricks_of(j.sh.N));
        F.brick0 = G.bricks;
        F.d = j.sh.d;
        F.flags = j.flags;
        G.bricks += F.nbricks;
        G.count++;
        ws_off += F.nbricks;
        res[order[oi]] = std::move(r);
    }

    // the workspace is free once earlier computations' emit kernels finished
    if ((e = cudaStreamWaitEvent(st, h->ws_free, 0)) != cudaSuccess) return fail(from_cuda(e));
    for (int i = 0; i < nf; i++)
        if ((e = cudaMemsetAsync(res[i]->small, 0, sizeof(SmallBlock), st)) != cudaSuccess) return fail(from_cuda(e));
    if ((e = cudaMemcpyAsync(L->desc_dev, L->desc_host, L->bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(from_cuda(e));
    const FieldDev *Ddev = static_cast<const FieldDev *>(L->desc_dev);
    if (h->timing) {
        for (auto &ev : L->ev)
            if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(from_cuda(e));
        cudaEventRecord(L->ev[0], st);
    }
    for (auto &G : groups) {
        if ((e = launch_classify_d(G.d, Ddev + G.first, G.count, G.bricks, st)) != cudaSuccess) return fail(from_cuda(e));
        h->launches++;
    }
    cudaEvent_t k1;
    if ((e = cudaEventCreateWithFlags(&k1, cudaEventDisableTiming)) != cudaSuccess) return fail(from_cuda(e));
    cudaEventRecord(k1, st);
    if (h->timing) cudaEventRecord(L->ev[1], st);
    for (auto &G : groups) {
        if ((e = launch_resolve(Ddev + G.first, G.count, G.bricks, st)) != cudaSuccess) {
            cudaEventDestroy(k1);
            return fail(from_cuda(e));
        }
        h->launches++;
    }
    if (h->timing) cudaEventRecord(L->ev[2], st);
    // node counts: side stream waits for classify only
    void *hcounts = nullptr;
    if ((e = h->hpool.alloc(&hcounts, sizeof(SmallBlock) * size_t(nf))) != cudaSuccess) {
        cudaEventDestroy(k1);
        return fail(from_cuda(e));
    }
    cudaStreamWaitEvent(h->side, k1, 0);
    for (int i = 0; i < nf; i++)
        cudaMemcpyAsync(static_cast<SmallBlock *>(hcounts) + i, res[i]->small, sizeof(SmallBlock),
                        cudaMemcpyDeviceToHost, h->side);
    e = cudaStreamSynchronize(h->side);
    cudaEventDestroy(k1);
    if (e != cudaSuccess) {
        h->hpool.release(hcounts);
        return fail(from_cuda(e));
    }
    eg_status first_err = EG_OK;
    for (int i = 0; i < nf; i++) {
        const SmallBlock &sb = static_cast<SmallBlock *>(hcounts)[i];
        Result &r = *res[i];
        r.M = sb.totals[0];
        r.S = sb.totals[1];
        r.P = sb.totals[2];
        r.err = sb.err;
        if (sb.err & kErrNaN) first_err = EG_ERR_NAN;
    }
    h->hpool.release(hcounts);
    if (first_err != EG_OK) return fail(first_err);

    // exact result buffers
    for (int oi = 0; oi < nf; oi++) {
        Result &r = *res[order[oi]];
        FieldDev &F = D[oi];
        struct { void **p; size_t b; } want[] = {
            {&r.maxima, r.M * 4}, {&r.max_val, r.M * 4}, {&r.saddles, r.S * 4}, {&r.sad_b0, r.S},
            {&r.sad_val, r.S * 4}, {&r.row_ptr, (r.S + 1) * 8}, {&r.col, r.P * 4}};
        for (auto &w : want)
            if ((e = h->pool.alloc(w.p, std::max<size_t>(w.b, 4))) != cudaSuccess) return fail(from_cuda(e));
        F.maxima = static_cast<uint32_t *>(r.maxima);
        F.max_val = static_cast<float *>(r.max_val);
        F.saddles = static_cast<uint32_t *>(r.saddles);
        F.sad_b0 = static_cast<uint8_t *>(r.sad_b0);
        F.sad_val = static_cast<float *>(r.sad_val);
        F.row_ptr = static_cast<uint64_t *>(r.row_ptr);
        F.col = static_cast<uint32_t *>(r.col);
    }
    // classify has finished (we waited for it), so the host table may change
    if ((e = cudaMemcpyAsync(L->desc_dev, L->desc_host, L->bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(from_cuda(e));
    // emit: one ticket counter and look-back array per dimension group, in
    // consecutive slices of the emit workspace
    {
        size_t need = 0;
        for (auto &G : groups) need += emit_workspace_bytes(G.bricks);
        if ((e = cudaMemsetAsync(h->ws_emit, 0, need, st)) != cudaSuccess) return fail(from_cuda(e));
        char *ws = static_cast<char *>(h->ws_emit);
        size_t pos = 0;
        if (h->timing) cudaEventRecord(L->ev[3], st);
        for (auto &G : groups) {
            if ((e = launch_emit_d(G.d, Ddev + G.first, G.count, G.bricks, ws + pos, h->sm_count, st)) != cudaSuccess)
                return fail(from_cuda(e));
            h->launches++;
            pos += emit_workspace_bytes(G.bricks);
        }
    }
    if (h->timing) cudaEventRecord(L->ev[4], st);
    cudaEventRecord(h->ws_free, st);
    ids.resize(nf);
    for (int i = 0; i < nf; i++) {
        Result &r = *res[i];
        if ((e = cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming)) != cudaSuccess) return fail(from_cuda(e));
        cudaEventRecord(r.done, st);
    }
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
        SmallBlock sb;
        e = cudaMemcpy(&sb, r.small, sizeof(SmallBlock), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return from_cuda(e);
        r.A = sb.totals[3];
        r.err |= sb.err;
        r.have_A = true;
        if (r.launch && r.launch.use_count() == 1) release_launch(h, r.launch.get());
    }
    if (r.err & kErrNaN) return EG_ERR_NAN;
    if (r.err & kErrNotConverged) return EG_ERR_NOT_CONVERGED;
    if (r.err & kErrTimeout) return EG_ERR_TIMEOUT;
    if (r.err & kErrInternal) return EG_ERR_INTERNAL;
    return EG_OK;
}

void fill_counts(const Result &r, eg_graph *out)
{
    out->d = r.d;
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
    if ((e = cudaEventCreateWithFlags(&h->ws_free, cudaEventDisableTiming)) != cudaSuccess) return from_cuda(e);
    cudaEventRecord(h->ws_free, h->side);
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
        for (auto &kv : h->results)
            if (kv.second->done) cudaEventDestroy(kv.second->done);
        h->results.clear();
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
    std::vector<Job> jobs{{field, sh, h->cfg.flags & (kFlagMinimum | kFlagNoLabels)}};
    std::vector<uint64_t> ids;
    eg_status s = run_jobs(h, jobs, static_cast<cudaStream_t>(stream), ids);
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
    std::vector<Job> jobs{{static_cast<const float *>(h->stage), sh, h->cfg.flags & (kFlagMinimum | kFlagNoLabels)}};
    std::vector<uint64_t> ids;
    eg_status s = run_jobs(h, jobs, st, ids);
    if (s == EG_OK) *out = ids[0];
    return s;
}

eg_status eg_batch_submit(eg_handle h, const eg_field_desc *fields, int n, void *stream, eg_result_id *out_ids)
{
    if (!h || (n > 0 && (!fields || !out_ids)) || n < 0) return EG_ERR_ARG;
    if (n == 0) return EG_OK;
    std::vector<Job> jobs(n);
    for (int i = 0; i < n; i++) {
        if (!fields[i].field || !make_shape(fields[i].d, fields[i].extents, jobs[i].sh)) return EG_ERR_ARG;
        jobs[i].field = fields[i].field;
        jobs[i].flags = (h->cfg.flags | uint32_t(fields[i].flags)) & (kFlagMinimum | kFlagNoLabels);
    }
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    std::vector<uint64_t> ids;
    eg_status s = run_jobs(h, jobs, static_cast<cudaStream_t>(stream), ids);
    if (s == EG_OK)
        for (int i = 0; i < n; i++) out_ids[i] = ids[i];
    return s;
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
    struct { void *dst; const void *src; size_t b; } cp[] = {
        {out->maxima, r.maxima, r.M * 4}, {out->max_val, r.max_val, r.M * 4},
        {out->saddles, r.saddles, r.S * 4}, {out->sad_beta0, r.sad_b0, r.S},
        {out->sad_val, r.sad_val, r.S * 4}, {out->row_ptr, r.row_ptr, (r.S + 1) * 8},
        {out->col, r.col, r.A * 4}, {out->labels, r.lab, r.N * 4}};
    for (auto &c : cp)
        if (c.dst && c.b) {
            cudaError_t e = cudaMemcpy(c.dst, c.src, c.b, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return from_cuda(e);
        }
    return EG_OK;
}

eg_status eg_get_graph_device(eg_handle h, eg_result_id id, eg_graph *out)
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
    out->maxima = static_cast<uint32_t *>(r.maxima);
    out->max_val = static_cast<float *>(r.max_val);
    out->saddles = static_cast<uint32_t *>(r.saddles);
    out->sad_beta0 = static_cast<uint8_t *>(r.sad_b0);
    out->sad_val = static_cast<float *>(r.sad_val);
    out->row_ptr = static_cast<uint64_t *>(r.row_ptr);
    out->col = static_cast<uint32_t *>(r.col);
    out->labels = static_cast<uint32_t *>(r.lab);
    return EG_OK;
}

eg_status eg_release(eg_handle h, eg_result_id id)
{
    if (!h) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    cudaSetDevice(h->device);
    auto it = h->results.find(id);
    if (it == h->results.end()) return EG_ERR_ARG;
    Result &r = *it->second;
    if (r.done) {
        cudaEventSynchronize(r.done);
        cudaEventDestroy(r.done);
    }
    free_result_buffers(h, &r);
    if (r.launch && r.launch.use_count() == 1) release_launch(h, r.launch.get());
    h->results.erase(it);
    return EG_OK;
}

uint64_t eg_workspace_bytes(int d, const int64_t *extents)
{
    Shape sh;
    if (!make_shape(d, extents, sh)) return 0;
    const uint64_t b = bricks_of(sh.N);
    return b * kBrick * (4 + 8) + b * sizeof(uint4) + emit_workspace_bytes(b) + sh.N * 4;
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
    Launch &L = *it->second->launch;
    cudaError_t e = cudaEventSynchronize(L.ev[4]);
    if (e != cudaSuccess) return from_cuda(e);
    // ev: start | classify | resolve | (count read-back, buffer set-up) | emit
    float a = 0, b = 0, c = 0, t = 0;
    cudaEventElapsedTime(&a, L.ev[0], L.ev[1]);
    cudaEventElapsedTime(&b, L.ev[1], L.ev[2]);
    cudaEventElapsedTime(&c, L.ev[3], L.ev[4]);
    cudaEventElapsedTime(&t, L.ev[0], L.ev[4]);
    ms[0] = a;
    ms[1] = b;
    ms[2] = c;
    ms[3] = t;
    return EG_OK;
}

uint64_t eg_launch_count(eg_handle h) { return h ? h->launches.load() : 0; }

eg_status eg_debug_fail_alloc(eg_handle h, int k)
{
    if (!h || k < 0) return EG_ERR_ARG;
    std::lock_guard<std::mutex> g(h->mu);
    h->pool.fail_in = k;
    return EG_OK;
}

}  // extern "C"
