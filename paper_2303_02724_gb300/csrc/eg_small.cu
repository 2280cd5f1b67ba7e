// Fused path for one small field (1D-3D float32, at most kSmallMaxVertices
// vertices): classification (Sec. 3.3), path resolution (Sec. 3.4) and graph
// assembly (Sec. 2 arcs, CSR) in one cooperative launch.
//
// A field this small is too little work to fill the GPU in any one step, so
// the separate launches of the general path (and the count read-back between
// them) cost more than the steps themselves.  Here one launch runs them all,
// separated by grid barriers:
//   1. classification, one vertex per thread, a brick = one CTA's 256
//      consecutive vertex ids (the flat layout's per-vertex classifier, so the
//      records are those of the general path);
//   2. brick offsets and the totals M, S, P (one CTA scans the <= 256 brick
//      counts), while every thread resolves its vertex's label by following
//      the gradient pointers (concurrent walks read either a pointer or a
//      finished label on the same path, so the races are benign);
//   3. nodes and arc ends, one warp per brick;
//   4. CSR, one warp per brick, each adding up the arc counts of the bricks
//      before its own (its arc offset) and of all bricks (the total A);
// then the last CTA to finish copies the totals and the status word to the
// caller's page-locked host block, so no copy follows the kernel.
// Every barrier wait is bounded (kErrTimeout after about a second); a CTA
// that gave up at a barrier never arrives at the end, and the host block
// keeps the timeout status the caller put there.
#include <atomic>

#include "eg_emit.cuh"
#include "eg_flat.cuh"
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kSmallThreads = int(kSmallBrick);  // one vertex per thread, a brick per CTA

// Grid barrier over a count that only grows during the launch (zero at its
// start): barrier k (k = 1, 2, ...) lets the CTAs go once the count reaches k
// times the grid size, so the last arrival's increment releases the others
// without a reset or a second word.  Thread 0 waits for at most about a
// second, then sets kErrTimeout and the CTA leaves.
__device__ __forceinline__ bool count_barrier(unsigned *count, unsigned k, uint32_t *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = k * gridDim.x;
        __threadfence();
        if (atomicAdd(count, 1u) + 1u < target) {
            unsigned ns = 32;
            uint32_t spins = 0;
            while (*reinterpret_cast<volatile unsigned *>(count) < target) {
                if (++spins > kSpinLimit) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                ns = ns < 256 ? ns * 2 : 256;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__global__ void __launch_bounds__(kSmallThreads)
    k_small(const FieldDev F, unsigned *bar, uint32_t *next_err, unsigned *next_count, unsigned long long *htotals,
            uint32_t *herr)
{
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned s_cnt[3];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nb = F.nbricks;
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    const bool minimum = (F.flags & kFlagMinimum) != 0;
    // the next launch's status word and barrier count (no other launch of
    // this caller runs before this one ends)
    if (blockIdx.x == 0 && tid == 0) {
        *next_err = 0u;
        *next_count = 0u;
    }

    // 1: classification and the brick's records in index order
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        if (tid < 3) s_cnt[tid] = 0;
        const uint64_t v64 = uint64_t(b) * kSmallThreads + uint64_t(tid);
        const bool in = v64 < F.N;
        const uint32_t v = uint32_t(v64);
        int b0 = 1;
        uint64_t codes = 0;
        bool nan = false;
        if (in && chk(v, F.N, F.err)) F.lab[v] = classify_vertex<3, kF32>(F, s, v, minimum, b0, codes, nan);
        if (nan) atomicOr(F.err, kErrNaN);
        const bool crit = in && b0 != 1;
        uint32_t tot;
        const uint32_t pos = block_excl_scan(crit ? 1u : 0u, s_scan, &tot);  // (its barriers publish s_cnt = 0)
        const uint64_t q = uint64_t(b) * F.bcap + pos;
        if (crit && chk(q, rec_cap(F), F.err) && chk(pos, F.bcap, F.err)) {
            F.rec_sid[q] = v;
            F.rec_info[q] = (uint64_t(b0) << 56) | codes;
            F.rec_val[q] = F.f[v];
        }
        const unsigned nm = __reduce_add_sync(0xffffffffu, crit && b0 == 0 ? 1u : 0u);
        const unsigned ns = __reduce_add_sync(0xffffffffu, crit && b0 > 0 ? 1u : 0u);
        const unsigned np = __reduce_add_sync(0xffffffffu, crit && b0 > 0 ? unsigned(b0) : 0u);
        if (lane == 0) {
            if (nm) atomicAdd(&s_cnt[0], nm);
            if (ns) atomicAdd(&s_cnt[1], ns);
            if (np) atomicAdd(&s_cnt[2], np);
        }
        __syncthreads();
        if (tid == 0 && chk(b, nb, F.err)) F.bcnt[b] = make_uint4(s_cnt[0], s_cnt[1], s_cnt[2], 0u);
        __syncthreads();  // s_cnt is cleared again by the next brick
    }
    if (!count_barrier(bar, 1u, F.err)) return;

    // 2: brick offsets (CTA 0: one thread per brick), labels (every thread)
    if (blockIdx.x == 0) {
        uint4 c = make_uint4(0u, 0u, 0u, 0u);
        if (uint32_t(tid) < nb) c = F.bcnt[tid];
        uint32_t tm, ts, tp;
        const uint32_t om = block_excl_scan(c.x, s_scan, &tm);
        const uint32_t os = block_excl_scan(c.y, s_scan, &ts);
        const uint32_t op = block_excl_scan(c.z, s_scan, &tp);
        if (uint32_t(tid) < nb) F.boff[tid] = make_uint4(om, os, op, 0u);
        if (tid == 0) {
            F.totals[0] = tm;
            F.totals[1] = ts;
            F.totals[2] = tp;
        }
    }
    for (uint64_t v = uint64_t(blockIdx.x) * kSmallThreads + tid; v < F.N; v += uint64_t(gridDim.x) * kSmallThreads) {
        uint32_t u = F.lab[v];
        bool moved = false;
        // a path climbs strictly in the order, so it has fewer than N steps
        for (uint32_t steps = 0; u != uint32_t(v); steps++) {
            if (steps > F.N) {
                atomicOr(F.err, kErrNotConverged);
                break;
            }
            if (!chk(u, F.N, F.err)) break;
            const uint32_t w = F.lab[u];
            if (w == u) break;  // a maximum
            u = w;
            moved = true;
        }
        if (moved) F.lab[v] = u;
    }
    if (!count_barrier(bar, 2u, F.err)) return;

    // 3: nodes and arc ends; a brick per warp, the bricks dealt to the CTAs
    // first (warp w of CTA c takes bricks c + w G, c + (w + 8) G, ... for a
    // grid of G CTAs), so the latency-bound warps spread over every SM
    constexpr uint32_t kWarps = kSmallThreads / 32;
    const uint32_t b_first = blockIdx.x + gridDim.x * uint32_t(warp), b_step = gridDim.x * kWarps;
    for (uint32_t b = b_first; b < nb; b += b_step) nodes_brick<3>(F, b);
    if (!count_barrier(bar, 3u, F.err)) return;

    // 4: each warp adds up the arc counts before its brick and in all (at
    // most 256 bricks), then writes its brick's CSR (every warp writes the
    // same total A)
    for (uint32_t b = b_first; b < nb; b += b_step) {
        uint32_t pre = 0, all = 0;
        for (uint32_t i = uint32_t(lane); i < nb; i += 32) {
            const uint32_t a = F.acnt[i];
            all += a;
            pre += i < b ? a : 0u;
        }
        pre = __reduce_add_sync(0xffffffffu, pre);
        all = __reduce_add_sync(0xffffffffu, all);
        if (lane == 0) {
            F.aoff[b] = pre;
            F.totals[3] = all;
        }
        __syncwarp();
        csr_brick(F, b);
    }

    // arrival at the end (after three barriers the count is 3 G); the last
    // CTA sees every other CTA's writes
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(bar, 1u) == 4u * gridDim.x - 1u) {
            __threadfence();
#pragma unroll
            for (int q = 0; q < 4; q++) htotals[q] = *reinterpret_cast<volatile unsigned long long *>(F.totals + q);
            *herr = *reinterpret_cast<volatile uint32_t *>(F.err);
            __threadfence_system();
        }
    }
}

uint32_t small_bricks(uint64_t n) { return uint32_t((n + kSmallThreads - 1) / kSmallThreads); }

cudaError_t launch_small(const FieldDev &F, unsigned *bar, uint32_t *next_err, unsigned *next_count,
                         unsigned long long *htotals, uint32_t *herr, int sm_count, cudaStream_t st)
{
    if (F.nbricks == 0 || F.nbricks > uint32_t(kSmallThreads) || F.bcap != uint32_t(kSmallThreads))
        return cudaErrorInvalidValue;
    // (the same kernel and CTA size on every device of the build's architecture)
    static std::atomic<int> per_sm_cache{0};
    int per_sm = per_sm_cache.load();
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small, kSmallThreads, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
        per_sm_cache.store(per_sm);
    }
    uint64_t grid = uint64_t(sm_count > 0 ? sm_count : 1) * uint64_t(per_sm);
    if (grid > F.nbricks) grid = F.nbricks;
    FieldDev arg = F;
    void *args[] = {&arg, &bar, &next_err, &next_count, &htotals, &herr};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_small), dim3(unsigned(grid)), dim3(kSmallThreads),
                                       args, 0, st);
}

}  // namespace eg
