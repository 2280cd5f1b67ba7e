// Persistence-directed cancellation (Sec. 3.5) on a finished extremum graph,
// as data-parallel rounds.
//
// The paper's procedure is a serial priority queue: take the saddle of lowest
// cost, recompute its cost against the graph as it is now, discard it above
// the threshold, reinsert it if it is no longer the cheapest, else cancel it
// (every maximum it reaches but the highest is merged into the highest).  With
// costs that never fall (the paper's premise; see the note on multi-saddles
// below) every cancellation takes the saddle of lowest current (cost, id),
// cost = second highest adjacent maximum minus the saddle, in float32.
//
// Rounds.  Two saddles that reach no common maximum (after the merges so far)
// do not affect each other's cost.  A saddle s may be cancelled in the current
// round, ahead of the serial order, when no saddle x sharing a maximum with it
// could come first: x's cost can only fall to lb(x) = lowest adjacent maximum
// minus x (merges replace a maximum by a higher one, and a multi-saddle whose
// maxima merge can drop to its lowest one), so s is safe when
//   (cost(s), id(s)) < (lb(x), id(x))  for every such x.
// Safe saddles share no maximum with one another (two of them would each have
// to be below the other), so their merges are disjoint and all of them are
// cancelled at once, together with the global cheapest saddle, which the serial
// order takes next anyway.  Every round therefore cancels at least one saddle
// and the result equals the serial one.  A saddle that joins one maximum, or
// whose lb exceeds the threshold, can never be cancelled (lb never falls) and
// leaves the rounds for good.
//
// Multi-saddles: merging two maxima of a multi-saddle can lower its second
// highest maximum, so its cost can fall, which the paper's discard rule does
// not foresee; here the cost is always the current one (a saddle is
// cancelled as soon as it is the cheapest), which is what the serial queue
// does whenever costs never fall.
//
// One round = four kernels: evaluate (current maxima, cost and lb keys, the
// per-maximum minimum of lb keys, the global cheapest), second minima per
// maximum, decide + mark the merges, apply the merges.  Keys are
// (float32 bits of a non-negative cost) << 32 | saddle index, so one 64-bit
// atomicMin orders by cost, then by vertex id (saddles are in id order).
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kCancelThreads = 256;
constexpr int kMaxAdj = 20;  // most distinct maxima one saddle reaches (beta0+ bound, 5D)
constexpr unsigned long long kNoKey = ~0ull;

// maximum a higher than maximum b: (value, then id), reversed for the
// minimum graph
__device__ __forceinline__ bool c_higher(const CancelDev &C, uint32_t a, uint32_t b)
{
    const float fa = C.max_val[a], fb = C.max_val[b];
    const bool up = fa != fb ? fa > fb : C.maxima[a] > C.maxima[b];
    return C.minimum ? !up : up;
}

// Cost of saddle s against maximum m: 0 for equal values, else the
// difference rounded to float32 (never negative: a saddle is below every
// maximum it reaches).
__device__ __forceinline__ float c_cost(const CancelDev &C, float fs, uint32_t m)
{
    const float fm = C.max_val[m];
    if (fm == fs) return 0.0f;
    return C.minimum ? __fsub_rn(fs, fm) : __fsub_rn(fm, fs);
}

__device__ __forceinline__ unsigned long long c_key(float cost, uint32_t s)
{
    return (static_cast<unsigned long long>(__float_as_uint(cost)) << 32) | s;
}

// Distinct current maxima of saddle s from the per-arc snapshot.
__device__ __forceinline__ int c_adjacent(const CancelDev &C, uint32_t s, uint32_t (&u)[kMaxAdj])
{
    int n = 0;
    for (uint64_t a = C.row_ptr[s]; a < C.row_ptr[s + 1]; a++) {
        const uint32_t r = C.aroot[a];
        bool dup = false;
        for (int k = 0; k < n; k++) dup |= u[k] == r;
        if (!dup && n < kMaxAdj) u[n++] = r;
    }
    return n;
}

// Arc ends as indices into the (sorted) maxima list.
__global__ void k_cancel_ends(CancelDev C, const uint32_t *__restrict__ col, uint64_t A)
{
    const uint64_t a = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (a >= A) return;
    const uint32_t v = col[a];
    uint32_t lo = 0, hi = C.M;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (C.maxima[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    if (lo >= C.M || C.maxima[lo] != v) {
        atomicOr(C.err, kErrInternal);  // an arc end that is not a maximum
        lo = 0;
    }
    C.end[a] = lo;
}

__global__ void k_cancel_init(CancelDev C)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C.M) {
        C.root[i] = i;
        C.merge[i] = 0;
    }
    if (i < C.S) C.state[i] = 0;
}

// 1: current maxima of every waiting saddle, its keys, the per-maximum
// minimum lb key and the global cheapest cancellable saddle.
__global__ void __launch_bounds__(kCancelThreads) k_cancel_eval(CancelDev C)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long gk = kNoKey;
    if (s < C.S && C.state[s] == 0) {
        for (uint64_t a = C.row_ptr[s]; a < C.row_ptr[s + 1]; a++) C.aroot[a] = C.root[C.end[a]];
        uint32_t u[kMaxAdj];
        const int n = c_adjacent(C, s, u);
        if (n < 2) {
            C.state[s] = 2;  // joins one maximum: never cancelled
        } else {
            uint32_t h1 = u[0], h2 = 0xffffffffu, lo = u[0];
            for (int k = 1; k < n; k++) {
                if (c_higher(C, u[k], h1)) {
                    h2 = h1;
                    h1 = u[k];
                } else if (h2 == 0xffffffffu || c_higher(C, u[k], h2)) {
                    h2 = u[k];
                }
                if (c_higher(C, lo, u[k])) lo = u[k];
            }
            const float fs = C.sad_val[s];
            const float cost = c_cost(C, fs, h2), lb = c_cost(C, fs, lo);
            if (lb > C.tau) {
                C.state[s] = 2;  // its cost never falls below lb: never cancelled
            } else {
                const unsigned long long ck = c_key(cost, s), lk = c_key(lb, s);
                C.costkey[s] = ck;
                C.lbkey[s] = lk;
                C.high[s] = h1;
                for (int k = 0; k < n; k++) atomicMin(C.minlb + u[k], lk);
                if (cost <= C.tau) gk = ck;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, gk, o);
        gk = y < gk ? y : gk;
    }
    if ((threadIdx.x & 31) == 0 && gk != kNoKey) atomicMin(C.ctrl, gk);
}

// 2: per maximum, the smallest lb key other than the minimum's own holder.
__global__ void __launch_bounds__(kCancelThreads) k_cancel_second(CancelDev C)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.S || C.state[s] != 0) return;
    uint32_t u[kMaxAdj];
    const int n = c_adjacent(C, s, u);
    const unsigned long long lk = C.lbkey[s];
    for (int k = 0; k < n; k++)
        if (C.minlb[u[k]] != lk) atomicMin(C.min2 + u[k], lk);
}

// 3: cancel every safe saddle and the global cheapest; mark their merges.
__global__ void __launch_bounds__(kCancelThreads) k_cancel_decide(CancelDev C, uint32_t stamp)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= C.S || C.state[s] != 0) return;
    const unsigned long long ck = C.costkey[s];
    if (__uint_as_float(uint32_t(ck >> 32)) > C.tau) return;
    uint32_t u[kMaxAdj];
    const int n = c_adjacent(C, s, u);
    bool safe = ck == C.ctrl[0];
    if (!safe) {
        const unsigned long long lk = C.lbkey[s];
        safe = true;
        for (int k = 0; k < n; k++) {
            const unsigned long long m1 = C.minlb[u[k]];
            const unsigned long long other = m1 == lk ? C.min2[u[k]] : m1;
            safe &= other > ck;
        }
    }
    if (!safe) return;
    C.state[s] = 1;
    atomicAdd(C.ctrl + 1, 1ull);
    const uint32_t h1 = C.high[s];
    for (int k = 0; k < n; k++)
        if (u[k] != h1) C.merge[u[k]] = (static_cast<unsigned long long>(stamp) << 32) | h1;
}

// 4: every maximum follows the merge of its current survivor (one hop: a
// survivor of this round is merged nowhere this round).
__global__ void k_cancel_apply(CancelDev C, uint32_t stamp)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= C.M) return;
    const unsigned long long m = C.merge[C.root[i]];
    if (uint32_t(m >> 32) == stamp) C.root[i] = uint32_t(m);
}

// Results: keep flag per saddle, vertex id of each maximum's survivor.
__global__ void k_cancel_out(CancelDev C, uint8_t *alive, uint32_t *survivor)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C.S) alive[i] = C.state[i] != 1 ? 1 : 0;
    if (i < C.M) survivor[i] = C.maxima[C.root[i]];
}

static inline dim3 grid_of(uint64_t n) { return dim3(unsigned((n + kCancelThreads - 1) / kCancelThreads)); }

cudaError_t launch_cancel_setup(const CancelDev &C, const uint32_t *col, uint64_t A, cudaStream_t st)
{
    const uint64_t n = C.M > C.S ? C.M : C.S;
    if (n) k_cancel_init<<<grid_of(n), kCancelThreads, 0, st>>>(C);
    if (A) k_cancel_ends<<<grid_of(A), kCancelThreads, 0, st>>>(C, col, A);
    return cudaGetLastError();
}

cudaError_t launch_cancel_round(const CancelDev &C, uint32_t stamp, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(C.minlb, 0xff, sizeof(unsigned long long) * C.M, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(C.min2, 0xff, sizeof(unsigned long long) * C.M, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(C.ctrl, 0xff, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(C.ctrl + 1, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    if (C.S) {
        k_cancel_eval<<<grid_of(C.S), kCancelThreads, 0, st>>>(C);
        k_cancel_second<<<grid_of(C.S), kCancelThreads, 0, st>>>(C);
        k_cancel_decide<<<grid_of(C.S), kCancelThreads, 0, st>>>(C, stamp);
    }
    if (C.M) k_cancel_apply<<<grid_of(C.M), kCancelThreads, 0, st>>>(C, stamp);
    return cudaGetLastError();
}

cudaError_t launch_cancel_out(const CancelDev &C, uint8_t *alive, uint32_t *survivor, cudaStream_t st)
{
    const uint64_t n = C.M > C.S ? C.M : C.S;
    if (n) k_cancel_out<<<grid_of(n), kCancelThreads, 0, st>>>(C, alive, survivor);
    return cudaGetLastError();
}

}  // namespace eg
