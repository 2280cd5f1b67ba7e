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
// Rounds.  Cancelling s merges its dying maxima D(s) (all it reaches but the
// highest, h(s)) into h(s).  Until s is cancelled, its cost and D(s) can only
// change through a cancellation that merges a maximum of D(s) away, and such a
// cancellation must come from a saddle that reaches that maximum now (or one
// that reaches it later through a merge into it, which again needs a saddle
// that reaches it now).  A saddle x's cost can only fall to lb(x) = lowest
// maximum it reaches minus x (merges replace a maximum by a higher one, and a
// multi-saddle whose maxima merge can drop to its lowest one).  So s may be
// cancelled now, ahead of the serial order and with the serial result, when
//   (cost(s), id(s)) < (lb(x), id(x))  for every other saddle x reaching a
//   maximum of D(s).
// Merging h(s) itself away (into a higher maximum) leaves cost(s) and D(s)
// unchanged and only relabels the survivor, so saddles that share nothing but
// h(s) with s do not constrain it.  Two safe saddles never share a dying
// maximum (each would have to be below the other), so all safe saddles are
// cancelled at once, together with the global cheapest saddle, which the
// serial order takes next anyway; a survivor of one may die in another, and
// the merges of a round are followed as chains.  Every round cancels at least
// one saddle.  A saddle that joins one maximum, or whose lb exceeds the
// threshold, can never be cancelled (lb never falls) and leaves the rounds for
// good.
//
// Multi-saddles: merging two maxima of a multi-saddle can lower its second
// highest maximum, so its cost can fall, which the paper's discard rule does
// not foresee; here the cost is always the current one (a saddle is
// cancelled as soon as it is the cheapest), which is what the serial queue
// does whenever costs never fall.
//
// One round, over the list of saddles still waiting: (1) clear the
// per-maximum minima of the round before, evaluate (current maxima by
// following the merges, cost and lb keys, the per-maximum minimum of lb keys,
// the global cheapest) and keep the saddles that still wait in the next
// list; (2) second minima per maximum; (3) decide (cancel, and point each
// dying maximum at its survivor).  The per-maximum minima and the arcs'
// snapshots of their current maxima are kept twice, by the parity of the
// round: round r writes set r % 2 and clears set (r + 1) % 2, which round r - 1
// wrote, through that round's snapshots, so no reset pass is needed and a
// round takes three grid barriers.  All rounds run in one cooperative launch
// (late rounds often cancel one or two saddles between a few large maxima,
// so their number can be large; a launch per round would cost far more), one
// CTA of 1024 threads per SM, so that few CTAs meet at each barrier.  Keys are
// (float32 bits of a non-negative cost) << 32 | saddle index, so one 64-bit
// atomicMin orders by cost, then by vertex id (saddles are in id order).
#include <algorithm>

#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kCancelThreads = 1024;
constexpr int kSetupThreads = 256;
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

// Current survivor of maximum m: follow the merges (each goes to a strictly
// higher maximum) and shorten the chain behind (any ancestor is a valid
// parent, so concurrent shortening is harmless).
__device__ __forceinline__ uint32_t c_find(const CancelDev &C, uint32_t m)
{
    uint32_t r = m;
    for (uint32_t hops = 0; hops < C.M; hops++) {
        const uint32_t p = C.parent[r];
        if (p == r) break;
        r = p;
    }
    if (C.parent[m] != r) C.parent[m] = r;
    return r;
}

// Distinct current maxima of saddle s from the snapshot of set b.
__device__ __forceinline__ int c_adjacent(const CancelDev &C, int b, uint32_t s, uint32_t (&u)[kMaxAdj])
{
    int n = 0;
    for (uint64_t a = C.row_ptr[s]; a < C.row_ptr[s + 1]; a++) {
        const uint32_t r = C.aroot[b][a];
        bool dup = false;
        for (int k = 0; k < n; k++) dup |= u[k] == r;
        if (!dup && n < kMaxAdj) u[n++] = r;
    }
    return n;
}

// Phase 1 for one waiting saddle: its current maxima (snapshot b), keys, the
// per-maximum minimum lb key; returns its cost key if it may be cancelled
// (else kNoKey).
__device__ __forceinline__ unsigned long long c_eval(const CancelDev &C, int b, uint32_t s)
{
    for (uint64_t a = C.row_ptr[s]; a < C.row_ptr[s + 1]; a++) C.aroot[b][a] = c_find(C, C.end[a]);
    uint32_t u[kMaxAdj];
    const int n = c_adjacent(C, b, s, u);
    if (n < 2) {
        C.state[s] = 2;  // joins one maximum: never cancelled
        return kNoKey;
    }
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
        return kNoKey;
    }
    const unsigned long long ck = c_key(cost, s), lk = c_key(lb, s);
    C.costkey[s] = ck;
    C.lbkey[s] = lk;
    C.high[s] = h1;
    for (int k = 0; k < n; k++) atomicMin(C.minlb[b] + u[k], lk);
    return cost <= C.tau ? ck : kNoKey;
}

// Phase 1 shortcut for a saddle evaluated in the round before: when every
// maximum it reached then is still a survivor (no merge took one away; merges
// happen only in phase 3, so the survivors are fixed during phase 1), its
// maxima, keys and highest maximum are the same as then.  The snapshot of set
// b ^ 1 is carried over to set b and the stored lb key contributed; *ck
// receives its cost key if it may be cancelled.  Returns false (nothing
// written) when a maximum changed.
__device__ __forceinline__ bool c_unchanged(const CancelDev &C, int b, uint32_t s, unsigned long long *ck)
{
    const uint64_t a0 = C.row_ptr[s], a1 = C.row_ptr[s + 1];
    for (uint64_t a = a0; a < a1; a++) {
        const uint32_t r = C.aroot[b ^ 1][a];
        if (C.parent[r] != r) return false;
    }
    const unsigned long long lk = C.lbkey[s];
    for (uint64_t a = a0; a < a1; a++) {
        const uint32_t r = C.aroot[b ^ 1][a];
        C.aroot[b][a] = r;
        atomicMin(C.minlb[b] + r, lk);
    }
    const unsigned long long k = C.costkey[s];
    *ck = __uint_as_float(uint32_t(k >> 32)) <= C.tau ? k : kNoKey;
    return true;
}

// Clear the per-maximum minima of set b that saddle s wrote (through the
// snapshot of set b).
__device__ __forceinline__ void c_clear(const CancelDev &C, int b, uint32_t s)
{
    for (uint64_t a = C.row_ptr[s]; a < C.row_ptr[s + 1]; a++) {
        const uint32_t r = C.aroot[b][a];
        C.minlb[b][r] = kNoKey;
        C.min2[b][r] = kNoKey;
    }
}

// Phase 2: per maximum, the smallest lb key other than the minimum's holder.
__device__ __forceinline__ void c_second(const CancelDev &C, int b, uint32_t s)
{
    uint32_t u[kMaxAdj];
    const int n = c_adjacent(C, b, s, u);
    const unsigned long long lk = C.lbkey[s];
    for (int k = 0; k < n; k++)
        if (C.minlb[b][u[k]] != lk) atomicMin(C.min2[b] + u[k], lk);
}

// Phase 3: cancel the saddle if it is safe or the global cheapest; its dying
// maxima get their survivor as parent.  Returns 1 when it is cancelled.
__device__ __forceinline__ int c_decide(const CancelDev &C, int b, uint32_t s, unsigned long long gmin)
{
    const unsigned long long ck = C.costkey[s];
    if (__uint_as_float(uint32_t(ck >> 32)) > C.tau) return 0;
    uint32_t u[kMaxAdj];
    const int n = c_adjacent(C, b, s, u);
    const uint32_t h1 = C.high[s];
    bool safe = ck == gmin;
    if (!safe) {
        const unsigned long long lk = C.lbkey[s];
        safe = true;
        for (int k = 0; k < n; k++) {
            if (u[k] == h1) continue;  // the survivor: see above
            const unsigned long long m1 = C.minlb[b][u[k]];
            const unsigned long long other = m1 == lk ? C.min2[b][u[k]] : m1;
            safe &= other > ck;
        }
    }
    if (!safe) return 0;
    C.state[s] = 1;
    // the next round's finds read these (every eval of this round is done)
    for (int k = 0; k < n; k++)
        if (u[k] != h1) C.parent[u[k]] = h1;
    return 1;
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
        C.parent[i] = i;
        for (int b = 0; b < 2; b++) {
            C.minlb[b][i] = kNoKey;
            C.min2[b][i] = kNoKey;
        }
    }
    if (i < C.S) {
        C.state[i] = 0;
        C.list[0][i] = i;  // every saddle waits
    }
}

__device__ __forceinline__ unsigned long long c_read(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// All rounds in one cooperative launch: the CTAs share the lists with
// grid-stride loops, separated by grid barriers (three per round).  The
// control words of round r live in slot r % 3 ({cheapest key, cancellations,
// length of the list the round keeps}); slot (r + 1) % 3 is cleared during
// round r, which no CTA can still be reading (it was last used two rounds
// before).  Round r walks the list kept by round r - 1 (every saddle of it
// clears what it wrote then, and the ones cancelled since drop out), keeps
// the saddles that still wait after its evaluation, and runs phases 2 and 3
// over those.  The loop ends with the first round that cancels nothing (or
// keeps no saddle), or when a barrier gives up.  ctrl[9] receives the number
// of rounds.
__global__ void __launch_bounds__(kCancelThreads) k_cancel_rounds(CancelDev C)
{
    unsigned *bar = reinterpret_cast<unsigned *>(C.ctrl + 10);  // [0] count, [1] generation
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    int p = 0;
    unsigned long long n = C.S;
    uint32_t round = 0;
    while (round <= C.S) {
        unsigned long long *slot = C.ctrl + 3 * (round % 3);
        const int b = int(round & 1);
        if (tid == 0) {
            unsigned long long *nx = C.ctrl + 3 * ((round + 1) % 3);
            nx[0] = kNoKey;
            nx[1] = 0;
            nx[2] = 0;
        }
        // 1: clear the previous round's minima, evaluate, keep the waiting
        for (uint64_t base = tid - lane; base < n; base += stride) {
            const uint64_t i = base + lane;
            bool keep = false;
            uint32_t s = 0;
            unsigned long long k = kNoKey;
            if (i < n) {
                s = C.list[p][i];
                if (round > 0) c_clear(C, b ^ 1, s);
                if (C.state[s] == 0) {
                    // (every saddle of a later round's list was evaluated in the
                    // round before and still waits)
                    if (round == 0 || !c_unchanged(C, b, s, &k)) k = c_eval(C, b, s);
                    keep = C.state[s] == 0;
                }
            }
            // the warp's cheapest key, then one atomic per warp (every
            // candidate of the round would otherwise meet at one address)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, k, o);
                k = y < k ? y : k;
            }
            if (lane == 0 && k != kNoKey) atomicMin(slot, k);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (!m) continue;
            unsigned long long o = 0;
            if (lane == __ffs(m) - 1) o = atomicAdd(slot + 2, (unsigned long long)__popc(m));
            o = __shfl_sync(0xffffffffu, o, __ffs(m) - 1);
            if (keep) C.list[p ^ 1][o + __popc(m & ((1u << lane) - 1u))] = s;
        }
        if (!grid_barrier(bar, bar + 1, C.err)) break;
        n = c_read(slot + 2);
        p ^= 1;
        if (n == 0) {
            round++;
            break;
        }
        // 2: second minima
        for (uint64_t i = tid; i < n; i += stride) c_second(C, b, C.list[p][i]);
        if (!grid_barrier(bar, bar + 1, C.err)) break;
        // 3: decide
        const unsigned long long gmin = c_read(slot);
        for (uint64_t i = tid; i < n; i += stride)
            if (c_decide(C, b, C.list[p][i], gmin)) atomicAdd(slot + 1, 1ull);
        if (!grid_barrier(bar, bar + 1, C.err)) break;
        round++;
        if (c_read(slot + 1) == 0) break;
    }
    if (tid == 0) C.ctrl[9] = round;
}

// Results: keep flag per saddle, vertex id of each maximum's survivor.
__global__ void k_cancel_out(CancelDev C, uint8_t *alive, uint32_t *survivor)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < C.S) alive[i] = C.state[i] != 1 ? 1 : 0;
    if (i < C.M) survivor[i] = C.maxima[c_find(C, i)];
}

static inline dim3 grid_of(uint64_t n) { return dim3(unsigned((n + kSetupThreads - 1) / kSetupThreads)); }

cudaError_t launch_cancel_setup(const CancelDev &C, const uint32_t *col, uint64_t A, cudaStream_t st)
{
    const uint64_t n = C.M > C.S ? C.M : C.S;
    if (n) k_cancel_init<<<grid_of(n), kSetupThreads, 0, st>>>(C);
    if (A) k_cancel_ends<<<grid_of(A), kSetupThreads, 0, st>>>(C, col, A);
    return cudaGetLastError();
}

cudaError_t launch_cancel_rounds(const CancelDev &C, int sm_count, cudaStream_t st)
{
    if (C.S == 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cancel_rounds, kCancelThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    uint64_t grid = uint64_t(std::max(sm_count, 1));
    const uint64_t need = (uint64_t(C.S) + kCancelThreads - 1) / kCancelThreads;
    if (grid > need) grid = need;
    CancelDev arg = C;
    void *args[] = {&arg};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_cancel_rounds), dim3(unsigned(grid)),
                                       dim3(kCancelThreads), args, 0, st);
}

cudaError_t launch_cancel_out(const CancelDev &C, uint8_t *alive, uint32_t *survivor, cudaStream_t st)
{
    const uint64_t n = C.M > C.S ? C.M : C.S;
    if (n) k_cancel_out<<<grid_of(n), kSetupThreads, 0, st>>>(C, alive, survivor);
    return cudaGetLastError();
}

}  // namespace eg
