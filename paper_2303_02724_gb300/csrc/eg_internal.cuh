// Internal device-side definitions shared by the library's kernels.
//
// Neighbourhood (Sec. 3.2, Algorithm 1): the neighbours of a grid vertex are
// the in-bounds vertices v + delta with delta in {0,1}^D u {0,-1}^D, delta != 0,
// 2(2^D - 1) of them.  A non-zero delta is written as a bit pattern p over the
// axes (bit i set <=> component i is non-zero) and a sign.  Neighbour slot k:
//   k <  H = 2^D - 1 : negative, pattern p = H - k      (offset -sum_{i in p} s_i)
//   k >= H           : positive, pattern p = k - H + 1  (offset +sum_{i in p} s_i)
// With strides s_0 = 1, s_{i+1} = n_i s_i and every used axis of extent >= 2,
// sum_{i<j} s_i < s_j, so the linear offset grows with k: slot order is index
// order.  The centre vertex sits between slot H-1 and slot H.
//
// Link edges (the triangulation is a flag complex, Sec. 3.3): two neighbours
// are joined iff their difference is again an Algorithm-1 offset, which for
// patterns p, q reads
//   same sign      : p != q and (p subset of q or q subset of p)
//   opposite sign  : p and q disjoint.
//
// Order (simulation of simplicity, Sec. 3.3): w is higher than v iff
// f[w] > f[v], or f[w] == f[v] and w > v.  Values become monotone uint32 keys
// (-0 folded onto +0); inside one neighbourhood the index tie-break is the slot
// rank, so "higher" is a comparison of the 64-bit composite (key << 8 | rank).
// The minimum graph reverses the order: key -> ~key and rank -> 2H - rank.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace eg {

constexpr int kMaxDim = 4;
constexpr int kBrick = 1024;  // vertices per brick: a contiguous range of linear ids

// device status word bits (reported by eg_get_graph)
enum : uint32_t {
    kErrNaN = 1u,
    kErrNotConverged = 2u,
    kErrTimeout = 4u,
    kErrInternal = 8u,
};

// flags carried per field
enum : uint32_t { kFlagMinimum = 1u, kFlagNoLabels = 2u };

// One field as the kernels see it.  Plain pointers; filled on the host.
struct FieldDev {
    const float *f;        // [N] input values
    uint32_t *lab;         // [N] gradient pointer, then the label (maximum reached)
    uint32_t *rec_sid;     // [nbricks * kBrick] critical-vertex records, per brick slot
    uint64_t *rec_info;    // [nbricks * kBrick] beta0+ (bits 56..59) | rep slots (5 bits each)
    uint4 *bcnt;           // [nbricks] maxima, saddles, paths per brick
    uint32_t *maxima;      // [M]
    float *max_val;        // [M]
    uint32_t *saddles;     // [S]
    uint8_t *sad_b0;       // [S]
    float *sad_val;        // [S]
    uint64_t *row_ptr;     // [S+1]
    uint32_t *col;         // [A] (capacity P)
    unsigned long long *totals;  // [4] M, S, P, A
    uint32_t *err;         // device status word
    uint32_t n[kMaxDim];   // extents (1 beyond d)
    uint32_t s[kMaxDim];   // strides
    uint32_t N;            // vertex count (< 2^32)
    uint32_t nbricks;      // ceil(N / kBrick)
    uint64_t brick0;       // first global brick id of this field in its launch
    int32_t d;
    uint32_t flags;
};

// Monotone key of a float: a < b (IEEE, non-NaN) <=> key(a) < key(b); -0 == +0.
__device__ __forceinline__ uint32_t order_key(float x)
{
    uint32_t u = __float_as_uint(x);
    u = (u == 0x80000000u) ? 0u : u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int D>
struct Nbr {
    static constexpr int H = (1 << D) - 1;
    static constexpr int K = 2 * H;
    __host__ __device__ static constexpr bool neg(int k) { return k < H; }
    __host__ __device__ static constexpr uint32_t pat(int k) { return k < H ? uint32_t(H - k) : uint32_t(k - H + 1); }
    // rank in index order, centre = H
    __host__ __device__ static constexpr uint32_t rank(int k) { return k < H ? uint32_t(k) : uint32_t(k + 1); }
    __host__ __device__ static constexpr bool linked(int a, int b)
    {
        return a != b && (neg(a) == neg(b) ? ((pat(a) & pat(b)) == pat(a) || (pat(a) & pat(b)) == pat(b))
                                           : ((pat(a) & pat(b)) == 0u));
    }
    __host__ __device__ static constexpr uint32_t adj_mask(int a)
    {
        uint32_t m = 0;
        for (int b = 0; b < K; b++)
            if (linked(a, b)) m |= 1u << b;
        return m;
    }
};

// Linear offset (magnitude) of pattern p under strides s (runtime p).
__device__ __forceinline__ uint32_t pattern_offset(uint32_t p, const uint32_t *s)
{
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < kMaxDim; i++)
        if (p & (1u << i)) o += s[i];
    return o;
}

// Vertex reached from v through neighbour slot k (runtime k, D known).
template <int D>
__device__ __forceinline__ uint32_t slot_vertex(uint32_t v, int k, const uint32_t *s)
{
    using NB = Nbr<D>;
    uint32_t p = k < NB::H ? uint32_t(NB::H - k) : uint32_t(k - NB::H + 1);
    uint32_t o = pattern_offset(p, s);
    return k < NB::H ? v - o : v + o;
}

// ---------------------------------------------------------------------------
// Decoupled look-back (single-pass prefix over work items taken in ticket
// order).  Status word: bits 63..62 = 0 empty, 1 aggregate, 2 inclusive
// prefix; bits 61..0 value.  A warp inspects 32 predecessors per step; every
// wait is bounded and reports kErrTimeout instead of hanging.
// ---------------------------------------------------------------------------
constexpr uint64_t kLbAgg = 1ull << 62;
constexpr uint64_t kLbPre = 2ull << 62;
constexpr uint64_t kLbVal = (1ull << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p)
{
    return *reinterpret_cast<const volatile uint64_t *>(p);
}

__device__ __forceinline__ void st_volatile_u64(uint64_t *p, uint64_t v)
{
    *reinterpret_cast<volatile uint64_t *>(p) = v;
}

// Called by one full warp.  st: status array indexed by global item id;
// item: this item; first: the first item of its segment (predecessors before
// it count as zero).  Returns the exclusive prefix of agg over the segment.
__device__ __forceinline__ uint64_t warp_lookback(uint64_t *st, uint64_t item, uint64_t first,
                                                  uint64_t agg, uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    if (item == first) {
        if (lane == 0) st_volatile_u64(st + item, kLbPre | agg);
        return 0;
    }
    if (lane == 0) st_volatile_u64(st + item, kLbAgg | agg);
    uint64_t excl = 0;
    int64_t base = int64_t(item) - 1;
    uint32_t spins = 0;
    unsigned ns = 8;
    while (true) {
        int64_t j = base - lane;
        uint64_t w = (j >= int64_t(first)) ? ld_volatile_u64(st + j) : kLbPre;
        bool empty = (w >> 62) == 0;
        if (__any_sync(0xffffffffu, empty)) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            __nanosleep(ns);
            ns = ns < 256 ? ns * 2 : 256;
            continue;
        }
        unsigned pmask = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        int stop = pmask ? (__ffs(pmask) - 1) : 31;
        uint64_t val = (lane <= stop) ? (w & kLbVal) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
        excl += val;
        if (pmask) break;
        base -= 32;
    }
    if (lane == 0) st_volatile_u64(st + item, kLbPre | (excl + agg));
    return excl;
}

// Locate the field that owns global brick g (fields sorted by brick0).
__device__ __forceinline__ int find_field(const FieldDev *fields, int nf, uint64_t g)
{
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (fields[mid].brick0 <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim multiple of 32,
// <= 1024).  scratch: >= 33 words of shared memory.  Returns the exclusive
// prefix; *total receives the block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *scratch, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? scratch[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) scratch[lane] = wi - w;
        if (lane == nw - 1) scratch[32] = wi;
    }
    __syncthreads();
    uint32_t r = scratch[warp] + inc - x;
    *total = scratch[32];
    __syncthreads();
    return r;
}

}  // namespace eg
