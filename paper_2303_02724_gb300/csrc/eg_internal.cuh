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
// f[w] > f[v], or f[w] == f[v] and w > v.  Inside one neighbourhood the index
// tie-break is the slot rank.  The minimum graph reverses the order.
//
// A 2D field is processed as a 3D field with n2 = 1: the 3D neighbourhood
// restricted to the plane is exactly the 2D one (patterns without the z bit),
// with the same link edges and the same index order.
//
// Bricks: every kernel after classification works on bricks, contiguous
// ranges of linear vertex ids, in index order.  Flat layout: 1024 ids per
// brick.  Row layout (2D/3D with axis-0 extent <= 2048, 4D with axis-0 extent
// <= 1024): `ty` whole rows of one plane per brick (one row when it holds more
// than 1024 vertices), so brick b = plane b / nyb, row block b % nyb.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace eg {

constexpr int kMaxDim = 5;
constexpr int kFlatBrick = 1024;
constexpr int kMaxBrick = 4096;  // largest brick of any layout (slot capacity bound)

// Most upper-link components a vertex can have: the independence number of
// the link graph (3 in 2D, 6 in 3D, 10 in 4D, 20 in 5D).
template <int KD>
struct CompBound {
    static constexpr int value = KD == 5 ? 20 : 10;
};

// Record info word of a critical vertex (0 for a maximum).  Kernel
// dimensions up to 4: beta0+ in bits 56..59 and the neighbour slot of each
// component's representative as 5-bit fields from bit 0.  5D (62 slots, up to
// 20 components): bit k set iff slot k is a representative; beta0+ is the
// number of set bits.
template <int KD>
__device__ __forceinline__ int rec_b0(uint64_t info)
{
    if constexpr (KD == 5) return __popcll(info);
    else return int(info >> 56);
}

// The representatives' slots of a saddle record in ascending order (slot
// order is index order); returns their number.
template <int KD>
__device__ __forceinline__ int rec_slots(uint64_t info, int (&k)[CompBound<KD>::value])
{
    constexpr int kCap = CompBound<KD>::value;
    if constexpr (KD == 5) {
        int n = 0;
        for (uint64_t m = info; m && n < kCap; m &= m - 1) k[n++] = __ffsll((long long)m) - 1;
        return n;
    } else {
        int b0 = int((info >> 56) & 0xfu);
        if (b0 > kCap) b0 = kCap;
        for (int c = 0; c < b0; c++) {
            const int v = int((info >> (5 * c)) & 31u);
            int j = c;
            while (j > 0 && k[j - 1] > v) {
                k[j] = k[j - 1];
                j--;
            }
            k[j] = v;
        }
        return b0;
    }
}

// device status word bits (reported by eg_get_graph)
enum : uint32_t {
    kErrNaN = 1u,
    kErrNotConverged = 2u,
    kErrTimeout = 4u,
    kErrInternal = 8u,
    kErrBounds = 16u,  // bounds-checked build: an index out of its array (access skipped)
};

// Bounds-checked build (compiled with EG_CHECKED): every index the kernels
// compute into a field's arrays, the records, the shared-memory rings and the
// outputs is tested against the array's size before the access; an index out
// of range sets kErrBounds in the status word and the access is skipped (a
// load yields 0), so a faulty index is reported, never dereferenced.  The
// regular build compiles the tests away.
#ifdef EG_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// true iff i < n; in the checked build a false also sets kErrBounds
__device__ __forceinline__ bool chk(uint64_t i, uint64_t n, uint32_t *err)
{
    if constexpr (!kChecked) {
        return true;
    } else {
        if (i < n) return true;
        atomicOr(err, kErrBounds);
        return false;
    }
}

// pointer p inside [base, base + n) (elements of p's type)
template <typename T>
__device__ __forceinline__ bool chk_ptr(const T *p, const T *base, uint64_t n, uint32_t *err)
{
    if constexpr (!kChecked) {
        return true;
    } else {
        const bool ok = p >= base && uint64_t(p - base) < n;
        if (!ok) atomicOr(err, kErrBounds);
        return ok;
    }
}

// flags carried per field
enum : uint32_t { kFlagMinimum = 1u, kFlagNoLabels = 2u, kFlagPaths = 8u, kFlagNoFused = 16u };

// element types of a field (the values of eg_dtype)
enum : uint32_t {
    kF32 = 0, kF64 = 1, kI8 = 2, kU8 = 3, kI16 = 4, kU16 = 5, kI32 = 6, kU32 = 7, kI64 = 8, kU64 = 9,
    kNumTypes = 10
};

__host__ __device__ __forceinline__ uint32_t dtype_size(uint32_t t)
{
    return t == kI8 || t == kU8 ? 1u : (t == kI16 || t == kU16 ? 2u : (t == kF64 || t == kI64 || t == kU64 ? 8u : 4u));
}

// Integers of at most 16 bits: exact in float32 with order and ties kept, so
// they are widened to float32 and take the float32 kernels.
__host__ __device__ __forceinline__ bool dtype_narrow(uint32_t t) { return t >= kI8 && t <= kU16; }

// Raw bits of an element type and their order key: a < b (in the type; IEEE
// and non-NaN for floats) <=> key(a) < key(b); -0 and +0 share a key.
template <uint32_t DT>
struct TypeKey;
template <>
struct TypeKey<kF32> {
    using B = uint32_t;
    static __device__ __forceinline__ B key(B u)
    {
        u = (u == 0x80000000u) ? 0u : u;
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
    static __device__ __forceinline__ bool nan(B u) { return (u & 0x7fffffffu) > 0x7f800000u; }
};
template <>
struct TypeKey<kF64> {
    using B = uint64_t;
    static __device__ __forceinline__ B key(B u)
    {
        constexpr B sign = 1ull << 63;
        u = (u == sign) ? 0ull : u;
        return (u & sign) ? ~u : (u | sign);
    }
    static __device__ __forceinline__ bool nan(B u) { return (u & ~(1ull << 63)) > 0x7ff0000000000000ull; }
};
template <>
struct TypeKey<kI32> {
    using B = uint32_t;
    static __device__ __forceinline__ B key(B u) { return u ^ 0x80000000u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kU32> {
    using B = uint32_t;
    static __device__ __forceinline__ B key(B u) { return u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kI64> {
    using B = uint64_t;
    static __device__ __forceinline__ B key(B u) { return u ^ (1ull << 63); }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kI8> {
    using B = uint32_t;  // the 8 bits, zero-extended
    static __device__ __forceinline__ B key(B u) { return u ^ 0x80u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kU8> {
    using B = uint32_t;
    static __device__ __forceinline__ B key(B u) { return u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kI16> {
    using B = uint32_t;  // the 16 bits, zero-extended
    static __device__ __forceinline__ B key(B u) { return u ^ 0x8000u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kU16> {
    using B = uint32_t;
    static __device__ __forceinline__ B key(B u) { return u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};
template <>
struct TypeKey<kU64> {
    using B = uint64_t;
    static __device__ __forceinline__ B key(B u) { return u; }
    static __device__ __forceinline__ bool nan(B) { return false; }
};

// One field as the kernels see it.  Plain pointers; filled on the host.
struct FieldDev {
    const float *f;          // [N] float32 values the float32 kernels read: the field itself,
                             //     or its float32 image (8/16-bit integer fields)
    const void *fraw;        // [N] the field in its own element type (== f for float32)
    uint32_t *lab;           // [N] gradient pointer, then the label (maximum reached)
    // classification records: one slot of bcap entries per brick, index order
    uint32_t *rec_sid;       // vertex id
    uint64_t *rec_info;      // beta0+ (bits 56..59) | rep slots (5 bits each)
    float *rec_val;          // f at the vertex
    uint4 *bcnt;             // [nbricks] maxima, saddles, paths in the brick
    uint4 *boff;             // [nbricks] exclusive offsets: maxima, saddles, paths (lo, hi)
    uint32_t *acnt;          // [nbricks] unique arcs in the brick
    uint64_t *aoff;          // [nbricks] exclusive offsets of unique arcs
    uint32_t *ends;          // [P] sorted unique arc ends, at each saddle's path offset
    uint8_t *ucnt;           // [S] unique arc count per saddle
    // outputs
    uint32_t *maxima;        // [M]
    float *max_val;          // [M] float32 fields (null for other element types)
    uint32_t *saddles;       // [S]
    uint8_t *sad_b0;         // [S]
    float *sad_val;          // [S] float32 fields (null for other element types)
    void *max_raw;           // [M] value copies in the field's element type (non-float32 fields)
    void *sad_raw;           // [S]
    uint64_t *row_ptr;       // [S+1]
    uint32_t *col;           // [A]
    unsigned long long *totals;  // [4] M, S, P, A
    // arc geometry (only when requested, else null)
    uint64_t *path_ptr;      // [P + 1] path lengths, then offsets into path_vtx
    uint32_t *path_vtx;      // [V] saddle, representative, ..., maximum per path
    uint64_t *pbrick;        // [nbricks + 1] path vertices per brick, then offsets and the total
    uint32_t *err;           // device status word
    uint32_t n[kMaxDim];     // extents (1 beyond the kernel dimension)
    uint32_t s[kMaxDim];     // strides
    uint32_t N;              // vertex count (< 2^32)
    uint32_t nbricks;
    uint32_t bcap;           // record slot capacity per brick (= brick size)
    uint32_t ty;             // rows per brick (0: flat layout)
    uint32_t nyb;            // row blocks per plane (row layout)
    uint32_t zc;             // planes per classification work item (row layout)
    uint32_t nzc;            // work items along the slowest axis (row layout)
    uint32_t vec;            // axis-0 extent is a multiple of 4 and f is 16-byte aligned
    uint64_t brick0;         // first global brick id of this field in its launch
    uint64_t item0;          // first classification work item of this field in its launch
    uint64_t stile0;         // first scan tile of this field (all fields of a call)
    uint64_t rtile0;         // first resolution tile of this field (all fields of a call)
    uint32_t rt[3];          // log2 of the resolution tile extents (3D kernels; 0 tiles for 4D)
    int32_t kd;              // kernel dimension (2D fields run as 3D)
    uint32_t flags;
    uint32_t dtype;          // element type of fraw
};

// Record slots of a field (nbricks slots of bcap entries each).
__host__ __device__ __forceinline__ uint64_t rec_cap(const FieldDev &F) { return uint64_t(F.nbricks) * F.bcap; }

__host__ __device__ __forceinline__ void brick_range(const FieldDev &F, uint32_t b, uint64_t &v0, uint32_t &len)
{
    if (F.ty == 0) {
        v0 = uint64_t(b) * kFlatBrick;
        const uint64_t rem = uint64_t(F.N) - v0;
        len = rem < kFlatBrick ? uint32_t(rem) : uint32_t(kFlatBrick);
    } else {
        const uint32_t p = b / F.nyb, yb = b - p * F.nyb;
        const uint32_t y0 = yb * F.ty;
        const uint32_t rows = (F.n[1] - y0) < F.ty ? (F.n[1] - y0) : F.ty;
        v0 = (uint64_t(p) * F.n[1] + y0) * F.n[0];
        len = rows * F.n[0];
    }
}

template <int D>
struct Nbr {
    static constexpr int H = (1 << D) - 1;
    static constexpr int K = 2 * H;
    using Mask = typename std::conditional<(K > 32), uint64_t, uint32_t>::type;  // one bit per slot
    __host__ __device__ static constexpr bool neg(int k) { return k < H; }
    __host__ __device__ static constexpr uint32_t pat(int k) { return k < H ? uint32_t(H - k) : uint32_t(k - H + 1); }
    // rank in index order, centre = H
    __host__ __device__ static constexpr uint32_t rank(int k) { return k < H ? uint32_t(k) : uint32_t(k + 1); }
    __host__ __device__ static constexpr bool linked(int a, int b)
    {
        return a != b && (neg(a) == neg(b) ? ((pat(a) & pat(b)) == pat(a) || (pat(a) & pat(b)) == pat(b))
                                           : ((pat(a) & pat(b)) == 0u));
    }
    __host__ __device__ static constexpr Mask adj_mask(int a)
    {
        Mask m = 0;
        for (int b = 0; b < K; b++)
            if (linked(a, b)) m |= Mask(1) << b;
        return m;
    }
};

// Linear offset (magnitude) of pattern p under strides s (runtime p).
__host__ __device__ __forceinline__ uint32_t pattern_offset(uint32_t p, const uint32_t *s)
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

__device__ __forceinline__ int lowest_bit(uint32_t m) { return __ffs(m) - 1; }
__device__ __forceinline__ int lowest_bit(uint64_t m) { return __ffsll((long long)m) - 1; }

// Connected component of `seed` inside `upper` over the link edges (bitmask
// flood fill; each member is expanded once).
template <typename M>
__device__ __forceinline__ M link_flood(M seed, M upper, const M *s_adj)
{
    M comp = seed, frontier = seed;
    while (frontier) {
        const int k = lowest_bit(frontier);
        frontier &= frontier - 1;
        const M nb = s_adj[k] & upper & ~comp;
        comp |= nb;
        frontier |= nb;
    }
    return comp;
}

// ---------------------------------------------------------------------------
// Link components by axis patterns.  Pattern layout of the link of a D-dim
// vertex: the positive neighbour with axis pattern p (p = 1 .. 2^D - 1) at bit
// p, the negative one at bit 2^D + p.  Two link vertices are joined
// (Algorithm 1 on their difference) iff they have the same sign and
// comparable patterns, or opposite signs and disjoint patterns.  So the link
// neighbours of a set are the supersets of its patterns in the same half and
// the subsets of its patterns and of their complements, where reversing the
// 2^(D+1) bits maps pattern p of one half to pattern ~p of the other: one
// expansion step is a superset closure and a subset closure over the D
// pattern bits of both halves at once, register-only.
// ---------------------------------------------------------------------------
template <int D>
struct PatternLink {
    static constexpr int W = 1 << D;  // bits per half
    using Mask = typename std::conditional<(2 * W > 32), uint64_t, uint32_t>::type;
    // bit of neighbour slot k (slot order of Nbr<D>)
    __host__ __device__ static constexpr int bit(int k) { return k < W - 1 ? W + (W - 1 - k) : k - (W - 1) + 1; }
    // positions whose pattern lacks axis bit i, in both halves
    __host__ __device__ static constexpr Mask lacks(int i)
    {
        Mask m = 0;
        for (int j = 0; j < 2 * W; j++)
            if (!((j & (W - 1)) >> i & 1)) m |= Mask(1) << j;
        return m;
    }
    static __device__ __forceinline__ Mask reverse(Mask x)
    {
        if constexpr (sizeof(Mask) == 8) return __brevll(x);
        else if constexpr (2 * W == 32) return __brev(x);
        else return __brev(x) >> (32 - 2 * W);
    }
    // connected component of s inside u (s a subset of u); the set only
    // grows, so the loop ends within 2W steps
    static __device__ __forceinline__ Mask component(Mask s, Mask u)
    {
        while (true) {
            Mask up = s, dn = s | reverse(s);
#pragma unroll
            for (int i = 0; i < D; i++) {
                up |= (up & lacks(i)) << (1 << i);
                dn |= (dn >> (1 << i)) & lacks(i);
            }
            const Mask n = (up | dn) & u;
            if (n == s || n == u) return n;  // (nothing can join a component that is all of u)
            s = n;
        }
    }
};

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

// Grid-wide barrier of a cooperative kernel (every CTA is resident:
// cooperative launch); count and gen start at zero.  The last CTA to arrive
// resets the count and advances the generation; the others wait for the
// generation to change, for at most about a second (kSpinLimit rounds of a
// growing sleep), after which they set kErrTimeout and report failure
// instead of hanging.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, uint32_t *err)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = *reinterpret_cast<volatile unsigned *>(gen);
        __threadfence();
        if (atomicAdd(count, 1u) == gridDim.x - 1) {
            *reinterpret_cast<volatile unsigned *>(count) = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned ns = 32;
            uint32_t spins = 0;
            while (*reinterpret_cast<volatile unsigned *>(gen) == g) {
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
        const int64_t j = base - lane;
        const uint64_t w = (j >= int64_t(first)) ? ld_volatile_u64(st + j) : kLbPre;
        const bool empty = (w >> 62) == 0;
        if (__any_sync(0xffffffffu, empty)) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                break;
            }
            __nanosleep(ns);
            ns = ns < 256 ? ns * 2 : 256;
            continue;
        }
        const unsigned pmask = __ballot_sync(0xffffffffu, (w >> 62) == 2);
        const int stop = pmask ? (__ffs(pmask) - 1) : 31;
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

// Locate the field that owns global item g, given each field's first item
// (ascending).  `key` selects brick0 or item0.
template <bool kItems>
__device__ __forceinline__ int find_field(const FieldDev *fields, int nf, uint64_t g)
{
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const uint64_t first = kItems ? fields[mid].item0 : fields[mid].brick0;
        if (first <= g) lo = mid;
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
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? scratch[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) scratch[lane] = wi - w;
        if (lane == nw - 1) scratch[32] = wi;
    }
    __syncthreads();
    const uint32_t r = scratch[warp] + inc - x;
    *total = scratch[32];
    __syncthreads();
    return r;
}

}  // namespace eg
