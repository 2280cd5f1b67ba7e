// Arc bundling (Sec. 3.5): when several saddles connect the same two maxima,
// only the highest of them (value, then index; the lowest for the minimum
// graph) stands for that pair.  A saddle is kept when it stands for at least
// one pair of its arc ends; a saddle whose arcs all end at one maximum
// connects no pair and is kept.
//
// On the finished graph (saddle list, values, CSR of unique sorted ends):
//   k_bundle_pairs   counts the pairs (u(u-1)/2 for u unique ends)
//   k_bundle_insert  open-addressing hash table keyed by the pair (m1 < m2);
//                    each slot keeps the highest saddle key (atomicMax)
//   k_bundle_keep    a saddle is kept iff it owns some pair's slot
// The saddle key orders saddles by the simulated perturbation: the float's
// order-preserving bits (with -0 taken as +0) above the vertex id; both are
// complemented for the minimum graph.  Probing is bounded by the table size.
//
// Other element types (up to 64-bit values): the value key alone fills a
// 64-bit word, so the highest saddle of a pair is found in two rounds -- the
// largest value key per slot, then the largest vertex id among the saddles
// holding that value key -- and a saddle is kept iff it holds both for some
// pair.
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kBundleThreads = 256;
constexpr uint64_t kEmptyPair = ~0ull;

__device__ __forceinline__ uint64_t saddle_key(float v, uint32_t id, bool minimum)
{
    uint32_t b = __float_as_uint(v);
    if ((b << 1) == 0) b = 0;  // -0 == +0
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    const uint64_t k = (uint64_t(b) << 32) | id;
    return minimum ? ~k : k;
}

__device__ __forceinline__ uint64_t pair_slot(uint64_t key, uint32_t lg)
{
    return (key * 0x9e3779b97f4a7c15ull) >> (64 - lg);
}

__global__ void __launch_bounds__(kBundleThreads)
k_bundle_pairs(const uint64_t *row_ptr, uint64_t S, unsigned long long *count)
{
    const uint64_t i = uint64_t(blockIdx.x) * kBundleThreads + threadIdx.x;
    uint64_t n = 0;
    if (i < S) {
        const uint64_t u = row_ptr[i + 1] - row_ptr[i];
        n = u * (u - 1) / 2;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, (unsigned long long)n);
}

// Slot of `pair` (inserting it when `insert`), or kEmptyPair when the table
// is full (cannot happen: at least twice as many slots as pairs).
__device__ __forceinline__ uint64_t find_pair(unsigned long long *keys, uint32_t lg, uint64_t pair, bool insert)
{
    const uint64_t mask = (1ull << lg) - 1;
    uint64_t h = pair_slot(pair, lg);
    for (uint64_t probe = 0; probe <= mask; probe++, h = (h + 1) & mask) {
        unsigned long long cur = keys[h];
        if (cur == pair) return h;
        if (cur == kEmptyPair) {
            if (!insert) return kEmptyPair;
            cur = atomicCAS(keys + h, kEmptyPair, (unsigned long long)pair);
            if (cur == kEmptyPair || cur == pair) return h;
        }
    }
    return kEmptyPair;
}

__global__ void __launch_bounds__(kBundleThreads)
k_bundle_insert(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles, const float *sad_val,
                uint64_t S, bool minimum, unsigned long long *keys, unsigned long long *best, uint32_t lg,
                uint32_t *err)
{
    const uint64_t i = uint64_t(blockIdx.x) * kBundleThreads + threadIdx.x;
    if (i >= S) return;
    const uint64_t a0 = row_ptr[i], a1 = row_ptr[i + 1];
    const uint64_t k = saddle_key(sad_val[i], saddles[i], minimum);
    for (uint64_t a = a0; a < a1; a++)
        for (uint64_t b = a + 1; b < a1; b++) {
            const uint64_t pair = (uint64_t(col[a]) << 32) | col[b];
            const uint64_t h = find_pair(keys, lg, pair, true);
            if (h == kEmptyPair) atomicOr(err, kErrInternal);
            else atomicMax(best + h, (unsigned long long)k);
        }
}

__global__ void __launch_bounds__(kBundleThreads)
k_bundle_keep(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles, const float *sad_val,
              uint64_t S, bool minimum, unsigned long long *keys, const unsigned long long *best, uint32_t lg,
              uint8_t *keep)
{
    const uint64_t i = uint64_t(blockIdx.x) * kBundleThreads + threadIdx.x;
    if (i >= S) return;
    const uint64_t a0 = row_ptr[i], a1 = row_ptr[i + 1];
    const uint64_t k = saddle_key(sad_val[i], saddles[i], minimum);
    bool kept = a1 - a0 < 2;
    for (uint64_t a = a0; a < a1 && !kept; a++)
        for (uint64_t b = a + 1; b < a1 && !kept; b++) {
            const uint64_t pair = (uint64_t(col[a]) << 32) | col[b];
            const uint64_t h = find_pair(keys, lg, pair, false);
            kept = h != kEmptyPair && best[h] == k;
        }
    keep[i] = kept ? 1 : 0;
}

// Value key of saddle i of a non-float32 field (complemented for the minimum graph).
template <uint32_t DT>
__device__ __forceinline__ uint64_t typed_value_key(const void *sad_raw, uint64_t i, bool minimum)
{
    using TK = TypeKey<DT>;
    uint64_t b;
    if constexpr (DT == kI8 || DT == kU8) b = static_cast<const uint8_t *>(sad_raw)[i];
    else if constexpr (DT == kI16 || DT == kU16) b = static_cast<const uint16_t *>(sad_raw)[i];
    else if constexpr (sizeof(typename TK::B) == 4) b = static_cast<const uint32_t *>(sad_raw)[i];
    else b = static_cast<const unsigned long long *>(sad_raw)[i];
    const uint64_t k = uint64_t(TK::key(typename TK::B(b)));
    return minimum ? ~k : k;
}

// round 0: value keys; round 1: vertex ids among the saddles holding the
// slot's value key
template <uint32_t DT, int ROUND>
__global__ void __launch_bounds__(kBundleThreads)
k_bundle_typed_insert(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles, const void *sad_raw,
                      uint64_t S, bool minimum, unsigned long long *keys, unsigned long long *best,
                      unsigned int *best_id, uint32_t lg, uint32_t *err)
{
    const uint64_t i = uint64_t(blockIdx.x) * kBundleThreads + threadIdx.x;
    if (i >= S) return;
    const uint64_t a0 = row_ptr[i], a1 = row_ptr[i + 1];
    const uint64_t k = typed_value_key<DT>(sad_raw, i, minimum);
    const uint32_t id = minimum ? ~saddles[i] : saddles[i];
    for (uint64_t a = a0; a < a1; a++)
        for (uint64_t b = a + 1; b < a1; b++) {
            const uint64_t pair = (uint64_t(col[a]) << 32) | col[b];
            const uint64_t h = find_pair(keys, lg, pair, ROUND == 0);
            if (h == kEmptyPair) atomicOr(err, kErrInternal);
            else if (ROUND == 0) atomicMax(best + h, (unsigned long long)k);
            else if (best[h] == k) atomicMax(best_id + h, id);
        }
}

template <uint32_t DT>
__global__ void __launch_bounds__(kBundleThreads)
k_bundle_typed_keep(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles, const void *sad_raw,
                    uint64_t S, bool minimum, unsigned long long *keys, const unsigned long long *best,
                    const unsigned int *best_id, uint32_t lg, uint8_t *keep)
{
    const uint64_t i = uint64_t(blockIdx.x) * kBundleThreads + threadIdx.x;
    if (i >= S) return;
    const uint64_t a0 = row_ptr[i], a1 = row_ptr[i + 1];
    const uint64_t k = typed_value_key<DT>(sad_raw, i, minimum);
    const uint32_t id = minimum ? ~saddles[i] : saddles[i];
    bool kept = a1 - a0 < 2;
    for (uint64_t a = a0; a < a1 && !kept; a++)
        for (uint64_t b = a + 1; b < a1 && !kept; b++) {
            const uint64_t pair = (uint64_t(col[a]) << 32) | col[b];
            const uint64_t h = find_pair(keys, lg, pair, false);
            kept = h != kEmptyPair && best[h] == k && best_id[h] == id;
        }
    keep[i] = kept ? 1 : 0;
}

template <uint32_t DT>
cudaError_t launch_bundle_typed_t(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles,
                                  const void *sad_raw, uint64_t S, bool minimum, unsigned long long *keys,
                                  unsigned long long *best, unsigned int *best_id, uint32_t lg, uint8_t *keep,
                                  uint32_t *err, cudaStream_t st)
{
    const dim3 grid = dim3(static_cast<unsigned>((S + kBundleThreads - 1) / kBundleThreads));
    k_bundle_typed_insert<DT, 0><<<grid, kBundleThreads, 0, st>>>(row_ptr, col, saddles, sad_raw, S, minimum, keys,
                                                                  best, best_id, lg, err);
    k_bundle_typed_insert<DT, 1><<<grid, kBundleThreads, 0, st>>>(row_ptr, col, saddles, sad_raw, S, minimum, keys,
                                                                  best, best_id, lg, err);
    k_bundle_typed_keep<DT><<<grid, kBundleThreads, 0, st>>>(row_ptr, col, saddles, sad_raw, S, minimum, keys, best,
                                                            best_id, lg, keep);
    return cudaGetLastError();
}

cudaError_t launch_bundle_typed(uint32_t dtype, const uint64_t *row_ptr, const uint32_t *col,
                                const uint32_t *saddles, const void *sad_raw, uint64_t S, bool minimum,
                                unsigned long long *keys, unsigned long long *best, unsigned int *best_id,
                                uint32_t lg, uint8_t *keep, uint32_t *err, cudaStream_t st)
{
    if (S == 0) return cudaSuccess;
#define EG_BUNDLE_CASE(T) \
    case T: return launch_bundle_typed_t<T>(row_ptr, col, saddles, sad_raw, S, minimum, keys, best, best_id, lg, \
                                            keep, err, st);
    switch (dtype) {
        EG_BUNDLE_CASE(kF64)
        EG_BUNDLE_CASE(kI8)
        EG_BUNDLE_CASE(kU8)
        EG_BUNDLE_CASE(kI16)
        EG_BUNDLE_CASE(kU16)
        EG_BUNDLE_CASE(kI32)
        EG_BUNDLE_CASE(kU32)
        EG_BUNDLE_CASE(kI64)
        EG_BUNDLE_CASE(kU64)
    default: return cudaErrorInvalidValue;
    }
#undef EG_BUNDLE_CASE
}

cudaError_t launch_bundle_pairs(const uint64_t *row_ptr, uint64_t S, unsigned long long *count, cudaStream_t st)
{
    if (S == 0) return cudaSuccess;
    k_bundle_pairs<<<dim3(static_cast<unsigned>((S + kBundleThreads - 1) / kBundleThreads)), kBundleThreads, 0,
                     st>>>(row_ptr, S, count);
    return cudaGetLastError();
}

cudaError_t launch_bundle(const uint64_t *row_ptr, const uint32_t *col, const uint32_t *saddles,
                          const float *sad_val, uint64_t S, bool minimum, unsigned long long *keys,
                          unsigned long long *best, uint32_t lg, uint8_t *keep, uint32_t *err, cudaStream_t st)
{
    if (S == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>((S + kBundleThreads - 1) / kBundleThreads));
    k_bundle_insert<<<grid, kBundleThreads, 0, st>>>(row_ptr, col, saddles, sad_val, S, minimum, keys, best, lg,
                                                     err);
    k_bundle_keep<<<grid, kBundleThreads, 0, st>>>(row_ptr, col, saddles, sad_val, S, minimum, keys, best, lg,
                                                   keep);
    return cudaGetLastError();
}

}  // namespace eg
