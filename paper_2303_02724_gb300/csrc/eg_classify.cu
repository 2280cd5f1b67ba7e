// Steps (a) + (c): per-vertex classification (Sec. 3.3, Table 1).
//
// For every vertex v: the gradient pointer asc(v) = highest vertex of the
// upper link (Sec. 3.3), or v at a maximum; beta0+(v), the number of
// connected components of the upper link, found with a bitmask flood fill
// over the link edges of the upper neighbours (the union-find of Sec. 3.3
// restated on a <= 30-bit register mask); and for a saddle the highest vertex
// of each component (UpperLinkRep, Sec. 3.4), recorded as its neighbour slot.
//
// This is the general kernel (any d in 1..4, any extents): one CTA per flat
// brick of kFlatBrick consecutive vertex ids, neighbour values read through
// the read-only cache.  2D/3D float32 fields with rows of at most 1024
// vertices use the plane-marching kernel of eg_classify_zm.cu instead.
//
// It is also the classifier of the 32- and 64-bit element types (Sec. 5):
// values are loaded as raw bits and mapped to order keys of the same width
// (key(a) < key(b) iff a < b in the type itself), so the comparison is exact
// in the type; the simulated-perturbation rank sits below the key.
//
// Every maximum and saddle of a brick is written, in index order, into that
// brick's record slot, so a scan over per-brick counts gives global positions.
#include "eg_flat.cuh"
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kClassifyThreads = 256;
constexpr int kVpt = kFlatBrick / kClassifyThreads;

// Classification of brick b of field F (one CTA, kClassifyThreads threads).
template <int D, uint32_t DT>
__device__ __forceinline__ void classify_brick(const FieldDev &F, uint32_t b)
{
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned s_cnt[3];
    const int tid = threadIdx.x;
    if (tid < 3) s_cnt[tid] = 0;
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    const bool minimum = (F.flags & kFlagMinimum) != 0;
    const uint64_t v0 = uint64_t(b) * kFlatBrick;
    const uint64_t slot = uint64_t(b) * F.bcap;
    __syncthreads();

    // classify this thread's vertices first (no barrier in between, so warps
    // run ahead of one another while their loads are in flight), then place
    // the records with one block scan per round
    int b0s[kVpt];
    uint64_t codess[kVpt];
    bool anynan = false;
#pragma unroll 1
    for (int i = 0; i < kVpt; i++) {
        const uint64_t v64 = v0 + uint64_t(i) * kClassifyThreads + tid;
        b0s[i] = 1;
        codess[i] = 0;
        if (v64 < F.N) {
            bool nan;
            int b0;
            uint64_t codes;
            const uint32_t v = uint32_t(v64);
            F.lab[v] = classify_vertex<D, DT>(F, s, v, minimum, b0, codes, nan);
            anynan |= nan;
            b0s[i] = b0;
            codess[i] = codes;
        }
    }
    uint32_t running = 0, nm = 0, ns = 0, np = 0;
#pragma unroll
    for (int i = 0; i < kVpt; i++) {
        const uint64_t v64 = v0 + uint64_t(i) * kClassifyThreads + tid;
        const int b0 = b0s[i];
        const bool crit = v64 < F.N && b0 != 1;
        uint32_t tot;
        const uint32_t pos = block_excl_scan(crit ? 1u : 0u, s_scan, &tot);
        if (crit && chk(slot + running + pos, rec_cap(F), F.err) && chk(running + pos, F.bcap, F.err)) {
            F.rec_sid[slot + running + pos] = uint32_t(v64);
            F.rec_info[slot + running + pos] = D == 5 ? codess[i] : ((uint64_t(b0) << 56) | codess[i]);
            // (other element types get their value copies from the field
            // itself once the graph is assembled)
            float fv = 0.f;
            if constexpr (DT == kF32) fv = F.f[v64];
            F.rec_val[slot + running + pos] = fv;
            if (b0 == 0) nm++;
            else {
                ns++;
                np += b0;
            }
        }
        running += tot;
    }
    if (anynan) atomicOr(F.err, kErrNaN);
    nm = __reduce_add_sync(0xffffffffu, nm);
    ns = __reduce_add_sync(0xffffffffu, ns);
    np = __reduce_add_sync(0xffffffffu, np);
    if ((tid & 31) == 0) {
        if (nm) atomicAdd(&s_cnt[0], nm);
        if (ns) atomicAdd(&s_cnt[1], ns);
        if (np) atomicAdd(&s_cnt[2], np);
    }
    __syncthreads();
    if (tid == 0 && chk(b, F.nbricks, F.err)) F.bcnt[b] = make_uint4(s_cnt[0], s_cnt[1], s_cnt[2], 0u);
}

template <int D, uint32_t DT>
__global__ void __launch_bounds__(kClassifyThreads)
k_classify(const FieldDev *__restrict__ fields, int nf)
{
    const uint64_t g = fields[0].brick0 + blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    classify_brick<D, DT>(F, uint32_t(g - F.brick0));
}

// Single-field variant with the descriptor passed by value (no descriptor
// table in device memory); used by the allocation-free entry point.
template <int D>
__global__ void __launch_bounds__(kClassifyThreads)
k_classify_one(const FieldDev F)
{
    classify_brick<D, kF32>(F, blockIdx.x);
}

template <int D, uint32_t DT>
cudaError_t launch_classify(const FieldDev *fields, int nf, uint64_t bricks, cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    k_classify<D, DT><<<dim3(unsigned(bricks)), kClassifyThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

template <int D>
cudaError_t launch_classify_typed(uint32_t dtype, const FieldDev *fields, int nf, uint64_t bricks, cudaStream_t st)
{
    switch (dtype) {
    case kF32: return launch_classify<D, kF32>(fields, nf, bricks, st);
    case kF64: return launch_classify<D, kF64>(fields, nf, bricks, st);
    case kI32: return launch_classify<D, kI32>(fields, nf, bricks, st);
    case kU32: return launch_classify<D, kU32>(fields, nf, bricks, st);
    case kI64: return launch_classify<D, kI64>(fields, nf, bricks, st);
    case kU64: return launch_classify<D, kU64>(fields, nf, bricks, st);
    default: return cudaErrorInvalidValue;  // narrow integers are classified as their float32 image
    }
}

cudaError_t launch_classify_one(int kd, const FieldDev &F, cudaStream_t st)
{
    if (F.nbricks == 0) return cudaSuccess;
    if (kd == 4) k_classify_one<4><<<dim3(F.nbricks), kClassifyThreads, 0, st>>>(F);
    else if (kd == 3) k_classify_one<3><<<dim3(F.nbricks), kClassifyThreads, 0, st>>>(F);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_classify_flat(int kd, uint32_t dtype, const FieldDev *fields, int nf, uint64_t bricks,
                                 cudaStream_t st)
{
    switch (kd) {
    case 3: return launch_classify_typed<3>(dtype, fields, nf, bricks, st);
    case 4: return launch_classify_typed<4>(dtype, fields, nf, bricks, st);
    case 5: return launch_classify_typed<5>(dtype, fields, nf, bricks, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace eg
