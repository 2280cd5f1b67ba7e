// Element types other than float32 (Sec. 5 lists 8- to 64-bit integers and
// 32/64-bit floats).
//
// k_widen   An 8- or 16-bit integer is exactly representable in float32, and
//           the conversion keeps both the order and the ties of the values,
//           so such a field is widened once into a float32 image that the
//           float32 classifiers (plane-marching or flat) read; the result is
//           the same as comparing the integers themselves.
// k_values  The value copies of the maxima and saddles come from the field
//           itself, in its own type, once the graph is assembled (the
//           classification records carry float32 values only).
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kTypedThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kTypedThreads)
k_widen(const FieldDev *__restrict__ Fp, uint64_t n)
{
    const T *src = static_cast<const T *>(Fp->fraw);
    float *dst = const_cast<float *>(Fp->f);
    const uint64_t stride = uint64_t(gridDim.x) * kTypedThreads;
    for (uint64_t i = uint64_t(blockIdx.x) * kTypedThreads + threadIdx.x; i < n; i += stride)
        dst[i] = float(src[i]);
}

// T: an unsigned integer of the element's size (the values are copied as bits).
template <typename T>
__global__ void __launch_bounds__(kTypedThreads)
k_values(const FieldDev *__restrict__ Fp)
{
    const FieldDev &F = *Fp;
    const T *src = static_cast<const T *>(F.fraw);
    T *mo = static_cast<T *>(F.max_raw);
    T *so = static_cast<T *>(F.sad_raw);
    const uint64_t M = F.totals[0], S = F.totals[1];
    const uint64_t stride = uint64_t(gridDim.x) * kTypedThreads;
    for (uint64_t i = uint64_t(blockIdx.x) * kTypedThreads + threadIdx.x; i < M + S; i += stride) {
        if (i < M) mo[i] = src[F.maxima[i]];
        else so[i - M] = src[F.saddles[i - M]];
    }
}

static unsigned grid_for(uint64_t work, int sm_count)
{
    const uint64_t want = (work + kTypedThreads - 1) / kTypedThreads;
    const uint64_t cap = uint64_t(sm_count > 0 ? sm_count : 1) * 8;
    return unsigned(want < 1 ? 1 : (want < cap ? want : cap));
}

cudaError_t launch_widen(uint32_t dtype, const FieldDev *field, uint64_t n, int sm_count, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const dim3 grid(grid_for(n, sm_count));
    switch (dtype) {
    case kI8: k_widen<int8_t><<<grid, kTypedThreads, 0, st>>>(field, n); break;
    case kU8: k_widen<uint8_t><<<grid, kTypedThreads, 0, st>>>(field, n); break;
    case kI16: k_widen<int16_t><<<grid, kTypedThreads, 0, st>>>(field, n); break;
    case kU16: k_widen<uint16_t><<<grid, kTypedThreads, 0, st>>>(field, n); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_values(uint32_t dtype, const FieldDev *field, int sm_count, cudaStream_t st)
{
    // the counts are only known on the device: a grid sized for the GPU,
    // striding over M + S
    const dim3 grid(unsigned(sm_count > 0 ? sm_count : 1) * 4);
    switch (dtype_size(dtype)) {
    case 1: k_values<uint8_t><<<grid, kTypedThreads, 0, st>>>(field); break;
    case 2: k_values<uint16_t><<<grid, kTypedThreads, 0, st>>>(field); break;
    case 4: k_values<uint32_t><<<grid, kTypedThreads, 0, st>>>(field); break;
    default: k_values<unsigned long long><<<grid, kTypedThreads, 0, st>>>(field); break;
    }
    return cudaGetLastError();
}

}  // namespace eg
