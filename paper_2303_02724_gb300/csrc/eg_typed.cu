// Element types other than float32 (Sec. 5 lists 8- to 64-bit integers and
// 32/64-bit floats).
//
// An 8- or 16-bit integer is exactly representable in float32, and the
// conversion keeps both the order and the ties of the values, so such a field
// is widened once into a float32 image that the float32 classifiers
// (plane-marching or flat) read; the result is the same as comparing the
// integers themselves.  (The 32/64-bit types are compared as order keys of
// their own width by the flat classifier; the value copies of every
// non-float32 type come from the field itself, in the node kernel.)
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kWidenThreads = 256;

// 16 bytes of the field per step: 16 (8-bit) or 8 (16-bit) elements, written
// as float4s; the ragged tail (and a field not aligned to 16 bytes) one
// element per thread.
template <typename T>
__global__ void __launch_bounds__(kWidenThreads)
k_widen(const FieldDev *__restrict__ Fp, uint64_t n)
{
    constexpr int kPer = 16 / int(sizeof(T));
    const T *src = static_cast<const T *>(Fp->fraw);
    float *dst = const_cast<float *>(Fp->f);
    const uint64_t tid = uint64_t(blockIdx.x) * kWidenThreads + threadIdx.x;
    const uint64_t stride = uint64_t(gridDim.x) * kWidenThreads;
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    const uint64_t nvec = aligned ? n / kPer : 0;
    for (uint64_t i = tid; i < nvec; i += stride) {
        const uint4 q = reinterpret_cast<const uint4 *>(src)[i];
        T e[kPer];
        static_assert(sizeof(e) == sizeof(q), "one 16-byte chunk");
        memcpy(e, &q, sizeof(q));
        float4 *o = reinterpret_cast<float4 *>(dst + i * kPer);
#pragma unroll
        for (int j = 0; j < kPer / 4; j++)
            o[j] = make_float4(float(e[4 * j]), float(e[4 * j + 1]), float(e[4 * j + 2]), float(e[4 * j + 3]));
    }
    for (uint64_t i = nvec * kPer + tid; i < n; i += stride) dst[i] = float(src[i]);
}

cudaError_t launch_widen(uint32_t dtype, const FieldDev *field, uint64_t n, int sm_count, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const uint64_t want = (n / 8 + kWidenThreads - 1) / kWidenThreads;
    const uint64_t cap = uint64_t(sm_count > 0 ? sm_count : 1) * 8;
    const dim3 grid(unsigned(want < 1 ? 1 : (want < cap ? want : cap)));
    switch (dtype) {
    case kI8: k_widen<int8_t><<<grid, kWidenThreads, 0, st>>>(field, n); break;
    case kU8: k_widen<uint8_t><<<grid, kWidenThreads, 0, st>>>(field, n); break;
    case kI16: k_widen<int16_t><<<grid, kWidenThreads, 0, st>>>(field, n); break;
    case kU16: k_widen<uint16_t><<<grid, kWidenThreads, 0, st>>>(field, n); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace eg
