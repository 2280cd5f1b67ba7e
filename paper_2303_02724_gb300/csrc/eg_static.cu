// Allocation-free labels: eg_labels_static (declared in eg.h).
//
// Every other entry point draws its device memory from the handle's pool,
// which grows with cudaMalloc.  Some callers cannot let a library do that:
// their device memory is owned by another allocator (a framework's caching
// allocator, a fixed arena carved out at start-up), they run under a hard
// memory budget, or they sit in a latency-critical loop where cudaMalloc and
// cudaFree may synchronise the whole device.  This entry point uses no memory
// but the caller's input and output buffers and one scratch array compiled
// into the library.
//
// The scratch array lives in device memory as a file-scope __device__
// variable, so every GPU that loads this library holds it until the process
// exits.  Its size is fixed by EG_STATIC_MAX_VERTICES: per vertex one
// classification record (16 bytes) plus per-brick counts and a status word.
//
// Host code must not hand the array's name to a kernel: in host code it is
// only a stand-in for the symbol.  The device address is looked up with
// cudaGetSymbolAddress, with the caller's device current, at the start of
// every call.  The lookup is a host-side query; the first one on a device
// loads this library's device code there, which is what creates the array.
// No address is cached, so a device reset (which unloads the module and may
// move the array) cannot leave a stale address behind.
#include <cstdint>

#include "eg.h"
#include "eg_internal.cuh"
#include "eg_kernels.h"

using namespace eg;

namespace {

constexpr uint64_t kStaticN = EG_STATIC_MAX_VERTICES;
constexpr uint64_t kStaticBricks = (kStaticN + kFlatBrick - 1) / kFlatBrick;
// layout in bytes: rec_info u64[N] | rec_sid u32[N] | rec_val f32[N] | bcnt uint4[bricks] | status
constexpr size_t kOffInfo = 0;
constexpr size_t kOffSid = kOffInfo + 8 * kStaticN;
constexpr size_t kOffVal = kOffSid + 4 * kStaticN;
constexpr size_t kOffCnt = kOffVal + 4 * kStaticN;
constexpr size_t kOffErr = kOffCnt + 16 * kStaticBricks;
constexpr size_t kScratchBytes = kOffErr + 256;

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of the scratch array on the current device.
eg_status scratch_address(unsigned char **out)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return EG_ERR_CUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return EG_OK;
}

}  // namespace

extern "C" eg_status eg_labels_static(const float *field, int d, const int64_t *extents, uint32_t flags,
                                      uint32_t *labels, void *stream)
{
    if (!field || !labels || !extents || d < 1 || d > 4) return EG_ERR_ARG;
    if (flags & ~uint32_t(EG_FLAG_MINIMUM_GRAPH)) return EG_ERR_ARG;
    uint64_t N = 1;
    uint32_t n[kMaxDim], s[kMaxDim];
    for (int i = 0; i < kMaxDim; i++) {
        n[i] = 1;
        s[i] = 0;
    }
    for (int i = 0; i < d; i++) {
        if (extents[i] < 1 || extents[i] > int64_t(kStaticN)) return EG_ERR_ARG;
        s[i] = uint32_t(N);
        N *= uint64_t(extents[i]);
        if (N > kStaticN) return EG_ERR_ARG;  // beyond the scratch array
        n[i] = uint32_t(extents[i]);
    }
    for (int i = d; i < kMaxDim; i++) s[i] = uint32_t(N);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // the call ends in a read-back and a stream synchronisation, neither of
    // which a stream under capture allows
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) {
        cudaGetLastError();
        return EG_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return EG_ERR_ARG;
    unsigned char *scr = nullptr;
    eg_status st = scratch_address(&scr);
    if (st != EG_OK) return st;

    FieldDev F{};
    F.f = field;
    F.lab = labels;
    F.rec_info = reinterpret_cast<uint64_t *>(scr + kOffInfo);
    F.rec_sid = reinterpret_cast<uint32_t *>(scr + kOffSid);
    F.rec_val = reinterpret_cast<float *>(scr + kOffVal);
    F.bcnt = reinterpret_cast<uint4 *>(scr + kOffCnt);
    F.err = reinterpret_cast<uint32_t *>(scr + kOffErr);
    for (int i = 0; i < kMaxDim; i++) {
        F.n[i] = n[i];
        F.s[i] = s[i];
    }
    F.N = uint32_t(N);
    F.nbricks = uint32_t((N + kFlatBrick - 1) / kFlatBrick);
    F.bcap = kFlatBrick;
    F.ty = 0;
    F.kd = d == 4 ? 4 : 3;
    F.flags = (flags & EG_FLAG_MINIMUM_GRAPH) ? kFlagMinimum : 0u;

    // the status word keeps the previous call's bits: clear it first
    cudaError_t e = cudaMemsetAsync(F.err, 0, sizeof(uint32_t), cs);
    if (e == cudaSuccess) e = launch_classify_one(F.kd, F, cs);
    if (e == cudaSuccess) e = launch_resolve_one(F, cs);
    uint32_t herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, F.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EG_ERR_CUDA;
    }
    if (herr & kErrNaN) return EG_ERR_NAN;
    if (herr & kErrNotConverged) return EG_ERR_NOT_CONVERGED;
    if (herr) return EG_ERR_INTERNAL;
    return EG_OK;
}
