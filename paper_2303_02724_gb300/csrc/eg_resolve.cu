// Step (b): every vertex gets the label of the maximum its gradient path
// reaches (Algorithm 2's inner loop, run for all vertices at once).
//
// lab[] holds the gradient pointers on entry and the labels on exit.  Each
// thread follows the pointers from its vertices to a fixed point (a maximum,
// lab[m] == m) and stores it; kIlp walks per thread advance in lock-step so
// their dependent loads overlap.  Threads write only their own vertices; a
// reader that meets an already-finished vertex sees its maximum instead of its
// gradient pointer, which lies on the same path, so the races are benign and
// later walks get shorter.  A walk longer than N steps is impossible (the
// order strictly increases along a path); the bound is a guard that reports
// kErrNotConverged instead of looping.
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kResolveThreads = 256;

// Resolve the labels of brick b of field F, kIlp walks in flight per thread.
template <int kIlp>
__device__ __forceinline__ void resolve_brick(const FieldDev &F, uint32_t b)
{
    uint64_t v0;
    uint32_t len;
    brick_range(F, b, v0, len);
    uint32_t *lab = F.lab;
    for (uint32_t base = threadIdx.x; base < len; base += kIlp * kResolveThreads) {
        uint32_t v[kIlp], u[kIlp];
        uint32_t live = 0;
#pragma unroll
        for (int q = 0; q < kIlp; q++) {
            const uint32_t i = base + q * kResolveThreads;
            v[q] = uint32_t(v0) + i;
            u[q] = v[q];
            if (i < len) {
                u[q] = lab[v[q]];
                if (u[q] != v[q]) live |= 1u << q;
            }
        }
        uint32_t moved = 0, steps = 0;
        while (live) {
#pragma unroll
            for (int q = 0; q < kIlp; q++)
                if ((live >> q) & 1u) {
                    const uint32_t w = lab[u[q]];
                    if (w == u[q]) {
                        live &= ~(1u << q);
                    } else {
                        u[q] = w;
                        moved |= 1u << q;
                    }
                }
            if (++steps > F.N) {
                atomicOr(F.err, kErrNotConverged);
                break;
            }
        }
#pragma unroll
        for (int q = 0; q < kIlp; q++)
            if ((moved >> q) & 1u) lab[v[q]] = u[q];
    }
}

template <int kIlp>
__global__ void __launch_bounds__(kResolveThreads)
k_resolve_chase(const FieldDev *__restrict__ fields, int nf)
{
    const uint64_t g = blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    resolve_brick<kIlp>(F, uint32_t(g - F.brick0));
}

// Single-field variant with the descriptor passed by value.
__global__ void __launch_bounds__(kResolveThreads)
k_resolve_one(const FieldDev F)
{
    resolve_brick<4>(F, blockIdx.x);
}

cudaError_t launch_resolve_one(const FieldDev &F, cudaStream_t st)
{
    if (F.nbricks == 0) return cudaSuccess;
    k_resolve_one<<<dim3(F.nbricks), kResolveThreads, 0, st>>>(F);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const FieldDev *fields, int nf, uint64_t total_bricks, int walks, cudaStream_t st)
{
    if (total_bricks == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>(total_bricks));
    if (walks <= 2) k_resolve_chase<2><<<grid, kResolveThreads, 0, st>>>(fields, nf);
    else if (walks <= 4) k_resolve_chase<4><<<grid, kResolveThreads, 0, st>>>(fields, nf);
    else k_resolve_chase<8><<<grid, kResolveThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
