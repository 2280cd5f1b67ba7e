// Step (b): every vertex gets the label of the maximum its gradient path
// reaches (Algorithm 2's inner loop, run for all vertices at once).
//
// lab[] holds the gradient pointers on entry and the labels on exit.  Each
// thread follows the pointers from its vertex to a fixed point (a maximum,
// lab[m] == m) and stores it.  Threads write only their own vertex; a reader
// that meets an already-finished vertex sees its maximum instead of its
// gradient pointer, which lies on the same path, so the races are benign and
// later walks get shorter.  A walk longer than N steps is impossible (the
// order strictly increases along a path); the bound is a guard that reports
// kErrNotConverged instead of looping.
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kResolveThreads = 256;

__global__ void __launch_bounds__(kResolveThreads)
k_resolve_chase(const FieldDev *__restrict__ fields, int nf)
{
    const uint64_t g = blockIdx.x;
    const int fi = find_field(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint64_t v0 = (g - F.brick0) * kBrick;
    uint32_t *lab = F.lab;
    for (int i = threadIdx.x; i < kBrick; i += kResolveThreads) {
        const uint64_t v64 = v0 + i;
        if (v64 >= F.N) break;
        const uint32_t v = uint32_t(v64);
        uint32_t u = lab[v];
        if (u == v) continue;
        uint64_t steps = 0;
        while (true) {
            uint32_t w = lab[u];
            if (w == u) break;
            u = w;
            if (++steps > F.N) {
                atomicOr(F.err, kErrNotConverged);
                break;
            }
        }
        lab[v] = u;
    }
}

cudaError_t launch_resolve(const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st)
{
    if (total_bricks == 0) return cudaSuccess;
    k_resolve_chase<<<dim3(unsigned(total_bricks)), kResolveThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
