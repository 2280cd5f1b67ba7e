// Steps (d) + (e): arcs and graph assembly.
//
// k_nodes (one warp per brick): the brick's maxima and saddles go to their
// final, index-sorted positions (brick offsets from scan A plus an in-brick
// scan); for every saddle s and every upper-link component C recorded by the
// classification, the arc end is label(rep(C)) (Sec. 3.4, Algorithm 2:
// following the gradient from UpperLinkRep reaches that maximum; Sec. 2: arc
// (s, m) iff s bounds the descending manifold of m).  The ends of a saddle are
// sorted and de-duplicated in registers and parked at the saddle's path offset;
// the brick's unique-arc count feeds scan B.
//
// k_csr (one warp per brick): row_ptr from the unique counts (scan B offsets
// plus an in-brick scan) and col, copied from the parked ends.
#include "eg_emit.cuh"
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kEmitThreads = 256;

// One warp per brick (kEmitThreads / 32 bricks per CTA): the brick's maxima and
// saddles go to their final positions, each saddle's sorted unique arc ends are
// parked at its path offset, and the brick's unique-arc count is stored.
template <int KD>
__global__ void __launch_bounds__(kEmitThreads)
k_nodes(const FieldDev *__restrict__ fields, int nf, uint64_t base, uint64_t bricks)
{
    const uint64_t t = uint64_t(blockIdx.x) * (kEmitThreads / 32) + (threadIdx.x >> 5);
    if (t >= bricks) return;
    const uint64_t g = base + t;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    nodes_brick<KD>(F, uint32_t(g - F.brick0));
}

// One warp per brick: row_ptr from the unique counts (scan offsets plus an
// in-brick warp scan) and col, copied from the parked ends.
__global__ void __launch_bounds__(kEmitThreads)
k_csr(const FieldDev *__restrict__ fields, int nf, uint64_t bricks)
{
    const uint64_t g = uint64_t(blockIdx.x) * (kEmitThreads / 32) + (threadIdx.x >> 5);
    if (g >= bricks) return;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    csr_brick(F, uint32_t(g - F.brick0));
}

cudaError_t launch_nodes_d(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks, cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>((bricks + kEmitThreads / 32 - 1) / (kEmitThreads / 32)));
    if (kd == 5) k_nodes<5><<<grid, kEmitThreads, 0, st>>>(fields, nf, base, bricks);
    else if (kd == 4) k_nodes<4><<<grid, kEmitThreads, 0, st>>>(fields, nf, base, bricks);
    else k_nodes<3><<<grid, kEmitThreads, 0, st>>>(fields, nf, base, bricks);
    return cudaGetLastError();
}

cudaError_t launch_csr(const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st)
{
    if (total_bricks == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>((total_bricks + kEmitThreads / 32 - 1) / (kEmitThreads / 32)));
    k_csr<<<grid, kEmitThreads, 0, st>>>(fields, nf, total_bricks);
    return cudaGetLastError();
}

}  // namespace eg
