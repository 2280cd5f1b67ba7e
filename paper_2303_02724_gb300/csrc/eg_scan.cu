// Prefix sums over the bricks of every field (step e, stream compaction).
//
// scan A: per-brick (maxima, saddles, paths) counts from classification ->
//         exclusive offsets per brick, and the field totals M, S, P.
// scan B: per-brick unique-arc counts -> exclusive offsets, and the total A.
//
// Single pass: scan tiles of kScanTile consecutive bricks of one field are
// taken in ticket order and chained with a segmented decoupled look-back (the
// chain restarts at each field's first tile).
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ uint64_t block_excl_scan64(uint64_t x, uint64_t *scratch, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint64_t w = lane < nw ? scratch[lane] : 0;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) scratch[lane] = wi - w;
        if (lane == nw - 1) scratch[32] = wi;
    }
    __syncthreads();
    const uint64_t r = scratch[warp] + inc - x;
    *total = scratch[32];
    __syncthreads();
    return r;
}

// Field owning scan tile t (fields ordered by first tile `stile0`).
__device__ __forceinline__ int field_of_tile(const FieldDev *fields, int nf, uint64_t t)
{
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fields[mid].stile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// NV = 3: scan A (bcnt -> boff, totals[0..2]); NV = 1: scan B (acnt -> aoff, totals[3]).
template <int NV>
__global__ void __launch_bounds__(kScanThreads)
k_scan_bricks(const FieldDev *__restrict__ fields, int nf, uint64_t total_tiles, unsigned long long *ticket,
              uint64_t *lb)
{
    __shared__ unsigned long long s_t;
    __shared__ uint64_t s_scan[NV][33];
    __shared__ uint64_t s_pref[NV];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_t = atomicAdd(ticket, 1ull);
    __syncthreads();
    const uint64_t t = s_t;
    if (t >= total_tiles) return;
    const int fi = field_of_tile(fields, nf, t);
    const FieldDev &F = fields[fi];
    const uint64_t first_tile = F.stile0;
    const uint32_t b0 = uint32_t(t - first_tile) * kScanTile;
    uint64_t loc[NV][kScanPer];
    uint64_t sum[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) sum[q] = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        const uint32_t b = b0 + uint32_t(tid) * kScanPer + j;
        uint64_t c[3] = {0, 0, 0};
        if (b < F.nbricks) {
            if (NV == 3) {
                const uint4 x = F.bcnt[b];
                c[0] = x.x;
                c[1] = x.y;
                c[2] = x.z;
            } else {
                c[0] = F.acnt[b];
            }
        }
#pragma unroll
        for (int q = 0; q < NV; q++) {
            loc[q][j] = sum[q];
            sum[q] += c[q];
        }
    }
    uint64_t ex[NV], tot[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) ex[q] = block_excl_scan64(sum[q], s_scan[q], &tot[q]);
    if (warp < NV) {
        const uint64_t p = warp_lookback(lb + uint64_t(warp) * total_tiles, t, first_tile, tot[warp], F.err);
        if (lane == 0) s_pref[warp] = p;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanPer; j++) {
        const uint32_t b = b0 + uint32_t(tid) * kScanPer + j;
        if (b >= F.nbricks) break;
        if (NV == 3) {
            const uint64_t po = s_pref[2] + ex[2] + loc[2][j];
            F.boff[b] = make_uint4(uint32_t(s_pref[0] + ex[0] + loc[0][j]), uint32_t(s_pref[1] + ex[1] + loc[1][j]),
                                   uint32_t(po), uint32_t(po >> 32));
        } else {
            F.aoff[b] = s_pref[0] + ex[0] + loc[0][j];
        }
    }
    // the field's last tile publishes the totals
    if (tid == 0 && b0 + kScanTile >= F.nbricks) {
        if (NV == 3) {
            F.totals[0] = s_pref[0] + tot[0];
            F.totals[1] = s_pref[1] + tot[1];
            F.totals[2] = s_pref[2] + tot[2];
        } else {
            F.totals[3] = s_pref[0] + tot[0];
        }
    }
}

// Zero every field's totals and status word (through the descriptor table, so
// a captured graph can replay it for new result buffers).
__global__ void k_init_fields(const FieldDev *__restrict__ fields, int nf)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const FieldDev &F = fields[i];
    F.totals[0] = F.totals[1] = F.totals[2] = F.totals[3] = 0;
    *F.err = 0;
}

cudaError_t launch_init_fields(const FieldDev *fields, int nf, cudaStream_t st)
{
    if (nf <= 0) return cudaSuccess;
    k_init_fields<<<dim3(unsigned((nf + 127) / 128)), 128, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

// Test hook: one warp waits, through the look-back, for a predecessor that
// never publishes; the bounded wait must give up and report kErrTimeout.
__global__ void k_lookback_orphan(uint64_t *st, uint32_t *err)
{
    warp_lookback(st, 1, 0, 1, err);
}

cudaError_t launch_lookback_orphan(uint64_t *st, uint32_t *err, cudaStream_t s)
{
    k_lookback_orphan<<<1, 32, 0, s>>>(st, err);
    return cudaGetLastError();
}

uint64_t scan_tiles(uint32_t nbricks) { return (uint64_t(nbricks) + kScanTile - 1) / kScanTile; }

size_t scan_workspace_bytes(uint64_t total_tiles) { return 256 + 4 * total_tiles * sizeof(uint64_t); }

cudaError_t launch_scan(bool arcs, const FieldDev *fields, int nf, uint64_t total_tiles, void *ws, cudaStream_t st)
{
    if (total_tiles == 0) return cudaSuccess;
    auto *ticket = reinterpret_cast<unsigned long long *>(ws) + (arcs ? 1 : 0);
    auto *lb = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(ws) + 256) + (arcs ? 3 * total_tiles : 0);
    if (arcs)
        k_scan_bricks<1><<<dim3(unsigned(total_tiles)), kScanThreads, 0, st>>>(fields, nf, total_tiles, ticket,
                                                                               lb);
    else
        k_scan_bricks<3><<<dim3(unsigned(total_tiles)), kScanThreads, 0, st>>>(fields, nf, total_tiles, ticket,
                                                                               lb);
    return cudaGetLastError();
}

}  // namespace eg
