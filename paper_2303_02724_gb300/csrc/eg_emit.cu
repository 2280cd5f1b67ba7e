// Steps (d) + (e): arcs and graph assembly.
//
// k_nodes (one CTA per brick): the brick's maxima and saddles go to their
// final, index-sorted positions (brick offsets from scan A plus an in-brick
// scan); for every saddle s and every upper-link component C recorded by the
// classification, the arc end is label(rep(C)) (Sec. 3.4, Algorithm 2:
// following the gradient from UpperLinkRep reaches that maximum; Sec. 2: arc
// (s, m) iff s bounds the descending manifold of m).  The ends of a saddle are
// sorted and de-duplicated in registers and parked at the saddle's path offset;
// the brick's unique-arc count feeds scan B.
//
// k_csr (one CTA per brick): row_ptr from the unique counts (scan B offsets
// plus an in-brick scan) and col, copied from the parked ends.
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kEmitThreads = 256;
constexpr int kRpt = 1;
constexpr int kChunk = kEmitThreads * kRpt;

__device__ __forceinline__ uint64_t block_excl_scan_u64(uint64_t x, uint64_t *scratch, uint64_t *total)
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

// Sorted unique arc ends of one saddle; returns their count.
template <int KD>
__device__ __forceinline__ int saddle_ends(const uint32_t *lab, const uint32_t (&s)[kMaxDim], uint32_t sid,
                                           uint64_t info, uint32_t (&t)[kMaxComp])
{
    const int b0 = int((info >> 56) & 0xfu);
    int n = 0;
    for (int c = 0; c < b0 && c < kMaxComp; c++) {
        const int k = int((info >> (5 * c)) & 31u);
        const uint32_t m = lab[slot_vertex<KD>(sid, k, s)];
        int j = n;
        bool dup = false;
        while (j > 0 && t[j - 1] >= m) {
            if (t[j - 1] == m) {
                dup = true;
                break;
            }
            j--;
        }
        if (dup) continue;
        for (int q = n; q > j; q--) t[q] = t[q - 1];
        t[j] = m;
        n++;
    }
    return n;
}

template <int KD>
__global__ void __launch_bounds__(kEmitThreads)
k_nodes(const FieldDev *__restrict__ fields, int nf, uint64_t base)
{
    __shared__ uint64_t s_scan[33];
    __shared__ unsigned s_asum;
    const int tid = threadIdx.x;
    const uint64_t g = base + blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint32_t b = uint32_t(g - F.brick0);
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    const uint4 c = F.bcnt[b];
    const uint4 o = F.boff[b];
    const uint32_t nrec = c.x + c.y;
    const uint64_t m_off = o.x, s_off = o.y, p_off = uint64_t(o.z) | (uint64_t(o.w) << 32);
    const uint64_t capM = F.totals[0], capS = F.totals[1], capP = F.totals[2];
    const uint64_t slot = uint64_t(b) * F.bcap;
    if (tid == 0) s_asum = 0;
    uint64_t run = 0;  // packed running prefix: maxima | saddles << 16 | paths << 32
    uint32_t asum = 0;
    uint32_t tmp[kMaxComp];
    for (uint32_t chunk = 0; chunk < nrec; chunk += kChunk) {
        uint32_t sid[kRpt];
        uint64_t info[kRpt];
        float val[kRpt];
        uint64_t mine = 0;
#pragma unroll
        for (int j = 0; j < kRpt; j++) {
            const uint32_t r = chunk + uint32_t(tid) * kRpt + j;
            info[j] = ~0ull;
            if (r < nrec) {
                sid[j] = F.rec_sid[slot + r];
                info[j] = F.rec_info[slot + r];
                val[j] = F.rec_val[slot + r];
                const uint64_t b0 = info[j] >> 56;
                mine += b0 == 0 ? 1ull : ((1ull << 16) | (b0 << 32));
            }
        }
        uint64_t tot;
        uint64_t pos = run + block_excl_scan_u64(mine, s_scan, &tot);
        run += tot;
#pragma unroll
        for (int j = 0; j < kRpt; j++) {
            if (info[j] == ~0ull) continue;
            const uint64_t b0 = info[j] >> 56;
            const uint64_t lm = pos & 0xffffu, ls = (pos >> 16) & 0xffffu, lp = pos >> 32;
            if (b0 == 0) {
                const uint64_t q = m_off + lm;
                if (q < capM) {
                    F.maxima[q] = sid[j];
                    F.max_val[q] = val[j];
                } else {
                    atomicOr(F.err, kErrInternal);
                }
                pos += 1;
            } else {
                const uint64_t q = s_off + ls, p = p_off + lp;
                const int u = saddle_ends<KD>(F.lab, s, sid[j], info[j], tmp);
                if (q < capS && p + b0 <= capP) {
                    F.saddles[q] = sid[j];
                    F.sad_b0[q] = uint8_t(b0);
                    F.sad_val[q] = val[j];
                    F.ucnt[q] = uint8_t(u);
                    for (int e = 0; e < u; e++) F.ends[p + e] = tmp[e];
                } else {
                    atomicOr(F.err, kErrInternal);
                }
                asum += uint32_t(u);
                pos += (1ull << 16) | (b0 << 32);
            }
        }
    }
    asum = __reduce_add_sync(0xffffffffu, asum);
    if ((tid & 31) == 0 && asum) atomicAdd(&s_asum, asum);
    __syncthreads();
    if (tid == 0) F.acnt[b] = s_asum;
}

__global__ void __launch_bounds__(kEmitThreads)
k_csr(const FieldDev *__restrict__ fields, int nf)
{
    __shared__ uint64_t s_scan[33];
    const int tid = threadIdx.x;
    const uint64_t g = blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint32_t b = uint32_t(g - F.brick0);
    const uint4 c = F.bcnt[b];
    const uint4 o = F.boff[b];
    const uint32_t ns = c.y;
    const uint64_t s_off = o.y, p_off = uint64_t(o.z) | (uint64_t(o.w) << 32);
    const uint64_t a_off = F.aoff[b];
    const uint64_t capS = F.totals[1], capP = F.totals[2], capA = F.totals[3];
    uint64_t run = 0;  // packed running prefix: unique arcs | paths << 32
    for (uint32_t chunk = 0; chunk < ns; chunk += kChunk) {
        uint32_t u[kRpt], b0[kRpt];
        uint64_t mine = 0;
#pragma unroll
        for (int j = 0; j < kRpt; j++) {
            const uint32_t r = chunk + uint32_t(tid) * kRpt + j;
            u[j] = 0;
            b0[j] = 0;
            if (r < ns && s_off + r < capS) {
                u[j] = F.ucnt[s_off + r];
                b0[j] = F.sad_b0[s_off + r];
                mine += uint64_t(u[j]) | (uint64_t(b0[j]) << 32);
            }
        }
        uint64_t tot;
        uint64_t pos = run + block_excl_scan_u64(mine, s_scan, &tot);
        run += tot;
#pragma unroll
        for (int j = 0; j < kRpt; j++) {
            const uint32_t r = chunk + uint32_t(tid) * kRpt + j;
            if (r < ns && s_off + r < capS) {
                const uint64_t a = a_off + (pos & 0xffffffffu), p = p_off + (pos >> 32);
                F.row_ptr[s_off + r] = a;
                if (a + u[j] <= capA && p + u[j] <= capP) {
                    for (uint32_t e = 0; e < u[j]; e++) F.col[a + e] = F.ends[p + e];
                } else {
                    atomicOr(F.err, kErrInternal);
                }
                pos += uint64_t(u[j]) | (uint64_t(b0[j]) << 32);
            }
        }
    }
    if (tid == 0 && b == F.nbricks - 1) {
        if (s_off + ns == capS && a_off + F.acnt[b] == capA) F.row_ptr[capS] = capA;
        else atomicOr(F.err, kErrInternal);
    }
}

cudaError_t launch_nodes_d(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks, cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    if (kd == 4) k_nodes<4><<<dim3(unsigned(bricks)), kEmitThreads, 0, st>>>(fields, nf, base);
    else k_nodes<3><<<dim3(unsigned(bricks)), kEmitThreads, 0, st>>>(fields, nf, base);
    return cudaGetLastError();
}

cudaError_t launch_csr(const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st)
{
    if (total_bricks == 0) return cudaSuccess;
    k_csr<<<dim3(unsigned(total_bricks)), kEmitThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
