// Arc geometry (the paths Algorithm 2 traces): for every saddle s and every
// component of its upper link, the vertices s, rep, gradient(rep), ..., up to
// the maximum reached, where rep is the component's highest vertex
// (UpperLinkRep, Sec. 3.4).  Gathered while lab[] still holds the gradient
// pointers, i.e. between classification and resolution.
//
// Output (CSR): path_ptr[P + 1] offsets into path_vtx; paths ordered by saddle
// (index order, the order of the saddle list) and, within a saddle, by
// ascending representative (ascending neighbour slot: slot order is index
// order).  The path index of a saddle's first component is its offset in the
// saddle-path numbering of scan A (Sigma beta0+ over earlier saddles).
//
// Three launches: k_path_len stores every path's length at path_ptr[p] and
// every brick's total in pbrick[]; k_path_scan turns pbrick into offsets (one
// CTA per field) and stores the total in pbrick[nbricks] and path_ptr[P];
// k_path_write replaces the lengths by offsets and writes the vertices.
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kPathThreads = 256;
constexpr int kScanPathThreads = 1024;

// Gradient steps from r to its maximum (bounded: a path has fewer than N steps).
__device__ __forceinline__ uint32_t gradient_steps(const uint32_t *lab, uint32_t r, uint32_t N, uint32_t *err)
{
    uint32_t n = 0;
    for (uint32_t u = r;;) {
        const uint32_t w = lab[u];
        if (w == u) break;
        u = w;
        if (++n > N) {
            atomicOr(err, kErrNotConverged);
            break;
        }
    }
    return n;
}

// Exclusive warp scan of a 64-bit value; *total receives the warp sum.
__device__ __forceinline__ uint64_t path_warp_scan(uint64_t x, uint64_t *total)
{
    const int lane = threadIdx.x & 31;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    *total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - x;
}

// One warp per brick: path lengths (2 + gradient steps) at path_ptr[p], the
// brick's total in pbrick[b].
template <int KD>
__global__ void __launch_bounds__(kPathThreads)
k_path_len(const FieldDev *__restrict__ fields, int nf, uint64_t base, uint64_t bricks)
{
    const int lane = threadIdx.x & 31;
    const uint64_t t = uint64_t(blockIdx.x) * (kPathThreads / 32) + (threadIdx.x >> 5);
    if (t >= bricks) return;
    const uint64_t g = base + t;
    const FieldDev &F = fields[find_field<false>(fields, nf, g)];
    if (!F.path_ptr) return;
    const uint32_t b = uint32_t(g - F.brick0);
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    const uint4 c = F.bcnt[b];
    const uint4 o = F.boff[b];
    const uint32_t nrec = c.x + c.y;
    const uint64_t p_off = uint64_t(o.z) | (uint64_t(o.w) << 32), capP = F.totals[2];
    const uint64_t slot = uint64_t(b) * F.bcap;
    uint64_t prun = 0, sum = 0;
    for (uint32_t chunk = 0; chunk < nrec; chunk += 32) {
        const uint32_t r = chunk + uint32_t(lane);
        const uint64_t info = r < nrec ? F.rec_info[slot + r] : 0ull;
        const uint64_t b0 = uint64_t(rec_b0<KD>(info));
        uint64_t tot;
        const uint64_t lp = prun + path_warp_scan(b0, &tot);
        prun += tot;
        if (b0 == 0) continue;
        const uint32_t sid = F.rec_sid[slot + r];
        int k[CompBound<KD>::value];
        const int nc = rec_slots<KD>(info, k);
        for (int q = 0; q < nc; q++) {
            const uint64_t len = 2 + gradient_steps(F.lab, slot_vertex<KD>(sid, k[q], s), F.N, F.err);
            const uint64_t p = p_off + lp + uint64_t(q);
            if (p < capP) F.path_ptr[p] = len;
            else atomicOr(F.err, kErrInternal);
            sum += len;
        }
    }
#pragma unroll
    for (int o2 = 16; o2 >= 1; o2 >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o2);
    if (lane == 0) F.pbrick[b] = sum;
}

// One CTA per field: exclusive scan of pbrick[0, nbricks) in place; the total
// goes to pbrick[nbricks] and path_ptr[P].
__global__ void __launch_bounds__(kScanPathThreads)
k_path_scan(const FieldDev *__restrict__ fields)
{
    __shared__ uint64_t s_w[kScanPathThreads / 32];
    __shared__ uint64_t s_carry;
    const FieldDev &F = fields[blockIdx.x];
    if (!F.path_ptr) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = F.nbricks;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < n; base += kScanPathThreads) {
        const uint32_t i = base + uint32_t(tid);
        const uint64_t x = i < n ? F.pbrick[i] : 0ull;
        uint64_t wt;
        const uint64_t ex = path_warp_scan(x, &wt);
        if (lane == 0) s_w[warp] = wt;
        __syncthreads();
        uint64_t before = s_carry;
        for (int w = 0; w < warp; w++) before += s_w[w];
        if (i < n) F.pbrick[i] = before + ex;
        __syncthreads();
        if (tid == kScanPathThreads - 1) s_carry = before + ex + x;
        __syncthreads();
    }
    if (tid == 0) {
        F.pbrick[n] = s_carry;
        F.path_ptr[F.totals[2]] = s_carry;
    }
}

// One warp per brick: path offsets (brick offset + in-brick prefix) replace
// the lengths, and the vertices are written.
template <int KD>
__global__ void __launch_bounds__(kPathThreads)
k_path_write(const FieldDev *__restrict__ fields, int nf, uint64_t base, uint64_t bricks)
{
    const int lane = threadIdx.x & 31;
    const uint64_t t = uint64_t(blockIdx.x) * (kPathThreads / 32) + (threadIdx.x >> 5);
    if (t >= bricks) return;
    const uint64_t g = base + t;
    const FieldDev &F = fields[find_field<false>(fields, nf, g)];
    if (!F.path_ptr || !F.path_vtx) return;
    const uint32_t b = uint32_t(g - F.brick0);
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    const uint4 c = F.bcnt[b];
    const uint4 o = F.boff[b];
    const uint32_t nrec = c.x + c.y;
    const uint64_t p_off = uint64_t(o.z) | (uint64_t(o.w) << 32), capP = F.totals[2];
    const uint64_t capV = F.pbrick[F.nbricks];
    const uint64_t slot = uint64_t(b) * F.bcap;
    uint64_t prun = 0, vrun = F.pbrick[b];
    for (uint32_t chunk = 0; chunk < nrec; chunk += 32) {
        const uint32_t r = chunk + uint32_t(lane);
        const uint64_t info = r < nrec ? F.rec_info[slot + r] : 0ull;
        const uint64_t b0 = uint64_t(rec_b0<KD>(info));
        // this saddle's paths and their total length (lengths from k_path_len)
        uint64_t L = 0;
        const bool mine = b0 != 0 && p_off + prun < capP;
        uint64_t tot;
        const uint64_t lp = prun + path_warp_scan(b0, &tot);
        prun += tot;
        if (mine)
            for (uint64_t q = 0; q < b0; q++)
                if (p_off + lp + q < capP) L += F.path_ptr[p_off + lp + q];
        const uint64_t lv = vrun + path_warp_scan(L, &tot);
        vrun += tot;
        if (b0 == 0) continue;
        const uint32_t sid = F.rec_sid[slot + r];
        int k[CompBound<KD>::value];
        const int nc = rec_slots<KD>(info, k);
        uint64_t at = lv;
        for (int q = 0; q < nc; q++) {
            const uint64_t p = p_off + lp + uint64_t(q);
            if (p >= capP) {
                atomicOr(F.err, kErrInternal);
                break;
            }
            const uint64_t len = F.path_ptr[p];
            F.path_ptr[p] = at;
            if (at + len > capV || len < 2) {
                atomicOr(F.err, kErrInternal);
                break;
            }
            uint32_t u = slot_vertex<KD>(sid, k[q], s);
            F.path_vtx[at] = sid;
            F.path_vtx[at + 1] = u;
            for (uint64_t j = 2; j < len; j++) {
                u = F.lab[u];
                F.path_vtx[at + j] = u;
            }
            at += len;
        }
    }
}

cudaError_t launch_path_len(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks, cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>((bricks + kPathThreads / 32 - 1) / (kPathThreads / 32)));
    if (kd == 5) k_path_len<5><<<grid, kPathThreads, 0, st>>>(fields, nf, base, bricks);
    else if (kd == 4) k_path_len<4><<<grid, kPathThreads, 0, st>>>(fields, nf, base, bricks);
    else k_path_len<3><<<grid, kPathThreads, 0, st>>>(fields, nf, base, bricks);
    return cudaGetLastError();
}

cudaError_t launch_path_scan(const FieldDev *fields, int nf, cudaStream_t st)
{
    if (nf == 0) return cudaSuccess;
    k_path_scan<<<dim3(static_cast<unsigned>(nf)), kScanPathThreads, 0, st>>>(fields);
    return cudaGetLastError();
}

cudaError_t launch_path_write(int kd, const FieldDev *fields, int nf, uint64_t base, uint64_t bricks,
                              cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>((bricks + kPathThreads / 32 - 1) / (kPathThreads / 32)));
    if (kd == 5) k_path_write<5><<<grid, kPathThreads, 0, st>>>(fields, nf, base, bricks);
    else if (kd == 4) k_path_write<4><<<grid, kPathThreads, 0, st>>>(fields, nf, base, bricks);
    else k_path_write<3><<<grid, kPathThreads, 0, st>>>(fields, nf, base, bricks);
    return cudaGetLastError();
}

}  // namespace eg
