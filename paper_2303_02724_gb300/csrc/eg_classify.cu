// Steps (a) + (c): per-vertex classification (Sec. 3.3, Table 1).
//
// For every vertex v: the gradient pointer asc(v) = highest vertex of the
// upper link (Sec. 3.3), or v at a maximum; beta0+(v), the number of
// connected components of the upper link, found with a bitmask flood fill
// over the link edges of the upper neighbours (the union-find of Sec. 3.3
// restated on a <= 30-bit register mask); and for a saddle the highest vertex
// of each component (UpperLinkRep, Sec. 3.4), recorded as its neighbour slot.
//
// Work unit: a brick of kBrick consecutive vertex ids.  Every maximum and
// saddle of a brick is written, in index order, into that brick's record slot,
// so a later scan over per-brick counts gives global positions directly.
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kClassifyThreads = 256;
constexpr int kVpt = kBrick / kClassifyThreads;

template <int D>
__device__ __forceinline__ uint32_t link_flood(uint32_t seed, uint32_t upper, const uint32_t *s_adj)
{
    uint32_t comp = seed, frontier = seed;
    while (frontier) {
        int k = __ffs(frontier) - 1;
        frontier &= frontier - 1;
        uint32_t nb = s_adj[k] & upper & ~comp;
        comp |= nb;
        frontier |= nb;
    }
    return comp;
}

// Classify vertex v of field F.  Returns asc(v); sets b0 and the packed rep
// slots (5 bits per component, component order arbitrary).
template <int D>
__device__ __forceinline__ uint32_t classify_vertex(const FieldDev &F, const uint32_t (&s)[kMaxDim],
                                                    uint32_t v, const uint32_t *s_adj, bool minimum,
                                                    int &b0, uint64_t &codes, bool &nan)
{
    using NB = Nbr<D>;
    constexpr int K = NB::K;
    // coordinates -> in-bounds masks per axis
    uint32_t pok = 0, mok = 0, rem = v;
#pragma unroll
    for (int i = 0; i < D; i++) {
        uint32_t c;
        if (i < D - 1) {
            c = rem % F.n[i];
            rem /= F.n[i];
        } else {
            c = rem;
        }
        if (c + 1 < F.n[i]) pok |= 1u << i;
        if (c > 0) mok |= 1u << i;
    }
    const uint32_t flip = minimum ? 0xffffffffu : 0u;
    float fv = __ldg(F.f + v);
    nan = fv != fv;
    const uint64_t cc = (uint64_t(order_key(fv) ^ flip) << 8) | uint64_t(NB::H);
    uint64_t cmp[K];
    uint32_t upper = 0, asc = v;
    uint64_t best = 0;
    int bestk = -1;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const uint32_t p = NB::pat(k);
        const bool inb = NB::neg(k) ? ((p & ~mok) == 0) : ((p & ~pok) == 0);
        uint64_t ck = 0;
        uint32_t w = 0;
        if (inb) {
            uint32_t o = 0;
#pragma unroll
            for (int i = 0; i < D; i++)
                if (p & (1u << i)) o += s[i];
            w = NB::neg(k) ? v - o : v + o;
            const uint32_t r = minimum ? uint32_t(2 * NB::H) - NB::rank(k) : NB::rank(k);
            ck = (uint64_t(order_key(__ldg(F.f + w)) ^ flip) << 8) | r;
        }
        cmp[k] = ck;
        if (ck > cc) {
            upper |= 1u << k;
            if (ck > best) {
                best = ck;
                bestk = k;
                asc = w;
            }
        }
    }
    codes = 0;
    if (upper == 0) {
        b0 = 0;
        return v;
    }
    uint32_t comp = link_flood<D>(1u << bestk, upper, s_adj);
    b0 = 1;
    if (comp == upper) return asc;
    codes = uint64_t(bestk);
    uint32_t left = upper & ~comp;
    while (left) {
        uint32_t c2 = link_flood<D>(left & (~left + 1u), upper, s_adj);
        left &= ~c2;
        uint64_t rb = 0;
        int rk = 0;
#pragma unroll
        for (int k = 0; k < K; k++)
            if (((c2 >> k) & 1u) && cmp[k] > rb) {
                rb = cmp[k];
                rk = k;
            }
        codes |= uint64_t(rk) << (5 * b0);
        b0++;
    }
    return asc;
}

template <int D>
__global__ void __launch_bounds__(kClassifyThreads)
k_classify(const FieldDev *__restrict__ fields, int nf)
{
    using NB = Nbr<D>;
    __shared__ uint32_t s_adj[NB::K];
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned s_cnt[3];
    const int tid = threadIdx.x;
    if (tid < NB::K) s_adj[tid] = NB::adj_mask(tid);
    if (tid < 3) s_cnt[tid] = 0;
    const uint64_t g = blockIdx.x;
    const int fi = find_field(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint32_t b = uint32_t(g - F.brick0);
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    const bool minimum = (F.flags & kFlagMinimum) != 0;
    const uint64_t v0 = uint64_t(b) * kBrick;
    uint32_t *rsid = F.rec_sid + v0;
    uint64_t *rinfo = F.rec_info + v0;
    __syncthreads();

    uint32_t running = 0, nm = 0, ns = 0, np = 0;
    bool anynan = false;
#pragma unroll 1
    for (int i = 0; i < kVpt; i++) {
        const uint64_t v64 = v0 + uint64_t(i) * kClassifyThreads + tid;
        const bool valid = v64 < F.N;
        int b0 = 1;
        uint64_t codes = 0;
        if (valid) {
            bool nan;
            const uint32_t v = uint32_t(v64);
            uint32_t asc = classify_vertex<D>(F, s, v, s_adj, minimum, b0, codes, nan);
            anynan |= nan;
            F.lab[v] = asc;
        }
        const bool crit = valid && b0 != 1;
        uint32_t tot;
        const uint32_t pos = block_excl_scan(crit ? 1u : 0u, s_scan, &tot);
        if (crit) {
            rsid[running + pos] = uint32_t(v64);
            rinfo[running + pos] = (uint64_t(b0) << 56) | codes;
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
    if (tid == 0) {
        F.bcnt[b] = make_uint4(s_cnt[0], s_cnt[1], s_cnt[2], 0u);
        if (s_cnt[0]) atomicAdd(&F.totals[0], (unsigned long long)s_cnt[0]);
        if (s_cnt[1]) atomicAdd(&F.totals[1], (unsigned long long)s_cnt[1]);
        if (s_cnt[2]) atomicAdd(&F.totals[2], (unsigned long long)s_cnt[2]);
    }
}

template <int D>
cudaError_t launch_classify(const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st)
{
    if (total_bricks == 0) return cudaSuccess;
    k_classify<D><<<dim3(unsigned(total_bricks)), kClassifyThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

cudaError_t launch_classify_d(int d, const FieldDev *fields, int nf, uint64_t total_bricks, cudaStream_t st)
{
    switch (d) {
    case 1: return launch_classify<1>(fields, nf, total_bricks, st);
    case 2: return launch_classify<2>(fields, nf, total_bricks, st);
    case 3: return launch_classify<3>(fields, nf, total_bricks, st);
    case 4: return launch_classify<4>(fields, nf, total_bricks, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace eg
