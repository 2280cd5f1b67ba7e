// Steps (d) + (e): arcs and graph assembly.
//
// For every saddle s and every upper-link component C recorded by the
// classification, the arc end is label(rep(C)) (Sec. 3.4, Algorithm 2:
// following the gradient from UpperLinkRep reaches that maximum; Sec. 2: arc
// (s, m) iff s bounds the descending manifold of m).  Each saddle's ends are
// sorted and de-duplicated in registers.
//
// Bricks are taken in ticket order by a persistent grid; one decoupled
// look-back per brick yields, for maxima, saddles and unique arcs at once,
// the number produced by all earlier bricks of the same field, so every
// output lands at its final, index-sorted position in a single pass:
//   maxima[M], max_val[M], saddles[S], sad_b0[S], sad_val[S],
//   row_ptr[S+1] (uint64), col[A].
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kEmitThreads = 256;
constexpr int kRpt = kBrick / kEmitThreads;  // records per thread

// Sorted unique arc ends of one saddle; returns their count.
template <int D>
__device__ __forceinline__ int saddle_ends(const FieldDev &F, const uint32_t (&s)[kMaxDim], uint32_t sid,
                                           uint64_t info, uint32_t (&t)[10])
{
    const int b0 = int((info >> 56) & 0xfu);
    int n = 0;
    for (int c = 0; c < b0 && c < 10; c++) {
        const int k = int((info >> (5 * c)) & 31u);
        const uint32_t rep = slot_vertex<D>(sid, k, s);
        uint32_t m = F.lab[rep];
        // insertion into the sorted prefix, dropping duplicates
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

template <int D>
__global__ void __launch_bounds__(kEmitThreads)
k_emit(const FieldDev *__restrict__ fields, int nf, uint64_t total, unsigned long long *ticket,
       uint64_t *lb)
{
    __shared__ unsigned long long s_t;
    __shared__ uint32_t s_scan[33];
    __shared__ uint64_t s_pref[3];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    while (true) {
        if (tid == 0) s_t = atomicAdd(ticket, 1ull);
        __syncthreads();
        const uint64_t t = s_t;
        __syncthreads();
        if (t >= total) break;
        const int fi = find_field(fields, nf, t);
        const FieldDev &F = fields[fi];
        const uint32_t b = uint32_t(t - F.brick0);
        uint32_t s[kMaxDim];
#pragma unroll
        for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
        const uint4 c = F.bcnt[b];
        const uint32_t nrec = c.x + c.y;
        const uint64_t slot = uint64_t(b) * kBrick;
        uint32_t sid[kRpt];
        uint64_t info[kRpt];
        uint32_t lm = 0, ls = 0, la = 0;
        uint32_t tmp[10];
#pragma unroll
        for (int j = 0; j < kRpt; j++) {
            const uint32_t r = uint32_t(tid) * kRpt + j;
            info[j] = ~0ull;
            sid[j] = 0;
            if (r < nrec) {
                sid[j] = F.rec_sid[slot + r];
                info[j] = F.rec_info[slot + r];
                if ((info[j] >> 56) == 0) lm++;
                else {
                    ls++;
                    la += uint32_t(saddle_ends<D>(F, s, sid[j], info[j], tmp));
                }
            }
        }
        uint32_t tm, ts, ta;
        uint32_t em = block_excl_scan(lm, s_scan, &tm);
        uint32_t es = block_excl_scan(ls, s_scan, &ts);
        uint32_t ea = block_excl_scan(la, s_scan, &ta);
        if (warp < 3) {
            const uint32_t agg = warp == 0 ? tm : (warp == 1 ? ts : ta);
            uint64_t p = warp_lookback(lb + uint64_t(warp) * total, t, F.brick0, agg, F.err);
            if (lane == 0) s_pref[warp] = p;
        }
        __syncthreads();
        uint64_t mo = s_pref[0] + em, so = s_pref[1] + es, ao = s_pref[2] + ea;
        // capacities from the classification counts; a failed look-back must
        // never turn into an out-of-range store
        const uint64_t capM = F.totals[0], capS = F.totals[1], capP = F.totals[2];
#pragma unroll
        for (int j = 0; j < kRpt; j++) {
            if (info[j] == ~0ull) continue;
            const uint32_t v = sid[j];
            if ((info[j] >> 56) == 0) {
                if (mo >= capM) {
                    atomicOr(F.err, kErrInternal);
                    continue;
                }
                F.maxima[mo] = v;
                F.max_val[mo] = F.f[v];
                mo++;
            } else {
                const int n = saddle_ends<D>(F, s, v, info[j], tmp);
                if (so >= capS || ao + n > capP) {
                    atomicOr(F.err, kErrInternal);
                    continue;
                }
                F.saddles[so] = v;
                F.sad_b0[so] = uint8_t(info[j] >> 56);
                F.sad_val[so] = F.f[v];
                F.row_ptr[so] = ao;
                for (int q = 0; q < n; q++) F.col[ao + q] = tmp[q];
                ao += n;
                so++;
            }
        }
        if (b == F.nbricks - 1 && tid == 0) {
            const uint64_t S = s_pref[1] + ts, A = s_pref[2] + ta;
            if (S == capS && A <= capP) {
                F.row_ptr[S] = A;
                F.totals[3] = A;
            } else {
                atomicOr(F.err, kErrInternal);
            }
        }
        __syncthreads();
    }
}

size_t emit_workspace_bytes(uint64_t total_bricks) { return 256 + 3 * total_bricks * sizeof(uint64_t); }

template <int D>
static cudaError_t launch_emit(const FieldDev *fields, int nf, uint64_t total, void *ws, int sm_count,
                               cudaStream_t st)
{
    if (total == 0) return cudaSuccess;
    auto *ticket = reinterpret_cast<unsigned long long *>(ws);
    auto *lb = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(ws) + 256);
    uint64_t grid = uint64_t(sm_count) * 4;
    if (grid > total) grid = total;
    k_emit<D><<<dim3(unsigned(grid)), kEmitThreads, 0, st>>>(fields, nf, total, ticket, lb);
    return cudaGetLastError();
}

cudaError_t launch_emit_d(int d, const FieldDev *fields, int nf, uint64_t total, void *ws, int sm_count,
                          cudaStream_t st)
{
    switch (d) {
    case 1: return launch_emit<1>(fields, nf, total, ws, sm_count, st);
    case 2: return launch_emit<2>(fields, nf, total, ws, sm_count, st);
    case 3: return launch_emit<3>(fields, nf, total, ws, sm_count, st);
    case 4: return launch_emit<4>(fields, nf, total, ws, sm_count, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace eg
