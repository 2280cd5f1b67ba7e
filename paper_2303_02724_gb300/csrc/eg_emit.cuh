// Arc and graph assembly bodies (steps d + e), one warp per brick: shared by
// the emit kernels (eg_emit.cu) and the fused small-field kernel
// (eg_small.cu).
#pragma once

#include "eg_internal.cuh"

namespace eg {

// Sorted unique arc ends of one saddle; returns their count.
template <int KD>
__device__ __forceinline__ int saddle_ends(const uint32_t *lab, const uint32_t (&s)[kMaxDim], uint32_t sid,
                                           uint64_t info, uint32_t (&t)[CompBound<KD>::value], uint32_t N,
                                           uint32_t *err)
{
    // the representatives in record order (the ends are sorted below)
    constexpr int kCap = CompBound<KD>::value;
    const int b0 = rec_b0<KD>(info);
    uint64_t rest = info;
    int n = 0;
    for (int c = 0; c < b0 && c < kCap; c++) {
        int k;
        if constexpr (KD == 5) {
            k = __ffsll((long long)rest) - 1;
            rest &= rest - 1;
        } else {
            k = int((info >> (5 * c)) & 31u);
        }
        const uint32_t rv = slot_vertex<KD>(sid, k, s);
        const uint32_t m = chk(rv, N, err) ? lab[rv] : 0u;
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

// Value copy of a vertex of a non-float32 field: the element's bits.
__device__ __forceinline__ void copy_value(const FieldDev &F, uint32_t v, void *dst, uint64_t q)
{
    switch (dtype_size(F.dtype)) {
    case 1: static_cast<uint8_t *>(dst)[q] = static_cast<const uint8_t *>(F.fraw)[v]; break;
    case 2: static_cast<uint16_t *>(dst)[q] = static_cast<const uint16_t *>(F.fraw)[v]; break;
    case 4: static_cast<uint32_t *>(dst)[q] = static_cast<const uint32_t *>(F.fraw)[v]; break;
    default:
        static_cast<unsigned long long *>(dst)[q] = static_cast<const unsigned long long *>(F.fraw)[v];
        break;
    }
}

// Inclusive warp scan of a packed 64-bit counter; returns the exclusive value,
// *total receives the warp sum.
__device__ __forceinline__ uint64_t warp_excl_scan_u64(uint64_t x, uint64_t *total)
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

// One warp (all 32 lanes) assembles brick b: the brick's maxima and saddles
// go to their final positions, each saddle's sorted unique arc ends are parked
// at its path offset, and the brick's unique-arc count is stored.
template <int KD>
__device__ __forceinline__ void nodes_brick(const FieldDev &F, uint32_t b)
{
    const int lane = threadIdx.x & 31;
    uint32_t s[kMaxDim];
#pragma unroll
    for (int i = 0; i < kMaxDim; i++) s[i] = F.s[i];
    if (!chk(b, F.nbricks, F.err)) return;
    const uint4 c = F.bcnt[b];
    const uint4 o = F.boff[b];
    const uint32_t nrec = c.x + c.y;
    const uint64_t m_off = o.x, s_off = o.y, p_off = uint64_t(o.z) | (uint64_t(o.w) << 32);
    const uint64_t capM = F.totals[0], capS = F.totals[1], capP = F.totals[2];
    const uint64_t slot = uint64_t(b) * F.bcap;
    uint64_t run = 0;  // maxima | saddles << 16 | paths << 32 of earlier rounds
    uint32_t asum = 0;
    uint32_t tmp[CompBound<KD>::value];
    for (uint32_t chunk = 0; chunk < nrec; chunk += 32) {
        const uint32_t r = chunk + uint32_t(lane);
        uint32_t sid = 0;
        uint64_t info = ~0ull;
        float val = 0.f;
        uint64_t mine = 0;
        const bool have = r < nrec && chk(slot + r, rec_cap(F), F.err) && chk(r, F.bcap, F.err);
        if (have) {
            sid = F.rec_sid[slot + r];
            info = F.rec_info[slot + r];
            val = F.rec_val[slot + r];
            const uint64_t b0 = uint64_t(rec_b0<KD>(info));
            mine = b0 == 0 ? 1ull : ((1ull << 16) | (b0 << 32));
        }
        uint64_t tot;
        const uint64_t pos = run + warp_excl_scan_u64(mine, &tot);
        run += tot;
        if (!have) continue;
        const uint64_t b0 = uint64_t(rec_b0<KD>(info));
        const uint64_t lm = pos & 0xffffu, ls = (pos >> 16) & 0xffffu, lp = pos >> 32;
        if (b0 == 0) {
            const uint64_t q = m_off + lm;
            if (q < capM) {
                F.maxima[q] = sid;
                if (F.max_val) F.max_val[q] = val;
                else copy_value(F, sid, F.max_raw, q);  // other element types: from the field
            } else {
                atomicOr(F.err, kErrInternal);
            }
        } else {
            const uint64_t q = s_off + ls, p = p_off + lp;
            const int u = saddle_ends<KD>(F.lab, s, sid, info, tmp, F.N, F.err);
            if (q < capS && p + b0 <= capP) {
                F.saddles[q] = sid;
                F.sad_b0[q] = uint8_t(b0);
                if (F.sad_val) F.sad_val[q] = val;
                else copy_value(F, sid, F.sad_raw, q);
                F.ucnt[q] = uint8_t(u);
                for (int e = 0; e < u; e++) F.ends[p + e] = tmp[e];
            } else {
                atomicOr(F.err, kErrInternal);
            }
            asum += uint32_t(u);
        }
    }
    asum = __reduce_add_sync(0xffffffffu, asum);
    if (lane == 0) F.acnt[b] = asum;
}

// One warp (all 32 lanes): row_ptr of brick b's saddles from the unique
// counts (scan B offsets plus an in-brick scan) and col, copied from the
// parked ends.
__device__ __forceinline__ void csr_brick(const FieldDev &F, uint32_t b)
{
    const int lane = threadIdx.x & 31;
    if (!chk(b, F.nbricks, F.err)) return;
    const uint4 c = F.bcnt[b];
    const uint4 o = F.boff[b];
    const uint32_t ns = c.y;
    const uint64_t s_off = o.y, p_off = uint64_t(o.z) | (uint64_t(o.w) << 32);
    const uint64_t a_off = F.aoff[b];
    const uint64_t capS = F.totals[1], capP = F.totals[2], capA = F.totals[3];
    uint64_t run = 0;  // unique arcs | paths << 32 of earlier rounds
    for (uint32_t chunk = 0; chunk < ns; chunk += 32) {
        const uint32_t r = chunk + uint32_t(lane);
        uint32_t u = 0, b0 = 0;
        const bool ok = r < ns && s_off + r < capS;
        if (ok) {
            u = F.ucnt[s_off + r];
            b0 = F.sad_b0[s_off + r];
        }
        uint64_t tot;
        const uint64_t pos = run + warp_excl_scan_u64(uint64_t(u) | (uint64_t(b0) << 32), &tot);
        run += tot;
        if (!ok) continue;
        const uint64_t a = a_off + (pos & 0xffffffffu), p = p_off + (pos >> 32);
        F.row_ptr[s_off + r] = a;
        if (a + u <= capA && p + u <= capP) {
            for (uint32_t e = 0; e < u; e++) F.col[a + e] = F.ends[p + e];
        } else {
            atomicOr(F.err, kErrInternal);
        }
    }
    if (lane == 0 && b == F.nbricks - 1) {
        if (s_off + ns == capS && a_off + F.acnt[b] == capA) F.row_ptr[capS] = capA;
        else atomicOr(F.err, kErrInternal);
    }
}

}  // namespace eg
