// Steps (a) + (c) for 5D float32 fields (and the float32 image of 8/16-bit
// integer fields) whose rows hold at most kR5MaxRow vertices: row classifier
// (Sec. 3.3, Table 1; UpperLinkRep of Sec. 3.4).
//
// A brick is `ty` whole rows (axis 0) of one (z, w, u) plane, classified by
// one CTA in up to kR5Passes passes of one vertex per thread (bricks of about
// 1024 vertices, the size the resolver and the assembly work best on).  The
// neighbour with axis pattern p (bit 0: axis 0, bits 1..4: axes 1..4) and sign
// lies in row q = p >> 1 (offset along the axes of q) at column x - (p & 1)
// (negative) or x + (p & 1) (positive),
// so 31 rows are read: the centre row and 15 on each side, one coalesced value
// per thread per row and the column x - 1 or x + 1 from the same cache lines.  Rows are consumed as they arrive, in slot order: the upper bits
// (set-compares accumulated with FMAs into floats whose exponent pins the
// integer part) and the running extreme with its slot, so only the centre
// value and a few accumulators stay live.  Out-of-domain rows and columns read
// NaN, which fails every ordered comparison.
//
// Per vertex, as in the general classifier (the same slot order, tie rules and
// record format):
//   upper   a negative slot needs a strictly higher value, a positive one a
//           higher or equal value (simulated perturbation: positive slots have
//           larger indices); mirrored for the minimum graph;
//   asc     the highest upper neighbour, ties to the later slot (the minimum
//           graph: the lowest, ties to the earlier slot);
//   beta0+  the component of the gradient slot inside the upper link
//           (PatternLink<5> closure); a saddle when it is not the whole link,
//           and then every other component and its highest slot, from values
//           reloaded through the cache (saddles are rare).
#include <type_traits>

#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kR5Threads = kR5CtaThreads;

namespace {

__device__ __forceinline__ float r5_set(int op, float a, float b)
{
    float d;
    switch (op) {
    case 0: asm("set.gt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    case 1: asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    case 2: asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    default: asm("set.le.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    }
    return d;
}

// offset of the row with axis pattern q (bits over axes 1..4)
__device__ __forceinline__ uint32_t r5_row_off(int q, uint32_t s1, uint32_t s2, uint32_t s3, uint32_t s4)
{
    return ((q & 1) ? s1 : 0u) + ((q & 2) ? s2 : 0u) + ((q & 4) ? s3 : 0u) + ((q & 8) ? s4 : 0u);
}

}  // namespace

template <bool MIN>
__global__ void __launch_bounds__(kR5Threads) k_classify_r5(const FieldDev *__restrict__ fields, int nf)
{
    using PL = PatternLink<5>;
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned s_cnt[3];
    const uint64_t g = fields[0].brick0 + blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint32_t b = uint32_t(g - F.brick0);
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 3) s_cnt[tid] = 0;

    const uint32_t n0 = F.n[0], n1 = F.n[1], n2 = F.n[2], n3 = F.n[3], n4 = F.n[4];
    const uint32_t s1 = F.s[1], s2 = F.s[2], s3 = F.s[3], s4 = F.s[4];
    const uint32_t p = b / F.nyb, yb = b - p * F.nyb;
    const uint32_t z = p % n2, w = (p / n2) % n3, u = p / (n2 * n3);
    const uint32_t y0 = yb * F.ty;
    const uint32_t brows = min(F.ty, n1 - y0);
    const uint32_t rpp = uint32_t(kR5Threads) / n0;  // rows per pass
    const uint32_t rr0 = uint32_t(tid) / n0, x = uint32_t(tid) - rr0 * n0;
    const bool left_ok = x > 0, right_ok = x + 1 < n0;
    const float qnan = __int_as_float(0x7fc00000);
    uint32_t running = 0;
    bool anynan = false;
    uint32_t nm = 0, ns = 0, np = 0;
    for (uint32_t pass = 0; pass * rpp < brows; pass++) {
        const uint32_t r = pass * rpp + rr0;
        const uint32_t y = y0 + r;
        const bool rowok = rr0 < rpp && r < brows;
        const uint32_t v = (((u * n3 + w) * n2 + z) * n1 + y) * n0 + x;  // (meaningful when rowok)
        // axes 1..4 along which the vertex may step down (lo) or up (hi)
        const uint32_t lo = (y > 0 ? 1u : 0u) | (z > 0 ? 2u : 0u) | (w > 0 ? 4u : 0u) | (u > 0 ? 8u : 0u);
        const uint32_t hi =
            (y + 1 < n1 ? 1u : 0u) | (z + 1 < n2 ? 2u : 0u) | (w + 1 < n3 ? 4u : 0u) | (u + 1 < n4 ? 8u : 0u);
        const float c = (rowok && chk(v, F.N, F.err)) ? __ldg(F.f + v) : qnan;

        // row q's value at column x, and at column x - 1 (negative rows) or
        // x + 1 (positive rows)
        auto row = [&](auto inner, int q, bool neg, float &vx, float &vside) {
            const bool ok = decltype(inner)::value ? true
                                                   : rowok && (neg ? (lo & uint32_t(q)) == uint32_t(q)
                                                                   : (hi & uint32_t(q)) == uint32_t(q));
            const uint32_t o = r5_row_off(q, s1, s2, s3, s4);
            const uint32_t rb = neg ? v - o : v + o;
            vx = (ok && chk(rb, F.N, F.err)) ? __ldg(F.f + rb) : qnan;
            // (a second load from the same cache lines costs fewer instructions
            // than a shuffle with its lane-edge fix-up)
            if (neg) vside = (ok && left_ok && chk(rb - 1, F.N, F.err)) ? __ldg(F.f + rb - 1) : qnan;
            else vside = (ok && right_ok && chk(rb + 1, F.N, F.err)) ? __ldg(F.f + rb + 1) : qnan;
        };

        // upper bits in the pattern layout: positive pattern p at bit p, negative
        // at bit 32 + p; four accumulators of at most 16 bits each
        float aP0 = 8388608.f, aP1 = 8388608.f, aN0 = 8388608.f, aN1 = 8388608.f;
        // running extreme over all 62 values (NaN ignored) and the slot of its
        // last (minimum graph: first) occurrence; that slot is upper whenever
        // the link has an upper neighbour: an extreme strictly beyond c is
        // upper in either half, and an extreme equal to c is upper exactly in
        // the half the tie rule prefers (positive slots come later), so the
        // upper test need not gate the update
        float best = MIN ? __int_as_float(0x7f800000) : __int_as_float(0xff800000);
        int bestk = -1;
        auto consider = [&](int k, float nb) {  // slot k (Nbr<5> order), value nb
            const bool neg = k < 31;
            const int pt = neg ? 31 - k : k - 30;
            const float up = r5_set(neg ? (MIN ? 3 : 0) : (MIN ? 2 : 1), nb, c);
            if (neg) {
                if (pt < 16) aN0 = __fmaf_rn(up, float(1u << pt), aN0);
                else aN1 = __fmaf_rn(up, float(1u << (pt - 16)), aN1);
            } else {
                if (pt < 16) aP0 = __fmaf_rn(up, float(1u << pt), aP0);
                else aP1 = __fmaf_rn(up, float(1u << (pt - 16)), aP1);
            }
            // slots arrive in increasing order: ties go to the later slot (>=),
            // in the minimum graph to the earlier one (<)
            const bool t = MIN ? nb < best : nb >= best;
            best = MIN ? fminf(best, nb) : fmaxf(best, nb);
            bestk = t ? k : bestk;
        };
        auto scan = [&](auto inner) {
            // negative rows q = 15 .. 1: slots 30 - 2q (pattern 2q + 1, column x - 1)
            // and 31 - 2q (pattern 2q, column x)
#pragma unroll
            for (int q = 15; q >= 1; q--) {
                float vx, vl;
                row(inner, q, true, vx, vl);
                consider(30 - 2 * q, vl);
                consider(31 - 2 * q, vx);
            }
            // centre row: slot 30 (pattern 1, column x - 1) and 31 (column x + 1)
            consider(30, (rowok && left_ok && chk(v - 1, F.N, F.err)) ? __ldg(F.f + v - 1) : qnan);
            consider(31, (rowok && right_ok && chk(v + 1, F.N, F.err)) ? __ldg(F.f + v + 1) : qnan);
            // positive rows q = 1 .. 15: slots 30 + 2q (pattern 2q, column x) and
            // 31 + 2q (pattern 2q + 1, column x + 1)
#pragma unroll
            for (int q = 1; q <= 15; q++) {
                float vx, vr;
                row(inner, q, false, vx, vr);
                consider(30 + 2 * q, vx);
                consider(31 + 2 * q, vr);
            }
        };
        // a vertex with room along axes 1..4 on both sides (most of them; the
        // whole warp agrees, as it lies in one row) takes a copy of the scan
        // without the rows' domain tests
        if (rowok && lo == 15u && hi == 15u) scan(std::true_type{});
        else scan(std::false_type{});
        const uint32_t up_pos = (__float_as_uint(aP0) & 0xffffu) | ((__float_as_uint(aP1) & 0xffffu) << 16);
        const uint32_t up_neg = (__float_as_uint(aN0) & 0xffffu) | ((__float_as_uint(aN1) & 0xffffu) << 16);
        const uint64_t U = uint64_t(up_pos) | (uint64_t(up_neg) << 32);

        uint32_t asc = v;
        uint64_t info = 0;
        bool crit = false;
        if (rowok && U != 0 && bestk >= 0) {
            const bool gneg = bestk < 31;
            const int gp = gneg ? 31 - bestk : bestk - 30;
            const uint32_t o = ((gp & 1) ? 1u : 0u) + r5_row_off(gp >> 1, s1, s2, s3, s4);
            asc = gneg ? v - o : v + o;
            // the gradient's component; seeded with its whole half when that half
            // holds its full pattern (comparable to every pattern of the half)
            const uint64_t half = gneg ? 0xffffffff00000000ull : 0x00000000ffffffffull;
            const uint64_t full = gneg ? (1ull << 63) : (1ull << 31);
            const uint64_t seed = (U & full) ? (U & half) : (1ull << PL::bit(bestk));
            const uint64_t comp = PL::component(seed, U);
            if (comp != U) {
                // a saddle: every other component's highest slot, from reloaded values
                uint64_t codes = 1ull << bestk;
                for (uint64_t lft = U & ~comp; lft;) {
                    const uint64_t c2 = PL::component(lft & (~lft + 1ull), U);
                    lft &= ~c2;
                    float rb = 0.f;
                    int rk = -1;
                    for (uint64_t m = c2; m;) {
                        const int bit = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        // pattern-layout bit -> slot: positive pattern p is slot 30 + p,
                        // negative pattern p is slot 31 - p
                        const int k = bit < 32 ? 30 + bit : 31 - (bit - 32);
                        const int pk = bit < 32 ? bit : bit - 32;
                        const uint32_t ok2 = ((pk & 1) ? 1u : 0u) + r5_row_off(pk >> 1, s1, s2, s3, s4);
                        const uint32_t wv = bit < 32 ? v + ok2 : v - ok2;
                        const float nb = chk(wv, F.N, F.err) ? __ldg(F.f + wv) : qnan;
                        // slots in decreasing order along the negative half: compare
                        // with the slot index for the tie rule
                        const bool better = rk < 0 || (MIN ? (nb < rb || (nb == rb && k < rk))
                                                           : (nb > rb || (nb == rb && k > rk)));
                        if (better) {
                            rb = nb;
                            rk = k;
                        }
                    }
                    codes |= 1ull << rk;
                }
                info = codes;
                crit = true;
                ns++;
                np += uint32_t(__popcll(codes));
            }
        } else if (rowok && U == 0) {
            crit = true;  // a maximum (or a NaN, flagged below)
            nm++;
        }
        if (rowok && chk(v, F.N, F.err)) F.lab[v] = asc;
        anynan |= rowok && c != c;

        // this pass's records after the earlier passes': threads are in (row, x)
        // order, so the brick's records stay in index order
        uint32_t tot;
        const uint32_t pos = running + block_excl_scan(crit ? 1u : 0u, s_scan, &tot);
        running += tot;
        const uint64_t qd = uint64_t(b) * F.bcap + pos;
        if (crit && chk(qd, rec_cap(F), F.err) && chk(pos, F.bcap, F.err)) {
            F.rec_sid[qd] = v;
            F.rec_info[qd] = info;
            F.rec_val[qd] = c;
        }
    }
    if (anynan) atomicOr(F.err, kErrNaN);
    nm = __reduce_add_sync(0xffffffffu, nm);
    ns = __reduce_add_sync(0xffffffffu, ns);
    np = __reduce_add_sync(0xffffffffu, np);
    if (lane == 0) {
        if (nm) atomicAdd(&s_cnt[0], nm);
        if (ns) atomicAdd(&s_cnt[1], ns);
        if (np) atomicAdd(&s_cnt[2], np);
    }
    __syncthreads();
    if (tid == 0 && chk(b, F.nbricks, F.err)) F.bcnt[b] = make_uint4(s_cnt[0], s_cnt[1], s_cnt[2], 0u);
}

cudaError_t launch_classify_r5(bool minimum, const FieldDev *fields, int nf, uint64_t bricks, cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    if (minimum) k_classify_r5<true><<<dim3(unsigned(bricks)), kR5Threads, 0, st>>>(fields, nf);
    else k_classify_r5<false><<<dim3(unsigned(bricks)), kR5Threads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
