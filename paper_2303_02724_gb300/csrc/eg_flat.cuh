// Per-vertex classification in any dimension (Sec. 3.3, Table 1; the
// UpperLinkRep of Sec. 3.4), reading the neighbours through the read-only
// cache: shared by the flat classifier (eg_classify.cu) and the fused
// small-field kernel (eg_small.cu).
#pragma once

#include "eg_internal.cuh"

namespace eg {

// Raw bits of element v: float32 reads F.f (the field, or the float32 image of
// a narrow integer field), every other type reads the field itself.
template <uint32_t DT>
__device__ __forceinline__ typename TypeKey<DT>::B load_bits(const FieldDev &F, uint32_t v)
{
    using B = typename TypeKey<DT>::B;
    if (!chk(v, F.N, F.err)) return B(0);
    if constexpr (DT == kF32) return __float_as_uint(__ldg(F.f + v));
    else if constexpr (sizeof(B) == 8) return B(__ldg(static_cast<const unsigned long long *>(F.fraw) + v));
    else return B(__ldg(static_cast<const unsigned int *>(F.fraw) + v));
}

// Classify vertex v of field F.  Returns asc(v); sets b0 and the
// representatives' slots in the record format of the dimension (rec_b0,
// rec_slots): 5-bit fields up to 4D (component order arbitrary), a slot mask
// in 5D.
//
// Inside one neighbourhood the simulated perturbation needs no index
// arithmetic: slot order is index order, so among equal values a positive
// slot (larger index) is higher than the centre and a negative one lower;
// among neighbours, the later slot is higher.  The minimum graph complements
// the keys and mirrors both rules.
template <int D, uint32_t DT>
__device__ __forceinline__ uint32_t classify_vertex(const FieldDev &F, const uint32_t (&s)[kMaxDim],
                                                    uint32_t v, bool minimum, int &b0, uint64_t &codes, bool &nan)
{
    using NB = Nbr<D>;
    using PL = PatternLink<D>;
    using M = typename PL::Mask;  // the upper link in the pattern layout
    using TK = TypeKey<DT>;
    using B = typename TK::B;
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
    const B flip = minimum ? ~B(0) : B(0);
    const B bv = load_bits<DT>(F, v);
    nan = TK::nan(bv);
    const B kv = TK::key(bv) ^ flip;
    // key of the neighbour in slot k (in bounds; reloaded through the cache
    // for saddles rather than kept in registers for every vertex)
    auto nkey = [&](int k) {
        const uint32_t p = NB::pat(k);
        uint32_t o = 0;
#pragma unroll
        for (int i = 0; i < D; i++)
            if (p & (1u << i)) o += s[i];
        return TK::key(load_bits<DT>(F, NB::neg(k) ? v - o : v + o)) ^ flip;
    };
    M upper = 0;
    uint32_t asc = v;
    B best = 0;
    int bestk = -1;
#pragma unroll
    for (int k = 0; k < K; k++) {
        const uint32_t p = NB::pat(k);
        const bool inb = NB::neg(k) ? ((p & ~mok) == 0) : ((p & ~pok) == 0);
        B kw = 0;
        bool up = false;
        uint32_t w = 0;
        if (inb) {
            uint32_t o = 0;
#pragma unroll
            for (int i = 0; i < D; i++)
                if (p & (1u << i)) o += s[i];
            w = NB::neg(k) ? v - o : v + o;
            kw = TK::key(load_bits<DT>(F, w)) ^ flip;
            // ties: higher iff the slot lies above the centre in the order
            up = (NB::neg(k) == minimum) ? kw >= kv : kw > kv;
        }
        if (up) {
            upper |= M(1) << PL::bit(k);
            // the highest upper neighbour; among equal keys the later slot
            // (maximum graph) or the earlier one (minimum graph)
            if (bestk < 0 || (minimum ? kw > best : kw >= best)) {
                best = kw;
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
    const M comp = PL::component(M(1) << PL::bit(bestk), upper);
    b0 = 1;
    if (comp == upper) return asc;
    codes = D == 5 ? (1ull << bestk) : uint64_t(bestk);
    M left = upper & ~comp;
    while (left) {
        const M c2 = PL::component(left & (~left + M(1)), upper);
        left &= ~c2;
        B rb = 0;
        int rk = -1;
#pragma unroll
        for (int k = 0; k < K; k++)
            if ((c2 >> PL::bit(k)) & 1u) {
                const B kk = nkey(k);
                if (rk < 0 || (minimum ? kk > rb : kk >= rb)) {
                    rb = kk;
                    rk = k;
                }
            }
        codes |= D == 5 ? (1ull << rk) : (uint64_t(rk) << (5 * b0));
        b0++;
    }
    return asc;
}

}  // namespace eg
