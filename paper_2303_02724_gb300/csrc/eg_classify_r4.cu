// Steps (a) + (c) for 4D float32 fields (and the float32 image of 8/16-bit
// integer fields) whose rows hold at most 1024 vertices: row classifier
// (Sec. 3.3, Table 1; UpperLinkRep of Sec. 3.4).
//
// A brick is `ty` whole rows (axis 0) of one (z, w) plane; one CTA per brick.
// Each thread classifies 4 consecutive vertices x .. x+3 of one row from
// register copies of the row segments their 30-neighbourhoods touch.  The
// neighbour with pattern p (bit 0: axis 0, bits 1..3: axes 1..3) and sign s
// lies in row q = p >> 1 (offset s along the axes of q) at column x + s*(p&1),
// so 15 rows are read: the centre row at x-1 .. x+4, the seven negative rows
// at x-1 .. x+3, the seven positive rows at x .. x+4.  Columns x .. x+3 come
// from one 16-byte load, the end columns from one more load of the same cache
// lines.  Out-of-domain rows and columns read NaN, which fails every
// ordered comparison and is skipped by min/max, so no bounds test enters the
// per-vertex work.
//
// Per vertex:
//   upper   bit k set iff neighbour k is higher (value, then index: ties go
//           to the positive slots, which have larger indices): 30
//           set-compares accumulated with FMAs into two 15-bit halves;
//   asc     the highest neighbour: the larger of the two halves' maxima
//           (the positive half wins ties: larger indices), then the highest
//           slot of that half holding it;
//   beta0+  the component of the gradient slot inside the upper mask (bitmask
//           flood over the link edges); a saddle when it is not the whole
//           mask, and then every other component and its highest vertex.
// The minimum graph mirrors every comparison and tie rule.
#include <type_traits>

#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kR4Threads = kR4CtaThreads;
constexpr int kR4Vx = kR4Vertices;  // vertices per thread along axis 0

namespace {

__device__ __forceinline__ float r4_set(int op, float a, float b)
{
    float d;
    switch (op) {
    case 0: asm("set.gt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    case 1: asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    case 2: asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    case 3: asm("set.le.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    default: asm("set.eq.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b)); break;
    }
    return d;
}

__device__ __forceinline__ float r4_max3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float r4_min3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Extreme of 15 values (NaN ignored unless all are NaN).
template <bool MIN>
__device__ __forceinline__ float r4_ext15(const float *v)
{
    if (MIN) {
        const float a = r4_min3(v[0], v[1], v[2]), b = r4_min3(v[3], v[4], v[5]), c = r4_min3(v[6], v[7], v[8]);
        const float d = r4_min3(v[9], v[10], v[11]), e = r4_min3(v[12], v[13], v[14]);
        return fminf(r4_min3(a, b, c), fminf(d, e));
    }
    const float a = r4_max3(v[0], v[1], v[2]), b = r4_max3(v[3], v[4], v[5]), c = r4_max3(v[6], v[7], v[8]);
    const float d = r4_max3(v[9], v[10], v[11]), e = r4_max3(v[12], v[13], v[14]);
    return fmaxf(r4_max3(a, b, c), fmaxf(d, e));
}

// Connected component of `s` inside `u`, both in the pattern layout of the 4D
// link: the positive neighbour with axis pattern p (p = 1..15) at bit p, the
// negative one at bit 16 + p.  Two link vertices are joined (Algorithm 1 on
// their difference) iff they have the same sign and comparable patterns, or
// opposite signs and disjoint patterns; so the link neighbours of a set are
// the supersets of its patterns (same half), and the subsets of its patterns
// and of their complements (a bit reversal maps pattern p of one half to
// pattern ~p of the other).  Each step is register-only bit arithmetic
// (superset and subset closures over the four pattern bits of both halves
// at once); the set only grows, so the loop ends within 30 steps.
__device__ __forceinline__ uint32_t r4_component(uint32_t s, uint32_t u)
{
    while (true) {
        uint32_t up = s, dn = s | __brev(s);
        up |= (up & 0x55555555u) << 1;
        up |= (up & 0x33333333u) << 2;
        up |= (up & 0x0f0f0f0fu) << 4;
        up |= (up & 0x00ff00ffu) << 8;
        dn |= (dn >> 1) & 0x55555555u;
        dn |= (dn >> 2) & 0x33333333u;
        dn |= (dn >> 4) & 0x0f0f0f0fu;
        dn |= (dn >> 8) & 0x00ff00ffu;
        const uint32_t n = (up | dn) & u;
        if (n == s) return s;
        s = n;
    }
}

// Pattern layout -> slot mask (slot k: negative k < 15 has pattern 15 - k,
// positive k >= 15 has pattern k - 14).
__device__ __forceinline__ uint32_t r4_slots(uint32_t c) { return ((c & 0xfffeu) << 14) | (__brev(c) & 0x7fffu); }

// Highest slot of `mask` (value, then rank; the minimum graph: lowest value,
// then lowest rank).
template <bool MIN>
__device__ __forceinline__ int r4_top(const float (&nb)[30], uint32_t mask)
{
    float best = 0.f;
    int rk = -1;
#pragma unroll
    for (int k = 0; k < 30; k++)
        if (((mask >> k) & 1u) && (rk < 0 || (MIN ? nb[k] < best : nb[k] >= best))) {
            best = nb[k];
            rk = k;
        }
    return rk;
}

}  // namespace

template <bool MIN>
__global__ void __launch_bounds__(kR4Threads, 3)
k_classify_r4(const FieldDev *__restrict__ fields, int nf)
{
    __shared__ uint32_t s_scan[33];
    __shared__ uint4 s_warp[kR4Threads / 32];  // per-warp counts of maxima, saddles, arc ends
    const uint64_t g = fields[0].brick0 + blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint32_t b = uint32_t(g - F.brick0);
    const int tid = threadIdx.x, lane = tid & 31;

    const uint32_t n0 = F.n[0], n1 = F.n[1], n2 = F.n[2], n3 = F.n[3];
    const uint32_t p = b / F.nyb, yb = b - p * F.nyb;
    const uint32_t z = p % n2, w = p / n2;
    const uint32_t y0 = yb * F.ty;
    const uint32_t brows = min(F.ty, n1 - y0);
    const uint32_t txn = (n0 + kR4Vx - 1) / kR4Vx;
    const uint32_t r = uint32_t(tid) / txn, xt = uint32_t(tid) - r * txn;
    const uint32_t x = kR4Vx * xt;
    const uint32_t y = y0 + r;
    const bool rowok = r < brows;
    const bool vec = F.vec != 0;
    const uint32_t s1 = n0, s2 = n0 * n1, s3 = s2 * n2;
    const uint32_t vrow = ((w * n2 + z) * n1 + y) * n0;  // id of (0, y, z, w) (meaningful when rowok)
    const float qnan = __int_as_float(0x7fc00000);
    const bool first_t = xt == 0, last_t = x + kR4Vx >= n0;

    // columns x .. x+3 of the row at offset `off` (sign sg) from this thread's
    // row, NaN outside the domain
    auto seg = [&](auto inner, uint32_t q, bool neg, float *v) {
        const uint32_t dy = q & 1u, dz = (q >> 1) & 1u, dw = (q >> 2) & 1u;
        bool ok = rowok;
        if (!decltype(inner)::value) {
            if (neg) ok = ok && y >= dy && z >= dz && w >= dw;
            else ok = ok && y + dy < n1 && z + dz < n2 && w + dw < n3;
        }
        const uint32_t off = dy * s1 + dz * s2 + dw * s3;
        const uint32_t rb = neg ? vrow - off : vrow + off;  // (only used when ok)
        if (ok && !(chk(uint64_t(rb) + x, F.N, F.err) && chk(uint64_t(rb) + min(x + kR4Vx, n0) - 1, F.N, F.err)))
            ok = false;
        if (decltype(inner)::value || (ok && vec && x + 3 < n0)) {
            const float4 q4 = __ldg(reinterpret_cast<const float4 *>(F.f + rb + x));
            v[0] = q4.x;
            v[1] = q4.y;
            v[2] = q4.z;
            v[3] = q4.w;
        } else {
#pragma unroll
            for (int j = 0; j < kR4Vx; j++) v[j] = (ok && x + j < n0) ? __ldg(F.f + rb + x + j) : qnan;
        }
        return ok ? rb : 0xffffffffu;
    };
    // column x-1 (left) and x+4 (right) of a row whose segment is v
    // (a load from the same cache lines costs fewer instructions than a
    // shuffle from the neighbouring lane with its fix-up at the warp's edges)
    auto left = [&](uint32_t rb, const float *v) {
        return (rb != 0xffffffffu && !first_t && chk(uint64_t(rb) + x - 1, F.N, F.err)) ? __ldg(F.f + rb + x - 1) : qnan;
    };
    auto right = [&](uint32_t rb, const float *v) {
        return (rb != 0xffffffffu && !last_t && chk(uint64_t(rb) + x + kR4Vx, F.N, F.err)) ? __ldg(F.f + rb + x + kR4Vx)
                                                                                             : qnan;
    };

    // C: centre row, columns x-1 .. x+4 (index j+1 for column x+j)
    // Nr[q]: negative row q, columns x-1 .. x+3; Pr[q]: positive row q, x .. x+4
    float C[kR4Vx + 2], Nr[7][kR4Vx + 1], Pr[7][kR4Vx + 1];
    auto loads = [&](auto inner) {
        {
            const uint32_t rb = seg(inner, 0, false, &C[1]);
            C[0] = left(rb, &C[1]);
            C[kR4Vx + 1] = right(rb, &C[1]);
        }
#pragma unroll
        for (int q = 1; q < 8; q++) {
            const uint32_t rn = seg(inner, uint32_t(q), true, &Nr[q - 1][1]);
            Nr[q - 1][0] = left(rn, &Nr[q - 1][1]);
            const uint32_t rp = seg(inner, uint32_t(q), false, &Pr[q - 1][0]);
            Pr[q - 1][kR4Vx] = right(rp, &Pr[q - 1][0]);
        }
    };
    // a thread with room on both sides along axes 1..3 and 16-byte rows
    // (most threads; a warp agrees whenever it lies in one row) loads through
    // a copy without the rows' domain tests
    if (rowok && vec && y >= 1 && y + 1 < n1 && z >= 1 && z + 1 < n2 && w >= 1 && w + 1 < n3)
        loads(std::true_type{});
    else
        loads(std::false_type{});

    // the 30 neighbour values of vertex i in slot order (slot k: k < 15
    // negative with pattern 15 - k, k >= 15 positive with pattern k - 14)
    auto neighbours = [&](int i, float (&nb)[30]) {
#pragma unroll
        for (int k = 0; k < 30; k++) {
            const bool neg = k < 15;
            const int pt = neg ? 15 - k : k - 14;
            const int q = pt >> 1, xb = pt & 1;
            if (q == 0) nb[k] = neg ? C[i] : C[i + 2];  // (pattern 1: the axis-0 neighbours)
            else if (neg) nb[k] = xb ? Nr[q - 1][i] : Nr[q - 1][i + 1];
            else nb[k] = xb ? Pr[q - 1][i + 1] : Pr[q - 1][i];
        }
    };

    // ---- per vertex: upper mask, gradient slot, and the seed of its component
    uint32_t asc[kR4Vx], Um[kR4Vx], comp[kR4Vx];
    int gslot[kR4Vx];
#pragma unroll
    for (int i = 0; i < kR4Vx; i++) {
        const float c = C[i + 1];
        float nb[30];
        neighbours(i, nb);
        // upper mask: negative slots need a strictly higher value, positive
        // slots a higher or equal one (mirrored for the minimum graph); each
        // test is 1.0 or 0.0, accumulated as bit k of a float whose exponent
        // pins the integer part (2^23 + a 15-bit mask is exact)
        float an = 8388608.f, ap = 8388608.f;
#pragma unroll
        for (int k = 0; k < 15; k++) an = __fmaf_rn(r4_set(MIN ? 3 : 0, nb[k], c), float(1u << k), an);
#pragma unroll
        for (int k = 0; k < 15; k++) ap = __fmaf_rn(r4_set(MIN ? 2 : 1, nb[15 + k], c), float(1u << k), ap);
        const uint32_t un = __float_as_uint(an) & 0x7fffu, up = __float_as_uint(ap) & 0x7fffu;
        // gradient: the half holding the extreme value (ties: the positive
        // half for the maximum graph, the negative half for the minimum
        // graph), then its highest (lowest) slot holding that value
        const float mN = r4_ext15<MIN>(nb), mP = r4_ext15<MIN>(nb + 15);
        // (a half without in-domain neighbours has a NaN extreme and loses)
        const bool pos = (MIN ? (mP < mN) : (mP >= mN)) || (mN != mN);
        const float mw = pos ? mP : mN;
        float ae = 8388608.f;
#pragma unroll
        for (int j = 0; j < 15; j++) ae = __fmaf_rn(r4_set(4, pos ? nb[15 + j] : nb[j], mw), float(1u << j), ae);
        const uint32_t eq = __float_as_uint(ae) & 0x7fffu;
        const uint32_t v = vrow + x + uint32_t(i);
        // the winning half holds an upper slot with the extreme value
        // whenever the mask is not empty; the fallback only keeps the slot in
        // range
        const uint32_t cand = eq & (pos ? up : un);
        int slot;
        if (cand) slot = (MIN ? (__ffs(cand) - 1) : (31 - __clz(cand))) + (pos ? 15 : 0);
        else slot = (un | up) ? (MIN ? (__ffs(un | (up << 15)) - 1) : (31 - __clz(un | (up << 15)))) : 0;
        const int pt = slot < 15 ? 15 - slot : slot - 14;
        const uint32_t o = ((pt & 1) ? 1u : 0u) + ((pt & 2) ? s1 : 0u) + ((pt & 4) ? s2 : 0u) + ((pt & 8) ? s3 : 0u);
        asc[i] = (un | up) ? (slot < 15 ? v - o : v + o) : v;
        gslot[i] = slot;
        // the upper link in the pattern layout; the seed of the gradient's
        // component: its whole half when that half holds its full pattern
        // (comparable to every pattern of the half), else the gradient alone
        const uint32_t U = (up << 1) | __brev(un);
        Um[i] = U;
        const uint32_t half = slot < 15 ? 0xffff0000u : 0x0000ffffu;
        const uint32_t full = slot < 15 ? 0x80000000u : 0x00008000u;
        comp[i] = (U & full) ? (U & half) : (1u << (slot < 15 ? 31 - slot : slot - 14));
    }
    // ---- the gradient's component inside each upper link: the four
    // closures advance together (independent chains); bounded by 30 steps
    for (int it = 0; it < 30; it++) {
        bool grew = false;
#pragma unroll
        for (int i = 0; i < kR4Vx; i++) {
            uint32_t s0 = comp[i], upc = s0, dn = s0 | __brev(s0);
            upc |= (upc & 0x55555555u) << 1;
            upc |= (upc & 0x33333333u) << 2;
            upc |= (upc & 0x0f0f0f0fu) << 4;
            upc |= (upc & 0x00ff00ffu) << 8;
            dn |= (dn >> 1) & 0x55555555u;
            dn |= (dn >> 2) & 0x33333333u;
            dn |= (dn >> 4) & 0x0f0f0f0fu;
            dn |= (dn >> 8) & 0x00ff00ffu;
            const uint32_t nx = (upc | dn) & Um[i];
            grew |= nx != s0 && nx != Um[i];  // (a whole upper link cannot grow)
            comp[i] = nx;
        }
        if (!grew) break;
    }
    // ---- maxima, saddles (every other component and its highest slot)
    uint64_t info[kR4Vx];
    uint32_t crit = 0, nm = 0, ns = 0, np = 0;
    bool anynan = false;
#pragma unroll
    for (int i = 0; i < kR4Vx; i++) {
        const bool ok = rowok && x + i < n0;
        const uint32_t U = Um[i];
        uint64_t inf = 0;
        bool cv = false;
        if (ok && U == 0) {
            cv = true;
            nm++;
            anynan |= C[i + 1] != C[i + 1];  // a NaN value has no upper neighbour
        } else if (ok && comp[i] != U) {
            // the upper neighbours' values, reloaded through the cache: saddles
            // are rare, and keeping the row segments live until here would
            // make every vertex's registers spill
            float nb[30];
            const uint32_t up_slots = r4_slots(U), vi = vrow + x + uint32_t(i);
#pragma unroll
            for (int k = 0; k < 30; k++) {
                nb[k] = qnan;
                if ((up_slots >> k) & 1u) {
                    const int pt = k < 15 ? 15 - k : k - 14;
                    const uint32_t o = ((pt & 1) ? 1u : 0u) + ((pt & 2) ? s1 : 0u) + ((pt & 4) ? s2 : 0u) +
                                       ((pt & 8) ? s3 : 0u);
                    const uint32_t w = k < 15 ? vi - o : vi + o;
                    if (chk(w, F.N, F.err)) nb[k] = __ldg(F.f + w);
                }
            }
            uint64_t codes = uint64_t(gslot[i]);
            int b0 = 1;
            for (uint32_t lft = U & ~comp[i]; lft;) {
                const uint32_t c2 = r4_component(lft & (~lft + 1u), U);
                lft &= ~c2;
                codes |= uint64_t(r4_top<MIN>(nb, r4_slots(c2))) << (5 * b0);
                b0++;
            }
            inf = (uint64_t(b0) << 56) | codes;
            cv = true;
            ns++;
            np += uint32_t(b0);
        }
        info[i] = inf;
        if (cv) crit |= 1u << i;
    }
    if (rowok && chk(uint64_t(vrow) + x + min(uint32_t(kR4Vx), n0 - x) - 1, F.N, F.err)) {
        uint32_t *dst = F.lab + vrow + x;
        if (vec && x + 3 < n0) {
            *reinterpret_cast<uint4 *>(dst) = make_uint4(asc[0], asc[1], asc[2], asc[3]);
        } else {
#pragma unroll
            for (int i = 0; i < kR4Vx; i++)
                if (x + i < n0) dst[i] = asc[i];
        }
    }
    // the brick's counts per warp (published by the scan's barriers)
    nm = __reduce_add_sync(0xffffffffu, nm);
    ns = __reduce_add_sync(0xffffffffu, ns);
    np = __reduce_add_sync(0xffffffffu, np);
    if (lane == 0) s_warp[tid >> 5] = make_uint4(nm, ns, np, 0u);
    // records of the brick in index order: threads are in (row, x) order
    uint32_t tot;
    const uint32_t pos0 = block_excl_scan(uint32_t(__popc(crit)), s_scan, &tot);
    const uint64_t slot0 = uint64_t(b) * F.bcap;
    uint32_t k = 0;
#pragma unroll
    for (int i = 0; i < kR4Vx; i++)
        if ((crit >> i) & 1u) {
            const uint64_t qd = slot0 + pos0 + k++;
            if (!chk(qd, rec_cap(F), F.err) || !chk(qd - slot0, F.bcap, F.err)) continue;
            F.rec_sid[qd] = vrow + x + uint32_t(i);
            F.rec_info[qd] = info[i];
            F.rec_val[qd] = C[i + 1];
        }
    if (anynan) atomicOr(F.err, kErrNaN);
    if (tid == 0 && chk(b, F.nbricks, F.err)) {
        uint4 c = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int w = 0; w < kR4Threads / 32; w++) {
            const uint4 q = s_warp[w];
            c.x += q.x;
            c.y += q.y;
            c.z += q.z;
        }
        F.bcnt[b] = c;
    }
}

cudaError_t launch_classify_r4(bool minimum, const FieldDev *fields, int nf, uint64_t bricks, cudaStream_t st)
{
    if (bricks == 0) return cudaSuccess;
    if (minimum) k_classify_r4<true><<<dim3(unsigned(bricks)), kR4Threads, 0, st>>>(fields, nf);
    else k_classify_r4<false><<<dim3(unsigned(bricks)), kR4Threads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
