// Steps (a) + (c) for 2D and 3D fields whose rows hold at most 2048 vertices:
// plane-marching classification (Sec. 3.3, Table 1; 2D runs as 3D, n2 = 1).
//
// A CTA owns `ty` whole rows of the grid (a row block) and marches along the
// slowest axis over `zc` planes.  A ring of four plane buffers in shared
// memory holds planes z-1, z, z+1 while plane z+2 streams in with cp.async;
// each buffer holds rows y0-1 .. y0+ty of one plane, rows separated by eight
// NaN.  Out-of-domain rows and planes are NaN as well, and NaN fails every
// ordered comparison, is skipped by min/max and equals nothing, so no bounds
// test is needed.
//
// Each thread classifies 8 consecutive vertices of one row of plane z from
// register copies of the 7 row segments their 14-neighbourhoods touch.  Per
// vertex:
//   upper   bit k set iff neighbour k is higher (value, then index: ties go to
//           the positive slots, which have larger indices); 14 set-compares
//           whose 0/1 results are accumulated with FMAs;
//   asc     the highest neighbour: the largest value (three-operand max), then
//           the highest slot rank holding it;
//   saddle  beta0+ >= 2, looked up in a table of 2-bit classes indexed by the
//           upper mask (built on the host from the link graph); the components
//           and their highest vertices (UpperLinkRep, Sec. 3.4) are then found
//           by flood fill, for saddles only, after the plane.
// The minimum graph mirrors every comparison and the tie rule.
//
// One row block of one plane is one brick (contiguous ids): asc goes to lab;
// its maxima and saddles go, in index order, to the brick's record slot.  The
// records are written by each warp cooperatively after a block scan of the
// counts: lane j writes the warp's j-th record (coalesced) and, for a saddle,
// also resolves its components, so the saddle work is spread over the lanes.
#include <atomic>

#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kZmThreads = 256;

__device__ __forceinline__ void cp_async16(float *smem, const float *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(float *smem, const float *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Shared-memory geometry of one field's ring buffers (in floats).
struct ZmGeom {
    uint32_t n0, n1, n2, ty, rstride, rb;
};

// Ring buffer: rows of n0 values rounded up to a multiple of 8 and followed by
// 8 NaN (each row's trailing pad is the next row's leading pad), 8 more at each
// end; reads of columns -1 .. n0+7 stay inside the buffer.
__host__ __device__ __forceinline__ uint32_t zm_rstride(uint32_t n0) { return ((n0 + 7) & ~7u) + 8; }

__host__ __device__ __forceinline__ uint32_t zm_ring_floats(uint32_t n0, uint32_t ty)
{
    return ((ty + 2) * zm_rstride(n0) + 16 + 3) & ~3u;
}

// Stored position of column x in a ring row: in every group of 8 columns the
// two halves trade places when bit 2 of the group index is set, so that the
// 16-byte loads of the eight lanes of a quarter-warp (consecutive groups) hit
// distinct banks.  A permutation inside each group; pads stay pads.
__device__ __forceinline__ int zm_col(int x) { return x ^ (((x >> 5) & 1) << 2); }

// This thread's first copy unit (row r0, unit c0 of the row) and the stride
// between its units (dr rows + dc units), for units of 16 bytes (vec) or 4
// bytes per row; fixed for a work item, so no division per plane.
struct ZmCopy {
    uint32_t r0, c0, dr, dc, upr;
};

__device__ __forceinline__ ZmCopy zm_copy_plan(uint32_t n0, bool vec)
{
    ZmCopy P;
    P.upr = vec ? (n0 >> 2) : n0;
    P.r0 = uint32_t(threadIdx.x) / P.upr;
    P.c0 = uint32_t(threadIdx.x) - P.r0 * P.upr;
    P.dr = uint32_t(kZmThreads) / P.upr;
    P.dc = uint32_t(kZmThreads) - P.dr * P.upr;
    return P;
}

// Stream rows [ylo, yhi) of plane z into ring slot `buf` (or NaN-fill the slot
// when z is past the last plane).  Always commits one cp.async group.
__device__ __forceinline__ void zm_load_plane(const FieldDev &F, const ZmGeom &G, const ZmCopy &P, float *buf, int z,
                                              uint32_t y0, uint32_t ylo, uint32_t yhi, bool vec, const float *ring)
{
    const uint32_t rows = yhi - ylo;
    float *dst0 = buf + 8 + (ylo - y0 + 1) * G.rstride;
    if (z < 0) {
        cp_async_commit();
        return;
    }
    const bool fill = uint32_t(z) >= G.n2;
    const float *src0 = F.f + (uint64_t(fill ? 0 : z) * G.n1 + ylo) * G.n0;
    const uint32_t w = vec ? 4u : 1u;  // floats per unit
    for (uint32_t r = P.r0, c = P.c0; r < rows;) {
        float *d = dst0 + r * G.rstride + zm_col(int(w * c));
        if (!chk_ptr<float>(d + w - 1, ring, 4 * uint64_t(G.rb), F.err) || !chk_ptr<float>(d, ring, 4 * uint64_t(G.rb), F.err)) {
            r += P.dr;
            c += P.dc;
            if (c >= P.upr) {
                c -= P.upr;
                r++;
            }
            continue;
        }
        if (fill) {
            const float qnan = __int_as_float(0x7fc00000);
            if (vec)
                *reinterpret_cast<float4 *>(d) = make_float4(qnan, qnan, qnan, qnan);
            else
                *d = qnan;
        } else {
            const float *g = src0 + uint64_t(r) * G.n0 + w * c;
            if (!chk_ptr(g + w - 1, F.f, F.N, F.err) || !chk_ptr(g, F.f, F.N, F.err)) {
            } else if (vec) {
                cp_async16(d, g);
            } else {
                cp_async4(d, g);
            }
        }
        r += P.dr;
        c += P.dc;
        if (c >= P.upr) {
            c -= P.upr;
            r++;
        }
    }
    cp_async_commit();
}

// Float comparisons that return 1.0f / 0.0f (false for NaN operands).
__device__ __forceinline__ float set_gt(float a, float b)
{
    float d;
    asm("set.gt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float set_ge(float a, float b)
{
    float d;
    asm("set.ge.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float set_lt(float a, float b)
{
    float d;
    asm("set.lt.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float set_le(float a, float b)
{
    float d;
    asm("set.le.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float set_eq(float a, float b)
{
    float d;
    asm("set.eq.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Three-operand max / min (NaN operands are ignored unless all are NaN).
__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Largest / smallest of 14 values in seven three-operand steps.
__device__ __forceinline__ float max7x2(const float (&v)[14])
{
    const float a = max3f(v[0], v[1], v[2]), b = max3f(v[3], v[4], v[5]);
    const float c = max3f(v[6], v[7], v[8]), d = max3f(v[9], v[10], v[11]);
    return fmaxf(max3f(a, b, v[12]), max3f(c, d, v[13]));
}
__device__ __forceinline__ float min7x2(const float (&v)[14])
{
    const float a = min3f(v[0], v[1], v[2]), b = min3f(v[3], v[4], v[5]);
    const float c = min3f(v[6], v[7], v[8]), d = min3f(v[9], v[10], v[11]);
    return fminf(min3f(a, b, v[12]), min3f(c, d, v[13]));
}

// The 14 neighbour values of column xx of ring row `row` of plane buffer C (D
// and U at float offsets dD, dU from C), in slot order.
__device__ __forceinline__ void ring_nbrs(const float *row, int xx, int rs, int dD, int dU, float (&nb)[14])
{
    const int cm = zm_col(xx - 1), c0 = zm_col(xx), cp = zm_col(xx + 1);
    const float *d0 = row + dD - rs, *d1 = row + dD;
    const float *r0 = row - rs, *r2 = row + rs;
    const float *u1 = row + dU, *u2 = row + dU + rs;
    // (-1,-1,-1) (0,-1,-1) (-1,0,-1) (0,0,-1) (-1,-1,0) (0,-1,0) (-1,0,0)
    // (1,0,0) (0,1,0) (1,1,0) (0,0,1) (1,0,1) (0,1,1) (1,1,1)
    nb[0] = d0[cm];
    nb[1] = d0[c0];
    nb[2] = d1[cm];
    nb[3] = d1[c0];
    nb[4] = r0[cm];
    nb[5] = r0[c0];
    nb[6] = row[cm];
    nb[7] = row[cp];
    nb[8] = r2[c0];
    nb[9] = r2[cp];
    nb[10] = u1[c0];
    nb[11] = u1[cp];
    nb[12] = u2[c0];
    nb[13] = u2[cp];
}

// Highest slot of `mask` (value, then rank; the minimum graph takes the
// lowest value and the lowest rank).
template <bool MIN>
__device__ __forceinline__ int masked_top(const float (&nb)[14], uint32_t mask)
{
    float best = 0.f;
    int rk = -1;
#pragma unroll
    for (int k = 0; k < 14; k++)
        if (((mask >> k) & 1u) && (rk < 0 || (MIN ? nb[k] < best : nb[k] >= best))) {
            best = nb[k];
            rk = k;
        }
    return rk;
}

// Upper-link components of one saddle and the highest vertex of each
// (UpperLinkRep, Sec. 3.4), packed as 5-bit slots with beta0+ in bits 56..59.
// first: the gradient slot (highest of all upper neighbours, hence the
// representative of its component); cls: 1 when the table says exactly two
// components.  low[m] (host-built table): the component of mask m holding
// m's lowest set bit; a2 = low[upper].  Removing whole components leaves the
// others intact, so low[] peels them off one by one.
template <bool MIN>
__device__ __forceinline__ uint64_t saddle_info(const float (&nb)[14], uint32_t upper, int first, uint32_t cls,
                                                uint32_t a2, const uint16_t *low)
{
    uint64_t codes = uint64_t(first);
    if (cls == 1) {
        const uint32_t other = ((a2 >> first) & 1u) ? (upper ^ a2) : a2;
        codes |= uint64_t(masked_top<MIN>(nb, other)) << 5;
        return (2ull << 56) | codes;
    }
    int b0 = 1;
    for (uint32_t left = upper, c = a2; left; c = left ? uint32_t(__ldg(low + left)) : 0u) {
        c = (c & left) ? (c & left) : left;  // (never empty; guarantees progress)
        left &= ~c;
        if ((c >> first) & 1u) continue;  // the gradient's component: coded first
        codes |= uint64_t(masked_top<MIN>(nb, c)) << (5 * b0);
        b0++;
    }
    return (uint64_t(b0) << 56) | codes;
}

constexpr int kVx = 8;  // vertices per thread along axis 0

template <bool MIN>
__global__ void __launch_bounds__(kZmThreads, 3)
k_classify_zm(const FieldDev *__restrict__ fields, int nf, const uint32_t *__restrict__ lut, uint64_t total_items,
              unsigned long long *ticket)
{
    extern __shared__ float4 zm_smem4[];
    float *ring = reinterpret_cast<float *>(zm_smem4);
    __shared__ uint32_t s_lut[1024];
    __shared__ uint32_t s_off[14];
    __shared__ uint32_t s_warp[kZmThreads / 32];
    __shared__ unsigned s_cnt[4];
    // per-vertex classification of this step (upper mask | gradient slot << 14 |
    // class << 18), thread-major, read back by the record writers
    __shared__ __align__(16) uint32_t s_um[kZmThreads * kVx];

    __shared__ unsigned long long s_item;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint16_t *lowc = reinterpret_cast<const uint16_t *>(lut + 1024);
    for (int i = tid; i < 1024; i += kZmThreads) s_lut[i] = __ldg(lut + i);
    // persistent work queue: take items in ticket order until none are left
    while (true) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(ticket, 1ull);
    __syncthreads();
    const uint64_t g = s_item;
    if (g >= total_items) break;
    const int fi = find_field<true>(fields, nf, g);
    const FieldDev &F = fields[fi];
    const uint32_t item = uint32_t(g - F.item0);
    ZmGeom G;
    G.n0 = F.n[0];
    G.n1 = F.n[1];
    G.n2 = F.n[2];
    G.ty = F.ty;
    G.rstride = zm_rstride(G.n0);
    G.rb = zm_ring_floats(G.n0, G.ty);
    const uint32_t yb = item % F.nyb, zci = item / F.nyb;
    const uint32_t y0 = yb * G.ty;
    const uint32_t brows = min(G.ty, G.n1 - y0);  // rows of this row block
    const uint32_t ylo = y0 > 0 ? y0 - 1 : 0;
    const uint32_t yhi = min(G.n1, y0 + G.ty + 1);
    const int zs = int(zci * F.zc);
    const int ze = int(min(G.n2, zci * F.zc + F.zc));
    const bool vec = F.vec != 0;
    const ZmCopy P = zm_copy_plan(G.n0, vec);

    if (tid < 14) {
        const uint32_t p = Nbr<3>::pat(tid);
        const uint32_t mag = ((p & 1u) ? 1u : 0u) + ((p & 2u) ? G.n0 : 0u) + ((p & 4u) ? G.n0 * G.n1 : 0u);
        s_off[tid] = Nbr<3>::neg(tid) ? 0u - mag : mag;
    }
    if (tid < 4) s_cnt[tid] = 0;
    {
        const float qnan = __int_as_float(0x7fc00000);
        for (uint32_t i = tid; i < 4 * G.rb; i += kZmThreads) ring[i] = qnan;
    }
    __syncthreads();

    zm_load_plane(F, G, P, ring + ((zs - 1) & 3) * G.rb, zs - 1, y0, ylo, yhi, vec, ring);
    zm_load_plane(F, G, P, ring + (zs & 3) * G.rb, zs, y0, ylo, yhi, vec, ring);
    zm_load_plane(F, G, P, ring + ((zs + 1) & 3) * G.rb, zs + 1, y0, ylo, yhi, vec, ring);

    // thread t owns vertices x .. x+7 of brick row r; threads are in (row, x)
    // order, which is the brick's index order
    const uint32_t txn = (G.n0 + kVx - 1) / kVx;
    const bool active = uint32_t(tid) < txn * G.ty;
    const uint32_t txt = uint32_t(tid) % txn, r = uint32_t(tid) / txn;
    const uint32_t x = kVx * txt;
    const uint32_t rs = G.rstride;
    const uint32_t rr = r + 1;  // ring row of this thread's grid row
    bool anynan = false;
    uint32_t prev_brick = 0xffffffffu;

    for (int z = zs; z < ze; z++) {
        __syncthreads();  // A: previous step done (ring slot, counters final)
        if (tid == 0 && prev_brick != 0xffffffffu) {
            if (chk(prev_brick, F.nbricks, F.err)) F.bcnt[prev_brick] = make_uint4(s_cnt[0], s_cnt[1] - s_cnt[0], s_cnt[2], 0u);
            s_cnt[0] = s_cnt[1] = s_cnt[2] = s_cnt[3] = 0;
        }
        zm_load_plane(F, G, P, ring + ((z + 2) & 3) * G.rb, z + 2, y0, ylo, yhi, vec, ring);
        cp_async_wait1();
        __syncthreads();  // B: plane z+1 visible, counters reset

        const float *Db = ring + ((z - 1) & 3) * G.rb + 8;
        const float *Cb = ring + (z & 3) * G.rb + 8;
        const float *Ub = ring + ((z + 1) & 3) * G.rb + 8;
        const int dD = int(Db - Cb), dU = int(Ub - Cb);
        const uint32_t brick = uint32_t(z) * F.nyb + yb;
        const uint64_t slot0 = uint64_t(brick) * F.bcap;
        const bool rowok = active && r < brows;
        const uint32_t vrow = uint32_t((uint64_t(z) * G.n1 + y0 + r) * G.n0) + x;
        uint32_t um[kVx];  // upper mask | gradient slot << 14 | class << 18
        uint32_t crit = 0, nm = 0;
        // ---- phase 1: gradient pointer, upper mask, saddle test.  Out-of-domain
        // neighbours read NaN pads, which fail every ordered comparison, are
        // ignored by min/max and never equal anything.
        // row segments: C rows r-1..r+1 at x-1..x+8, D rows r-1..r at
        // x-1..x+7, U rows r..r+1 at x..x+8 (lanes without vertices read ring
        // row 1 and discard it).
        float C[3][kVx + 2], D[2][kVx + 1], U[2][kVx + 1];
        {
            const uint32_t rl = rowok ? rr : 1u;
            const float qnan = __int_as_float(0x7fc00000);
            const bool first_t = txt == 0, last_t = txt + 1 == txn;
            // 8 values of columns x..x+7 of ring row `row`
            const uint64_t ringn = 4 * uint64_t(G.rb);
            auto seg = [&](const float *row, float *v) {
                if (!chk_ptr(row + x - 8, ring, ringn, F.err) || !chk_ptr(row + x + 15, ring, ringn, F.err)) {
#pragma unroll
                    for (int b = 0; b < kVx; b++) v[b] = qnan;
                } else if (vec) {
                    const uint32_t h = (x >> 3) & 4u;  // stored order of the two halves
                    const float4 q0 = *reinterpret_cast<const float4 *>(row + x + h);
                    const float4 q1 = *reinterpret_cast<const float4 *>(row + x + (h ^ 4u));
                    v[0] = q0.x; v[1] = q0.y; v[2] = q0.z; v[3] = q0.w;
                    v[4] = q1.x; v[5] = q1.y; v[6] = q1.z; v[7] = q1.w;
                } else {
#pragma unroll
                    for (int b = 0; b < kVx; b++) v[b] = row[zm_col(int(x) + b)];
                }
            };
            // columns x-1 and x+8, read from the ring (cheaper than a shuffle
            // from the neighbouring lane with a fix-up read at the warp's edges)
            auto left = [&](const float *row, float) {
                if (first_t) return qnan;
                return chk_ptr(row + zm_col(int(x) - 1), ring, ringn, F.err) ? row[zm_col(int(x) - 1)] : qnan;
            };
            auto right = [&](const float *row, float) {
                if (last_t) return qnan;
                return chk_ptr(row + zm_col(int(x) + kVx), ring, ringn, F.err) ? row[zm_col(int(x) + kVx)] : qnan;
            };
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float *row = Cb + (rl - 1 + a) * rs;
                seg(row, &C[a][1]);
                C[a][0] = left(row, C[a][kVx]);
                C[a][kVx + 1] = right(row, C[a][1]);
            }
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const float *drow = Db + (rl - 1 + a) * rs;
                const float *urow = Ub + (rl + a) * rs;
                seg(drow, &D[a][1]);
                D[a][0] = left(drow, D[a][kVx]);
                seg(urow, &U[a][0]);
                U[a][kVx] = right(urow, U[a][0]);
            }
        }
        if (rowok) {
            uint32_t asc[kVx];
#pragma unroll
            for (int i = 0; i < kVx; i++) {
                const float c = C[1][i + 1];
                // slot order: (-1,-1,-1) (0,-1,-1) (-1,0,-1) (0,0,-1) (-1,-1,0) (0,-1,0)
                // (-1,0,0) | (1,0,0) (0,1,0) (1,1,0) (0,0,1) (1,0,1) (0,1,1) (1,1,1)
                const float nb[14] = {D[0][i], D[0][i + 1], D[1][i], D[1][i + 1], C[0][i],     C[0][i + 1],
                                      C[1][i], C[1][i + 2], C[2][i + 1], C[2][i + 2], U[0][i], U[0][i + 1],
                                      U[1][i], U[1][i + 1]};
                // upper: negative slots (smaller index) need a strictly higher
                // value, positive slots a higher or equal one (maximum graph); the
                // minimum graph mirrors both.  Each test yields 0.0 or 1.0 and is
                // accumulated as bit k of a float whose exponent pins the
                // integer part (2^23 + mask is exact), on the FMA pipe.
                float au = 8388608.f;
#pragma unroll
                for (int k = 0; k < 14; k++) {
                    const float t = MIN ? (k < 7 ? set_le(nb[k], c) : set_lt(nb[k], c))
                                        : (k < 7 ? set_gt(nb[k], c) : set_ge(nb[k], c));
                    au = __fmaf_rn(t, float(1u << k), au);
                }
                uint32_t upper = __float_as_uint(au) & 0x3fffu;
                // gradient: the extreme neighbour value, then the highest (maximum
                // graph) or lowest (minimum graph) slot holding it among the upper
                // neighbours
                const float m = MIN ? min7x2(nb) : max7x2(nb);
                float ae = 8388608.f;
#pragma unroll
                for (int k = 0; k < 14; k++) ae = __fmaf_rn(set_eq(nb[k], m), float(1u << k), ae);
                const uint32_t eq = __float_as_uint(ae) & 0x3fffu;
                const bool ok = x + i < G.n0;
                const uint32_t v = vrow + i;
                uint32_t a = v;
                bool cv = false;
                uint32_t cls = 0, slot = 0;
                if (upper) {
                    uint32_t cand = eq & upper;
                    cand = cand ? cand : upper;  // (never empty; keeps the slot in range)
                    slot = MIN ? uint32_t(__ffs(cand) - 1) : uint32_t(31 - __clz(cand));
                    a = v + s_off[slot];
                    cls = (s_lut[upper >> 4] >> ((upper & 15) << 1)) & 3u;
                    cv = cls != 0;
                } else {
                    cv = true;
                    nm += ok ? 1u : 0u;
                    anynan |= ok && (c != c);  // a NaN value has no upper neighbour
                }
                asc[i] = a;
                um[i] = upper | (slot << 14) | (cls << 18);
                if (ok) crit |= cv ? (1u << i) : 0u;
            }
            uint4 *um4 = reinterpret_cast<uint4 *>(s_um + tid * kVx);
            um4[0] = make_uint4(um[0], um[1], um[2], um[3]);
            um4[1] = make_uint4(um[4], um[5], um[6], um[7]);
            uint32_t *dst = F.lab + vrow;
            if (!chk(uint64_t(vrow) + min(uint32_t(kVx), G.n0 - x) - 1, F.N, F.err)) {
            } else if (vec) {
                // n0 is a multiple of 4, so x+3 < n0; the second half may be past the row
                *reinterpret_cast<uint4 *>(dst) = make_uint4(asc[0], asc[1], asc[2], asc[3]);
                if (x + 7 < G.n0) *reinterpret_cast<uint4 *>(dst + 4) = make_uint4(asc[4], asc[5], asc[6], asc[7]);
            } else {
#pragma unroll
                for (int i = 0; i < kVx; i++)
                    if (x + i < G.n0) dst[i] = asc[i];
            }
        }
        // ---- order-preserving compaction: threads are in index order
        const uint32_t cnt = __popc(crit);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_warp[warp] = inc;
        nm = __reduce_add_sync(0xffffffffu, nm);
        if (lane == 0 && nm) atomicAdd(&s_cnt[0], nm);
        __syncthreads();  // C: warp totals visible
        uint32_t pw = 0, tot = 0;  // this warp's first record, the brick's record count
#pragma unroll
        for (int w = 0; w < kZmThreads / 32; w++) {
            const uint32_t t = s_warp[w];
            pw += w < warp ? t : 0u;
            tot += t;
        }
        // ---- records, in index order, written by the warp cooperatively: lane
        // j of a round writes the warp's record j (coalesced) and, for a
        // saddle, finds its upper-link components and their highest vertices
        const uint32_t excl = inc - cnt, cw = __shfl_sync(0xffffffffu, inc, 31);
        uint32_t np = 0;
        for (uint32_t base = 0; base < cw; base += 32) {
            const uint32_t j = base + lane;
            // owner: the last lane whose first record is at or before j
            uint32_t own = 0, own_excl = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, excl, own + st);
                if (e <= j) {
                    own += st;
                    own_excl = e;
                }
            }
            const uint32_t ocrit = __shfl_sync(0xffffffffu, crit, own);
            const uint32_t ovrow = __shfl_sync(0xffffffffu, vrow, own);
            const uint32_t ox = __shfl_sync(0xffffffffu, x, own);
            const uint32_t orr = __shfl_sync(0xffffffffu, rr, own);
            if (j < cw) {
                // vertex i of the owner: its (j - own_excl)-th critical vertex
                uint32_t k = j - own_excl, m = ocrit, i = 0;
                const uint32_t c4 = __popc(m & 15u);
                if (k >= c4) { i = 4; k -= c4; m >>= 4; }
                const uint32_t c2 = __popc(m & 3u);
                if (k >= c2) { i += 2; k -= c2; m >>= 2; }
                if (k >= (m & 1u)) i += 1;
                const uint32_t w = s_um[(uint32_t(warp) * 32u + own) * kVx + i];
                const uint32_t upper = w & 0x3fffu, sl = w >> 14;
                const float *orow = Cb + orr * rs;
                const uint64_t q = slot0 + pw + j;
                // (the record stays inside its brick's slot; the 14
                // neighbours lie within one row and one plane of the ring)
                const bool qok = chk(q, rec_cap(F), F.err) && chk(pw + j, F.bcap, F.err);
                const bool nok = chk_ptr(orow + dD - int(rs) + zm_col(int(ox + i) - 1), ring, 4 * uint64_t(G.rb), F.err) &&
                                 chk_ptr(orow + dU + int(rs) + zm_col(int(ox + i) + 1), ring, 4 * uint64_t(G.rb), F.err) &&
                                 chk_ptr(orow - int(rs), ring, 4 * uint64_t(G.rb), F.err) &&
                                 chk_ptr(orow + int(rs) + zm_col(int(ox + i) + 1), ring, 4 * uint64_t(G.rb), F.err);
                if (!qok || !nok) continue;
                F.rec_sid[q] = ovrow + i;
                F.rec_val[q] = orow[zm_col(int(ox + i))];
                uint64_t inf = 0;
                if (upper) {
                    const uint32_t cls = sl >> 4;
                    const uint32_t a2 = __ldg(lowc + upper);
                    float nb[14];
                    ring_nbrs(orow, int(ox + i), int(rs), dD, dU, nb);
                    inf = saddle_info<MIN>(nb, upper, int(sl & 15u), cls, a2, lowc);
                    np += uint32_t(inf >> 56);
                }
                F.rec_info[q] = inf;
            }
        }
        np = __reduce_add_sync(0xffffffffu, np);
        if (lane == 0 && np) atomicAdd(&s_cnt[2], np);
        if (tid == 0) s_cnt[1] = tot;  // critical vertices; maxima subtracted below
        prev_brick = brick;
    }
    __syncthreads();
    if (tid == 0 && prev_brick != 0xffffffffu)
        if (chk(prev_brick, F.nbricks, F.err)) F.bcnt[prev_brick] = make_uint4(s_cnt[0], s_cnt[1] - s_cnt[0], s_cnt[2], 0u);
    if (anynan) atomicOr(F.err, kErrNaN);
    // drain this item's outstanding (empty) copy groups before the ring is reused
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
}

cudaError_t prepare_classify_zm()
{
    // allow the opt-in maximum of dynamic shared memory, once per device
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (done_mask.load() & bit) return cudaSuccess;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    for (auto kern : {k_classify_zm<false>, k_classify_zm<true>}) {
        cudaFuncAttributes fa{};
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        const int dyn = optin - int(fa.sharedSizeBytes);
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
    }
    done_mask.fetch_or(bit);
    return cudaSuccess;
}

size_t zm_smem_bytes(uint32_t n0, uint32_t ty) { return size_t(4) * zm_ring_floats(n0, ty) * sizeof(float); }

cudaError_t launch_classify_zm(bool minimum, const FieldDev *fields, int nf, uint64_t total_items, size_t smem,
                               const uint32_t *lut, unsigned long long *ticket, int sm_count, int ctas_per_sm,
                               cudaStream_t st)
{
    if (total_items == 0) return cudaSuccess;
    auto kern = minimum ? k_classify_zm<true> : k_classify_zm<false>;
    cudaError_t e = prepare_classify_zm();
    if (e != cudaSuccess) return e;
    // (the row layout bounds the ring at 4 x (4 rows x 1032 + 16) floats = 66 KB)
    uint64_t grid = uint64_t(sm_count > 0 ? sm_count : 1) * uint64_t(ctas_per_sm > 0 ? ctas_per_sm : 3);
    if (grid > total_items) grid = total_items;
    kern<<<dim3(unsigned(grid)), kZmThreads, smem, st>>>(fields, nf, lut, total_items, ticket);
    return cudaGetLastError();
}

}  // namespace eg
