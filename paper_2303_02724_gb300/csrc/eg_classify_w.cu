// Steps (a) + (c) for 2D and 3D float32 fields whose rows hold at most 2048
// vertices: warp-marching classification (Sec. 3.3, Table 1; 2D runs as 3D,
// n2 = 1).
//
// Every warp works on its own: it takes a work item (a run of 32 x 8
// consecutive vertices of one plane -- whole row pieces in index order -- and
// a range of planes) from a ticket counter and marches along the slowest axis
// through the planes.  Lane l owns 8 consecutive vertices of one row.  Per
// plane it reads the 7 row segments its vertices' 14-neighbourhoods touch
// (columns x-1 .. x+8 of rows y-1..y of the plane below, y-1..y+1 of its own
// plane and y..y+1 of the plane above) straight from global memory with
// 16-byte loads (the segments of neighbouring rows and planes are read again
// by the warps next to it and on the next plane, and come from L1/L2), the
// end columns from the neighbouring lanes by shuffle.  Out-of-domain values
// are NaN, which fails every ordered comparison, is skipped by min/max and
// equals nothing, so no bounds test is needed in the classification.  No
// shared-memory staging and no block-wide barrier: a warp's vertices of one
// plane are one brick (a contiguous range of ids), and its records are
// written in index order with warp shuffles alone.
//
// Per vertex:
//   upper   bit k set iff neighbour k is higher (value, then index: ties go to
//           the positive slots, which have larger indices); 14 set-compares
//           whose 0/1 results are accumulated with FMAs;
//   asc     the highest neighbour: the largest value (three-operand max), then
//           the highest slot rank holding it;
//   saddle  beta0+ >= 2, from a table of 2-bit classes indexed by the upper
//           mask (built on the host from the link graph).
// The gradient goes out as a 4-bit code (a pointer for fields of 2^31
// vertices or more).  Records of maxima and saddles: a saddle with two
// components gets its two representatives (UpperLinkRep, Sec. 3.4: the
// gradient slot, and the highest slot of the other component, whose values
// are read again from L1); a saddle with three or more is completed by
// k_saddle_multi.  The minimum graph mirrors every comparison and the tie
// rule.
#include <algorithm>
#include <atomic>

#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kWThreads = 256;
constexpr int kWWarps = kWThreads / 32;
constexpr int kVx = 8;  // vertices per lane along axis 0
constexpr unsigned kFull = 0xffffffffu;

// Record info of a saddle with three or more upper-link components, left for
// k_saddle_multi: bit 63, the gradient slot in bits 16..19, the upper mask in
// bits 0..13 (a real info word never has bit 63 set).
constexpr uint64_t kInfoPending = 1ull << 63;

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

// Neighbour slot k (slot order of Nbr<3>) as a signed step per axis.
__device__ __forceinline__ void slot_step(int k, int &dx, int &dy, int &dz)
{
    const uint32_t p = Nbr<3>::pat(k);
    const int sg = Nbr<3>::neg(k) ? -1 : 1;
    dx = sg * int(p & 1u);
    dy = sg * int((p >> 1) & 1u);
    dz = sg * int((p >> 2) & 1u);
}

// Info word of a saddle with three or more upper-link components, from its 14
// neighbour values read from the field (NaN outside the domain).
template <bool MIN>
__device__ __forceinline__ uint64_t multi_info(const FieldDev &F, uint32_t v, uint64_t pending, const uint16_t *lowc)
{
    const uint32_t n0 = F.n[0], n1 = F.n[1], n2 = F.n[2];
    const uint32_t x = v % n0, t = v / n0, y = t % n1, z = t / n1;
    float nb[14];
#pragma unroll
    for (int k = 0; k < 14; k++) {
        int dx, dy, dz;
        slot_step(k, dx, dy, dz);
        const int xx = int(x) + dx, yy = int(y) + dy, zz = int(z) + dz;
        const bool in = xx >= 0 && xx < int(n0) && yy >= 0 && yy < int(n1) && zz >= 0 && zz < int(n2);
        nb[k] = in ? F.f[(uint64_t(uint32_t(zz)) * n1 + uint32_t(yy)) * n0 + uint32_t(xx)] : __int_as_float(0x7fc00000);
    }
    const uint32_t upper = uint32_t(pending & 0x3fffu);
    return saddle_info<MIN>(nb, upper, int((pending >> 16) & 15u), 2u, __ldg(lowc + upper), lowc);
}

// The warp's view of one field.
struct WGeom {
    const float *f;
    uint32_t n0, n1, n2;
    bool vec;  // rows start on 16-byte boundaries (n0 % 4 == 0, aligned field)
};

__device__ __forceinline__ void cp_async16(float *smem, const float *gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem)
{
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Per-warp staging of one plane: three row tracks (rows y-1, y, y+1 of every
// lane), each 32 lanes x 8 values plus the two end columns of the warp (x-1 of
// lane 0, x+8 of lane 31).  A lane's two 16-byte halves are stored swapped
// when bit 2 of the lane is set, so the eight lanes of a quarter-warp read
// distinct banks.
constexpr int kTrack = 32 * kVx + 4;  // (the two end columns, padded to 16 bytes)
constexpr int kSlot = 3 * kTrack;

__device__ __forceinline__ int half_pos(int lane, int i) { return ((i & 4) ^ (((lane >> 2) & 1) << 2)) | (i & 3); }

// Copy rows y-1, y, y+1 of plane zz into a slot (NaN outside the field);
// always commits one group of asynchronous copies.
__device__ __forceinline__ void stage_plane(const WGeom &G, float *slot, bool valid, int y, int zz, uint32_t x,
                                            bool first_t, bool last_t, int lane)
{
    const float qnan = __int_as_float(0x7fc00000);
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const int yy = y - 1 + t;
        float *dst = slot + t * kTrack;
        float *mine = dst + lane * kVx;
        const bool in = valid && yy >= 0 && yy < int(G.n1) && zz >= 0 && zz < int(G.n2);
        const float *row = G.f + (in ? (uint64_t(uint32_t(zz)) * G.n1 + uint32_t(yy)) * G.n0 : 0ull);
        if (in && G.vec && x + kVx <= G.n0) {
            const int h = ((lane >> 2) & 1) << 2;
            cp_async16(mine + h, row + x);
            cp_async16(mine + (h ^ 4), row + x + 4);
        } else {
#pragma unroll
            for (int i = 0; i < kVx; i++) {
                if (in && x + i < G.n0) cp_async4(mine + half_pos(lane, i), row + x + i);
                else mine[half_pos(lane, i)] = qnan;
            }
        }
        if (lane == 0) {
            if (in && !first_t) cp_async4(dst + 32 * kVx, row + x - 1);
            else dst[32 * kVx] = qnan;
        }
        if (lane == 31) {
            if (in && !last_t) cp_async4(dst + 32 * kVx + 1, row + x + kVx);
            else dst[32 * kVx + 1] = qnan;
        }
    }
    cp_async_commit();
}

// Columns x-1 .. x+8 of one staged row track (end columns from the
// neighbouring lanes, or the warp's end columns).
__device__ __forceinline__ void read_row(const float *src, int lane, bool first_t, bool last_t, float (&v)[10])
{
    const float qnan = __int_as_float(0x7fc00000);
    const int h = ((lane >> 2) & 1) << 2;
    const float4 a = *reinterpret_cast<const float4 *>(src + lane * kVx + h);
    const float4 b = *reinterpret_cast<const float4 *>(src + lane * kVx + (h ^ 4));
    v[1] = a.x; v[2] = a.y; v[3] = a.z; v[4] = a.w;
    v[5] = b.x; v[6] = b.y; v[7] = b.z; v[8] = b.w;
    float l = __shfl_up_sync(kFull, v[8], 1);
    float r = __shfl_down_sync(kFull, v[1], 1);
    if (lane == 0) l = src[32 * kVx];
    if (lane == 31) r = src[32 * kVx + 1];
    v[0] = first_t ? qnan : l;
    v[9] = last_t ? qnan : r;
}

__device__ __forceinline__ int warp_slot_base(int warp) { return warp * 3 * kSlot; }
constexpr size_t kWSmemDyn = size_t(kWWarps) * 3 * kSlot * sizeof(float);

template <bool MIN>
__global__ void __launch_bounds__(kWThreads, 2)
k_classify_w(const FieldDev *__restrict__ fields, int nf, const uint32_t *__restrict__ lut, uint64_t total_items,
             unsigned long long *ticket, int fbase, uint64_t *mlist, unsigned long long *mcount, uint64_t mcap)
{
    __shared__ uint32_t s_lut[1024];
    // per warp: the classification word of every vertex of the current plane
    // (upper mask | gradient slot << 14 | class << 18), lane-major, and the
    // 14 neighbour offsets of the current field
    __shared__ __align__(16) uint32_t s_um[kWWarps][32 * kVx];
    __shared__ uint32_t s_off[kWWarps][14];
    // per warp: planes z-1, z, z+1 staged (slot = plane mod 3)
    extern __shared__ __align__(16) float w_smem[];
    float *stage = w_smem + warp_slot_base(threadIdx.x >> 5);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint16_t *lowc = reinterpret_cast<const uint16_t *>(lut + 1024);
    for (int i = tid; i < 1024; i += kWThreads) s_lut[i] = __ldg(lut + i);
    __syncthreads();
    while (true) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(ticket, 1ull);
        g = __shfl_sync(kFull, g, 0);
        if (g >= total_items) break;
        const int fi = find_field<true>(fields, nf, g);
        const FieldDev &F = fields[fi];
        const uint32_t item = uint32_t(g - F.item0);
        const uint32_t wpp = F.wpp, gpr = F.gpr;
        const uint32_t w = item % wpp, zci = item / wpp;
        WGeom G;
        G.f = F.f;
        G.n0 = F.n[0];
        G.n1 = F.n[1];
        G.n2 = F.n[2];
        G.vec = F.vec != 0;
        const int zs = int(zci * F.zc), ze = int(min(G.n2, zci * F.zc + F.zc));
        if (lane < 14) {
            const uint32_t p = Nbr<3>::pat(lane);
            const uint32_t mag = ((p & 1u) ? 1u : 0u) + ((p & 2u) ? G.n0 : 0u) + ((p & 4u) ? G.n0 * G.n1 : 0u);
            s_off[warp][lane] = Nbr<3>::neg(lane) ? 0u - mag : mag;
        }
        __syncwarp();
        // this lane's 8 vertices: group gi of the plane's row-major groups
        const uint32_t gi = 32u * w + uint32_t(lane);
        const bool valid = gi < G.n1 * gpr;
        const uint32_t y = valid ? gi / gpr : 0u, xg = valid ? gi - y * gpr : 0u, x = kVx * xg;
        const bool first_t = xg == 0, last_t = !valid || xg + 1 == gpr;
        bool anynan = false;
        auto slot_of = [&](int p) { return stage + ((p + 3) % 3) * kSlot; };
        stage_plane(G, slot_of(zs - 1), valid, int(y), zs - 1, x, first_t, last_t, lane);
        stage_plane(G, slot_of(zs), valid, int(y), zs, x, first_t, last_t, lane);
        stage_plane(G, slot_of(zs + 1), valid, int(y), zs + 1, x, first_t, last_t, lane);

        for (int z = zs; z < ze; z++) {
            const uint32_t brick = uint32_t(z) * wpp + w;
            const uint32_t vrow = uint32_t((uint64_t(uint32_t(z)) * G.n1 + y) * G.n0) + x;
            // rows: A = y-1, B = y, C = y+1; D = plane z-1, C = plane z, U = plane z+1
            float DA[10], DB[10], CA[10], CB[10], CC[10], UB[10], UC[10];
            cp_async_wait0();  // plane z+1 (the last one staged) has landed
            __syncwarp();
            {
                const float *Ds = slot_of(z - 1), *Cs = slot_of(z), *Us = slot_of(z + 1);
                read_row(Ds, lane, first_t, last_t, DA);
                read_row(Ds + kTrack, lane, first_t, last_t, DB);
                read_row(Cs, lane, first_t, last_t, CA);
                read_row(Cs + kTrack, lane, first_t, last_t, CB);
                read_row(Cs + 2 * kTrack, lane, first_t, last_t, CC);
                read_row(Us + kTrack, lane, first_t, last_t, UB);
                read_row(Us + 2 * kTrack, lane, first_t, last_t, UC);
            }
            __syncwarp();  // every lane has read plane z-1's slot: plane z+2 may replace it
            if (z + 1 < ze) stage_plane(G, slot_of(z + 2), valid, int(y), z + 2, x, first_t, last_t, lane);
            uint32_t um[kVx];
            uint32_t crit = 0, nm = 0, code = 0;
#pragma unroll
            for (int i = 0; i < kVx; i++) {
                const float c = CB[i + 1];
                // slot order: (-1,-1,-1) (0,-1,-1) (-1,0,-1) (0,0,-1) (-1,-1,0) (0,-1,0)
                // (-1,0,0) | (1,0,0) (0,1,0) (1,1,0) (0,0,1) (1,0,1) (0,1,1) (1,1,1)
                const float nb[14] = {DA[i], DA[i + 1], DB[i], DB[i + 1], CA[i], CA[i + 1], CB[i],
                                      CB[i + 2], CC[i + 1], CC[i + 2], UB[i + 1], UB[i + 2], UC[i + 1], UC[i + 2]};
                // upper: negative slots (smaller index) need a strictly higher
                // value, positive slots a higher or equal one (maximum graph);
                // the minimum graph mirrors both.  Each test yields 0.0 or 1.0
                // and is accumulated as bit k of a float whose exponent pins the
                // integer part (2^23 + mask is exact), on the FMA pipe.
                float au = 8388608.f;
#pragma unroll
                for (int k = 0; k < 14; k++) {
                    const float t = MIN ? (k < 7 ? set_le(nb[k], c) : set_lt(nb[k], c))
                                        : (k < 7 ? set_gt(nb[k], c) : set_ge(nb[k], c));
                    au = __fmaf_rn(t, float(1u << k), au);
                }
                const uint32_t upper = __float_as_uint(au) & 0x3fffu;
                // gradient: the extreme neighbour value, then the highest
                // (maximum graph) or lowest (minimum graph) slot holding it
                // among the upper neighbours
                const float m = MIN ? min7x2(nb) : max7x2(nb);
                float ae = 8388608.f;
#pragma unroll
                for (int k = 0; k < 14; k++) ae = __fmaf_rn(set_eq(nb[k], m), float(1u << k), ae);
                const uint32_t eq = __float_as_uint(ae) & 0x3fffu;
                const bool ok = valid && x + i < G.n0;
                uint32_t cls = 0, slot = 0;
                bool cv;
                if (upper) {
                    uint32_t cand = eq & upper;
                    cand = cand ? cand : upper;  // (never empty; keeps the slot in range)
                    slot = MIN ? uint32_t(__ffs(cand) - 1) : uint32_t(31 - __clz(cand));
                    cls = (s_lut[upper >> 4] >> ((upper & 15) << 1)) & 3u;
                    cv = cls != 0;
                } else {
                    cv = true;
                    nm += ok ? 1u : 0u;
                    anynan |= ok && (c != c);  // a NaN value has no upper neighbour
                }
                um[i] = upper | (slot << 14) | (cls << 18);
                code |= (ok && upper ? slot : kCodeMax) << (4 * i);
                if (ok) crit |= cv ? (1u << i) : 0u;
            }
            if (valid) {
                if (F.code) {
                    F.code[code_word(F.n0p, uint64_t(uint32_t(z)) * G.n1 + y, x)] = code;
                } else {
                    uint32_t a[kVx];
#pragma unroll
                    for (int i = 0; i < kVx; i++)
                        a[i] = (um[i] & 0x3fffu) ? vrow + i + s_off[warp][(um[i] >> 14) & 15u] : vrow + i;
                    if (G.vec && x + kVx <= G.n0) {  // (vrow is a multiple of 4 then)
                        uint4 *dst = reinterpret_cast<uint4 *>(F.lab + vrow);
                        dst[0] = make_uint4(a[0], a[1], a[2], a[3]);
                        dst[1] = make_uint4(a[4], a[5], a[6], a[7]);
                    } else {
#pragma unroll
                        for (int i = 0; i < kVx; i++)
                            if (x + i < G.n0) F.lab[vrow + i] = a[i];
                    }
                }
            }
            uint4 *um4 = reinterpret_cast<uint4 *>(&s_um[warp][lane * kVx]);
            um4[0] = make_uint4(um[0], um[1], um[2], um[3]);
            um4[1] = make_uint4(um[4], um[5], um[6], um[7]);
            __syncwarp();
            // ---- records in index order: lanes are in index order
            const uint32_t cnt = __popc(crit);
            uint32_t inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t excl = inc - cnt, cw = __shfl_sync(kFull, inc, 31);
            nm = __reduce_add_sync(kFull, nm);
            const uint64_t slot0 = uint64_t(brick) * F.bcap;
            uint32_t np = 0;
            for (uint32_t base = 0; base < cw; base += 32) {
                const uint32_t j = base + lane;
                // owner: the last lane whose first record is at or before j
                uint32_t own = 0, own_excl = 0;
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const uint32_t e = __shfl_sync(kFull, excl, own + st);
                    if (e <= j) {
                        own += st;
                        own_excl = e;
                    }
                }
                const uint32_t ocrit = __shfl_sync(kFull, crit, own);
                const uint32_t ovrow = __shfl_sync(kFull, vrow, own);
                bool pend = false;
                uint64_t q = 0;
                if (j < cw) {
                    // vertex i of the owner: its (j - own_excl)-th critical vertex
                    uint32_t k = j - own_excl, mk = ocrit, i = 0;
                    const uint32_t c4 = __popc(mk & 15u);
                    if (k >= c4) { i = 4; k -= c4; mk >>= 4; }
                    const uint32_t c2 = __popc(mk & 3u);
                    if (k >= c2) { i += 2; k -= c2; mk >>= 2; }
                    if (k >= (mk & 1u)) i += 1;
                    const uint32_t wd = s_um[warp][own * kVx + i];
                    const uint32_t upper = wd & 0x3fffu, sl = wd >> 14;
                    const uint32_t v = ovrow + i;
                    q = slot0 + j;
                    F.rec_sid[q] = v;
                    F.rec_val[q] = __ldg(G.f + v);
                    uint64_t inf = 0;
                    if (upper) {
                        const uint32_t cls = sl >> 4;
                        const int first = int(sl & 15u);
                        if (cls == 1) {
                            // two components: the gradient's, represented by
                            // the gradient slot, and the other one (the
                            // component of the mask's lowest set bit, or the
                            // rest), whose highest vertex is found among its
                            // own slots (upper neighbours exist: no bounds test)
                            const uint32_t a2 = __ldg(lowc + upper);
                            uint32_t other = ((a2 >> first) & 1u) ? (upper ^ a2) : a2;
                            float best = 0.f;
                            int rk = -1;
                            while (other) {
                                const int kk = __ffs(other) - 1;
                                other &= other - 1;
                                const float val = __ldg(G.f + (v + s_off[warp][kk]));
                                if (rk < 0 || (MIN ? val < best : val >= best)) {
                                    best = val;
                                    rk = kk;
                                }
                            }
                            inf = (2ull << 56) | uint64_t(first) | (uint64_t(rk) << 5);
                            np += 2;
                        } else {
                            // three or more (rare): completed by k_saddle_multi,
                            // which also adds their paths to the brick's count
                            inf = kInfoPending | (uint64_t(first) << 16) | upper;
                            pend = true;
                        }
                    }
                    F.rec_info[q] = inf;
                }
                // pending records onto the list (warp-aggregated); if it is
                // full, the record is completed here from the field
                const unsigned pm = __ballot_sync(kFull, pend);
                if (pm) {
                    unsigned long long at = 0;
                    if (lane == __ffs(pm) - 1) at = atomicAdd(mcount, (unsigned long long)__popc(pm));
                    at = __shfl_sync(kFull, at, __ffs(pm) - 1) + __popc(pm & ((1u << lane) - 1u));
                    if (pend) {
                        if (at < mcap) {
                            mlist[at] = (uint64_t(fbase + fi) << 40) | q;
                        } else {
                            const uint64_t inf = multi_info<MIN>(F, F.rec_sid[q], F.rec_info[q], lowc);
                            F.rec_info[q] = inf;
                            np += uint32_t(inf >> 56);
                        }
                    }
                }
            }
            np = __reduce_add_sync(kFull, np);
            if (lane == 0) F.bcnt[brick] = make_uint4(nm, cw - nm, np, 0u);
            __syncwarp();  // s_um is rewritten on the next plane
        }
        if (__any_sync(kFull, anynan) && lane == 0) atomicOr(F.err, kErrNaN);
        cp_async_wait0();  // nothing in flight into the staging slots
        __syncwarp();
    }
}

// Saddles with three or more upper-link components left pending by the
// classifier (the list holds field << 40 | record slot): their record info
// (components and their highest vertices, Sec. 3.4), and their paths added
// to their brick's count, before scan A.
__global__ void __launch_bounds__(256)
k_saddle_multi(const FieldDev *__restrict__ fields, const uint64_t *mlist, const unsigned long long *mcount,
               uint64_t mcap, const uint32_t *__restrict__ lut)
{
    const uint16_t *lowc = reinterpret_cast<const uint16_t *>(lut + 1024);
    unsigned long long n = *mcount;
    if (n > mcap) n = mcap;
    for (unsigned long long i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t e = mlist[i];
        const FieldDev &F = fields[uint32_t(e >> 40)];
        const uint64_t q = e & ((1ull << 40) - 1);
        const uint64_t inf = (F.flags & kFlagMinimum) ? multi_info<true>(F, F.rec_sid[q], F.rec_info[q], lowc)
                                                      : multi_info<false>(F, F.rec_sid[q], F.rec_info[q], lowc);
        F.rec_info[q] = inf;
        atomicAdd(&F.bcnt[q / F.bcap].z, uint32_t(inf >> 56));
    }
}

cudaError_t launch_saddle_multi(const FieldDev *fields, const uint64_t *mlist, const unsigned long long *mcount,
                                uint64_t mcap, const uint32_t *lut, int sm_count, cudaStream_t st)
{
    const dim3 grid = dim3(unsigned(std::max(sm_count, 1) * 2));
    k_saddle_multi<<<grid, 256, 0, st>>>(fields, mlist, mcount, mcap, lut);
    return cudaGetLastError();
}

cudaError_t prepare_classify_w()
{
    // the staging slots take more than the default 48 KB: raise the limit,
    // once per device
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (done_mask.load() & bit) return cudaSuccess;
    for (auto kern : {k_classify_w<false>, k_classify_w<true>})
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kWSmemDyn))) !=
            cudaSuccess)
            return e;
    done_mask.fetch_or(bit);
    return cudaSuccess;
}

cudaError_t launch_classify_w(bool minimum, const FieldDev *fields, int nf, uint64_t total_items, const uint32_t *lut,
                              unsigned long long *ticket, int sm_count, int ctas_per_sm, int fbase, uint64_t *mlist,
                              unsigned long long *mcount, uint64_t mcap, cudaStream_t st)
{
    if (total_items == 0) return cudaSuccess;
    auto kern = minimum ? k_classify_w<true> : k_classify_w<false>;
    // persistent: enough CTAs for every SM (or one warp per item, if fewer)
    uint64_t grid = uint64_t(sm_count > 0 ? sm_count : 1) * uint64_t(ctas_per_sm > 0 ? ctas_per_sm : 2);
    const uint64_t need = (total_items + kWWarps - 1) / kWWarps;
    if (grid > need) grid = need;
    cudaError_t e = prepare_classify_w();
    if (e != cudaSuccess) return e;
    kern<<<dim3(unsigned(grid)), kWThreads, kWSmemDyn, st>>>(fields, nf, lut, total_items, ticket, fbase, mlist,
                                                           mcount, mcap);
    return cudaGetLastError();
}

}  // namespace eg
