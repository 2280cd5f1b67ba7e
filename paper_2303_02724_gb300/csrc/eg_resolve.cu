// Step (b): every vertex gets the label of the maximum its gradient path
// reaches (Algorithm 2's inner loop, run for all vertices at once).
//
// lab[] holds the gradient pointers on entry and the labels on exit.  For
// fields with few maxima (long gradient paths) a tiled pass runs first (below):
// it labels every vertex whose path ends inside its tile and points every
// other vertex at the first vertex of its path outside the tile, so the walks
// here take one step for a labelled vertex and cross a tile per step for the
// others.  Each
// thread follows the pointers from its vertices to a fixed point (a maximum,
// lab[m] == m) and stores it; kIlp walks per thread advance in lock-step so
// their dependent loads overlap.  Threads write only their own vertices; a
// reader that meets an already-finished vertex sees its maximum instead of its
// gradient pointer, which lies on the same path, so the races are benign and
// later walks get shorter.  A walk longer than N steps is impossible (the
// order strictly increases along a path); the bound is a guard that reports
// kErrNotConverged instead of looping.
#include <algorithm>

#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kResolveThreads = 256;

// Resolve the labels of brick b of field F, kIlp walks in flight per thread.
template <int kIlp>
__device__ __forceinline__ void resolve_brick(const FieldDev &F, uint32_t b)
{
    if (F.wpp) return;  // warp-layout fields: resolved by k_resolve_cwalk
    uint64_t v0;
    uint32_t len;
    brick_range(F, b, v0, len);
    uint32_t *lab = F.lab;
    for (uint32_t base = threadIdx.x; base < len; base += kIlp * kResolveThreads) {
        uint32_t v[kIlp], u[kIlp];
        uint32_t live = 0;
#pragma unroll
        for (int q = 0; q < kIlp; q++) {
            const uint32_t i = base + q * kResolveThreads;
            v[q] = uint32_t(v0) + i;
            u[q] = v[q];
            if (i < len) {
                u[q] = lab[v[q]];
                if (u[q] != v[q]) live |= 1u << q;
            }
        }
        uint32_t moved = 0, steps = 0;
        while (live) {
#pragma unroll
            for (int q = 0; q < kIlp; q++)
                if ((live >> q) & 1u) {
                    const uint32_t w = lab[u[q]];
                    if (w == u[q]) {
                        live &= ~(1u << q);
                    } else {
                        u[q] = w;
                        moved |= 1u << q;
                    }
                }
            if (++steps > F.N) {
                atomicOr(F.err, kErrNotConverged);
                break;
            }
        }
#pragma unroll
        for (int q = 0; q < kIlp; q++)
            if ((moved >> q) & 1u) lab[v[q]] = u[q];
    }
}

template <int kIlp>
__global__ void __launch_bounds__(kResolveThreads)
k_resolve_chase(const FieldDev *__restrict__ fields, int nf)
{
    const uint64_t g = blockIdx.x;
    const int fi = find_field<false>(fields, nf, g);
    const FieldDev &F = fields[fi];
    resolve_brick<kIlp>(F, uint32_t(g - F.brick0));
}

// Single-field variant with the descriptor passed by value.
__global__ void __launch_bounds__(kResolveThreads)
k_resolve_one(const FieldDev F)
{
    resolve_brick<4>(F, blockIdx.x);
}

cudaError_t launch_resolve_one(const FieldDev &F, cudaStream_t st)
{
    if (F.nbricks == 0) return cudaSuccess;
    k_resolve_one<<<dim3(F.nbricks), kResolveThreads, 0, st>>>(F);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const FieldDev *fields, int nf, uint64_t total_bricks, int walks, cudaStream_t st)
{
    if (total_bricks == 0) return cudaSuccess;
    const dim3 grid = dim3(static_cast<unsigned>(total_bricks));
    if (walks <= 2) k_resolve_chase<2><<<grid, kResolveThreads, 0, st>>>(fields, nf);
    else if (walks <= 4) k_resolve_chase<4><<<grid, kResolveThreads, 0, st>>>(fields, nf);
    else k_resolve_chase<8><<<grid, kResolveThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tiled pass (fields run by the 3D kernels, only when maxima are rarer than 1
// in 100 vertices: long paths; otherwise the CTA returns and the brick walks
// do everything).
//
// One CTA takes a tile of TX x TY x TZ vertices (powers of two, kTileMax in
// all).  It reads the tile's gradient pointers once (coalesced rows) and keeps
// a 16-bit word per vertex in shared memory: the tile-local index of its
// gradient target, or, for a terminal (a maximum, or a vertex whose target lies
// outside the tile), its own index marked kDone (and kOut when it leaves).
// Pointer jumping (w <- word[w] until every word is marked kDone) gives every
// vertex its terminal in a few rounds.  A vertex ending on a maximum gets its
// label; any other gets its terminal's gradient target, the first vertex of
// its path outside the tile.
// ---------------------------------------------------------------------------
constexpr int kTileThreads = 256;
constexpr uint32_t kTileMax = 8192;
constexpr uint16_t kDone = 0x8000u, kOut = 0x4000u, kIdx = 0x3fffu;
constexpr int kTb = 8;  // elements per thread per pass (loads in flight)

void resolve_tile_shape(uint32_t n0, uint32_t n1, uint32_t n2, uint32_t rt[3], uint64_t *tiles)
{
    if (n2 > 1) {
        rt[0] = 5; rt[1] = 4; rt[2] = 4;  // 32 x 16 x 16
    } else if (n1 > 1) {
        rt[0] = 5; rt[1] = 8; rt[2] = 0;  // 32 x 256
    } else {
        rt[0] = 13; rt[1] = 0; rt[2] = 0;  // 8192
    }
    const uint64_t tx = (uint64_t(n0) + (1u << rt[0]) - 1) >> rt[0];
    const uint64_t ty = (uint64_t(n1) + (1u << rt[1]) - 1) >> rt[1];
    const uint64_t tz = (uint64_t(n2) + (1u << rt[2]) - 1) >> rt[2];
    *tiles = tx * ty * tz;
}

__global__ void __launch_bounds__(kTileThreads)
k_resolve_tile(const FieldDev *__restrict__ fields, int nf)
{
    __shared__ uint16_t s_w[kTileMax];
    const uint64_t g = blockIdx.x;
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fields[mid].rtile0 <= g) lo = mid;
        else hi = mid - 1;
    }
    const FieldDev &F = fields[lo];
    // dense maxima: short paths, the walks are faster on their own
    if (F.kd != 3 || uint64_t(F.totals[0]) * 100 >= uint64_t(F.N)) return;
    const uint32_t lx = F.rt[0], ly = F.rt[1], lz = F.rt[2];
    const uint32_t TX = 1u << lx, TY = 1u << ly, T = 1u << (lx + ly + lz);
    const uint32_t n0 = F.n[0], n1 = F.n[1], n2 = F.n[2];
    const uint32_t s1 = n0, s2 = n0 * n1;
    const uint32_t ntx = (n0 + TX - 1) >> lx, nty = (n1 + TY - 1) >> ly;
    uint32_t t = uint32_t(g - F.rtile0);
    const uint32_t tx = t % ntx;
    t /= ntx;
    const uint32_t tyi = t % nty, tz = t / nty;
    const uint32_t x0 = tx << lx, y0 = tyi << ly, z0 = tz << lz;
    const uint32_t ex = min(TX, n0 - x0), ey = min(TY, n1 - y0), ez = min(1u << lz, n2 - z0);
    uint32_t *lab = F.lab;
    auto inside = [&](uint32_t i) {
        return (i & (TX - 1)) < ex && ((i >> lx) & (TY - 1)) < ey && (i >> (lx + ly)) < ez;
    };
    auto gid = [&](uint32_t i) {
        return (z0 + (i >> (lx + ly))) * s2 + (y0 + ((i >> lx) & (TY - 1))) * s1 + x0 + (i & (TX - 1));
    };
    // gradient target of tile vertex i: its pointer, or decoded from its code
    auto target = [&](uint32_t i) {
        const uint32_t v = gid(i);
        if (!F.code) return lab[v];
        const uint32_t row = (z0 + (i >> (lx + ly))) * n1 + y0 + ((i >> lx) & (TY - 1)), x = x0 + (i & (TX - 1));
        const uint32_t c = (F.code[code_word(F.n0p, row, x)] >> ((x & 7u) * 4u)) & 15u;
        return c == kCodeMax ? v : slot_vertex<3>(v, int(c), F.s);
    };
    // 1: tile-local gradient targets (every thread runs the same trip counts)
    for (uint32_t i0 = 0; i0 < T; i0 += kTb * kTileThreads) {
        uint32_t a[kTb];
#pragma unroll
        for (int b = 0; b < kTb; b++) {
            const uint32_t i = i0 + b * kTileThreads + threadIdx.x;
            a[b] = inside(i) ? target(i) : 0u;
        }
#pragma unroll
        for (int b = 0; b < kTb; b++) {
            const uint32_t i = i0 + b * kTileThreads + threadIdx.x;
            uint16_t w = uint16_t(i) | kDone;  // a maximum, or outside the field
            if (inside(i)) {
                const uint32_t v = gid(i);
                if (a[b] != v) {
                    // a - v = +-(dz s2 + dy s1 + dx), d* in {0, 1}; axes of extent
                    // 1 never move, so peeling the largest stride first is exact
                    const uint32_t ix = i & (TX - 1), iy = (i >> lx) & (TY - 1), iz = i >> (lx + ly);
                    const bool neg = a[b] < v;
                    uint32_t d = neg ? v - a[b] : a[b] - v;
                    const uint32_t dz = d >= s2 ? 1u : 0u;
                    d -= dz * s2;
                    const uint32_t dy = d >= s1 ? 1u : 0u;
                    d -= dy * s1;
                    const int jx = neg ? int(ix) - int(d) : int(ix + d);
                    const int jy = neg ? int(iy) - int(dy) : int(iy + dy);
                    const int jz = neg ? int(iz) - int(dz) : int(iz + dz);
                    const bool in = jx >= 0 && jx < int(ex) && jy >= 0 && jy < int(ey) && jz >= 0 && jz < int(ez);
                    w = in ? uint16_t(uint32_t(jx) + (uint32_t(jy) << lx) + (uint32_t(jz) << (lx + ly)))
                           : uint16_t(uint16_t(i) | kDone | kOut);
                }
            }
            s_w[i] = w;
        }
    }
    __syncthreads();
    // 2: pointer jumping to the terminals (a path has fewer than T steps, so
    // at most log2(T) + 1 rounds change anything)
    for (int round = 0; round <= 14; round++) {
        int changed = 0;
        for (uint32_t i = threadIdx.x; i < T; i += kTileThreads) {
            const uint16_t w = s_w[i];
            if (!(w & kDone)) {
                s_w[i] = s_w[w & kIdx];
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    // 3: the label of every vertex that ends on a maximum; for the others the
    // first vertex outside the tile: their terminal's gradient target (with
    // pointers, terminals keep their entry; with codes every vertex is written)
    for (uint32_t i0 = 0; i0 < T; i0 += kTb * kTileThreads) {
#pragma unroll
        for (int b = 0; b < kTb; b++) {
            const uint32_t i = i0 + b * kTileThreads + threadIdx.x;
            const uint16_t w = s_w[i];
            if (!inside(i)) continue;
            if (F.code) lab[gid(i)] = (w & kOut) ? target(w & kIdx) : gid(w & kIdx);
            else if ((w & kIdx) != i) lab[gid(i)] = (w & kOut) ? lab[gid(w & kIdx)] : gid(w & kIdx);
        }
    }
}

// ---------------------------------------------------------------------------
// Resolution of code fields (gradients as 4-bit codes): one thread per group
// of 8 consecutive vertices of a row (the classifier's groups; one code word).
// Fields with dense maxima (short paths): the 8 gradient paths are followed
// through the codes in lock-step (the code array is 1/8 of the pointers', so
// it mostly stays in L2); a path still going after kWalkCap steps leaves its
// current vertex with kLabelExit set and goes on the exit list, which
// k_resolve_exits finishes.  Fields with few maxima (long paths) had the tiled
// pass first, which left a label or the first vertex outside its tile in
// every entry of lab[]: the walks follow lab[] to a fixed point.
// ---------------------------------------------------------------------------
constexpr int kWalkThreads = 256;
constexpr int kWalkCap = 64;

uint64_t walk_blocks(uint32_t n0, uint32_t n1, uint32_t n2)
{
    const uint64_t groups = uint64_t((n0 + 7) / 8) * n1 * n2;
    return (groups + kWalkThreads - 1) / kWalkThreads;
}

__global__ void __launch_bounds__(kWalkThreads)
k_resolve_cwalk(const FieldDev *__restrict__ fields, int nf, uint64_t *xlist, unsigned long long *xcount)
{
    __shared__ uint32_t s_coff[14], s_voff[14];
    const uint64_t g = blockIdx.x;
    int fi = 0;
    {
        int lo = 0, hi = nf - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (fields[mid].ctile0 <= g) lo = mid;
            else hi = mid - 1;
        }
        fi = lo;
    }
    const FieldDev &F = fields[fi];
    if (!F.wpp) return;
    const uint32_t n0 = F.n[0], n1 = F.n[1], n0p = F.n0p, gpr = (n0 + 7) / 8;
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 14) {
        const uint32_t p = Nbr<3>::pat(tid);
        const uint32_t co = (p & 1u) + ((p & 2u) ? n0p : 0u) + ((p & 4u) ? n0p * n1 : 0u);
        const uint32_t vo = (p & 1u) + ((p & 2u) ? n0 : 0u) + ((p & 4u) ? n0 * n1 : 0u);
        s_coff[tid] = Nbr<3>::neg(tid) ? 0u - co : co;
        s_voff[tid] = Nbr<3>::neg(tid) ? 0u - vo : vo;
    }
    __syncthreads();
    const uint64_t gi = (g - F.ctile0) * kWalkThreads + uint64_t(tid);
    const bool valid = gi < uint64_t(gpr) * n1 * F.n[2];
    const uint32_t row = valid ? uint32_t(gi / gpr) : 0u, x = valid ? 8u * uint32_t(gi - uint64_t(row) * gpr) : 0u;
    const uint32_t nv = valid ? min(8u, n0 - x) : 0u;
    const uint32_t vrow = row * n0 + x;
    uint32_t *lab = F.lab;
    uint32_t v[8];
    uint32_t live = 0;
    if (!F.code || uint64_t(F.totals[0]) * 100 < uint64_t(F.N)) {
        // gradient pointers, or after the tiled pass (labels or the first
        // vertex outside a tile): follow lab[] to a fixed point (a maximum)
#pragma unroll
        for (int i = 0; i < 8; i++) {
            v[i] = vrow + i;
            if (uint32_t(i) < nv) {
                const uint32_t u = lab[vrow + i];
                if (u != vrow + i) {
                    v[i] = u;
                    live |= 1u << i;
                }
            }
        }
        const uint32_t moved = live;
        uint32_t steps = 0;
        while (live) {
#pragma unroll
            for (int i = 0; i < 8; i++)
                if ((live >> i) & 1u) {
                    const uint32_t w = lab[v[i]];
                    if (w == v[i]) live &= ~(1u << i);
                    else v[i] = w;
                }
            if (++steps > F.N) {
                atomicOr(F.err, kErrNotConverged);
                break;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; i++)
            if ((moved >> i) & 1u) lab[vrow + i] = v[i];
        return;
    }
    // dense maxima: walk the codes, two walks in flight per lane; a slot whose
    // walk ends (a maximum, or the step cap) takes the lane's next vertex, so
    // the lane's time is the sum of its 8 walks, not 8 times the longest
    const uint32_t crow = row * n0p + x;
    const uint32_t w0 = valid ? F.code[crow >> 3] : 0xffffffffu;
    const uint32_t *code = F.code;
    uint32_t next = 0;
    uint32_t sj[2], sci[2], sv[2], sh[2];
    bool act[2];
    auto start = [&](int k) {
        act[k] = false;
        while (next < nv) {
            const uint32_t j = next++;
            const uint32_t c = (w0 >> (4 * j)) & 15u;
            if (c == kCodeMax) {
                lab[vrow + j] = vrow + j;  // a maximum labels itself
                continue;
            }
            sj[k] = j;
            sci[k] = crow + j + s_coff[c];
            sv[k] = vrow + j + s_voff[c];
            sh[k] = 1;
            act[k] = true;
            return;
        }
    };
    start(0);
    start(1);
    while (act[0] || act[1]) {
#pragma unroll
        for (int k = 0; k < 2; k++)
            if (act[k]) {
                const uint32_t c = (code[sci[k] >> 3] >> ((sci[k] & 7u) * 4u)) & 15u;
                if (c == kCodeMax) {
                    lab[vrow + sj[k]] = sv[k];
                    start(k);
                } else if (sh[k] >= kWalkCap) {
                    // still going: the current vertex lies on the path;
                    // k_resolve_exits continues from its entry
                    lab[vrow + sj[k]] = sv[k] | kLabelExit;
                    live |= 1u << sj[k];
                    start(k);
                } else {
                    sci[k] += s_coff[c];
                    sv[k] += s_voff[c];
                    sh[k]++;
                }
            }
    }
    // exit list (warp-aggregated)
    const uint32_t ne = __popc(live);
    uint32_t inc = ne;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
    if (tot == 0) return;
    unsigned long long b0 = 0;
    if (lane == 31) b0 = atomicAdd(xcount, (unsigned long long)tot);
    b0 = __shfl_sync(0xffffffffu, b0, 31) + (inc - ne);
    for (uint32_t m = live; m; m &= m - 1)
        xlist[b0++] = (uint64_t(uint32_t(fi)) << 32) | (vrow + uint32_t(__ffs(m) - 1));
}

// Vertices whose path left the neighbourhood of their tile: follow exits to a
// label (every vertex carries its label or an exit by now).  Concurrent
// threads may replace an exit by the label on the same path: either leads to
// the same maximum.
__global__ void __launch_bounds__(kWalkThreads)
k_resolve_exits(const FieldDev *__restrict__ fields, const uint64_t *xlist, const unsigned long long *xcount)
{
    const unsigned long long n = *xcount;
    for (unsigned long long i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t e = xlist[i];
        const FieldDev &F = fields[uint32_t(e >> 32)];
        const uint32_t v = uint32_t(e);
        uint32_t *lab = F.lab;
        const uint32_t first = lab[v] & ~kLabelExit;  // the first exit of v's path
        uint32_t w = lab[first];
        uint32_t steps = 0;
        while (w & kLabelExit) {
            w = lab[w & ~kLabelExit];
            if (++steps > F.N) {
                atomicOr(F.err, kErrNotConverged);
                break;
            }
        }
        w &= ~kLabelExit;
        lab[v] = w;
        if (steps) lab[first] = w;  // the first exit lies on the same path: later walks stop there
    }
}

cudaError_t launch_resolve_codes(const FieldDev *fields, int nf, uint64_t blocks, uint64_t *xlist,
                                 unsigned long long *xcount, int sm_count, cudaStream_t st)
{
    if (blocks == 0) return cudaSuccess;
    k_resolve_cwalk<<<dim3(static_cast<unsigned>(blocks)), kWalkThreads, 0, st>>>(fields, nf, xlist, xcount);
    k_resolve_exits<<<dim3(unsigned(std::max(sm_count, 1) * 8)), kWalkThreads, 0, st>>>(fields, xlist, xcount);
    return cudaGetLastError();
}

cudaError_t launch_resolve_tiles(const FieldDev *fields, int nf, uint64_t tiles, cudaStream_t st)
{
    if (tiles == 0) return cudaSuccess;
    k_resolve_tile<<<dim3(static_cast<unsigned>(tiles)), kTileThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
