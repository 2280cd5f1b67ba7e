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
    if (F.code) return;  // resolved by the code tiles (below)
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
    // dense maxima: short paths, the brick walks are faster on their own
    if (F.kd != 3 || F.code || uint64_t(F.totals[0]) * 100 >= uint64_t(F.N)) return;
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
    // 1: tile-local gradient targets (every thread runs the same trip counts)
    for (uint32_t i0 = 0; i0 < T; i0 += kTb * kTileThreads) {
        uint32_t a[kTb];
#pragma unroll
        for (int b = 0; b < kTb; b++) {
            const uint32_t i = i0 + b * kTileThreads + threadIdx.x;
            a[b] = inside(i) ? lab[gid(i)] : 0u;
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
    // first vertex outside the tile: their terminal's gradient target, still
    // in lab[] (terminals keep their entry)
    for (uint32_t i0 = 0; i0 < T; i0 += kTb * kTileThreads) {
#pragma unroll
        for (int b = 0; b < kTb; b++) {
            const uint32_t i = i0 + b * kTileThreads + threadIdx.x;
            const uint16_t w = s_w[i];
            if (inside(i) && (w & kIdx) != i) lab[gid(i)] = (w & kOut) ? lab[gid(w & kIdx)] : gid(w & kIdx);
        }
    }
}

// ---------------------------------------------------------------------------
// Resolution from gradient codes (fields classified by the plane-marching
// kernel): one CTA per tile of 32 x 16 x 16 vertices (32 x 256 in 2D).  The
// CTA copies the 4-bit codes of the tile and of a halo of kCodeHalo vertices
// on every side into shared memory, one byte per vertex; cells outside the
// field and the outermost layer of the halo are marked kShell.  Every vertex
// of the tile then follows its gradient path through shared memory: a path
// that reaches a maximum gives the label; a path that reaches the shell leaves
// the tile's neighbourhood, and the vertex gets that shell vertex with
// kLabelExit set and goes on the exit list.  Paths are short on most fields,
// so the halo keeps most of them inside; k_resolve_exits follows the rest,
// from exit to exit (each crossing at least kCodeHalo + 1 steps), to a label.
// ---------------------------------------------------------------------------
constexpr int kCodeThreads = 256;
constexpr int kCodeHalo = 4;
constexpr int kCodeIlp = 4;
constexpr uint8_t kShell = 0xff;
constexpr uint32_t kCodeSmem3 = (32 + 2 * kCodeHalo) * (16 + 2 * kCodeHalo) * (16 + 2 * kCodeHalo);
constexpr uint32_t kCodeSmem2 = (32 + 2 * kCodeHalo) * (256 + 2 * kCodeHalo);
constexpr uint32_t kCodeSmem = kCodeSmem3 > kCodeSmem2 ? kCodeSmem3 : kCodeSmem2;

// log2 of the core tile extents of a code field
__host__ __device__ __forceinline__ void code_tile_shape(uint32_t n2, uint32_t &lx, uint32_t &ly, uint32_t &lz)
{
    lx = 5;
    if (n2 > 1) {
        ly = 4;
        lz = 4;
    } else {
        ly = 8;
        lz = 0;
    }
}

uint64_t code_tiles(uint32_t n0, uint32_t n1, uint32_t n2)
{
    uint32_t lx, ly, lz;
    code_tile_shape(n2, lx, ly, lz);
    return ((uint64_t(n0) + (1u << lx) - 1) >> lx) * ((uint64_t(n1) + (1u << ly) - 1) >> ly) *
           ((uint64_t(n2) + (1u << lz) - 1) >> lz);
}

__global__ void __launch_bounds__(kCodeThreads)
k_resolve_codes(const FieldDev *__restrict__ fields, int nf, uint64_t *xlist, unsigned long long *xcount)
{
    __shared__ uint8_t s_c[kCodeSmem];
    __shared__ int32_t s_loff[14];
    __shared__ uint32_t s_goff[14];
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
    if (!F.code) return;
    uint32_t lx, ly, lz;
    code_tile_shape(F.n[2], lx, ly, lz);
    const uint32_t n0 = F.n[0], n1 = F.n[1], n2 = F.n[2];
    const int H = kCodeHalo;
    const int HZ = n2 > 1 ? kCodeHalo : 0;
    const int EX = (1 << lx) + 2 * H, EY = (1 << ly) + 2 * H, EZ = (1 << lz) + 2 * HZ;
    const uint32_t ntx = (n0 + (1u << lx) - 1) >> lx, nty = (n1 + (1u << ly) - 1) >> ly;
    uint32_t t = uint32_t(g - F.ctile0);
    const uint32_t tx = t % ntx;
    t /= ntx;
    const uint32_t tyi = t % nty, tz = t / nty;
    const int x0 = int(tx << lx), y0 = int(tyi << ly), z0 = int(tz << lz);
    const int tid = threadIdx.x;
    if (tid < 14) {
        const uint32_t p = Nbr<3>::pat(tid);
        const int lo = int(p & 1u) + EX * int((p >> 1) & 1u) + EX * EY * int((p >> 2) & 1u);
        const uint32_t go = (p & 1u) + ((p & 2u) ? F.s[1] : 0u) + ((p & 4u) ? F.s[2] : 0u);
        s_loff[tid] = Nbr<3>::neg(tid) ? -lo : lo;
        s_goff[tid] = Nbr<3>::neg(tid) ? 0u - go : go;
    }
    // 1: codes of the tile and its halo, one byte per cell (each extended row
    // spans the 6 code words from x0 - 8 to x0 + 40)
    const int nrows = EY * EZ;
    const int wpr = ((1 << lx) + 16) / 8;  // words per extended row
    const int xw0 = (x0 - 8) >> 3;          // first word (may be -1)
    for (int i = tid; i < nrows * wpr; i += kCodeThreads) {
        const int row = i / wpr, wi = i - row * wpr;
        const int ry = row % EY, rz = row / EY;
        const int gy = y0 - H + ry, gz = z0 - HZ + rz;
        const int w = xw0 + wi;
        const bool rowin = gy >= 0 && gy < int(n1) && gz >= 0 && gz < int(n2);
        const bool win = rowin && w >= 0 && w < int(F.n0p >> 3);
        const uint32_t word = win ? F.code[(uint64_t(uint32_t(gz)) * n1 + uint32_t(gy)) * (F.n0p >> 3) + uint32_t(w)] : 0u;
        const bool edge_yz = ry == 0 || ry == EY - 1 || (HZ && (rz == 0 || rz == EZ - 1));
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int gx = 8 * w + j, ux = gx - (x0 - H);
            if (ux < 0 || ux >= EX) continue;
            const bool in = win && gx < int(n0);
            const bool shell = !in || edge_yz || ux == 0 || ux == EX - 1;
            s_c[(rz * EY + ry) * EX + ux] = shell ? kShell : uint8_t((word >> (4 * j)) & 15u);
        }
    }
    __syncthreads();
    // 2: walks from every vertex of the tile (kCodeIlp in lock-step)
    const uint32_t T = 1u << (lx + ly + lz);
    const uint32_t s1 = F.s[1], s2 = F.s[2];
    uint32_t *lab = F.lab;
    const int lane = tid & 31;
    for (uint32_t base = 0; base < T; base += kCodeIlp * kCodeThreads) {
        int u[kCodeIlp];
        uint32_t gv[kCodeIlp], gu[kCodeIlp];
        uint32_t live = 0, inmask = 0;
#pragma unroll
        for (int q = 0; q < kCodeIlp; q++) {
            const uint32_t i = base + uint32_t(q * kCodeThreads + tid);
            const uint32_t cx = i & ((1u << lx) - 1), cy = (i >> lx) & ((1u << ly) - 1), cz = i >> (lx + ly);
            const uint32_t gx = uint32_t(x0) + cx, gy = uint32_t(y0) + cy, gz = uint32_t(z0) + cz;
            u[q] = int(cx + H) + EX * (int(cy + H) + EY * int(cz + HZ));
            gv[q] = gx + gy * s1 + gz * s2;
            gu[q] = gv[q];
            if (i < T && gx < n0 && gy < n1 && gz < n2) {
                inmask |= 1u << q;
                live |= 1u << q;
            }
        }
        uint32_t exits = 0, steps = 0;
        while (live) {
#pragma unroll
            for (int q = 0; q < kCodeIlp; q++)
                if ((live >> q) & 1u) {
                    const uint32_t c = s_c[u[q]];
                    if (c == kCodeMax) {
                        live &= ~(1u << q);
                    } else if (c == kShell) {
                        live &= ~(1u << q);
                        exits |= 1u << q;
                    } else {
                        u[q] += s_loff[c];
                        gu[q] += s_goff[c];
                    }
                }
            if (++steps > uint32_t(EX * EY * EZ)) {  // a path visits each cell once
                atomicOr(F.err, kErrNotConverged);
                break;
            }
        }
#pragma unroll
        for (int q = 0; q < kCodeIlp; q++) {
            const bool ex = (exits >> q) & 1u;
            if ((inmask >> q) & 1u) lab[gv[q]] = ex ? (gu[q] | kLabelExit) : gu[q];
            // exit list: warp-aggregated append
            const unsigned m = __ballot_sync(0xffffffffu, ex);
            if (m) {
                unsigned long long b0 = 0;
                if (lane == __ffs(m) - 1) b0 = atomicAdd(xcount, (unsigned long long)__popc(m));
                b0 = __shfl_sync(0xffffffffu, b0, __ffs(m) - 1);
                if (ex) xlist[b0 + __popc(m & ((1u << lane) - 1u))] = (uint64_t(uint32_t(fi)) << 32) | gv[q];
            }
        }
    }
}

// Vertices whose path left the neighbourhood of their tile: follow exits to a
// label (every vertex carries its label or an exit by now).  Concurrent
// threads may replace an exit by the label on the same path: either leads to
// the same maximum.
__global__ void __launch_bounds__(kCodeThreads)
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

cudaError_t launch_resolve_codes(const FieldDev *fields, int nf, uint64_t tiles, uint64_t *xlist,
                                 unsigned long long *xcount, int sm_count, cudaStream_t st)
{
    if (tiles == 0) return cudaSuccess;
    k_resolve_codes<<<dim3(static_cast<unsigned>(tiles)), kCodeThreads, 0, st>>>(fields, nf, xlist, xcount);
    k_resolve_exits<<<dim3(unsigned(std::max(sm_count, 1) * 8)), kCodeThreads, 0, st>>>(fields, xlist, xcount);
    return cudaGetLastError();
}

cudaError_t launch_resolve_tiles(const FieldDev *fields, int nf, uint64_t tiles, cudaStream_t st)
{
    if (tiles == 0) return cudaSuccess;
    k_resolve_tile<<<dim3(static_cast<unsigned>(tiles)), kTileThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
