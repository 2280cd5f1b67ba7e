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
#include "eg_internal.cuh"
#include "eg_kernels.h"

namespace eg {

constexpr int kResolveThreads = 256;

// Resolve the labels of brick b of field F, kIlp walks in flight per thread.
template <int kIlp>
__device__ __forceinline__ void resolve_brick(const FieldDev &F, uint32_t b)
{
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
            if (i < len && chk(v[q], F.N, F.err)) {
                u[q] = lab[v[q]];
                if (u[q] != v[q]) live |= 1u << q;
            }
        }
        uint32_t moved = 0, steps = 0;
        while (live) {
#pragma unroll
            for (int q = 0; q < kIlp; q++)
                if ((live >> q) & 1u) {
                    if (!chk(u[q], F.N, F.err)) {
                        live &= ~(1u << q);
                        moved &= ~(1u << q);
                        continue;
                    }
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
constexpr uint32_t kTileSmallField = 1u << 20;  // fields up to this size always take the tiled pass

void resolve_tile_shape(uint32_t n0, uint32_t n1, uint32_t n2, bool alone, uint32_t rt[3], uint64_t *tiles)
{
    if (alone && uint64_t(n0) * n1 * n2 <= kTileSmallField) {
        // a small field launched on its own: 1024-vertex tiles, so that its
        // tiles spread over the GPU (in a batch the other fields fill it)
        if (n2 > 1) {
            rt[0] = 4; rt[1] = 3; rt[2] = 3;  // 16 x 8 x 8
        } else if (n1 > 1) {
            rt[0] = 5; rt[1] = 5; rt[2] = 0;  // 32 x 32
        } else {
            rt[0] = 10; rt[1] = 0; rt[2] = 0;  // 1024
        }
    } else if (n2 > 1) {
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
    // dense maxima: short paths, the brick walks are faster on their own --
    // unless the field is small, where a few long paths (e.g. up the slopes of
    // smooth regions) set the walks' latency and the tiles cut them short
    if (F.kd != 3 || (uint64_t(F.totals[0]) * 100 >= uint64_t(F.N) && F.N > kTileSmallField)) return;
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
            a[b] = inside(i) && chk(gid(i), F.N, F.err) ? lab[gid(i)] : 0u;
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
            if (chk(i, kTileMax, F.err)) s_w[i] = w;
        }
    }
    __syncthreads();
    // 2: pointer jumping to the terminals (a path has fewer than T steps, so
    // at most log2(T) + 1 rounds change anything)
    for (int round = 0; round <= 14; round++) {
        int changed = 0;
        for (uint32_t i = threadIdx.x; i < T; i += kTileThreads) {
            const uint16_t w = s_w[i];
            if (!(w & kDone) && chk(w & kIdx, kTileMax, F.err)) {
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
            if (inside(i) && (w & kIdx) != i && chk(gid(i), F.N, F.err) && chk(gid(w & kIdx), F.N, F.err))
                lab[gid(i)] = (w & kOut) ? lab[gid(w & kIdx)] : gid(w & kIdx);
        }
    }
}

cudaError_t launch_resolve_tiles(const FieldDev *fields, int nf, uint64_t tiles, cudaStream_t st)
{
    if (tiles == 0) return cudaSuccess;
    k_resolve_tile<<<dim3(static_cast<unsigned>(tiles)), kTileThreads, 0, st>>>(fields, nf);
    return cudaGetLastError();
}

}  // namespace eg
