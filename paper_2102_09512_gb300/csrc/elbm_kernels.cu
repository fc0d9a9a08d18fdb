// Kernels of one lattice x store combination, selected at compile time by
// ELBM_D (2 or 3) and ELBM_ST (elbm::StoreKind).  Built once per combination so
// the eight variants compile in parallel.
//
//   init_kernel        f = f^eq, g = g^eq of (rho, u, T)              (Eqs. 27eq, geq_i)
//   fields_kernel      rho, u, T of the current populations           (Eqs. density..E)
//   moments_kernel     two-pass schedule, pass 1: Q~_aaa field        (Eq. anomalya)
//   collide_kernel     two-pass schedule, pass 2: pull, collide, store (Eqs. fLBGK, gLBGK)
//   fused2d_kernel     D2Q9 one-kernel step: tile + halo moments in shared memory
//   fused3d_kernel     D3Q27 one-kernel step: xy tile + halo, marching along z
//   totals_kernel      FP64 totals of the current state (per-CTA partials)
//
// Streaming is "pull": the value of direction i at node x is read from x - c_i of
// the source store and the post-collision value is written at x in the destination
// store (ping-pong), so every store is coalesced and no two threads write one slot.
#include <cuda_runtime.h>

#include "elbm_internal.h"
#include "elbm_node.cuh"

#ifndef ELBM_D
#error "ELBM_D must be defined (2 or 3)"
#endif
#ifndef ELBM_ST
#error "ELBM_ST must be defined (elbm::StoreKind)"
#endif

namespace elbm {
namespace {

constexpr int kD = ELBM_D;
constexpr int kST = ELBM_ST;
using Cd = Codec<kST>;
using S = typename Cd::S;
using R = typename Cd::R;
constexpr int Q = Lat<kD>::Q;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long node_index(const KParams& p, int x, int y, int z) {
    return (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * (long long)z);
}

// Pull-gather of the 2Q populations arriving at node (x, y, z): direction i is read
// at (x - c_x, y - c_y, z - c_z) with ghost nodes resolved by map_axis.
struct PullRows {
    long long row[3][3];   // node index of (0, y - c_y, z - c_z) for b = c_y+1, c = c_z+1
    int xs[3];             // x - c_x for a = c_x+1
};

// With PULL = false every direction is read at the node itself (no streaming);
// that form is used once, to collide the initial state.
template <bool PULL = true>
__device__ __forceinline__ void pull_rows(const KParams& p, int x, int y, int z, PullRows& r) {
    r.xs[0] = PULL ? map_axis(x + 1, p.nx, p.per_x) : x;
    r.xs[1] = x;
    r.xs[2] = PULL ? map_axis(x - 1, p.nx, p.per_x) : x;
    int ys[3] = {PULL ? map_axis(y + 1, p.ny, p.per_y) : y, y, PULL ? map_axis(y - 1, p.ny, p.per_y) : y};
    int zs[3] = {z, z, z};
    if (kD == 3 && PULL) {
        zs[0] = map_axis(z + 1, p.nz, p.per_z);
        zs[2] = map_axis(z - 1, p.nz, p.per_z);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            r.row[b][c] = (long long)p.nx * ((long long)ys[b] + (long long)p.ny * (long long)zs[c]);
}

__device__ __forceinline__ void gather(const KParams& p, const S* __restrict__ src, const PullRows& r,
                                       R* f, R* g) {
    const size_t N = (size_t)p.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int a = i % 3, b = (i / 3) % 3, c = (kD == 3) ? i / 9 : 1;
        const size_t n = (size_t)(r.row[b][c] + r.xs[a]);
        f[i] = Cd::load(src, (size_t)i * N + n, p.rest32[i]);
        g[i] = Cd::load(src, (size_t)(Q + i) * N + n, p.rest32[Q + i]);
    }
}

__device__ __forceinline__ void store_node(const KParams& p, S* __restrict__ dst, long long n,
                                           const R* f, const R* g) {
    const size_t N = (size_t)p.N;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        dst[(size_t)i * N + (size_t)n] = Cd::enc(f[i], p.rest32[i]);
        dst[(size_t)(Q + i) * N + (size_t)n] = Cd::enc(g[i], p.rest32[Q + i]);
    }
}

// Totals of one node: rho, rho u_x, rho u_y, rho u_z, rho E.
__device__ __forceinline__ void node_totals(const Moments<R>& m, R rE, R v[5]) {
    v[0] = m.rho;
    v[1] = m.rho * m.ux;
    v[2] = m.rho * m.uy;
    v[3] = m.rho * m.uz;
    v[4] = rE;
}

template <typename T>
__device__ __forceinline__ T sum_g(const T* g) {
    T s = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) s += g[i];
    return s;
}

// Kahan-compensated running sum in the arithmetic type.
struct Acc5 {
    R s[5], c[5];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 5; ++k) s[k] = c[k] = R(0);
    }
    __device__ __forceinline__ void add(const R v[5]) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const R y = v[k] - c[k];
            const R t = s[k] + y;
            c[k] = (t - s[k]) - y;
            s[k] = t;
        }
    }
};

// Block-wide FP64 sum of 5 values per thread; thread 0 writes out[0..4].
__device__ __forceinline__ void block_sum5(double v[5], double* __restrict__ out) {
    __shared__ double red[32][5];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) red[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double t = lane < nw ? red[lane][k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) out[k] = t;
        }
    }
}

__device__ __forceinline__ void flag_if(bool bad, int* __restrict__ status) {
    // every thread of the warp reaches this call
    const unsigned any = __ballot_sync(0xffffffffu, bad);
    if (any && (threadIdx.x & 31) == 0 && status) atomicOr(status, 1);
}

// ---------------------------------------------------------------------------
// initial state and field extraction
// ---------------------------------------------------------------------------
__global__ void init_kernel(const __grid_constant__ KParams p, const double* __restrict__ rho,
                            const double* __restrict__ u, const double* __restrict__ T,
                            S* __restrict__ pop, int* __restrict__ status) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (n < p.N) {
        const R r = (R)rho[n], t = (R)T[n];
        const R ux = (R)u[n], uy = (R)u[p.N + n], uz = kD == 3 ? (R)u[2 * p.N + n] : R(0);
        bad = !(r > R(0)) || !(t > R(0)) || !isfinite(r) || !isfinite(t) || !isfinite(ux) ||
              !isfinite(uy) || !isfinite(uz);
        R f[Q], g[Q];
        equilibria<kD, R>(r, ux, uy, uz, t, R(1) / R(p.gm1), f, g);
        store_node(p, pop, n, f, g);
    }
    flag_if(bad, status);
}

__global__ void fields_kernel(const __grid_constant__ KParams p, const S* __restrict__ pop,
                              double* __restrict__ rho, double* __restrict__ u,
                              double* __restrict__ T, int* __restrict__ status) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (n < p.N) {
        R f[Q], g[Q];
        const size_t N = (size_t)p.N;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = Cd::load(pop, (size_t)i * N + n, p.rest32[i]);
            g[i] = Cd::load(pop, (size_t)(Q + i) * N + n, p.rest32[Q + i]);
        }
        Moments<R> m;
        node_moments<kD, R, false>(f, g, R(p.gm1), m);
        rho[n] = m.rho;
        u[n] = m.ux;
        u[p.N + n] = m.uy;
        if (kD == 3) u[2 * p.N + n] = m.uz;
        T[n] = m.T;
        bad = nonphysical(m);
    }
    flag_if(bad, status);
}

// FP64 totals of the current state: one partial per CTA (grid-stride loop).
__global__ void totals_kernel(const __grid_constant__ KParams p, const S* __restrict__ pop,
                              double* __restrict__ partials) {
    double s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
    const size_t N = (size_t)p.N;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < p.N;
         n += (long long)gridDim.x * blockDim.x) {
        R f[Q], g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            f[i] = Cd::load(pop, (size_t)i * N + n, p.rest32[i]);
            g[i] = Cd::load(pop, (size_t)(Q + i) * N + n, p.rest32[Q + i]);
        }
        double v[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double fi = (double)f[i];
            v[0] += fi;
            if (cx_of(i) != 0) v[1] += cx_of(i) * fi;
            if (cy_of(i) != 0) v[2] += cy_of(i) * fi;
            if (cz_of<kD>(i) != 0) v[3] += cz_of<kD>(i) * fi;
            v[4] += (double)g[i];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {   // Neumaier
            const double t = s[k] + v[k];
            c[k] += fabs(s[k]) >= fabs(v[k]) ? (s[k] - t) + v[k] : (v[k] - t) + s[k];
            s[k] = t;
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) s[k] += c[k];
    block_sum5(s, partials + 5 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// two-pass schedule
// ---------------------------------------------------------------------------
// Pass 1: Q~_aaa at every node from the pulled (post-stream) populations.
template <bool PULL>
__global__ void moments_kernel(const __grid_constant__ KParams p, const S* __restrict__ src,
                               R* __restrict__ qf) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int x = (int)(n % p.nx);
    const int y = (int)((n / p.nx) % p.ny);
    const int z = (int)(n / ((long long)p.nx * p.ny));
    PullRows r;
    pull_rows<PULL>(p, x, y, z, r);
    R f[Q], g[Q];
    gather(p, src, r, f, g);
    Moments<R> m;
    node_moments<kD, R, false>(f, g, R(p.gm1), m);
    qf[n] = anomaly(m.rho, m.ux, m.T);
    qf[p.N + n] = anomaly(m.rho, m.uy, m.T);
    if (kD == 3) qf[2 * p.N + n] = anomaly(m.rho, m.uz, m.T);
}

// Pass 2: pull, moments, derivative of Q~ from the field, collide, store.
template <bool PULL>
__global__ void collide_kernel(const __grid_constant__ KParams p, const S* __restrict__ src,
                               S* __restrict__ dst, const R* __restrict__ qf,
                               double* __restrict__ partials, int* __restrict__ status) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double tot[5] = {0, 0, 0, 0, 0};
    bool bad = false;
    if (n < p.N) {
        const int x = (int)(n % p.nx);
        const int y = (int)((n / p.nx) % p.ny);
        const int z = (int)(n / ((long long)p.nx * p.ny));
        PullRows r;
        pull_rows<PULL>(p, x, y, z, r);
        R f[Q], g[Q];
        gather(p, src, r, f, g);
        Moments<R> m;
        node_moments<kD, R, true>(f, g, R(p.gm1), m);
        bad = nonphysical(m);
        const long long N = p.N;
        const int xm = map_axis(x - 1, p.nx, p.per_x), xp = map_axis(x + 1, p.nx, p.per_x);
        const int ym = map_axis(y - 1, p.ny, p.per_y), yp = map_axis(y + 1, p.ny, p.per_y);
        const R Dx = dQ(p.deriv, m.ux, qf[node_index(p, xm, y, z)], qf[n], qf[node_index(p, xp, y, z)]);
        const R Dy = dQ(p.deriv, m.uy, qf[N + node_index(p, x, ym, z)], qf[N + n],
                        qf[N + node_index(p, x, yp, z)]);
        R Dz = R(0);
        if (kD == 3) {
            const int zm = map_axis(z - 1, p.nz, p.per_z), zp = map_axis(z + 1, p.nz, p.per_z);
            Dz = dQ(p.deriv, m.uz, qf[2 * N + node_index(p, x, y, zm)], qf[2 * N + n],
                    qf[2 * N + node_index(p, x, y, zp)]);
        }
        R v[5];
        node_totals(m, sum_g(g), v);
#pragma unroll
        for (int k = 0; k < 5; ++k) tot[k] = (double)v[k];
        collide<kD, R>(f, g, m, Dx, Dy, Dz, p);
        store_node(p, dst, n, f, g);
    }
    flag_if(bad, status);
    block_sum5(tot, partials + 5 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// fused schedule
// ---------------------------------------------------------------------------
constexpr int TX = 32;

// Moments of the node (hx, hy, z) (already mapped), returning one anomaly component.
__device__ __forceinline__ R halo_anomaly(const KParams& p, const S* __restrict__ src, int hx, int hy,
                                          int z, int axis) {
    PullRows r;
    pull_rows(p, hx, hy, z, r);
    R f[Q], g[Q];
    gather(p, src, r, f, g);
    Moments<R> m;
    node_moments<kD, R, false>(f, g, R(p.gm1), m);
    return anomaly(m.rho, axis == 0 ? m.ux : (axis == 1 ? m.uy : m.uz), m.T);
}

// Halo ring of an xy tile: 2*TX row nodes (need Q~_yyy) and 2*TY column nodes (need
// Q~_xxx).  Corner nodes are never needed: the stencil uses axis neighbours only.
template <int TY>
__device__ __forceinline__ void tile_halo(const KParams& p, const S* __restrict__ src, int z, int x0,
                                          int y0, int xl, int yl, R (*qx)[TX + 2], R (*qy)[TX]) {
    const int h = threadIdx.x + TX * threadIdx.y;
    if (h < TX) {
        if (h <= xl) qy[0][h] = halo_anomaly(p, src, x0 + h, map_axis(y0 - 1, p.ny, p.per_y), z, 1);
    } else if (h < 2 * TX) {
        const int hx = h - TX;
        if (hx <= xl) qy[yl + 2][hx] = halo_anomaly(p, src, x0 + hx, map_axis(y0 + yl + 1, p.ny, p.per_y), z, 1);
    } else if (h < 2 * TX + TY) {
        const int hy = h - 2 * TX;
        if (hy <= yl) qx[hy][0] = halo_anomaly(p, src, map_axis(x0 - 1, p.nx, p.per_x), y0 + hy, z, 0);
    } else if (h < 2 * TX + 2 * TY) {
        const int hy = h - 2 * TX - TY;
        if (hy <= yl) qx[hy][xl + 2] = halo_anomaly(p, src, map_axis(x0 + xl + 1, p.nx, p.per_x), y0 + hy, z, 0);
    }
}

// D2Q9: one thread per node of a TX x TY tile.  Phase 1 pulls the populations into
// registers and puts Q~ of the tile and its halo ring into shared memory; phase 2
// collides and stores.  One launch per step, no intermediate field in HBM.
template <int TY>
__global__ void __launch_bounds__(TX * TY)
fused2d_kernel(const __grid_constant__ KParams p, const S* __restrict__ src, S* __restrict__ dst,
               double* __restrict__ partials, int* __restrict__ status) {
    __shared__ R qx[TY][TX + 2];
    __shared__ R qy[TY + 2][TX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    const int xl = min(x0 + TX, p.nx) - 1 - x0, yl = min(y0 + TY, p.ny) - 1 - y0;

    R f[Q], g[Q];
    Moments<R> m;
    if (active) {
        PullRows r;
        pull_rows(p, x, y, 0, r);
        gather(p, src, r, f, g);
        node_moments<kD, R, true>(f, g, R(p.gm1), m);
        qx[ty][tx + 1] = anomaly(m.rho, m.ux, m.T);
        qy[ty + 1][tx] = anomaly(m.rho, m.uy, m.T);
    }
    tile_halo<TY>(p, src, 0, x0, y0, xl, yl, qx, qy);
    __syncthreads();

    double tot[5] = {0, 0, 0, 0, 0};
    bool bad = false;
    if (active) {
        bad = nonphysical(m);
        const R Dx = dQ(p.deriv, m.ux, qx[ty][tx], qx[ty][tx + 1], qx[ty][tx + 2]);
        const R Dy = dQ(p.deriv, m.uy, qy[ty][tx], qy[ty + 1][tx], qy[ty + 2][tx]);
        R v[5];
        node_totals(m, sum_g(g), v);
#pragma unroll
        for (int k = 0; k < 5; ++k) tot[k] = (double)v[k];
        collide<kD, R>(f, g, m, Dx, Dy, R(0), p);
        store_node(p, dst, node_index(p, x, y, 0), f, g);
    }
    flag_if(bad, status);
    block_sum5(tot, partials + 5 * (blockIdx.x + gridDim.x * blockIdx.y));
}

// D3Q27: a CTA owns a TX x TY column of nodes and marches along z over a segment of
// p.tz planes.  For plane z it needs Q~ at z-1, z, z+1 (z-components, kept in
// registers as a rolling window) and at the x/y neighbours in plane z (shared
// memory, halo ring recomputed from the pulled populations).  Per plane: moments
// of plane z+1 (tile + halo) into buffer b^1, barrier, collide plane z from buffer
// b.  The populations of plane z are pulled again for the collision; they were
// read one plane earlier by this CTA and its neighbours, so the re-read is an L2
// hit and HBM sees each population about once per step.
template <int TY>
__global__ void __launch_bounds__(TX * TY, 2)
fused3d_kernel(const __grid_constant__ KParams p, const S* __restrict__ src, S* __restrict__ dst,
               double* __restrict__ partials, int* __restrict__ status) {
    __shared__ R qx[2][TY][TX + 2];
    __shared__ R qy[2][TY + 2][TX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * p.tz, ze = min(zb + p.tz, p.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    const int xl = min(x0 + TX, p.nx) - 1 - x0, yl = min(y0 + TY, p.ny) - 1 - y0;

    // Q~ of the tile and its halo in plane z -> buffer b; returns Q~_zzz of (x, y, z)
    auto plane_moments = [&](int z, int b, bool with_xy) -> R {
        R qz = R(0);
        if (active) {
            PullRows r;
            pull_rows(p, x, y, z, r);
            R f[Q], g[Q];
            gather(p, src, r, f, g);
            Moments<R> m;
            node_moments<kD, R, false>(f, g, R(p.gm1), m);
            if (with_xy) {
                qx[b][ty][tx + 1] = anomaly(m.rho, m.ux, m.T);
                qy[b][ty + 1][tx] = anomaly(m.rho, m.uy, m.T);
            }
            qz = anomaly(m.rho, m.uz, m.T);
        }
        if (with_xy) tile_halo<TY>(p, src, z, x0, y0, xl, yl, qx[b], qy[b]);
        return qz;
    };

    Acc5 acc;
    acc.zero();
    bool bad = false;
    R qz_prev = plane_moments(map_axis(zb - 1, p.nz, p.per_z), 0, false);
    R qz_cur = plane_moments(zb, 0, true);
    for (int z = zb; z < ze; ++z) {
        const int b = (z - zb) & 1;
        const bool last = (z + 1 == ze);
        __syncthreads();   // buffer b^1 is free (collision of z-1 is done)
        const R qz_next = plane_moments(map_axis(z + 1, p.nz, p.per_z), b ^ 1, !last);
        __syncthreads();   // buffer b complete for plane z
        if (active) {
            PullRows r;
            pull_rows(p, x, y, z, r);
            R f[Q], g[Q];
            gather(p, src, r, f, g);
            Moments<R> m;
            node_moments<kD, R, true>(f, g, R(p.gm1), m);
            bad |= nonphysical(m);
            const R Dx = dQ(p.deriv, m.ux, qx[b][ty][tx], qx[b][ty][tx + 1], qx[b][ty][tx + 2]);
            const R Dy = dQ(p.deriv, m.uy, qy[b][ty][tx], qy[b][ty + 1][tx], qy[b][ty + 2][tx]);
            const R Dz = dQ(p.deriv, m.uz, qz_prev, qz_cur, qz_next);
            R v[5];
            node_totals(m, sum_g(g), v);
            acc.add(v);
            collide<kD, R>(f, g, m, Dx, Dy, Dz, p);
            store_node(p, dst, node_index(p, x, y, z), f, g);
        }
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
    flag_if(bad, status);
    double tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) tot[k] = (double)acc.s[k] - (double)acc.c[k];
    block_sum5(tot, partials + 5 * (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kTY2 = 8;                  // D2Q9 fused tile 32 x 8
constexpr int kTY3 = 8;                  // D3Q27 fused tile 32 x 8
constexpr int kTotalsBlocks = 2 * 152;   // totals_kernel grid (grid-stride)

inline unsigned blocks_1d(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

dim3 fused_grid(const KParams& p) {
    if (kD == 2) return dim3((p.nx + TX - 1) / TX, (p.ny + kTY2 - 1) / kTY2, 1);
    return dim3((p.nx + TX - 1) / TX, (p.ny + kTY3 - 1) / kTY3, (p.nz + p.tz - 1) / p.tz);
}

int max_blocks(const KParams& p) {
    long long a = blocks_1d(p.N);
    dim3 gf = fused_grid(p);
    long long b = (long long)gf.x * gf.y * gf.z;
    long long m = a > b ? a : b;
    if (m < kTotalsBlocks) m = kTotalsBlocks;
    return (int)m;
}

// The stored state is post-collision: after step n the store holds C(X_n), where
// X_n is the post-stream state of the method and C the collision, and a step is
// pull (X_{n+1} = S(C(X_n))) followed by collide.  Initialisation therefore writes
// X_0 = (f^eq, g^eq) into the spare store and collides it in place of streaming.
// Moments of C(X_n) equal those of X_n (the collision conserves them), so field
// extraction and totals read each node's own values.
cudaError_t launch_init(const KParams& p, const double* rho, const double* u, const double* T, void* pop,
                        void* spare, void* qfield, double* partials, int* status, cudaStream_t s,
                        long long* launches) {
    const unsigned nb = blocks_1d(p.N);
    init_kernel<<<nb, kThreads, 0, s>>>(p, rho, u, T, (S*)spare, status);
    moments_kernel<false><<<nb, kThreads, 0, s>>>(p, (const S*)spare, (R*)qfield);
    collide_kernel<false><<<nb, kThreads, 0, s>>>(p, (const S*)spare, (S*)pop, (const R*)qfield, partials, status);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_fields(const KParams& p, const void* pop, double* rho, double* u, double* T, int* status,
                          cudaStream_t s, long long* launches) {
    fields_kernel<<<blocks_1d(p.N), kThreads, 0, s>>>(p, (const S*)pop, rho, u, T, status);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_twopass(const KParams& p, const void* src, void* dst, void* qfield, double* partials,
                           int* nblocks, int* status, cudaStream_t s, long long* launches) {
    const unsigned nb = blocks_1d(p.N);
    moments_kernel<true><<<nb, kThreads, 0, s>>>(p, (const S*)src, (R*)qfield);
    collide_kernel<true><<<nb, kThreads, 0, s>>>(p, (const S*)src, (S*)dst, (const R*)qfield, partials, status);
    *launches += 2;
    *nblocks = (int)nb;
    return cudaGetLastError();
}

cudaError_t launch_fused(const KParams& p, const void* src, void* dst, double* partials, int* nblocks,
                         int* status, cudaStream_t s, long long* launches) {
    const dim3 grid = fused_grid(p);
    if constexpr (kD == 2) {
        fused2d_kernel<kTY2><<<grid, dim3(TX, kTY2), 0, s>>>(p, (const S*)src, (S*)dst, partials, status);
    } else {
        fused3d_kernel<kTY3><<<grid, dim3(TX, kTY3), 0, s>>>(p, (const S*)src, (S*)dst, partials, status);
    }
    ++*launches;
    *nblocks = (int)(grid.x * grid.y * grid.z);
    return cudaGetLastError();
}

cudaError_t launch_totals(const KParams& p, const void* pop, double* partials, int* nblocks, cudaStream_t s,
                          long long* launches) {
    totals_kernel<<<kTotalsBlocks, kThreads, 0, s>>>(p, (const S*)pop, partials);
    ++*launches;
    *nblocks = kTotalsBlocks;
    return cudaGetLastError();
}

const Ops kOps = {kD, kST, sizeof(S), sizeof(R), max_blocks, launch_init, launch_fields,
                  launch_twopass, launch_fused, launch_totals};

}  // namespace

#define ELBM_CAT2(a, b) a##b
#define ELBM_CAT(a, b) ELBM_CAT2(a, b)
const Ops* ELBM_CAT(ops_, ELBM_OPS_NAME)() { return &kOps; }

}  // namespace elbm
