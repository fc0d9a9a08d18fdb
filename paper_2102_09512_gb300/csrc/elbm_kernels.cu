// Kernels of one lattice x store combination, selected at compile time by
// ELBM_D (2 or 3) and ELBM_ST (elbm::StoreKind).  Built once per combination so
// the eight variants compile in parallel.
//
//   init_kernel          f = f^eq, g = g^eq of (rho, u, T)              (Eqs. 27eq, geq_i)
//   fields_kernel        rho, u, T of the current populations           (Eqs. density..E)
//   totals_kernel        FP64 totals of the current state (per-CTA partials)
//   moments_kernel       two-pass schedule, pass 1: Q~_aaa field        (Eq. anomalya)
//   collide_kernel       two-pass schedule, pass 2: pull, collide, store (Eqs. fLBGK, gLBGK)
//   fused2d_kernel       D2Q9 one-kernel step: tile + halo moments in shared memory
//   fused3d_kernel       D3Q27 one-kernel step: xy tile + halo marching along z, the pulled
//                        populations of each plane prefetched into shared memory with
//                        cp.async one plane ahead
//   fused3d_reread_kernel  D3Q27 one-kernel step without the shared-memory plane buffers:
//                        the populations of a plane are gathered twice (moments of the
//                        next plane, then the collision), the second time from L2
//
// Layout: element [i * N + n] holds the pair (f_i, g_i) of direction i at node n.
// Streaming is "pull": the pair of direction i at node x is read from x - c_i of the
// source store and the post-collision pair is written at x in the destination store
// (ping-pong), so every store is coalesced and no two threads write one element.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <type_traits>

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
using P = typename Cd::P;
using R = typename Cd::R;
constexpr int Q = Lat<kD>::Q;
constexpr bool DEV = Cd::DEV;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long node_index(const KParams& p, int x, int y, int z) {
    return (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * (long long)z);
}

// Source nodes of the pull at node (x, y, z): direction i = a + 3b + 9c is read at
// (xs[a], ys[b], zs[c]) = (x - c_x, y - c_y, z - c_z) with ghosts resolved by map_axis.
// Node indices fit in 32 bits (N <= 2^31); only the per-direction plane offset
// i * N needs 64 bits, and it is the same for every thread.
struct PullRows {
    int row[3][3];   // node index of (0, ys[b], zs[c])
    int xs[3];
    unsigned gmask;  // bit i: direction i is pulled from beyond a fixed-state face
};

// Fixed-state faces (D2Q9): is coordinate v of axis a beyond a fixed face, and the
// ghost values there (the fixed state's equilibria as raw stored values, its Q~).
__device__ __forceinline__ bool beyond_fixed(const KParams& p, int a, int v, int n) {
    return (v < 0 && p.fix_lo[a]) || (v >= n && p.fix_hi[a]);
}
__device__ __forceinline__ void fixed_pair(const KParams& p, int i, R& f, R& g) {
    if constexpr (sizeof(R) == 8) {
        f = p.fixd[i][0];
        g = p.fixd[i][1];
    } else {
        f = p.fixf[i].x;
        g = p.fixf[i].y;
    }
}
__device__ __forceinline__ R fixed_Q(const KParams& p, int a) {
    if constexpr (sizeof(R) == 8) return p.fixQd[a];
    else return p.fixQf[a];
}

// Directions of node (x, y) whose pull source lies beyond a fixed-state face (D2Q9;
// bit i for direction i): their pairs are the fixed state's, not a stored node's.
// FIX = false: a kernel compiled for grids without fixed faces (always 0).
template <bool FIX = true>
__device__ __forceinline__ unsigned fixed_mask(const KParams& p, int x, int y) {
    unsigned m = 0u;
    if constexpr (kD == 2 && FIX) {
        if (p.has_fixed) {
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (beyond_fixed(p, 0, x + 1 - a, p.nx) || beyond_fixed(p, 1, y + 1 - b, p.ny))
                        m |= 1u << (a + 3 * b);
        }
    }
    return m;
}

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
            r.row[b][c] = p.nx * (ys[b] + p.ny * zs[c]);
    r.gmask = PULL ? fixed_mask(p, x, y) : 0u;
}

// Address of the pair of direction i pulled by node r in store s.
__device__ __forceinline__ const P* src_ptr(const KParams& p, const P* __restrict__ s, const PullRows& r, int i) {
    const int a = i % 3, b = (i / 3) % 3, c = (kD == 3) ? i / 9 : 1;
    return (s + (size_t)i * (size_t)p.N) + (unsigned)(r.row[b][c] + r.xs[a]);
}

__device__ __forceinline__ void gather(const KParams& p, const P* __restrict__ src, const PullRows& r,
                                       R* f, R* g) {
#pragma unroll
    for (int i = 0; i < Q; ++i) Cd::dec(*src_ptr(p, src, r, i), f[i], g[i]);
    if (r.gmask) {   // sources beyond a fixed-state face (the load above read a clamped node)
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if ((r.gmask >> i) & 1u) fixed_pair(p, i, f[i], g[i]);
    }
}

// The post-collision pairs C(X_n)_i of node n as stored: in place (p.aa = 0), or in the AA
// single-store layouts (p.aa = 1: direction i at opp(i) of the node; p.aa = 2: direction i
// pushed to the node's neighbour n + c_i, periodic).
__device__ __forceinline__ void load_local(const KParams& p, const P* __restrict__ pop, long long n, R* f,
                                           R* g) {
    if (p.aa == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) Cd::dec(pop[(size_t)i * (size_t)p.N + (size_t)n], f[i], g[i]);
    } else if (p.aa == 1) {
#pragma unroll
        for (int i = 0; i < Q; ++i) Cd::dec(pop[(size_t)(Q - 1 - i) * (size_t)p.N + (size_t)n], f[i], g[i]);
    } else {
        const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny), z = (int)(n / ((long long)p.nx * p.ny));
        PullRows r;
        pull_rows(p, x, y, z, r);   // the pull source of opp(i) is n + c_i
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int k = Q - 1 - i, a = k % 3, b = (k / 3) % 3, c = (kD == 3) ? k / 9 : 1;
            Cd::dec(*((pop + (size_t)i * (size_t)p.N) + (unsigned)(r.row[b][c] + r.xs[a])), f[i], g[i]);
        }
    }
}

__device__ __forceinline__ void store_node(const KParams& p, P* __restrict__ dst, long long n, const R* f,
                                           const R* g) {
    const unsigned nn = (unsigned)n;
#pragma unroll
    for (int i = 0; i < Q; ++i) (dst + (size_t)i * (size_t)p.N)[nn] = Cd::enc(f[i], g[i]);
}

// Totals of one node: rho, rho u_x, rho u_y, rho u_z, rho E.
__device__ __forceinline__ void node_totals(const Moments<R>& m, R rE, R v[5]) {
    v[0] = m.rho;
    v[1] = m.rho * m.ux;
    v[2] = m.rho * m.uy;
    v[3] = m.rho * m.uz;
    v[4] = rE;
}

// Per-thread running sum of the node totals over the planes of a z segment:
// Kahan-compensated in FP64; in FP32 a plain sum (at most p.tz terms of per-node
// values that are themselves FP32 results), which saves the registers of the
// compensation terms.
struct Acc5 {
    R s[5], c[5];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 5; ++k) s[k] = c[k] = R(0);
    }
    __device__ __forceinline__ void add(const R v[5]) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if constexpr (sizeof(R) == 8) {
                const R y = v[k] - c[k];
                const R t = s[k] + y;
                c[k] = (t - s[k]) - y;
                s[k] = t;
            } else {
                s[k] += v[k];
            }
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

// The same sum for kernels that reduce once per small tile: the sum within each warp runs
// in the arithmetic type T (an FP64 shuffle tree per 256-node tile costs more than the
// tile's whole update on GB300's narrow FP64 pipe), the sum of the warp partials in FP64.
// With T = double it is block_sum5.  An FP32 warp partial of 32 node values carries a
// relative rounding error of about 1e-7, below the rounding of the FP32 values summed.
template <typename T>
__device__ __forceinline__ void block_sum5_warp(T v[5], double* __restrict__ out) {
    if constexpr (sizeof(T) == 8) {
        block_sum5(v, out);
    } else {
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
            for (int k = 0; k < 5; ++k) red[warp][k] = (double)v[k];
        __syncthreads();
        if (tid < 5) {
            const int nw = (nthreads + 31) >> 5;
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += red[w][tid];
            out[tid] = t;
        }
    }
}

__device__ __forceinline__ void flag_if(bool bad, int* __restrict__ status) {
    // every thread of the warp reaches this call
    const unsigned any = __ballot_sync(0xffffffffu, bad);
    if (any && (threadIdx.x & 31) == 0 && status) atomicOr(status, 1);
}

// Asynchronous global -> shared copy of one pair (cp.async, bypasses registers).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// Waits until at most N of this thread's most recent cp.async groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_pending() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// initial state and field extraction
// ---------------------------------------------------------------------------
// Nodes n0 .. n0 + cnt - 1; the fields hold those nodes only (u component-major with
// stride cnt).
__global__ void init_kernel(const __grid_constant__ KParams p, const double* __restrict__ rho,
                            const double* __restrict__ u, const double* __restrict__ T,
                            P* __restrict__ pop, int* __restrict__ status, long long n0, long long cnt) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = n0 + k;
    bool bad = false;
    if (k < cnt) {
        const R r = (R)rho[k], t = (R)T[k];
        const R ux = (R)u[k], uy = (R)u[cnt + k], uz = kD == 3 ? (R)u[2 * cnt + k] : R(0);
        bad = !(r > R(0)) || !(t > R(0)) || !isfinite(r) || !isfinite(t) || !isfinite(ux) ||
              !isfinite(uy) || !isfinite(uz);
        R f[Q], g[Q];
        equilibria<kD, R>(r, ux, uy, uz, t, U_of_T(t, p), f, g);
        if constexpr (DEV) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[i] -= R(p.rest2[i].x);
                g[i] -= R(p.rest2[i].y);
            }
        }
        store_node(p, pop, n, f, g);
    }
    flag_if(bad, status);
}

// Nodes n0 .. n0 + cnt - 1 into fields of cnt nodes (u component-major with stride cnt).
__global__ void fields_kernel(const __grid_constant__ KParams p, const P* __restrict__ pop,
                              double* __restrict__ rho, double* __restrict__ u,
                              double* __restrict__ T, int* __restrict__ status, long long n0, long long cnt) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = n0 + k;
    bool bad = false;
    if (k < cnt) {
        R f[Q], g[Q];
        load_local(p, pop, n, f, g);
        Moments<R> m;
        node_moments<kD, R, false, DEV>(f, g, p, m);
        rho[k] = m.rho;
        u[k] = m.ux;
        u[cnt + k] = m.uy;
        if (kD == 3) u[2 * cnt + k] = m.uz;
        T[k] = m.T;
        bad = nonphysical(m);
    }
    flag_if(bad, status);
}

// FP64 totals of the current state: one partial per CTA (grid-stride loop).
__global__ void totals_kernel(const __grid_constant__ KParams p, const P* __restrict__ pop,
                              double* __restrict__ partials) {
    double s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < p.N;
         n += (long long)gridDim.x * blockDim.x) {
        R f[Q], g[Q];
        load_local(p, pop, n, f, g);
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
        if constexpr (DEV) {   // moment sums of the rest state (no momentum)
            v[0] += (double)p.rest_rho;
            v[4] += (double)p.rest_E;
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

// Velocity of node n from its f values only (rho and rho u).
__device__ __forceinline__ void node_velocity(const KParams& p, const P* __restrict__ pop, long long n, R u[3]) {
    R rho = 0, j[3] = {0, 0, 0};
    R fs[Q], gs[Q];
    load_local(p, pop, n, fs, gs);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R f = fs[i];
        rho += f;
        if (cx_of(i)) j[0] += cx_of(i) * f;
        if (cy_of(i)) j[1] += cy_of(i) * f;
        if (cz_of<kD>(i)) j[2] += cz_of<kD>(i) * f;
    }
    if constexpr (DEV) rho += R(p.rest_rho);
    const R inv = qdiv(R(1), rho);
    u[0] = j[0] * inv;
    u[1] = j[1] * inv;
    u[2] = j[2] * inv;
}

// Turbulence statistics of the current state (one FP64 partial vector per CTA):
// sums of rho, rho^2, rho u.u, u.u, theta^2, T, T^2, (d u_x / d x)^2, |omega|^2, u_x^2
// and mu(T) |omega|^2, with the velocity gradient by second-order central differences
// (boundary nodes use the ghost values of the boundary map): dilatation
// theta = div u, vorticity omega = curl u, mu = mu0 (T/T0)^mu_exp (Eq. mu law).
constexpr int kStats = kStatsSums;
__global__ void stats_kernel(const __grid_constant__ KParams p, const P* __restrict__ pop,
                             double* __restrict__ partials) {
    double acc[kStats] = {};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < p.N;
         n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny), z = (int)(n / ((long long)p.nx * p.ny));
        R f[Q], g[Q];
        load_local(p, pop, n, f, g);
        Moments<R> m;
        node_moments<kD, R, false, DEV>(f, g, p, m);
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // G[a][b] = d u_a / d x_b
        R up[3], um[3];
        node_velocity(p, pop, node_index(p, map_axis(x + 1, p.nx, p.per_x), y, z), up);
        node_velocity(p, pop, node_index(p, map_axis(x - 1, p.nx, p.per_x), y, z), um);
#pragma unroll
        for (int a = 0; a < 3; ++a) G[a][0] = 0.5 * ((double)up[a] - (double)um[a]);
        node_velocity(p, pop, node_index(p, x, map_axis(y + 1, p.ny, p.per_y), z), up);
        node_velocity(p, pop, node_index(p, x, map_axis(y - 1, p.ny, p.per_y), z), um);
#pragma unroll
        for (int a = 0; a < 3; ++a) G[a][1] = 0.5 * ((double)up[a] - (double)um[a]);
        if (kD == 3) {
            node_velocity(p, pop, node_index(p, x, y, map_axis(z + 1, p.nz, p.per_z)), up);
            node_velocity(p, pop, node_index(p, x, y, map_axis(z - 1, p.nz, p.per_z)), um);
#pragma unroll
            for (int a = 0; a < 3; ++a) G[a][2] = 0.5 * ((double)up[a] - (double)um[a]);
        }
        const double theta = G[0][0] + G[1][1] + G[2][2];
        const double wx = G[2][1] - G[1][2], wy = G[0][2] - G[2][0], wz = G[1][0] - G[0][1];
        const double rho = m.rho, T = m.T;
        const double uu = (double)m.ux * m.ux + (double)m.uy * m.uy + (double)m.uz * m.uz;
        acc[0] += rho;
        acc[1] += rho * rho;
        acc[2] += rho * uu;
        acc[3] += uu;
        acc[4] += theta * theta;
        acc[5] += T;
        acc[6] += T * T;
        const double w2 = wx * wx + wy * wy + wz * wz;
        const double mu = p.mu_exp != 0.0 ? p.mu0 * pow(T / p.T0, p.mu_exp) : p.mu0;
        acc[7] += G[0][0] * G[0][0];
        acc[8] += w2;
        acc[9] += (double)m.ux * m.ux;
        acc[10] += mu * w2;
    }
    // block reduction of kStats values, five at a time
    static_assert(kStats <= 15, "three passes of five values");
    __shared__ double tail[5];
    for (int base = 0; base < kStats; base += 5) {
        double v5[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) v5[k] = base + k < kStats ? acc[base + k] : 0.0;
        block_sum5(v5, tail);
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < 5 && base + k < kStats; ++k) partials[(size_t)kStats * blockIdx.x + base + k] = tail[k];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// two-pass schedule
// ---------------------------------------------------------------------------
// Pass 1: Q~_aaa at every node from the pulled (post-stream) populations.
template <bool PULL>
__global__ void moments_kernel(const __grid_constant__ KParams p, const P* __restrict__ src,
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
    node_moments<kD, R, false, DEV>(f, g, p, m);
    qf[n] = anomaly(m.rho, m.ux, m.T);
    qf[p.N + n] = anomaly(m.rho, m.uy, m.T);
    if (kD == 3) qf[2 * p.N + n] = anomaly(m.rho, m.uz, m.T);
}

// Pass 2: pull, moments, derivative of Q~ from the field, collide, store.
template <bool PULL>
__global__ void collide_kernel(const __grid_constant__ KParams p, const P* __restrict__ src,
                               P* __restrict__ dst, const R* __restrict__ qf,
                               double* __restrict__ partials, int* __restrict__ status) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    R tot[5] = {0, 0, 0, 0, 0};
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
        node_moments<kD, R, true, DEV>(f, g, p, m);
        bad = nonphysical(m);
        const long long N = p.N;
        const int xm = map_axis(x - 1, p.nx, p.per_x), xp = map_axis(x + 1, p.nx, p.per_x);
        const int ym = map_axis(y - 1, p.ny, p.per_y), yp = map_axis(y + 1, p.ny, p.per_y);
        R qxm = qf[node_index(p, xm, y, z)], qxp = qf[node_index(p, xp, y, z)];
        R qym = qf[N + node_index(p, x, ym, z)], qyp = qf[N + node_index(p, x, yp, z)];
        if (kD == 2 && p.has_fixed) {
            if (beyond_fixed(p, 0, x - 1, p.nx)) qxm = fixed_Q(p, 0);
            if (beyond_fixed(p, 0, x + 1, p.nx)) qxp = fixed_Q(p, 0);
            if (beyond_fixed(p, 1, y - 1, p.ny)) qym = fixed_Q(p, 1);
            if (beyond_fixed(p, 1, y + 1, p.ny)) qyp = fixed_Q(p, 1);
        }
        const R Dx = dQ(p.deriv, m.ux, qxm, qf[n], qxp);
        const R Dy = dQ(p.deriv, m.uy, qym, qf[N + n], qyp);
        R Dz = R(0);
        if (kD == 3) {
            const int zm = map_axis(z - 1, p.nz, p.per_z), zp = map_axis(z + 1, p.nz, p.per_z);
            Dz = dQ(p.deriv, m.uz, qf[2 * N + node_index(p, x, y, zm)], qf[2 * N + n],
                    qf[2 * N + node_index(p, x, y, zp)]);
        }
        node_totals(m, m.rE, tot);
        collide<kD, R, DEV>(f, g, m, Dx, Dy, Dz, p);
        store_node(p, dst, n, f, g);
    }
    flag_if(bad, status);
    block_sum5_warp(tot, partials + 5 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// AA single-store layout (periodic grids, two-pass schedule)
// ---------------------------------------------------------------------------
// One store A holds the post-collision state C(X_n) in one of two layouts that alternate
// with the step:
//   L0: C(X_n)_i(x) at A[opp(i)][x]          (swapped at the node)
//   L1: C(X_n)_i(x) at A[i][x + c_i]         (pushed to the neighbour, periodic wrap)
// A step from L0 pulls f_i(y) = C(X_n)_i(y - c_i) = A[opp(i)][y - c_i] and pushes the new
// C(X_n+1)_i(y) to A[i][y + c_i] (-> L1); a step from L1 reads f_i(y) = A[i][y] at the node
// itself and writes C(X_n+1)_i(y) to A[opp(i)][y] (-> L0).  In both, the slots a node
// writes are exactly the slots it read (for a step from L0, direction i's write target
// A[i][y + c_i] is direction opp(i)'s source), so with the Q~ field computed in a first pass
// every slot is read and written by one thread only.  A periodic map is a bijection; a
// clamped (zero-gradient) face would let two nodes read one slot that one of them writes.
__host__ __device__ constexpr int opp(int i) { return Q - 1 - i; }

// Address of direction j's pair in the row/column of direction k's pull source (PullRows of
// the node): a step from L0 reads A[opp(i)] at the source of i and writes A[i] at the
// source of opp(i).
__device__ __forceinline__ P* aa_ptr(const KParams& p, P* A, const PullRows& r, int j, int k) {
    const int a = k % 3, b = (k / 3) % 3, c = (kD == 3) ? k / 9 : 1;
    return (A + (size_t)j * (size_t)p.N) + (unsigned)(r.row[b][c] + r.xs[a]);
}

template <bool FROM_L1>
__device__ __forceinline__ void aa_gather(const KParams& p, P* A, const PullRows& r, long long n, R* f, R* g) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const P v = FROM_L1 ? A[(size_t)i * (size_t)p.N + (size_t)n] : *aa_ptr(p, A, r, opp(i), i);
        Cd::dec(v, f[i], g[i]);
    }
}
template <bool FROM_L1>
__device__ __forceinline__ void aa_store(const KParams& p, P* A, const PullRows& r, long long n, const R* f,
                                         const R* g) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const P v = Cd::enc(f[i], g[i]);
        if (FROM_L1) A[(size_t)opp(i) * (size_t)p.N + (size_t)n] = v;
        else *aa_ptr(p, A, r, i, opp(i)) = v;
    }
}

// Pass 1 of an AA step: Q~_aaa of every node from its post-stream populations.
template <bool FROM_L1>
__global__ void aa_moments_kernel(const __grid_constant__ KParams p, P* A, R* __restrict__ qf) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny), z = (int)(n / ((long long)p.nx * p.ny));
    PullRows r;
    if (!FROM_L1) pull_rows(p, x, y, z, r);
    R f[Q], g[Q];
    aa_gather<FROM_L1>(p, A, r, n, f, g);
    Moments<R> m;
    node_moments<kD, R, false, DEV>(f, g, p, m);
    qf[n] = anomaly(m.rho, m.ux, m.T);
    qf[p.N + n] = anomaly(m.rho, m.uy, m.T);
    if (kD == 3) qf[2 * p.N + n] = anomaly(m.rho, m.uz, m.T);
}

// Pass 2 of an AA step: the same reads, the derivative of Q~ from the field, collision, and
// the writes into the slots just read.
// Two CTAs per SM (at most 128 registers) for the FP32-arithmetic stores: the L0 form holds
// the pull offsets for its pushed writes and would take 156 (FP32) / 182 (FP16) registers,
// one CTA of 8 warps per SM, which made it twice as slow as the L1 form (AA step at 256^3,
// FP32 6.1 -> 7.8 GLUPS, FP16 7.6 -> 10.7 with the cap, despite about 100 bytes of spills).
// FP64 keeps one CTA (the cap would spill 0.8 KB per thread).
constexpr int kAaMinBlocks = sizeof(R) == 4 ? 2 : 1;
template <bool FROM_L1>
__global__ void __launch_bounds__(kThreads1D, kAaMinBlocks)
aa_collide_kernel(const __grid_constant__ KParams p, P* A, const R* __restrict__ qf,
                                  double* __restrict__ partials, int* __restrict__ status) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    R tot[5] = {0, 0, 0, 0, 0};
    bool bad = false;
    if (n < p.N) {
        const int x = (int)(n % p.nx), y = (int)((n / p.nx) % p.ny), z = (int)(n / ((long long)p.nx * p.ny));
        PullRows r;
        if (!FROM_L1) pull_rows(p, x, y, z, r);
        R f[Q], g[Q];
        aa_gather<FROM_L1>(p, A, r, n, f, g);
        Moments<R> m;
        node_moments<kD, R, true, DEV>(f, g, p, m);
        bad = nonphysical(m);
        const long long N = p.N;
        const int xm = map_axis(x - 1, p.nx, p.per_x), xp = map_axis(x + 1, p.nx, p.per_x);
        const int ym = map_axis(y - 1, p.ny, p.per_y), yp = map_axis(y + 1, p.ny, p.per_y);
        const R Dx = dQ(p.deriv, m.ux, qf[node_index(p, xm, y, z)], qf[n], qf[node_index(p, xp, y, z)]);
        const R Dy = dQ(p.deriv, m.uy, qf[N + node_index(p, x, ym, z)], qf[N + n], qf[N + node_index(p, x, yp, z)]);
        R Dz = R(0);
        if (kD == 3) {
            const int zm = map_axis(z - 1, p.nz, p.per_z), zp = map_axis(z + 1, p.nz, p.per_z);
            Dz = dQ(p.deriv, m.uz, qf[2 * N + node_index(p, x, y, zm)], qf[2 * N + n],
                    qf[2 * N + node_index(p, x, y, zp)]);
        }
        node_totals(m, m.rE, tot);
        collide<kD, R, DEV>(f, g, m, Dx, Dy, Dz, p);
        aa_store<FROM_L1>(p, A, r, n, f, g);
    }
    flag_if(bad, status);
    block_sum5_warp(tot, partials + 5 * blockIdx.x);
}

// ---------------------------------------------------------------------------
// fused schedules
// ---------------------------------------------------------------------------
constexpr int TX = 32;

// Halo ring of a TX x TY tile: 2*TX row nodes (they need Q~_yyy) and 2*TY column
// nodes (Q~_xxx).  Corners are never needed: the stencil uses axis neighbours only.
// Halo node h: [0,TX) row below, [TX,2TX) row above, then the left and right columns.
// Returns false for slots outside a ragged tile; (hx, hy) are mapped by the BCs and
// (sx, sy) is where its Q~ goes: qy[sy][sx] for rows, qx[sy][sx] for columns.
template <int TY>
__device__ __forceinline__ bool halo_node(const KParams& p, int h, int x0, int y0, int xl, int yl, int& hx,
                                          int& hy, int& sx, int& sy, int& axis) {
    if (h < TX) {
        hx = x0 + h; hy = map_axis(y0 - 1, p.ny, p.per_y); sx = h; sy = 0; axis = 1;
        return h <= xl;
    }
    if (h < 2 * TX) {
        const int k = h - TX;
        hx = x0 + k; hy = map_axis(y0 + yl + 1, p.ny, p.per_y); sx = k; sy = yl + 2; axis = 1;
        return k <= xl;
    }
    if (h < 2 * TX + TY) {
        const int k = h - 2 * TX;
        hx = map_axis(x0 - 1, p.nx, p.per_x); hy = y0 + k; sx = 0; sy = k; axis = 0;
        return k <= yl;
    }
    const int k = h - 2 * TX - TY;
    hx = map_axis(x0 + xl + 1, p.nx, p.per_x); hy = y0 + k; sx = xl + 2; sy = k; axis = 0;
    return k <= yl;
}

// D2Q9: one thread per node of a TX x TY tile.  Phase 1 pulls the populations into
// registers and puts Q~ of the tile and its halo ring into shared memory; phase 2
// collides and stores.  One launch per step, no intermediate field in HBM.  The tile
// body is shared by the per-lattice kernel and the persistent ensemble kernel;
// `partial` (may be null) receives the tile's totals.
template <int TY, bool CAL, bool ONE_WAIT>
__device__ __forceinline__ void fused2d_tile(const KParams& p, const P* __restrict__ src, P* __restrict__ dst,
                                             int bx, int by, double* __restrict__ partial,
                                             int* __restrict__ status) {
    __shared__ R qx[TY][TX + 2];
    __shared__ R qy[TY + 2][TX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = bx * TX, y0 = by * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    const int xl = min(x0 + TX, p.nx) - 1 - x0, yl = min(y0 + TY, p.ny) - 1 - y0;

    // ONE_WAIT: both gathers (the node's and its halo node's pairs) are issued before any
    // arithmetic, so the tile waits for memory once; the persistent ensemble kernel keeps
    // the node's gather and moments first, which needs fewer registers (64, no spills)
    const int h = tx + TX * ty;
    int hx = 0, hy = 0, sx = 0, sy = 0, axis = 0;
    const bool hv = h < 2 * TX + 2 * TY && halo_node<TY>(p, h, x0, y0, xl, yl, hx, hy, sx, sy, axis);
    // the unmapped halo coordinate is (x0 + sx - 1, y0 + sy) for columns and (x0 + sx, y0 + sy - 1)
    // for rows; beyond a fixed face the halo's Q~ is the fixed state's
    const bool hfixed = hv && p.has_fixed &&
                        (axis == 1 ? beyond_fixed(p, 1, y0 + sy - 1, p.ny) : beyond_fixed(p, 0, x0 + sx - 1, p.nx));
    R f[Q], g[Q];
    Moments<R> m;
    auto halo_q = [&](const R* hf, const R* hg) {
        Moments<R> hm;
        node_moments<kD, R, false, DEV, CAL>(hf, hg, p, hm);
        return anomaly(hm.rho, axis == 1 ? hm.uy : hm.ux, hm.T);
    };
    auto store_halo_q = [&](R q) {
        if (axis == 1) qy[sy][sx] = q;
        else qx[sy][sx] = q;
    };
    if constexpr (ONE_WAIT) {
        R hf[Q], hg[Q];
        if (active) {
            PullRows r;
            pull_rows(p, x, y, 0, r);
            gather(p, src, r, f, g);
        }
        if (hv && !hfixed) {
            PullRows r;
            pull_rows(p, hx, hy, 0, r);
            gather(p, src, r, hf, hg);
        }
        if (active) {
            node_moments<kD, R, true, DEV, CAL>(f, g, p, m);
            qx[ty][tx + 1] = anomaly(m.rho, m.ux, m.T);
            qy[ty + 1][tx] = anomaly(m.rho, m.uy, m.T);
        }
        if (hv) store_halo_q(hfixed ? fixed_Q(p, axis) : halo_q(hf, hg));
    } else {
        if (active) {
            PullRows r;
            pull_rows(p, x, y, 0, r);
            gather(p, src, r, f, g);
            node_moments<kD, R, true, DEV, CAL>(f, g, p, m);
            qx[ty][tx + 1] = anomaly(m.rho, m.ux, m.T);
            qy[ty + 1][tx] = anomaly(m.rho, m.uy, m.T);
        }
        if (hv) {
            R q;
            if (hfixed) {
                q = fixed_Q(p, axis);
            } else {
                PullRows r;
                pull_rows(p, hx, hy, 0, r);
                R hf[Q], hg[Q];
                gather(p, src, r, hf, hg);
                q = halo_q(hf, hg);
            }
            store_halo_q(q);
        }
    }
    __syncthreads();

    R tot[5] = {0, 0, 0, 0, 0};
    bool bad = false;
    if (active) {
        bad = nonphysical(m);
        const R Dx = dQ(p.deriv, m.ux, qx[ty][tx], qx[ty][tx + 1], qx[ty][tx + 2]);
        const R Dy = dQ(p.deriv, m.uy, qy[ty][tx], qy[ty + 1][tx], qy[ty + 2][tx]);
        if (partial) node_totals(m, m.rE, tot);
        collide<kD, R, DEV, CAL>(f, g, m, Dx, Dy, R(0), p);
        store_node(p, dst, node_index(p, x, y, 0), f, g);
    }
    flag_if(bad, status);
    if (partial) block_sum5_warp(tot, partial);
    __syncthreads();   // the shared arrays are reused by the next tile of a persistent CTA
}

template <int TY, bool CAL>
__global__ void __launch_bounds__(TX * TY)
fused2d_kernel(const __grid_constant__ KParams p, const P* __restrict__ src, P* __restrict__ dst,
               double* __restrict__ partials, int* __restrict__ status) {
    fused2d_tile<TY, CAL, true>(p, src, dst, blockIdx.x, blockIdx.y, partials + 5 * (blockIdx.x + gridDim.x * blockIdx.y),
                     status);
}

// Persistent D2Q9 ensemble step: the tiles of all instances form one work list
// (instance k owns tiles [tile_start[k], tile_start[k+1]), tiles_x[k] per row); CTA
// b processes tiles b, b + gridDim.x, ...  Instance k's populations start at element
// offset[k] of both stores; its parameters are params[k].  No totals are kept.
template <int TY, bool CAL>
__global__ void __launch_bounds__(TX * TY)
ensemble2d_kernel(const EnsembleArgs a, const P* __restrict__ src, P* __restrict__ dst, int* __restrict__ status) {
    __shared__ int s_start[kMaxEnsemble + 1];
    __shared__ int s_tx[kMaxEnsemble];
    const int tid = threadIdx.x + TX * threadIdx.y;
    for (int k = tid; k <= a.n; k += TX * TY) s_start[k] = a.tile_start[k];
    for (int k = tid; k < a.n; k += TX * TY) s_tx[k] = a.tiles_x[k];
    __syncthreads();
    int k = 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        while (t >= s_start[k + 1]) ++k;   // t increases, so k only moves forward
        const int local = t - s_start[k];
        const int bx = local % s_tx[k], by = local / s_tx[k];
        const long long off = a.offset[k];
        fused2d_tile<TY, CAL, false>(a.params[k], src + off, dst + off, bx, by, nullptr, status);
    }
}

// Q~_zzz of the node (x, y, z) by a direct gather (used once per z segment).
template <bool CAL>
__device__ __forceinline__ R direct_anomaly_z(const KParams& p, const P* __restrict__ src, int x, int y, int z) {
    PullRows r;
    pull_rows(p, x, y, z, r);
    R f[Q], g[Q];
    gather(p, src, r, f, g);
    Moments<R> m;
    node_moments<kD, R, false, DEV, CAL>(f, g, p, m);
    return anomaly(m.rho, m.uz, m.T);
}

// D3Q27, pipelined.  A CTA owns a TX x TY column of nodes and marches along z over a
// segment of p.tz planes.  For every plane q it needs the pulled pairs of its TX*TY
// nodes and of the 2TX+2TY halo nodes; these are copied with cp.async into one of
// two shared-memory plane buffers, laid out [direction][slot].  Thread t copies and
// reads only its own slots (its node, and halo node t for t < 2TX+2TY), so the
// population buffers need no barrier: each thread waits for its own copies.  Only
// the Q~ arrays (double-buffered by plane parity) are shared, and one barrier per
// plane orders both of their hazards.  Per plane z:
//   wait for this thread's copies of plane z+1; barrier;
//   moments of plane z+1 (tile and halo) -> Q~ in shared memory, moments kept in
//       registers for the next iteration;
//   read the pairs of plane z from shared memory, prefetch plane z+2 into the same
//       slots;
//   collide plane z (moments and Q~ from the previous iteration, the rolling Q~_zzz
//       registers) and store.
// Every population leaves HBM once per step; the collision overlaps the prefetch.
template <int TY, int NB>
struct Pipe {
    static constexpr int NT = TX * TY;
    static constexpr int NH = 2 * TX + 2 * TY;
    static constexpr int NS = NT + NH;
    static constexpr size_t buf_bytes = (size_t)NB * Q * NS * sizeof(P);
    static constexpr size_t q_bytes = (size_t)2 * (TY * (TX + 2) + (TY + 2) * TX) * sizeof(R);
    static constexpr size_t smem_bytes = buf_bytes + q_bytes;
};

// Base of every direction plane of the source and destination stores, computed on the
// host: the kernel then forms each population address as one 32-bit node offset added
// to a base read from the parameter bank, instead of a 64-bit i * N product per access.
struct DirPlanes {
    const P* src[Q];
    P* dst[Q];
};
__device__ __forceinline__ const P* dir_src(const DirPlanes& pl, const PullRows& r, int i) {
    const int a = i % 3, b = (i / 3) % 3, c = (kD == 3) ? i / 9 : 1;
    return pl.src[i] + (unsigned)(r.row[b][c] + r.xs[a]);
}

template <int TY, int NB>
struct PipeBytes {
    static constexpr size_t value = Pipe<TY, NB>::smem_bytes;
};

// The collision's per-direction updates of f and g as one two-lane FP32 operation (FFMA2):
// FP16 19.9 -> 20.4 GLUPS at 256^3, FP32 unchanged (the same results bit for bit).
#ifndef ELBM_FFMA2
#define ELBM_FFMA2 1
#endif
constexpr bool kFFMA2 = ELBM_FFMA2;

// Store of a post-collision pair.  With ELBM_STCS the store is marked streaming (evict
// first), so that the step's writes do not push the planes prefetched ahead out of L2.
#ifndef ELBM_STCS
#define ELBM_STCS 1
#endif
__device__ __forceinline__ void store_pair(P* ptr, P v) {
    if constexpr (ELBM_STCS && sizeof(P) <= 8) __stcs(ptr, v);
    else *ptr = v;
}

// L2 prefetch of one box of a direction plane through the tensor-copy unit (no shared
// memory, no L1; a hint: boxes that leave the tensor are clipped).  x * element size
// must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int w) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];\n" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(x), "r"(y), "r"(w)
                 : "memory");
}

template <int TY, int NB, int MINB, bool EARLY, int DD, bool CAL>
__global__ void __launch_bounds__(TX * TY, MINB)
fused3d_kernel(const __grid_constant__ KParams p, const __grid_constant__ DirPlanes pl,
               const P* __restrict__ src, double* __restrict__ partials, int* __restrict__ status,
               const __grid_constant__ CUtensorMap pmap, int pref) {
    using PP = Pipe<TY, NB>;
    static_assert(NB == 2, "plane z+2 is prefetched into the slots of plane z");
    static_assert(sizeof(R) == 4 && DD == 3, "the pipelined kernel is D3Q27 in FP32");
    constexpr int NT = PP::NT, NH = PP::NH, NS = PP::NS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P* buf = reinterpret_cast<P*>(smem_raw);                       // [NB][Q][NS]
    R* qxs = reinterpret_cast<R*>(smem_raw + PP::buf_bytes);       // [2][TY][TX+2]
    R* qys = qxs + 2 * TY * (TX + 2);                              // [2][TY+2][TX]
    auto QX = [&](int b, int row, int col) -> R& { return qxs[(b * TY + row) * (TX + 2) + col]; };
    auto QY = [&](int b, int row, int col) -> R& { return qys[(b * (TY + 2) + row) * TX + col]; };

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * p.tz, ze = min(zb + p.tz, p.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    const int xl = min(x0 + TX, p.nx) - 1 - x0, yl = min(y0 + TY, p.ny) - 1 - y0;

    // this thread's halo node (if any) is fixed for the whole segment
    int hx = 0, hy = 0, hsx = 0, hsy = 0, haxis = 0;
    const bool has_halo = tid < NH && halo_node<TY>(p, tid, x0, y0, xl, yl, hx, hy, hsx, hsy, haxis);

    // copies of plane q (already mapped) into buffer sb
    auto issue_plane = [&](int q, int sb, bool with_halo) {
        P* bb = buf + (size_t)sb * Q * NS;
        if (active) {
            PullRows r;
            pull_rows(p, x, y, q, r);
#pragma unroll
            for (int i = 0; i < Q; ++i) cp_async<sizeof(P)>(bb + i * NS + tid, dir_src(pl, r, i));
        }
        if (with_halo && has_halo) {
            PullRows r;
            pull_rows(p, hx, hy, q, r);
#pragma unroll
            for (int i = 0; i < Q; ++i) cp_async<sizeof(P)>(bb + i * NS + NT + tid, dir_src(pl, r, i));
        }
        cp_async_commit();
    };
    // moments of the node in slot `slot` of buffer sb (the pressure tensor only for
    // tile nodes: halo nodes contribute Q~ alone)
    auto slot_moments = [&](int sb, int slot, Moments<R>& m, auto full) {
        const P* bb = buf + (size_t)sb * Q * NS + slot;
        if constexpr (DEV) {   // sums straight from the stored pairs
            node_moments_stored<kD, kST, decltype(full)::value, CAL>([&](int i) { return bb[i * NS]; }, p, m);
        } else {
            R f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) Cd::dec(bb[i * NS], f[i], g[i]);
            node_moments<kD, R, decltype(full)::value, DEV, CAL>(f, g, p, m);
        }
    };
    using Full = std::true_type;
    using Lite = std::false_type;
    // pref > 0: plane q's pulled source windows are prefetched into L2 `pref` planes
    // before their cp.async copies are issued (one tensor-prefetch box per direction,
    // issued by lanes of the last warp, which has no halo work), so that the copies of
    // the plane buffer find their lines in L2.  The box for direction i (pmap: TX x TY+2
    // pairs) covers the tile's own columns x0 .. x0 + TX - 1 and rows y0 - 1 - c_y ..
    // y0 + TY - c_y of source plane q - c_z.  The columns the pulls take beyond the tile
    // (x0 - 1 - c_x, x0 + TX - c_x) are left to the neighbouring tiles' boxes: a box
    // widened to them must start on a 16-byte boundary and then carries whole lines of
    // the neighbours' columns, which in FP32 cost 15 % more DRAM reads and 11 % of the step.
    const int pf_lane = tid - (NT - 32);
    auto prefetch_plane = [&](int q) {
        if (pf_lane >= 0 && pf_lane < Q) {
            const int i = pf_lane, b = (i / 3) % 3, c = i / 9;
            // x0 is a multiple of TX (x0 * pair size a multiple of 16 bytes); rows clamped
            tma_prefetch_3d(&pmap, x0, max(y0 - b, 0), i * p.nz + map_axis(q + 1 - c, p.nz, p.per_z));
        }
    };

    Acc5 acc;
    acc.zero();
    bool bad = false;

    // prologue: Q~_zzz below the segment, planes zb and zb+1 in flight, moments of zb
    R qz_prev = R(0), qz_cur = R(0), qz_next = R(0);
    if (active) qz_prev = direct_anomaly_z<CAL>(p, src, x, y, map_axis(zb - 1, p.nz, p.per_z));
    for (int d = 2; d < 2 + pref && zb + d <= ze; ++d) prefetch_plane(map_axis(zb + d, p.nz, p.per_z));
    issue_plane(zb, 0, true);
    issue_plane(map_axis(zb + 1, p.nz, p.per_z), 1 % NB, zb + 1 < ze);
    Moments<R> m_cur, m_next;
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    if (active) {
        slot_moments(0, tid, m_cur, Full());
        QX(0, ty, tx + 1) = anomaly(m_cur.rho, m_cur.ux, m_cur.T);
        QY(0, ty + 1, tx) = anomaly(m_cur.rho, m_cur.uy, m_cur.T);
        qz_cur = anomaly(m_cur.rho, m_cur.uz, m_cur.T);
    }
    if (has_halo) {
        Moments<R> hm;
        slot_moments(0, NT + tid, hm, Lite());
        if (haxis == 1) QY(0, hsy, hsx) = anomaly(hm.rho, hm.uy, hm.T);
        else QX(0, hsy, hsx) = anomaly(hm.rho, hm.ux, hm.T);
    }

    for (int z = zb; z < ze; ++z) {
        const int k = z - zb;
        const int bq = k & 1;               // Q~ buffer of plane z
        const int sz = k % NB;              // population buffer of plane z
        const int sn = (k + 1) % NB;        // ... of plane z+1
        const bool last = (z + 1 == ze);
        cp_async_wait_all();
        __syncthreads();

        // EARLY: plane z is read into registers and plane z+2 requested before the
        // moments of plane z+1, so the copy overlaps them too (both planes are live
        // in registers meanwhile, which only a one-CTA-per-SM launch affords)
        P pk[Q];   // the pulled pairs of plane z, as stored
        if (pref > 0 && z + 2 + pref <= ze) prefetch_plane(map_axis(z + 2 + pref, p.nz, p.per_z));
        if (EARLY) {
            if (active) {
                const P* bb = buf + (size_t)sz * Q * NS + tid;
#pragma unroll
                for (int i = 0; i < Q; ++i) pk[i] = bb[i * NS];
            }
            if (z + 2 <= ze) issue_plane(map_axis(z + 2, p.nz, p.per_z), sz, z + 2 < ze);
        }

        if (active) {
            slot_moments(sn, tid, m_next, Full());
            qz_next = anomaly(m_next.rho, m_next.uz, m_next.T);
            if (!last) {
                QX(bq ^ 1, ty, tx + 1) = anomaly(m_next.rho, m_next.ux, m_next.T);
                QY(bq ^ 1, ty + 1, tx) = anomaly(m_next.rho, m_next.uy, m_next.T);
            }
        }
        if (!last && has_halo) {
            Moments<R> hm;
            slot_moments(sn, NT + tid, hm, Lite());
            if (haxis == 1) QY(bq ^ 1, hsy, hsx) = anomaly(hm.rho, hm.uy, hm.T);
            else QX(bq ^ 1, hsy, hsx) = anomaly(hm.rho, hm.ux, hm.T);
        }

        if (!EARLY) {
            if (active) {
                const P* bb = buf + (size_t)sz * Q * NS + tid;
#pragma unroll
                for (int i = 0; i < Q; ++i) pk[i] = bb[i * NS];
            }
            if (z + 2 <= ze) issue_plane(map_axis(z + 2, p.nz, p.per_z), sz, z + 2 < ze);
        }
        if (active) {
            bad |= nonphysical(m_cur);
            const R Dx = dQ(p.deriv, m_cur.ux, QX(bq, ty, tx), QX(bq, ty, tx + 1), QX(bq, ty, tx + 2));
            const R Dy = dQ(p.deriv, m_cur.uy, QY(bq, ty, tx), QY(bq, ty + 1, tx), QY(bq, ty + 2, tx));
            const R Dz = dQ(p.deriv, m_cur.uz, qz_prev, qz_cur, qz_next);
            R v[5];
            node_totals(m_cur, m_cur.rE, v);
            acc.add(v);
            // collide and store pair by pair, decoding each just before its update
            Relax<kD, R, DEV, CAL> rx;
            rx.init(m_cur, Dx, Dy, Dz, p);
            const unsigned n = (unsigned)node_index(p, x, y, z);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                R f, g;
                Cd::dec(pk[i], f, g);
                if constexpr (kFFMA2) {
                    const float2 o = rx.fg(i, make_float2(f, g), p);
                    store_pair(pl.dst[i] + n, Cd::enc(o.x, o.y));
                } else {
                    store_pair(pl.dst[i] + n, Cd::enc(rx.f(i, f, p), rx.g(i, g, p)));
                }
            }
        }
        m_cur = m_next;
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
    cp_async_wait_all();
    flag_if(bad, status);
    R tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) tot[k] = acc.s[k] - acc.c[k];
    block_sum5_warp(tot, partials + 5 * (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
}

// ---------------------------------------------------------------------------
// D3Q27 with tensor-copy (TMA) plane staging
// ---------------------------------------------------------------------------
// The tensor-copy engine (cp.async.bulk.tensor, the TMA unit) moves a box of a direction
// plane from global to shared memory; the copies of one plane count their bytes on an
// mbarrier, which the consuming threads wait on.
__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return static_cast<unsigned>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival that also announces `bytes` of copies for the current phase.
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
// One arrival, made when this thread's earlier cp.async copies have landed (counts as
// one of the arrivals the mbarrier was initialised with).
__device__ __forceinline__ void mbar_arrive_cp_async(unsigned bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Waits for the phase of parity `parity` to complete, for at most about one second;
// false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}
// Box {x, y, w} of a rank-3 tensor map into shared memory (128-byte aligned), completing
// on the mbarrier.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y, int w,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(w), "r"(bar)
        : "memory");
}

// Shared-memory plan of the TMA-staged kernel.  For every direction i the buffer of
// plane q holds a box of RB rows x BW columns of the SOURCE plane q - c_z: rows
// y0 - 1 - c_y ... y0 + TY - c_y and columns x0 - XO ... x0 + TX + XO - 1, so that node
// (x, y) of the tile and its halo ring finds its pulled pair of direction i at box row
// y - y0 + 1 and column x - x0 + XO - c_x (one box element per destination node and
// direction).  XO keeps the box's first column 16-byte aligned; each box starts on a
// 128-byte boundary (BOXP elements apart).
template <int TY>
struct Tma {
    static constexpr int XO = 16 / (int)sizeof(P);
    static constexpr int BW = TX + 2 * XO;
    static constexpr int RB = TY + 2;
    static constexpr int BOX = RB * BW;
    static constexpr int BOXP = ((BOX * (int)sizeof(P) + 127) / 128) * 128 / (int)sizeof(P);
    static constexpr unsigned plane_bytes = (unsigned)(Q * BOX * sizeof(P));   // bytes the 27 boxes deliver
    static constexpr size_t buf_bytes = (size_t)2 * Q * BOXP * sizeof(P);
    static constexpr size_t q_bytes = (size_t)2 * (TY * (TX + 2) + (TY + 2) * TX) * sizeof(R);
    static constexpr size_t smem_bytes = buf_bytes + q_bytes + 2 * sizeof(unsigned long long);
};

// D3Q27, pipelined on tensor copies.  The same march as fused3d_kernel (a TX x TY
// column over a z segment, two plane buffers, plane z+2 requested while plane z+1's
// moments and plane z's collision run), with a plane's arrival counted on one mbarrier.
// A CTA whose boxes lie inside the grid for every direction requests a plane as 27
// tensor copies (one box per direction, issued by six threads of each of warps 3..7)
// and one thread announces their bytes; a CTA at an x or y face, where a box would wrap
// around a periodic axis or clamp at a zero-gradient one, copies each pulled pair with
// cp.async into the same box positions (the boundary map resolves the source), and each
// thread arrives when its copies have landed.  Per plane z:
//   wait for plane z+1's phase; read the pairs of plane z into registers; barrier
//   (every thread has read plane z's buffer; the Q~ arrays are free); request plane
//   z+2 into plane z's buffer; moments of plane z+1 (tile and halo) -> Q~; collide
//   plane z and store.
// A wait that gives up (about one second) latches kStatusTimeoutBit, and the CTA stops
// after waiting, again bounded, for the copies it still has in flight.
// A selectable schedule: at 256^3 it runs level with fused3d_kernel (within 1 %).  It
// executes fewer instructions and waits far less at the plane barrier, but the boxes
// carry 11-19 % more pairs than the pulls use (corners, and the columns that keep the
// box 16-byte aligned) and the kernel draws 12-25 % more DRAM reads.
#ifndef ELBM_PREF_TMA
#define ELBM_PREF_TMA 0   // measured: FP32 11.16 -> 10.95 GLUPS with it at 256^3, FP16 19.3 -> 19.5
#endif
constexpr bool kPrefTma = ELBM_PREF_TMA;

template <int TY, int MINB, int DD, bool CAL>
__global__ void __launch_bounds__(TX * TY, MINB)
fused3d_tma_kernel(const __grid_constant__ KParams p, const __grid_constant__ DirPlanes pl,
                   const __grid_constant__ CUtensorMap tmap, const P* __restrict__ src,
                   double* __restrict__ partials, int* __restrict__ status) {
    using TT = Tma<TY>;
    static_assert(sizeof(R) == 4 && DD == 3, "the TMA-staged kernel is D3Q27 in FP32 arithmetic");
    constexpr int NT = TX * TY, NH = 2 * TX + 2 * TY, XO = TT::XO, BW = TT::BW, BOXP = TT::BOXP;
    static_assert(NT >= 96 + 5 * 32, "tensor copies are issued by warps 3..7");
    extern __shared__ __align__(128) unsigned char tma_smem[];   // tensor-copy destinations: 128-byte aligned
    P* buf = reinterpret_cast<P*>(tma_smem);                                // [2][Q][BOXP]
    R* qxs = reinterpret_cast<R*>(tma_smem + TT::buf_bytes);                // [2][TY][TX+2]
    R* qys = qxs + 2 * TY * (TX + 2);                                       // [2][TY+2][TX]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(tma_smem + TT::buf_bytes + TT::q_bytes);
    auto QX = [&](int b, int row, int col) -> R& { return qxs[(b * TY + row) * (TX + 2) + col]; };
    auto QY = [&](int b, int row, int col) -> R& { return qys[(b * (TY + 2) + row) * TX + col]; };

    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * p.tz, ze = min(zb + p.tz, p.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    const int xl = min(x0 + TX, p.nx) - 1 - x0, yl = min(y0 + TY, p.ny) - 1 - y0;
    const int nslot = (ty + 1) * BW + tx + XO;   // this node in a direction's box (before -c_x)
    // every box of this CTA inside the grid: columns x0 - XO .. x0 + TX + XO - 1, rows
    // y0 - 2 .. y0 + TY + 1 (the union over c_y)
    const bool boxed = x0 >= XO && x0 + TX + XO <= p.nx && y0 >= 2 && y0 + TY + 1 < p.ny;

    // this thread's halo node: its box position is the unmapped one, or, beyond a
    // zero-gradient face, that of the clamped node it copies (whose pairs the tile node
    // there already brings: such a halo thread copies nothing)
    int hx = 0, hy = 0, hsx = 0, hsy = 0, haxis = 0, hslot = 0;
    const bool has_halo = tid < NH && halo_node<TY>(p, tid, x0, y0, xl, yl, hx, hy, hsx, hsy, haxis);
    bool halo_copies = false;
    if (has_halo) {
        const int ux = haxis == 1 ? x0 + hsx : x0 + hsx - 1;
        const int uy = haxis == 1 ? y0 + hsy - 1 : y0 + hsy;
        const bool clamped = (ux < 0 || ux >= p.nx) ? !p.per_x : ((uy < 0 || uy >= p.ny) ? !p.per_y : false);
        halo_copies = !clamped;
        hslot = ((clamped ? hy : uy) - y0 + 1) * BW + ((clamped ? hx : ux) - x0 + XO);
    }

    unsigned issued = 0u;   // planes requested per buffer: buffer 0 in the low half, 1 in the high
    auto issue_plane = [&](int q, int sb) {
        const unsigned bar = smem_u32(&bars[sb]);
        issued += sb ? 0x10000u : 1u;
        P* bb = buf + (size_t)sb * Q * BOXP;
        if (boxed) {
            if (tid == 0) mbar_expect_tx(bar, TT::plane_bytes + p.inject_tx);
            const int w = (tid >> 5) - 3, lane = tid & 31;
            if (w >= 0 && lane < 6 && 6 * w + lane < Q) {
                const int i = 6 * w + lane;
                const int b = (i / 3) % 3, c = i / 9;
                const int zs = map_axis(q + 1 - c, p.nz, p.per_z);   // q - c_z
                tma_load_3d(smem_u32(bb + (size_t)i * BOXP), &tmap, x0 - XO, y0 - b, i * p.nz + zs, bar);
            }
        } else {
            if (active) {
                PullRows r;
                pull_rows(p, x, y, q, r);
#pragma unroll
                for (int i = 0; i < Q; ++i) cp_async<sizeof(P)>(bb + i * BOXP + nslot - cx_of(i), dir_src(pl, r, i));
            }
            if (halo_copies) {
                PullRows r;
                pull_rows(p, hx, hy, q, r);
#pragma unroll
                for (int i = 0; i < Q; ++i) cp_async<sizeof(P)>(bb + i * BOXP + hslot - cx_of(i), dir_src(pl, r, i));
            }
            mbar_arrive_cp_async(bar);
        }
    };
    auto slot_moments = [&](int sb, int slot, Moments<R>& m, auto full) {
        const P* bb = buf + (size_t)sb * Q * BOXP + slot;
        if constexpr (DEV) {   // sums straight from the stored pairs
            node_moments_stored<kD, kST, decltype(full)::value, CAL>([&](int i) { return bb[i * BOXP - cx_of(i)]; },
                                                                       p, m);
        } else {
            R f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) Cd::dec(bb[i * BOXP - cx_of(i)], f[i], g[i]);
            node_moments<kD, R, decltype(full)::value, DEV, CAL>(f, g, p, m);
        }
    };
    using Full = std::true_type;
    using Lite = std::false_type;

    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), boxed ? 1 : NT);
        mbar_init(smem_u32(&bars[1]), boxed ? 1 : NT);
    }
    __syncthreads();

    Acc5 acc;
    acc.zero();
    bool bad = false, late = false;

    // prologue: Q~_zzz below the segment, planes zb and zb+1 in flight, moments of zb
    R qz_prev = R(0), qz_cur = R(0), qz_next = R(0);
    if (active) qz_prev = direct_anomaly_z<CAL>(p, src, x, y, map_axis(zb - 1, p.nz, p.per_z));
    // L2 prefetch of the plane after the two in flight, by lanes of the last warp, one
    // staging box per direction (ELBM_PREF_TMA, off by default)
    const int pf_lane = tid - (NT - 32);
    auto prefetch_plane = [&](int q) {
        if (kPrefTma && pf_lane >= 0 && pf_lane < Q) {
            const int i = pf_lane, b = (i / 3) % 3, c = i / 9;
            tma_prefetch_3d(&tmap, max(x0 - XO, 0), max(y0 - b, 0), i * p.nz + map_axis(q + 1 - c, p.nz, p.per_z));
        }
    };
    if (zb + 2 <= ze) prefetch_plane(map_axis(zb + 2, p.nz, p.per_z));
    issue_plane(zb, 0);
    issue_plane(map_axis(zb + 1, p.nz, p.per_z), 1);
    Moments<R> m_cur, m_next;
    late |= !mbar_wait(smem_u32(&bars[0]), 0);
    if (active) {
        slot_moments(0, nslot, m_cur, Full());
        QX(0, ty, tx + 1) = anomaly(m_cur.rho, m_cur.ux, m_cur.T);
        QY(0, ty + 1, tx) = anomaly(m_cur.rho, m_cur.uy, m_cur.T);
        qz_cur = anomaly(m_cur.rho, m_cur.uz, m_cur.T);
    }
    if (has_halo) {
        Moments<R> hm;
        slot_moments(0, hslot, hm, Lite());
        if (haxis == 1) QY(0, hsy, hsx) = anomaly(hm.rho, hm.uy, hm.T);
        else QX(0, hsy, hsx) = anomaly(hm.rho, hm.ux, hm.T);
    }

    bool gave_up = false;
    for (int z = zb; z < ze; ++z) {
        const int k = z - zb;
        const int sz = k & 1, sn = sz ^ 1;   // buffers (and Q~ arrays) of planes z and z+1
        const bool last = (z + 1 == ze);
        late |= !mbar_wait(smem_u32(&bars[sn]), ((k + 1) >> 1) & 1);
        P pk[Q];   // the pulled pairs of plane z, as stored
        if (active) {
            const P* bb = buf + (size_t)sz * Q * BOXP + nslot;
#pragma unroll
            for (int i = 0; i < Q; ++i) pk[i] = bb[i * BOXP - cx_of(i)];
        }
        if (__syncthreads_or(late)) {
            gave_up = true;
            break;
        }
        if (z + 3 <= ze) prefetch_plane(map_axis(z + 3, p.nz, p.per_z));
        if (z + 2 <= ze) issue_plane(map_axis(z + 2, p.nz, p.per_z), sz);

        if (active) {
            slot_moments(sn, nslot, m_next, Full());
            qz_next = anomaly(m_next.rho, m_next.uz, m_next.T);
            if (!last) {
                QX(sn, ty, tx + 1) = anomaly(m_next.rho, m_next.ux, m_next.T);
                QY(sn, ty + 1, tx) = anomaly(m_next.rho, m_next.uy, m_next.T);
            }
        }
        if (!last && has_halo) {
            Moments<R> hm;
            slot_moments(sn, hslot, hm, Lite());
            if (haxis == 1) QY(sn, hsy, hsx) = anomaly(hm.rho, hm.uy, hm.T);
            else QX(sn, hsy, hsx) = anomaly(hm.rho, hm.ux, hm.T);
        }
        if (active) {
            bad |= nonphysical(m_cur);
            const R Dx = dQ(p.deriv, m_cur.ux, QX(sz, ty, tx), QX(sz, ty, tx + 1), QX(sz, ty, tx + 2));
            const R Dy = dQ(p.deriv, m_cur.uy, QY(sz, ty, tx), QY(sz, ty + 1, tx), QY(sz, ty + 2, tx));
            const R Dz = dQ(p.deriv, m_cur.uz, qz_prev, qz_cur, qz_next);
            R v[5];
            node_totals(m_cur, m_cur.rE, v);
            acc.add(v);
            Relax<kD, R, DEV, CAL> rx;
            rx.init(m_cur, Dx, Dy, Dz, p);
            const unsigned n = (unsigned)node_index(p, x, y, z);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                R f, g;
                Cd::dec(pk[i], f, g);
                if constexpr (kFFMA2) {
                    const float2 o = rx.fg(i, make_float2(f, g), p);
                    store_pair(pl.dst[i] + n, Cd::enc(o.x, o.y));
                } else {
                    store_pair(pl.dst[i] + n, Cd::enc(rx.f(i, f, p), rx.g(i, g, p)));
                }
            }
        }
        m_cur = m_next;
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
    if (gave_up) {
        // the last phase of each buffer may still have copies in flight
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const unsigned n = b ? issued >> 16 : issued & 0xffffu;
            if (n) mbar_wait(smem_u32(&bars[b]), (n - 1) & 1);
        }
        if (tid == 0) atomicOr(status, kStatusTimeoutBit);
    }
    cp_async_wait_all();
    flag_if(bad, status);
    R tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) tot[k] = acc.s[k] - acc.c[k];
    block_sum5_warp(tot, partials + 5 * (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
}

// D3Q27 without plane buffers: for plane z it computes Q~ of plane z+1 (tile + halo)
// from a first gather, then gathers plane z again (an L2 hit) to collide it.
template <int TY, bool CAL>
__global__ void __launch_bounds__(TX * TY, 2)
fused3d_reread_kernel(const __grid_constant__ KParams p, const P* __restrict__ src, P* __restrict__ dst,
                      double* __restrict__ partials, int* __restrict__ status) {
    __shared__ R qx[2][TY][TX + 2];
    __shared__ R qy[2][TY + 2][TX];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + TX * ty;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zb = blockIdx.z * p.tz, ze = min(zb + p.tz, p.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool active = x < p.nx && y < p.ny;
    const int xl = min(x0 + TX, p.nx) - 1 - x0, yl = min(y0 + TY, p.ny) - 1 - y0;
    int hx = 0, hy = 0, hsx = 0, hsy = 0, haxis = 0;
    const bool has_halo = tid < 2 * TX + 2 * TY && halo_node<TY>(p, tid, x0, y0, xl, yl, hx, hy, hsx, hsy, haxis);

    // Q~ of the tile and its halo in plane z -> buffer b; returns Q~_zzz of (x, y, z)
    auto plane_moments = [&](int z, int b, bool with_xy) -> R {
        R qz = R(0);
        if (active) {
            PullRows r;
            pull_rows(p, x, y, z, r);
            R f[Q], g[Q];
            gather(p, src, r, f, g);
            Moments<R> m;
            node_moments<kD, R, false, DEV, CAL>(f, g, p, m);
            if (with_xy) {
                qx[b][ty][tx + 1] = anomaly(m.rho, m.ux, m.T);
                qy[b][ty + 1][tx] = anomaly(m.rho, m.uy, m.T);
            }
            qz = anomaly(m.rho, m.uz, m.T);
        }
        if (with_xy && has_halo) {
            PullRows r;
            pull_rows(p, hx, hy, z, r);
            R f[Q], g[Q];
            gather(p, src, r, f, g);
            Moments<R> m;
            node_moments<kD, R, false, DEV, CAL>(f, g, p, m);
            if (haxis == 1) qy[b][hsy][hsx] = anomaly(m.rho, m.uy, m.T);
            else qx[b][hsy][hsx] = anomaly(m.rho, m.ux, m.T);
        }
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
            node_moments<kD, R, true, DEV, CAL>(f, g, p, m);
            bad |= nonphysical(m);
            const R Dx = dQ(p.deriv, m.ux, qx[b][ty][tx], qx[b][ty][tx + 1], qx[b][ty][tx + 2]);
            const R Dy = dQ(p.deriv, m.uy, qy[b][ty][tx], qy[b][ty + 1][tx], qy[b][ty + 2][tx]);
            const R Dz = dQ(p.deriv, m.uz, qz_prev, qz_cur, qz_next);
            R v[5];
            node_totals(m, m.rE, v);
            acc.add(v);
            collide<kD, R, DEV, CAL>(f, g, m, Dx, Dy, Dz, p);
            store_node(p, dst, node_index(p, x, y, z), f, g);
        }
        qz_prev = qz_cur;
        qz_cur = qz_next;
    }
    flag_if(bad, status);
    R tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) tot[k] = acc.s[k] - acc.c[k];
    block_sum5_warp(tot, partials + 5 * (blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)));
}

// ---------------------------------------------------------------------------
// D2Q9, row march
// ---------------------------------------------------------------------------
// The two-dimensional form of the pipelined D3Q27 kernel: a CTA of W threads owns a
// strip of W nodes of a row and marches along y over a segment of rows [y0, ye); the
// row plays the part of the plane.  For every row it needs the pulled pairs of its W
// nodes and of the two nodes at the strip's ends (the halo of the x derivative);
// they are copied with cp.async into one of two shared-memory row buffers one row ahead
// ([direction][slot], slot 0 the left end, 1..W the strip, W+1 or the ragged end + 1
// the right end).  Each thread copies and reads only its own slots; the Q~_xxx row
// (double-buffered by row parity) is the only shared array, so one barrier per row
// orders it.  Q~_yyy of the rows below, at and above the current one rolls in registers.
// Per row y: wait for this thread's copies of row y+1; barrier; read row y's pairs into
// registers and request row y+2 into their slots; moments of row y+1 (strip and ends)
// -> Q~ (registers kept for the next row); collide row y and store.  Every population
// leaves HBM once per step; a segment re-reads about two rows (the row below it and
// the row above it).
template <int W, int NB = 2>
struct March2 {
    static constexpr int NS = W + 2;
    static constexpr int NBUF = NB;   // row buffers: rows y (collide), y+1 (moments), up to y+NB-1 in flight
    static constexpr size_t buf_bytes = (size_t)NB * Q * NS * sizeof(P);
    static constexpr size_t q_bytes = (size_t)2 * NS * sizeof(R);
    static constexpr size_t smem_bytes = buf_bytes + q_bytes;
};

// Per-direction plane bases of one lattice's stores: from the kernel parameters (one
// lattice), or formed from the instance's base (ensemble).
struct PlanesParam {
    const DirPlanes* pl;
    const P* base;
    __device__ __forceinline__ const P* s(int i) const { return pl->src[i]; }
    __device__ __forceinline__ P* d(int i) const { return pl->dst[i]; }
};
struct PlanesBase {
    const P* src;
    P* dst;
    size_t N;
    const P* base;
    __device__ __forceinline__ const P* s(int i) const { return src + (size_t)i * N; }
    __device__ __forceinline__ P* d(int i) const { return dst + (size_t)i * N; }
};

// Q~_yyy of node (x, y) (y mapped) by a direct gather, with the fixed-state pairs where
// its pulls cross a fixed face (used once per segment).
template <bool CAL>
__device__ __forceinline__ R direct_anomaly_y(const KParams& p, const P* __restrict__ src, int x, int y) {
    PullRows r;
    pull_rows(p, x, y, 0, r);
    R f[Q], g[Q];
    gather(p, src, r, f, g);
    Moments<R> m;
    node_moments<kD, R, false, DEV, CAL>(f, g, p, m);
    return anomaly(m.rho, m.uy, m.T);
}

// FIX = false compiles the march for grids without fixed-state faces: the face tests and
// the per-direction substitutions fold away (FP16 store at 4096^2: 46.7 -> 50.0 GLUPS,
// 80 -> 72 registers, seven CTAs per SM instead of six).
template <int W, int NB, bool CAL, bool FIX, class PL>
__device__ __forceinline__ void march2d_segment(const KParams& p, const PL& pl, int x0, int y0, int ye,
                                                unsigned char* smem, Acc5& acc, bool& bad) {
    using MC = March2<W, NB>;
    static_assert(NB == 2 || NB == 3, "two or three row buffers");
    constexpr int NS = MC::NS;
    P* buf = reinterpret_cast<P*>(smem);                   // [NB][Q][NS]
    R* qxs = reinterpret_cast<R*>(smem + MC::buf_bytes);   // [2][NS]
    const int t = threadIdx.x;
    const int x = x0 + t;
    const bool active = x < p.nx;
    const int xl = min(x0 + W, p.nx) - 1 - x0;   // last local column of the strip
    const int nslot = t + 1;
    // the strip's ends: thread 0 the left one (slot 0), thread 1 the right one (slot xl + 2);
    // beyond a fixed-state face an end carries the fixed state's Q~ and is not copied
    const bool has_halo = t < 2;
    const int hux = t == 0 ? x0 - 1 : x0 + xl + 1;
    const int hx = map_axis(hux, p.nx, p.per_x);
    const bool fixed_faces = FIX && p.has_fixed;
    const bool hfixed = has_halo && fixed_faces && beyond_fixed(p, 0, hux, p.nx);
    const int hslot = t == 0 ? 0 : xl + 2;

    auto issue_row = [&](int yq, int sb, bool with_halo) {   // yq already mapped
        P* bb = buf + (size_t)sb * Q * NS;
        if (active) {
            PullRows r;
            pull_rows(p, x, yq, 0, r);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                cp_async<sizeof(P)>(bb + i * NS + nslot, pl.s(i) + (unsigned)(r.row[(i / 3) % 3][1] + r.xs[i % 3]));
        }
        if (with_halo && has_halo && !hfixed) {
            PullRows r;
            pull_rows(p, hx, yq, 0, r);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                cp_async<sizeof(P)>(bb + i * NS + hslot, pl.s(i) + (unsigned)(r.row[(i / 3) % 3][1] + r.xs[i % 3]));
        }
        cp_async_commit();
    };
    // moments of the node in slot `slot` of buffer sb; gm marks the pairs that are the
    // fixed state's (pulled across a fixed face)
    auto row_moments = [&](int sb, int slot, unsigned gm, Moments<R>& m, auto full) {
        const P* bb = buf + (size_t)sb * Q * NS + slot;
        if constexpr (DEV) {
            if (!gm) {   // sums straight from the stored pairs
                node_moments_stored<kD, kST, decltype(full)::value, CAL>([&](int i) { return bb[i * NS]; }, p, m);
                return;
            }
        }
        R f[Q], g[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) Cd::dec(bb[i * NS], f[i], g[i]);
        if (gm) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if ((gm >> i) & 1u) fixed_pair(p, i, f[i], g[i]);
        }
        node_moments<kD, R, decltype(full)::value, DEV, CAL>(f, g, p, m);
    };
    using Full = std::true_type;
    using Lite = std::false_type;
    auto QX = [&](int b, int slot) -> R& { return qxs[b * NS + slot]; };
    auto halo_q = [&](int sb, int yq) {
        if (hfixed) return fixed_Q(p, 0);
        Moments<R> hm;
        row_moments(sb, hslot, fixed_mask<FIX>(p, hx, yq), hm, Lite());
        return anomaly(hm.rho, hm.ux, hm.T);
    };

    // prologue: Q~_yyy of the row below the segment, rows y0 and y0+1 in flight, moments of y0
    R qy_prev = R(0), qy_cur = R(0), qy_next = R(0);
    if (active) {
        if (fixed_faces && beyond_fixed(p, 1, y0 - 1, p.ny)) qy_prev = fixed_Q(p, 1);
        else qy_prev = direct_anomaly_y<CAL>(p, pl.base, x, map_axis(y0 - 1, p.ny, p.per_y));
    }
    // rows y0 .. y0+NB-1 in flight (a row past ye is not needed; its group stays empty)
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (y0 + j <= ye) issue_row(map_axis(y0 + j, p.ny, p.per_y), j, y0 + j < ye);
        else cp_async_commit();
    }
    Moments<R> m_cur, m_next;
    cp_async_wait_pending<NB - 1>();   // row y0 has landed
    __syncthreads();
    if (active) {
        row_moments(0, nslot, fixed_mask<FIX>(p, x, y0), m_cur, Full());
        QX(0, nslot) = anomaly(m_cur.rho, m_cur.ux, m_cur.T);
        qy_cur = anomaly(m_cur.rho, m_cur.uy, m_cur.T);
    }
    if (has_halo) QX(0, hslot) = halo_q(0, y0);

    for (int y = y0; y < ye; ++y) {
        const int k = y - y0;
        const int bq = k & 1;                          // Q~ row of y (y+1: bq ^ 1)
        const int sz = k % NB, sn = (k + 1) % NB;      // row buffers of rows y and y+1
        const bool last = (y + 1 == ye);
        cp_async_wait_pending<NB - 2>();               // row y+1 has landed (y+2.. may be in flight)
        __syncthreads();
        P pk[Q];   // the pulled pairs of row y, as stored
        if (active) {
            const P* bb = buf + (size_t)sz * Q * NS + nslot;
#pragma unroll
            for (int i = 0; i < Q; ++i) pk[i] = bb[i * NS];
        }
        if (y + NB <= ye) issue_row(map_axis(y + NB, p.ny, p.per_y), sz, y + NB < ye);
        else cp_async_commit();   // keep one group per row for the wait count

        const int yn = map_axis(y + 1, p.ny, p.per_y);
        if (active) {
            if (fixed_faces && beyond_fixed(p, 1, y + 1, p.ny)) {
                qy_next = fixed_Q(p, 1);   // the last row of the grid: nothing after it
            } else {
                row_moments(sn, nslot, fixed_mask<FIX>(p, x, yn), m_next, Full());
                qy_next = anomaly(m_next.rho, m_next.uy, m_next.T);
                if (!last) QX(bq ^ 1, nslot) = anomaly(m_next.rho, m_next.ux, m_next.T);
            }
        }
        if (!last && has_halo) QX(bq ^ 1, hslot) = halo_q(sn, yn);

        if (active) {
            bad |= nonphysical(m_cur);
            const R Dx = dQ(p.deriv, m_cur.ux, QX(bq, nslot - 1), QX(bq, nslot), QX(bq, nslot + 1));
            const R Dy = dQ(p.deriv, m_cur.uy, qy_prev, qy_cur, qy_next);
            R v[5];
            node_totals(m_cur, m_cur.rE, v);
            acc.add(v);
            Relax<kD, R, DEV, CAL> rx;
            rx.init(m_cur, Dx, Dy, R(0), p);
            const unsigned gm = fixed_mask<FIX>(p, x, y);
            const unsigned n = (unsigned)(x + p.nx * y);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                R f, g;
                Cd::dec(pk[i], f, g);
                if ((gm >> i) & 1u) fixed_pair(p, i, f, g);
                pl.d(i)[n] = Cd::enc(rx.f(i, f, p), rx.g(i, g, p));
            }
        }
        m_cur = m_next;
        qy_prev = qy_cur;
        qy_cur = qy_next;
    }
    cp_async_wait_all();
    __syncthreads();   // the shared buffers are reused by the next segment of a persistent CTA
}

// One lattice: CTA (bx, by) marches strip bx over rows [by * p.tz, min((by + 1) * p.tz, ny)).
#ifndef ELBM_MARCH_MINB
#define ELBM_MARCH_MINB 0
#endif
#if ELBM_MARCH_MINB > 0
#define ELBM_MARCH_BOUNDS(W) __launch_bounds__(W, ELBM_MARCH_MINB)
#else
#define ELBM_MARCH_BOUNDS(W) __launch_bounds__(W)
#endif
template <int W, int NB, bool CAL, bool FIX>
__global__ void ELBM_MARCH_BOUNDS(W)
march2d_kernel(const __grid_constant__ KParams p, const __grid_constant__ DirPlanes pl, const P* __restrict__ src,
               double* __restrict__ partials, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char march_smem[];
    const int x0 = blockIdx.x * W, y0 = blockIdx.y * p.tz, ye = min(y0 + p.tz, p.ny);
    Acc5 acc;
    acc.zero();
    bool bad = false;
    march2d_segment<W, NB, CAL, FIX>(p, PlanesParam{&pl, src}, x0, y0, ye, march_smem, acc, bad);
    flag_if(bad, status);
    R tot[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) tot[k] = acc.s[k] - acc.c[k];
    block_sum5_warp(tot, partials + 5 * (blockIdx.x + gridDim.x * blockIdx.y));
}

// Persistent ensemble step on the row march: the work list holds (instance, strip, segment)
// units (instance k owns units [tile_start[k], tile_start[k+1]), tiles_x[k] strips per
// segment row); CTA b takes units b, b + gridDim.x, ...  No totals are kept.
template <int W, int NB, bool CAL>
__global__ void __launch_bounds__(W)
ensemble_march2d_kernel(const EnsembleArgs a, const P* __restrict__ src, P* __restrict__ dst, int seg,
                        int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char march_smem[];
    __shared__ int s_start[kMaxEnsemble + 1];
    __shared__ int s_tx[kMaxEnsemble];
    for (int k = threadIdx.x; k <= a.n; k += W) s_start[k] = a.tile_start[k];
    for (int k = threadIdx.x; k < a.n; k += W) s_tx[k] = a.tiles_x[k];
    __syncthreads();
    bool bad = false;
    Acc5 acc;
    acc.zero();
    int k = 0;
    for (int u = blockIdx.x; u < a.ntiles; u += gridDim.x) {
        while (u >= s_start[k + 1]) ++k;   // u increases, so k only moves forward
        const int local = u - s_start[k];
        const int bx = local % s_tx[k], by = local / s_tx[k];
        const KParams& p = a.params[k];
        const long long off = a.offset[k];
        const int y0 = by * seg;
        march2d_segment<W, NB, CAL, true>(p, PlanesBase{src + off, dst + off, (size_t)p.N, src + off}, bx * W, y0,
                                min(y0 + seg, p.ny), march_smem, acc, bad);
    }
    flag_if(bad, status);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
constexpr int kThreads = kThreads1D;
constexpr int kTY2 = 8;                  // D2Q9 tile kernel: 32 x 8 tiles
constexpr int kW2 = kMarchW2;            // D2Q9 row march: strips of kW2 nodes
#ifndef ELBM_MARCH_NB
#define ELBM_MARCH_NB 2
#endif
constexpr int kNBM = ELBM_MARCH_NB;      // row buffers of the march (2: one row in flight, 3: two)
using MarchCfg = March2<kW2, kNBM>;
// Strip width of the single-lattice D2Q9 march: 256 nodes for the 16-bit stores, whose
// march is issue-bound and pays for the strip's two halo nodes half as often per node
// (FP16 at 4096^2: 52.8 -> 55.2 GLUPS), kW2 for FP32 and FP64, which are bandwidth-bound
// (256 measured 39.2 against 44.9 GLUPS in FP32).  The persistent ensemble keeps kW2.
#ifndef ELBM_MARCH_W16
#define ELBM_MARCH_W16 256
#endif
constexpr int kW2L = sizeof(P) == 4 ? ELBM_MARCH_W16 : kW2;
using MarchCfgL = March2<kW2L, kNBM>;
#ifndef ELBM_TY3
#define ELBM_TY3 8
#endif
constexpr int kTY3 = ELBM_TY3;           // D3Q27 re-read and tensor-copy kernels: tiles 32 x kTY3
// Pipelined (cp.async) D3Q27 kernel: tiles 32 x kTYP.  Taller FP32 tiles (more warps per
// SM, relatively fewer halo nodes) measured slower at 256^3: 10 rows 7 %, 12 rows 37 %
// (their plane buffers leave the L1 cache that the 8-byte cp.async copies go through
// 60 KB and 28 KB instead of about 90 KB, and cap the registers at 168); 8 it is.
#ifndef ELBM_TYP_F32
#define ELBM_TYP_F32 8
#endif
constexpr int kTYP = (kST == ST_F32) ? ELBM_TYP_F32 : kTY3;
constexpr int kTotalsBlocks = 2 * 152;   // totals_kernel grid (grid-stride)
// Pipelined D3Q27 kernel per store: two plane buffers.  FP32 pairs make them 145 KB
// (one CTA per SM, up to 255 registers; a third buffer would leave L1 almost no
// room and measured 35 % slower); FP16/BF16 pairs are half the size (two CTAs per
// SM); FP64 uses the re-read kernel (its plane buffers would not fit).  With one CTA
// per SM the registers also hold plane z while plane z+1's moments are computed, so
// the prefetch of plane z+2 starts one phase earlier (EARLY; 10 % faster at 256^3;
// with two CTAs per SM and 128 registers it measured 1 % slower).
#ifndef ELBM_PIPE_NB_F32
#define ELBM_PIPE_NB_F32 2
#endif
#ifndef ELBM_PIPE_NB_F16
#define ELBM_PIPE_NB_F16 2
#endif
constexpr bool kPipe = (kST != ST_F64);
constexpr int kNB = (kST == ST_F32) ? ELBM_PIPE_NB_F32 : ELBM_PIPE_NB_F16;
constexpr int kMinB = (PipeBytes<kTYP, kNB>::value * 2 + 2048 <= 228 * 1024) ? 2 : 1;
using PipeCfg = Pipe<kTYP, kNB>;
#ifndef ELBM_EARLY
#define ELBM_EARLY 1
#endif
constexpr bool kEarly = ELBM_EARLY && kMinB == 1;
// TMA-staged D3Q27 kernel: FP32 plane buffers (155 KB) leave room for one CTA per SM,
// FP16/BF16 ones (88 KB) for two.
using TmaCfg = Tma<kTY3>;
constexpr int kTmaMinB = (TmaCfg::smem_bytes * 2 + 4096 <= 228 * 1024) ? 2 : 1;

// Can the TMA-staged kernel run this grid?  The tensor map's row pitch nx * pair size
// must be a multiple of 16 bytes (nx a multiple of 2 for FP32 pairs, 4 for FP16/BF16).
int tma_supported(const KParams& p) {
    if (kD != 3 || !kPipe) return 0;
    return p.nx % TmaCfg::XO == 0 && !p.has_fixed;
}

// Tensor map of a population store as rank 3: x (nx pairs), y (ny), w = i * nz + z (the
// planes of all directions); box TmaCfg::BW x RB x 1 (kTmapStage: the TMA-staged
// kernel's copies) or TX x kTYP + 2 x 1 (kTmapPrefetch: the default pipelined kernel's
// L2 prefetch of a tile's source rows).  The encoder is the driver's, reached through
// the runtime (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();   // leave no sticky error behind
        return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
}

int encode_tmap(const KParams& p, const void* base, CUtensorMap* out, int kind) {
    if (!tma_supported(p) || (kind != kTmapStage && kind != kTmapPrefetch)) return 0;
    static const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();   // resolved once, thread-safe
    if (!encode) return -1;
    const cuuint64_t dims[3] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz * Q};
    const cuuint64_t strides[2] = {(cuuint64_t)p.nx * sizeof(P), (cuuint64_t)p.nx * p.ny * sizeof(P)};
    const cuuint32_t box[3] = {(cuuint32_t)(kind == kTmapStage ? TmaCfg::BW : TX),
                               (cuuint32_t)(kind == kTmapStage ? TmaCfg::RB : kTYP + 2), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUtensorMapDataType dt = sizeof(P) == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
#ifndef ELBM_TMAP_PROMO
#define ELBM_TMAP_PROMO CU_TENSOR_MAP_L2_PROMOTION_L2_128B
#endif
    const CUresult r = encode(out, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              (CUtensorMapL2promotion)ELBM_TMAP_PROMO, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 1 : -1;
}

inline unsigned blocks_1d(long long n) { return (unsigned)blocks_1d_of(n); }

// Per-direction plane bases of both stores for the kernels.
DirPlanes dir_planes(const KParams& p, const void* src, void* dst) {
    DirPlanes pl;
    for (int i = 0; i < Q; ++i) {
        pl.src[i] = (const P*)src + (size_t)i * (size_t)p.N;
        pl.dst[i] = (P*)dst + (size_t)i * (size_t)p.N;
    }
    return pl;
}

// Grid of the default fused kernel: D2Q9 row march (strips x row segments of p.tz rows),
// D3Q27 pipelined kernel (32 x kTYP column tiles x z segments of p.tz planes).
dim3 fused_grid(const KParams& p) {
    if (kD == 2) return dim3((p.nx + kW2L - 1) / kW2L, (p.ny + p.tz - 1) / p.tz, 1);
    const int ty = kPipe ? kTYP : kTY3;
    return dim3((p.nx + TX - 1) / TX, (p.ny + ty - 1) / ty, (p.nz + p.tz - 1) / p.tz);
}
// Grid of the D3Q27 re-read and tensor-copy kernels (32 x kTY3 tiles).
dim3 grid3_ty3(const KParams& p) {
    return dim3((p.nx + TX - 1) / TX, (p.ny + kTY3 - 1) / kTY3, (p.nz + p.tz - 1) / p.tz);
}
// Grid of the D2Q9 tile kernel (the re-read schedule of D2Q9): 32 x kTY2 tiles.
dim3 tile2d_grid(const KParams& p) { return dim3((p.nx + TX - 1) / TX, (p.ny + kTY2 - 1) / kTY2, 1); }

int max_blocks(const KParams& p) {
    long long a = blocks_1d(p.N);
    dim3 gf = fused_grid(p);
    long long b = (long long)gf.x * gf.y * gf.z;
    long long m = a > b ? a : b;
    const dim3 gt = kD == 2 ? tile2d_grid(p) : grid3_ty3(p);
    const long long c = (long long)gt.x * gt.y * gt.z;
    if (c > m) m = c;
    if (m < kTotalsBlocks) m = kTotalsBlocks;
    return (int)m;
}

cudaError_t launch_init(const KParams& p, const double* rho, const double* u, const double* T, void* pop,
                        void* spare, void* qfield, double* partials, int* status, cudaStream_t s,
                        long long* launches) {
    // The stored state is post-collision: after step n the store holds C(X_n), where
    // X_n is the post-stream state of the method and C the collision, and a step is
    // pull (X_{n+1} = S(C(X_n))) followed by collide.  Initialisation therefore writes
    // X_0 = (f^eq, g^eq) into the spare store and collides it in place of streaming.
    // Moments of C(X_n) equal those of X_n (the collision conserves them), so field
    // extraction and totals read each node's own values.
    const unsigned nb = blocks_1d(p.N);
    init_kernel<<<nb, kThreads, 0, s>>>(p, rho, u, T, (P*)spare, status, 0, p.N);
    moments_kernel<false><<<nb, kThreads, 0, s>>>(p, (const P*)spare, (R*)qfield);
    collide_kernel<false><<<nb, kThreads, 0, s>>>(p, (const P*)spare, (P*)pop, (const R*)qfield, partials, status);
    *launches += 3;
    return cudaGetLastError();
}

// f^eq, g^eq of nodes n0 .. n0 + cnt - 1 written in place into pop (fields of those nodes
// only).  For the AA single store this is the first half of initialisation: a step from
// layout L1 (node-local reads, swapped writes) then collides the equilibria without
// streaming, leaving C(X_0) in layout L0.
cudaError_t launch_init_nodes(const KParams& p, const double* rho, const double* u, const double* T, void* pop,
                              long long n0, long long cnt, int* status, cudaStream_t s, long long* launches) {
    init_kernel<<<blocks_1d(cnt), kThreads, 0, s>>>(p, rho, u, T, (P*)pop, status, n0, cnt);
    ++*launches;
    return cudaGetLastError();
}

// rho, u, T of nodes n0 .. n0 + cnt - 1 into fields of cnt nodes.
cudaError_t launch_fields_nodes(const KParams& p, const void* pop, double* rho, double* u, double* T,
                                long long n0, long long cnt, int* status, cudaStream_t s, long long* launches) {
    fields_kernel<<<blocks_1d(cnt), kThreads, 0, s>>>(p, (const P*)pop, rho, u, T, status, n0, cnt);
    ++*launches;
    return cudaGetLastError();
}

// One AA step on the single store A: from layout L1 (node-local reads, swapped writes) or
// from L0 (pulled reads, pushed writes).
cudaError_t launch_step_aa(const KParams& p, void* A, void* qfield, double* partials, int* nblocks, int* status,
                           cudaStream_t s, long long* launches, int from_l1) {
    const unsigned nb = blocks_1d(p.N);
    if (from_l1) {
        aa_moments_kernel<true><<<nb, kThreads, 0, s>>>(p, (P*)A, (R*)qfield);
        aa_collide_kernel<true><<<nb, kThreads, 0, s>>>(p, (P*)A, (const R*)qfield, partials, status);
    } else {
        aa_moments_kernel<false><<<nb, kThreads, 0, s>>>(p, (P*)A, (R*)qfield);
        aa_collide_kernel<false><<<nb, kThreads, 0, s>>>(p, (P*)A, (const R*)qfield, partials, status);
    }
    *launches += 2;
    *nblocks = (int)nb;
    return cudaGetLastError();
}

cudaError_t launch_fields(const KParams& p, const void* pop, double* rho, double* u, double* T, int* status,
                          cudaStream_t s, long long* launches) {
    fields_kernel<<<blocks_1d(p.N), kThreads, 0, s>>>(p, (const P*)pop, rho, u, T, status, 0, p.N);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_twopass(const KParams& p, const void* src, void* dst, void* qfield, double* partials,
                           int* nblocks, int* status, cudaStream_t s, long long* launches) {
    const unsigned nb = blocks_1d(p.N);
    moments_kernel<true><<<nb, kThreads, 0, s>>>(p, (const P*)src, (R*)qfield);
    collide_kernel<true><<<nb, kThreads, 0, s>>>(p, (const P*)src, (P*)dst, (const R*)qfield, partials, status);
    *launches += 2;
    *nblocks = (int)nb;
    return cudaGetLastError();
}

// A template so that the branch of the other lattice is never instantiated; CAL as in
// the kernels (the caloric form only for handles with a Cv(T) model).
#ifndef ELBM_PREF
#define ELBM_PREF 1
#endif
constexpr int kPref = ELBM_PREF;   // planes of L2 prefetch ahead of the cp.async copies (with a tensor map)

template <int DD, bool CAL>
cudaError_t launch_fused_cal(const KParams& p, const void* src, void* dst, double* partials, int* status,
                             cudaStream_t s, bool reread, const CUtensorMap* pmap = nullptr) {
    const dim3 grid = fused_grid(p);
    if constexpr (DD == 2) {
        if (reread || p.tile2d) {   // the tile kernel: one 32 x kTY2 tile per CTA, no march
            fused2d_kernel<kTY2, CAL><<<tile2d_grid(p), dim3(TX, kTY2), 0, s>>>(p, (const P*)src, (P*)dst, partials,
                                                                               status);
        } else {
            auto kern = p.has_fixed ? march2d_kernel<kW2L, kNBM, CAL, true> : march2d_kernel<kW2L, kNBM, CAL, false>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)MarchCfgL::smem_bytes);
            if (e != cudaSuccess) return e;
            DirPlanes pl = dir_planes(p, src, dst);
            kern<<<grid, kW2L, MarchCfgL::smem_bytes, s>>>(p, pl, (const P*)src, partials, status);
        }
    } else {
        bool launched = false;
        if constexpr (kPipe) {
            if (!reread) {
                auto kern = fused3d_kernel<kTYP, kNB, kMinB, kEarly, DD, CAL>;
                // the dynamic shared-memory limit is a per-function attribute; setting it
                // again is cheap and keeps this correct for every device of the process
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)PipeCfg::smem_bytes);
                if (e != cudaSuccess) return e;
                DirPlanes pl = dir_planes(p, src, dst);
                CUtensorMap none;
                std::memset(&none, 0, sizeof(none));
                kern<<<grid, dim3(TX, kTYP), PipeCfg::smem_bytes, s>>>(p, pl, (const P*)src, partials, status,
                                                                       pmap ? *pmap : none, pmap ? kPref : 0);
                launched = true;
            }
        }
        if (!launched)
            fused3d_reread_kernel<kTY3, CAL><<<grid3_ty3(p), dim3(TX, kTY3), 0, s>>>(p, (const P*)src, (P*)dst, partials,
                                                                              status);
    }
    return cudaGetLastError();
}

template <int DD, bool CAL>
cudaError_t launch_tma_cal(const KParams& p, const void* src, void* dst, const CUtensorMap* map, double* partials,
                           int* status, cudaStream_t s) {
    if constexpr (DD == 3 && kPipe) {
        auto kern = fused3d_tma_kernel<kTY3, kTmaMinB, DD, CAL>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TmaCfg::smem_bytes);
        if (e != cudaSuccess) return e;
        DirPlanes pl = dir_planes(p, src, dst);
        kern<<<grid3_ty3(p), dim3(TX, kTY3), TmaCfg::smem_bytes, s>>>(p, pl, *map, (const P*)src, partials, status);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

// TMA-staged fused step; map is the tensor map of src (encode_tmap, kTmapStage).
cudaError_t launch_fused_tma(const KParams& p, const void* src, void* dst, const CUtensorMap* map,
                             double* partials, int* nblocks, int* status, cudaStream_t s, long long* launches) {
    if (!tma_supported(p) || !map) return cudaErrorInvalidValue;
    const cudaError_t e = p.eos ? launch_tma_cal<kD, true>(p, src, dst, map, partials, status, s)
                                : launch_tma_cal<kD, false>(p, src, dst, map, partials, status, s);
    ++*launches;
    const dim3 grid = grid3_ty3(p);
    *nblocks = (int)(grid.x * grid.y * grid.z);
    return e;
}

template <int DD>
cudaError_t launch_fused(const KParams& p, const void* src, void* dst, double* partials, int* nblocks,
                         int* status, cudaStream_t s, long long* launches, bool reread,
                         const CUtensorMap* pmap = nullptr) {
    const cudaError_t e = p.eos ? launch_fused_cal<DD, true>(p, src, dst, partials, status, s, reread, pmap)
                                : launch_fused_cal<DD, false>(p, src, dst, partials, status, s, reread, pmap);
    ++*launches;
    const dim3 grid = DD == 2 ? ((reread || p.tile2d) ? tile2d_grid(p) : fused_grid(p))
                              : ((reread && kPipe) ? grid3_ty3(p) : fused_grid(p));
    *nblocks = (int)(grid.x * grid.y * grid.z);
    return e;
}

cudaError_t launch_fused_default(const KParams& p, const void* src, void* dst, double* partials, int* nblocks,
                                 int* status, cudaStream_t s, long long* launches) {
    return launch_fused<kD>(p, src, dst, partials, nblocks, status, s, launches, false);
}

cudaError_t launch_fused_reread(const KParams& p, const void* src, void* dst, double* partials, int* nblocks,
                                int* status, cudaStream_t s, long long* launches) {
    return launch_fused<kD>(p, src, dst, partials, nblocks, status, s, launches, true);
}

// The default fused step with src's prefetch tensor map at hand (encode_tmap,
// kTmapPrefetch: L2 prefetch of the planes ahead).
cudaError_t launch_fused_pf(const KParams& p, const void* src, void* dst, const CUtensorMap* map, double* partials,
                            int* nblocks, int* status, cudaStream_t s, long long* launches) {
    return launch_fused<kD>(p, src, dst, partials, nblocks, status, s, launches, false, map);
}

template <bool CAL>
cudaError_t launch_ensemble_march(const EnsembleArgs& a, const void* src, void* dst, int* status, int seg, int grid,
                                  cudaStream_t s) {
    auto kern = ensemble_march2d_kernel<kW2, kNBM, CAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)MarchCfg::smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<grid, kW2, MarchCfg::smem_bytes, s>>>(a, (const P*)src, (P*)dst, seg, status);
    return cudaGetLastError();
}

// Persistent ensemble step and `grid` CTAs: ty = 4, 8 or 16 runs one 32 x ty tile per work
// unit; ty = kMarchSegs (32, 64 or 128) runs the row march over strips of kW2 nodes and
// segments of ty rows.
cudaError_t launch_ensemble(const EnsembleArgs& a, const void* src, void* dst, int* status, int ty, int grid,
                            cudaStream_t s, long long* launches) {
    if constexpr (kD == 2) {
        if (ty > 16) {
            ++*launches;
            return a.caloric ? launch_ensemble_march<true>(a, src, dst, status, ty, grid, s)
                             : launch_ensemble_march<false>(a, src, dst, status, ty, grid, s);
        }
        if (a.caloric) {
            if (ty == 4) ensemble2d_kernel<4, true><<<grid, dim3(TX, 4), 0, s>>>(a, (const P*)src, (P*)dst, status);
            else if (ty == 16)
                ensemble2d_kernel<16, true><<<grid, dim3(TX, 16), 0, s>>>(a, (const P*)src, (P*)dst, status);
            else ensemble2d_kernel<8, true><<<grid, dim3(TX, 8), 0, s>>>(a, (const P*)src, (P*)dst, status);
        } else {
            if (ty == 4) ensemble2d_kernel<4, false><<<grid, dim3(TX, 4), 0, s>>>(a, (const P*)src, (P*)dst, status);
            else if (ty == 16)
                ensemble2d_kernel<16, false><<<grid, dim3(TX, 16), 0, s>>>(a, (const P*)src, (P*)dst, status);
            else ensemble2d_kernel<8, false><<<grid, dim3(TX, 8), 0, s>>>(a, (const P*)src, (P*)dst, status);
        }
        ++*launches;
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

// Occupancy (resident CTAs per SM) of the ensemble kernel with tile height ty (or, above
// 16, of the row-march form).
int ensemble_occupancy(int ty) {
    int nb = 0;
    if constexpr (kD == 2) {
        cudaError_t e;
        if (ty > 16) {
            auto kern = ensemble_march2d_kernel<kW2, kNBM, false>;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfg::smem_bytes) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kW2, MarchCfg::smem_bytes) != cudaSuccess)
                return 0;
            return nb;
        }
        // the constant-gamma form (the caloric one differs by a few registers at most)
        if (ty == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ensemble2d_kernel<4, false>, TX * 4, 0);
        else if (ty == 16)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ensemble2d_kernel<16, false>, TX * 16, 0);
        else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ensemble2d_kernel<8, false>, TX * 8, 0);
        if (e != cudaSuccess) return 0;
    }
    return nb;
}

cudaError_t launch_stats(const KParams& p, const void* pop, double* partials, int* nblocks, cudaStream_t s,
                         long long* launches) {
    stats_kernel<<<kTotalsBlocks, kThreads, 0, s>>>(p, (const P*)pop, partials);
    ++*launches;
    *nblocks = kTotalsBlocks;
    return cudaGetLastError();
}

cudaError_t launch_totals(const KParams& p, const void* pop, double* partials, int* nblocks, cudaStream_t s,
                          long long* launches) {
    totals_kernel<<<kTotalsBlocks, kThreads, 0, s>>>(p, (const P*)pop, partials);
    ++*launches;
    *nblocks = kTotalsBlocks;
    return cudaGetLastError();
}

// Resident CTAs per SM of the default fused kernel for grid p (a template so that the
// kernel of the other lattice is never instantiated).
template <int DD>
int fused_occupancy_impl(const KParams& p) {
    int n = 0;
    if constexpr (DD == 3 && kPipe) {
        auto kern = fused3d_kernel<kTYP, kNB, kMinB, kEarly, DD, false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PipeCfg::smem_bytes) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX * kTYP, PipeCfg::smem_bytes) != cudaSuccess)
            return 0;
    } else if constexpr (DD == 3) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused3d_reread_kernel<kTY3, false>, TX * kTY3, 0) !=
            cudaSuccess)
            return 0;
    } else {
        auto kern = p.has_fixed ? march2d_kernel<kW2L, kNBM, false, true> : march2d_kernel<kW2L, kNBM, false, false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MarchCfgL::smem_bytes) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kW2L, MarchCfgL::smem_bytes) != cudaSuccess)
            return 0;
    }
    return n;
}
int fused_occupancy(const KParams& p) { return fused_occupancy_impl<kD>(p); }

const Ops kOps = {kD,          kST,           sizeof(P) / 2,  sizeof(R),            max_blocks,
                  launch_init, launch_fields, launch_twopass, launch_fused_default, launch_fused_reread,
                  launch_totals, launch_ensemble, ensemble_occupancy, launch_stats,
                  kD == 3 ? (kPipe ? kTYP : kTY3) : 1, fused_occupancy, launch_fused_tma, tma_supported, encode_tmap,
                  launch_fused_pf, launch_init_nodes, launch_fields_nodes, launch_step_aa, kW2L};

}  // namespace

#define ELBM_CAT2(a, b) a##b
#define ELBM_CAT(a, b) ELBM_CAT2(a, b)
const Ops* ELBM_CAT(ops_, ELBM_OPS_NAME)() { return &kOps; }

}  // namespace elbm
