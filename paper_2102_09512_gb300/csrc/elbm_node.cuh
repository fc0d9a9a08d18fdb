// Per-node arithmetic of the two-population compressible LB step, for sm_103a.
//
// Everything here acts on the 2Q populations of ONE node held in registers:
// moments (Eqs. density, momentum, energy, P), temperature from the total energy
// (Eqs. U, E with constant Cv = 1/(gamma-1), R = 1), the anomaly Q~_aaa
// (Eq. anomalya), the relaxation rates (Eqs. mu, Pr), the extended f-equilibrium
// (Eqs. productform, extf, Pa_star), the operator product-form g-equilibrium
// (Eq. geq_i) in closed form, the quasi-equilibrium g* (Eqs. gstar, qstar1) and
// the BGK relaxation (Eqs. fLBGK, gLBGK).
//
// Direction i = a + 3b + 9c with (c_x, c_y, c_z) = (a-1, b-1, c-1); D2Q9 uses
// i = a + 3b.  All loops over directions are fully unrolled, so every index is a
// compile-time constant and the populations stay in registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace elbm {

enum StoreKind { ST_F64 = 0, ST_F32 = 1, ST_F16DEV = 2, ST_BF16DEV = 3 };

// Kernel parameters, passed by value (__grid_constant__).
struct KParams {
    int nx, ny, nz;
    int per_x, per_y, per_z;     // 1: periodic axis, 0: zero-gradient (clamped)
    long long N;                 // nx * ny * nz
    double gm1;                  // gamma - 1  (so Cv = 1 / gm1)
    double Pr, mu0, T0, mu_exp;
    int deriv;                   // 0 upwind, 1 central
    int tz;                      // segment length of the fused kernels (D3Q27: z planes, D2Q9: rows)
    int tile2d;                  // D2Q9: the default fused schedule runs the one-tile-per-CTA kernel
                                 // (grids whose row march would not fill the device)
    int aa;                      // layout of the store read by the diagnostics: 0 in place; AA single
                                 // store: 1 swapped at the node, 2 pushed to the neighbour
    float2 rest2[27];            // rest-state pair (f_i, g_i) of every direction, deviation stores
    float rest_rho, rest_Pxx, rest_Pyy, rest_Pzz, rest_E;   // their moment sums
    // The same parameters precomputed in both arithmetic types, so that no kernel
    // converts or divides a double per node (the FP64 pipe of GB300 is narrow).
    // fixed-state faces (D2Q9): flags per axis face and the ghost values
    int has_fixed, fix_lo[3], fix_hi[3];
    double fixd[9][2];           // ghost pair (f_i, g_i), FP64 store representation
    float2 fixf[9];              // the same as raw stored values of the FP32 path
    double fixQd[3];             // Q~_aaa of the fixed state
    float fixQf[3];
    // caloric equation of state: 0 constant Cv (d_Cv, gm1); 1 Cv(T) cubic, U(T) quartic
    int eos;
    double cvd[4], Ud[4];        // Cv(T) = sum cvd[k] T^k, U(T) = T sum Ud[k] T^k (Ud[k] = cvd[k]/(k+1))
    float cvf[4], Uf[4];
    int powlaw;                                            // mu_exp != 0
    unsigned inject_tx;          // fault injection: extra bytes each TMA plane announces (0 in use)
    double d_Cv, d_invT0;
    float f_gm1, f_Cv, f_Pr, f_mu0, f_invT0, f_mu_exp;
};

// Parameter in the arithmetic type R.
template <typename R> __device__ __forceinline__ R par(double d, float f);
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

// ---------------------------------------------------------------------------
// Storage codecs.  The store keeps, for every direction i and node n, the pair
// (f_i, g_i) in one element P (double2 / float2 / half2 / bfloat162): both values
// are pulled from the same source node, so one access moves both.  The deviation
// stores (DEV) hold (f_i - f_i^rest, g_i - g_i^rest) rounded to nearest even; the
// kernels keep working on these raw stored values (see node_moments and collide),
// so decoding is a conversion only.
// ---------------------------------------------------------------------------
template <int ST> struct Codec;

template <> struct Codec<ST_F64> {
    using P = double2;
    using R = double;
    static constexpr bool DEV = false;
    __device__ __forceinline__ static void dec(P v, R& f, R& g) { f = v.x; g = v.y; }
    __device__ __forceinline__ static P enc(R f, R g) { return make_double2(f, g); }
};
template <> struct Codec<ST_F32> {
    using P = float2;
    using R = float;
    static constexpr bool DEV = false;
    __device__ __forceinline__ static void dec(P v, R& f, R& g) { f = v.x; g = v.y; }
    __device__ __forceinline__ static P enc(R f, R g) { return make_float2(f, g); }
};
// Mixed-precision add and subtract (sm_100 and later): a 16-bit operand a, exact in
// FP32, combined with an FP32 operand c and rounded once to FP32 — the same result as
// converting a first, in one instruction.  The deviation stores use them to sum moments
// straight from the stored pairs.
__device__ __forceinline__ float mixed_add_f16(unsigned short a, float c) {
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
}
__device__ __forceinline__ float mixed_sub_f16(unsigned short a, float c) {
    float d;
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
}
__device__ __forceinline__ float mixed_add_bf16(unsigned short a, float c) {
    float d;
    asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
}
__device__ __forceinline__ float mixed_sub_bf16(unsigned short a, float c) {
    float d;
    asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(c));
    return d;
}

template <> struct Codec<ST_F16DEV> {
    using P = __half2;
    using R = float;
    static constexpr bool DEV = true;
    __device__ __forceinline__ static void dec(P v, R& f, R& g) {
        const float2 d = __half22float2(v);
        f = d.x;
        g = d.y;
    }
    __device__ __forceinline__ static P enc(R f, R g) { return __floats2half2_rn(f, g); }
    // f or g component of a stored pair: to FP32, plus / minus an FP32 value
    __device__ __forceinline__ static float f32(P v, int k) { return __half2float(k ? __high2half(v) : __low2half(v)); }
    __device__ __forceinline__ static float add(P v, int k, float c) {
        return mixed_add_f16(__half_as_ushort(k ? __high2half(v) : __low2half(v)), c);
    }
    __device__ __forceinline__ static float sub(P v, int k, float c) {
        return mixed_sub_f16(__half_as_ushort(k ? __high2half(v) : __low2half(v)), c);
    }
};
template <> struct Codec<ST_BF16DEV> {
    using P = __nv_bfloat162;
    using R = float;
    static constexpr bool DEV = true;
    __device__ __forceinline__ static void dec(P v, R& f, R& g) {
        const float2 d = __bfloat1622float2(v);
        f = d.x;
        g = d.y;
    }
    __device__ __forceinline__ static P enc(R f, R g) { return __floats2bfloat162_rn(f, g); }
    __device__ __forceinline__ static float f32(P v, int k) {
        return __bfloat162float(k ? __high2bfloat16(v) : __low2bfloat16(v));
    }
    __device__ __forceinline__ static float add(P v, int k, float c) {
        return mixed_add_bf16(__bfloat16_as_ushort(k ? __high2bfloat16(v) : __low2bfloat16(v)), c);
    }
    __device__ __forceinline__ static float sub(P v, int k, float c) {
        return mixed_sub_bf16(__bfloat16_as_ushort(k ? __high2bfloat16(v) : __low2bfloat16(v)), c);
    }
};

// ---------------------------------------------------------------------------
// Lattice
// ---------------------------------------------------------------------------
template <int D> struct Lat {
    static constexpr int Q = (D == 3) ? 27 : 9;
    static constexpr int NC = (D == 3) ? 3 : 1;      // number of c_z values
};
__host__ __device__ constexpr int cx_of(int i) { return i % 3 - 1; }
__host__ __device__ constexpr int cy_of(int i) { return (i / 3) % 3 - 1; }
template <int D> __host__ __device__ constexpr int cz_of(int i) { return D == 3 ? i / 9 - 1 : 0; }

// Index mapping of one axis: periodic wrap or zero-gradient clamp (the ghost is a
// copy of the adjacent interior node).  Valid for x in [-1, n].
__device__ __forceinline__ int map_axis(int x, int n, int periodic) {
    if (x < 0) return periodic ? x + n : 0;
    if (x >= n) return periodic ? x - n : n - 1;
    return x;
}

// Division in the arithmetic type: exact for FP64, the fast hardware form for FP32
// (a few ulp; every quotient here is of moderate magnitude).
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qpow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float qpow(float a, float b) { return __powf(a, b); }

// ---------------------------------------------------------------------------
// Caloric equation of state (Eqs. U, E; R = 1): U(T) = int_0^T Cv dT and its inverse
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R cubic(const double* cd, const float* cf, R T) {
    return par<R>(cd[0], cf[0]) + T * (par<R>(cd[1], cf[1]) + T * (par<R>(cd[2], cf[2]) + T * par<R>(cd[3], cf[3])));
}
// CAL = false compiles the constant-Cv model only (the kernels launch that form when
// the handle's model is constant gamma); CAL = true branches on the handle's model.
template <typename R, bool CAL = true>
__device__ __forceinline__ R U_of_T(R T, const KParams& p) {
    if (!CAL || !p.eos) return T * par<R>(p.d_Cv, p.f_Cv);
    return T * cubic<R>(p.Ud, p.Uf, T);
}
// T from U: constant Cv directly; otherwise Newton's method on the increasing U(T)
// from T = U / Cv(0), a fixed 8 iterations (enough for T <= 1 with the stated Cv).
template <typename R, bool CAL = true>
__device__ __forceinline__ R T_of_U(R U, const KParams& p) {
    if (!CAL || !p.eos) return U * par<R>(p.gm1, p.f_gm1);
    R T = U / par<R>(p.cvd[0], p.cvf[0]);
#pragma unroll
    for (int k = 0; k < 8; ++k) T -= (T * cubic<R>(p.Ud, p.Uf, T) - U) / cubic<R>(p.cvd, p.cvf, T);
    return T;
}

// ---------------------------------------------------------------------------
// Moments
// ---------------------------------------------------------------------------
template <typename R> struct Moments {
    R rho, ux, uy, uz, T, rE;
    R Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;   // sum c c f (pre-collision)
};

// Moments of f: rho, rho u and (FULL) the pressure tensor sum c c f.  f holds the raw
// stored values; for the deviation stores (DEV) the moment sums of the rest state are
// added (the rest state carries no momentum and no off-diagonal stress, by symmetry).
template <int D, typename R, bool FULL, bool DEV>
__device__ __forceinline__ void f_moments(const R* f, const KParams& p, R& rho, R& jx, R& jy, R& jz,
                                          R P6[6]) {
    constexpr int NC = Lat<D>::NC;
    // per (b, c) row sums over c_x
    R t[3][3], d[3][3], e[3][3];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int i0 = 3 * b + 9 * c;
            R lo = f[i0], mid = f[i0 + 1], hi = f[i0 + 2];
            e[b][c] = hi + lo;
            d[b][c] = hi - lo;
            t[b][c] = e[b][c] + mid;
        }
    // sums over c_z first (columns b), then over c_y: depth 2 + 2
    R tb[3], db[3], eb[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        tb[b] = t[b][0];
        db[b] = d[b][0];
        eb[b] = e[b][0];
        if (D == 3) {
            tb[b] = (t[b][0] + t[b][2]) + t[b][1];
            db[b] = (d[b][0] + d[b][2]) + d[b][1];
            eb[b] = (e[b][0] + e[b][2]) + e[b][1];
        }
    }
    rho = (tb[0] + tb[2]) + tb[1];
    jx = (db[0] + db[2]) + db[1];
    jy = tb[2] - tb[0];
    jz = 0;
    R Pxx = (eb[0] + eb[2]) + eb[1], Pyy = tb[2] + tb[0], Pxy = db[2] - db[0];
    R Pzz = 0, Pxz = 0, Pyz = 0;
    if (D == 3) {
        const R tzh = (t[0][2] + t[2][2]) + t[1][2], tzl = (t[0][0] + t[2][0]) + t[1][0];
        const R dzh = (d[0][2] + d[2][2]) + d[1][2], dzl = (d[0][0] + d[2][0]) + d[1][0];
        jz = tzh - tzl;
        Pzz = tzh + tzl;
        Pxz = dzh - dzl;
        Pyz = (t[2][2] - t[0][2]) - (t[2][0] - t[0][0]);
    }
    if constexpr (DEV) {
        rho += R(p.rest_rho);
        Pxx += R(p.rest_Pxx);
        Pyy += R(p.rest_Pyy);
        Pzz += R(p.rest_Pzz);
    }
    if (FULL) {
        P6[0] = Pxx; P6[1] = Pyy; P6[2] = Pzz;
        P6[3] = Pxy; P6[4] = Pxz; P6[5] = Pyz;
    }
}

// rho E = sum of g, as a balanced tree (short dependency chains).
template <int D, typename R, bool DEV>
__device__ __forceinline__ R g_energy(const R* g, const KParams& p) {
    R gs[Lat<D>::Q];
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) gs[i] = g[i];
#pragma unroll
    for (int w = 1; w < Lat<D>::Q; w *= 2)
#pragma unroll
        for (int i = 0; i + w < Lat<D>::Q; i += 2 * w) gs[i] += gs[i + w];
    R rE = gs[0];
    if constexpr (DEV) rE += R(p.rest_E);
    return rE;
}

// u = j / rho and T from E = Cv T + u^2/2.
template <typename R, bool CAL = true>
__device__ __forceinline__ void finish_moments(R rho, R jx, R jy, R jz, R rE, const KParams& p, Moments<R>& m) {
    const R inv = qdiv(R(1), rho);
    m.rho = rho;
    m.rE = rE;
    m.ux = jx * inv;
    m.uy = jy * inv;
    m.uz = jz * inv;
    const R u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    m.T = T_of_U<R, CAL>(rE * inv - R(0.5) * u2, p);
}

// The same moments straight from the stored pairs of a deviation store: pair(i) returns
// the stored (f_i, g_i) of direction i.  Per (c_y, c_z) row one component is converted and
// the other two enter through mixed-precision adds (hi + lo, hi - lo, mid + (hi + lo));
// the energy is the sum of the nine row sums of g.  The rounding is that of f_moments
// and g_energy on the converted values, up to the order of the energy sum.
template <int D, int ST, bool FULL, bool CAL = true, class Pair>
__device__ __forceinline__ void node_moments_stored(Pair pair, const KParams& p, Moments<float>& m) {
    using Cd = Codec<ST>;
    using R = float;
    constexpr int NC = Lat<D>::NC;
    R t[3][3], d[3][3], e[3][3], gr[3][3];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int i0 = 3 * b + 9 * c;
            const auto lo = pair(i0), mid = pair(i0 + 1), hi = pair(i0 + 2);
            const R lo32 = Cd::f32(lo, 0);
            e[b][c] = Cd::add(hi, 0, lo32);
            d[b][c] = Cd::sub(hi, 0, lo32);
            t[b][c] = Cd::add(mid, 0, e[b][c]);
            gr[b][c] = Cd::add(hi, 1, Cd::add(mid, 1, Cd::f32(lo, 1)));
        }
    R tb[3], db[3], eb[3], gb[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        tb[b] = t[b][0];
        db[b] = d[b][0];
        eb[b] = e[b][0];
        gb[b] = gr[b][0];
        if (D == 3) {
            tb[b] = (t[b][0] + t[b][2]) + t[b][1];
            db[b] = (d[b][0] + d[b][2]) + d[b][1];
            eb[b] = (e[b][0] + e[b][2]) + e[b][1];
            gb[b] = (gr[b][0] + gr[b][2]) + gr[b][1];
        }
    }
    R rho = (tb[0] + tb[2]) + tb[1];
    const R jx = (db[0] + db[2]) + db[1];
    const R jy = tb[2] - tb[0];
    R jz = 0;
    R Pxx = (eb[0] + eb[2]) + eb[1], Pyy = tb[2] + tb[0], Pxy = db[2] - db[0];
    R Pzz = 0, Pxz = 0, Pyz = 0;
    if (D == 3) {
        const R tzh = (t[0][2] + t[2][2]) + t[1][2], tzl = (t[0][0] + t[2][0]) + t[1][0];
        const R dzh = (d[0][2] + d[2][2]) + d[1][2], dzl = (d[0][0] + d[2][0]) + d[1][0];
        jz = tzh - tzl;
        Pzz = tzh + tzl;
        Pxz = dzh - dzl;
        Pyz = (t[2][2] - t[0][2]) - (t[2][0] - t[0][0]);
    }
    rho += R(p.rest_rho);
    const R rE = ((gb[0] + gb[2]) + gb[1]) + R(p.rest_E);
    finish_moments<R, CAL>(rho, jx, jy, jz, rE, p, m);
    if (FULL) {
        m.Pxx = Pxx + R(p.rest_Pxx);
        m.Pyy = Pyy + R(p.rest_Pyy);
        m.Pzz = Pzz + R(p.rest_Pzz);
        m.Pxy = Pxy; m.Pxz = Pxz; m.Pyz = Pyz;
    }
}

// All moments of one node: f_moments, g_energy, finish_moments.
template <int D, typename R, bool FULL, bool DEV, bool CAL = true>
__device__ __forceinline__ void node_moments(const R* f, const R* g, const KParams& p, Moments<R>& m) {
    R rho, jx, jy, jz, P6[6];
    f_moments<D, R, FULL, DEV>(f, p, rho, jx, jy, jz, P6);
    const R rE = g_energy<D, R, DEV>(g, p);
    finish_moments<R, CAL>(rho, jx, jy, jz, rE, p, m);
    if (FULL) {
        m.Pxx = P6[0]; m.Pyy = P6[1]; m.Pzz = P6[2];
        m.Pxy = P6[3]; m.Pxz = P6[4]; m.Pyz = P6[5];
    }
}

// Q~_aaa = rho u_a (1 - 3T - u_a^2)  (Eq. anomalya, R = 1)
template <typename R>
__device__ __forceinline__ R anomaly(R rho, R ua, R T) {
    return rho * ua * (R(1) - R(3) * T - ua * ua);
}

// Discrete derivative of Q~_aaa at a node from its own value and the two axis
// neighbours: upwind by the sign of u_a at the node (strict '>'), or central.
template <typename R>
__device__ __forceinline__ R dQ(int deriv, R ua, R qm, R q0, R qp) {
    if (deriv) return R(0.5) * (qp - qm);
    return ua > R(0) ? (q0 - qm) : (qp - q0);
}

// Unphysical-state test used to latch ELBM_ERR_NONPHYSICAL.
template <typename R>
__device__ __forceinline__ bool nonphysical(const Moments<R>& m) {
    return !(m.rho > R(0)) || !(m.T > R(0)) || !isfinite(m.rho) || !isfinite(m.T) ||
           !isfinite(m.ux) || !isfinite(m.uy) || !isfinite(m.uz);
}

// ---------------------------------------------------------------------------
// Equilibria and collision
// ---------------------------------------------------------------------------
// Psi triplet at (xi, P), indexed a = c + 1 (Eqs. phi0S, phiPlusS, phiMinusS).
template <typename R>
__device__ __forceinline__ void psi3(R xi, R P, R out[3]) {
    out[0] = R(0.5) * (P - xi);
    out[1] = R(1) - P;
    out[2] = R(0.5) * (P + xi);
}

// Per-axis factors of g^eq.  Applying Psi_c(O, O^2) (Eq. Operator) to functions of
// one velocity component u gives
//   on 1:       phi_c = Psi_c(u, T + u^2)                      (as f^eq)
//   on u^2/2:   psi_0 = u^2/2 - s,  psi_{+-1} = (s +- o)/2,
//   with o = O(u^2/2) = T u + u^3/2 and s = O^2(u^2/2) = T^2 + (5/2) T u^2 + u^4/2.
// With E = Cv T + sum_b u_b^2/2 this gives
//   g^eq_i = rho [ Cv T phi_x phi_y phi_z + psi_x phi_y phi_z + phi_x psi_y phi_z
//                  + phi_x phi_y psi_z ].
template <typename R>
__device__ __forceinline__ void gfactors(R u, R T, R phi[3], R ps[3]) {
    const R u2 = u * u;
    psi3(u, T + u2, phi);
    const R o = T * u + R(0.5) * u2 * u;
    const R s = T * T + R(2.5) * T * u2 + R(0.5) * u2 * u2;
    ps[0] = R(0.5) * (s - o);
    ps[1] = R(0.5) * u2 - s;
    ps[2] = R(0.5) * (s + o);
}

// Equilibria f^eq and g^eq of (rho, u, T) into f, g (full populations; used for
// initialisation).
template <int D, typename R>
__device__ __forceinline__ void equilibria(R rho, R ux, R uy, R uz, R T, R U, R* f, R* g) {
    R X[3], Y[3], Z[3], sx[3], sy[3], sz[3];
    gfactors(ux, T, X, sx);
    gfactors(uy, T, Y, sy);
    if (D == 3) gfactors(uz, T, Z, sz);
    else { Z[0] = Z[2] = 0; Z[1] = 1; sz[0] = sz[1] = sz[2] = 0; }
    const R CvT = U;   // U(T): Cv T for constant Cv
#pragma unroll
    for (int c = 0; c < Lat<D>::NC; ++c) {
        const int cc = (D == 3) ? c : 1;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const R A = Y[b] * Z[cc];
            const R B = sy[b] * Z[cc] + Y[b] * sz[cc];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int i = a + 3 * b + 9 * c;
                f[i] = rho * X[a] * A;
                g[i] = rho * ((CvT * X[a] + sx[a]) * A + X[a] * B);
            }
        }
    }
}

// Relaxation rate omega (Eqs. mu, Pr) from the local pressure P = rho T, and omega_1.
template <typename R>
__device__ __forceinline__ R rate_w(R rho, R T, const KParams& p) {
    R mu = par<R>(p.mu0, p.f_mu0);
    if (p.powlaw) mu = mu * qpow(T * par<R>(p.d_invT0, p.f_invT0), par<R>(p.mu_exp, p.f_mu_exp));
    const R P = rho * T;
    return qdiv(R(2) * P, R(2) * mu + P);
}
template <typename R>
__device__ __forceinline__ R rate_w1(R w, const KParams& p) {
    const R Pr = par<R>(p.Pr, p.f_Pr);
    return qdiv(R(2) * Pr * w, R(2) - w + Pr * w);
}

// One collision, direction by direction.  init() evaluates the per-node factors;
// f(i, f_i) and g(i, g_i) return the post-collision values of direction i from the raw
// stored values (populations, or their deviations from the rest state when DEV).
//   f_i <- (1 - w) f_i + w f^ex_i            (Eqs. fLBGK, extf, Pa_star)
//   g_i <- (1 - w1) g_i + w1 g^eq_i + corr_i (Eqs. gLBGK, geq_i, gstar, qstar1)
// with w and w1 folded into the row factors of the product forms.  For DEV the rest
// state r_i is carried as (1 - w)(r_i + d_i) + w f^ex_i - r_i = (1 - w) d_i +
// w (f^ex_i - r_i).  corr_i is the quasi-equilibrium term, nonzero only for |c_i| = 1:
// q* - q^eq = u.(P - P^eq + div Q~ / 2) with P^eq = rho T I + rho u u and
// div Q~ = diag(D), and g_i += (omega - omega_1)(g^eq_i - g*_i) =
// -(omega - omega_1) c_i.(q* - q^eq) / 2.  m must carry the pressure tensor.
template <int D, typename R, bool DEV, bool CAL = true>
struct Relax {
    R omw, omw1, w, w1;
    R X[3], Y[3], Z[3], wr;                      // f^ex factors
    R gx[3], gy[3], gz[3], sy[3], sz[3], ax[3];  // g^eq factors
    R w1r;
    R h, dq[3];                                  // (omega - omega_1)/2 and q* - q^eq

    __device__ __forceinline__ void init(const Moments<R>& m, R Dx, R Dy, R Dz, const KParams& p) {
        const R rho = m.rho, T = m.T, ux = m.ux, uy = m.uy, uz = m.uz;
        w = rate_w(rho, T, p);
        w1 = rate_w1(w, p);
        // extended f-equilibrium
        const R k = qdiv(R(2) - w, R(2) * rho * w);
        psi3(ux, T + ux * ux + k * Dx, X);
        psi3(uy, T + uy * uy + k * Dy, Y);
        if (D == 3) psi3(uz, T + uz * uz + k * Dz, Z);
        else { Z[0] = Z[2] = 0; Z[1] = 1; }
        omw = R(1) - w;
        wr = w * rho;
        // g-equilibrium
        R sx[3];
        gfactors(ux, T, gx, sx);
        gfactors(uy, T, gy, sy);
        if (D == 3) gfactors(uz, T, gz, sz);
        else { gz[0] = gz[2] = 0; gz[1] = 1; sz[0] = sz[1] = sz[2] = 0; }
        const R CvT = U_of_T<R, CAL>(T, p);   // U(T) (Cv T for constant Cv)
#pragma unroll
        for (int a = 0; a < 3; ++a) ax[a] = CvT * gx[a] + sx[a];
        omw1 = R(1) - w1;
        w1r = w1 * rho;
        // quasi-equilibrium
        const R rT = rho * T;
        const R dxx = m.Pxx - rT - rho * ux * ux, dyy = m.Pyy - rT - rho * uy * uy;
        const R dxy = m.Pxy - rho * ux * uy;
        R dqx = ux * dxx + uy * dxy + R(0.5) * ux * Dx;
        R dqy = ux * dxy + uy * dyy + R(0.5) * uy * Dy;
        R dqz = 0;
        if (D == 3) {
            const R dzz = m.Pzz - rT - rho * uz * uz;
            const R dxz = m.Pxz - rho * ux * uz, dyz = m.Pyz - rho * uy * uz;
            dqx += uz * dxz;
            dqy += uz * dyz;
            dqz = ux * dxz + uy * dyz + uz * dzz + R(0.5) * uz * Dz;
        }
        h = R(0.5) * (w - w1);
        dq[0] = dqx;
        dq[1] = dqy;
        dq[2] = dqz;
    }

    // i is a compile-time constant after unrolling, so every branch below folds away
    __device__ __forceinline__ R f(int i, R fi, const KParams& p) const {
        const int a = cx_of(i) + 1, b = cy_of(i) + 1, c = (D == 3) ? cz_of<D>(i) + 1 : 1;
        const R yz = wr * Y[b] * Z[c];
        R t = X[a] * yz;
        if constexpr (DEV) t = fma(-w, R(p.rest2[i].x), t);
        return fma(omw, fi, t);
    }
    // Both updates of direction i at once, as two-lane FP32 arithmetic (FFMA2, sm_100 and
    // later): the same operations in the same order as f() and g(), so the same results.
    __device__ __forceinline__ float2 fg(int i, float2 v, const KParams& p) const {
        static_assert(sizeof(R) == 4, "two-lane form of the FP32 arithmetic");
        const int a = cx_of(i) + 1, b = cy_of(i) + 1, c = (D == 3) ? cz_of<D>(i) + 1 : 1;
        const R yz = wr * Y[b] * Z[c];
        const R A = w1r * gy[b] * gz[c];
        const R B = w1r * (sy[b] * gz[c] + gy[b] * sz[c]);
        float2 t = make_float2(X[a] * yz, fma(ax[a], A, gx[a] * B));
        if constexpr (DEV) t = __ffma2_rn(make_float2(-w, -w1), p.rest2[i], t);
        float2 o = __ffma2_rn(make_float2(omw, omw1), v, t);
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of<D>(i);
        if (cx * cx + cy * cy + cz * cz == 1) {
            const R q = cx != 0 ? dq[0] : (cy != 0 ? dq[1] : dq[2]);
            if (cx + cy + cz < 0) o.y += h * q;
            else o.y -= h * q;
        }
        return o;
    }
    __device__ __forceinline__ R g(int i, R gi, const KParams& p) const {
        constexpr int Q = Lat<D>::Q;
        const int a = cx_of(i) + 1, b = cy_of(i) + 1, c = (D == 3) ? cz_of<D>(i) + 1 : 1;
        const R A = w1r * gy[b] * gz[c];
        const R B = w1r * (sy[b] * gz[c] + gy[b] * sz[c]);
        R t = fma(ax[a], A, gx[a] * B);
        if constexpr (DEV) t = fma(-w1, R(p.rest2[i].y), t);
        R v = fma(omw1, gi, t);
        // unit-speed directions: the correction enters with the sign of -c_i
        const int cx = cx_of(i), cy = cy_of(i), cz = cz_of<D>(i);
        if (cx * cx + cy * cy + cz * cz == 1) {
            const R q = cx != 0 ? dq[0] : (cy != 0 ? dq[1] : dq[2]);
            if (cx + cy + cz < 0) v += h * q;
            else v -= h * q;
        }
        return v;
    }
};

// One collision in place on the raw stored values f, g.
template <int D, typename R, bool DEV, bool CAL = true>
__device__ __forceinline__ void collide(R* f, R* g, const Moments<R>& m, R Dx, R Dy, R Dz,
                                        const KParams& p) {
    Relax<D, R, DEV, CAL> r;
    r.init(m, Dx, Dy, Dz, p);
#pragma unroll
    for (int i = 0; i < Lat<D>::Q; ++i) {
        f[i] = r.f(i, f[i], p);
        g[i] = r.g(i, g[i], p);
    }
}

}  // namespace elbm
