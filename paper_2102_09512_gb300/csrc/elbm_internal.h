// Host-side interface between the C ABI (elbm_api.cu) and the kernel translation
// units (elbm_kernels.cu, compiled once per lattice x store kind).
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the library does not link the driver)
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "elbm.h"
#include "elbm_node.cuh"

namespace elbm {

// Internal energy U(T) = int_0^T Cv dT of the problem's caloric equation of state.
inline double host_U(const elbm_params& p, double T) {
    if (p.eos == ELBM_EOS_CV_POLY)
        return T * (p.cv[0] + T * (p.cv[1] / 2.0 + T * (p.cv[2] / 3.0 + T * p.cv[3] / 4.0)));
    return T / (p.gamma - 1.0);
}

// f^eq and g^eq of a uniform state for D2Q9 in FP64 on the host (Eqs. 27eq, geq_i in
// the per-axis closed form of the kernels): phi = Psi(u, T + u^2),
// psi = {(s - o)/2, u^2/2 - s, (s + o)/2} with o = T u + u^3/2, s = T^2 + 5/2 T u^2 + u^4/2,
// f_i = rho phi_x phi_y, g_i = rho [(U phi_x + psi_x) phi_y + phi_x psi_y] with U = U(T).
inline void host_equilibria_d2q9(double rho, const double u[3], double T, double U, double f[9], double g[9]) {
    double ph[2][3], ps[2][3];
    for (int a = 0; a < 2; ++a) {
        const double v = u[a], v2 = v * v, P = T + v2;
        ph[a][0] = 0.5 * (P - v);
        ph[a][1] = 1.0 - P;
        ph[a][2] = 0.5 * (P + v);
        const double o = T * v + 0.5 * v2 * v, s = T * T + 2.5 * T * v2 + 0.5 * v2 * v2;
        ps[a][0] = 0.5 * (s - o);
        ps[a][1] = 0.5 * v2 - s;
        ps[a][2] = 0.5 * (s + o);
    }
    for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
            f[a + 3 * b] = rho * ph[0][a] * ph[1][b];
            g[a + 3 * b] = rho * ((U * ph[0][a] + ps[0][a]) * ph[1][b] + ph[0][a] * ps[1][b]);
        }
}

// Validates a problem statement and fills the kernel parameters (host only, no CUDA
// call, no allocation).  Returns ELBM_OK, ELBM_ERR_ARG or ELBM_ERR_UNSUPPORTED; *D_out is 2 or 3.
inline int fill_kparams(const elbm_params& p, KParams& k, int* D_out) {
    auto finite_pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    int D;
    if (p.lattice == ELBM_D2Q9) D = 2;
    else if (p.lattice == ELBM_D3Q27) D = 3;
    else return ELBM_ERR_ARG;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (D == 2 && p.nz != 1)) return ELBM_ERR_ARG;
    if (!(std::isfinite(p.gamma) && p.gamma > 1.0)) return ELBM_ERR_ARG;
    if (!finite_pos(p.Pr) || !finite_pos(p.mu0) || !finite_pos(p.T0) || !std::isfinite(p.mu_exp))
        return ELBM_ERR_ARG;
    if (p.eos != ELBM_EOS_GAMMA && p.eos != ELBM_EOS_CV_POLY) return ELBM_ERR_ARG;
    if (p.eos == ELBM_EOS_CV_POLY &&
        (!finite_pos(p.cv[0]) || !std::isfinite(p.cv[1]) || !std::isfinite(p.cv[2]) || !std::isfinite(p.cv[3])))
        return ELBM_ERR_ARG;
    bool any_fixed = false;
    for (int f = 0; f < 6; ++f) {
        if (p.bc[f] != ELBM_BC_PERIODIC && p.bc[f] != ELBM_BC_ZEROGRAD && p.bc[f] != ELBM_BC_FIXED)
            return ELBM_ERR_ARG;
        any_fixed |= p.bc[f] == ELBM_BC_FIXED;
    }
    if (any_fixed) {
        if (!finite_pos(p.fix_rho) || !finite_pos(p.fix_T) || !std::isfinite(p.fix_u[0]) ||
            !std::isfinite(p.fix_u[1]) || !std::isfinite(p.fix_u[2]))
            return ELBM_ERR_ARG;
        if (D != 2) return ELBM_ERR_UNSUPPORTED;
    }
    for (int a = 0; a < 3; ++a)
        if ((p.bc[2 * a] == ELBM_BC_PERIODIC) != (p.bc[2 * a + 1] == ELBM_BC_PERIODIC)) return ELBM_ERR_ARG;
    if (p.store < ELBM_F64 || p.store > ELBM_BF16DEV) return ELBM_ERR_ARG;
    if (p.deriv != ELBM_DERIV_UPWIND && p.deriv != ELBM_DERIV_CENTRAL) return ELBM_ERR_ARG;
    const bool dev = p.store == ELBM_F16DEV || p.store == ELBM_BF16DEV;
    if (dev && (!finite_pos(p.rho_ref) || !finite_pos(p.T_ref) || p.T_ref >= 1.0)) return ELBM_ERR_ARG;

    std::memset(&k, 0, sizeof(k));
    k.nx = p.nx;
    k.ny = p.ny;
    k.nz = p.nz;
    k.per_x = p.bc[0] == ELBM_BC_PERIODIC;
    k.per_y = p.bc[2] == ELBM_BC_PERIODIC;
    k.per_z = p.bc[4] == ELBM_BC_PERIODIC;
    k.N = (long long)p.nx * p.ny * p.nz;
    k.gm1 = p.gamma - 1.0;
    k.Pr = p.Pr;
    k.mu0 = p.mu0;
    k.T0 = p.T0;
    k.mu_exp = p.mu_exp;
    k.deriv = p.deriv;
    k.powlaw = p.mu_exp != 0.0;
    k.d_Cv = 1.0 / (p.gamma - 1.0);
    k.eos = p.eos == ELBM_EOS_CV_POLY;
    for (int j = 0; j < 4; ++j) {
        k.cvd[j] = k.eos ? p.cv[j] : 0.0;
        k.Ud[j] = k.cvd[j] / (j + 1);
        k.cvf[j] = (float)k.cvd[j];
        k.Uf[j] = (float)k.Ud[j];
    }
    k.d_invT0 = 1.0 / p.T0;
    k.f_gm1 = (float)k.gm1;
    k.f_Cv = (float)k.d_Cv;
    k.f_Pr = (float)p.Pr;
    k.f_mu0 = (float)p.mu0;
    k.f_invT0 = (float)k.d_invT0;
    k.f_mu_exp = (float)p.mu_exp;
    if (any_fixed) {
        // ghosts of the fixed-state faces: f^eq, g^eq and Q~ of the fixed state (D2Q9)
        k.has_fixed = 1;
        for (int a = 0; a < 3; ++a) {
            k.fix_lo[a] = p.bc[2 * a] == ELBM_BC_FIXED;
            k.fix_hi[a] = p.bc[2 * a + 1] == ELBM_BC_FIXED;
        }
        double fe[9], ge[9];
        host_equilibria_d2q9(p.fix_rho, p.fix_u, p.fix_T, host_U(p, p.fix_T), fe, ge);
        for (int i = 0; i < 9; ++i) {
            k.fixd[i][0] = fe[i];
            k.fixd[i][1] = ge[i];
        }
        for (int a = 0; a < 3; ++a) {
            k.fixQd[a] = p.fix_rho * p.fix_u[a] * (1.0 - 3.0 * p.fix_T - p.fix_u[a] * p.fix_u[a]);
            k.fixQf[a] = (float)k.fixQd[a];
        }
    }
    // z segment of the fused D3Q27 kernels: longer for FP32 (one CTA per SM, so
    // fewer prologues per plane matter more), measured at 256^3; D2Q9: rows per
    // segment of the row march (both refined for the device at handle creation)
    if (D == 3) {
        const int tz = p.store == ELBM_F32 ? 64 : 32;
        k.tz = p.nz < tz ? p.nz : tz;
    } else {
        k.tz = p.ny < 32 ? p.ny : 32;
    }
    if (dev) {
        // Rest state f^eq(rho_ref, 0, T_ref), g^eq(rho_ref, 0, T_ref): with u = 0 the
        // per-axis factors are phi = (T/2, 1-T, T/2) and psi = (T^2/2, -T^2, T^2/2).
        const int Q = D == 3 ? 27 : 9;
        const double T0 = p.T_ref, U0 = host_U(p, T0);
        const double phi[3] = {0.5 * T0, 1.0 - T0, 0.5 * T0};
        const double psi[3] = {0.5 * T0 * T0, -T0 * T0, 0.5 * T0 * T0};
        double srho = 0, sxx = 0, syy = 0, szz = 0, sE = 0;
        for (int i = 0; i < Q; ++i) {
            const int a = i % 3, b = (i / 3) % 3, c = D == 3 ? i / 9 : 1;
            const double pz = D == 3 ? phi[c] : 1.0, sz = D == 3 ? psi[c] : 0.0;
            k.rest2[i].x = (float)(p.rho_ref * phi[a] * phi[b] * pz);
            k.rest2[i].y = (float)(p.rho_ref * ((U0 * phi[a] + psi[a]) * phi[b] * pz +
                                                phi[a] * (psi[b] * pz + phi[b] * sz)));
            // moment sums of the stored (rounded) rest values
            srho += k.rest2[i].x;
            if (a != 1) sxx += k.rest2[i].x;
            if (b != 1) syy += k.rest2[i].x;
            if (D == 3 && c != 1) szz += k.rest2[i].x;
            sE += k.rest2[i].y;
        }
        k.rest_rho = (float)srho;
        k.rest_Pxx = (float)sxx;
        k.rest_Pyy = (float)syy;
        k.rest_Pzz = (float)szz;
        k.rest_E = (float)sE;
    }
    if (k.has_fixed) {
        // the same ghosts as raw stored values of the FP32 arithmetic path (deviations
        // from the rest state for the deviation stores)
        for (int i = 0; i < 9; ++i) {
            const double rf = dev ? (double)k.rest2[i].x : 0.0, rg = dev ? (double)k.rest2[i].y : 0.0;
            k.fixf[i].x = (float)(k.fixd[i][0] - rf);
            k.fixf[i].y = (float)(k.fixd[i][1] - rg);
        }
    }
    *D_out = D;
    return ELBM_OK;
}

// Threads per CTA of the one-dimensional launches (initialisation, field extraction, the
// two passes of the two-pass schedule).  The two-pass step writes one partial vector of
// step totals per CTA of that grid, so every scratch layout sizes its partials by
// blocks_1d_of(N).
constexpr int kThreads1D = 256;
inline long long blocks_1d_of(long long n) { return (n + kThreads1D - 1) / kThreads1D; }

// Scratch of the allocation-free step (elbm_step_noalloc): status word, per-CTA partials
// of the two-pass step, Q~ field (D values of the arithmetic type per node); offsets
// 256-byte aligned.  The static device array that holds it has kNoallocScratchBytes; a
// grid whose layout needs more is rejected before anything is launched.
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
struct NoallocLayout {
    size_t status, partials, qfield, bytes;
};
inline NoallocLayout noalloc_layout(long long N, int D, size_t real_bytes) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    NoallocLayout l;
    l.status = 0;
    l.partials = up(sizeof(int));
    l.qfield = up(l.partials + (size_t)blocks_1d_of(N) * 5 * sizeof(double));
    l.bytes = up(l.qfield + (size_t)D * (size_t)N * real_bytes);
    return l;
}

// D2Q9 row march: a CTA owns a strip of kMarchW2 nodes of a row and marches along y;
// the persistent ensemble runs it with segments of one of kMarchSegs rows (a schedule
// value above 16; 4, 8 and 16 select the one-tile-per-unit kernel with 32 x ty tiles).
#ifndef ELBM_MARCH_W
#define ELBM_MARCH_W 128
#endif
constexpr int kMarchW2 = ELBM_MARCH_W;
constexpr int kMarchSegs[3] = {32, 64, 128};

// Layout of the auxiliary buffer (all offsets 256-byte aligned).
struct AuxLayout {
    size_t status;      // int32 status word
    size_t totals;      // up to 12 doubles: finalised totals
    size_t fin_count;   // uint32 arrival counter of the finalisation (zero between launches)
    size_t fin_scratch; // per-CTA (sum, compensation) pairs of the finalisation
    size_t partials;    // max_blocks x 5 doubles: per-CTA totals
    size_t qfield;      // D x N values of Q~ (two-pass schedule), arithmetic type
    size_t staging;     // 5 x N doubles (host field transfers)
    size_t bytes;
    int max_blocks;
};

// Device-side description of a D2Q9 ensemble (arrays live in the ensemble's
// auxiliary buffer).
// Bits of the device status word: a non-physical state (rho <= 0, T <= 0 or not
// finite) and a bounded device wait that gave up.
constexpr int kStatusNonphysicalBit = 1;
constexpr int kStatusTimeoutBit = 2;

constexpr int kMaxEnsemble = 1024;
struct EnsembleArgs {
    const KParams* params;      // [n] per-instance parameters
    const long long* offset;    // [n] element offset of instance k in both stores
    const int* tile_start;      // [n+1] prefix sums of the instances' tile counts
    const int* tiles_x;         // [n] tiles per row of instance k
    int n, ntiles;
    int caloric;                // some instance has a Cv(T) model (selects the kernel form)
};

// Launchers for one (lattice, store) combination.  Each returns the first CUDA
// error it meets and adds the number of kernels it launched to *launches.
// Per-CTA partial sums of the turbulence statistics (stats_kernel, elbm_turbulence_stats).
constexpr int kStatsSums = 11;

struct Ops {
    int D, store;
    size_t value_bytes;   // bytes per stored population value
    size_t real_bytes;    // bytes of the arithmetic type (Q~ field)
    int (*max_blocks)(const KParams& p);
    cudaError_t (*init)(const KParams& p, const double* rho, const double* u, const double* T,
                        void* pop, void* spare, void* qfield, double* partials, int* status,
                        cudaStream_t s, long long* launches);
    cudaError_t (*fields)(const KParams& p, const void* pop, double* rho, double* u, double* T,
                          int* status, cudaStream_t s, long long* launches);
    cudaError_t (*step_twopass)(const KParams& p, const void* src, void* dst, void* qfield,
                                double* partials, int* nblocks, int* status, cudaStream_t s,
                                long long* launches);
    cudaError_t (*step_fused)(const KParams& p, const void* src, void* dst, double* partials,
                              int* nblocks, int* status, cudaStream_t s, long long* launches);
    cudaError_t (*step_fused_reread)(const KParams& p, const void* src, void* dst, double* partials,
                                     int* nblocks, int* status, cudaStream_t s, long long* launches);
    cudaError_t (*conservation)(const KParams& p, const void* pop, double* partials, int* nblocks,
                                cudaStream_t s, long long* launches);
    cudaError_t (*step_ensemble)(const EnsembleArgs& a, const void* src, void* dst, int* status, int ty,
                                 int grid, cudaStream_t s, long long* launches);
    int (*ensemble_occupancy)(int ty);
    cudaError_t (*stats)(const KParams& p, const void* pop, double* partials, int* nblocks, cudaStream_t s,
                         long long* launches);   // kStatsSums partial sums per CTA
    int fused_tile_y;             // D3Q27: tile height of the fused kernels (tile width 32); D2Q9: 1 (row march)
    // resident CTAs per SM of the default fused kernel for the grid p (the D2Q9 march is
    // compiled with and without fixed-state faces; 0: unknown)
    int (*fused_occupancy)(const KParams& p);
    cudaError_t (*step_fused_tma)(const KParams& p, const void* src, void* dst, const CUtensorMap* src_map,
                                  double* partials, int* nblocks, int* status, cudaStream_t s, long long* launches);
    int (*tma_supported)(const KParams& p);   // the grid suits the TMA-staged D3Q27 kernel
    // tensor map of a store: 1 made, 0 not applicable, -1 the driver refused.  kind
    // kTmapStage: the boxes the TMA-staged kernel copies; kTmapPrefetch: the boxes the
    // default fused kernel prefetches into L2
    int (*encode_tmap)(const KParams& p, const void* base, CUtensorMap* out, int kind);
    // the default fused step given src's prefetch tensor map (L2 prefetch of the planes ahead)
    cudaError_t (*step_fused_pf)(const KParams& p, const void* src, void* dst, const CUtensorMap* src_map,
                                 double* partials, int* nblocks, int* status, cudaStream_t s, long long* launches);
    // equilibria of nodes n0 .. n0 + cnt - 1 written in place (fields of those nodes only),
    // and rho, u, T of such a range (chunked host transfers)
    cudaError_t (*init_nodes)(const KParams& p, const double* rho, const double* u, const double* T, void* pop,
                              long long n0, long long cnt, int* status, cudaStream_t s, long long* launches);
    cudaError_t (*fields_nodes)(const KParams& p, const void* pop, double* rho, double* u, double* T,
                                long long n0, long long cnt, int* status, cudaStream_t s, long long* launches);
    // AA single-store layout (periodic grids): one two-pass step on the store A from layout
    // L1 (from_l1 = 1: node-local reads, swapped writes) or from layout L0 (pulled reads,
    // pushed writes)
    cudaError_t (*step_aa)(const KParams& p, void* A, void* qfield, double* partials, int* nblocks, int* status,
                           cudaStream_t s, long long* launches, int from_l1);
    int march_width;   // D2Q9: strip width of the single-lattice row march of this store
};

// z-segment length of the fused D3Q27 kernels.  Each CTA marches one (tile, segment)
// column; the grid runs in waves of sms * per_sm CTAs.  The choice maximises the fill
// of the last wave times tz / (tz + 2), the second factor charging each segment about
// two planes of prologue (the Q~ plane below it and the plane above it).  Ties keep
// the longer segment.  Without device information the fallback is kept.
inline int choose_segment(double tiles, int nplanes, int sms, int per_sm, int fallback) {
    if (sms <= 0 || per_sm <= 0) return fallback < nplanes ? fallback : nplanes;
    const double slots = (double)sms * per_sm;
    const int lo = nplanes < 16 ? nplanes : 16, hi = 128;
    int best = fallback < nplanes ? fallback : nplanes;
    double best_score = -1.0;
    for (int nseg = 1; nseg <= nplanes; ++nseg) {
        const int tz = (nplanes + nseg - 1) / nseg;
        if (tz > hi) continue;
        if (tz < lo) break;
        const int ns = (nplanes + tz - 1) / tz;
        const double waves = tiles * ns / slots;
        const double fill = waves / std::ceil(waves);
        const double score = fill * tz / (tz + 2.0);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = tz;
        }
    }
    return best;
}
inline int choose_tz(const KParams& k, int ty, int sms, int per_sm, int fallback) {
    const double tiles = (double)((k.nx + 31) / 32) * (double)((k.ny + ty - 1) / ty);
    return choose_segment(tiles, k.nz, sms, per_sm, fallback);
}
// The same choice for the D2Q9 row march: strips of `width` nodes, segments of rows.
inline int choose_rows(const KParams& k, int sms, int per_sm, int fallback, int width) {
    return choose_segment((double)((k.nx + width - 1) / width), k.ny, sms, per_sm, fallback);
}
// D2Q9 schedule for a device of `sms` SMs: the row segment, and whether the grid is too
// small for the march (fewer strips x segments than SMs), in which case the default fused
// schedule runs the one-tile-per-CTA kernel instead.  Without device information the
// march with the fallback segment is kept.
inline void plan_d2q9(KParams& k, int sms, int per_sm, int width) {
    k.tz = choose_rows(k, sms, per_sm, k.tz, width);
    const long long ctas = (long long)((k.nx + width - 1) / width) * ((k.ny + k.tz - 1) / k.tz);
    k.tile2d = sms > 0 && ctas < sms;
}

constexpr int kTmapStage = 0, kTmapPrefetch = 1;   // encode_tmap kinds

const Ops* ops_d2_f64();
const Ops* ops_d2_f32();
const Ops* ops_d2_f16();
const Ops* ops_d2_bf16();
const Ops* ops_d3_f64();
const Ops* ops_d3_f32();
const Ops* ops_d3_f16();
const Ops* ops_d3_bf16();

}  // namespace elbm
