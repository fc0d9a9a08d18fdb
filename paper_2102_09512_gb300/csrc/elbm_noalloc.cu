// elbm_step_noalloc: one time step of the two-pass schedule for callers that cannot
// allocate device memory.
//
// Some callers of this library are not allowed to call cudaMalloc: a solver embedded
// in a host application that owns the whole device memory pool and hands the library
// only the buffers it reads and writes, or a fixed-budget deployment whose device
// memory is reserved once at start-up.  The handle-based API needs a caller-owned
// auxiliary buffer for its scratch (the Q~ field, reduction partials, the status
// word); this entry point instead keeps that scratch in one fixed, file-scope device
// array, so the caller passes only the two population stores.
//
// The array is a static __device__ object: every GPU that loads the library holds
// it (kNoallocScratchBytes) until the process exits, whether or not the entry point
// is called.  Host code cannot use the array's name as a device address; the entry
// point looks the address up with cudaGetSymbolAddress once per device, with that
// device current, on the first call made on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "elbm.h"
#include "elbm_internal.h"

namespace {

using namespace elbm;

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

const Ops* ops_for(int D, int store) {
    switch (store) {
        case ELBM_F64: return D == 2 ? ops_d2_f64() : ops_d3_f64();
        case ELBM_F32: return D == 2 ? ops_d2_f32() : ops_d3_f32();
        case ELBM_F16DEV: return D == 2 ? ops_d2_f16() : ops_d3_f16();
        case ELBM_BF16DEV: return D == 2 ? ops_d2_bf16() : ops_d3_bf16();
    }
    return nullptr;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Device address of the scratch array on the current device (set-up on first use).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ELBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ELBM_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ELBM_OK;
}

}  // namespace

extern "C" int elbm_step_noalloc(const elbm_params* prm, const void* src, void* dst, void* stream) {
    if (!prm || !src || !dst || src == dst) return ELBM_ERR_ARG;
    if (((uintptr_t)src | (uintptr_t)dst) % kAlign) return ELBM_ERR_ARG;
    const elbm_params& p = *prm;
    int D;
    if (p.lattice == ELBM_D2Q9) D = 2;
    else if (p.lattice == ELBM_D3Q27) D = 3;
    else return ELBM_ERR_ARG;
    if (p.nx < 1 || p.ny < 1 || p.nz < 1 || (D == 2 && p.nz != 1)) return ELBM_ERR_ARG;
    if (!(std::isfinite(p.gamma) && p.gamma > 1.0)) return ELBM_ERR_ARG;
    if (!finite_pos(p.Pr) || !finite_pos(p.mu0) || !finite_pos(p.T0) || !std::isfinite(p.mu_exp))
        return ELBM_ERR_ARG;
    for (int k = 0; k < 6; ++k)
        if (p.bc[k] != ELBM_BC_PERIODIC && p.bc[k] != ELBM_BC_ZEROGRAD) return ELBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if ((p.bc[2 * a] == ELBM_BC_PERIODIC) != (p.bc[2 * a + 1] == ELBM_BC_PERIODIC)) return ELBM_ERR_ARG;
    if (p.store < ELBM_F64 || p.store > ELBM_BF16DEV) return ELBM_ERR_ARG;
    if (p.deriv != ELBM_DERIV_UPWIND && p.deriv != ELBM_DERIV_CENTRAL) return ELBM_ERR_ARG;
    const bool dev = p.store == ELBM_F16DEV || p.store == ELBM_BF16DEV;
    if (dev && (!finite_pos(p.rho_ref) || !finite_pos(p.T_ref) || p.T_ref >= 1.0)) return ELBM_ERR_ARG;
    const Ops* ops = ops_for(D, p.store);
    if (!ops) return ELBM_ERR_ARG;

    KParams k;
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
    k.tz = p.nz < 32 ? p.nz : 32;
    if (dev) {   // rest state f^eq(rho_ref, 0, T_ref), g^eq(rho_ref, 0, T_ref) of the deviation stores
        const int Q = D == 3 ? 27 : 9;
        const double T0 = p.T_ref, Cv = 1.0 / (p.gamma - 1.0);
        const double phi[3] = {0.5 * T0, 1.0 - T0, 0.5 * T0};
        const double psi[3] = {0.5 * T0 * T0, -T0 * T0, 0.5 * T0 * T0};
        for (int i = 0; i < Q; ++i) {
            const int a = i % 3, b = (i / 3) % 3, c = D == 3 ? i / 9 : 1;
            const double pz = D == 3 ? phi[c] : 1.0, sz = D == 3 ? psi[c] : 0.0;
            k.rest32[i] = (float)(p.rho_ref * phi[a] * phi[b] * pz);
            k.rest32[Q + i] = (float)(p.rho_ref * ((Cv * T0 * phi[a] + psi[a]) * phi[b] * pz +
                                                   phi[a] * (psi[b] * pz + phi[b] * sz)));
        }
    }

    // scratch layout: status word | per-CTA partials | Q~ field
    const size_t status_off = 0;
    const size_t partials_off = align_up(sizeof(int));
    const size_t nblocks = (size_t)((k.N + 255) / 256);
    const size_t qfield_off = align_up(partials_off + nblocks * 5 * sizeof(double));
    const size_t need = align_up(qfield_off + (size_t)D * (size_t)k.N * ops->real_bytes);
    if (need > kNoallocScratchBytes) return ELBM_ERR_UNSUPPORTED;   // grid too large for the static scratch

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != ELBM_OK) return rc;
    char* s = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;
    int* status = (int*)(s + status_off);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return ELBM_ERR_CUDA;
    int nb = 0;
    long long launches = 0;
    cudaError_t e = ops->step_twopass(k, src, dst, s + qfield_off, (double*)(s + partials_off), &nb, status, st,
                                      &launches);
    return e == cudaSuccess ? ELBM_OK : ELBM_ERR_CUDA;
}
