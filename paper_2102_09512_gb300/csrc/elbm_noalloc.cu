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
    KParams k;
    int D = 0;
    const int vrc = fill_kparams(p, k, &D);
    if (vrc != ELBM_OK) return vrc;
    const Ops* ops = ops_for(D, p.store);
    if (!ops) return ELBM_ERR_ARG;

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
