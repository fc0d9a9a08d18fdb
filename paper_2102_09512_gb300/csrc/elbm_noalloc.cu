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
// device current, on the first call made on it.  The address belongs to the device's
// context: if the caller resets the device (cudaDeviceReset) the module is loaded again
// in a new context, so the cached address is keyed by the context's unique id and the
// first call after a reset looks it up again.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "elbm.h"
#include "elbm_internal.h"

namespace {

using namespace elbm;

constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

// kNoallocScratchBytes (16 MiB) per device, from elbm_internal.h
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // id of the context the address belongs to

// Unique id of the calling thread's current context (0 if none or if the driver does not
// offer the query); the driver entry points are resolved through the runtime, so the
// library does not link the driver.
unsigned long long current_context_id() {
    struct Api {
        PFN_cuCtxGetCurrent_v4000 get = nullptr;
        PFN_cuCtxGetId_v12000 id = nullptr;
    };
    static const Api api = [] {
        Api a;
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            a.get = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            a.id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
        cudaGetLastError();   // leave no sticky error behind
        return a;
    }();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!api.get || !api.id || api.get(&ctx) != CUDA_SUCCESS || !ctx || api.id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

const Ops* ops_for(int D, int store) {
    switch (store) {
        case ELBM_F64: return D == 2 ? ops_d2_f64() : ops_d3_f64();
        case ELBM_F32: return D == 2 ? ops_d2_f32() : ops_d3_f32();
        case ELBM_F16DEV: return D == 2 ? ops_d2_f16() : ops_d3_f16();
        case ELBM_BF16DEV: return D == 2 ? ops_d2_bf16() : ops_d3_bf16();
    }
    return nullptr;
}

// Device address of the scratch array on the current device: looked up on the first call
// made on the device, and again on the first call after its context changed (a reset).
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ELBM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ELBM_ERR_CUDA;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();   // the lookup made the runtime's context current
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

    // scratch layout: status word | per-CTA partials of the two-pass step | Q~ field
    const NoallocLayout lay = noalloc_layout(k.N, D, ops->real_bytes);
    if (lay.bytes > kNoallocScratchBytes) return ELBM_ERR_UNSUPPORTED;   // grid too large for the static scratch

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc != ELBM_OK) return rc;
    char* s = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;
    int* status = (int*)(s + lay.status);
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return ELBM_ERR_CUDA;
    int nb = 0;
    long long launches = 0;
    cudaError_t e = ops->step_twopass(k, src, dst, s + lay.qfield, (double*)(s + lay.partials), &nb, status, st,
                                      &launches);
    return e == cudaSuccess ? ELBM_OK : ELBM_ERR_CUDA;
}
