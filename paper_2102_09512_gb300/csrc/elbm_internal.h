// Host-side interface between the C ABI (elbm_api.cu) and the kernel translation
// units (elbm_kernels.cu, compiled once per lattice x store kind).
#pragma once

#include <cuda_runtime.h>

#include "elbm_node.cuh"

namespace elbm {

// Layout of the auxiliary buffer (all offsets 256-byte aligned).
struct AuxLayout {
    size_t status;      // int32 status word
    size_t totals;      // 8 doubles: finalised totals
    size_t partials;    // max_blocks x 5 doubles: per-CTA totals
    size_t qfield;      // D x N values of Q~ (two-pass schedule), arithmetic type
    size_t staging;     // 5 x N doubles (host field transfers)
    size_t bytes;
    int max_blocks;
};

// Launchers for one (lattice, store) combination.  Each returns the first CUDA
// error it meets and adds the number of kernels it launched to *launches.
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
};

const Ops* ops_d2_f64();
const Ops* ops_d2_f32();
const Ops* ops_d2_f16();
const Ops* ops_d2_bf16();
const Ops* ops_d3_f64();
const Ops* ops_d3_f32();
const Ops* ops_d3_f16();
const Ops* ops_d3_bf16();

}  // namespace elbm
