// C ABI of the library (declared in include/elbm.h): parameter validation, buffer
// binding, schedule selection and the host side of the diagnostics.  No kernel here
// touches the populations except the small reduction finaliser.
#include <cuda.h>   // driver types (CUpointer_attribute); the driver is reached through the runtime
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "elbm.h"
#include "elbm_internal.h"

using namespace elbm;

struct elbm_handle {
    elbm_params prm;
    const Ops* ops;
    KParams kp;
    int D, Q;
    long long N;
    size_t pop_bytes;
    AuxLayout aux;
    void* pop[2];
    CUtensorMap tmap[2];     // tensor maps of pop[0], pop[1] (TMA-staged D3Q27 kernel)
    CUtensorMap pfmap[2];    // ... with the L2-prefetch boxes of the default fused kernel
    bool tmap_ready;
    char* auxp;
    cudaStream_t stream;
    bool bound;
    int cur;                 // index of the store holding the current state
    int kernel;              // elbm_kernel
    int layout;              // elbm_layout
    int step_blocks;         // CTAs that wrote step partials in the last step
    long long steps;
    long long launches;
    // CUDA graphs of graph_steps steps (0: off), one per starting store / layout parity;
    // dropped whenever a pointer, the kernel choice or a kernel parameter changes
    int graph_steps = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long graph_launches = 0;   // kernel launches one replay issues
    void drop_graphs() {
        for (auto& g : gexec) {
            if (g) cudaGraphExecDestroy(g);
            g = nullptr;
        }
    }
    ~elbm_handle() { drop_graphs(); }
};

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
// Host field transfers of an AA handle go through the staging area in chunks of this many
// nodes (a ping-pong handle stages the whole grid at once).
constexpr long long kStagingChunk = 1LL << 25;

const Ops* pick_ops(int D, int store) {
    if (D == 2) {
        switch (store) {
            case ELBM_F64: return ops_d2_f64();
            case ELBM_F32: return ops_d2_f32();
            case ELBM_F16DEV: return ops_d2_f16();
            case ELBM_BF16DEV: return ops_d2_bf16();
        }
    } else {
        switch (store) {
            case ELBM_F64: return ops_d3_f64();
            case ELBM_F32: return ops_d3_f32();
            case ELBM_F16DEV: return ops_d3_f16();
            case ELBM_BF16DEV: return ops_d3_bf16();
        }
    }
    return nullptr;
}

// Compensated FP64 sum over nb partial vectors of `width` values (width <= kMaxWidth).
constexpr int kMaxWidth = 12;   // widest partial vector: step totals 5, statistics kStatsSums
static_assert(kStatsSums <= kMaxWidth, "finalize width");
// The sum runs on kFinBlocks CTAs: CTA b takes a contiguous range of the partial vectors,
// each thread a Neumaier sum of its share, the CTA a fixed pairwise tree of the threads'
// (sum, compensation) pairs; the last CTA to finish (a counter in the auxiliary buffer,
// zero between launches) adds the kFinBlocks pairs in order and writes the result.  The
// order of every operation is fixed, so the result does not depend on the schedule.
constexpr int kFinBlocks = 32;
constexpr int kFinThreads = 128;

__device__ __forceinline__ void neumaier_add(double& s, double& c, double v) {
    const double t = s + v;
    c += fabs(s) >= fabs(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

__global__ void __launch_bounds__(kFinThreads)
finalize_kernel(const double* __restrict__ partials, int nb, int width, double* __restrict__ scratch,
                unsigned* __restrict__ count, double* __restrict__ out) {
    const int tid = threadIdx.x;
    double s[kMaxWidth] = {}, c[kMaxWidth] = {};
    const int chunk = (nb + gridDim.x - 1) / gridDim.x;
    const int j0 = blockIdx.x * chunk, j1 = min(j0 + chunk, nb);
    for (int j = j0 + tid; j < j1; j += kFinThreads)
        for (int k = 0; k < width; ++k) neumaier_add(s[k], c[k], partials[(size_t)width * j + k]);
    __shared__ double rs[kMaxWidth][kFinThreads], rc[kMaxWidth][kFinThreads];
    for (int k = 0; k < width; ++k) {
        rs[k][tid] = s[k];
        rc[k][tid] = c[k];
    }
    __syncthreads();
    for (int w = kFinThreads / 2; w > 0; w /= 2) {   // pairs (s, c) + (s', c') -> (s + s', c + c' + error)
        if (tid < w) {
            for (int k = 0; k < width; ++k) {
                double a = rs[k][tid], cc = rc[k][tid] + rc[k][tid + w];
                neumaier_add(a, cc, rs[k][tid + w]);
                rs[k][tid] = a;
                rc[k][tid] = cc;
            }
        }
        __syncthreads();
    }
    if (tid < width) {
        scratch[2 * (kMaxWidth * blockIdx.x + tid)] = rs[tid][0];
        scratch[2 * (kMaxWidth * blockIdx.x + tid) + 1] = rc[tid][0];
    }
    __threadfence();   // this CTA's pair is visible before its arrival is counted
    __syncthreads();
    __shared__ bool last;
    if (tid == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (tid < width) {
        double ss = 0.0, cc = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            neumaier_add(ss, cc, __ldcg(scratch + 2 * (kMaxWidth * b + tid)));
            cc += __ldcg(scratch + 2 * (kMaxWidth * b + tid) + 1);
        }
        out[tid] = ss + cc;
    }
    if (tid == 0) *count = 0u;   // ready for the next launch on this stream
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ELBM_OK : ELBM_ERR_CUDA; }

// Nodes staged per host field transfer.
long long staging_nodes(const elbm_handle* h) {
    return h->layout == ELBM_LAYOUT_AA && h->N > kStagingChunk ? kStagingChunk : h->N;
}

// Layout of the auxiliary buffer (all offsets 256-byte aligned).
void compute_aux(elbm_handle* h) {
    AuxLayout& a = h->aux;
    a.max_blocks = h->ops->max_blocks(h->kp);
    size_t off = 0;
    a.status = off;
    off = align_up(off + sizeof(int));
    a.totals = off;
    off = align_up(off + kMaxWidth * sizeof(double));
    a.fin_count = off;
    off = align_up(off + sizeof(unsigned));
    a.fin_scratch = off;
    off = align_up(off + (size_t)2 * kMaxWidth * kFinBlocks * sizeof(double));
    a.partials = off;
    off = align_up(off + (5 + kStatsSums) * sizeof(double) * (size_t)a.max_blocks);
    a.qfield = off;
    off = align_up(off + (size_t)h->D * (size_t)h->N * h->ops->real_bytes);
    a.staging = off;
    off = align_up(off + (size_t)5 * (size_t)staging_nodes(h) * sizeof(double));
    a.bytes = off;
}

// Kernel parameters for the diagnostics: how the current state C(X_n) is laid out in the
// store (in place, or the AA layout of the step parity).
KParams diag_params(const elbm_handle* h) {
    KParams k = h->kp;
    k.aa = h->layout == ELBM_LAYOUT_AA ? (h->steps % 2 == 0 ? 1 : 2) : 0;
    return k;
}

int* status_ptr(elbm_handle* h) { return (int*)(h->auxp + h->aux.status); }
double* totals_ptr(elbm_handle* h) { return (double*)(h->auxp + h->aux.totals); }
double* step_partials(elbm_handle* h) { return (double*)(h->auxp + h->aux.partials); }
// query partials hold up to kStatsSums values per CTA (turbulence statistics)
double* query_partials(elbm_handle* h) {
    return (double*)(h->auxp + h->aux.partials) + 5 * (size_t)h->aux.max_blocks;
}
double* staging(elbm_handle* h) { return (double*)(h->auxp + h->aux.staging); }

// Host fields in page-locked memory that the device maps (cudaHostAlloc, cudaMallocHost
// or cudaHostRegister under unified addressing) are read and written by the field
// kernels themselves, over the host link, with no staging copy.  mapped_host returns the
// device address of such a buffer when [p, p + bytes) lies inside one allocation (the
// driver's range attributes), else nullptr, and the transfer goes through the staging
// area with cudaMemcpyAsync: a short or pageable buffer never reaches a kernel.
using PointerAttrFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
PointerAttrFn pointer_attr_fn() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();   // leave no sticky error behind
        return nullptr;
    }
    return reinterpret_cast<PointerAttrFn>(fn);
}

const void* mapped_host(const void* p, size_t bytes) {
    static const PointerAttrFn attr = pointer_attr_fn();   // resolved once, thread-safe
    if (!attr || !p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const CUdeviceptr dp = (CUdeviceptr)(uintptr_t)a.devicePointer;
    CUdeviceptr start = 0;
    size_t size = 0;
    if (attr(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, dp) != CUDA_SUCCESS ||
        attr(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, dp) != CUDA_SUCCESS)
        return nullptr;
    if (dp < start || bytes > size || dp - start > size - bytes) return nullptr;
    return a.devicePointer;
}

// Synchronise, read and clear the latched device status.
int sync_status(elbm_handle* h) {
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, status_ptr(h), sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    if (st != 0) {
        e = cudaMemsetAsync(status_ptr(h), 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return ELBM_ERR_CUDA;
        return (st & kStatusTimeoutBit) ? ELBM_ERR_TIMEOUT : ELBM_ERR_NONPHYSICAL;
    }
    return ELBM_OK;
}

// Reduction of nb per-CTA partial sums into out (host memory), enqueued on the handle's
// stream: written by the kernel itself when out is page-locked mapped memory, else
// reduced into the totals slot and copied; finalize_to_host also synchronises and reads
// the status.
int finalize_async(elbm_handle* h, const double* partials, int nb, double* out, int width = 5) {
    double* direct = (double*)mapped_host(out, (size_t)width * sizeof(double));
    const int grid = nb < kFinBlocks ? (nb > 0 ? nb : 1) : kFinBlocks;
    finalize_kernel<<<grid, kFinThreads, 0, h->stream>>>(partials, nb, width,
                                                         (double*)(h->auxp + h->aux.fin_scratch),
                                                         (unsigned*)(h->auxp + h->aux.fin_count),
                                                         direct ? direct : totals_ptr(h));
    ++h->launches;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !direct)
        e = cudaMemcpyAsync(out, totals_ptr(h), width * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    return e == cudaSuccess ? ELBM_OK : ELBM_ERR_CUDA;
}
int finalize_to_host(elbm_handle* h, const double* partials, int nb, double* out, int width = 5) {
    const int rc = finalize_async(h, partials, nb, out, width);
    return rc != ELBM_OK ? rc : sync_status(h);
}

// One step enqueued on stream st from the handle's current state; advances the store
// index and the step count.
cudaError_t step_one(elbm_handle* h, cudaStream_t st) {
    cudaError_t e;
    if (h->layout == ELBM_LAYOUT_AA) {   // the layout alternates: L0 after an even number of steps
        e = h->ops->step_aa(h->kp, h->pop[0], h->auxp + h->aux.qfield, step_partials(h), &h->step_blocks,
                            status_ptr(h), st, &h->launches, (int)(h->steps % 2));
        if (e == cudaSuccess) ++h->steps;
        return e;
    }
    const void* src = h->pop[h->cur];
    void* dst = h->pop[1 - h->cur];
    if (h->kernel == ELBM_KERNEL_TWOPASS)
        e = h->ops->step_twopass(h->kp, src, dst, h->auxp + h->aux.qfield, step_partials(h), &h->step_blocks,
                                 status_ptr(h), st, &h->launches);
    else if (h->kernel == ELBM_KERNEL_FUSED_REREAD)
        e = h->ops->step_fused_reread(h->kp, src, dst, step_partials(h), &h->step_blocks, status_ptr(h), st,
                                      &h->launches);
    else if (h->kernel == ELBM_KERNEL_FUSED_TMA)
        e = h->tmap_ready ? h->ops->step_fused_tma(h->kp, src, dst, &h->tmap[h->cur], step_partials(h),
                                                   &h->step_blocks, status_ptr(h), st, &h->launches)
                          : cudaErrorNotSupported;
    else if (h->tmap_ready)
        e = h->ops->step_fused_pf(h->kp, src, dst, &h->pfmap[h->cur], step_partials(h), &h->step_blocks,
                                  status_ptr(h), st, &h->launches);
    else
        e = h->ops->step_fused(h->kp, src, dst, step_partials(h), &h->step_blocks, status_ptr(h), st, &h->launches);
    if (e == cudaSuccess) {
        h->cur = 1 - h->cur;
        ++h->steps;
    }
    return e;
}

// The parity a graph starts from: the store holding the state (ping-pong) or the layout of
// the step parity (AA).  A graph of an even number of steps ends at the parity it began.
int graph_parity(const elbm_handle* h) { return h->layout == ELBM_LAYOUT_AA ? (int)(h->steps % 2) : h->cur; }

// Captures graph_steps steps from the current parity on a private stream; the handle's
// state is restored afterwards (the replays advance it).
cudaError_t build_step_graph(elbm_handle* h, cudaGraphExec_t* out) {
    cudaStream_t cap;
    cudaError_t err = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (err != cudaSuccess) return err;
    const int cur = h->cur;
    const long long steps = h->steps, launches = h->launches;
    cudaGraph_t g = nullptr;
    err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        cudaError_t le = cudaSuccess;
        for (int k = 0; k < h->graph_steps && le == cudaSuccess; ++k) le = step_one(h, cap);
        h->graph_launches = h->launches - launches;
        err = cudaStreamEndCapture(cap, &g);
        if (err == cudaSuccess) err = le;
    }
    h->cur = cur;
    h->steps = steps;
    h->launches = launches;
    if (err == cudaSuccess) err = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return err;
}

}  // namespace

extern "C" {

int elbm_create(const elbm_params* prm, elbm_handle** out) {
    if (!prm || !out) return ELBM_ERR_ARG;
    *out = nullptr;
    const elbm_params& p = *prm;
    KParams kp;
    int D = 0;
    const int rc = fill_kparams(p, kp, &D);
    if (rc != ELBM_OK) return rc;
    const long long N = kp.N;
    if (N > (1LL << 31)) return ELBM_ERR_UNSUPPORTED;

    elbm_handle* h = new (std::nothrow) elbm_handle();
    if (!h) return ELBM_ERR_ARG;
    h->prm = p;
    h->D = D;
    h->Q = D == 3 ? 27 : 9;
    h->N = N;
    h->ops = pick_ops(D, p.store);
    h->kernel = ELBM_KERNEL_FUSED;
    h->layout = ELBM_LAYOUT_PINGPONG;

    h->kp = kp;
    {
        // z segments (D3Q27) or row segments (D2Q9) sized for the waves of this device
        // (current device at creation)
        int dev = -1, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
        {
            if (D == 3) h->kp.tz = choose_tz(kp, h->ops->fused_tile_y, sms, h->ops->fused_occupancy(h->kp), kp.tz);
            else plan_d2q9(h->kp, sms, h->ops->fused_occupancy(h->kp), h->ops->march_width);
        }
        else
            cudaGetLastError();   // no device: keep the fallback, clear the error
    }
    const KParams& k = h->kp;

    h->pop_bytes = (size_t)2 * h->Q * (size_t)N * h->ops->value_bytes;
    compute_aux(h);
    *out = h;
    return ELBM_OK;
}

int elbm_bytes_required(const elbm_handle* h, size_t* pop_bytes, size_t* aux_bytes) {
    if (!h) return ELBM_ERR_ARG;
    if (pop_bytes) *pop_bytes = h->pop_bytes;
    if (aux_bytes) *aux_bytes = h->aux.bytes;
    return ELBM_OK;
}

int elbm_bind(elbm_handle* h, void* pop_a, void* pop_b, void* aux, void* stream) {
    if (!h || !pop_a || !aux) return ELBM_ERR_ARG;
    const bool aa = h->layout == ELBM_LAYOUT_AA;
    if (aa) {
        if (pop_b && pop_b != pop_a) return ELBM_ERR_ARG;   // one store
        pop_b = pop_a;
    } else if (!pop_b || pop_a == pop_b) {
        return ELBM_ERR_ARG;
    }
    if (((uintptr_t)pop_a | (uintptr_t)pop_b | (uintptr_t)aux) % kAlign) return ELBM_ERR_ARG;
    h->drop_graphs();
    h->pop[0] = pop_a;
    h->pop[1] = pop_b;
    h->tmap_ready = false;
    if (!aa && h->ops->tma_supported(h->kp))
        h->tmap_ready = h->ops->encode_tmap(h->kp, pop_a, &h->tmap[0], kTmapStage) == 1 &&
                        h->ops->encode_tmap(h->kp, pop_b, &h->tmap[1], kTmapStage) == 1 &&
                        h->ops->encode_tmap(h->kp, pop_a, &h->pfmap[0], kTmapPrefetch) == 1 &&
                        h->ops->encode_tmap(h->kp, pop_b, &h->pfmap[1], kTmapPrefetch) == 1;
    h->auxp = (char*)aux;
    h->stream = (cudaStream_t)stream;
    h->cur = 0;
    h->bound = true;
    cudaError_t e = cudaMemsetAsync(status_ptr(h), 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->auxp + h->aux.fin_count, 0, sizeof(unsigned), h->stream);
    return cuda_status(e);
}

// AA: C(X_0) in layout L0 from equilibria already written in place (a step from layout L1
// collides them without streaming).
int aa_collide_initial(elbm_handle* h) {
    int nb = 0;
    return cuda_status(h->ops->step_aa(h->kp, h->pop[0], h->auxp + h->aux.qfield, query_partials(h), &nb,
                                       status_ptr(h), h->stream, &h->launches, 1));
}

int elbm_set_fields_device(elbm_handle* h, const double* rho, const double* u, const double* T) {
    if (!h || !h->bound || !rho || !u || !T) return ELBM_ERR_ARG;
    h->cur = 0;
    h->steps = 0;
    if (h->layout == ELBM_LAYOUT_AA) {
        const int rc = cuda_status(h->ops->init_nodes(h->kp, rho, u, T, h->pop[0], 0, h->N, status_ptr(h),
                                                      h->stream, &h->launches));
        return rc != ELBM_OK ? rc : aa_collide_initial(h);
    }
    return cuda_status(h->ops->init(h->kp, rho, u, T, h->pop[0], h->pop[1], h->auxp + h->aux.qfield,
                                    query_partials(h), status_ptr(h), h->stream, &h->launches));
}

int elbm_set_fields(elbm_handle* h, const double* rho, const double* u, const double* T) {
    if (!h || !h->bound || !rho || !u || !T) return ELBM_ERR_ARG;
    {
        const size_t b = (size_t)h->N * sizeof(double);
        const double* dr = (const double*)mapped_host(rho, b);
        const double* du = dr ? (const double*)mapped_host(u, (size_t)h->D * b) : nullptr;
        const double* dT = du ? (const double*)mapped_host(T, b) : nullptr;
        if (dT) {   // page-locked fields: the initialisation kernel reads them directly
            const int rc = elbm_set_fields_device(h, dr, du, dT);
            return rc != ELBM_OK ? rc : sync_status(h);
        }
    }
    if (h->layout == ELBM_LAYOUT_AA) {   // chunks of staging_nodes(h) nodes
        h->cur = 0;
        h->steps = 0;
        const long long N = h->N, C = staging_nodes(h);
        double* st = staging(h);
        for (long long n0 = 0; n0 < N; n0 += C) {
            const long long c = N - n0 < C ? N - n0 : C;
            cudaError_t e = cudaMemcpyAsync(st, rho + n0, c * sizeof(double), cudaMemcpyHostToDevice, h->stream);
            for (int d = 0; d < h->D && e == cudaSuccess; ++d)
                e = cudaMemcpyAsync(st + (1 + d) * c, u + d * N + n0, c * sizeof(double), cudaMemcpyHostToDevice,
                                    h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(st + (1 + h->D) * c, T + n0, c * sizeof(double), cudaMemcpyHostToDevice,
                                    h->stream);
            if (e == cudaSuccess)
                e = h->ops->init_nodes(h->kp, st, st + c, st + (1 + h->D) * c, h->pop[0], n0, c, status_ptr(h),
                                       h->stream, &h->launches);
            if (e != cudaSuccess) return ELBM_ERR_CUDA;
        }
        const int rc = aa_collide_initial(h);
        return rc != ELBM_OK ? rc : sync_status(h);
    }
    const size_t N = (size_t)h->N;
    double* st = staging(h);
    cudaError_t e = cudaMemcpyAsync(st, rho, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st + N, u, (size_t)h->D * N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st + (1 + h->D) * N, T, N * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    int rc = elbm_set_fields_device(h, st, st + N, st + (1 + h->D) * N);
    if (rc != ELBM_OK) return rc;
    return sync_status(h);
}

int elbm_step(elbm_handle* h, int nsteps) {
    if (!h || !h->bound || nsteps < 0) return ELBM_ERR_ARG;
    if (h->kernel == ELBM_KERNEL_FUSED_TMA && !h->tmap_ready) return ELBM_ERR_UNSUPPORTED;
    int s = 0;
    if (h->graph_steps > 0) {   // whole groups of graph_steps steps, each one graph replay
        for (; s + h->graph_steps <= nsteps; s += h->graph_steps) {
            cudaGraphExec_t& g = h->gexec[graph_parity(h)];
            cudaError_t e = g ? cudaSuccess : build_step_graph(h, &g);
            if (e == cudaSuccess) e = cudaGraphLaunch(g, h->stream);
            if (e != cudaSuccess) return ELBM_ERR_CUDA;
            h->steps += h->graph_steps;   // an even count: the store index is where it was
            h->launches += h->graph_launches;
        }
    }
    for (; s < nsteps; ++s)
        if (step_one(h, h->stream) != cudaSuccess) return ELBM_ERR_CUDA;
    return ELBM_OK;
}

int elbm_set_step_graph(elbm_handle* h, int steps_per_graph) {
    if (!h || steps_per_graph < 0 || steps_per_graph > 1024 || steps_per_graph % 2) return ELBM_ERR_ARG;
    h->drop_graphs();
    h->graph_steps = steps_per_graph;
    return ELBM_OK;
}

int elbm_get_fields_device(elbm_handle* h, double* rho, double* u, double* T) {
    if (!h || !h->bound || !rho || !u || !T) return ELBM_ERR_ARG;
    return cuda_status(h->ops->fields(diag_params(h), h->pop[h->cur], rho, u, T, status_ptr(h), h->stream,
                                      &h->launches));
}

int elbm_get_fields(elbm_handle* h, double* rho, double* u, double* T) {
    if (!h || !h->bound || !rho || !u || !T) return ELBM_ERR_ARG;
    {
        const size_t b = (size_t)h->N * sizeof(double);
        double* dr = (double*)mapped_host(rho, b);
        double* du = dr ? (double*)mapped_host(u, (size_t)h->D * b) : nullptr;
        double* dT = du ? (double*)mapped_host(T, b) : nullptr;
        if (dT) {   // page-locked fields: the field kernel writes them directly
            const int rc = elbm_get_fields_device(h, dr, du, dT);
            return rc != ELBM_OK ? rc : sync_status(h);
        }
    }
    if (h->layout == ELBM_LAYOUT_AA) {   // chunks of staging_nodes(h) nodes
        const long long N = h->N, C = staging_nodes(h);
        const KParams k = diag_params(h);
        double* st = staging(h);
        for (long long n0 = 0; n0 < N; n0 += C) {
            const long long c = N - n0 < C ? N - n0 : C;
            cudaError_t e = h->ops->fields_nodes(k, h->pop[0], st, st + c, st + (1 + h->D) * c, n0, c,
                                                 status_ptr(h), h->stream, &h->launches);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(rho + n0, st, c * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            for (int d = 0; d < h->D && e == cudaSuccess; ++d)
                e = cudaMemcpyAsync(u + d * N + n0, st + (1 + d) * c, c * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(T + n0, st + (1 + h->D) * c, c * sizeof(double), cudaMemcpyDeviceToHost,
                                    h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // the staging area is reused
            if (e != cudaSuccess) return ELBM_ERR_CUDA;
        }
        return sync_status(h);
    }
    const size_t N = (size_t)h->N;
    double* st = staging(h);
    int rc = elbm_get_fields_device(h, st, st + N, st + (1 + h->D) * N);
    if (rc != ELBM_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(rho, st, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(u, st + N, (size_t)h->D * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(T, st + (1 + h->D) * N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    return sync_status(h);
}

int elbm_conservation(elbm_handle* h, double out[5]) {
    if (!h || !h->bound || !out) return ELBM_ERR_ARG;
    int nb = 0;
    cudaError_t e = h->ops->conservation(diag_params(h), h->pop[h->cur], query_partials(h), &nb, h->stream,
                                         &h->launches);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    return finalize_to_host(h, query_partials(h), nb, out);
}

int elbm_turbulence_stats(elbm_handle* h, double out[13]) {
    if (!h || !h->bound || !out) return ELBM_ERR_ARG;
    int nb = 0;
    double* part = query_partials(h);   // kStatsSums values x (<= max_blocks) CTAs
    cudaError_t e = h->ops->stats(diag_params(h), h->pop[h->cur], part, &nb, h->stream, &h->launches);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    double sums[kStatsSums];
    const int rc = finalize_to_host(h, part, nb, sums, kStatsSums);
    if (rc != ELBM_OK) return rc;
    const double N = (double)h->N;
    const double mrho = sums[0] / N, mT = sums[5] / N;
    out[0] = mrho;                                               // <rho>
    out[1] = std::sqrt(std::fmax(sums[1] / N - mrho * mrho, 0.0));   // rho_rms
    out[2] = 0.5 * sums[2] / N;                                  // K = <rho u.u>/2
    out[3] = std::sqrt(sums[3] / N / h->D);                      // u_rms = sqrt(<u.u>/D)
    out[4] = std::sqrt(sums[4] / N);                             // theta_rms
    out[5] = mT;                                                 // <T>
    out[6] = std::sqrt(std::fmax(sums[6] / N - mT * mT, 0.0));   // T_rms
    out[7] = sums[7] / N;                                        // <(d u_x/d x)^2>
    out[8] = std::sqrt(sums[8] / N);                             // omega_rms = sqrt(<|omega|^2>)
    out[9] = 0.5 * sums[8] / N;                                  // enstrophy = <|omega|^2>/2
    out[10] = sums[10] / N;                                      // dissipation <mu |omega|^2>
    // Taylor microscale and its Reynolds number (Eq. Taylor_Re, with the square root)
    const double lam = sums[7] > 0.0 ? std::sqrt(sums[9] / sums[7]) : 0.0;
    out[11] = lam;                                               // lambda = sqrt(<u_x^2>/<(d u_x/d x)^2>)
    out[12] = mrho * out[3] * lam / h->prm.mu0;                  // Re_lambda = <rho> u_rms lambda / mu0
    return ELBM_OK;
}

int elbm_step_totals(elbm_handle* h, double out[5]) {
    if (!h || !h->bound || !out) return ELBM_ERR_ARG;
    if (h->steps == 0) return ELBM_ERR_ARG;
    return finalize_to_host(h, step_partials(h), h->step_blocks, out);
}

int elbm_step_totals_async(elbm_handle* h, double out[5]) {
    if (!h || !h->bound || !out) return ELBM_ERR_ARG;
    if (h->steps == 0) return ELBM_ERR_ARG;
    return finalize_async(h, step_partials(h), h->step_blocks, out);
}

int elbm_set_kernel(elbm_handle* h, int kernel) {
    if (!h || (kernel != ELBM_KERNEL_FUSED && kernel != ELBM_KERNEL_TWOPASS && kernel != ELBM_KERNEL_FUSED_REREAD &&
               kernel != ELBM_KERNEL_FUSED_TMA))
        return ELBM_ERR_ARG;
    if (kernel == ELBM_KERNEL_FUSED_TMA && !h->ops->tma_supported(h->kp)) return ELBM_ERR_UNSUPPORTED;
    if (h->layout == ELBM_LAYOUT_AA && kernel != ELBM_KERNEL_TWOPASS) return ELBM_ERR_UNSUPPORTED;
    h->kernel = kernel;
    h->drop_graphs();
    return ELBM_OK;
}

int elbm_set_layout(elbm_handle* h, int layout) {
    if (!h || h->bound || (layout != ELBM_LAYOUT_PINGPONG && layout != ELBM_LAYOUT_AA)) return ELBM_ERR_ARG;
    if (layout == ELBM_LAYOUT_AA && !(h->kp.per_x && h->kp.per_y && h->kp.per_z)) return ELBM_ERR_UNSUPPORTED;
    h->layout = layout;
    h->kernel = layout == ELBM_LAYOUT_AA ? ELBM_KERNEL_TWOPASS : ELBM_KERNEL_FUSED;
    compute_aux(h);
    return ELBM_OK;
}

int elbm_set_tile_z(elbm_handle* h, int tz) {
    if (!h || tz < 1) return ELBM_ERR_ARG;
    KParams k = h->kp;
    const int planes = h->D == 3 ? h->prm.nz : h->prm.ny;   // the marched axis
    k.tz = tz < planes ? tz : planes;
    k.tile2d = 0;   // D2Q9: an explicit row segment selects the row march
    if (h->ops->max_blocks(k) > h->aux.max_blocks) return ELBM_ERR_ARG;   // partials would not fit
    h->kp.tz = k.tz;
    h->kp.tile2d = 0;
    h->drop_graphs();
    return ELBM_OK;
}

int elbm_get_populations(elbm_handle* h, void* host_dst) {
    if (!h || !h->bound || !host_dst) return ELBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(host_dst, h->pop[h->cur], h->pop_bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    return sync_status(h);
}

int elbm_set_populations(elbm_handle* h, const void* host_src) {
    if (!h || !h->bound || !host_src) return ELBM_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(h->pop[h->cur], host_src, h->pop_bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return ELBM_ERR_CUDA;
    return sync_status(h);
}

int elbm_sync(elbm_handle* h) {
    if (!h || !h->bound) return ELBM_ERR_ARG;
    return sync_status(h);
}

int elbm_inject_wait_timeout(elbm_handle* h, int on) {
    if (!h || (on != 0 && on != 1)) return ELBM_ERR_ARG;
    h->kp.inject_tx = on ? 16u : 0u;
    h->drop_graphs();
    return ELBM_OK;
}

long long elbm_steps_done(const elbm_handle* h) { return h ? h->steps : -1; }

long long elbm_launch_count(const elbm_handle* h) { return h ? h->launches : -1; }

int elbm_velocity(int lattice, int i, int c[3]) {
    const int Q = lattice == ELBM_D3Q27 ? 27 : (lattice == ELBM_D2Q9 ? 9 : 0);
    if (!Q || i < 0 || i >= Q || !c) return ELBM_ERR_ARG;
    c[0] = i % 3 - 1;
    c[1] = (i / 3) % 3 - 1;
    c[2] = Q == 27 ? i / 9 - 1 : 0;
    return ELBM_OK;
}

int elbm_destroy(elbm_handle* h) {
    delete h;
    return ELBM_OK;
}

const char* elbm_status_str(int code) {
    switch (code) {
        case ELBM_OK: return "ok";
        case ELBM_ERR_ARG: return "invalid argument";
        case ELBM_ERR_UNSUPPORTED: return "unsupported combination";
        case ELBM_ERR_CUDA: return "CUDA runtime error";
        case ELBM_ERR_NONPHYSICAL: return "non-physical state (non-finite, rho <= 0 or T <= 0)";
        case ELBM_ERR_TIMEOUT: return "bounded device wait timed out";
    }
    return "unknown status";
}

}  // extern "C"
