// Ensembles of independent D2Q9 instances of uneven sizes (one population store
// holding all instances back to back), stepped either by one persistent launch over
// the work units of every instance (replayed from CUDA graphs of several steps) or by
// one launch per instance.  A work unit is a 32 x ty tile (ty = 4, 8, 16) or a strip of
// kMarchW2 nodes marched along y over a segment of rows (kMarchSegs); the persistent
// schedule (unit and CTAs per SM) is chosen by a small autotuner that times the
// candidates on the bound buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "elbm.h"
#include "elbm_internal.h"

using namespace elbm;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kTileX = 32;
constexpr int kNSched = 6;
constexpr int kTYs[kNSched] = {4, 8, 16, kMarchSegs[0], kMarchSegs[1], kMarchSegs[2]};
// steps per CUDA graph of the persistent schedule (even, so a replay ends in the store
// it started from); shorter requests use one-step graphs
constexpr int kGraphSteps = 8;

const Ops* ops_2d(int store) {
    switch (store) {
        case ELBM_F64: return ops_d2_f64();
        case ELBM_F32: return ops_d2_f32();
        case ELBM_F16DEV: return ops_d2_f16();
        case ELBM_BF16DEV: return ops_d2_bf16();
    }
    return nullptr;
}

int ty_index(int ty) {
    for (int t = 0; t < kNSched; ++t)
        if (kTYs[t] == ty) return t;
    return 1;
}
bool valid_ty(int ty) {
    for (int t = 0; t < kNSched; ++t)
        if (kTYs[t] == ty) return true;
    return false;
}

// tuned schedules, cached per (store, size class = log2 of the total node count)
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, std::pair<int, int>> g_tune_cache;

}  // namespace

struct elbm_ensemble {
    int n = 0;
    int store = 0;
    const Ops* ops = nullptr;
    std::vector<KParams> kp;
    std::vector<long long> offset;             // element offsets
    std::vector<int> tile_start[kNSched], tiles_x[kNSched];  // work units per schedule
    long long total_nodes = 0, max_nodes = 0;
    size_t pop_bytes = 0;
    // aux layout
    size_t a_status = 0, a_params = 0, a_offset = 0, a_tstart[kNSched] = {}, a_tx[kNSched] = {};
    size_t a_qfield = 0, a_partials = 0, a_staging = 0, aux_bytes = 0;
    int max_blocks = 0;
    // binding
    void* pop[2] = {nullptr, nullptr};
    char* aux = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false;
    int cur = 0;
    // schedule
    int mode = ELBM_ENSEMBLE_PERSISTENT;
    int ty = kMarchSegs[1], ctas_per_sm = 2, grid = 0;
    bool use_graph = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};    // one step from store c to store 1-c
    cudaGraphExec_t graphk[2] = {nullptr, nullptr};   // kGraphSteps steps from store c back to c
    long long steps = 0, launches = 0;

    int* status() { return (int*)(aux + a_status); }
    EnsembleArgs args(int tyi) const {
        EnsembleArgs a;
        a.params = (const KParams*)(aux + a_params);
        a.offset = (const long long*)(aux + a_offset);
        a.tile_start = (const int*)(aux + a_tstart[tyi]);
        a.tiles_x = (const int*)(aux + a_tx[tyi]);
        a.n = n;
        a.ntiles = tile_start[tyi][n];
        a.caloric = 0;
        for (const KParams& k : kp) a.caloric |= k.eos;
        return a;
    }
    void drop_graphs() {
        for (auto* gs : {graph, graphk})
            for (int c = 0; c < 2; ++c)
                if (gs[c]) {
                    cudaGraphExecDestroy(gs[c]);
                    gs[c] = nullptr;
                }
    }
};

namespace {

int ens_sync(elbm_ensemble* e) {
    int st = 0;
    cudaError_t c = cudaMemcpyAsync(&st, e->status(), sizeof(int), cudaMemcpyDeviceToHost, e->stream);
    if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);
    if (c != cudaSuccess) return ELBM_ERR_CUDA;
    if (st != 0) {
        if (cudaMemsetAsync(e->status(), 0, sizeof(int), e->stream) != cudaSuccess) return ELBM_ERR_CUDA;
        if (cudaStreamSynchronize(e->stream) != cudaSuccess) return ELBM_ERR_CUDA;
        return ELBM_ERR_NONPHYSICAL;
    }
    return ELBM_OK;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

void set_schedule(elbm_ensemble* e, int ty, int ctas) {
    e->ty = ty;
    e->ctas_per_sm = ctas;
    const long long ntiles = e->tile_start[ty_index(ty)][e->n];
    long long g = (long long)ctas * sm_count();
    e->grid = (int)(g < ntiles ? g : ntiles);
    e->drop_graphs();
}

cudaError_t launch_persistent(elbm_ensemble* e, const void* src, void* dst, cudaStream_t s) {
    return e->ops->step_ensemble(e->args(ty_index(e->ty)), src, dst, e->status(), e->ty, e->grid, s, &e->launches);
}

// graph of `steps` persistent steps starting from store c (alternating stores)
cudaError_t build_graph(elbm_ensemble* e, int c, int steps, cudaGraphExec_t* out) {
    cudaStream_t cap;
    cudaError_t err = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (err != cudaSuccess) return err;
    cudaGraph_t g = nullptr;
    err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        const long long before = e->launches;
        cudaError_t le = cudaSuccess;
        for (int s = 0; s < steps && le == cudaSuccess; ++s)
            le = launch_persistent(e, e->pop[(c + s) & 1], e->pop[(c + s + 1) & 1], cap);
        e->launches = before;   // counted when the graph is launched
        err = cudaStreamEndCapture(cap, &g);
        if (err == cudaSuccess) err = le;
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    return err;
}

int step_once(elbm_ensemble* e) {
    const int c = e->cur;
    cudaError_t err = cudaSuccess;
    if (e->mode == ELBM_ENSEMBLE_PER_INSTANCE) {
        for (int k = 0; k < e->n && err == cudaSuccess; ++k) {
            const size_t off = (size_t)e->offset[k] * e->ops->value_bytes * 2;
            int nb = 0;
            err = e->ops->step_fused(e->kp[k], (const char*)e->pop[c] + off, (char*)e->pop[1 - c] + off,
                                     (double*)(e->aux + e->a_partials), &nb, e->status(), e->stream, &e->launches);
        }
    } else if (e->use_graph) {
        if (!e->graph[c]) err = build_graph(e, c, 1, &e->graph[c]);
        if (err == cudaSuccess) err = cudaGraphLaunch(e->graph[c], e->stream);
        ++e->launches;
    } else {
        err = launch_persistent(e, e->pop[c], e->pop[1 - c], e->stream);
    }
    if (err != cudaSuccess) return ELBM_ERR_CUDA;
    e->cur = 1 - c;
    ++e->steps;
    return ELBM_OK;
}

}  // namespace

extern "C" {

int elbm_ensemble_create(const elbm_params* params, int n, elbm_ensemble** out) {
    if (!params || !out || n < 1 || n > kMaxEnsemble) return ELBM_ERR_ARG;
    *out = nullptr;
    const int store = params[0].store;
    const Ops* ops = ops_2d(store);
    if (!ops) return ELBM_ERR_ARG;
    elbm_ensemble* e = new (std::nothrow) elbm_ensemble();
    if (!e) return ELBM_ERR_ARG;
    e->n = n;
    e->store = store;
    e->ops = ops;
    e->kp.resize(n);
    e->offset.resize(n);
    long long off = 0;
    for (int k = 0; k < n; ++k) {
        int D = 0;
        if (params[k].store != store || params[k].lattice != ELBM_D2Q9) { delete e; return ELBM_ERR_ARG; }
        if (fill_kparams(params[k], e->kp[k], &D) != ELBM_OK) { delete e; return ELBM_ERR_ARG; }
        e->offset[k] = off;
        off += 9LL * e->kp[k].N;   // pair elements of instance k
        e->total_nodes += e->kp[k].N;
        if (e->kp[k].N > e->max_nodes) e->max_nodes = e->kp[k].N;
    }
    if (e->total_nodes > (1LL << 31)) { delete e; return ELBM_ERR_UNSUPPORTED; }
    for (int t = 0; t < kNSched; ++t) {
        e->tile_start[t].resize(n + 1);
        e->tiles_x[t].resize(n);
        const int width = kTYs[t] > 16 ? kMarchW2 : kTileX;   // march strips or tiles
        int acc = 0;
        for (int k = 0; k < n; ++k) {
            const int txn = (e->kp[k].nx + width - 1) / width, tyn = (e->kp[k].ny + kTYs[t] - 1) / kTYs[t];
            e->tile_start[t][k] = acc;
            e->tiles_x[t][k] = txn;
            acc += txn * tyn;
        }
        e->tile_start[t][n] = acc;
    }
    e->pop_bytes = (size_t)off * ops->value_bytes * 2;
    // aux layout
    // per-CTA partials of the one-launch-per-instance mode: its row segments are chosen
    // for the device at bind, no shorter than 16 rows, so size for that
    int maxb = 0;
    for (int k = 0; k < n; ++k) {
        KParams shortest = e->kp[k];
        shortest.tz = shortest.ny < 16 ? shortest.ny : 16;
        const int b = std::max(ops->max_blocks(e->kp[k]), ops->max_blocks(shortest));
        if (b > maxb) maxb = b;
    }
    e->max_blocks = maxb;
    size_t o = 0;
    e->a_status = o; o = align_up(o + sizeof(int));
    e->a_params = o; o = align_up(o + (size_t)n * sizeof(KParams));
    e->a_offset = o; o = align_up(o + (size_t)n * sizeof(long long));
    for (int t = 0; t < kNSched; ++t) {
        e->a_tstart[t] = o; o = align_up(o + (size_t)(n + 1) * sizeof(int));
        e->a_tx[t] = o; o = align_up(o + (size_t)n * sizeof(int));
    }
    e->a_partials = o; o = align_up(o + (size_t)maxb * 5 * sizeof(double));
    e->a_qfield = o; o = align_up(o + (size_t)2 * e->max_nodes * ops->real_bytes);
    e->a_staging = o; o = align_up(o + (size_t)4 * e->max_nodes * sizeof(double));
    e->aux_bytes = o;
    set_schedule(e, kMarchSegs[1], 2);
    e->grid = 0;   // set at bind (needs the device)
    *out = e;
    return ELBM_OK;
}

int elbm_ensemble_bytes_required(const elbm_ensemble* e, size_t* pop_bytes, size_t* aux_bytes) {
    if (!e) return ELBM_ERR_ARG;
    if (pop_bytes) *pop_bytes = e->pop_bytes;
    if (aux_bytes) *aux_bytes = e->aux_bytes;
    return ELBM_OK;
}

int elbm_ensemble_bind(elbm_ensemble* e, void* pop_a, void* pop_b, void* aux, void* stream) {
    if (!e || !pop_a || !pop_b || !aux || pop_a == pop_b) return ELBM_ERR_ARG;
    if (((uintptr_t)pop_a | (uintptr_t)pop_b | (uintptr_t)aux) % kAlign) return ELBM_ERR_ARG;
    e->drop_graphs();
    e->pop[0] = pop_a;
    e->pop[1] = pop_b;
    e->aux = (char*)aux;
    e->stream = (cudaStream_t)stream;
    e->cur = 0;
    e->bound = true;
    // the one-launch-per-instance mode runs each instance as a single lattice would on this device
    const int sms = sm_count();
    for (KParams& k : e->kp) plan_d2q9(k, sms, e->ops->fused_occupancy(k), e->ops->march_width);
    cudaError_t c = cudaMemsetAsync(e->status(), 0, sizeof(int), e->stream);
    if (c == cudaSuccess)
        c = cudaMemcpyAsync(e->aux + e->a_params, e->kp.data(), e->kp.size() * sizeof(KParams),
                            cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess)
        c = cudaMemcpyAsync(e->aux + e->a_offset, e->offset.data(), e->offset.size() * sizeof(long long),
                            cudaMemcpyHostToDevice, e->stream);
    for (int t = 0; t < kNSched && c == cudaSuccess; ++t) {
        c = cudaMemcpyAsync(e->aux + e->a_tstart[t], e->tile_start[t].data(), (e->n + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, e->stream);
        if (c == cudaSuccess)
            c = cudaMemcpyAsync(e->aux + e->a_tx[t], e->tiles_x[t].data(), e->n * sizeof(int),
                                cudaMemcpyHostToDevice, e->stream);
    }
    if (c == cudaSuccess) c = cudaStreamSynchronize(e->stream);
    if (c != cudaSuccess) return ELBM_ERR_CUDA;
    set_schedule(e, e->ty, e->ctas_per_sm);
    return ELBM_OK;
}

int elbm_ensemble_set_fields(elbm_ensemble* e, int k, const double* rho, const double* u, const double* T) {
    if (!e || !e->bound || k < 0 || k >= e->n || !rho || !u || !T) return ELBM_ERR_ARG;
    const KParams& p = e->kp[k];
    const size_t N = (size_t)p.N;
    double* st = (double*)(e->aux + e->a_staging);
    cudaError_t c = cudaMemcpyAsync(st, rho, N * sizeof(double), cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess) c = cudaMemcpyAsync(st + N, u, 2 * N * sizeof(double), cudaMemcpyHostToDevice, e->stream);
    if (c == cudaSuccess) c = cudaMemcpyAsync(st + 3 * N, T, N * sizeof(double), cudaMemcpyHostToDevice, e->stream);
    if (c != cudaSuccess) return ELBM_ERR_CUDA;
    const size_t off = (size_t)e->offset[k] * e->ops->value_bytes * 2;
    c = e->ops->init(p, st, st + N, st + 3 * N, (char*)e->pop[e->cur] + off, (char*)e->pop[1 - e->cur] + off,
                     e->aux + e->a_qfield, (double*)(e->aux + e->a_partials), e->status(), e->stream, &e->launches);
    if (c != cudaSuccess) return ELBM_ERR_CUDA;
    e->steps = 0;
    return ens_sync(e);
}

int elbm_ensemble_get_fields(elbm_ensemble* e, int k, double* rho, double* u, double* T) {
    if (!e || !e->bound || k < 0 || k >= e->n || !rho || !u || !T) return ELBM_ERR_ARG;
    const KParams& p = e->kp[k];
    const size_t N = (size_t)p.N;
    double* st = (double*)(e->aux + e->a_staging);
    const size_t off = (size_t)e->offset[k] * e->ops->value_bytes * 2;
    cudaError_t c = e->ops->fields(p, (const char*)e->pop[e->cur] + off, st, st + N, st + 3 * N, e->status(),
                                   e->stream, &e->launches);
    if (c == cudaSuccess) c = cudaMemcpyAsync(rho, st, N * sizeof(double), cudaMemcpyDeviceToHost, e->stream);
    if (c == cudaSuccess) c = cudaMemcpyAsync(u, st + N, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, e->stream);
    if (c == cudaSuccess) c = cudaMemcpyAsync(T, st + 3 * N, N * sizeof(double), cudaMemcpyDeviceToHost, e->stream);
    if (c != cudaSuccess) return ELBM_ERR_CUDA;
    return ens_sync(e);
}

int elbm_ensemble_set_mode(elbm_ensemble* e, int mode, int use_graph) {
    if (!e || (mode != ELBM_ENSEMBLE_PERSISTENT && mode != ELBM_ENSEMBLE_PER_INSTANCE)) return ELBM_ERR_ARG;
    e->mode = mode;
    e->use_graph = use_graph != 0;
    return ELBM_OK;
}

int elbm_ensemble_set_schedule(elbm_ensemble* e, int tile_y, int ctas_per_sm) {
    if (!e || !valid_ty(tile_y) || ctas_per_sm < 1 || ctas_per_sm > 32) return ELBM_ERR_ARG;
    set_schedule(e, tile_y, ctas_per_sm);
    return ELBM_OK;
}

int elbm_ensemble_get_schedule(const elbm_ensemble* e, int* tile_y, int* ctas_per_sm, int* grid) {
    if (!e) return ELBM_ERR_ARG;
    if (tile_y) *tile_y = e->ty;
    if (ctas_per_sm) *ctas_per_sm = e->ctas_per_sm;
    if (grid) *grid = e->grid;
    return ELBM_OK;
}

int elbm_ensemble_tune(elbm_ensemble* e, int trial_steps, int use_cache) {
    if (!e || !e->bound || trial_steps < 1) return ELBM_ERR_ARG;
    int sc = 0;
    for (long long v = e->total_nodes; v > 1; v >>= 1) ++sc;
    const std::pair<int, int> key(e->store, sc);
    if (use_cache) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            set_schedule(e, it->second.first, it->second.second);
            return ELBM_OK;
        }
    }
    // Candidates run src -> dst without swapping, so the state in the current store
    // is left as it was.
    cudaEvent_t t0, t1;
    if (cudaEventCreate(&t0) != cudaSuccess) return ELBM_ERR_CUDA;
    if (cudaEventCreate(&t1) != cudaSuccess) { cudaEventDestroy(t0); return ELBM_ERR_CUDA; }
    float best = -1.f;
    int best_ty = 8, best_c = 1;
    const long long launches0 = e->launches;
    int rc = ELBM_OK;
    for (int t = 0; t < kNSched && rc == ELBM_OK; ++t) {
        const int ty = kTYs[t];
        const int occ = e->ops->ensemble_occupancy(ty);
        for (int c = 1; c <= occ && rc == ELBM_OK; ++c) {
            set_schedule(e, ty, c);
            if (launch_persistent(e, e->pop[e->cur], e->pop[1 - e->cur], e->stream) != cudaSuccess) { rc = ELBM_ERR_CUDA; break; }
            cudaEventRecord(t0, e->stream);
            for (int s = 0; s < trial_steps; ++s)
                if (launch_persistent(e, e->pop[e->cur], e->pop[1 - e->cur], e->stream) != cudaSuccess) rc = ELBM_ERR_CUDA;
            cudaEventRecord(t1, e->stream);
            if (cudaEventSynchronize(t1) != cudaSuccess) { rc = ELBM_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, t0, t1);
            if (best < 0.f || ms < best) { best = ms; best_ty = ty; best_c = c; }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    e->launches = launches0;
    set_schedule(e, best_ty, best_c);
    if (rc != ELBM_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = {best_ty, best_c};
    }
    return ens_sync(e);
}

int elbm_ensemble_step(elbm_ensemble* e, int nsteps) {
    if (!e || !e->bound || nsteps < 0) return ELBM_ERR_ARG;
    int s = 0;
    if (e->mode == ELBM_ENSEMBLE_PERSISTENT && e->use_graph) {
        // whole groups of kGraphSteps steps from one graph each (the store parity is back
        // where it started after each group)
        for (; s + kGraphSteps <= nsteps; s += kGraphSteps) {
            const int c = e->cur;
            cudaError_t err = cudaSuccess;
            if (!e->graphk[c]) err = build_graph(e, c, kGraphSteps, &e->graphk[c]);
            if (err == cudaSuccess) err = cudaGraphLaunch(e->graphk[c], e->stream);
            if (err != cudaSuccess) return ELBM_ERR_CUDA;
            e->launches += kGraphSteps;
            e->steps += kGraphSteps;
        }
    }
    for (; s < nsteps; ++s) {
        const int rc = step_once(e);
        if (rc != ELBM_OK) return rc;
    }
    return ELBM_OK;
}

int elbm_ensemble_sync(elbm_ensemble* e) {
    if (!e || !e->bound) return ELBM_ERR_ARG;
    return ens_sync(e);
}

long long elbm_ensemble_launch_count(const elbm_ensemble* e) { return e ? e->launches : -1; }

long long elbm_ensemble_nodes(const elbm_ensemble* e) { return e ? e->total_nodes : -1; }

int elbm_ensemble_destroy(elbm_ensemble* e) {
    if (e) e->drop_graphs();
    delete e;
    return ELBM_OK;
}

}  // extern "C"
