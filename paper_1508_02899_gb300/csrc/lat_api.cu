// Host side of the C ABI declared in include/lat.h: argument validation, the stability checks
// of Eq. (cfl) and Eq. (stabLapl), context scratch, CUDA-graph capture of multi-step runs,
// the launch-shape autotuner and the moment reductions.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "lat_internal.h"
#include "lat2d.h"
#include "learn.h"

using namespace lat;

namespace {

__global__ void k_set_noise_window(DevState* st, long long base, long long rows) {
    st->noise_base = base;
    st->noise_rows = rows;
}
__global__ void k_clear_status(DevState* st) { st->status = 0u; }

}  // namespace

struct lat_ctx {
    int d = 1;
    int dtype = LAT_F32;
    int nv = 0;
    int n_inst = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;      // capture stream (graphs are launched on `stream`)
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    long long h_step = 0;
    int sm_count = 0;

    // 1D instances and work items
    std::vector<Inst1D> h_inst;
    Inst1D* d_inst = nullptr;
    long long total_x = 0;
    int2* d_items = nullptr;
    int* d_inst_begin = nullptr;
    std::vector<int> h_inst_begin;
    int nitems = 0;
    double* d_partials = nullptr;
    double* d_glob = nullptr;
    double* h_glob = nullptr;       // pinned

    // flow
    int flow_kind = LAT_FLOW_NONE;
    int nmodes = 0;
    int k1d[kMaxModes1D] = {0};
    bool frozen = true;
    const void* field = nullptr;
    double* d_amp = nullptr;        // [2][n_inst][2M]
    float* d_ampf = nullptr;        // FP32 copy for the FP32 kernels
    long long amp_stride = 0;
    double* d_noise = nullptr;
    long long noise_cap = 0;        // doubles
    long long noise_row_len = 0;    // doubles per row

    DevState* d_state = nullptr;
    DevState* h_state = nullptr;    // pinned

    // drag scheme (1D)
    int scheme = LAT_SCHEME_UPWIND;
    double mu = 2.0 / 3.0;

    // launch shape: kernel variant (plain loads or bulk-copy ring), threads per block (= tile
    // width), ring slots, resident blocks per SM of the persistent grid, launch mode
    int variant = STEP1D_PLAIN, block = 256, slots = 3, bps = 4, mode = 0;
    bool ring_ok = false;

    // cached graphs keyed by the number of steps (buffers are picked by the device step parity)
    std::map<int, cudaGraphExec_t> graphs;

    // observables scratch (FP64): per-cell rho, prefix sums or summed-area table, outputs
    double* d_obs = nullptr;
    size_t obs_cap = 0;

    // 2D
    Ctx2D* c2 = nullptr;
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
    fprintf(stderr, "lat: %s failed: %s\n", what, cudaGetErrorString(e));
    return LAT_ECUDA;
}
#define CK(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);         \
    } while (0)

void drop_graphs(lat_ctx* c) {
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

int status_code(unsigned st) {
    if (st & ST_NUMERIC) return LAT_ENUMERIC;
    if (st & ST_CFL) return LAT_ECFL;
    if (st & ST_OVERFLOW) return LAT_EOVERFLOW;
    if (st & ST_TIMEOUT) return LAT_ETIMEOUT;
    if (st & ST_NOISE) return LAT_ENOISE;
    return LAT_OK;
}

int tile_of(const lat_ctx* c) { return c->block; }

// Rebuild the (instance, x-tile) work list for the current tile width.
int build_items(lat_ctx* c) {
    const int tile = tile_of(c);
    std::vector<int2> items;
    c->h_inst_begin.assign(c->n_inst + 1, 0);
    for (int i = 0; i < c->n_inst; ++i) {
        c->h_inst_begin[i] = (int)items.size();
        for (int x0 = 0; x0 < c->h_inst[i].nx; x0 += tile) items.push_back(make_int2(i, x0));
    }
    c->h_inst_begin[c->n_inst] = (int)items.size();
    if (c->d_items) cudaFree(c->d_items);
    if (c->d_inst_begin) cudaFree(c->d_inst_begin);
    if (c->d_partials) cudaFree(c->d_partials);
    c->d_items = nullptr;
    c->d_inst_begin = nullptr;
    c->d_partials = nullptr;
    c->nitems = (int)items.size();
    if (cudaMalloc(&c->d_items, sizeof(int2) * items.size()) != cudaSuccess ||
        cudaMalloc(&c->d_inst_begin, sizeof(int) * (c->n_inst + 1)) != cudaSuccess ||
        cudaMalloc(&c->d_partials,
                   sizeof(double) * 6 * std::max(kPcConsumerWarps, tile / 32) * items.size()) !=
            cudaSuccess)
        return LAT_ENOMEM;
    CK(cudaMemcpy(c->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_inst_begin, c->h_inst_begin.data(), sizeof(int) * (c->n_inst + 1),
                  cudaMemcpyHostToDevice));
    drop_graphs(c);
    return LAT_OK;
}

// The 1D globals [instances][M, P, E] of the last reduction to host memory: into the pinned
// context buffer (wait: the caller synchronises and copies them on), or straight into the
// caller's pinned buffer.
int copy_globals_1d(lat_ctx* c, double* gdst, bool wait) {
    if (!gdst) return LAT_OK;
    CK(cudaMemcpyAsync(wait ? c->h_glob : gdst, c->d_glob, sizeof(double) * 3 * c->n_inst,
                       cudaMemcpyDeviceToHost, c->stream));
    return LAT_OK;
}

int persistent_grid(const lat_ctx* c) {
    return std::max(1, std::min(c->nitems, c->bps * c->sm_count));
}

Step1DArgs step_args(const lat_ctx* c, int k, int dry) {
    Step1DArgs a;
    memset(&a, 0, sizeof(a));
    a.f[0] = c->f[0];
    a.f[1] = c->f[1];
    (void)k;
    a.inst = c->d_inst;
    a.items = c->d_items;
    a.item_begin = 0;
    a.item_end = c->nitems;
    a.flow_kind = c->flow_kind;
    a.nmodes = c->nmodes;
    for (int m = 0; m < kMaxModes1D; ++m) a.k[m] = c->k1d[m];
    a.amp = c->d_amp;
    a.amp_w = c->d_amp;
    a.ampf = c->d_ampf;
    a.ampf_w = c->d_ampf;
    a.amp_stride = c->amp_stride;
    a.noise = c->d_noise;
    a.field = c->field;
    a.st = c->d_state;
    a.dry = dry;
    a.frozen = c->frozen ? 1 : 0;
    a.scheme = c->scheme;
    a.mu = c->mu;
    return a;
}

// Enqueue n steps of a 1D context on stream s (used directly and under capture).
int enqueue_steps_1d(lat_ctx* c, int n, cudaStream_t s) {
    for (int k = 0; k < n; ++k) {
        Step1DArgs a = step_args(c, k, 0);
        if (c->mode == 1) {
            for (int i = 0; i < c->n_inst; ++i) {
                a.item_begin = c->h_inst_begin[i];
                a.item_end = c->h_inst_begin[i + 1];
                CK(launch_step1d(c->dtype, c->nv, c->variant, c->block, c->slots,
                                 a.item_end - a.item_begin, a, k, s));
            }
        } else {
            CK(launch_step1d(c->dtype, c->nv, c->variant, c->block, c->slots, persistent_grid(c),
                             a, k, s));
        }
    }
    CK(launch_advance_step(c->d_state, n, s));
    return LAT_OK;
}

int validate_common(double L, int nx, double tau_p, double kappa, double dt, int nv, int d) {
    if (!(L > 0) || nx < 1 || !(dt > 0) || !(kappa >= 0) || !(tau_p > 0) || isnan(tau_p))
        return LAT_EINVAL;
    if (nv < 1 || nv % 2 == 0 || nv > 129) return LAT_EINVAL;
    const double dx = L / nx, dv = dx / dt;
    const int J = (nv - 1) / 2;
    const double g = isinf(tau_p) ? 0.0 : dt / tau_p;
    // Eq. (cfl) at rest (u = 0): largest |a| dt / dv = g J; unsplit 2D adds both components.
    if (g * J * d > 1.0) return LAT_ECFL;
    // Eq. (stabLapl) for the d-dimensional five-point (d = 2) or three-point (d = 1) Laplacian.
    if (2.0 * d * kappa * dt / (dv * dv) > 1.0) return LAT_ECFL;
    return LAT_OK;
}

int alloc_common(lat_ctx* c) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
    if (cudaMalloc(&c->d_state, sizeof(DevState)) != cudaSuccess) return LAT_ENOMEM;
    if (cudaMallocHost(&c->h_state, sizeof(DevState)) != cudaSuccess) return LAT_ENOMEM;
    CK(cudaMemsetAsync(c->d_state, 0, sizeof(DevState), c->stream));
    return LAT_OK;
}

}  // namespace

extern "C" {

const char* lat_strerror(int s) {
    switch (s) {
        case LAT_OK: return "ok";
        case LAT_EINVAL: return "invalid argument";
        case LAT_ECFL: return "stability condition violated (Eq. cfl or Eq. stabLapl)";
        case LAT_ENOMEM: return "device allocation failed";
        case LAT_ECUDA: return "CUDA runtime error";
        case LAT_ENUMERIC: return "non-finite value in f";
        case LAT_ETIMEOUT: return "bounded device wait gave up";
        case LAT_EOVERFLOW: return "reduced-precision value exceeded its line scale";
        case LAT_ENOISE: return "noise table exhausted (flow frozen for the remaining steps)";
        default: return "unknown status";
    }
}

int lat_ensemble_init(lat_ctx** out, int n_inst, const lat_instance* inst, int nv, int dtype,
                      void* f_a, void* f_b, void* stream) {
    if (!out || !inst || n_inst < 1 || !f_a || !f_b || f_a == f_b) return LAT_EINVAL;
    if (dtype != LAT_F32 && dtype != LAT_F64) return LAT_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n_inst; ++i) {
        int v = validate_common(inst[i].L, inst[i].nx, inst[i].tau_p, inst[i].kappa, inst[i].dt,
                                nv, 1);
        if (v != LAT_OK) return v;
    }
    lat_ctx* c = new lat_ctx();
    c->d = 1;
    c->dtype = dtype;
    c->nv = nv;
    c->n_inst = n_inst;
    c->stream = (cudaStream_t)stream;
    c->f[0] = f_a;
    c->f[1] = f_b;
    c->h_inst.resize(n_inst);
    long long off = 0, xoff = 0;
    for (int i = 0; i < n_inst; ++i) {
        Inst1D& q = c->h_inst[i];
        memset(&q, 0, sizeof(q));
        q.off = off;
        q.xoff = xoff;
        q.nx = inst[i].nx;
        q.dx = inst[i].L / inst[i].nx;
        q.dv = q.dx / inst[i].dt;
        q.inv_dv = 1.0 / q.dv;
        q.g = isinf(inst[i].tau_p) ? 0.0 : inst[i].dt / inst[i].tau_p;
        q.r = inst[i].kappa * inst[i].dt / (q.dv * q.dv);
        q.ou_e = 1.0;
        q.ou_s = 0.0;
        q.pow2 = (q.nx & (q.nx - 1)) == 0 ? 1 : 0;
        q.two_over_nx = 2.0 / q.nx;
        q.dt = inst[i].dt;
        off += (long long)nv * inst[i].nx;
        xoff += inst[i].nx;
    }
    c->total_x = xoff;
    int rc = alloc_common(c);
    if (rc == LAT_OK && cudaMalloc(&c->d_inst, sizeof(Inst1D) * n_inst) != cudaSuccess)
        rc = LAT_ENOMEM;
    if (rc == LAT_OK && cudaMalloc(&c->d_glob, sizeof(double) * 3 * n_inst) != cudaSuccess)
        rc = LAT_ENOMEM;
    if (rc == LAT_OK && cudaMallocHost(&c->h_glob, sizeof(double) * 4 * n_inst) != cudaSuccess)
        rc = LAT_ENOMEM;
    if (rc == LAT_OK &&
        cudaMemcpy(c->d_inst, c->h_inst.data(), sizeof(Inst1D) * n_inst, cudaMemcpyHostToDevice) !=
            cudaSuccess)
        rc = LAT_ECUDA;
    if (rc == LAT_OK) {
        // default launch shape: the producer/consumer bulk-copy pipeline where every instance
        // allows it, else plain loads with 256 threads; one x column per thread
        c->ring_ok = step1d_ring_supported(dtype, nv);
        for (int i = 0; i < n_inst; ++i)
            if (inst[i].nx % 4 != 0 || inst[i].nx < step1d_ring_min_nx()) c->ring_ok = false;
        if (c->ring_ok) {
            c->variant = STEP1D_PC;
            c->block = step1d_ring_tile();
            c->slots = 2;
            c->bps = std::max(1, step1d_ring_occupancy(nv, 2, STEP1D_PC));
        } else {
            c->variant = STEP1D_PLAIN;
            c->block = std::min(256, step1d_max_block(dtype, nv, STEP1D_PLAIN));
            c->bps = 4;
        }
        rc = build_items(c);
    }
    if (rc != LAT_OK) {
        lat_free(c);
        return rc;
    }
    *out = c;
    return LAT_OK;
}

int lat_init(lat_ctx** out, const lat_grid* g, void* f_a, void* f_b, void* stream) {
    if (!out || !g) return LAT_EINVAL;
    if (g->d == 1) {
        if (g->ny != 1) return LAT_EINVAL;
        lat_instance in;
        in.nx = g->nx;
        in.L = g->L;
        in.tau_p = g->tau_p;
        in.kappa = g->kappa;
        in.dt = g->dt;
        return lat_ensemble_init(out, 1, &in, g->nv, g->dtype, f_a, f_b, stream);
    }
    if (g->d != 2) return LAT_EINVAL;
    if (!f_a || !f_b || f_a == f_b || g->ny < 1) return LAT_EINVAL;
    int v = validate_common(g->L, g->nx, g->tau_p, g->kappa, g->dt, g->nv, 2);
    if (v != LAT_OK) return v;
    *out = nullptr;
    lat_ctx* c = new lat_ctx();
    c->d = 2;
    c->dtype = g->dtype;
    c->nv = g->nv;
    c->n_inst = 1;
    c->stream = (cudaStream_t)stream;
    c->f[0] = f_a;
    c->f[1] = f_b;
    int rc = alloc_common(c);
    if (rc == LAT_OK) rc = ctx2d_create(&c->c2, g, c->d_state, c->sm_count, c->stream);
    if (rc == LAT_OK) rc = ctx2d_init_state(c->c2, c->f, c->cur, c->stream);
    if (rc != LAT_OK) {
        lat_free(c);
        return rc;
    }
    *out = c;
    return LAT_OK;
}

int lat_set_flow(lat_ctx* c, const lat_flow* fl) {
    if (!c || !fl) return LAT_EINVAL;
    const bool frozen = !(fl->tau_f > 0) || isinf(fl->tau_f);
    if (c->d == 2) {
        drop_graphs(c);
        return ctx2d_set_flow(c->c2, fl, frozen, c->stream);
    }
    if (fl->kind == LAT_FLOW_NONE) {
        c->flow_kind = LAT_FLOW_NONE;
        c->nmodes = 0;
    } else if (fl->kind == LAT_FLOW_FIELD) {
        if (!fl->field) return LAT_EINVAL;
        c->flow_kind = LAT_FLOW_FIELD;
        c->field = fl->field;
        c->nmodes = 0;
    } else if (fl->kind == LAT_FLOW_MODES) {
        if (fl->nmodes < 1 || fl->nmodes > kMaxModes1D || !fl->k || !fl->amp0) return LAT_EINVAL;
        if (!frozen && !(fl->sigma >= 0)) return LAT_EINVAL;
        const int M2 = 2 * fl->nmodes;
        const long long stride = (long long)c->n_inst * M2;
        double* amp = nullptr;
        float* ampf = nullptr;
        if (cudaMalloc(&amp, sizeof(double) * 2 * stride) != cudaSuccess) return LAT_ENOMEM;
        if (cudaMalloc(&ampf, sizeof(float) * 2 * stride) != cudaSuccess) {
            cudaFree(amp);
            return LAT_ENOMEM;
        }
        // both parities start from amp0 so that a frozen flow reads the same values every step
        std::vector<float> a32(fl->amp0, fl->amp0 + stride);
        CK(cudaMemcpy(amp, fl->amp0, sizeof(double) * stride, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(amp + stride, fl->amp0, sizeof(double) * stride, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ampf, a32.data(), sizeof(float) * stride, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ampf + stride, a32.data(), sizeof(float) * stride, cudaMemcpyHostToDevice));
        if (c->d_amp) cudaFree(c->d_amp);
        if (c->d_ampf) cudaFree(c->d_ampf);
        c->d_amp = amp;
        c->d_ampf = ampf;
        c->amp_stride = stride;
        c->flow_kind = LAT_FLOW_MODES;
        c->nmodes = fl->nmodes;
        for (int m = 0; m < kMaxModes1D; ++m) c->k1d[m] = m < fl->nmodes ? fl->k[m] : 0;
        c->noise_row_len = stride;
        for (int i = 0; i < c->n_inst; ++i) {
            Inst1D& q = c->h_inst[i];
            const double dt = q.dt;
            if (frozen) {
                q.ou_e = 1.0;
                q.ou_s = 0.0;
            } else {
                q.ou_e = exp(-dt / fl->tau_f);
                q.ou_s = fl->sigma * sqrt(1.0 - q.ou_e * q.ou_e);
            }
        }
        CK(cudaMemcpy(c->d_inst, c->h_inst.data(), sizeof(Inst1D) * c->n_inst,
                      cudaMemcpyHostToDevice));
    } else {
        return LAT_EINVAL;
    }
    c->frozen = frozen || fl->kind != LAT_FLOW_MODES;
    k_set_noise_window<<<1, 1, 0, c->stream>>>(c->d_state, c->h_step, 0);
    CK(cudaGetLastError());
    drop_graphs(c);
    return LAT_OK;
}

int lat_set_noise(lat_ctx* c, const double* noise, long long rows) {
    if (!c || rows < 0 || (rows > 0 && !noise)) return LAT_EINVAL;
    if (c->d == 2) {
        int rc = ctx2d_set_noise(c->c2, noise, rows, c->h_step, c->stream);
        if (rc == LAT_OK) drop_graphs(c);
        return rc;
    }
    if (c->flow_kind != LAT_FLOW_MODES) return LAT_EINVAL;
    const long long need = rows * c->noise_row_len;
    if (need > c->noise_cap) {
        CK(cudaStreamSynchronize(c->stream));
        double* p = nullptr;
        if (cudaMalloc(&p, sizeof(double) * need) != cudaSuccess) return LAT_ENOMEM;
        if (c->d_noise) cudaFree(c->d_noise);
        c->d_noise = p;
        c->noise_cap = need;
        drop_graphs(c);
    }
    if (need > 0)
        CK(cudaMemcpyAsync(c->d_noise, noise, sizeof(double) * need, cudaMemcpyHostToDevice,
                           c->stream));
    k_set_noise_window<<<1, 1, 0, c->stream>>>(c->d_state, c->h_step, rows);
    CK(cudaGetLastError());
    return LAT_OK;
}

}  // extern "C"

namespace {

// Capture (once) the graph of n steps of a 1D context.
int graph_for(lat_ctx* c, int n, cudaGraphExec_t* out) {
    auto it = c->graphs.find(n);
    if (it == c->graphs.end()) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_steps_1d(c, n, c->cap);
        cudaError_t e = cudaStreamEndCapture(c->cap, &g);
        if (rc != LAT_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (c->graphs.size() >= 8) drop_graphs(c);
        it = c->graphs.emplace(n, ge).first;
    }
    *out = it->second;
    return LAT_OK;
}

}  // namespace

extern "C" {

int lat_prepare(lat_ctx* c, int n) {
    if (!c || n < 1) return LAT_EINVAL;
    if (c->d == 2) return ctx2d_prepare(c->c2, c->f, n);
    if (c->mode != 0) return LAT_OK;
    cudaGraphExec_t ge;
    return graph_for(c, n, &ge);
}

int lat_step(lat_ctx* c, int n) {
    if (!c || n < 0) return LAT_EINVAL;
    if (n == 0) return LAT_OK;
    if (c->d == 2) {
        int rc = ctx2d_step(c->c2, c->f, n, c->stream);
        if (rc != LAT_OK) return rc;
    } else if (c->mode != 0) {
        int rc = enqueue_steps_1d(c, n, c->stream);
        if (rc != LAT_OK) return rc;
    } else {
        cudaGraphExec_t ge;
        int rc = graph_for(c, n, &ge);
        if (rc != LAT_OK) return rc;
        CK(cudaGraphLaunch(ge, c->stream));
    }
    c->h_step += n;
    c->cur = (int)(c->h_step & 1);
    return LAT_OK;
}

int lat_status(lat_ctx* c) {
    if (!c) return LAT_EINVAL;
    CK(cudaMemcpyAsync(c->h_state, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost,
                       c->stream));
    k_clear_status<<<1, 1, 0, c->stream>>>(c->d_state);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->stream));
    return status_code(c->h_state->status);
}

}  // extern "C"

namespace {

// The moments of the current state, enqueued: per-cell arrays on the device, the globals to host
// memory (gdst, or none): through the pinned context buffer and a synchronisation (wait), or by
// an asynchronous copy into the caller's pinned buffer.
int enqueue_moments(lat_ctx* c, double* rho, double* mean_v, double* mean_v2, double* gdst,
                    bool wait) {
    if (c->d == 2)
        return ctx2d_moments(c->c2, c->f[c->cur], c->cur, rho, mean_v, mean_v2, gdst, wait,
                             c->stream);
    Mom1DArgs a;
    a.f = c->f[c->cur];
    a.inst = c->d_inst;
    a.items = c->d_items;
    a.nitems = c->nitems;
    a.nv = c->nv;
    a.rho = rho;
    a.mean_v = mean_v;
    a.mean_v2 = mean_v2;
    a.partials = c->d_partials;
    a.st = c->d_state;
    const int grid = std::max(1, std::min(c->nitems, 8 * c->sm_count));
    CK(launch_moments1d(c->dtype, tile_of(c), 1, grid, a, c->stream));
    CK(launch_finalize1d(c->d_partials, c->d_inst_begin, c->d_inst, c->n_inst, c->d_glob,
                         tile_of(c) / 32, c->stream));
    return copy_globals_1d(c, gdst, wait);
}

// n steps and the moments of the state the last one writes (fused into it where the launch
// allows it), enqueued; gdst and wait as for enqueue_moments.
int enqueue_step_moments(lat_ctx* c, int n, double* rho, double* mean_v, double* mean_v2,
                         double* gdst, bool wait) {
    if (c->d == 2 && ctx2d_moments_fusable(c->c2)) {
        if (n > 1) {
            int rc = lat_step(c, n - 1);
            if (rc != LAT_OK) return rc;
        }
        int rc = ctx2d_step_moments(c->c2, c->f, rho, mean_v, mean_v2, gdst, wait, c->stream);
        if (rc != LAT_OK) return rc;
        c->h_step += 1;
        c->cur = (int)(c->h_step & 1);
        return LAT_OK;
    }
    const bool fused = c->d == 1 && c->variant == STEP1D_PC && c->mode != 1 &&
                       step1d_moments_supported(c->dtype, c->nv);
    if (!fused) {
        int rc = lat_step(c, n);
        if (rc != LAT_OK) return rc;
        return enqueue_moments(c, rho, mean_v, mean_v2, gdst, wait);
    }
    if (n > 1) {
        int rc = lat_step(c, n - 1);
        if (rc != LAT_OK) return rc;
    }
    Step1DArgs a = step_args(c, 0, 0);
    a.m_rho = rho;
    a.m_mv = mean_v;
    a.m_mv2 = mean_v2;
    a.m_partials = c->d_partials;
    CK(launch_step1d_moments(c->nv, persistent_grid(c), a, c->stream));
    CK(launch_advance_step(c->d_state, 1, c->stream));
    CK(launch_finalize1d(c->d_partials, c->d_inst_begin, c->d_inst, c->n_inst, c->d_glob,
                         kPcConsumerWarps, c->stream));
    c->h_step += 1;
    c->cur = (int)(c->h_step & 1);
    return copy_globals_1d(c, gdst, wait);
}

}  // namespace

extern "C" {

int lat_moments(lat_ctx* c, double* rho, double* mean_v, double* mean_v2, double* globals) {
    if (!c) return LAT_EINVAL;
    int rc = enqueue_moments(c, rho, mean_v, mean_v2, globals, true);
    if (rc != LAT_OK) return rc;
    rc = lat_status(c);  // synchronises
    if (globals && c->d == 1) memcpy(globals, c->h_glob, sizeof(double) * 3 * c->n_inst);
    return rc;
}

int lat_step_moments(lat_ctx* c, int n, double* rho, double* mean_v, double* mean_v2,
                     double* globals) {
    if (!c || n < 1) return LAT_EINVAL;
    int rc = enqueue_step_moments(c, n, rho, mean_v, mean_v2, globals, true);
    if (rc != LAT_OK) return rc;
    rc = lat_status(c);  // synchronises
    if (globals && c->d == 1) memcpy(globals, c->h_glob, sizeof(double) * 3 * c->n_inst);
    return rc;
}

int lat_step_moments_async(lat_ctx* c, int n, double* globals) {
    if (!c || n < 1 || !globals) return LAT_EINVAL;
    return enqueue_step_moments(c, n, nullptr, nullptr, nullptr, globals, false);
}

int lat_current(const lat_ctx* c) { return c ? c->cur : -1; }

int lat_restrict(const float* fine, int nv_fine, int nx, int ny, float* coarse, void* stream) {
    if (!fine || !coarse || nx < 1 || ny < 1 || nv_fine < 5 || (nv_fine - 1) % 4 != 0)
        return LAT_EINVAL;
    if (launch_restrict(fine, nv_fine, nx, ny, coarse, (cudaStream_t)stream) != cudaSuccess)
        return LAT_ECUDA;
    return LAT_OK;
}

int lat_learn(lat_ctx* c, const float* params, int mode) {
    if (!c || c->d != 2) return LAT_EINVAL;
    int rc = ctx2d_learn_set(c->c2, params, mode, c->stream);
    if (rc == LAT_OK) drop_graphs(c);
    return rc;
}

int lat_learn_corrections(lat_ctx* c, float* G, int reuse_inputs) {
    if (!c || c->d != 2) return LAT_EINVAL;
    return ctx2d_learn_corr(c->c2, c->f, c->cur, G, reuse_inputs ? 1 : 0, c->stream);
}

int lat_learn_grad(lat_ctx* c, int nsteps, const float* target, double rho_weight, double* loss,
                   float* grad) {
    if (!c || c->d != 2 || !target || !loss || !grad || !(rho_weight >= 0)) return LAT_EINVAL;
    int rc = ctx2d_learn_grad(c->c2, c->f, c->cur, nsteps, target, rho_weight, loss, grad,
                              c->stream);
    if (rc != LAT_OK) return rc;
    return lat_status(c);
}

int lat_encode(lat_ctx* c, const float* src) {
    if (!c || !src || c->d != 2 || (c->dtype != LAT_F16 && c->dtype != LAT_BF16))
        return LAT_EINVAL;
    int rc = ctx2d_encode(c->c2, src, c->f, c->cur, c->stream);
    if (rc != LAT_OK) return rc;
    return lat_status(c);
}

int lat_decode(lat_ctx* c, float* dst, float* scales) {
    if (!c || (!dst && !scales) || c->d != 2 || (c->dtype != LAT_F16 && c->dtype != LAT_BF16))
        return LAT_EINVAL;
    int rc = ctx2d_decode(c->c2, c->f, c->cur, dst, scales, c->stream);
    if (rc != LAT_OK) return rc;
    return lat_status(c);
}

long long lat_steps_done(const lat_ctx* c) { return c ? c->h_step : -1; }

namespace {

// Grows the observables scratch to n doubles (device).
int obs_scratch(lat_ctx* c, size_t n) {
    if (c->obs_cap >= n) return LAT_OK;
    if (c->d_obs) cudaFree(c->d_obs);
    c->d_obs = nullptr;
    c->obs_cap = 0;
    if (cudaMalloc(&c->d_obs, sizeof(double) * n) != cudaSuccess) return LAT_ENOMEM;
    c->obs_cap = n;
    return LAT_OK;
}

}  // namespace

int lat_coarse_moment(lat_ctx* c, int nw, const int* widths, double* out) {
    if (!c || nw < 1 || nw > 256 || !widths || !out) return LAT_EINVAL;
    int nx = 0, ny = 1, nv = 0;
    double dx = 0, dv = 0;
    long long ncell;
    int nmin;
    if (c->d == 2) {
        ctx2d_geometry(c->c2, &nx, &ny, &nv, &dx, &dv);
        ncell = (long long)nx * ny;
        nmin = std::min(nx, ny);
    } else {
        ncell = c->total_x;
        nmin = c->h_inst.empty() ? 0 : c->h_inst[0].nx;
        for (const Inst1D& in : c->h_inst) nmin = std::min(nmin, in.nx);
    }
    for (int q = 0; q < nw; ++q)
        if (widths[q] < 1 || widths[q] > nmin) return LAT_EINVAL;
    const int nout = (c->d == 2 ? 1 : c->n_inst) * nw;
    const size_t table = c->d == 2 ? 2 * (size_t)(ny + 1) * (nx + 1)
                                   : 2 * (size_t)(c->total_x + c->n_inst);
    const size_t ints = (nw + 1) / 2;  // widths, two per double
    int rc = obs_scratch(c, (size_t)ncell + table + nout + ints);
    if (rc != LAT_OK) return rc;
    double* rho = c->d_obs;
    double* tab = rho + ncell;
    double* d_out = tab + table;
    int* d_w = reinterpret_cast<int*>(d_out + nout);
    // per-cell rho (also raises the pending status)
    rc = lat_moments(c, rho, nullptr, nullptr, nullptr);
    if (rc != LAT_OK) return rc;
    CK(cudaMemcpyAsync(d_w, widths, sizeof(int) * nw, cudaMemcpyHostToDevice, c->stream));
    if (c->d == 2)
        CK(launch_coarse2d(rho, nx, ny, dx, d_w, nw, tab, d_out, c->sm_count, c->stream));
    else
        CK(launch_coarse1d(rho, c->d_inst, c->n_inst, c->total_x, d_w, nw, tab, d_out,
                           c->sm_count, c->stream));
    CK(cudaMemcpyAsync(out, d_out, sizeof(double) * nout, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LAT_OK;
}

int lat_s1(lat_ctx* c, int ns, const int* seps, double* num, double* den) {
    if (!c || c->d != 1 || ns < 1 || ns > 256 || !seps || !num || !den) return LAT_EINVAL;
    if (c->dtype != LAT_F32 && c->dtype != LAT_F64) return LAT_EINVAL;
    int nmin = c->h_inst.empty() ? 0 : c->h_inst[0].nx;
    for (const Inst1D& in : c->h_inst) nmin = std::min(nmin, in.nx);
    for (int q = 0; q < ns; ++q)
        if (seps[q] < 0 || seps[q] >= nmin) return LAT_EINVAL;
    const int nout = c->n_inst * ns;
    int rc = obs_scratch(c, (size_t)c->total_x + 2 * (size_t)nout + (ns + 1) / 2);
    if (rc != LAT_OK) return rc;
    double* rho = c->d_obs;
    double* d_num = rho + c->total_x;
    double* d_den = d_num + nout;
    int* d_s = reinterpret_cast<int*>(d_den + nout);
    rc = lat_moments(c, rho, nullptr, nullptr, nullptr);
    if (rc != LAT_OK) return rc;
    CK(cudaMemcpyAsync(d_s, seps, sizeof(int) * ns, cudaMemcpyHostToDevice, c->stream));
    CK(launch_s1_1d(c->dtype, c->f[c->cur], c->d_inst, c->n_inst, c->nv, rho, d_s, ns, d_num,
                    d_den, c->sm_count, c->stream));
    CK(cudaMemcpyAsync(num, d_num, sizeof(double) * nout, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(den, d_den, sizeof(double) * nout, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return LAT_OK;
}

int lat_set_scheme(lat_ctx* c, int scheme, double mu) {
    if (!c) return LAT_EINVAL;
    if (scheme != LAT_SCHEME_UPWIND && scheme != LAT_SCHEME_KOREN) return LAT_EINVAL;
    if (c->d == 2) {
        if (scheme == LAT_SCHEME_KOREN && !(mu > 0.0 && mu <= 2.0)) return LAT_EINVAL;
        const int rc = ctx2d_set_scheme(c->c2, scheme, mu);
        if (rc == LAT_OK) drop_graphs(c);
        return rc;
    }
    if (scheme == LAT_SCHEME_KOREN) {
        if (c->dtype != LAT_F32 && c->dtype != LAT_F64) return LAT_EINVAL;
        if (!step1d_limiter_supported(c->nv)) return LAT_EINVAL;
        if (!(mu > 0.0 && mu <= 2.0)) return LAT_EINVAL;
        // each Heun stage is positive for nu (1 + mu) <= 1; at rest nu = (dt/tau_p) J
        const int J = (c->nv - 1) / 2;
        for (const Inst1D& in : c->h_inst)
            if (in.g * J * (1.0 + mu) > 1.0) return LAT_ECFL;
    }
    c->scheme = scheme;
    if (scheme == LAT_SCHEME_KOREN) c->mu = mu;
    drop_graphs(c);
    return LAT_OK;
}

int lat_set_launch(lat_ctx* c, int kernel, int block, int blocks_per_sm, int mode) {
    if (!c) return LAT_EINVAL;
    if (c->d == 2) {
        int rc = ctx2d_set_launch(c->c2, kernel, block, blocks_per_sm, mode);
        if (rc == LAT_OK) drop_graphs(c);
        return rc;
    }
    int variant = c->variant, slots = c->slots, nb = c->block;
    if (kernel == 1) {
        variant = STEP1D_PLAIN;
        if (c->variant != STEP1D_PLAIN && !block) nb = std::min(256, step1d_max_block(c->dtype, c->nv, STEP1D_PLAIN));
    } else if (kernel >= 2 && kernel <= 7) {
        if (!c->ring_ok) return LAT_EINVAL;
        variant = kernel <= 4 ? STEP1D_RING : STEP1D_PC;
        slots = kernel <= 4 ? kernel : kernel - 3;
        nb = step1d_ring_tile();
    } else if (kernel != 0) {
        return LAT_EINVAL;
    }
    const bool piped = variant != STEP1D_PLAIN;
    if (block && !piped) nb = block;
    if (block && piped && block != step1d_ring_tile()) return LAT_EINVAL;
    int nbps = blocks_per_sm ? blocks_per_sm : c->bps;
    // a kept block count is clamped to what the newly chosen pipeline shape can hold
    if (!blocks_per_sm && piped)
        nbps = std::max(1, std::min(nbps, step1d_ring_occupancy(c->nv, slots, variant)));
    const int nmode = mode >= 0 ? mode : c->mode;
    if (nb < 32 || nb > 1024 || nb % 32 != 0 || nbps < 1 || nbps > 64 || nmode > 2)
        return LAT_EINVAL;
    if (nb > step1d_max_block(c->dtype, c->nv, variant)) return LAT_EINVAL;
    if (piped && nbps > step1d_ring_occupancy(c->nv, slots, variant)) return LAT_EINVAL;
    const bool retile = nb != tile_of(c);
    c->variant = variant;
    c->slots = slots;
    c->block = nb;
    c->bps = nbps;
    c->mode = nmode;
    drop_graphs(c);
    return retile ? build_items(c) : LAT_OK;
}

int lat_autotune(lat_ctx* c, int reps, double* best) {
    if (!c || reps < 1) return LAT_EINVAL;
    if (c->d == 2) return ctx2d_autotune(c->c2, c->f, reps, best, c->stream);
    struct Cand {
        int kernel, block, bps;
    };
    std::vector<Cand> cands;
    for (int b : {128, 256, 512})
        for (int p : {1, 2, 3, 4, 6, 8})
            if (b * p <= 2048 && b <= step1d_max_block(c->dtype, c->nv, STEP1D_PLAIN))
                cands.push_back({1, b, p});
    if (c->ring_ok)
        for (int sl : {2, 3, 4}) {
            const int occ = step1d_ring_occupancy(c->nv, sl, STEP1D_RING);
            for (int p = 1; p <= occ; ++p) cands.push_back({sl, 0, p});
            const int occp = step1d_ring_occupancy(c->nv, sl, STEP1D_PC);
            for (int p = 1; p <= occp; ++p) cands.push_back({sl + 3, 0, p});
        }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int mode_save = c->mode;
    double best_us = 1e300;
    Cand bc{0, 0, 0};
    for (const Cand& q : cands) {
        if (lat_set_launch(c, q.kernel, q.block, q.bps, 0) != LAT_OK) continue;
        Step1DArgs a = step_args(c, 0, 1);
        const int grid = persistent_grid(c);
        CK(launch_step1d(c->dtype, c->nv, c->variant, c->block, c->slots, grid, a, 0, c->stream));
        CK(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < reps; ++r)
            CK(launch_step1d(c->dtype, c->nv, c->variant, c->block, c->slots, grid, a, 0,
                             c->stream));
        CK(cudaEventRecord(e1, c->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double us = 1000.0 * ms / reps;
        if (us < best_us) {
            best_us = us;
            bc = q;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the dry runs may have flagged CFL on the current state; the next real step flags it again
    k_clear_status<<<1, 1, 0, c->stream>>>(c->d_state);
    int rc = lat_set_launch(c, bc.kernel, bc.block, bc.bps, mode_save);
    if (best) {
        best[0] = bc.kernel;
        best[1] = c->block;
        best[2] = bc.bps;
        best[3] = best_us;
    }
    return rc;
}

}  // extern "C"

// ---- host density I/O and checkpoints ----------------------------------------------------------
namespace {

constexpr long long kConvChunk = 1ll << 26;  // values per FP32 <-> FP64 conversion pass

size_t elem_bytes(int dtype) {
    return dtype == LAT_F64 ? 8 : (dtype == LAT_F32 ? 4 : 2);
}

// Values of one density buffer (all instances).
long long state_values(const lat_ctx* c) {
    if (c->d == 2) {
        int nx, ny, nv;
        double dx, dv;
        ctx2d_geometry(c->c2, &nx, &ny, &nv, &dx, &dv);
        return (long long)nv * nv * nx * ny;
    }
    return (long long)c->nv * c->total_x;
}

// RAII device scratch of the I/O calls.
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t bytes) { return cudaMalloc(&p, bytes) == cudaSuccess; }
};

// FNV-1a over the bytes of the values that fix a context's lattice, so that an image is only
// restored into a context of the same geometry and parameters.
struct Fnv {
    unsigned long long h = 1469598103934665603ull;
    template <class T>
    void add(const T& v) {
        const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
        for (size_t i = 0; i < sizeof(T); ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

struct ImgHeader {
    char magic[8];
    int version, d, dtype, nv, nx, ny, n_inst, flow_kind, nmodes, reserved;
    long long values;        // density values (all instances)
    long long step;
    long long noise_start;   // the first stored noise row applies at step + noise_start
    long long noise_rows;
    long long noise_row_len; // doubles per row
    long long f_bytes, sc_bytes, flow_bytes, noise_bytes;
    unsigned long long lattice_hash;
};
const char kImgMagic[8] = {'L', 'A', 'T', 'S', 'T', 'A', 'T', 'E'};
constexpr int kImgVersion = 1;

// What a context's image holds, from its host fields and its device state word (synchronises).
int image_layout(lat_ctx* c, ImgHeader* h, DevState* ds) {
    memset(h, 0, sizeof(*h));
    memcpy(h->magic, kImgMagic, 8);
    h->version = kImgVersion;
    h->d = c->d;
    h->dtype = c->dtype;
    h->nv = c->nv;
    h->n_inst = c->n_inst;
    h->values = state_values(c);
    Fnv fh;
    long long row_len = 0;
    bool moving = false;  // a modal flow that consumes noise rows
    if (c->d == 2) {
        int nx, ny, nv;
        double dx, dv;
        ctx2d_geometry(c->c2, &nx, &ny, &nv, &dx, &dv);
        Ctx2DDyn dy;
        ctx2d_dyn(c->c2, &dy);
        h->nx = nx;
        h->ny = ny;
        h->flow_kind = dy.flow_kind;
        h->nmodes = dy.nmodes;
        fh.add(nx), fh.add(ny), fh.add(nv), fh.add(dx), fh.add(dv), fh.add(dy.g), fh.add(dy.r);
        h->sc_bytes = (long long)dy.nlines * (sizeof(float) + sizeof(unsigned));
        h->flow_bytes = dy.flow_kind == LAT_FLOW_MODES ? (long long)sizeof(double) * dy.nmodes : 0;
        row_len = dy.nmodes;
        moving = dy.flow_kind == LAT_FLOW_MODES && !dy.frozen;
    } else {
        h->nx = (int)std::min<long long>(c->total_x, 0x7fffffff);
        h->ny = 1;
        h->flow_kind = c->flow_kind;
        h->nmodes = c->flow_kind == LAT_FLOW_MODES ? c->nmodes : 0;
        for (const Inst1D& q : c->h_inst) {
            fh.add(q.nx), fh.add(q.dx), fh.add(q.dv), fh.add(q.g), fh.add(q.r);
            fh.add(q.ou_e), fh.add(q.ou_s);
        }
        h->flow_bytes = c->flow_kind == LAT_FLOW_MODES
                            ? (long long)(sizeof(double) + sizeof(float)) * c->amp_stride
                            : 0;
        row_len = c->flow_kind == LAT_FLOW_MODES ? c->noise_row_len : 0;
        moving = c->flow_kind == LAT_FLOW_MODES && !c->frozen;
    }
    h->lattice_hash = fh.h;
    h->f_bytes = h->values * (long long)elem_bytes(c->dtype);
    CK(cudaMemcpyAsync(ds, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    h->step = ds->step;
    h->noise_row_len = row_len;
    if (row_len > 0 && moving && ds->noise_rows > 0) {
        const long long skip = std::max(0ll, ds->step - ds->noise_base);
        h->noise_rows = std::max(0ll, ds->noise_rows - skip);
        h->noise_start = std::max(0ll, ds->noise_base - ds->step);
    }
    h->noise_bytes = (long long)sizeof(double) * h->noise_rows * row_len;
    return LAT_OK;
}

long long image_bytes(const ImgHeader& h) {
    return (long long)sizeof(ImgHeader) + h.f_bytes + h.sc_bytes + h.flow_bytes + h.noise_bytes;
}

}  // namespace

extern "C" {

int lat_get_density(lat_ctx* c, double* f_host) {
    if (!c || !f_host) return LAT_EINVAL;
    const long long n = state_values(c);
    void* cur = c->f[c->cur];
    if (c->dtype == LAT_F64) {
        CK(cudaMemcpyAsync(f_host, cur, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    } else if (c->dtype == LAT_F32) {
        const long long chunk = std::min(n, kConvChunk);
        DevBuf t;
        if (!t.alloc(sizeof(double) * chunk)) return LAT_ENOMEM;
        for (long long i = 0; i < n; i += chunk) {
            const long long m = std::min(chunk, n - i);
            CK(launch_f32_to_f64(static_cast<const float*>(cur) + i, (double*)t.p, m, c->stream));
            CK(cudaMemcpyAsync(f_host + i, t.p, sizeof(double) * m, cudaMemcpyDeviceToHost,
                               c->stream));
            CK(cudaStreamSynchronize(c->stream));  // t is reused by the next pass
        }
    } else {
        DevBuf t32, t64;
        if (!t32.alloc(sizeof(float) * n) || !t64.alloc(sizeof(double) * n)) return LAT_ENOMEM;
        int rc = ctx2d_decode(c->c2, c->f, c->cur, (float*)t32.p, nullptr, c->stream);
        if (rc != LAT_OK) return rc;
        CK(launch_f32_to_f64((const float*)t32.p, (double*)t64.p, n, c->stream));
        CK(cudaMemcpyAsync(f_host, t64.p, sizeof(double) * n, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return lat_status(c);  // synchronises
}

int lat_set_density(lat_ctx* c, const double* f_host) {
    if (!c || !f_host) return LAT_EINVAL;
    const long long n = state_values(c);
    void* cur = c->f[c->cur];
    if (c->dtype == LAT_F64) {
        CK(cudaMemcpyAsync(cur, f_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    } else if (c->dtype == LAT_F32) {
        const long long chunk = std::min(n, kConvChunk);
        DevBuf t;
        if (!t.alloc(sizeof(double) * chunk)) return LAT_ENOMEM;
        for (long long i = 0; i < n; i += chunk) {
            const long long m = std::min(chunk, n - i);
            CK(cudaMemcpyAsync(t.p, f_host + i, sizeof(double) * m, cudaMemcpyHostToDevice,
                               c->stream));
            CK(launch_f64_to_f32((const double*)t.p, static_cast<float*>(cur) + i, m, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    } else {
        DevBuf t32, t64;
        if (!t32.alloc(sizeof(float) * n) || !t64.alloc(sizeof(double) * n)) return LAT_ENOMEM;
        CK(cudaMemcpyAsync(t64.p, f_host, sizeof(double) * n, cudaMemcpyHostToDevice,
                           c->stream));
        CK(launch_f64_to_f32((const double*)t64.p, (float*)t32.p, n, c->stream));
        int rc = ctx2d_encode(c->c2, (const float*)t32.p, c->f, c->cur, c->stream);
        if (rc != LAT_OK) return rc;
        CK(cudaStreamSynchronize(c->stream));
    }
    return lat_status(c);
}

int lat_state_bytes(lat_ctx* c, long long* bytes) {
    if (!c || !bytes) return LAT_EINVAL;
    ImgHeader h;
    int rc = image_layout(c, &h, c->h_state);
    if (rc != LAT_OK) return rc;
    *bytes = image_bytes(h);
    return LAT_OK;
}

int lat_get_state(lat_ctx* c, void* image, long long bytes) {
    if (!c || !image) return LAT_EINVAL;
    ImgHeader h;
    DevState ds;
    int rc = image_layout(c, &h, c->h_state);
    if (rc != LAT_OK) return rc;
    ds = *c->h_state;
    if (bytes < image_bytes(h)) return LAT_EINVAL;
    const int par = (int)(h.step & 1);
    unsigned char* p = static_cast<unsigned char*>(image);
    memcpy(p, &h, sizeof(h));
    p += sizeof(h);
    CK(cudaMemcpyAsync(p, c->f[par], h.f_bytes, cudaMemcpyDeviceToHost, c->stream));
    p += h.f_bytes;
    if (h.sc_bytes) {
        Ctx2DDyn dy;
        ctx2d_dyn(c->c2, &dy);
        CK(cudaMemcpyAsync(p, dy.sc + (size_t)par * dy.nlines, sizeof(float) * dy.nlines,
                           cudaMemcpyDeviceToHost, c->stream));
        p += sizeof(float) * dy.nlines;
        CK(cudaMemcpyAsync(p, dy.mx + (size_t)par * dy.nlines, sizeof(unsigned) * dy.nlines,
                           cudaMemcpyDeviceToHost, c->stream));
        p += sizeof(unsigned) * dy.nlines;
    }
    if (h.flow_bytes) {
        if (c->d == 2) {
            Ctx2DDyn dy;
            ctx2d_dyn(c->c2, &dy);
            CK(cudaMemcpyAsync(p, dy.phase + (size_t)par * dy.nmodes, h.flow_bytes,
                               cudaMemcpyDeviceToHost, c->stream));
        } else {
            const size_t na = (size_t)c->amp_stride;
            CK(cudaMemcpyAsync(p, c->d_amp + (size_t)par * na, sizeof(double) * na,
                               cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(p + sizeof(double) * na, c->d_ampf + (size_t)par * na,
                               sizeof(float) * na, cudaMemcpyDeviceToHost, c->stream));
        }
        p += h.flow_bytes;
    }
    if (h.noise_bytes) {
        const double* table = c->d == 2 ? [&] {
            Ctx2DDyn dy;
            ctx2d_dyn(c->c2, &dy);
            return (const double*)dy.noise;
        }() : c->d_noise;
        const long long skip = std::max(0ll, ds.step - ds.noise_base);
        CK(cudaMemcpyAsync(p, table + skip * h.noise_row_len, h.noise_bytes,
                           cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return LAT_OK;
}

int lat_set_state(lat_ctx* c, const void* image, long long bytes) {
    if (!c || !image || bytes < (long long)sizeof(ImgHeader)) return LAT_EINVAL;
    ImgHeader img;
    memcpy(&img, image, sizeof(img));
    ImgHeader mine;
    int rc = image_layout(c, &mine, c->h_state);
    if (rc != LAT_OK) return rc;
    if (memcmp(img.magic, kImgMagic, 8) != 0 || img.version != kImgVersion) return LAT_EINVAL;
    if (img.d != mine.d || img.dtype != mine.dtype || img.nv != mine.nv || img.nx != mine.nx ||
        img.ny != mine.ny || img.n_inst != mine.n_inst || img.values != mine.values ||
        img.flow_kind != mine.flow_kind || img.nmodes != mine.nmodes ||
        img.lattice_hash != mine.lattice_hash || img.f_bytes != mine.f_bytes ||
        img.sc_bytes != mine.sc_bytes || img.flow_bytes != mine.flow_bytes ||
        img.noise_row_len != mine.noise_row_len || img.step < 0 || img.noise_rows < 0 ||
        img.noise_start < 0 || img.noise_bytes != (long long)sizeof(double) * img.noise_rows *
                                                      img.noise_row_len)
        return LAT_EINVAL;
    if (bytes < image_bytes(img)) return LAT_EINVAL;
    const long long need = img.noise_rows * img.noise_row_len;
    double* table = nullptr;
    if (c->d == 2) {
        rc = ctx2d_noise_reserve(c->c2, need, c->stream);
        if (rc != LAT_OK) return rc;
        Ctx2DDyn dy;
        ctx2d_dyn(c->c2, &dy);
        table = dy.noise;
    } else if (need > c->noise_cap) {
        CK(cudaStreamSynchronize(c->stream));
        double* q = nullptr;
        if (cudaMalloc(&q, sizeof(double) * need) != cudaSuccess) return LAT_ENOMEM;
        if (c->d_noise) cudaFree(c->d_noise);
        c->d_noise = q;
        c->noise_cap = need;
        table = q;
    } else {
        table = c->d_noise;
    }
    const int par = (int)(img.step & 1);
    const unsigned char* p = static_cast<const unsigned char*>(image) + sizeof(ImgHeader);
    CK(cudaMemcpyAsync(c->f[par], p, img.f_bytes, cudaMemcpyHostToDevice, c->stream));
    p += img.f_bytes;
    if (img.sc_bytes) {
        Ctx2DDyn dy;
        ctx2d_dyn(c->c2, &dy);
        CK(cudaMemcpyAsync(dy.sc + (size_t)par * dy.nlines, p, sizeof(float) * dy.nlines,
                           cudaMemcpyHostToDevice, c->stream));
        p += sizeof(float) * dy.nlines;
        CK(cudaMemcpyAsync(dy.mx + (size_t)par * dy.nlines, p, sizeof(unsigned) * dy.nlines,
                           cudaMemcpyHostToDevice, c->stream));
        p += sizeof(unsigned) * dy.nlines;
    }
    if (img.flow_bytes) {
        // both parities: a frozen flow reads either, a moving one overwrites the other
        for (int q = 0; q < 2; ++q) {
            if (c->d == 2) {
                Ctx2DDyn dy;
                ctx2d_dyn(c->c2, &dy);
                CK(cudaMemcpyAsync(dy.phase + (size_t)q * dy.nmodes, p, img.flow_bytes,
                                   cudaMemcpyHostToDevice, c->stream));
            } else {
                const size_t na = (size_t)c->amp_stride;
                CK(cudaMemcpyAsync(c->d_amp + (size_t)q * na, p, sizeof(double) * na,
                                   cudaMemcpyHostToDevice, c->stream));
                CK(cudaMemcpyAsync(c->d_ampf + (size_t)q * na, p + sizeof(double) * na,
                                   sizeof(float) * na, cudaMemcpyHostToDevice, c->stream));
            }
        }
        p += img.flow_bytes;
    }
    if (img.noise_bytes)
        CK(cudaMemcpyAsync(table, p, img.noise_bytes, cudaMemcpyHostToDevice, c->stream));
    CK(launch_set_devstate(c->d_state, img.step, img.step + img.noise_start, img.noise_rows,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->h_step = img.step;
    c->cur = par;
    drop_graphs(c);
    if (c->d == 2) ctx2d_drop_graphs(c->c2);
    return LAT_OK;
}

int lat_debug_stall(lat_ctx* c, int on) {
    if (!c) return LAT_EINVAL;
    CK(launch_set_stall(c->d_state, on ? 1u : 0u, c->stream));
    return LAT_OK;
}

void lat_free(lat_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graphs(c);
    if (c->c2) ctx2d_destroy(c->c2);
    cudaFree(c->d_inst);
    cudaFree(c->d_items);
    cudaFree(c->d_inst_begin);
    cudaFree(c->d_partials);
    cudaFree(c->d_glob);
    cudaFree(c->d_amp);
    cudaFree(c->d_ampf);
    cudaFree(c->d_noise);
    cudaFree(c->d_state);
    cudaFree(c->d_obs);
    if (c->h_glob) cudaFreeHost(c->h_glob);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

}  // extern "C"
