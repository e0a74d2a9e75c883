// lbm_runtime.cu -- the C-ABI (include/lbmadj.h): context, device buffers,
// convergence loops and result read-back.
//
// Each solve phase runs in blocks of K steps.  A block is captured once as a
// CUDA graph (K-1 plain fused steps, one reducing step, the deterministic
// finalize kernel and the copy of the sums to pinned host memory) and then
// replayed, so a block costs one graph launch and one host synchronisation.
// The residual |I(t) - I(t-K)| / |I(t)| is evaluated on the host from the FP64
// sums (Sec. 3.1, Fig. 8 text).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbmadj.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return fail(_e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,    \
                        std::string(#expr) + ": " + cudaGetErrorString(_e));             \
    } while (0)

enum Phase { PH_FLOW = 0, PH_THERM = 1, PH_ADJ = 2, PH_TADJ = 3 };

}  // namespace

int lbm::set_error(int status, const char* msg) {
    g_err = msg;
    return status;
}

struct lbm_ctx {
    int device = 0;
    int stencil = 1, Q = 19, storage = 1;
    bool thermal = false;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0, np = 0;
    size_t pb = 4, ab = 4, rb = 4;  // population / adjoint / aux element bytes

    cudaStream_t stream = nullptr;  // internal work stream
    cudaStream_t user = nullptr;    // caller's stream (ordering only)
    cudaEvent_t ev = nullptr;

    void* f[2] = {nullptr, nullptr};
    void* fa[2] = {nullptr, nullptr};
    void* g[2] = {nullptr, nullptr};
    void* ga[2] = {nullptr, nullptr};
    int fcur = 0, facur = 0, gcur = 0, gacur = 0;

    uint8_t* flags = nullptr;
    void* gamma = nullptr;
    void* bc = nullptr;
    void* u = nullptr;      // 3 planes
    void* rho = nullptr;
    void* T = nullptr;
    void* gpost = nullptr;  // 7 planes
    void* cpl = nullptr;    // 3 planes
    void* sT = nullptr;
    void* gcn = nullptr;
    void* sens = nullptr;
    double* partials = nullptr;
    double* dres = nullptr;
    double* hres = nullptr;  // pinned, 4 doubles

    Geom geom{};
    lbm_params prm{0.6, 1.0, 0, 0.0, 1.0, 0.0, 0.0, 0.0};
    lbm_objective obj{1.0, 0.0, 0.0};
    long long n_in = 0, n_nw = 0;
    bool have_flags = false, have_gamma = false, have_bc = false, have_params = false;
    bool fwd_done = false, adj_done = false;
    bool flow_done = false, tadj_done = false;  // phase-level completion (lbm_solve_phase)
    bool g_fresh = false;  // temperature populations hold the initial state, not yet collided
    bool fstate = false, astate = false;  // populations hold a usable (warm-start) state
    double J_p = 0.0, J_T = 0.0, J_Q = 0.0;
    double J() const { return J_p + (thermal ? J_T + J_Q : 0.0); }
    double last_I[4] = {0, 0, 0, 0};

    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    std::vector<uint8_t> hflags;   // host copy of the flags (per-face boundary values)
    int mirror = 0;                // axes with symmetry planes (lbm_set_symmetry)
    int adj_scheme = LBM_ADJOINT_DISCRETE;  // lbm_set_adjoint_scheme
    lbm_batch* holder = nullptr;   // batch whose memory budget counts this context

    void drop_graphs() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
    }
};

namespace {
// a destroyed context stops counting against its batch's memory budget
void batch_forget(lbm_batch* b, lbm_ctx* c);

void* dalloc(size_t bytes, cudaError_t* err) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess && *err == cudaSuccess) *err = e;
    return e == cudaSuccess ? p : nullptr;
}

void free_all(lbm_ctx* c) {
    c->drop_graphs();
    void* bufs[] = {c->f[0], c->f[1], c->fa[0], c->fa[1], c->g[0], c->g[1], c->ga[0], c->ga[1],
                    c->flags, c->gamma, c->bc, c->u, c->rho, c->T, c->gpost, c->cpl, c->sT,
                    c->gcn, c->sens, c->partials, c->dres};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (c->hres) cudaFreeHost(c->hres);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->stream) cudaStreamDestroy(c->stream);
}

// order ctx work after the caller's stream, and the caller's stream after it
lbm_status enter(lbm_ctx* c) {
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaEventRecord(c->ev, c->user));
    CUDA_TRY(cudaStreamWaitEvent(c->stream, c->ev, 0));
    return LBM_OK;
}

lbm_status leave(lbm_ctx* c) {
    CUDA_TRY(cudaEventRecord(c->ev, c->stream));
    CUDA_TRY(cudaStreamWaitEvent(c->user, c->ev, 0));
    return LBM_OK;
}

FlowLaunch flow_base(lbm_ctx* c) {
    FlowLaunch a;
    std::memset(&a, 0, sizeof(a));
    a.flags = c->flags;
    a.gamma = c->gamma;
    a.bc = c->bc;
    a.u = c->u;
    a.cpl = c->cpl;
    a.sT = c->sT;
    a.partials = c->partials;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.np = c->np;
    a.omega = 1.0 / c->prm.tau;
    a.rho0 = c->prm.rho0;
    a.src_in = c->n_in > 0 ? c->obj.w_pin / (3.0 * (double)c->n_in) : 0.0;
    a.ascale = 1.0;
    a.model = c->prm.gamma_model;
    a.mirror = c->mirror;
    return a;
}

ThermLaunch therm_base(lbm_ctx* c) {
    ThermLaunch a;
    std::memset(&a, 0, sizeof(a));
    a.flags = c->flags;
    a.gamma = c->gamma;
    a.bc = c->bc;
    a.u = c->u;
    a.gpost = c->gpost;
    a.gcn = c->gcn;
    a.partials = c->partials;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.np = c->np;
    a.rho0 = c->prm.rho0;
    a.kappa_f = c->prm.kappa_f;
    a.k_ratio = c->prm.k_ratio;
    a.q = c->prm.q_flux;
    a.T0 = c->prm.T0;
    a.src_T = c->n_nw > 0 ? c->obj.w_tmean / (double)c->n_nw : 0.0;
    a.ascale = 1.0;
    a.beta = c->prm.beta_max;
    a.src_q = c->obj.w_qgen * c->prm.beta_max;
    a.mirror = c->mirror;
    return a;
}

// values a phase's reducing step sums: flow |u| and inlet rho; temperature T
// and the heat source Q; the adjoints sum |f*| or |g*|
int phase_nv(int ph) { return ph == PH_FLOW || ph == PH_THERM ? 2 : 1; }

// enqueue one step of a phase on stream s; the reducing variant writes the
// per-block partial sums (and the fields of the post-boundary state)
cudaError_t enqueue_step(lbm_ctx* c, int ph, bool reduce, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (ph == PH_FLOW) {
        FlowLaunch a = flow_base(c);
        a.fin = c->f[c->fcur];
        a.fout = c->f[1 - c->fcur];
        a.out0 = c->rho;
        a.out1 = c->u;
        e = flow_launch(c->stencil, c->storage, reduce ? FOP_STEP_RED : FOP_STEP, a, c->geom, s);
        c->fcur ^= 1;
    } else if (ph == PH_THERM) {
        ThermLaunch a = therm_base(c);
        a.gin = c->g[c->gcur];
        a.gout = c->g[1 - c->gcur];
        a.out0 = c->T;
        a.out1 = c->gpost;
        e = thermal_launch(c->storage, reduce ? TOP_STEP_RED : TOP_STEP, a, c->geom, s);
        c->gcur ^= 1;
    } else if (ph == PH_ADJ) {
        FlowLaunch a = flow_base(c);
        a.ain = c->fa[c->facur];
        a.aout = c->fa[1 - c->facur];
        FlowOp op = c->thermal ? (reduce ? FOP_ADJ_T_RED : FOP_ADJ_T) : (reduce ? FOP_ADJ_RED : FOP_ADJ);
        if (c->adj_scheme == LBM_ADJOINT_CONTINUOUS) op = reduce ? FOP_ADJ_CONT_RED : FOP_ADJ_CONT;
        e = flow_launch(c->stencil, c->storage, op, a, c->geom, s);
        c->facur ^= 1;
    } else {
        ThermLaunch a = therm_base(c);
        a.ain = c->ga[c->gacur];
        a.aout = c->ga[1 - c->gacur];
        e = thermal_launch(c->storage, reduce ? TOP_ADJ_RED : TOP_ADJ, a, c->geom, s);
        c->gacur ^= 1;
    }
    return e;
}

int& parity_of(lbm_ctx* c, int ph) {
    return ph == PH_FLOW ? c->fcur : (ph == PH_THERM ? c->gcur : (ph == PH_ADJ ? c->facur : c->gacur));
}

// enqueue a block of k steps ending with a reduction, the finalize kernel and
// the copy of the sums to c->hres
cudaError_t enqueue_block(lbm_ctx* c, int ph, int k, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < k && e == cudaSuccess; ++i) e = enqueue_step(c, ph, i == k - 1, s);
    if (e != cudaSuccess) return e;
    e = finalize_launch(c->partials, c->geom.nblocks, phase_nv(ph), c->dres, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(c->hres, c->dres, sizeof(double) * phase_nv(ph), cudaMemcpyDeviceToHost, s);
}

lbm_status run_block(lbm_ctx* c, int ph, int k) {
    int& par = parity_of(c, ph);
    auto key = std::make_tuple(ph, k, par);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        int par0 = par;
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_block(c, ph, k, c->stream);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
        par = par0;  // capture only recorded the work
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            (void)cudaGetLastError();
            return fail(LBM_ERR_CUDA, std::string("graph capture failed: ") +
                                          cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        cudaGraphExec_t exec = nullptr;
        cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e3 != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e3));
        it = c->graphs.emplace(key, exec).first;
    }
    CUDA_TRY(cudaGraphLaunch(it->second, c->stream));
    if (k % 2) par ^= 1;
    return LBM_OK;
}

double rel_change(double cur, double prev) {
    double d = std::fabs(cur - prev);
    if (d == 0.0) return 0.0;
    return cur != 0.0 ? d / std::fabs(cur) : INFINITY;
}

// run a phase to tolerance (or a fixed number of steps when tol <= 0)
// NVTX ranges name each solve phase and batch step on a profiler's timeline
// (ncu --nvtx, Nsight Systems); with no tool attached a push/pop costs a call
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

lbm_status run_phase(lbm_ctx* c, int ph, const lbm_solve_opts* o, long long* steps_out,
                     double* res_out, double* I_out) {
    static const char* const kPhaseNames[4] = {"lbm flow", "lbm temperature", "lbm flow adjoint",
                                               "lbm temperature adjoint"};
    NvtxRange range(kPhaseNames[ph & 3]);
    const int K = o->check_every;
    long long steps = 0;
    double res = INFINITY;
    double prev = c->last_I[ph];
    double cur = prev;
    while (steps < o->max_steps) {
        long long k = std::min<long long>(K, o->max_steps - steps);
        lbm_status st = run_block(c, ph, (int)k);
        if (st != LBM_OK) return st;
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        steps += k;
        double denom = (double)(c->n_nw > 0 ? c->n_nw : 1);
        cur = c->hres[0] / denom;
        if (ph == PH_FLOW)
            c->J_p = c->n_in > 0 ? c->obj.w_pin * c->hres[1] / (3.0 * (double)c->n_in) : 0.0;
        if (ph == PH_THERM) {
            c->J_T = c->obj.w_tmean * cur;
            c->J_Q = -c->obj.w_qgen * c->hres[1];  // Eq. 72: J_Q = -sum Q
        }
        if (!std::isfinite(cur) || (phase_nv(ph) > 1 && !std::isfinite(c->hres[1]))) {
            *steps_out = steps;
            *res_out = NAN;
            *I_out = cur;
            c->last_I[ph] = cur;
            return fail(LBM_ERR_DIVERGED, "non-finite residual quantity after " +
                                              std::to_string(steps) + " steps");
        }
        res = rel_change(cur, prev);
        prev = cur;
        if (o->tol > 0 && res < o->tol) break;
    }
    c->last_I[ph] = cur;
    *steps_out = steps;
    *res_out = res;
    *I_out = cur;
    if (o->tol > 0 && !(res < o->tol)) return LBM_NOT_CONVERGED;
    return LBM_OK;
}

lbm_status check_opts(const lbm_solve_opts* o) {
    if (!o) return fail(LBM_ERR_ARG, "opts is null");
    if (o->max_steps < 0) return fail(LBM_ERR_ARG, "max_steps < 0");
    if (o->check_every <= 0) return fail(LBM_ERR_ARG, "check_every must be > 0");
    if (std::isnan(o->tol)) return fail(LBM_ERR_ARG, "tol is NaN");
    return LBM_OK;
}

lbm_status ready(lbm_ctx* c) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is null");
    if (!c->have_flags) return fail(LBM_ERR_ORDER, "lbm_set_flags has not been called");
    if (!c->have_gamma) return fail(LBM_ERR_ORDER, "lbm_set_gamma has not been called");
    if (!c->have_bc) return fail(LBM_ERR_ORDER, "boundary values have not been set (lbm_set_bc_values / lbm_set_bc)");
    if (!c->have_params) return fail(LBM_ERR_ORDER, "lbm_set_params has not been called");
    return LBM_OK;
}

// copy n values of dtype (host or device) into the ctx aux buffer dst (R type)
lbm_status copy_in(lbm_ctx* c, void* dst, const void* src, size_t n, int dtype, int on_device) {
    const bool r64 = c->rb == 8;
    const bool s64 = dtype == LBM_DTYPE_F64;
    if (on_device) {
        CUDA_TRY(convert_launch(src, s64, dst, r64, (long long)n, c->stream));
    } else if (s64 == r64) {
        CUDA_TRY(cudaMemcpyAsync(dst, src, n * c->rb, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } else {
        std::vector<char> tmp(n * c->rb);
        for (size_t i = 0; i < n; ++i) {
            double v = s64 ? ((const double*)src)[i] : (double)((const float*)src)[i];
            if (r64)
                ((double*)tmp.data())[i] = v;
            else
                ((float*)tmp.data())[i] = (float)v;
        }
        CUDA_TRY(cudaMemcpyAsync(dst, tmp.data(), n * c->rb, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

// copy nplanes planes of N values (stride np) out of an aux buffer
lbm_status copy_out(lbm_ctx* c, void* dst, const void* src, int nplanes, int dtype, int on_device) {
    const bool r64 = c->rb == 8;
    const bool d64 = dtype == LBM_DTYPE_F64;
    const size_t db = d64 ? 8 : 4;
    if (on_device) {
        for (int p = 0; p < nplanes; ++p)
            CUDA_TRY(convert_launch((const char*)src + p * c->np * c->rb, r64,
                                    (char*)dst + p * c->N * db, d64, c->N, c->stream));
    } else {
        std::vector<char> tmp(c->N * c->rb);
        for (int p = 0; p < nplanes; ++p) {
            CUDA_TRY(cudaMemcpyAsync(tmp.data(), (const char*)src + p * c->np * c->rb, c->N * c->rb,
                                     cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            for (long long i = 0; i < c->N; ++i) {
                double v = r64 ? ((double*)tmp.data())[i] : (double)((float*)tmp.data())[i];
                if (d64)
                    ((double*)dst)[p * c->N + i] = v;
                else
                    ((float*)dst)[p * c->N + i] = (float)v;
            }
        }
    }
    return LBM_OK;
}

lbm_status init_flow(lbm_ctx* c) {
    FlowLaunch a = flow_base(c);
    a.fout = c->f[0];
    a.out0 = c->rho;
    a.out1 = c->u;
    c->fcur = 0;
    CUDA_TRY(flow_launch(c->stencil, c->storage, FOP_INIT_F, a, c->geom, c->stream));
    c->last_I[PH_FLOW] = 0.0;
    return LBM_OK;
}

lbm_status init_temperature(lbm_ctx* c) {
    ThermLaunch t = therm_base(c);
    t.gout = c->g[0];
    t.out0 = c->T;
    t.out1 = c->gpost;
    c->gcur = 0;
    CUDA_TRY(thermal_launch(c->storage, TOP_INIT_G, t, c->geom, c->stream));
    c->last_I[PH_THERM] = c->prm.T0;
    c->g_fresh = true;
    return LBM_OK;
}

// the stored temperature populations are post-collision ones: collide the
// initial state once with the frozen flow before the first temperature step
lbm_status collide_initial_temperature(lbm_ctx* c) {
    if (!c->g_fresh) return LBM_OK;
    ThermLaunch t = therm_base(c);
    t.gout = c->g[c->gcur];
    CUDA_TRY(thermal_launch(c->storage, TOP_COLLIDE_INIT, t, c->geom, c->stream));
    c->g_fresh = false;
    return LBM_OK;
}

lbm_status init_forward(lbm_ctx* c) {
    lbm_status st = init_flow(c);
    if (st == LBM_OK && c->thermal) st = init_temperature(c);
    return st;
}

lbm_status init_flow_adjoint(lbm_ctx* c) {
    FlowLaunch a = flow_base(c);
    a.aout = c->fa[0];
    c->facur = 0;
    CUDA_TRY(flow_launch(c->stencil, c->storage, FOP_INIT_A, a, c->geom, c->stream));
    c->last_I[PH_ADJ] = 0.0;
    return LBM_OK;
}

lbm_status init_temperature_adjoint(lbm_ctx* c) {
    ThermLaunch t = therm_base(c);
    t.aout = c->ga[0];
    c->gacur = 0;
    CUDA_TRY(thermal_launch(c->storage, TOP_INIT_A, t, c->geom, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->cpl, 0, 3 * c->np * c->rb, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->sT, 0, c->np * c->rb, c->stream));
    c->last_I[PH_TADJ] = 0.0;
    return LBM_OK;
}

lbm_status init_adjoint(lbm_ctx* c) {
    lbm_status st = init_flow_adjoint(c);
    if (st == LBM_OK && c->thermal) st = init_temperature_adjoint(c);
    return st;
}

// thermal-to-flow coupling and thermal sensitivity from the current
// temperature adjoint iterate (run once the temperature adjoint has finished)
lbm_status run_coupling(lbm_ctx* c) {
    ThermLaunch t = therm_base(c);
    t.gin = c->g[c->gcur];
    t.ain = c->ga[c->gacur];
    t.out0 = c->cpl;
    t.out1 = c->sT;
    CUDA_TRY(thermal_launch(c->storage, TOP_COUPLING, t, c->geom, c->stream));
    return LBM_OK;
}

// One phase of the solve sequence flow -> temperature -> temperature adjoint
// (+ coupling) -> flow adjoint, with its order checks and state bookkeeping.
// do_reset restarts the phase's populations (the flow phase restarts the
// temperature populations too, the temperature-adjoint phase the flow-adjoint
// ones: a restarted phase invalidates the warm start of the phases after it).
lbm_status solve_phase(lbm_ctx* c, int ph, const lbm_solve_opts* o, bool do_reset,
                       long long* steps, double* res, double* I) {
    *steps = 0;
    *res = 0;
    *I = 0;
    lbm_status st = LBM_OK;
    if (ph == PH_FLOW) {
        if (do_reset || !c->fstate) {
            if ((st = init_forward(c)) != LBM_OK) return st;
            c->fstate = true;
        }
        c->flow_done = c->fwd_done = c->tadj_done = c->adj_done = false;
    } else if (ph == PH_THERM) {
        if (!c->flow_done) return fail(LBM_ERR_ORDER, "the temperature phase needs a completed flow phase");
        if (do_reset && (st = init_temperature(c)) != LBM_OK) return st;
        if ((st = collide_initial_temperature(c)) != LBM_OK) return st;
        c->fwd_done = c->tadj_done = c->adj_done = false;
    } else if (ph == PH_TADJ) {
        if (!c->fwd_done) return fail(LBM_ERR_ORDER, "the temperature adjoint needs a completed forward solve");
        if (do_reset || !c->astate) {
            if ((st = init_adjoint(c)) != LBM_OK) return st;
            c->astate = true;
        }
        c->tadj_done = c->adj_done = false;
    } else {
        if (!c->fwd_done) return fail(LBM_ERR_ORDER, "the flow adjoint needs a completed forward solve");
        if (c->adj_scheme == LBM_ADJOINT_CONTINUOUS && (c->stencil != LBM_D2Q9 || c->thermal || c->mirror))
            return fail(LBM_ERR_UNSUPPORTED,
                        "the continuous adjoint is built for D2Q9 flow without symmetry planes");
        if (c->thermal && !c->tadj_done)
            return fail(LBM_ERR_ORDER, "the flow adjoint needs a completed temperature adjoint");
        if (!c->astate) {
            if ((st = init_adjoint(c)) != LBM_OK) return st;
            c->astate = true;
        } else if (do_reset) {
            if ((st = init_flow_adjoint(c)) != LBM_OK) return st;
        }
        c->adj_done = false;
    }
    st = run_phase(c, ph, o, steps, res, I);
    if (st < 0) {
        // a failed phase leaves no usable warm start for its lattice pair
        if (ph == PH_FLOW || ph == PH_THERM) c->fstate = false;
        else c->astate = false;
        return st;
    }
    if (ph == PH_FLOW) {
        c->flow_done = true;
        c->fwd_done = !c->thermal;
    } else if (ph == PH_THERM) {
        c->fwd_done = true;
    } else if (ph == PH_TADJ) {
        lbm_status s2 = run_coupling(c);
        if (s2 != LBM_OK) return s2;
        c->tadj_done = true;
    } else {
        c->adj_done = true;
    }
    return st;
}

double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm_check_addressing(int stencil, int nx, int ny, int nz, long long* mismatches) {
    if (!mismatches) return fail(LBM_ERR_ARG, "mismatches is null");
    if (stencil < 0 || stencil > 2) return fail(LBM_ERR_ARG, "unknown stencil");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(LBM_ERR_ARG, "lattice sizes must be positive");
    if ((long long)nx * ny * nz > (1LL << 24)) return fail(LBM_ERR_ARG, "at most 2^24 nodes (a host loop)");
    *mismatches = addressing_mismatches(stencil, nx, ny, nz);
    return LBM_OK;
}

const char* lbm_version(void) { return "lbmadj 0.1 (sm_103a)"; }

lbm_status lbm_create(lbm_ctx** out, int stencil, int nx, int ny, int nz, int storage, int thermal) {
    if (!out) return fail(LBM_ERR_ARG, "out is null");
    *out = nullptr;
    if (stencil != LBM_D2Q9 && stencil != LBM_D3Q19) return fail(LBM_ERR_ARG, "unknown stencil");
    if (storage < LBM_FP64 || storage > LBM_BF16_OFS) return fail(LBM_ERR_ARG, "unknown storage");
    if (nx <= 0 || ny <= 0 || nz <= 0) return fail(LBM_ERR_ARG, "lattice sizes must be positive");
    if (stencil == LBM_D2Q9 && nz != 1) return fail(LBM_ERR_ARG, "D2Q9 needs nz == 1");
    if (stencil == LBM_D2Q9 && thermal) return fail(LBM_ERR_UNSUPPORTED, "thermal lattice needs D3Q19");
    if (stencil == LBM_D2Q9 && storage > LBM_FP32)
        return fail(LBM_ERR_UNSUPPORTED, "16-bit storage is built for D3Q19 only");
    if ((long long)nx * ny * nz > (1LL << 31) - 1024) return fail(LBM_ERR_ARG, "lattice too large");
    lbm_ctx* c = new lbm_ctx();
    cudaGetDevice(&c->device);
    c->stencil = stencil;
    c->Q = stencil == LBM_D2Q9 ? 9 : 19;
    c->storage = storage;
    c->thermal = thermal != 0;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = (long long)nx * ny * nz;
    c->np = (c->N + 63) / 64 * 64;
    c->pb = pop_bytes(storage);
    c->ab = adj_bytes(storage);
    c->rb = aux_bytes(storage);
    c->geom = make_geom(nx, ny, nz);
    cudaError_t e = cudaSuccess;
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(LBM_ERR_CUDA, std::string("stream/event: ") + cudaGetErrorString(e));
    }
    const size_t np = (size_t)c->np;
    for (int b = 0; b < 2; ++b) {
        c->f[b] = dalloc(np * c->Q * c->pb, &e);
        c->fa[b] = dalloc(np * c->Q * c->ab, &e);
        if (c->thermal) {
            c->g[b] = dalloc(np * 7 * heat_bytes(storage), &e);
            c->ga[b] = dalloc(np * 7 * c->ab, &e);
        }
    }
    c->flags = (uint8_t*)dalloc(np, &e);
    c->gamma = dalloc(np * c->rb, &e);
    c->bc = dalloc(np * 4 * c->rb, &e);
    c->u = dalloc(np * 3 * c->rb, &e);
    c->rho = dalloc(np * c->rb, &e);
    c->sens = dalloc(np * c->rb, &e);
    if (c->thermal) {
        c->T = dalloc(np * c->rb, &e);
        c->gpost = dalloc(np * 7 * c->rb, &e);
        c->cpl = dalloc(np * 3 * c->rb, &e);
        c->sT = dalloc(np * c->rb, &e);
        c->gcn = dalloc(np * c->rb, &e);
    }
    c->partials = (double*)dalloc(sizeof(double) * 2 * (size_t)c->geom.nblocks, &e);
    c->dres = (double*)dalloc(sizeof(double) * 4, &e);
    if (e == cudaSuccess) e = cudaMallocHost(&c->hres, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 1 /* WALL */, np, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bc, 0, np * 4 * c->rb, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->gamma, 0, np * c->rb, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                    std::string("allocation: ") + cudaGetErrorString(e));
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->holder) batch_forget(c->holder, c);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* s) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is null");
    c->user = (cudaStream_t)s;
    return LBM_OK;
}

lbm_status lbm_set_flags(lbm_ctx* c, const uint8_t* flags, size_t n, int on_device) {
    if (!c || !flags) return fail(LBM_ERR_ARG, "null argument");
    if ((long long)n != c->N) return fail(LBM_ERR_ARG, "flags: n != nx*ny*nz");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    std::vector<uint8_t> h(n);
    if (on_device) {
        CUDA_TRY(cudaMemcpyAsync(h.data(), flags, n, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(h.data(), flags, n);
    }
    long long nin = 0, nnw = 0;
    for (size_t i = 0; i < n; ++i) {
        int fl = h[i], type = fl & 7, code = (fl >> 3) & 7;
        if (fl & 0x80) return fail(LBM_ERR_ARG, "flag bit 7 set at node " + std::to_string(i));
        if (type > 3) return fail(LBM_ERR_ARG, "unknown node type at node " + std::to_string(i));
        if ((type >= 2 || (fl & 0x40)) && (code > 5 || (c->stencil == LBM_D2Q9 && code > 3)))
            return fail(LBM_ERR_ARG, "bad normal code at node " + std::to_string(i));
        if ((fl & 0x40) && type != 1 && type != 3)
            return fail(LBM_ERR_ARG, "bit 6 on a node that is neither a wall nor a fixed-density node");
        nin += type == 2;
        nnw += type != 1;
    }
    CUDA_TRY(cudaMemcpyAsync(c->flags, h.data(), n, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->hflags.swap(h);
    // the captured step graphs read the flags from device memory, but their
    // objective source terms are baked from N_in and N_nonwall: recapture only
    // when those counts change
    if (!c->have_flags || nin != c->n_in || nnw != c->n_nw) c->drop_graphs();
    c->n_in = nin;
    c->n_nw = nnw;
    c->have_flags = true;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    c->fstate = c->astate = false;
    return leave(c);
}

lbm_status lbm_set_gamma(lbm_ctx* c, const void* gamma, size_t n, int dtype, int on_device) {
    if (!c || !gamma) return fail(LBM_ERR_ARG, "null argument");
    if ((long long)n != c->N) return fail(LBM_ERR_ARG, "gamma: n != nx*ny*nz");
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_ERR_ARG, "bad dtype");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    st = copy_in(c, c->gamma, gamma, n, dtype, on_device);
    if (st != LBM_OK) return st;
    c->have_gamma = true;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    return leave(c);
}

lbm_status lbm_set_bc_values(lbm_ctx* c, const void* v, size_t n, int dtype, int on_device) {
    if (!c || !v) return fail(LBM_ERR_ARG, "null argument");
    if ((long long)n != 4 * c->N) return fail(LBM_ERR_ARG, "bc values: n != 4*nx*ny*nz");
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_ERR_ARG, "bad dtype");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    st = copy_in(c, c->bc, v, n, dtype, on_device);
    if (st != LBM_OK) return st;
    c->have_bc = true;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    return leave(c);
}

lbm_status lbm_set_params(lbm_ctx* c, const lbm_params* p) {
    if (!c || !p) return fail(LBM_ERR_ARG, "null argument");
    if (!(p->tau > 0.5)) return fail(LBM_ERR_ARG, "tau must be > 0.5");
    if (!(p->rho0 > 0)) return fail(LBM_ERR_ARG, "rho0 must be > 0");
    if (p->gamma_model != LBM_GAMMA_EQ12 && p->gamma_model != LBM_GAMMA_LINEAR)
        return fail(LBM_ERR_ARG, "unknown gamma model");
    if (c->thermal && !(p->kappa_f >= 0)) return fail(LBM_ERR_ARG, "kappa_f must be >= 0");
    if (c->thermal && !(p->k_ratio > 0)) return fail(LBM_ERR_ARG, "k_ratio must be > 0");
    if (!std::isfinite(p->q_flux) || !std::isfinite(p->T0)) return fail(LBM_ERR_ARG, "non-finite q_flux / T0");
    if (!(p->beta_max >= 0) || !std::isfinite(p->beta_max)) return fail(LBM_ERR_ARG, "beta_max must be >= 0");
    if (p->beta_max != 0 && !c->thermal) return fail(LBM_ERR_ARG, "beta_max needs the thermal lattice");
    // the captured graphs bake these values into their launches: recapture
    // only when one of them changes
    const lbm_params& q = c->prm;
    const bool same = c->have_params && q.tau == p->tau && q.rho0 == p->rho0 &&
                      q.gamma_model == p->gamma_model && q.kappa_f == p->kappa_f &&
                      q.k_ratio == p->k_ratio && q.q_flux == p->q_flux && q.T0 == p->T0 &&
                      q.beta_max == p->beta_max;
    if (!same) c->drop_graphs();
    c->prm = *p;
    c->have_params = true;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    return LBM_OK;
}

lbm_status lbm_set_objective(lbm_ctx* c, const lbm_objective* o) {
    if (!c || !o) return fail(LBM_ERR_ARG, "null argument");
    if (!std::isfinite(o->w_pin) || !std::isfinite(o->w_tmean) || !std::isfinite(o->w_qgen))
        return fail(LBM_ERR_ARG, "non-finite weights");
    if (o->w_qgen != 0 && !c->thermal) return fail(LBM_ERR_ARG, "w_qgen needs the thermal lattice");
    if (c->obj.w_pin != o->w_pin || c->obj.w_tmean != o->w_tmean || c->obj.w_qgen != o->w_qgen)
        c->drop_graphs();
    c->obj = *o;
    c->adj_done = c->tadj_done = false;
    return LBM_OK;
}

lbm_status lbm_set_adjoint_scheme(lbm_ctx* c, int scheme) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is null");
    if (scheme != LBM_ADJOINT_DISCRETE && scheme != LBM_ADJOINT_CONTINUOUS)
        return fail(LBM_ERR_ARG, "unknown adjoint scheme");
    if (scheme == LBM_ADJOINT_CONTINUOUS && (c->stencil != LBM_D2Q9 || c->thermal))
        return fail(LBM_ERR_UNSUPPORTED, "the continuous adjoint is built for D2Q9 flow lattices");
    if (scheme != c->adj_scheme) {
        c->drop_graphs();
        c->astate = false;  // the stored adjoint means another quantity
    }
    c->adj_scheme = scheme;
    c->adj_done = c->tadj_done = false;
    return LBM_OK;
}

lbm_status lbm_set_symmetry(lbm_ctx* c, int axes) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is null");
    if (axes < 0 || axes > 7) return fail(LBM_ERR_ARG, "axes must be a mask of bits 0 (x), 1 (y), 2 (z)");
    if (c->stencil == LBM_D2Q9 && (axes & 4)) return fail(LBM_ERR_ARG, "D2Q9 lattices have no z axis");
    if (axes != c->mirror) c->drop_graphs();  // the captured launches carry the mask
    c->mirror = axes;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    return LBM_OK;
}

lbm_status lbm_physics_to_params(const lbm_physics* ph, lbm_params* out) {
    if (!ph || !out) return fail(LBM_ERR_ARG, "null argument");
    const double vals[] = {ph->re, ph->u_ref, ph->l_ref, ph->dp, ph->pr, ph->rho0,
                           ph->k_ratio, ph->q_flux, ph->T0, ph->beta_max};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(LBM_ERR_ARG, "non-finite physics value");
    if (!(ph->re > 0)) return fail(LBM_ERR_ARG, "re must be > 0");
    if (!(ph->l_ref > 0)) return fail(LBM_ERR_ARG, "l_ref must be > 0");
    if (!(ph->rho0 > 0)) return fail(LBM_ERR_ARG, "rho0 must be > 0");
    if (ph->pr < 0) return fail(LBM_ERR_ARG, "pr must be >= 0");
    double U = ph->u_ref;
    if (!(U > 0)) {
        if (!(ph->dp > 0)) return fail(LBM_ERR_ARG, "needs u_ref > 0 or a pressure drop dp > 0");
        U = std::sqrt(ph->dp / ph->rho0);  // Eq. 70
    }
    const double nu = U * ph->l_ref / ph->re;  // Re = U L / nu
    lbm_params p;
    p.tau = 0.5 + 3.0 * nu;                    // Eq. 3: nu = (tau - 1/2) c_s^2, c_s^2 = 1/3
    p.rho0 = ph->rho0;
    p.gamma_model = ph->gamma_model;
    p.kappa_f = ph->pr > 0 ? nu / ph->pr : 0.0;
    p.k_ratio = ph->k_ratio;
    p.q_flux = ph->q_flux;
    p.T0 = ph->T0;
    p.beta_max = ph->beta_max;
    *out = p;
    return LBM_OK;
}

lbm_status lbm_set_physics(lbm_ctx* c, const lbm_physics* ph) {
    if (!c || !ph) return fail(LBM_ERR_ARG, "null argument");
    if (c->thermal && !(ph->pr > 0)) return fail(LBM_ERR_ARG, "pr must be > 0 with the thermal lattice");
    lbm_params p;
    lbm_status st = lbm_physics_to_params(ph, &p);
    if (st != LBM_OK) return st;
    return lbm_set_params(c, &p);
}

lbm_status lbm_set_bc(lbm_ctx* c, int face, int kind, const void* values, size_t n, int dtype,
                      int on_device) {
    if (!c || !values) return fail(LBM_ERR_ARG, "null argument");
    if (face < 0 || face > 5) return fail(LBM_ERR_ARG, "face must be 0..5");
    if (c->stencil == LBM_D2Q9 && face > 3) return fail(LBM_ERR_ARG, "D2Q9 lattices have faces 0..3");
    if (kind != LBM_VEL && kind != LBM_PRES) return fail(LBM_ERR_ARG, "kind must be LBM_VEL or LBM_PRES");
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_ERR_ARG, "bad dtype");
    if (!c->have_flags) return fail(LBM_ERR_ORDER, "lbm_set_flags has not been called");
    // the face as a 2-D block of nodes: start node, row width, row pitch, rows
    const long long nx = c->nx, ny = c->ny, nz = c->nz;
    const int ax = face >> 1, hi = face & 1;
    long long start = 0, width = 0, pitch = 0, rows = 0;
    if (ax == 0) { start = hi ? nx - 1 : 0; width = 1; pitch = nx; rows = ny * nz; }
    else if (ax == 1) { start = hi ? nx * (ny - 1) : 0; width = nx; pitch = nx * ny; rows = nz; }
    else { start = hi ? nx * ny * (nz - 1) : 0; width = nx * ny; pitch = nx * ny; rows = 1; }
    std::vector<long long> slot;  // position in the face block of each matching node, node order
    for (long long r = 0; r < rows; ++r)
        for (long long w = 0; w < width; ++w) {
            const uint8_t fl = c->hflags[start + r * pitch + w];
            if ((fl & 7) == kind && ((fl >> 3) & 7) == face) slot.push_back(r * width + w);
        }
    const size_t m = slot.size();
    if (m == 0) return fail(LBM_ERR_ARG, "no node of this kind with this normal on the face");
    if (n != 4 && n != 4 * m) return fail(LBM_ERR_ARG, "values: n must be 4 or 4 x the face's nodes of this kind");
    std::vector<double> v(n);
    const size_t eb = dtype == LBM_DTYPE_F64 ? 8 : 4;
    std::vector<char> raw(n * eb);
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    if (on_device) {
        CUDA_TRY(cudaMemcpyAsync(raw.data(), values, n * eb, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(raw.data(), values, n * eb);
    }
    for (size_t i = 0; i < n; ++i)
        v[i] = eb == 8 ? ((const double*)raw.data())[i] : (double)((const float*)raw.data())[i];
    for (double x : v)
        if (!std::isfinite(x)) return fail(LBM_ERR_ARG, "non-finite boundary value");
    // read the face block, write the matching nodes' four values, put it back
    const size_t rb = c->rb, nb = 4 * rb;
    std::vector<char> blk((size_t)(rows * width) * nb);
    char* base = (char*)c->bc + (size_t)start * nb;
    CUDA_TRY(cudaMemcpy2DAsync(blk.data(), width * nb, base, pitch * nb, width * nb, rows,
                               cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (size_t k = 0; k < m; ++k)
        for (int j = 0; j < 4; ++j) {
            const double x = v[(n == 4 ? 0 : 4 * k) + j];
            char* dst = blk.data() + (size_t)slot[k] * nb + j * rb;
            if (rb == 8) *(double*)dst = x;
            else *(float*)dst = (float)x;
        }
    CUDA_TRY(cudaMemcpy2DAsync(base, pitch * nb, blk.data(), width * nb, width * nb, rows,
                               cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->have_bc = true;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    return leave(c);
}

lbm_status lbm_forward(lbm_ctx* c, const lbm_solve_opts* o, lbm_report* rep) {
    lbm_status st = ready(c);
    if (st != LBM_OK) return st;
    if ((st = check_opts(o)) != LBM_OK) return st;
    double t0 = now_ms();
    if ((st = enter(c)) != LBM_OK) return st;
    long long s1 = 0, s2 = 0;
    double res = 0, I = 0;
    lbm_status st1 = solve_phase(c, PH_FLOW, o, o->reset != 0, &s1, &res, &I);
    lbm_status st2 = LBM_OK;
    if (st1 >= 0 && c->thermal) {
        double r2 = 0, I2 = 0;
        st2 = solve_phase(c, PH_THERM, o, false, &s2, &r2, &I2);
        res = std::max(res, r2);
        I = I2;
    }
    lbm_status final = st1 < 0 ? st1 : (st2 < 0 ? st2 : (st1 > 0 ? st1 : st2));
    if (rep) {
        rep->steps = s1 + s2;
        rep->residual = res;
        rep->I = I;
        rep->J = c->J();
        rep->ms = now_ms() - t0;
        rep->status = final;
    }
    lbm_status lv = leave(c);
    return final != LBM_OK ? final : lv;
}

lbm_status lbm_adjoint(lbm_ctx* c, const lbm_solve_opts* o, lbm_report* rep) {
    lbm_status st = ready(c);
    if (st != LBM_OK) return st;
    if ((st = check_opts(o)) != LBM_OK) return st;
    if (!c->fwd_done) return fail(LBM_ERR_ORDER, "lbm_adjoint needs a completed lbm_forward");
    double t0 = now_ms();
    if ((st = enter(c)) != LBM_OK) return st;
    long long s1 = 0, s2 = 0;
    double res = 0, I = 0;
    lbm_status st1 = LBM_OK, st2 = LBM_OK;
    if (c->thermal) st1 = solve_phase(c, PH_TADJ, o, o->reset != 0, &s1, &res, &I);
    if (st1 >= 0) {
        double r2 = 0, I2 = 0;
        st2 = solve_phase(c, PH_ADJ, o, !c->thermal && o->reset != 0, &s2, &r2, &I2);
        res = std::max(res, r2);
        I = I2;
    }
    lbm_status final = st1 < 0 ? st1 : (st2 < 0 ? st2 : (st1 > 0 ? st1 : st2));
    if (rep) {
        rep->steps = s1 + s2;
        rep->residual = res;
        rep->I = I;
        rep->J = c->J();
        rep->ms = now_ms() - t0;
        rep->status = final;
    }
    lbm_status lv = leave(c);
    return final != LBM_OK ? final : lv;
}

lbm_status lbm_solve_phase(lbm_ctx* c, int phase, const lbm_solve_opts* o, lbm_report* rep) {
    lbm_status st = ready(c);
    if (st != LBM_OK) return st;
    if ((st = check_opts(o)) != LBM_OK) return st;
    if (phase < PH_FLOW || phase > PH_TADJ) return fail(LBM_ERR_ARG, "unknown phase");
    if ((phase == PH_THERM || phase == PH_TADJ) && !c->thermal)
        return fail(LBM_ERR_ARG, "temperature phase without the thermal lattice");
    double t0 = now_ms();
    if ((st = enter(c)) != LBM_OK) return st;
    long long steps = 0;
    double res = 0, I = 0;
    lbm_status final = solve_phase(c, phase, o, o->reset != 0, &steps, &res, &I);
    if (rep) {
        rep->steps = steps;
        rep->residual = res;
        rep->I = I;
        rep->J = c->J();
        rep->ms = now_ms() - t0;
        rep->status = final;
    }
    if (final == LBM_ERR_ORDER || final == LBM_ERR_ARG) return final;
    lbm_status lv = leave(c);
    return final != LBM_OK ? final : lv;
}

lbm_status lbm_sensitivity(lbm_ctx* c, void* out, int dtype, int on_device) {
    if (!c || !out) return fail(LBM_ERR_ARG, "null argument");
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_ERR_ARG, "bad dtype");
    if (!c->adj_done) return fail(LBM_ERR_ORDER, "lbm_sensitivity needs a completed lbm_adjoint");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    FlowLaunch a = flow_base(c);
    a.ain = c->fa[c->facur];
    a.out0 = c->sens;
    const FlowOp op = c->adj_scheme == LBM_ADJOINT_CONTINUOUS ? FOP_SENS_CONT : (c->thermal ? FOP_SENS_T : FOP_SENS);
    CUDA_TRY(flow_launch(c->stencil, c->storage, op, a, c->geom, c->stream));
    st = copy_out(c, out, c->sens, 1, dtype, on_device);
    if (st != LBM_OK) return st;
    return leave(c);
}

lbm_status lbm_get_fields(lbm_ctx* c, void* rho, void* u, void* T, int dtype, int on_device) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is null");
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_ERR_ARG, "bad dtype");
    if (!c->fwd_done) return fail(LBM_ERR_ORDER, "lbm_get_fields needs a completed lbm_forward");
    if (T && !c->thermal) return fail(LBM_ERR_ARG, "T requested without the thermal lattice");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    if (rho && (st = copy_out(c, rho, c->rho, 1, dtype, on_device)) != LBM_OK) return st;
    if (u && (st = copy_out(c, u, c->u, 3, dtype, on_device)) != LBM_OK) return st;
    if (T && (st = copy_out(c, T, c->T, 1, dtype, on_device)) != LBM_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return leave(c);
}

lbm_status lbm_get_objective(lbm_ctx* c, double* J) {
    if (!c || !J) return fail(LBM_ERR_ARG, "null argument");
    if (!c->fwd_done) return fail(LBM_ERR_ORDER, "lbm_get_objective needs a completed lbm_forward");
    *J = c->J();
    return LBM_OK;
}

lbm_status lbm_get_adjoint(lbm_ctx* c, void* fstar, void* gstar, int dtype, int on_device) {
    if (!c) return fail(LBM_ERR_ARG, "ctx is null");
    if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return fail(LBM_ERR_ARG, "bad dtype");
    if (!c->adj_done) return fail(LBM_ERR_ORDER, "lbm_get_adjoint needs a completed lbm_adjoint");
    if (gstar && !c->thermal) return fail(LBM_ERR_ARG, "gstar requested without the thermal lattice");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    if (fstar && (st = copy_out(c, fstar, c->fa[c->facur], c->Q, dtype, on_device)) != LBM_OK) return st;
    if (gstar && (st = copy_out(c, gstar, c->ga[c->gacur], 7, dtype, on_device)) != LBM_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return leave(c);
}

// ---------------------------------------------------------------------------
// state checkpoint: a header, then the current buffer of every population set
// and the fields a resumed solve reads (plain copies, any memory kind)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct StateHeader {
    char magic[8];  // "LBMSTATE"
    int version;
    int stencil, storage, thermal;
    int nx, ny, nz;
    long long np, n_in, n_nw;
    int fstate, astate, fwd_done, adj_done;
    int flow_done, tadj_done, g_fresh;
    double J_p, J_T, J_Q;
    double last_I[4];
    double tau, rho0;
};

struct StatePart {
    void* buf;
    size_t bytes;
};

std::vector<StatePart> state_parts(lbm_ctx* c) {
    const size_t np = (size_t)c->np;
    std::vector<StatePart> v;
    v.push_back({c->f[c->fcur], np * c->Q * c->pb});
    v.push_back({c->fa[c->facur], np * c->Q * c->ab});
    v.push_back({c->rho, np * c->rb});
    v.push_back({c->u, np * 3 * c->rb});
    if (c->thermal) {
        v.push_back({c->g[c->gcur], np * 7 * heat_bytes(c->storage)});
        v.push_back({c->ga[c->gacur], np * 7 * c->ab});
        v.push_back({c->T, np * c->rb});
        v.push_back({c->gpost, np * 7 * c->rb});
        v.push_back({c->gcn, np * c->rb});
        v.push_back({c->cpl, np * 3 * c->rb});
        v.push_back({c->sT, np * c->rb});
    }
    return v;
}

constexpr size_t kStateAlign = 256;

size_t state_size(lbm_ctx* c) {
    size_t b = (sizeof(StateHeader) + kStateAlign - 1) / kStateAlign * kStateAlign;
    for (const StatePart& p : state_parts(c)) b += (p.bytes + kStateAlign - 1) / kStateAlign * kStateAlign;
    return b;
}

}  // namespace

extern "C" {

size_t lbm_state_bytes(lbm_ctx* c) { return c ? state_size(c) : 0; }

lbm_status lbm_export_state(lbm_ctx* c, void* dst, size_t bytes) {
    if (!c || !dst) return fail(LBM_ERR_ARG, "null argument");
    if (bytes < state_size(c)) return fail(LBM_ERR_ARG, "state buffer smaller than lbm_state_bytes");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "LBMSTATE", 8);
    h.version = 2;
    h.stencil = c->stencil;
    h.storage = c->storage;
    h.thermal = c->thermal;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.np = c->np;
    h.n_in = c->n_in;
    h.n_nw = c->n_nw;
    h.fstate = c->fstate;
    h.astate = c->astate;
    h.fwd_done = c->fwd_done;
    h.adj_done = c->adj_done;
    h.flow_done = c->flow_done;
    h.tadj_done = c->tadj_done;
    h.g_fresh = c->g_fresh;
    h.J_p = c->J_p;
    h.J_T = c->J_T;
    h.J_Q = c->J_Q;
    for (int k = 0; k < 4; ++k) h.last_I[k] = c->last_I[k];
    h.tau = c->prm.tau;
    h.rho0 = c->prm.rho0;
    char* d = (char*)dst;
    size_t off = (sizeof(StateHeader) + kStateAlign - 1) / kStateAlign * kStateAlign;
    for (const StatePart& p : state_parts(c)) {
        CUDA_TRY(cudaMemcpyAsync(d + off, p.buf, p.bytes, cudaMemcpyDefault, c->stream));
        off += (p.bytes + kStateAlign - 1) / kStateAlign * kStateAlign;
    }
    CUDA_TRY(cudaMemcpyAsync(d, &h, sizeof(h), cudaMemcpyDefault, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return leave(c);
}

lbm_status lbm_import_state(lbm_ctx* c, const void* src, size_t bytes) {
    if (!c || !src) return fail(LBM_ERR_ARG, "null argument");
    if (bytes < sizeof(StateHeader)) return fail(LBM_ERR_ARG, "state buffer smaller than its header");
    lbm_status st = enter(c);
    if (st != LBM_OK) return st;
    StateHeader h;
    CUDA_TRY(cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDefault, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (std::memcmp(h.magic, "LBMSTATE", 8) != 0 || h.version != 2)
        return fail(LBM_ERR_ARG, "not a state written by lbm_export_state");
    if (h.stencil != c->stencil || h.storage != c->storage || h.thermal != (int)c->thermal ||
        h.nx != c->nx || h.ny != c->ny || h.nz != c->nz || h.np != c->np)
        return fail(LBM_ERR_ARG, "state is for another lattice shape, stencil, storage or thermal setting");
    if (!c->have_flags || !c->have_params || h.n_in != c->n_in || h.n_nw != c->n_nw ||
        h.tau != c->prm.tau || h.rho0 != c->prm.rho0)
        return fail(LBM_ERR_ARG, "set the same flags and parameters before importing a state");
    if (bytes < state_size(c)) return fail(LBM_ERR_ARG, "state buffer smaller than lbm_state_bytes");
    c->fcur = c->facur = c->gcur = c->gacur = 0;
    const char* s = (const char*)src;
    size_t off = (sizeof(StateHeader) + kStateAlign - 1) / kStateAlign * kStateAlign;
    for (const StatePart& p : state_parts(c)) {
        CUDA_TRY(cudaMemcpyAsync(p.buf, s + off, p.bytes, cudaMemcpyDefault, c->stream));
        off += (p.bytes + kStateAlign - 1) / kStateAlign * kStateAlign;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->fstate = h.fstate;
    c->astate = h.astate;
    c->fwd_done = h.fwd_done;
    c->adj_done = h.adj_done;
    c->flow_done = h.flow_done;
    c->tadj_done = h.tadj_done;
    c->g_fresh = h.g_fresh;
    c->J_p = h.J_p;
    c->J_T = h.J_T;
    c->J_Q = h.J_Q;
    for (int k = 0; k < 4; ++k) c->last_I[k] = h.last_I[k];
    return leave(c);
}

lbm_status lbm_time_steps(lbm_ctx* c, int phase, int n, double* ms_per_step) {
    lbm_status st = ready(c);
    if (st != LBM_OK) return st;
    if (!ms_per_step || n <= 0 || phase < 0 || phase > 3) return fail(LBM_ERR_ARG, "bad argument");
    if ((phase == PH_THERM || phase == PH_TADJ) && !c->thermal)
        return fail(LBM_ERR_ARG, "temperature phase without the thermal lattice");
    if (phase != PH_FLOW && !c->fwd_done) return fail(LBM_ERR_ORDER, "needs a completed lbm_forward");
    if ((st = enter(c)) != LBM_OK) return st;
    const int m = n + (n & 1);  // an even count keeps the buffer parity
    int& par = parity_of(c, phase);
    const int par0 = par;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < m && e == cudaSuccess; ++i) e = enqueue_step(c, phase, false, c->stream);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
    par = par0;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        (void)cudaGetLastError();
        return fail(LBM_ERR_CUDA, "time_steps capture failed");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(e);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(cudaGraphLaunch(exec, c->stream));  // untimed: first replay uploads the graph
    CUDA_TRY(cudaEventRecord(e0, c->stream));
    CUDA_TRY(cudaGraphLaunch(exec, c->stream));
    CUDA_TRY(cudaEventRecord(e1, c->stream));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(exec);
    *ms_per_step = (double)ms / m;
    return leave(c);
}

}  // extern "C"

// ===========================================================================
// batched solves (serving)
// ===========================================================================
namespace {

enum SlotPhase { SP_FLOW = 0, SP_THERM = 1, SP_ADJ = 2, SP_TADJ = 3, SP_DONE = 4 };

struct BatchEntry {
    lbm_ctx* ctx = nullptr;
    int phase = SP_DONE;
    long long steps = 0;     // steps in the current phase
    long long total = 0;     // steps over all phases
    double tol = 0, res = INFINITY;
    long long max_steps = 0;
    int status = LBM_OK;     // worst warning / first error
    double t0 = 0;
    bool used = false;
    bool solo = false;       // runs its own single-lattice graph (at or above the solo threshold)
};

}  // namespace

struct lbm_batch {
    int device = 0;
    int storage = 1;
    int K = 1000;
    int max_slots = 0;
    int grid = 0;
    long long solo_tiles = 0; // lattices with at least this many tiles run solo (0: never)
    cudaStream_t stream = nullptr;
    std::vector<char> h_bank;   // host image of the __constant__ argument bank
    int4* d_tiles[4] = {nullptr, nullptr, nullptr, nullptr};
    long long tile_cap[4] = {0, 0, 0, 0};
    int* d_lists = nullptr;  // resident slot ids
    int* d_counts = nullptr; // tile count, slot count
    double* d_results = nullptr;
    double* h_results = nullptr;
    std::vector<BatchEntry> e;
    std::vector<std::pair<int, lbm_report>> done;
    bool dirty = true;
    std::map<int, cudaGraphExec_t> graphs;
    size_t budget = 0;                 // device bytes the counted contexts may hold (0: no limit)
    std::map<lbm_ctx*, size_t> held;   // counted contexts and their footprints
    size_t held_bytes = 0;
};

namespace {

// the __constant__ bank of a storage type serves one live batch at a time
bool g_bank_busy[4] = {false, false, false, false};

void batch_forget(lbm_batch* b, lbm_ctx* c) {
    auto it = b->held.find(c);
    if (it != b->held.end()) {
        b->held_bytes -= it->second;
        b->held.erase(it);
    }
    c->holder = nullptr;
}

void batch_slot_refresh(lbm_batch* b, int i) {
    BatchEntry& en = b->e[i];
    lbm_ctx* c = en.ctx;
    FlowLaunch f = flow_base(c);
    f.out0 = c->rho;
    f.out1 = c->u;
    ThermLaunch t = therm_base(c);
    t.out0 = c->T;
    t.out1 = c->gpost;
    void* bufs[4][2] = {{c->f[0], c->f[1]}, {c->g[0], c->g[1]}, {c->fa[0], c->fa[1]}, {c->ga[0], c->ga[1]}};
    const int ph = en.phase;
    const int cur_fa = ph == SP_ADJ ? c->facur : c->fcur;
    const int cur_th = ph == SP_TADJ ? c->gacur : c->gcur;
    batch_fill_slot(b->storage, b->h_bank.data(), i, f, t, bufs, cur_fa, cur_th, ph,
                    (int)c->geom.grid.x, (int)c->geom.grid.y, (int)c->geom.block.x, (int)c->geom.block.y);
}

// rebuild the argument bank, the tile table and the slot list on the device
lbm_status batch_upload(lbm_batch* b) {
    std::vector<int4> tiles;
    std::vector<int> list;
    for (int i = 0; i < b->max_slots; ++i) {
        BatchEntry& en = b->e[i];
        if (!en.used || en.phase == SP_DONE || en.solo) continue;
        batch_slot_refresh(b, i);
        const Geom& g = en.ctx->geom;
        // the single-lattice launch's blocks, in its block-id order
        for (unsigned z = 0; z < g.grid.z; ++z)
            for (unsigned by = 0; by < g.grid.y; ++by)
                for (unsigned bx = 0; bx < g.grid.x; ++bx) {
                    const int bid = (int)(bx + g.grid.x * (by + g.grid.y * z));
                    tiles.push_back(make_int4(i | (int)(z << 8), (int)(bx * g.block.x),
                                              (int)(by * g.block.y), bid));
                }
        list.push_back(i);
    }
    int counts[2] = {(int)tiles.size(), (int)list.size()};
    if ((long long)tiles.size() > b->tile_cap[0]) {
        if (b->d_tiles[0]) CUDA_TRY(cudaFree(b->d_tiles[0]));
        b->d_tiles[0] = nullptr;
        long long cap = std::max<long long>(1024, (long long)tiles.size() * 2);
        CUDA_TRY(cudaMalloc(&b->d_tiles[0], sizeof(int4) * cap));
        b->tile_cap[0] = cap;
        for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);  // they hold the old table
        b->graphs.clear();
    }
    if (!tiles.empty())
        CUDA_TRY(cudaMemcpyAsync(b->d_tiles[0], tiles.data(), sizeof(int4) * tiles.size(),
                                 cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(batch_upload_bank(b->storage, b->h_bank.data(), b->stream));
    if (!list.empty())
        CUDA_TRY(cudaMemcpyAsync(b->d_lists, list.data(), sizeof(int) * list.size(),
                                 cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaMemcpyAsync(b->d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice, b->stream));
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    b->dirty = false;
    return LBM_OK;
}

// phases present among the packed (not solo) running entries
int batch_mask(lbm_batch* b) {
    int m = 0;
    for (int i = 0; i < b->max_slots; ++i)
        if (b->e[i].used && !b->e[i].solo && b->e[i].phase != SP_DONE) m |= 1 << b->e[i].phase;
    return m;
}

int slot_to_ctx_phase(int ph) {
    return ph == SP_FLOW ? PH_FLOW : (ph == SP_THERM ? PH_THERM : (ph == SP_ADJ ? PH_ADJ : PH_TADJ));
}

cudaError_t batch_enqueue(lbm_batch* b) {
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < b->K && e == cudaSuccess; ++s)
        e = batch_launch(b->storage, s == b->K - 1, b->d_tiles[0], b->d_counts, s, b->grid, b->stream);
    if (e == cudaSuccess)
        e = batch_finalize_launch(b->storage, b->d_lists, b->d_counts + 1, b->d_results, b->grid,
                                  b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_results, b->d_results, sizeof(double) * 2 * b->max_slots,
                            cudaMemcpyDeviceToHost, b->stream);
    return e;
}

// a context moves to its next phase (or finishes); kernels it needs run on its stream
lbm_status batch_advance(lbm_batch* b, int i, int st) {
    BatchEntry& en = b->e[i];
    lbm_ctx* c = en.ctx;
    if (st < 0) {
        en.status = st;
        en.phase = SP_DONE;
    } else {
        if (st > 0 && en.status == LBM_OK) en.status = st;
        if (en.phase == SP_FLOW) {
            c->flow_done = true;
            if (c->thermal) {
                lbm_status s2 = collide_initial_temperature(c);
                if (s2 != LBM_OK) return s2;
                en.phase = SP_THERM;
            } else {
                c->fwd_done = true;
                en.phase = SP_ADJ;
            }
        } else if (en.phase == SP_THERM) {
            c->fwd_done = true;
            en.phase = c->thermal ? SP_TADJ : SP_ADJ;
        } else if (en.phase == SP_TADJ) {
            lbm_status s2 = run_coupling(c);
            if (s2 != LBM_OK) return s2;
            c->tadj_done = true;
            en.phase = SP_ADJ;
        } else if (en.phase == SP_ADJ) {
            c->adj_done = true;
            c->astate = true;
            en.phase = SP_DONE;
        }
        if (en.phase == SP_ADJ || en.phase == SP_TADJ) {
            if (!c->astate) {
                lbm_status s2 = init_adjoint(c);
                if (s2 != LBM_OK) return s2;
                c->astate = true;
            }
        }
        en.steps = 0;
        en.res = INFINITY;
    }
    if (en.phase == SP_DONE) {
        if (en.status < 0) {
            if (c->fwd_done == false) c->fstate = false;
            else c->astate = false;
        }
        lbm_report r;
        r.steps = en.total;
        r.residual = en.res;
        r.I = c->last_I[PH_ADJ];
        r.J = c->J();
        r.ms = now_ms() - en.t0;
        r.status = en.status;
        b->done.push_back(std::make_pair(i, r));
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    b->dirty = true;
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_footprint_bytes(int stencil, int nx, int ny, int nz, int storage, int thermal) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || storage < 0 || storage > 3) return 0;
    const size_t N = (size_t)nx * ny * nz, np = (N + 63) / 64 * 64;
    const int Q = stencil == LBM_D2Q9 ? 9 : 19;
    const size_t pb = pop_bytes(storage), ab = adj_bytes(storage), rb = aux_bytes(storage),
                 hb = heat_bytes(storage);
    size_t bytes = 2 * np * Q * (pb + ab) + np * (1 + rb * (1 + 4 + 3 + 1 + 1));
    if (thermal) bytes += 2 * np * 7 * (hb + ab) + np * rb * (1 + 7 + 3 + 1 + 1);
    Geom g = make_geom(nx, ny, nz);
    bytes += sizeof(double) * 2 * (size_t)g.nblocks + 64;
    return bytes;
}

lbm_status lbm_batch_create(lbm_batch** out, int storage, int check_every, int max_slots,
                            size_t hbm_budget_bytes) {
    if (!out) return fail(LBM_ERR_ARG, "out is null");
    *out = nullptr;
    if (storage == LBM_FP64) return fail(LBM_ERR_UNSUPPORTED, "batches are built for FP32 arithmetic storage");
    if (storage < LBM_FP32 || storage > LBM_BF16_OFS) return fail(LBM_ERR_ARG, "unknown storage");
    if (check_every <= 0 || (check_every & 1)) return fail(LBM_ERR_ARG, "check_every must be positive and even");
    if (max_slots <= 0 || max_slots > batch_max_slots())
        return fail(LBM_ERR_ARG, "max_slots must be in [1, " + std::to_string(batch_max_slots()) + "]");
    if (g_bank_busy[storage])
        return fail(LBM_ERR_ARG, "a batch of this storage type is already live in this process");
    lbm_batch* b = new lbm_batch();
    cudaGetDevice(&b->device);
    b->storage = storage;
    b->K = check_every;
    b->max_slots = max_slots;
    b->budget = hbm_budget_bytes;
    b->h_bank.assign(batch_bank_bytes(storage), 0);
    b->e.resize(max_slots);
    g_bank_busy[storage] = true;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->grid = std::max(1, sms) * batch_blocks_per_sm(storage);
    // every lattice on its own graph and stream by default: measured faster
    // than the packed persistent launch for every mix tried (16 x 32^3: 62.5
    // against 35.8 GLUPS; 32 x 16^3: 18.0 against 16.0; mixed shapes: 43.3
    // against 34.6); lbm_batch_set_solo_tiles selects the packed launch
    b->solo_tiles = 1;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_lists, sizeof(int) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counts, sizeof(int) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_results, sizeof(double) * 2 * max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_results, sizeof(double) * 2 * max_slots);
    if (e == cudaSuccess) e = cudaMemset(b->d_counts, 0, sizeof(int) * 8);
    if (e != cudaSuccess) {
        lbm_batch_destroy(b);
        return fail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : b->held) kv.first->holder = nullptr;
    for (int ph = 0; ph < 4; ++ph)
        if (b->d_tiles[ph]) cudaFree(b->d_tiles[ph]);
    g_bank_busy[b->storage] = false;
    if (b->d_lists) cudaFree(b->d_lists);
    if (b->d_counts) cudaFree(b->d_counts);
    if (b->d_results) cudaFree(b->d_results);
    if (b->h_results) cudaFreeHost(b->h_results);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

lbm_status lbm_batch_admit(lbm_batch* b, lbm_ctx* c, const lbm_solve_opts* o, int* slot) {
    if (!b || !c || !o) return fail(LBM_ERR_ARG, "null argument");
    if (c->stencil != LBM_D3Q19) return fail(LBM_ERR_ARG, "batches hold D3Q19 contexts");
    if (c->storage != b->storage) return fail(LBM_ERR_ARG, "context storage differs from the batch's");
    if (o->max_steps < 0 || std::isnan(o->tol)) return fail(LBM_ERR_ARG, "bad opts");
    lbm_status st = ready(c);
    if (st != LBM_OK) return st;
    int i = -1;
    for (int k = 0; k < b->max_slots; ++k)
        if (!b->e[k].used) {
            i = k;
            break;
        }
    if (i < 0) return fail(LBM_ERR_ARG, "batch is full");
    if (c->holder && c->holder != b) return fail(LBM_ERR_ARG, "context is counted by another batch");
    size_t fp = 0;
    if (c->holder != b) {
        fp = lbm_footprint_bytes(c->stencil, c->nx, c->ny, c->nz, c->storage, c->thermal);
        if (b->budget > 0 && b->held_bytes + fp > b->budget)
            return fail(LBM_ERR_OOM, "context needs " + std::to_string(fp) + " bytes; the batch holds " +
                                         std::to_string(b->held_bytes) + " of its " +
                                         std::to_string(b->budget) + "-byte budget");
    }
    if ((st = enter(c)) != LBM_OK) return st;
    if (o->reset || !c->fstate) {
        if ((st = init_forward(c)) != LBM_OK) return st;
        c->fstate = true;
    }
    if (o->reset) c->astate = false;
    c->fwd_done = c->adj_done = false;
    c->flow_done = c->tadj_done = false;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->holder != b) {
        b->held[c] = fp;
        b->held_bytes += fp;
        c->holder = b;
    }
    BatchEntry& en = b->e[i];
    en = BatchEntry();
    en.ctx = c;
    en.used = true;
    en.phase = SP_FLOW;
    en.tol = o->tol;
    en.max_steps = o->max_steps;
    en.t0 = now_ms();
    en.solo = b->solo_tiles > 0 && c->geom.nblocks >= b->solo_tiles;
    b->dirty = true;
    if (slot) *slot = i;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int* n_active) {
    if (!b) return fail(LBM_ERR_ARG, "batch is null");
    NvtxRange range("lbm batch step");
    CUDA_TRY(cudaSetDevice(b->device));
    // contexts whose phase has nothing to do (max_steps reached) move on first
    for (int i = 0; i < b->max_slots; ++i) {
        BatchEntry& en = b->e[i];
        while (en.used && en.phase != SP_DONE && en.steps >= en.max_steps) {
            lbm_status st = batch_advance(b, i, en.tol > 0 ? LBM_NOT_CONVERGED : LBM_OK);
            if (st != LBM_OK) return st;
        }
    }
    if (b->dirty) {
        lbm_status st = batch_upload(b);
        if (st != LBM_OK) return st;
    }
    // solo entries: K steps of the context's own single-lattice graph on its
    // stream, running concurrently with the packed launch below
    bool any_solo = false;
    for (int i = 0; i < b->max_slots; ++i) {
        BatchEntry& en = b->e[i];
        if (!en.used || en.phase == SP_DONE || !en.solo) continue;
        lbm_status st = run_block(en.ctx, slot_to_ctx_phase(en.phase), b->K);
        if (st != LBM_OK) return st;
        any_solo = true;
    }
    const int mask = batch_mask(b);
    if (mask || any_solo) {
        const int key = 0;  // one graph: the tables it reads live in device memory
        auto it = b->graphs.find(key);
        if (mask && it == b->graphs.end()) {
            cudaGraph_t g = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = batch_enqueue(b);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                (void)cudaGetLastError();
                return fail(LBM_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
            }
            cudaGraphExec_t x = nullptr;
            cudaError_t e3 = cudaGraphInstantiate(&x, g, 0);
            cudaGraphDestroy(g);
            if (e3 != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e3));
            it = b->graphs.emplace(key, x).first;
        }
        if (mask) CUDA_TRY(cudaGraphLaunch(it->second, b->stream));
        CUDA_TRY(cudaStreamSynchronize(b->stream));
        for (int i = 0; i < b->max_slots; ++i) {
            BatchEntry& en = b->e[i];
            if (en.used && en.phase != SP_DONE && en.solo) CUDA_TRY(cudaStreamSynchronize(en.ctx->stream));
        }
        for (int i = 0; i < b->max_slots; ++i) {
            BatchEntry& en = b->e[i];
            if (!en.used || en.phase == SP_DONE) continue;
            lbm_ctx* c = en.ctx;
            const int ph = en.phase;
            // map the slot phase to the context's residual bookkeeping
            const int cph = slot_to_ctx_phase(ph);
            const double* r = en.solo ? c->hres : b->h_results + 2 * i;
            const double denom = (double)(c->n_nw > 0 ? c->n_nw : 1);
            const double cur = r[0] / denom;
            if (ph == SP_FLOW) c->J_p = c->n_in > 0 ? c->obj.w_pin * r[1] / (3.0 * (double)c->n_in) : 0.0;
            if (ph == SP_THERM) {
                c->J_T = c->obj.w_tmean * cur;
                c->J_Q = -c->obj.w_qgen * r[1];
            }
            en.steps += b->K;
            en.total += b->K;
            const bool bad = !std::isfinite(cur) || (ph <= SP_THERM && !std::isfinite(r[1]));
            if (bad) {
                c->last_I[cph] = cur;
                lbm_status st = batch_advance(b, i, LBM_ERR_DIVERGED);
                if (st != LBM_OK) return st;
                continue;
            }
            en.res = rel_change(cur, c->last_I[cph]);
            c->last_I[cph] = cur;
            lbm_status st = LBM_OK;
            if (en.tol > 0 && en.res < en.tol)
                st = batch_advance(b, i, LBM_OK);
            else if (en.steps >= en.max_steps)
                st = batch_advance(b, i, en.tol > 0 ? LBM_NOT_CONVERGED : LBM_OK);
            if (st != LBM_OK) return st;
        }
    }
    if (n_active) {
        int n = 0;
        for (int i = 0; i < b->max_slots; ++i) n += b->e[i].used && b->e[i].phase != SP_DONE;
        *n_active = n;
    }
    return LBM_OK;
}

lbm_status lbm_batch_release(lbm_batch* b, lbm_ctx* c) {
    if (!b || !c) return fail(LBM_ERR_ARG, "null argument");
    if (c->holder != b) return fail(LBM_ERR_ARG, "context is not counted by this batch");
    for (int i = 0; i < b->max_slots; ++i)
        if (b->e[i].used && b->e[i].ctx == c)
            return fail(LBM_ERR_ORDER, "context is still in the batch (running or not yet polled)");
    batch_forget(b, c);
    return LBM_OK;
}

lbm_status lbm_batch_memory(lbm_batch* b, size_t* budget, size_t* held) {
    if (!b) return fail(LBM_ERR_ARG, "batch is null");
    if (budget) *budget = b->budget;
    if (held) *held = b->held_bytes;
    return LBM_OK;
}

lbm_status lbm_batch_set_solo_tiles(lbm_batch* b, long long min_tiles) {
    if (!b) return fail(LBM_ERR_ARG, "batch is null");
    if (min_tiles < 0) return fail(LBM_ERR_ARG, "min_tiles < 0");
    b->solo_tiles = min_tiles;
    return LBM_OK;
}

lbm_status lbm_batch_poll(lbm_batch* b, int* slots, lbm_ctx** ctxs, lbm_report* reps, int max, int* n) {
    if (!b || !n) return fail(LBM_ERR_ARG, "null argument");
    int k = 0;
    while (!b->done.empty() && k < max) {
        auto pr = b->done.front();
        b->done.erase(b->done.begin());
        const int i = pr.first;
        if (slots) slots[k] = i;
        if (ctxs) ctxs[k] = b->e[i].ctx;
        if (reps) reps[k] = pr.second;
        b->e[i] = BatchEntry();
        ++k;
    }
    *n = k;
    return LBM_OK;
}

}  // extern "C"
