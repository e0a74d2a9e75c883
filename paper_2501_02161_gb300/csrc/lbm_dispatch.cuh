// lbm_dispatch.cuh -- storage types, kernel-argument conversion and the
// per-(stencil, storage) launch switch.  Each storage type's kernels are
// instantiated in a translation unit of their own (lbm_storage_*.cu), so the
// library's kernels compile in parallel.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {
namespace dispatch {

// storage -> (population type, adjoint type, compute type)
template <int S> struct StorageTypes;
// T: flow populations, TG: temperature populations, TA: adjoint populations.
// The 16-bit modes narrow only the flow populations: the adjoint and the
// temperature lattice converge slowly (thousands of sweeps of a linear
// iteration), and 11- or 8-bit mantissas accumulate into percent-level errors
// there, so they stay FP32.
template <> struct StorageTypes<0> { using T = double; using TG = double; using TA = double; using R = double; };
template <> struct StorageTypes<1> { using T = float; using TG = float; using TA = float; using R = float; };
template <> struct StorageTypes<2> { using T = __half; using TG = float; using TA = float; using R = float; };
template <> struct StorageTypes<3> { using T = __nv_bfloat16; using TG = float; using TA = float; using R = float; };

template <int S>
FlowArgs<typename StorageTypes<S>::T, typename StorageTypes<S>::TA, typename StorageTypes<S>::R>
flow_args(const FlowLaunch& l) {
    using T = typename StorageTypes<S>::T;
    using TA = typename StorageTypes<S>::TA;
    using R = typename StorageTypes<S>::R;
    FlowArgs<T, TA, R> a;
    a.fin = (const T*)l.fin;
    a.fout = (T*)l.fout;
    a.ain = (const TA*)l.ain;
    a.aout = (TA*)l.aout;
    a.flags = l.flags;
    a.gamma = (const R*)l.gamma;
    a.bc = (const R*)l.bc;
    a.u = (const R*)l.u;
    a.cpl = (const R*)l.cpl;
    a.sT = (const R*)l.sT;
    a.out0 = (R*)l.out0;
    a.out1 = (R*)l.out1;
    a.partials = l.partials;
    a.nx = l.nx;
    a.ny = l.ny;
    a.nz = l.nz;
    a.np = l.np;
    a.omega = (R)l.omega;
    a.rho0 = (R)l.rho0;
    a.src_in = (R)l.src_in;
    a.ascale = (R)l.ascale;
    a.model = l.model;
    a.mirror = l.mirror;
    return a;
}

template <int S>
ThermArgs<typename StorageTypes<S>::TG, typename StorageTypes<S>::TA, typename StorageTypes<S>::R>
therm_args(const ThermLaunch& l) {
    using T = typename StorageTypes<S>::TG;
    using TA = typename StorageTypes<S>::TA;
    using R = typename StorageTypes<S>::R;
    ThermArgs<T, TA, R> a;
    a.gin = (const T*)l.gin;
    a.gout = (T*)l.gout;
    a.ain = (const TA*)l.ain;
    a.aout = (TA*)l.aout;
    a.flags = l.flags;
    a.gamma = (const R*)l.gamma;
    a.bc = (const R*)l.bc;
    a.u = (const R*)l.u;
    a.gpost = (const R*)l.gpost;
    a.gcn = (R*)l.gcn;
    a.out0 = (R*)l.out0;
    a.out1 = (R*)l.out1;
    a.partials = l.partials;
    a.nx = l.nx;
    a.ny = l.ny;
    a.nz = l.nz;
    a.np = l.np;
    a.rho0 = (R)l.rho0;
    a.kappa_f = (R)l.kappa_f;
    a.k_ratio = (R)l.k_ratio;
    a.q = (R)l.q;
    a.T0 = (R)l.T0;
    a.src_T = (R)l.src_T;
    a.ascale = (R)l.ascale;
    a.beta = (R)l.beta;
    a.src_q = (R)l.src_q;
    a.mirror = l.mirror;
    return a;
}

inline dim3 flat_grid(long long np) { return dim3((unsigned)((np + 255) / 256)); }

// launch a step kernel as a programmatic dependent of the previous kernel in
// the stream (the kernel waits for it with griddepcontrol.wait)
template <typename Arg>
void launch_pdl(void (*kernel)(Arg), const Geom& g, cudaStream_t s, const Arg& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = g.grid;
    cfg.blockDim = g.block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, a);
}

template <class L, int S, bool M>
void flow_dispatch_m(FlowOp op, const FlowLaunch& l, const Geom& g, cudaStream_t s) {
    using T = typename StorageTypes<S>::T;
    using TA = typename StorageTypes<S>::TA;
    using R = typename StorageTypes<S>::R;
    auto a = flow_args<S>(l);
    switch (op) {
        case FOP_INIT_F: k_flow_init<L, T, TA, R><<<flat_grid(l.np), 256, 0, s>>>(a, 0); break;
        case FOP_INIT_A: k_flow_init<L, T, TA, R><<<flat_grid(l.np), 256, 0, s>>>(a, 1); break;
        case FOP_STEP:
            // 16-bit populations with an even nx and no symmetry planes: two
            // nodes per thread
            if constexpr (sizeof(T) == 2 && L::Q == 19 && !M) {
                if ((l.nx % 2) == 0) {
                    launch_pdl(k_flow_step_pair<L, T, TA, R>,
                               make_geom(l.nx / 2, l.ny, l.nz, PairShape::threads), s, a);
                    break;
                }
            }
            launch_pdl(k_flow_step<L, T, TA, R, false, M>, g, s, a);
            break;
        case FOP_STEP_RED: launch_pdl(k_flow_step<L, T, TA, R, true, M>, g, s, a); break;
        case FOP_ADJ: launch_pdl(k_flow_adjoint<L, T, TA, R, false, false, M>, g, s, a); break;
        case FOP_ADJ_RED: launch_pdl(k_flow_adjoint<L, T, TA, R, true, false, M>, g, s, a); break;
        case FOP_ADJ_T: launch_pdl(k_flow_adjoint<L, T, TA, R, false, true, M>, g, s, a); break;
        case FOP_ADJ_T_RED: launch_pdl(k_flow_adjoint<L, T, TA, R, true, true, M>, g, s, a); break;
        case FOP_SENS: k_flow_sens<L, T, TA, R, false, M><<<g.grid, g.block, 0, s>>>(a); break;
        case FOP_SENS_T: k_flow_sens<L, T, TA, R, true, M><<<g.grid, g.block, 0, s>>>(a); break;
        case FOP_ADJ_CONT:
        case FOP_ADJ_CONT_RED:
        case FOP_SENS_CONT:
            // the continuous adjoint is built for D2Q9 without symmetry planes
            if constexpr (L::Q == 9 && !M) {
                if (op == FOP_ADJ_CONT)
                    launch_pdl(k_flow_adjoint_cont<L, T, TA, R, false>, g, s, a);
                else if (op == FOP_ADJ_CONT_RED)
                    launch_pdl(k_flow_adjoint_cont<L, T, TA, R, true>, g, s, a);
                else
                    k_flow_sens_cont<L, T, TA, R><<<g.grid, g.block, 0, s>>>(a);
            }
            break;
    }
}

// lattices with symmetry planes take the kernels that carry that path
template <class L, int S>
void flow_dispatch(FlowOp op, const FlowLaunch& l, const Geom& g, cudaStream_t s) {
    if (l.mirror)
        flow_dispatch_m<L, S, true>(op, l, g, s);
    else
        flow_dispatch_m<L, S, false>(op, l, g, s);
}

template <int S, bool M>
void therm_dispatch_m(ThermOp op, const ThermLaunch& l, const Geom& g, cudaStream_t s) {
    using T = typename StorageTypes<S>::TG;
    using TA = typename StorageTypes<S>::TA;
    using R = typename StorageTypes<S>::R;
    auto a = therm_args<S>(l);
    switch (op) {
        case TOP_INIT_G: k_thermal_init<T, TA, R><<<flat_grid(l.np), 256, 0, s>>>(a, 0); break;
        case TOP_INIT_A: k_thermal_init<T, TA, R><<<flat_grid(l.np), 256, 0, s>>>(a, 1); break;
        case TOP_STEP: launch_pdl(k_thermal_step<T, TA, R, false, M>, g, s, a); break;
        case TOP_STEP_RED: launch_pdl(k_thermal_step<T, TA, R, true, M>, g, s, a); break;
        case TOP_ADJ: launch_pdl(k_thermal_adjoint<T, TA, R, false, M>, g, s, a); break;
        case TOP_ADJ_RED: launch_pdl(k_thermal_adjoint<T, TA, R, true, M>, g, s, a); break;
        case TOP_COUPLING: k_thermal_coupling<T, TA, R, M><<<g.grid, g.block, 0, s>>>(a); break;
        case TOP_COLLIDE_INIT: k_thermal_collide_initial<T, TA, R><<<g.grid, g.block, 0, s>>>(a); break;
    }
}

template <int S>
void therm_dispatch(ThermOp op, const ThermLaunch& l, const Geom& g, cudaStream_t s) {
    if (l.mirror)
        therm_dispatch_m<S, true>(op, l, g, s);
    else
        therm_dispatch_m<S, false>(op, l, g, s);
}

}  // namespace dispatch

// one storage type's launches (defined in lbm_storage_*.cu)
template <int S>
cudaError_t flow_launch_storage(int stencil, FlowOp op, const FlowLaunch& a, const Geom& g, cudaStream_t s);
template <int S>
cudaError_t therm_launch_storage(ThermOp op, const ThermLaunch& a, const Geom& g, cudaStream_t s);

}  // namespace lbm
