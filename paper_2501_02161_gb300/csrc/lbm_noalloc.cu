// lbm_noalloc.cu -- lbm_flow_step_noalloc: one fused forward step with its
// reduction on caller-owned buffers, for callers that cannot allocate device
// memory.  The reduction scratch is a static device array of this file.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/lbmadj.h"
#include "lbm_internal.h"

namespace {

constexpr long long kMaxBlocks = 32768;  // 2 doubles per block: 512 KiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_scratch[2 * kMaxBlocks];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// device address of g_scratch on the current device, looked up once per device
cudaError_t scratch_address(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

lbm_status err(lbm_status s, const std::string& m) {
    return (lbm_status)lbm::set_error(s, m.c_str());
}

}  // namespace

extern "C" lbm_status lbm_flow_step_noalloc(const lbm_step_desc* d, void* stream) {
    if (!d) return err(LBM_ERR_ARG, "desc is null");
    if (d->stencil != LBM_D2Q9 && d->stencil != LBM_D3Q19) return err(LBM_ERR_ARG, "unknown stencil");
    if (d->storage < LBM_FP64 || d->storage > LBM_BF16_OFS) return err(LBM_ERR_ARG, "unknown storage");
    if (d->stencil == LBM_D2Q9 && d->storage > LBM_FP32)
        return err(LBM_ERR_UNSUPPORTED, "16-bit storage is built for D3Q19 only");
    if (d->nx <= 0 || d->ny <= 0 || d->nz <= 0) return err(LBM_ERR_ARG, "lattice sizes must be positive");
    if (d->stencil == LBM_D2Q9 && d->nz != 1) return err(LBM_ERR_ARG, "D2Q9 needs nz == 1");
    const long long N = (long long)d->nx * d->ny * d->nz;
    if (d->stride < N) return err(LBM_ERR_ARG, "stride < nx*ny*nz");
    if (!d->f_in || !d->f_out || !d->flags || !d->gamma || !d->bc || !d->rho || !d->u || !d->sums)
        return err(LBM_ERR_ARG, "null buffer in desc");
    if (d->f_in == d->f_out) return err(LBM_ERR_ARG, "f_out must not alias f_in");
    if (!(d->tau > 0.5) || !(d->rho0 > 0)) return err(LBM_ERR_ARG, "tau must be > 0.5 and rho0 > 0");
    if (d->gamma_model != LBM_GAMMA_EQ12 && d->gamma_model != LBM_GAMMA_LINEAR)
        return err(LBM_ERR_ARG, "unknown gamma model");
    lbm::Geom g = lbm::make_geom(d->nx, d->ny, d->nz);
    if (g.nblocks > kMaxBlocks)
        return err(LBM_ERR_ARG, "lattice needs " + std::to_string(g.nblocks) +
                                    " reduction blocks; the static scratch holds " +
                                    std::to_string(kMaxBlocks));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(LBM_ERR_ARG, "device ordinal out of range");
    double* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    lbm::FlowLaunch a = {};
    a.fin = d->f_in;
    a.fout = d->f_out;
    a.flags = d->flags;
    a.gamma = d->gamma;
    a.bc = d->bc;
    a.out0 = d->rho;
    a.out1 = d->u;
    a.partials = scratch;
    a.nx = d->nx;
    a.ny = d->ny;
    a.nz = d->nz;
    a.np = d->stride;
    a.omega = 1.0 / d->tau;
    a.rho0 = d->rho0;
    a.ascale = 1.0;
    a.model = d->gamma_model;
    cudaStream_t s = (cudaStream_t)stream;
    e = lbm::flow_launch(d->stencil, d->storage, lbm::FOP_STEP_RED, a, g, s);
    if (e == cudaSuccess) e = lbm::finalize_launch(scratch, g.nblocks, 2, d->sums, s);
    if (e != cudaSuccess) return err(LBM_ERR_CUDA, cudaGetErrorString(e));
    return LBM_OK;
}
