// lbm_internal.h -- type-erased launch interface between the C-ABI runtime
// and the templated kernels (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

struct Geom {
    dim3 grid;
    dim3 block;
    long long nblocks;  // grid.x * grid.y * grid.z (reduction partial count)
};

// (BX x BY) tiles of x-y planes, one thread per node, `threads` per block
// when the lattice is wide enough; BX divides nx when possible so no lane
// idles.
Geom make_geom(int nx, int ny, int nz, int threads = 256);

struct FlowLaunch {
    const void* fin;
    void* fout;
    const void* ain;
    void* aout;
    const uint8_t* flags;
    const void* gamma;
    const void* bc;
    const void* u;
    const void* cpl;
    const void* sT;
    void* out0;
    void* out1;
    double* partials;
    int nx, ny, nz;
    long long np;
    double omega, rho0, src_in, ascale;
    int model;
    int mirror;
};

struct ThermLaunch {
    const void* gin;
    void* gout;
    const void* ain;
    void* aout;
    const uint8_t* flags;
    const void* gamma;
    const void* bc;
    const void* u;
    const void* gpost;
    void* gcn;
    void* out0;
    void* out1;
    double* partials;
    int nx, ny, nz;
    long long np;
    double rho0, kappa_f, k_ratio, q, T0, src_T, ascale, beta, src_q;
    int mirror;
};

enum FlowOp {
    FOP_INIT_F = 0,
    FOP_INIT_A,
    FOP_STEP,
    FOP_STEP_RED,
    FOP_ADJ,
    FOP_ADJ_RED,
    FOP_ADJ_T,
    FOP_ADJ_T_RED,
    FOP_SENS,
    FOP_SENS_T,
    FOP_ADJ_CONT,      // continuous adjoint step (D2Q9 / D3Q19, no symmetry planes)
    FOP_ADJ_CONT_RED,
    FOP_SENS_CONT
};

enum ThermOp { TOP_INIT_G = 0, TOP_INIT_A, TOP_STEP, TOP_STEP_RED, TOP_ADJ, TOP_ADJ_RED, TOP_COUPLING,
               TOP_COLLIDE_INIT };

// storage codes follow lbm_storage; stencil codes follow lbm_stencil
cudaError_t flow_launch(int stencil, int storage, FlowOp op, const FlowLaunch& a, const Geom& g,
                        cudaStream_t s);
cudaError_t thermal_launch(int storage, ThermOp op, const ThermLaunch& a, const Geom& g,
                           cudaStream_t s);
// host run of the kernels' pull addressing over every node (stencil 0 D2Q9,
// 1 D3Q19, 2 D3Q7): the number of wrong or out-of-range sources
long long addressing_mismatches(int stencil, int nx, int ny, int nz);

cudaError_t finalize_launch(const double* partials, long long nblocks, int nv, double* out,
                            cudaStream_t s);
// element conversion between float/double buffers (device to device)
cudaError_t convert_launch(const void* src, int src_f64, void* dst, int dst_f64, long long n,
                           cudaStream_t s);

// batched (serving) kernels, D3Q19, storage 1-3: one launch per step over the
// tiles of all resident lattices (each in its own phase: 0 flow,
// 1 temperature, 2 flow adjoint, 3 temperature adjoint).  The lattices'
// arguments sit in a __constant__ bank per storage type, filled on the host.
size_t batch_bank_bytes(int storage);
int batch_max_slots();
int batch_blocks_per_sm(int storage);
void batch_fill_slot(int storage, void* bank, int slot, const FlowLaunch& f, const ThermLaunch& t,
                     void* const bufs[4][2], int cur_flow_or_adj, int cur_therm, int phase,
                     int gx, int gy, int bx, int by);
cudaError_t batch_upload_bank(int storage, const void* bank, cudaStream_t s);
cudaError_t batch_launch(int storage, bool reduce, const int4* tiles, const int* ntiles, int step,
                         int grid, cudaStream_t s);
cudaError_t batch_finalize_launch(int storage, const int* list, const int* nlist, double* results,
                                  int grid, cudaStream_t s);

// record an error message for lbm_last_error() and return the status
int set_error(int status, const char* msg);

// bytes per stored flow population / adjoint population / auxiliary value /
// temperature population
size_t pop_bytes(int storage);
size_t adj_bytes(int storage);
size_t aux_bytes(int storage);
size_t heat_bytes(int storage);

}  // namespace lbm
