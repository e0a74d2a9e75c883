// lbm_launch.cu -- template instantiation and dispatch of the kernels for each
// (stencil, storage) pair.
#include <algorithm>
#include <cstring>

#include "lbm_dispatch.cuh"

namespace lbm {

Geom make_geom(int nx, int ny, int nz, int threads) {
    Geom g;
    int bx = (nx % 128 == 0) ? 128 : ((nx % 64 == 0 || nx > 96) ? 64 : 32);
    if (bx > threads) bx = threads;
    int by = threads / bx;
    if (by > ny) by = ny;
    if (by < 1) by = 1;
    g.block = dim3(bx, by, 1);
    g.grid = dim3((nx + bx - 1) / bx, (ny + by - 1) / by, nz);
    g.nblocks = (long long)g.grid.x * g.grid.y * g.grid.z;
    return g;
}

namespace {

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (D)src[i];
}

}  // namespace

cudaError_t flow_launch(int stencil, int storage, FlowOp op, const FlowLaunch& a, const Geom& g,
                        cudaStream_t s) {
    if (stencil == 0 && storage > 1) return cudaErrorInvalidValue;
    switch (storage) {
        case 0: return flow_launch_storage<0>(stencil, op, a, g, s);
        case 1: return flow_launch_storage<1>(stencil, op, a, g, s);
        case 2: return flow_launch_storage<2>(stencil, op, a, g, s);
        case 3: return flow_launch_storage<3>(stencil, op, a, g, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t thermal_launch(int storage, ThermOp op, const ThermLaunch& a, const Geom& g,
                           cudaStream_t s) {
    switch (storage) {
        case 0: return therm_launch_storage<0>(op, a, g, s);
        case 1: return therm_launch_storage<1>(op, a, g, s);
        case 2: return therm_launch_storage<2>(op, a, g, s);
        case 3: return therm_launch_storage<3>(op, a, g, s);
        default: return cudaErrorInvalidValue;
    }
}

namespace {
// every (node, direction) pair: the source the kernels' offset arithmetic pulls
// from, against x - s e_i wrapped periodically by plain modular arithmetic
template <class L>
long long check_addressing(int nx, int ny, int nz) {
    long long bad = 0;
    const long long N = (long long)nx * ny * nz;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                Cell c;
                c.x = x;
                c.y = y;
                c.z = z;
                c.n = x + (long long)nx * (y + (long long)ny * z);
                c.active = true;
                const Nbr o = neighbours(c, nx, ny, nz);
                for (int i = 0; i < L::Q; ++i)
                    for (int sgn = -1; sgn <= 1; sgn += 2) {
                        const long long got = c.n + nbr_offset<L>(o, i, sgn);
                        const int xs = ((x + sgn * L::cx(i)) % nx + nx) % nx;
                        const int ys = ((y + sgn * L::cy(i)) % ny + ny) % ny;
                        const int zs = ((z + sgn * L::cz(i)) % nz + nz) % nz;
                        const long long want = xs + (long long)nx * (ys + (long long)ny * zs);
                        bad += (got != want || got < 0 || got >= N);
                    }
            }
    return bad;
}
}  // namespace

long long addressing_mismatches(int stencil, int nx, int ny, int nz) {
    if (stencil == 0) return check_addressing<D2Q9>(nx, ny, nz);
    if (stencil == 2) return check_addressing<D3Q7>(nx, ny, nz);
    return check_addressing<D3Q19>(nx, ny, nz);
}

cudaError_t finalize_launch(const double* partials, long long nblocks, int nv, double* out,
                            cudaStream_t s) {
    if (nv == 1)
        k_finalize<1><<<1, 256, 0, s>>>(partials, nblocks, out);
    else
        k_finalize<2><<<1, 256, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t convert_launch(const void* src, int src_f64, void* dst, int dst_f64, long long n,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n + 255) / 256));
    if (src_f64 && dst_f64)
        return cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s);
    if (!src_f64 && !dst_f64)
        return cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, s);
    if (src_f64)
        k_convert<double, float><<<grid, 256, 0, s>>>((const double*)src, (float*)dst, n);
    else
        k_convert<float, double><<<grid, 256, 0, s>>>((const float*)src, (double*)dst, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// batched (serving) kernels: D3Q19 with FP32 arithmetic (storage 1, 2, 3).
// One __constant__ bank per storage type holds the resident lattices'
// argument blocks; one batch per storage type may be live at a time.
// ---------------------------------------------------------------------------
namespace {
using dispatch::StorageTypes;
using dispatch::flow_args;
using dispatch::therm_args;

template <int S>
using BankT = BatchConst<typename StorageTypes<S>::T, typename StorageTypes<S>::TG,
                         typename StorageTypes<S>::TA, typename StorageTypes<S>::R>;

__constant__ BankT<1> c_bank1;
__constant__ BankT<2> c_bank2;
__constant__ BankT<3> c_bank3;

template <int S> struct Bank;
template <> struct Bank<1> { __device__ __forceinline__ static const BankT<1>& get() { return c_bank1; } };
template <> struct Bank<2> { __device__ __forceinline__ static const BankT<2>& get() { return c_bank2; } };
template <> struct Bank<3> { __device__ __forceinline__ static const BankT<3>& get() { return c_bank3; } };

template <typename... Args>
void launch_pdl_grid(void (*kernel)(Args...), int grid, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int S>
void batch_dispatch(bool reduce, const int4* tiles, const int* ntiles, int step, int grid,
                    cudaStream_t s) {
    using T = typename StorageTypes<S>::T;
    using TG = typename StorageTypes<S>::TG;
    using TA = typename StorageTypes<S>::TA;
    using R = typename StorageTypes<S>::R;
    if (reduce)
        launch_pdl_grid(k_batch<D3Q19, T, TG, TA, R, true, Bank<S>>, grid, s, tiles, ntiles, step);
    else
        launch_pdl_grid(k_batch<D3Q19, T, TG, TA, R, false, Bank<S>>, grid, s, tiles, ntiles, step);
}

template <int S>
void batch_finalize_dispatch(const int* list, const int* nlist, double* results, int grid,
                             cudaStream_t s) {
    using T = typename StorageTypes<S>::T;
    using TG = typename StorageTypes<S>::TG;
    using TA = typename StorageTypes<S>::TA;
    using R = typename StorageTypes<S>::R;
    k_batch_finalize<T, TG, TA, R, Bank<S>><<<grid, 256, 0, s>>>(list, nlist, results);
}

template <int S>
void fill(void* dst, int slot, const FlowLaunch& f, const ThermLaunch& t, void* const bufs[4][2],
          int cur_flow_or_adj, int cur_therm, int phase_flow, int phase_therm, int gx, int gy, int bx, int by) {
    BankT<S>* bank = (BankT<S>*)dst;
    for (int p = 0; p < 2; ++p) {
        FlowLaunch fl = f;
        ThermLaunch tl = t;
        const int pf = (cur_flow_or_adj + p) & 1, pt = (cur_therm + p) & 1;
        // the lattice's current phase decides which pair the parity swaps
        fl.fin = bufs[0][phase_flow == 0 ? pf : 0];
        fl.fout = bufs[0][phase_flow == 0 ? pf ^ 1 : 1];
        fl.ain = bufs[2][phase_flow == 2 ? pf : 0];
        fl.aout = bufs[2][phase_flow == 2 ? pf ^ 1 : 1];
        tl.gin = bufs[1][phase_therm == 1 ? pt : 0];
        tl.gout = bufs[1][phase_therm == 1 ? pt ^ 1 : 1];
        tl.ain = bufs[3][phase_therm == 3 ? pt : 0];
        tl.aout = bufs[3][phase_therm == 3 ? pt ^ 1 : 1];
        bank->f[slot][p] = flow_args<S>(fl);
        bank->t[slot][p] = therm_args<S>(tl);
    }
    int lg = 0;
    while ((1 << lg) < bx) ++lg;  // block widths are 32, 64 or 128
    bank->geom[slot] = make_int4(lg, by, gx * gy * f.nz, 0);
    bank->cur[slot] = 0;
    bank->phase[slot] = phase_flow >= 0 ? phase_flow : phase_therm;
}
}  // namespace

size_t batch_bank_bytes(int storage) {
    switch (storage) {
        case 1: return sizeof(BankT<1>);
        case 2: return sizeof(BankT<2>);
        case 3: return sizeof(BankT<3>);
        default: return 0;
    }
}

int batch_max_slots() { return kBatchSlots; }

void batch_fill_slot(int storage, void* bank, int slot, const FlowLaunch& f, const ThermLaunch& t,
                     void* const bufs[4][2], int cur_flow_or_adj, int cur_therm, int phase,
                     int gx, int gy, int bx, int by) {
    const int pf = (phase == 0 || phase == 2) ? phase : -1;
    const int pt = (phase == 1 || phase == 3) ? phase : -1;
    switch (storage) {
        case 1: fill<1>(bank, slot, f, t, bufs, cur_flow_or_adj, cur_therm, pf, pt, gx, gy, bx, by); break;
        case 2: fill<2>(bank, slot, f, t, bufs, cur_flow_or_adj, cur_therm, pf, pt, gx, gy, bx, by); break;
        case 3: fill<3>(bank, slot, f, t, bufs, cur_flow_or_adj, cur_therm, pf, pt, gx, gy, bx, by); break;
        default: break;
    }
}

cudaError_t batch_upload_bank(int storage, const void* bank, cudaStream_t s) {
    switch (storage) {
        case 1: return cudaMemcpyToSymbolAsync(c_bank1, bank, sizeof(BankT<1>), 0, cudaMemcpyHostToDevice, s);
        case 2: return cudaMemcpyToSymbolAsync(c_bank2, bank, sizeof(BankT<2>), 0, cudaMemcpyHostToDevice, s);
        case 3: return cudaMemcpyToSymbolAsync(c_bank3, bank, sizeof(BankT<3>), 0, cudaMemcpyHostToDevice, s);
        default: return cudaErrorInvalidValue;
    }
}

int batch_blocks_per_sm(int storage) {
    auto occ = [](const void* k) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, 256, 0);
        return n;
    };
    int m = 0;
    switch (storage) {
        case 1: {
            using T = StorageTypes<1>::T; using TG = StorageTypes<1>::TG; using TA = StorageTypes<1>::TA; using R = StorageTypes<1>::R;
            m = occ((const void*)k_batch<D3Q19, T, TG, TA, R, false, Bank<1>>);
            break;
        }
        case 2: {
            using T = StorageTypes<2>::T; using TG = StorageTypes<2>::TG; using TA = StorageTypes<2>::TA; using R = StorageTypes<2>::R;
            m = occ((const void*)k_batch<D3Q19, T, TG, TA, R, false, Bank<2>>);
            break;
        }
        case 3: {
            using T = StorageTypes<3>::T; using TG = StorageTypes<3>::TG; using TA = StorageTypes<3>::TA; using R = StorageTypes<3>::R;
            m = occ((const void*)k_batch<D3Q19, T, TG, TA, R, false, Bank<3>>);
            break;
        }
        default: break;
    }
    return m > 0 ? m : 4;
}

cudaError_t batch_launch(int storage, bool reduce, const int4* tiles, const int* ntiles, int step,
                         int grid, cudaStream_t s) {
    switch (storage) {
        case 1: batch_dispatch<1>(reduce, tiles, ntiles, step, grid, s); break;
        case 2: batch_dispatch<2>(reduce, tiles, ntiles, step, grid, s); break;
        case 3: batch_dispatch<3>(reduce, tiles, ntiles, step, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t batch_finalize_launch(int storage, const int* list, const int* nlist, double* results,
                                  int grid, cudaStream_t s) {
    switch (storage) {
        case 1: batch_finalize_dispatch<1>(list, nlist, results, grid, s); break;
        case 2: batch_finalize_dispatch<2>(list, nlist, results, grid, s); break;
        case 3: batch_finalize_dispatch<3>(list, nlist, results, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

size_t pop_bytes(int storage) { return storage == 0 ? 8 : (storage == 1 ? 4 : 2); }
size_t adj_bytes(int storage) { return storage == 0 ? 8 : 4; }
size_t heat_bytes(int storage) { return storage == 0 ? 8 : 4; }
size_t aux_bytes(int storage) { return storage == 0 ? 8 : 4; }

}  // namespace lbm
