// lbm_device.cuh -- device-side lattice tables, population storage policies and
// the fused kernels of the forward / adjoint lattice Boltzmann sweeps.
//
// Memory layout (structure of arrays): population i of node n lives at
// p[i*np + n], n = x + nx*(y + ny*z), np = node count rounded up to a multiple
// of 64 so every population plane starts 256-byte aligned.  One thread owns one
// node; a block is a (BX x BY) tile of an x-y plane so that a warp reads 32
// consecutive x of one plane of one population (coalesced, with the +/-1 shift
// of the pull straddling at most one extra 32-byte sector).
//
// The flow kernels work on offset populations h_i = f_i - w_i rho0 in every
// storage type (rho - rho0 = sum h, rho0 u = sum e h), so no FP32 digits are
// spent on the constant w_i rho0; 16-bit storage holds the same h.
//
// Forward step (Eq. 35-37): pull f_S,i(x) = f_C,i(x - e_i) with periodic wrap,
// boundary operator B at the node, BGK collision with the design coupling
// u <- gamma u (Eq. 12) and store f_C.  Adjoint step (Eq. 53-56): pull
// f*_S,i(x) = f*_i(x + e_i) (Eq. 61), C^T in moment form (Eq. 65), objective
// source, closed-form B^T (Eq. 59-60 generalised), store f*.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

enum : int { FLUID = 0, WALL = 1, VEL = 2, PRES = 3 };
constexpr int HEAT_BIT = 0x40;

// ---------------------------------------------------------------------------
// lattices (Eq. 5); D2Q9 in the order Eq. 7-8 use
// ---------------------------------------------------------------------------
struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    // rest; +/-x, +/-y, +/-z; (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
    // (1,0,-1) (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

// temperature lattice: rest 1/4, six axis directions 1/8 (c_s^2 = 1/4)
struct D3Q7 {
    static constexpr int Q = 7;
    __host__ __device__ static constexpr int cx(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
};

// ---------------------------------------------------------------------------
// population storage: full precision, or 16-bit offsets from a reference
// ---------------------------------------------------------------------------
template <typename T> struct Pop;
template <> struct Pop<double> {
    using R = double;
    __device__ __forceinline__ static R ld(const double* __restrict__ p, long long k, R) { return __ldg(p + k); }
    __device__ __forceinline__ static void st(double* __restrict__ p, long long k, R v, R) { p[k] = v; }
    __device__ __forceinline__ static double enc(R v, R) { return v; }
};
template <> struct Pop<float> {
    using R = float;
    __device__ __forceinline__ static R ld(const float* __restrict__ p, long long k, R) { return __ldg(p + k); }
    __device__ __forceinline__ static void st(float* __restrict__ p, long long k, R v, R) { p[k] = v; }
    __device__ __forceinline__ static float enc(R v, R) { return v; }
};
template <> struct Pop<__half> {
    using R = float;
    __device__ __forceinline__ static R ld(const __half* __restrict__ p, long long k, R off) {
        return off + __half2float(__ldg(p + k));
    }
    __device__ __forceinline__ static void st(__half* __restrict__ p, long long k, R v, R off) {
        p[k] = __float2half_rn(v - off);
    }
    __device__ __forceinline__ static __half enc(R v, R off) { return __float2half_rn(v - off); }
};
template <> struct Pop<__nv_bfloat16> {
    using R = float;
    __device__ __forceinline__ static R ld(const __nv_bfloat16* __restrict__ p, long long k, R off) {
        return off + __bfloat162float(__ldg(p + k));
    }
    __device__ __forceinline__ static void st(__nv_bfloat16* __restrict__ p, long long k, R v, R off) {
        p[k] = __float2bfloat16_rn(v - off);
    }
    __device__ __forceinline__ static __nv_bfloat16 enc(R v, R off) { return __float2bfloat16_rn(v - off); }
};

// ---------------------------------------------------------------------------
// rounding-explicit arithmetic.  The node functions are inlined into several
// kernels (the single-lattice steps and the packed serving kernel).  Written
// with these operations, every multiply, add and fused multiply-add is fixed
// in the source: the compiler can neither fuse nor split them differently from
// one kernel to the next, so a node rounds identically wherever it runs.
// Coefficients that are lattice constants (components of e_i in {-1, 0, 1})
// enter through compile-time branches, so no multiply by 0 or 1 is executed.
// ---------------------------------------------------------------------------
template <typename R> struct Ex;
template <> struct Ex<float> {
    __device__ __forceinline__ static float add(float a, float b) { return __fadd_rn(a, b); }
    __device__ __forceinline__ static float sub(float a, float b) { return __fsub_rn(a, b); }
    __device__ __forceinline__ static float mul(float a, float b) { return __fmul_rn(a, b); }
    __device__ __forceinline__ static float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <> struct Ex<double> {
    __device__ __forceinline__ static double add(double a, double b) { return __dadd_rn(a, b); }
    __device__ __forceinline__ static double sub(double a, double b) { return __dsub_rn(a, b); }
    __device__ __forceinline__ static double mul(double a, double b) { return __dmul_rn(a, b); }
    __device__ __forceinline__ static double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// a + s b for a sign s in {-1, 0, 1} known at compile time (s = 0 gives a)
template <typename R>
__device__ __forceinline__ R add_s(R a, int s, R b) {
    return s > 0 ? Ex<R>::add(a, b) : (s < 0 ? Ex<R>::sub(a, b) : a);
}

// e.v for a direction e with components in {-1, 0, 1} known at compile time,
// summed x, y, z in that order
template <typename R>
__device__ __forceinline__ R edot(int x, int y, int z, R v0, R v1, R v2) {
    R r = R(0);
    bool any = false;
    if (x) { r = x > 0 ? v0 : -v0; any = true; }
    if (y) { r = any ? add_s(r, y, v1) : (y > 0 ? v1 : -v1); any = true; }
    if (z) { r = any ? add_s(r, z, v2) : (z > 0 ? v2 : -v2); }
    return r;
}

template <class L, typename R>
__device__ __forceinline__ R edot_i(int i, R v0, R v1, R v2) {
    return edot<R>(L::cx(i), L::cy(i), L::cz(i), v0, v1, v2);
}

// ---------------------------------------------------------------------------
// kernel arguments (passed by value)
// ---------------------------------------------------------------------------
template <typename T, typename TA, typename R>
struct FlowArgs {
    const T* __restrict__ fin;       // forward populations (read)
    T* __restrict__ fout;            // forward populations (write)
    const TA* __restrict__ ain;      // adjoint populations (read)
    TA* __restrict__ aout;           // adjoint populations (write)
    const uint8_t* __restrict__ flags;
    const R* __restrict__ gamma;
    const R* __restrict__ bc;        // 4 values per node
    const R* __restrict__ u;         // frozen velocity, 3 planes of np
    const R* __restrict__ cpl;       // thermal coupling v / rho0, 3 planes (or null)
    const R* __restrict__ sT;        // thermal part of dJ/dgamma (or null)
    R* __restrict__ out0;            // rho (reducing step, init) / dJ/dgamma (sens)
    R* __restrict__ out1;            // u, 3 planes (reducing step, init)
    double* __restrict__ partials;   // per-block sums (reductions)
    int nx, ny, nz;
    long long np;
    R omega;                         // 1/tau
    R rho0;
    R src_in;                        // w_pin / (3 N_in): -dJ/df_i at VEL nodes
    R ascale;                        // adjoint storage scale: 1 in every storage mode
                                     // (the adjoint is stored at full precision)
    int model;                       // 0 EQ12, 1 LINEAR
    int mirror;                      // bit a: axis a has symmetry planes beyond both faces
};

template <typename T, typename TA, typename R>
struct ThermArgs {
    const T* __restrict__ gin;
    T* __restrict__ gout;
    const TA* __restrict__ ain;
    TA* __restrict__ aout;
    const uint8_t* __restrict__ flags;
    const R* __restrict__ gamma;
    const R* __restrict__ bc;
    const R* __restrict__ u;         // frozen flow velocity, 3 planes
    const R* __restrict__ gpost;     // frozen post-boundary g, 7 planes
    R* __restrict__ gcn;             // adjoint g*_C of the outlet's unknown (PRES nodes)
    R* __restrict__ out0;            // T (reducing step, init) / v (coupling, 3 planes)
    R* __restrict__ out1;            // post-boundary g (reducing step, init, 7 planes) / sT (coupling)
    double* __restrict__ partials;
    int nx, ny, nz;
    long long np;
    R rho0, kappa_f, k_ratio, q, T0;
    R src_T;                         // w_tmean / N_nonwall
    R ascale;
    R beta;                          // beta_max: heat source Q = beta (1 - gamma)(1 - T) (Eq. 69)
    R src_q;                         // w_qgen beta_max: -dJ_Q/dg_l = -src_q (1 - gamma)
    int mirror;                      // bit a: axis a has symmetry planes beyond both faces
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
struct Cell {
    int x, y, z;
    long long n;
    bool active;
};

__device__ __forceinline__ Cell this_cell(int nx, int ny) {
    Cell c;
    c.x = blockIdx.x * blockDim.x + threadIdx.x;
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z;
    c.active = (c.x < nx) && (c.y < ny);
    c.n = c.x + (long long)nx * (c.y + (long long)ny * c.z);
    return c;
}

// offsets (in nodes) from a node to its six axis neighbours, periodic wrap
// included; they fit in 32 bits because node counts stay below 2^31.  A pull
// then costs one integer add per population instead of a wrapped 3-D index.
struct Nbr {
    int xm, xp, ym, yp, zm, zp;
};

__host__ __device__ __forceinline__ Nbr neighbours(const Cell& c, int nx, int ny, int nz) {
    const int sy = nx, sz = nx * ny;
    Nbr o;
    o.xm = c.x == 0 ? nx - 1 : -1;
    o.xp = c.x == nx - 1 ? 1 - nx : 1;
    o.ym = c.y == 0 ? (ny - 1) * sy : -sy;
    o.yp = c.y == ny - 1 ? (1 - ny) * sy : sy;
    o.zm = c.z == 0 ? (nz - 1) * sz : -sz;
    o.zp = c.z == nz - 1 ? (1 - nz) * sz : sz;
    return o;
}

// offset of x + s e_i (s = +1 or -1); the selections fold at compile time
template <class L>
__host__ __device__ __forceinline__ int nbr_offset(const Nbr& o, int i, int s) {
    const int dx = s * L::cx(i), dy = s * L::cy(i), dz = s * L::cz(i);
    return (dx < 0 ? o.xm : (dx > 0 ? o.xp : 0)) + (dy < 0 ? o.ym : (dy > 0 ? o.yp : 0)) +
           (dz < 0 ? o.zm : (dz > 0 ? o.zp : 0));
}

// Symmetry planes.  Along an axis with planes (bit a of `mirror`) the faces
// are not a periodic seam: a pull x + s e_i that leaves the box reads the
// image of that node in the plane (half a node beyond the face) and the
// population with that component of e_i reversed.  Only nodes on such a face
// take this path.
__host__ __device__ __forceinline__ bool on_mirror_face(const Cell& c, int nx, int ny, int nz, int mirror) {
    return ((mirror & 1) && (c.x == 0 || c.x == nx - 1)) || ((mirror & 2) && (c.y == 0 || c.y == ny - 1)) ||
           ((mirror & 4) && (c.z == 0 || c.z == nz - 1));
}

__host__ __device__ __forceinline__ int reflect_coord(int v, int n, bool plane, bool& flipped) {
    if (v < 0) {
        if (plane) { flipped = true; return -1 - v; }
        return v + n;
    }
    if (v >= n) {
        if (plane) { flipped = true; return 2 * n - 1 - v; }
        return v - n;
    }
    return v;
}

// element index (plane * np + node) of the pull x + s e_i at a node on a
// symmetry-plane face
template <class L>
__host__ __device__ __forceinline__ long long mirror_src(const Cell& c, int nx, int ny, int nz, long long np,
                                                         int mirror, int i, int s) {
    bool f0 = false, f1 = false, f2 = false;
    const int x = reflect_coord(c.x + s * L::cx(i), nx, mirror & 1, f0);
    const int y = reflect_coord(c.y + s * L::cy(i), ny, mirror & 2, f1);
    const int z = reflect_coord(c.z + s * L::cz(i), nz, mirror & 4, f2);
    const int e0 = f0 ? -L::cx(i) : L::cx(i), e1 = f1 ? -L::cy(i) : L::cy(i), e2 = f2 ? -L::cz(i) : L::cz(i);
    int j = i;
#pragma unroll
    for (int k = 0; k < L::Q; ++k)
        if (L::cx(k) == e0 && L::cy(k) == e1 && L::cz(k) == e2) j = k;
    return (long long)j * np + x + (long long)nx * (y + (long long)ny * z);
}

// Programmatic dependent launch (sm_90+): a step kernel lets the next step's
// grid be scheduled as soon as all of its own blocks are running, and waits
// for the previous grid (completion and memory visibility) before it touches
// any population or output buffer.  Outside a programmatic launch both are
// no-ops.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ long long grid_block_id() {
    return blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
}

// per-block FP64 partial sums of NV values (warp shuffles + shared memory),
// written to partials[b*NV + k]; ends with a barrier so the block may reuse
// the shared scratch for another tile
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], double* __restrict__ partials, long long b) {
    __shared__ double sh[NV][32];
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < nwarps ? sh[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) partials[b * NV + k] = s;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// forward boundary operator: Zou-He with an axis-aligned inward normal
//   unknowns U = {i : e_i.n > 0};  K0 = sum_{e.n=0} f, K- = sum_{e.n<0} f
//   VEL: u given.  PRES: u = n (rho_out - K0 - 2K-)/rho0 (Eq. 8, first line)
//   f_i = f_opp(i) + 6 w_i rho0 e_i.u - e_i.N,  N = S/2 - rho0 u_t / 3
//   with S = sum_{e.n=0} e f (Eq. 7-8 written for any face); applied to the
//   offset populations h (w_i = w_opp(i), sum_{e.n=0} e w = 0)
// ---------------------------------------------------------------------------
template <class L, typename R>
__device__ __forceinline__ void zou_he(R (&f)[L::Q], int type, int code, const R* __restrict__ bc, R rho0) {
    using X = Ex<R>;
    const int ax = code >> 1;
    const int sg = (code & 1) ? -1 : 1;
    const int n0 = ax == 0 ? sg : 0, n1 = ax == 1 ? sg : 0, n2 = ax == 2 ? sg : 0;
    R K0 = 0, Km = 0, S0 = 0, S1 = 0, S2 = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int d = L::cx(i) * n0 + L::cy(i) * n1 + L::cz(i) * n2;
        if (d == 0) {
            K0 = X::add(K0, f[i]);
            S0 = add_s(S0, L::cx(i), f[i]);
            S1 = add_s(S1, L::cy(i), f[i]);
            S2 = add_s(S2, L::cz(i), f[i]);
        } else if (d < 0) {
            Km = X::add(Km, f[i]);
        }
    }
    R u0, u1, u2;
    if (type == VEL) {
        u0 = bc[0];
        u1 = bc[1];
        u2 = bc[2];
    } else {
        // sums of offset populations: sum_{e.n=0} w + 2 sum_{e.n<0} w = 1
        const R un = X::fma(R(-2), Km, X::sub(X::sub(bc[0], rho0), K0)) / rho0;
        u0 = X::mul(un, R(n0));
        u1 = X::mul(un, R(n1));
        u2 = X::mul(un, R(n2));
    }
    const R unn = X::fma(u2, R(n2), X::fma(u1, R(n1), X::mul(u0, R(n0))));
    const R t0 = X::fma(-unn, R(n0), u0), t1 = X::fma(-unn, R(n1), u1), t2 = X::fma(-unn, R(n2), u2);
    const R k3 = X::mul(rho0, R(1) / R(3));
    const R N0 = X::fma(-k3, t0, X::mul(R(0.5), S0));
    const R N1 = X::fma(-k3, t1, X::mul(R(0.5), S1));
    const R N2 = X::fma(-k3, t2, X::mul(R(0.5), S2));
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int d = L::cx(i) * n0 + L::cy(i) * n1 + L::cz(i) * n2;
        if (d > 0) {
            const R eu = edot_i<L>(i, u0, u1, u2);
            const R eN = edot_i<L>(i, N0, N1, N2);
            f[i] = X::sub(X::fma(X::mul(R(6.0 * L::w(i)), rho0), eu, f[L::opp(i)]), eN);
        }
    }
}

// adjoint boundary operator f* = B^T f*_C for a Zou-He node:
//   unknown j           : 0
//   e_j.n < 0           : c_j + c_opp(j)              (- 2P at PRES)
//   e_j.n = 0           : c_j - e_j.M / 2              (-  P at PRES)
// with M = sum_{k in U} e_k c_k and P = sum_{k in U} 6 w_k c_k.  In D2Q9 this is
// Eq. 59 (left velocity inlet) and Eq. 60 (bottom fixed-density outlet).
template <class L, typename R>
__device__ __forceinline__ void zou_he_adjoint(R (&c)[L::Q], int type, int code) {
    using X = Ex<R>;
    const int ax = code >> 1;
    const int sg = (code & 1) ? -1 : 1;
    const int n0 = ax == 0 ? sg : 0, n1 = ax == 1 ? sg : 0, n2 = ax == 2 ? sg : 0;
    R M0 = 0, M1 = 0, M2 = 0, P = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int d = L::cx(i) * n0 + L::cy(i) * n1 + L::cz(i) * n2;
        if (d > 0) {
            M0 = add_s(M0, L::cx(i), c[i]);
            M1 = add_s(M1, L::cy(i), c[i]);
            M2 = add_s(M2, L::cz(i), c[i]);
            P = X::fma(R(6.0 * L::w(i)), c[i], P);
        }
    }
    if (type != PRES) P = R(0);
    // in place: the unknowns are read (through opp) before they are zeroed
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int d = L::cx(i) * n0 + L::cy(i) * n1 + L::cz(i) * n2;
        if (d < 0)
            c[i] = X::fma(R(-2), P, X::add(c[i], c[L::opp(i)]));
        else if (d == 0)
            c[i] = X::sub(X::fma(R(-0.5), edot_i<L>(i, M0, M1, M2), c[i]), P);
    }
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int d = L::cx(i) * n0 + L::cy(i) * n1 + L::cz(i) * n2;
        if (d > 0) c[i] = R(0);
    }
}

template <class L, typename R>
__device__ __forceinline__ void bounce(R (&f)[L::Q]) {
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if (L::opp(i) > i) {
            const R t = f[i];
            f[i] = f[L::opp(i)];
            f[L::opp(i)] = t;
        }
    }
}

// the boundary operator B at a node, on its post-stream populations
template <class L, typename T, typename TA, typename R>
__device__ __forceinline__ void apply_boundary(const FlowArgs<T, TA, R>& a, long long n, int fl, R (&f)[L::Q]) {
    const int type = fl & 7;
    if (type == WALL)
        bounce<L>(f);
    else if (type >= VEL)
        zou_he<L>(f, type, (fl >> 3) & 7, a.bc + 4 * n, a.rho0);
}

// pull the post-collision populations of the upstream neighbours and apply B
// (MIRROR: the lattice may have symmetry planes; without it that path is
// compiled out)
template <class L, bool MIRROR, typename T, typename TA, typename R>
__device__ __forceinline__ int pull_forward(const FlowArgs<T, TA, R>& a, const Cell& c, R (&f)[L::Q]) {
    if (MIRROR && a.mirror && on_mirror_face(c, a.nx, a.ny, a.nz, a.mirror)) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            f[i] = Pop<T>::ld(a.fin, mirror_src<L>(c, a.nx, a.ny, a.nz, a.np, a.mirror, i, -1), R(0));
    } else {
        const Nbr o = neighbours(c, a.nx, a.ny, a.nz);
        const T* __restrict__ p = a.fin + c.n;
#pragma unroll
        for (int i = 0; i < L::Q; ++i, p += a.np) f[i] = Pop<T>::ld(p, nbr_offset<L>(o, i, -1), R(0));
    }
    const int fl = a.flags[c.n];
    apply_boundary<L>(a, c.n, fl, f);
    return fl;
}

// component a (0 x, 1 y, 2 z) of e_i
template <class L>
__host__ __device__ constexpr int ecomp_of(int i, int a) {
    return a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i));
}

// the first direction of a (direction, opposite) pair with a nonzero
// component a, in the order the pairs are visited
template <class L>
__host__ __device__ constexpr int first_pair_on(int a) {
    for (int i = 1; i < L::Q; ++i)
        if (L::opp(i) > i && ecomp_of<L>(i, a) != 0) return i;
    return -1;
}

// drho = rho - rho0 = sum h, u = sum e h / rho0.  A direction and its
// opposite enter the density through their sum and the momentum through
// their difference, so each pair is read once and a component's first term
// is assigned rather than added to zero.
template <class L, typename R>
__device__ __forceinline__ void moments(const R (&f)[L::Q], R rho0, R& rho, R& u0, R& u1, R& u2) {
    using X = Ex<R>;
    R r = f[0], j0 = 0, j1 = 0, j2 = 0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if (L::opp(i) < i) continue;
        const int j = L::opp(i);
        const R sum = X::add(f[i], f[j]);
        const R dif = X::sub(f[i], f[j]);
        r = X::add(r, sum);
        if (L::cx(i)) j0 = i == first_pair_on<L>(0) ? (L::cx(i) > 0 ? dif : -dif) : add_s(j0, L::cx(i), dif);
        if (L::cy(i)) j1 = i == first_pair_on<L>(1) ? (L::cy(i) > 0 ? dif : -dif) : add_s(j1, L::cy(i), dif);
        if (L::cz(i)) j2 = i == first_pair_on<L>(2) ? (L::cz(i) > 0 ? dif : -dif) : add_s(j2, L::cz(i), dif);
    }
    const R inv = R(1) / rho0;
    rho = r;
    u0 = X::mul(j0, inv);
    u1 = X::mul(j1, inv);
    u2 = X::mul(j2, inv);
}

// ---------------------------------------------------------------------------
// forward kernels
// ---------------------------------------------------------------------------
// moments and BGK collision with the design coupling of one node's
// post-boundary populations (in place); the reducing variant also writes the
// node's fields and its residual / objective terms.  g is the node's gamma.
template <class L, typename T, typename TA, typename R, bool REDUCE>
__device__ __forceinline__ void flow_collide(const FlowArgs<T, TA, R>& a, long long n, int fl, R g,
                                             R (&f)[L::Q], double (&acc)[2]) {
    const int type = fl & 7;
    R drho, u0, u1, u2;
    moments<L>(f, a.rho0, drho, u0, u1, u2);
    using X = Ex<R>;
    if (REDUCE) {  // the fields and the frozen velocity of this post-boundary state
        a.out0[n] = X::add(a.rho0, drho);
        a.out1[n] = u0;
        a.out1[a.np + n] = u1;
        a.out1[2 * a.np + n] = u2;
    }
    if (type != WALL) {
        if (REDUCE) {
            acc[0] = (double)sqrt(X::fma(u2, u2, X::fma(u1, u1, X::mul(u0, u0))));
            if (type == VEL) acc[1] = (double)X::add(a.rho0, drho);
        }
        R a0, a1, a2, amp;
        if (a.model == 0) {
            a0 = X::mul(g, u0); a1 = X::mul(g, u1); a2 = X::mul(g, u2); amp = R(1);
        } else {
            a0 = u0; a1 = u1; a2 = u2; amp = g;
        }
        const R uu = X::fma(a2, a2, X::fma(a1, a1, X::mul(a0, a0)));
        const R om = a.omega, om1 = X::sub(R(1), om);
        // h_eq,i = w_i (drho + k (3 e_i.a + 4.5 (e_i.a)^2 - 1.5 a.a)), k = rho0 amp.
        // A direction and its opposite share the even part and negate the odd
        // one, so each pair is evaluated once; 1/tau is folded into w_i.
        const R k = X::mul(a.rho0, amp);
        const R ev = X::fma(-X::mul(R(1.5), k), uu, drho);
        const R k45 = X::mul(R(4.5), k), k3 = X::mul(R(3), k);
        f[0] = X::fma(om1, f[0], X::mul(X::mul(om, R(L::w(0))), ev));
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            if (L::opp(i) < i) continue;
            const int j = L::opp(i);
            const R omw = X::mul(om, R(L::w(i)));
            const R eu = edot_i<L>(i, a0, a1, a2);
            const R even = X::mul(omw, X::fma(X::mul(k45, eu), eu, ev));
            const R odd = X::mul(X::mul(omw, k3), eu);
            f[i] = X::fma(om1, f[i], X::add(even, odd));
            f[j] = X::fma(om1, f[j], X::sub(even, odd));
        }
        // The collision conserves mass: sum h = drho before and after.  With
        // the weights and products rounded, the updated populations sum to
        // drho plus a few ulps of a term in |u|^2 that has the same sign at
        // every moving node; over the lattice and the thousands of steps of a
        // steady solve that bias integrates into an offset of the whole
        // density level and a velocity error growing downstream (measured:
        // 1e-5 to 7e-5 relative in FP32).  The rest population takes the
        // remainder instead, so every node conserves its mass to one rounding.
        // With 16-bit storage the rounding of the stored values (unbiased,
        // 1e-3 relative) is far larger than that bias, so the step that is
        // bound by its instruction count keeps the plain update.
        if constexpr (sizeof(T) >= 4) {
            R moved = f[1];
#pragma unroll
            for (int i = 2; i < L::Q; ++i) moved = X::add(moved, f[i]);
            f[0] = X::sub(drho, moved);
        }
    }
}

template <class L, typename T, typename TA, typename R, bool REDUCE, bool MIRROR = true>
__device__ __forceinline__ void flow_step_node(const FlowArgs<T, TA, R>& a, const Cell& c, double (&acc)[2]) {
    R f[L::Q];
    const int fl = pull_forward<L, MIRROR>(a, c, f);
    const R g = (fl & 7) != WALL ? a.gamma[c.n] : R(0);
    flow_collide<L, T, TA, R, REDUCE>(a, c.n, fl, g, f, acc);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        Pop<T>::st(a.fout, (size_t)i * a.np + c.n, f[i], R(0));
}

// resident 256-thread blocks per SM asked of the compiler for the forward
// step: with 16-bit populations 6 (40 registers, a few spilled bytes) beat 5
// (48) by 4 % at 320^3, where the kernel is issue-bound; FP32 keeps 5 (48
// registers, no spills; 6 blocks, 40 registers and 20 spilled bytes, were
// 3 % slower at both 64^3 and 320^3)
template <class L, typename T>
struct FwdMinBlocks {
    static constexpr int value = L::Q != 19 ? 1 : (sizeof(T) == 2 ? 6 : (sizeof(T) == 4 ? 5 : 1));
};

template <class L, typename T, typename TA, typename R, bool REDUCE, bool MIRROR>
__global__ void __launch_bounds__(256, (FwdMinBlocks<L, T>::value)) k_flow_step(FlowArgs<T, TA, R> a) {
    pdl_launch_dependents();
    pdl_wait();
    const Cell c = this_cell(a.nx, a.ny);
    double acc[2] = {0.0, 0.0};
    if (c.active) flow_step_node<L, T, TA, R, REDUCE, MIRROR>(a, c, acc);
    if (REDUCE) block_partials<2>(acc, a.partials, grid_block_id());
}

// ---------------------------------------------------------------------------
// 16-bit storage, two x-adjacent nodes per thread.  The populations of a node
// pair (x0, x0 + 1), x0 even, sit in one aligned 32-bit word of each plane, so
// a pull is one 32-bit load per direction when e_x = 0; when e_x = +1 (-1) the
// pair pulled is (x0 - 1, x0) ((x0 + 1, x0 + 2)): the two aligned words around
// it are loaded and one byte permute takes out the middle.  Each node then
// runs the same boundary and collision code as the one-node kernels (so its
// populations are bit-identical to theirs) and the results are stored as one
// packed word per plane (one round-to-nearest-even pair conversion).  Needs an
// even nx (every pair starts on an even node index); the reducing step keeps
// the one-node kernel, so the per-block sums are those of every other path.
// ---------------------------------------------------------------------------
template <typename T> struct Pair16;
template <> struct Pair16<__half> {
    __device__ __forceinline__ static void unpack(uint32_t w, float& lo, float& hi) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&w));
        lo = v.x;
        hi = v.y;
    }
    __device__ __forceinline__ static uint32_t pack(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};
template <> struct Pair16<__nv_bfloat16> {
    __device__ __forceinline__ static void unpack(uint32_t w, float& lo, float& hi) {
        lo = __uint_as_float(w << 16);          // a bf16 is the high half of an f32
        hi = __uint_as_float(w & 0xffff0000u);
    }
    __device__ __forceinline__ static uint32_t pack(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};

// block size and resident blocks per SM of the paired step (64 registers,
// a few bytes spilled).  Measured at 320^3, where the kernel is issue-bound:
// 128 x 8 moved 0.872 of the HBM copy rate (FP16), 256 x 4 0.838, 64 x 16
// 0.798, 512 x 2 0.769; 256 x 3 (80 registers, no spill) was 3 % slower than
// 256 x 4
struct PairShape {
    static constexpr int threads = 128, blocks = 8;
};

template <class L, typename T, typename TA, typename R>
__global__ void __launch_bounds__(PairShape::threads, PairShape::blocks) k_flow_step_pair(FlowArgs<T, TA, R> a) {
    pdl_launch_dependents();
    pdl_wait();
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    Cell c;
    c.x = 2 * px;
    c.y = blockIdx.y * blockDim.y + threadIdx.y;
    c.z = blockIdx.z;
    if (c.x >= a.nx || c.y >= a.ny) return;  // no block-wide step follows
    c.n = c.x + (long long)a.nx * (c.y + (long long)a.ny * c.z);
    c.active = true;
    const Nbr o = neighbours(c, a.nx, a.ny, a.nz);
    const int xm2 = c.x == 0 ? a.nx - 2 : -2;           // the pair to the left, wrapped
    const int xp2 = c.x + 2 == a.nx ? 2 - a.nx : 2;     // the pair to the right, wrapped
    const uint32_t* __restrict__ p = reinterpret_cast<const uint32_t*>(a.fin + c.n);
    const long long pstride = a.np >> 1;                // words per plane
    uint32_t w[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i, p += pstride) {
        const int dy = -L::cy(i), dz = -L::cz(i);
        const int oyz = (dy < 0 ? o.ym : (dy > 0 ? o.yp : 0)) + (dz < 0 ? o.zm : (dz > 0 ? o.zp : 0));
        const uint32_t mid = __ldg(p + (oyz >> 1));
        if (L::cx(i) > 0) {
            w[i] = __byte_perm(__ldg(p + ((oyz + xm2) >> 1)), mid, 0x5432);
        } else if (L::cx(i) < 0) {
            w[i] = __byte_perm(mid, __ldg(p + ((oyz + xp2) >> 1)), 0x5432);
        } else {
            w[i] = mid;
        }
    }
    const uchar2 fl2 = *reinterpret_cast<const uchar2*>(a.flags + c.n);
    const float2 g2 = *reinterpret_cast<const float2*>(a.gamma + c.n);
    R fa[L::Q], fb[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) Pair16<T>::unpack(w[i], fa[i], fb[i]);
    double acc[2];
    apply_boundary<L>(a, c.n, fl2.x, fa);
    flow_collide<L, T, TA, R, false>(a, c.n, fl2.x, (fl2.x & 7) != WALL ? g2.x : R(0), fa, acc);
    apply_boundary<L>(a, c.n + 1, fl2.y, fb);
    flow_collide<L, T, TA, R, false>(a, c.n + 1, fl2.y, (fl2.y & 7) != WALL ? g2.y : R(0), fb, acc);
    uint32_t* __restrict__ q = reinterpret_cast<uint32_t*>(a.fout + c.n);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) q[(size_t)i * pstride] = Pair16<T>::pack(fa[i], fb[i]);
}

// f = f^eq(rho0, 0) = w rho0, i.e. h = 0 (collision leaves it unchanged); f* = 0
template <class L, typename T, typename TA, typename R>
__global__ void k_flow_init(FlowArgs<T, TA, R> a, int which) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= a.np) return;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        if (which == 0)
            a.fout[(size_t)i * a.np + n] = Pop<T>::enc(R(0), R(0));
        else
            a.aout[(size_t)i * a.np + n] = Pop<TA>::enc(R(0), R(0));
    }
    if (which == 0) {  // fields of the initial state f = f^eq(rho0, 0)
        a.out0[n] = a.rho0;
        a.out1[n] = R(0);
        a.out1[a.np + n] = R(0);
        a.out1[2 * a.np + n] = R(0);
    }
}

// ---------------------------------------------------------------------------
// adjoint kernels
// ---------------------------------------------------------------------------
// adjoint moments of f*_S: A = sum w f*, M = sum w f* e, Qm = sum w f* e e^T
template <class L, typename R>
struct AdjMoments {
    R A, M0, M1, M2, Q00, Q11, Q22, Q01, Q02, Q12;
    // a direction and its opposite enter A and Q through their sum and M
    // through their difference (e_opp = -e), so each pair is read once
    __device__ __forceinline__ void compute(const R (&s)[L::Q]) {
        using X = Ex<R>;
        M0 = M1 = M2 = Q00 = Q11 = Q22 = Q01 = Q02 = Q12 = R(0);
        A = X::mul(R(L::w(0)), s[0]);
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            if (L::opp(i) < i) continue;
            const int j = L::opp(i);
            const R wp = X::mul(R(L::w(i)), X::add(s[i], s[j]));
            const R wd = X::mul(R(L::w(i)), X::sub(s[i], s[j]));
            const int x = L::cx(i), y = L::cy(i), z = L::cz(i);
            A = X::add(A, wp);
            if (x) { M0 = add_s(M0, x, wd); Q00 = X::add(Q00, wp); }
            if (y) { M1 = add_s(M1, y, wd); Q11 = X::add(Q11, wp); }
            if (z) { M2 = add_s(M2, z, wd); Q22 = X::add(Q22, wp); }
            Q01 = add_s(Q01, x * y, wp);
            Q02 = add_s(Q02, x * z, wp);
            Q12 = add_s(Q12, y * z, wp);
        }
    }
};

template <class L, bool MIRROR, typename T, typename TA, typename R>
__device__ __forceinline__ void pull_adjoint(const FlowArgs<T, TA, R>& a, const Cell& c, R (&s)[L::Q]) {
    if (MIRROR && a.mirror && on_mirror_face(c, a.nx, a.ny, a.nz, a.mirror)) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            s[i] = Pop<TA>::ld(a.ain, mirror_src<L>(c, a.nx, a.ny, a.nz, a.np, a.mirror, i, +1), R(0)) * a.ascale;
        return;
    }
    const Nbr o = neighbours(c, a.nx, a.ny, a.nz);
    const TA* __restrict__ p = a.ain + c.n;
#pragma unroll
    for (int i = 0; i < L::Q; ++i, p += a.np) s[i] = Pop<TA>::ld(p, nbr_offset<L>(o, i, +1), R(0)) * a.ascale;
}

// resident 256-thread blocks per SM requested from the compiler: the plain
// FP32-math D3Q19 adjoint fits 40 registers without spilling (6 blocks, 75 %
// occupancy), its thermal-coupling variant 48 (5 blocks); the reducing
// variants (one step in K) keep the compiler's choice
template <class L, typename R, bool REDUCE, bool THERMAL>
struct AdjMinBlocks {
    static constexpr int value =
        (L::Q == 19 && sizeof(R) == 4 && !REDUCE) ? (THERMAL ? 5 : 6) : 1;
};

// THERMAL: the coupling field is present; CPL_RT: decide at run time from
// whether a coupling field is given (one code path for mixed batches)
// adjoint collision at a non-wall node, in place (Eq. 63-65): f*_C,i =
// (1 - 1/tau) f*_S,i + (1/tau) sum_m (d f^eq_m / d f_i) f*_S,m
// [- dJ/df_i = 1/(3 N_in) at an inlet node when src] [+ thermal coupling]
template <class L, typename T, typename TA, typename R, bool THERMAL, bool CPL_RT>
__device__ __forceinline__ void adjoint_collide(const FlowArgs<T, TA, R>& a, long long n, bool src, R (&s)[L::Q]) {
    using X = Ex<R>;
    const R g = a.gamma[n];
    const R u0 = a.u[n], u1 = a.u[a.np + n], u2 = a.u[2 * a.np + n];
    AdjMoments<L, R> m;
    m.compute(s);
    const R Qu0 = X::fma(m.Q02, u2, X::fma(m.Q01, u1, X::mul(m.Q00, u0)));
    const R Qu1 = X::fma(m.Q12, u2, X::fma(m.Q11, u1, X::mul(m.Q01, u0)));
    const R Qu2 = X::fma(m.Q22, u2, X::fma(m.Q12, u1, X::mul(m.Q02, u0)));
    // sum_m (d f^eq_m / d f_i) f*_m = A + e_i . w
    const R c1 = X::mul(R(3), g);
    const R c2 = a.model == 0 ? X::mul(X::mul(R(9), g), g) : X::mul(R(9), g);
    const R c3 = a.model == 0 ? X::mul(c1, g) : c1;
    const R c3A = X::mul(c3, m.A);
    R w0 = X::fma(-c3A, u0, X::fma(c2, Qu0, X::mul(c1, m.M0)));
    R w1 = X::fma(-c3A, u1, X::fma(c2, Qu1, X::mul(c1, m.M1)));
    R w2 = X::fma(-c3A, u2, X::fma(c2, Qu2, X::mul(c1, m.M2)));
    const R om = a.omega;
    R base = X::mul(om, m.A);
    if (src) base = X::sub(base, a.src_in);
    // the coupling term enters through the same fused operation whether
    // it is present or zero, so every kernel variant rounds alike
    R v0 = 0, v1 = 0, v2 = 0;
    if (THERMAL || (CPL_RT && a.cpl != nullptr)) {
        v0 = a.cpl[n];
        v1 = a.cpl[a.np + n];
        v2 = a.cpl[2 * a.np + n];
    }
    w0 = X::fma(om, w0, v0);
    w1 = X::fma(om, w1, v1);
    w2 = X::fma(om, w2, v2);
    const R om1 = X::sub(R(1), om);
    s[0] = X::fma(om1, s[0], base);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        if (L::opp(i) < i) continue;
        const int j = L::opp(i);
        const R ew = edot_i<L>(i, w0, w1, w2);
        s[i] = X::fma(om1, s[i], X::add(base, ew));
        s[j] = X::fma(om1, s[j], X::sub(base, ew));
    }
}

template <class L, typename T, typename TA, typename R, bool REDUCE, bool THERMAL, bool CPL_RT = false,
          bool MIRROR = true>
__device__ __forceinline__ void flow_adjoint_node(const FlowArgs<T, TA, R>& a, const Cell& c, double (&acc)[1]) {
    R s[L::Q];
    pull_adjoint<L, MIRROR>(a, c, s);
    const int fl = a.flags[c.n];
    const int type = fl & 7;
    if (type == WALL) {
        bounce<L>(s);  // C^T = I, B^T = the same swap
    } else {
        adjoint_collide<L, T, TA, R, THERMAL, CPL_RT>(a, c.n, type == VEL, s);
        if (type >= VEL) zou_he_adjoint<L>(s, type, (fl >> 3) & 7);
    }
    const R inv = R(1) / a.ascale;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) Pop<TA>::st(a.aout, (size_t)i * a.np + c.n, s[i] * inv, R(0));
    if (REDUCE && type != WALL) {
        R t = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) t = Ex<R>::add(t, fabs(s[i]));
        acc[0] = (double)t;
    }
}

template <class L, typename T, typename TA, typename R, bool REDUCE, bool THERMAL, bool MIRROR>
__global__ void __launch_bounds__(256, (AdjMinBlocks<L, R, REDUCE, THERMAL>::value))
    k_flow_adjoint(FlowArgs<T, TA, R> a) {
    pdl_launch_dependents();
    pdl_wait();
    const Cell c = this_cell(a.nx, a.ny);
    double acc[1] = {0.0};
    if (c.active) flow_adjoint_node<L, T, TA, R, REDUCE, THERMAL, false, MIRROR>(a, c, acc);
    if (REDUCE) block_partials<1>(acc, a.partials, grid_block_id());
}

// J'(x) = -(1/tau) sum_i f*_S,i d f^eq_i / d gamma (Eq. 66), + thermal part
template <class L, typename T, typename TA, typename R, bool THERMAL, bool MIRROR>
__global__ void __launch_bounds__(256) k_flow_sens(FlowArgs<T, TA, R> a) {
    const Cell c = this_cell(a.nx, a.ny);
    if (!c.active) return;
    const int type = a.flags[c.n] & 7;
    if (type == WALL) {
        a.out0[c.n] = R(0);
        return;
    }
    R s[L::Q];
    pull_adjoint<L, MIRROR>(a, c, s);
    const R g = a.gamma[c.n];
    const R u0 = a.u[c.n], u1 = a.u[a.np + c.n], u2 = a.u[2 * a.np + c.n];
    AdjMoments<L, R> m;
    m.compute(s);
    const R Mu = m.M0 * u0 + m.M1 * u1 + m.M2 * u2;
    const R uQu = m.Q00 * u0 * u0 + m.Q11 * u1 * u1 + m.Q22 * u2 * u2 +
                  R(2) * (m.Q01 * u0 * u1 + m.Q02 * u0 * u2 + m.Q12 * u1 * u2);
    const R uu = u0 * u0 + u1 * u1 + u2 * u2;
    R br;
    if (a.model == 0)
        br = R(3) * Mu + R(9) * g * uQu - R(3) * g * uu * m.A;
    else
        br = R(3) * Mu + R(4.5) * uQu - R(1.5) * uu * m.A;
    R out = -a.rho0 * a.omega * br;
    if (THERMAL) out += a.sT[c.n];
    a.out0[c.n] = out;
}

// ---------------------------------------------------------------------------
// the continuous adjoint LBM (Sec. 2.3), the comparison the paper draws:
// collide (C^T, no source), stream backwards, then the boundary rows derived
// from the continuous Lagrangian (Eq. 27 fixed-density outlet, Eq. 29
// velocity inlet, where the objective enters) and bounce-back at walls.  The
// kernels store c = C^T f* (the post-collision adjoint); a step pulls
// c(x + e_i), applies the boundary rows at the node (the result is f*, whose
// mean sum |f*| the residual uses) and collides.  At an open node with
// inward normal n the values with e_k.n < 0 came through the periodic wrap:
//   outlet: f*_k = f*_opp(k) - 12 sum_{e_i.n > 0} w_i f*_i
//   inlet:  f*_k = f*_opp(k) - 2 w_pin / (3 N_in)
// which is Eq. 27 (bottom outlet) and Eq. 29 (left inlet) on every face.
// ---------------------------------------------------------------------------
template <class L, typename R>
__device__ __forceinline__ void cont_boundary(R (&s)[L::Q], int fl, R s_in) {
    using X = Ex<R>;
    const int type = fl & 7;
    if (type == WALL) {
        bounce<L>(s);
        return;
    }
    if (type < VEL) return;
    const int code = (fl >> 3) & 7;
    const int ax = code >> 1;
    const int sg = (code & 1) ? -1 : 1;
    const int n0 = ax == 0 ? sg : 0, n1 = ax == 1 ? sg : 0, n2 = ax == 2 ? sg : 0;
    R sub = s_in;
    if (type == PRES) {
        sub = R(0);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            if (L::cx(i) * n0 + L::cy(i) * n1 + L::cz(i) * n2 > 0) sub = X::fma(R(12.0 * L::w(i)), s[i], sub);
    }
#pragma unroll
    for (int k = 0; k < L::Q; ++k)
        if (L::cx(k) * n0 + L::cy(k) * n1 + L::cz(k) * n2 < 0) s[k] = X::sub(s[L::opp(k)], sub);
}

template <class L, typename T, typename TA, typename R, bool REDUCE>
__global__ void __launch_bounds__(256) k_flow_adjoint_cont(FlowArgs<T, TA, R> a) {
    pdl_launch_dependents();
    pdl_wait();
    const Cell c = this_cell(a.nx, a.ny);
    double acc[1] = {0.0};
    if (c.active) {
        R s[L::Q];
        pull_adjoint<L, false>(a, c, s);
        const int fl = a.flags[c.n];
        const int type = fl & 7;
        cont_boundary<L>(s, fl, Ex<R>::mul(R(2), a.src_in));
        if (REDUCE && type != WALL) {
            R t = 0;
#pragma unroll
            for (int i = 0; i < L::Q; ++i) t = Ex<R>::add(t, fabs(s[i]));
            acc[0] = (double)t;
        }
        if (type != WALL) adjoint_collide<L, T, TA, R, false, false>(a, c.n, false, s);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) Pop<TA>::st(a.aout, (size_t)i * a.np + c.n, s[i], R(0));
    }
    if (REDUCE) block_partials<1>(acc, a.partials, grid_block_id());
}

// J'(x) = -(1/tau) sum_i f*_i d f^eq_i / d gamma with the continuous adjoint
// f* of the last step (Eq. 32 without lambda); zero at walls
template <class L, typename T, typename TA, typename R>
__global__ void __launch_bounds__(256) k_flow_sens_cont(FlowArgs<T, TA, R> a) {
    const Cell c = this_cell(a.nx, a.ny);
    if (!c.active) return;
    const int fl = a.flags[c.n];
    if ((fl & 7) == WALL) {
        a.out0[c.n] = R(0);
        return;
    }
    R s[L::Q];
    pull_adjoint<L, false>(a, c, s);
    cont_boundary<L>(s, fl, Ex<R>::mul(R(2), a.src_in));
    const R g = a.gamma[c.n];
    const R u0 = a.u[c.n], u1 = a.u[a.np + c.n], u2 = a.u[2 * a.np + c.n];
    AdjMoments<L, R> m;
    m.compute(s);
    const R Mu = m.M0 * u0 + m.M1 * u1 + m.M2 * u2;
    const R uQu = m.Q00 * u0 * u0 + m.Q11 * u1 * u1 + m.Q22 * u2 * u2 +
                  R(2) * (m.Q01 * u0 * u1 + m.Q02 * u0 * u2 + m.Q12 * u1 * u2);
    const R uu = u0 * u0 + u1 * u1 + u2 * u2;
    R br;
    if (a.model == 0)
        br = R(3) * Mu + R(9) * g * uQu - R(3) * g * uu * m.A;
    else
        br = R(3) * Mu + R(4.5) * uQu - R(1.5) * uu * m.A;
    a.out0[c.n] = -a.rho0 * a.omega * br;
}

// ---------------------------------------------------------------------------
// temperature lattice (D3Q7), velocity frozen from the converged flow
//   g^eq_k = w_k T (1 + 4 e_k.(gamma u)),  tau_g = 1/2 + 4 kappa_f (gamma + (1-gamma) k_r)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R tau_g(R g, R kappa_f, R k_ratio) {
    using X = Ex<R>;
    return X::fma(X::mul(R(4), kappa_f), X::fma(X::sub(R(1), g), k_ratio, g), R(0.5));
}

template <typename R>
__device__ __forceinline__ R ecomp(int k, R u0, R u1, R u2) {  // e_k . u for D3Q7
    return edot<R>(D3Q7::cx(k), D3Q7::cy(k), D3Q7::cz(k), u0, u1, u2);
}

// thermal boundary operator: wall bounce-back (+ heat flux), Dirichlet inlet,
// outflow setting the unknown to its equilibrium share of the node's own T
template <typename R>
__device__ __forceinline__ void thermal_bc(R (&g)[7], int fl, const R* __restrict__ bc, R gam,
                                           R u0, R u1, R u2, R q) {
    const int type = fl & 7;
    if (type == FLUID) return;
    const int kn = ((fl >> 3) & 7) + 1;  // D3Q7 index of the inward normal
    if (type == WALL) {
        bounce<D3Q7>(g);
        if (fl & HEAT_BIT) {
#pragma unroll
            for (int k = 1; k < 7; ++k)
                if (k == kn) g[k] = Ex<R>::add(g[k], q);
        }
        return;
    }
    using X = Ex<R>;
    R K = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k)
        if (k != kn) K = X::add(K, g[k]);
    R val;
    if (type == VEL || (fl & HEAT_BIT)) {  // inlet: T held at T_in (bit 6 on a PRES node:
        val = X::sub(bc[3], K);           // a pressure-driven inlet, Eq. 70)
    } else {
        R en = 0;
#pragma unroll
        for (int k = 1; k < 7; ++k)
            if (k == kn) en = ecomp<R>(k, u0, u1, u2);
        const R wa = X::mul(R(0.125), X::fma(X::mul(R(4), gam), en, R(1)));
        val = X::mul(wa, K) / X::sub(R(1), wa);
    }
#pragma unroll
    for (int k = 1; k < 7; ++k)
        if (k == kn) g[k] = val;
}

template <bool MIRROR, typename T, typename TA, typename R>
__device__ __forceinline__ int thermal_pull(const ThermArgs<T, TA, R>& a, const Cell& c, R (&g)[7],
                                            R& gam, R& u0, R& u1, R& u2) {
    if (MIRROR && a.mirror && on_mirror_face(c, a.nx, a.ny, a.nz, a.mirror)) {
#pragma unroll
        for (int k = 0; k < 7; ++k)
            g[k] = Pop<T>::ld(a.gin, mirror_src<D3Q7>(c, a.nx, a.ny, a.nz, a.np, a.mirror, k, -1),
                              R(D3Q7::w(k)) * a.T0);
    } else {
        const Nbr o = neighbours(c, a.nx, a.ny, a.nz);
        const T* __restrict__ p = a.gin + c.n;
#pragma unroll
        for (int k = 0; k < 7; ++k, p += a.np)
            g[k] = Pop<T>::ld(p, nbr_offset<D3Q7>(o, k, -1), R(D3Q7::w(k)) * a.T0);
    }
    const int fl = a.flags[c.n];
    gam = a.gamma[c.n];
    u0 = a.u[c.n];
    u1 = a.u[a.np + c.n];
    u2 = a.u[2 * a.np + c.n];
    thermal_bc<R>(g, fl, a.bc + 4 * c.n, gam, u0, u1, u2, a.q);
    return fl;
}

// temperature collision at a non-wall node with the heat source w_k Q,
// Q = beta_max (1 - gamma)(1 - T) (Eq. 69, 71), in place; returns Q
template <typename T, typename TA, typename R>
__device__ __forceinline__ R thermal_collide(const ThermArgs<T, TA, R>& a, R (&g)[7], R tem, R gam, R u0, R u1,
                                             R u2) {
    using X = Ex<R>;
    const R qs = X::mul(X::mul(a.beta, X::sub(R(1), gam)), X::sub(R(1), tem));
    const R om = R(1) / tau_g<R>(gam, a.kappa_f, a.k_ratio);
    const R g4 = X::mul(R(4), gam);
#pragma unroll
    for (int k = 1; k < 7; ++k) {
        const R geq = X::mul(X::mul(R(D3Q7::w(k)), tem), X::fma(g4, ecomp<R>(k, u0, u1, u2), R(1)));
        g[k] = X::fma(R(D3Q7::w(k)), qs, X::fma(om, X::sub(geq, g[k]), g[k]));
    }
    // the collision turns T into T + Q (sum g^eq = T): the rest population
    // takes the remainder, so the heat balance holds to one rounding at every
    // node (see the flow collision)
    R moved = g[1];
#pragma unroll
    for (int k = 2; k < 7; ++k) moved = X::add(moved, g[k]);
    g[0] = X::sub(X::add(tem, qs), moved);
    return qs;
}

// one temperature step at a node; the reducing step also sums T (residual,
// mean-T objective) and Q (heat-generation objective, Eq. 72) over non-wall
// nodes
template <typename T, typename TA, typename R, bool REDUCE, bool MIRROR = true>
__device__ __forceinline__ void thermal_step_node(const ThermArgs<T, TA, R>& a, const Cell& c, double (&acc)[2]) {
    R g[7], gam, u0, u1, u2;
    const int fl = thermal_pull<MIRROR>(a, c, g, gam, u0, u1, u2);
    using X = Ex<R>;
    R tem = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) tem = X::add(tem, g[k]);
    if (REDUCE) {  // temperature and frozen post-boundary g of this state
        a.out0[c.n] = tem;
#pragma unroll
        for (int k = 0; k < 7; ++k) a.out1[(size_t)k * a.np + c.n] = g[k];
    }
    if ((fl & 7) != WALL) {
        const R qs = thermal_collide(a, g, tem, gam, u0, u1, u2);
        if (REDUCE) {
            acc[0] = (double)tem;
            acc[1] = (double)qs;
        }
    }
#pragma unroll
    for (int k = 0; k < 7; ++k)
        Pop<T>::st(a.gout, (size_t)k * a.np + c.n, g[k], R(D3Q7::w(k)) * a.T0);
}

// The temperature lattice starts from g = w T0 (post-boundary state of step
// 0).  The kernels store post-collision populations, so before the first
// step that state is collided once, with the frozen flow: unlike the flow's
// rest equilibrium it is not a fixed point of the collision (advection
// term, heat source).
template <typename T, typename TA, typename R>
__global__ void __launch_bounds__(256) k_thermal_collide_initial(ThermArgs<T, TA, R> a) {
    const Cell c = this_cell(a.nx, a.ny);
    if (!c.active) return;
    const int fl = a.flags[c.n];
    if ((fl & 7) == WALL) return;  // no collision at walls: w T0 stays
    R g[7];
    using X = Ex<R>;
    R tem = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        g[k] = X::mul(R(D3Q7::w(k)), a.T0);
        tem = X::add(tem, g[k]);
    }
    thermal_collide(a, g, tem, a.gamma[c.n], a.u[c.n], a.u[a.np + c.n], a.u[2 * a.np + c.n]);
#pragma unroll
    for (int k = 0; k < 7; ++k)
        Pop<T>::st(a.gout, (size_t)k * a.np + c.n, g[k], R(D3Q7::w(k)) * a.T0);
}

template <typename T, typename TA, typename R, bool REDUCE, bool MIRROR>
__global__ void __launch_bounds__(256) k_thermal_step(ThermArgs<T, TA, R> a) {
    pdl_launch_dependents();
    pdl_wait();
    const Cell c = this_cell(a.nx, a.ny);
    double acc[2] = {0.0, 0.0};
    if (c.active) thermal_step_node<T, TA, R, REDUCE, MIRROR>(a, c, acc);
    if (REDUCE) block_partials<2>(acc, a.partials, grid_block_id());
}

template <typename T, typename TA, typename R>
__global__ void k_thermal_init(ThermArgs<T, TA, R> a, int which) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= a.np) return;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        if (which == 0)
            a.gout[(size_t)k * a.np + n] = Pop<T>::enc(R(D3Q7::w(k)) * a.T0, R(D3Q7::w(k)) * a.T0);
        else
            a.aout[(size_t)k * a.np + n] = Pop<TA>::enc(R(0), R(0));
    }
    if (which == 0) {
        a.out0[n] = a.T0;
#pragma unroll
        for (int k = 0; k < 7; ++k) a.out1[(size_t)k * a.np + n] = R(D3Q7::w(k)) * a.T0;
    } else {
        a.gcn[n] = R(0);
    }
}

// adjoint of the thermal collision at one node:
//   g*_C,l = (1 - 1/tau_g) g*_S,l + (1/tau_g) sum_k w_k a_k g*_S,k
//            - beta_max (1 - gamma) sum_k w_k g*_S,k - dJ/dg_l
// (the source w_k Q of Eq. 71 has dQ/dg_l = -beta_max (1 - gamma))
template <typename R>
__device__ __forceinline__ void thermal_adjoint_collide(R (&s)[7], R gam, R u0, R u1, R u2, R om, R src,
                                                        R beta) {
    using X = Ex<R>;
    R B = 0, W = 0;
    const R g4 = X::mul(R(4), gam);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        B = X::fma(X::mul(R(D3Q7::w(k)), X::fma(g4, ecomp<R>(k, u0, u1, u2), R(1))), s[k], B);
        W = X::fma(R(D3Q7::w(k)), s[k], W);
    }
    const R bg = X::mul(beta, X::sub(R(1), gam));
    const R base = X::fma(om, B, X::fma(-bg, W, -src));
    const R om1 = X::sub(R(1), om);
#pragma unroll
    for (int k = 0; k < 7; ++k) s[k] = X::fma(om1, s[k], base);
}

template <bool MIRROR, typename T, typename TA, typename R>
__device__ __forceinline__ void thermal_pull_adjoint(const ThermArgs<T, TA, R>& a, const Cell& c, R (&s)[7]) {
    if (MIRROR && a.mirror && on_mirror_face(c, a.nx, a.ny, a.nz, a.mirror)) {
#pragma unroll
        for (int k = 0; k < 7; ++k)
            s[k] = Pop<TA>::ld(a.ain, mirror_src<D3Q7>(c, a.nx, a.ny, a.nz, a.np, a.mirror, k, +1), R(0)) *
                   a.ascale;
        return;
    }
    const Nbr o = neighbours(c, a.nx, a.ny, a.nz);
    const TA* __restrict__ p = a.ain + c.n;
#pragma unroll
    for (int k = 0; k < 7; ++k, p += a.np) s[k] = Pop<TA>::ld(p, nbr_offset<D3Q7>(o, k, +1), R(0)) * a.ascale;
}

template <typename T, typename TA, typename R, bool REDUCE, bool MIRROR = true>
__device__ __forceinline__ void thermal_adjoint_node(const ThermArgs<T, TA, R>& a, const Cell& c, double (&acc)[1]) {
    R s[7];
    thermal_pull_adjoint<MIRROR>(a, c, s);
    const int fl = a.flags[c.n];
    const int type = fl & 7;
    if (type == WALL) {
        bounce<D3Q7>(s);
    } else {
        const R gam = a.gamma[c.n];
        const R u0 = a.u[c.n], u1 = a.u[a.np + c.n], u2 = a.u[2 * a.np + c.n];
        const R om = R(1) / tau_g<R>(gam, a.kappa_f, a.k_ratio);
        // -dJ/dg_l: mean-T objective and heat-generation objective (Eq. 72)
        const R src = Ex<R>::fma(a.src_q, Ex<R>::sub(R(1), gam), a.src_T);
        thermal_adjoint_collide<R>(s, gam, u0, u1, u2, om, src, a.beta);
        if (type >= VEL) {
            const int kn = ((fl >> 3) & 7) + 1;
            R ckn = 0, en = 0;
#pragma unroll
            for (int k = 1; k < 7; ++k)
                if (k == kn) {
                    ckn = s[k];
                    en = ecomp<R>(k, u0, u1, u2);
                }
            R coef;
            if (type == VEL || (fl & HEAT_BIT)) {
                coef = R(-1);
            } else {
                const R wa = Ex<R>::mul(R(0.125), Ex<R>::fma(Ex<R>::mul(R(4), gam), en, R(1)));
                coef = wa / Ex<R>::sub(R(1), wa);
                a.gcn[c.n] = ckn;
            }
#pragma unroll
            for (int k = 0; k < 7; ++k) s[k] = (k == kn) ? R(0) : Ex<R>::fma(coef, ckn, s[k]);
        }
    }
    const R inv = R(1) / a.ascale;
#pragma unroll
    for (int k = 0; k < 7; ++k) Pop<TA>::st(a.aout, (size_t)k * a.np + c.n, s[k] * inv, R(0));
    if (REDUCE && type != WALL) {
        R t = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) t = Ex<R>::add(t, fabs(s[k]));
        acc[0] = (double)t;
    }
}

template <typename T, typename TA, typename R, bool REDUCE, bool MIRROR>
__global__ void __launch_bounds__(256) k_thermal_adjoint(ThermArgs<T, TA, R> a) {
    pdl_launch_dependents();
    pdl_wait();
    const Cell c = this_cell(a.nx, a.ny);
    double acc[1] = {0.0};
    if (c.active) thermal_adjoint_node<T, TA, R, REDUCE, MIRROR>(a, c, acc);
    if (REDUCE) block_partials<1>(acc, a.partials, grid_block_id());
}

// thermal-to-flow coupling v/rho0 (added as e_i.v/rho0 to f*_C,i) and the
// thermal part of dJ/dgamma, from the current thermal adjoint iterate:
//   v   = (4 gamma T / tau_g) sum_k w_k g*_S,k e_k
//         + [outlet] g*_C,n w K/(1 - w a)^2 4 gamma e_n
//   s_T = -sum_k g*_S,k d g_C,k/d gamma - [outlet] g*_C,n w K/(1 - w a)^2 4 e_n.u
// The outlet terms linearise the boundary operator at the post-stream state of
// the stored temperature iterate (K = sum of its known post-stream
// populations), the same point as the collision terms.
template <typename T, typename TA, typename R, bool MIRROR>
__global__ void __launch_bounds__(256) k_thermal_coupling(ThermArgs<T, TA, R> a) {
    const Cell c = this_cell(a.nx, a.ny);
    if (!c.active) return;
    const int fl = a.flags[c.n];
    const int type = fl & 7;
    R v0 = 0, v1 = 0, v2 = 0, sT = 0;
    if (type != WALL) {
        R s[7];
        thermal_pull_adjoint<MIRROR>(a, c, s);
        const R gam = a.gamma[c.n];
        const R u0 = a.u[c.n], u1 = a.u[a.np + c.n], u2 = a.u[2 * a.np + c.n];
        R gp[7], tem = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            gp[k] = a.gpost[(size_t)k * a.np + c.n];
            tem += gp[k];
        }
        const R tg = tau_g<R>(gam, a.kappa_f, a.k_ratio);
        const R om = R(1) / tg;
        const R dom = -R(4) * a.kappa_f * (R(1) - a.k_ratio) * om * om;  // d(1/tau_g)/d gamma
        R Mg0 = 0, Mg1 = 0, Mg2 = 0, s1 = 0, W = 0;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const R ws = R(D3Q7::w(k)) * s[k];
            Mg0 += R(D3Q7::cx(k)) * ws;
            Mg1 += R(D3Q7::cy(k)) * ws;
            Mg2 += R(D3Q7::cz(k)) * ws;
            W += ws;
            const R eu = ecomp<R>(k, u0, u1, u2);
            const R geq = R(D3Q7::w(k)) * tem * (R(1) + R(4) * gam * eu);
            s1 += s[k] * (-(gp[k] - geq) * dom + om * R(D3Q7::w(k)) * tem * R(4) * eu);
        }
        const R cf = R(4) * gam * tem * om;
        v0 = cf * Mg0;
        v1 = cf * Mg1;
        v2 = cf * Mg2;
        // heat source: d(w_k Q)/d gamma = -w_k beta_max (1 - T); and the
        // direct part of J_Q = -w_qgen sum beta_max (1 - gamma)(1 - T)
        const R omT = R(1) - tem;
        sT = -s1 + a.beta * omT * W + a.src_q * omT;
        if (type == PRES && !(fl & HEAT_BIT)) {  // outflow node (not a temperature inlet)
            const int kn = ((fl >> 3) & 7) + 1;
            R en = 0;
#pragma unroll
            for (int k = 1; k < 7; ++k)
                if (k == kn) en = ecomp<R>(k, u0, u1, u2);
            const R wa = R(0.125) * (R(1) + R(4) * gam * en);
            R K = 0;
            const Nbr o = neighbours(c, a.nx, a.ny, a.nz);
            const bool mf = MIRROR && a.mirror && on_mirror_face(c, a.nx, a.ny, a.nz, a.mirror);
#pragma unroll
            for (int k = 0; k < 7; ++k) {
                if (k == kn) continue;
                K += mf ? Pop<T>::ld(a.gin, mirror_src<D3Q7>(c, a.nx, a.ny, a.nz, a.np, a.mirror, k, -1),
                                     R(D3Q7::w(k)) * a.T0)
                        : Pop<T>::ld(a.gin + (long long)k * a.np + c.n, nbr_offset<D3Q7>(o, k, -1),
                                     R(D3Q7::w(k)) * a.T0);
            }
            const R dgda = R(0.125) * K / ((R(1) - wa) * (R(1) - wa));
            const R ckn = a.gcn[c.n];
            const R cb = ckn * dgda * R(4) * gam;
            v0 += cb * R(D3Q7::cx(kn));
            v1 += cb * R(D3Q7::cy(kn));
            v2 += cb * R(D3Q7::cz(kn));
            sT -= ckn * dgda * R(4) * en;
        }
    }
    const R inv = R(1) / a.rho0;
    a.out0[c.n] = v0 * inv;
    a.out0[a.np + c.n] = v1 * inv;
    a.out0[2 * a.np + c.n] = v2 * inv;
    a.out1[c.n] = sT;
}

// ---------------------------------------------------------------------------
// batched (serving) kernels: one persistent launch walks the tiles of every
// resident lattice in a phase.  A tile is one block of that lattice's own
// single-lattice launch geometry (same threads, same warps), so each lattice's
// arithmetic and partial sums are bit-identical to its single-lattice solve,
// whatever else is resident.  Each lattice's argument blocks live in
// __constant__ memory, one per step parity (buffers swapped), so the node code
// reads its arguments from the constant cache exactly as the single-lattice
// kernels read theirs from the parameter bank.
// ---------------------------------------------------------------------------
constexpr int kBatchSlots = 32;

template <typename T, typename TG, typename TA, typename R>
struct BatchConst {
    FlowArgs<T, TA, R> f[kBatchSlots][2];   // [slot][parity]: flow and flow-adjoint buffers
    ThermArgs<TG, TA, R> t[kBatchSlots][2]; // [slot][parity]: temperature and its adjoint
    int4 geom[kBatchSlots];                 // log2(block x), block y, blocks (partials), unused
    int cur[kBatchSlots];                   // parity of step 0 of a graph block
    int phase[kBatchSlots];                 // 0 flow, 1 temperature, 2 flow adjoint, 3 temperature adjoint
};

// one persistent launch per step covers the tiles of every resident lattice,
// each tile dispatching on its lattice's phase (uniform within a block):
// 0 flow, 1 temperature, 2 flow adjoint, 3 temperature adjoint.  A tile entry
// is (slot | z << 8, x0, y0, block id), so no division is needed.  The next
// tile's entry is loaded before the current tile is computed, so a block never
// waits on the tile table between tiles.  Four 256-thread blocks per SM leave
// 64 registers a thread: the union of the four node functions and the tile
// loop does not fit the single kernels' 40-48 without spilling.
template <class L, typename T, typename TG, typename TA, typename R, bool REDUCE, class Bank>
__global__ void __launch_bounds__(256, 4)
    k_batch(const int4* __restrict__ tiles, const int* __restrict__ ntiles, int step) {
    const BatchConst<T, TG, TA, R>& C = Bank::get();
    pdl_launch_dependents();
    pdl_wait();
    const int nt = *ntiles;
    int4 next = blockIdx.x < nt ? tiles[blockIdx.x] : make_int4(0, 0, 0, 0);
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int4 tl = next;
        if (t + (int)gridDim.x < nt) next = tiles[t + gridDim.x];
        const int sl = tl.x & 0xff;
        const int par = (C.cur[sl] + step) & 1;
        const int4 g = C.geom[sl];
        const int P = C.phase[sl];
        Cell c;
        const int tid = threadIdx.x;
        c.x = tl.y + (tid & ((1 << g.x) - 1));
        c.y = tl.z + (tid >> g.x);
        c.z = tl.x >> 8;
        const bool in_tile = tid < (g.y << g.x);
        if (P == 0 || P == 2) {
            const FlowArgs<T, TA, R>& a = C.f[sl][par];
            c.active = in_tile && c.x < a.nx && c.y < a.ny;
            c.n = c.x + (long long)a.nx * (c.y + (long long)a.ny * c.z);
            if (P == 0) {
                double acc[2] = {0.0, 0.0};
                if (c.active) flow_step_node<L, T, TA, R, REDUCE>(a, c, acc);
                if (REDUCE) block_partials<2>(acc, a.partials, tl.w);
            } else {
                double acc[1] = {0.0};
                if (c.active) flow_adjoint_node<L, T, TA, R, REDUCE, false, true>(a, c, acc);
                if (REDUCE) block_partials<1>(acc, a.partials, tl.w);
            }
        } else {
            const ThermArgs<TG, TA, R>& a = C.t[sl][par];
            c.active = in_tile && c.x < a.nx && c.y < a.ny;
            c.n = c.x + (long long)a.nx * (c.y + (long long)a.ny * c.z);
            if (P == 1) {
                double acc[2] = {0.0, 0.0};
                if (c.active) thermal_step_node<TG, TA, R, REDUCE>(a, c, acc);
                if (REDUCE) block_partials<2>(acc, a.partials, tl.w);
            } else {
                double acc[1] = {0.0};
                if (c.active) thermal_adjoint_node<TG, TA, R, REDUCE>(a, c, acc);
                if (REDUCE) block_partials<1>(acc, a.partials, tl.w);
            }
        }
    }
}

// per-lattice second stage of the batched reductions: one block per listed
// slot sums that slot's partials in the same fixed order as k_finalize
template <int NV, typename T, typename TG, typename TA, typename R, class Bank>
__device__ __forceinline__ void batch_finalize_slot(const BatchConst<T, TG, TA, R>& C, int slot,
                                                    double* __restrict__ results) {
    __shared__ double sh[NV][8];
    {
        const double* __restrict__ partials = C.f[slot][0].partials;
        const long long nblocks = C.geom[slot].z;
        double s[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] = 0.0;
        for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
            for (int k = 0; k < NV; ++k) s[k] += partials[b * NV + k];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = s[k];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) sh[k][warp] = t;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double t = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
                for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
                if (lane == 0) results[2 * slot + k] = t;
            }
        }
        __syncthreads();
    }
}

// the flow and temperature phases sum two values, the adjoints one
template <typename T, typename TG, typename TA, typename R, class Bank>
__global__ void __launch_bounds__(256) k_batch_finalize(const int* __restrict__ list,
                                                        const int* __restrict__ nlist,
                                                        double* __restrict__ results) {
    const BatchConst<T, TG, TA, R>& C = Bank::get();
    const int n = *nlist;
    for (int q = blockIdx.x; q < n; q += gridDim.x) {
        const int slot = list[q];
        if (C.phase[slot] <= 1)  // flow: |u| and inlet rho; temperature: T and Q
            batch_finalize_slot<2, T, TG, TA, R, Bank>(C, slot, results);
        else
            batch_finalize_slot<1, T, TG, TA, R, Bank>(C, slot, results);
    }
}

// deterministic second stage of every reduction: one block sums the per-block
// partials in a fixed order
template <int NV>
__global__ void __launch_bounds__(256) k_finalize(const double* __restrict__ partials, long long nblocks,
                                                  double* __restrict__ out) {
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = 0.0;
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += partials[b * NV + k];
    __shared__ double sh[NV][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = s[k];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) sh[k][warp] = t;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < (int)(blockDim.x >> 5) ? sh[k][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) out[k] = t;
        }
    }
}

}  // namespace lbm
