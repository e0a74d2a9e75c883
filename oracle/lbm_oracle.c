/*
 * lbm_oracle.c -- plain FP64 CPU reference for the forward lattice Boltzmann
 * solve, its discrete adjoint and the sensitivity dJ/dgamma.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load or call this library.  It shares no
 * code, header, table or helper with the CUDA library; both take their inputs
 * from the seeded generators and nothing else.
 *
 * What it computes (paper section / equation in brackets):
 *   forward step      f_C = C[f], f_S = S f_C (periodic), f = B[f_S]    [Eq. 35-37]
 *   collision         BGK, incompressible equilibrium with u <- gamma u   [Eq. 2, 4, 12, 36]
 *   boundaries        Zou-He velocity inlet / fixed-density outlet in any
 *                     axis-aligned orientation, full-way bounce-back walls [Eq. 7-9]
 *   adjoint step      f* = B^T f*_C, f*_S = S^T f*, f*_C = C^T f*_S - dJ/df [Eq. 53-56]
 *                     with C and B built as explicit per-node Q x Q matrices [Eq. 57, 62-65]
 *   sensitivity       J'(x) = -f*_S^T dC/dgamma                            [Eq. 66, without lambda]
 *   thermal lattice   D3Q7 BGK with a gamma-interpolated relaxation time    [Eq. 71]
 *                     and its discrete adjoint, derived with the same recipe
 *                     (the paper's supplement that states them is absent).
 *   comparison        the continuous adjoint LBM the paper argues against:
 *                     C^T, reverse streaming, Eq. 27 / 29 boundaries     [Eq. 25-32]
 *
 * Layout: array of structures, f[n*Q + i], node n = x + nx*(y + ny*z).
 * Node flags follow the documented byte layout (type in bits 0-2, inward
 * normal code in bits 3-5, bit 6: a heated wall, or a fixed-density node that
 * holds the temperature at T_in, i.e. a pressure-driven inlet).  Faces of the
 * box are periodic seams or, per P->mirror, symmetry planes.
 *
 * Plain loops on purpose: no blocking, no fusion beyond the equations.  The
 * outer node loops carry an OpenMP pragma so the CPU baseline can use the
 * host cores; results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 19

/* ORC_MUTATION plants one deliberate mistake (tests/test_oracle_mutations.py
 * checks that the pins catch each); the normal build leaves it at 0. */
#ifndef ORC_MUTATION
#define ORC_MUTATION 0
#endif

enum { T_FLUID = 0, T_WALL = 1, T_VEL = 2, T_PRES = 3 };

typedef struct {
    int stencil;      /* 0 D2Q9, 1 D3Q19 */
    int nx, ny, nz;
    double tau, rho0;
    int gamma_model;  /* 0: u <- gamma u inside f^eq (Eq. 12); 1: linear in gamma */
    int thermal;
    double kappa_f, k_ratio, q_flux;
    double w_pin, w_tmean;
    /* heat generation (Eq. 69, 71-72): source Q = beta_max (1 - gamma)(1 - T)
     * added as w_k Q in the temperature collision; objective weight w_qgen
     * of J_Q = -sum_nonwall Q.  Both 0 switch the variant off. */
    double beta_max, w_qgen;
    /* symmetry planes: bit a makes both faces of axis a mirrors half a node
     * beyond the boundary layers instead of a periodic seam (a box cannot be
     * periodic along an axis with a plane on one side; a face that is not
     * meant as a plane carries walls or open boundaries, whose pulls from
     * outside the box are overwritten or never read) */
    int mirror;
} orc_problem;

typedef struct {
    int Q;
    int e[QMAX][3];
    double w[QMAX];
    int opp[QMAX];
} lattice;

/* D2Q9, Eq. 5 weights; index order as used by Eq. 7-8:
 * 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-). */
static void make_d2q9(lattice* L) {
    static const int e[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    L->Q = 9;
    for (int i = 0; i < 9; i++) {
        L->e[i][0] = e[i][0];
        L->e[i][1] = e[i][1];
        L->e[i][2] = 0;
        L->w[i] = (i == 0) ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
}

/* D3Q19, Eq. 5 weights.  Order: rest; the six axis directions as +/- pairs;
 * the twelve edge directions as +/- pairs. */
static void make_d3q19(lattice* L) {
    static const int e[19][3] = {
        {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
        {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
        {1, 0, -1}, {-1, 0, 1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    L->Q = 19;
    for (int i = 0; i < 19; i++) {
        for (int a = 0; a < 3; a++) L->e[i][a] = e[i][a];
        L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
}

/* D3Q7 for temperature: rest weight 1/4, axis weights 1/8, c_s^2 = 1/4. */
static void make_d3q7(lattice* L) {
    static const int e[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    L->Q = 7;
    for (int i = 0; i < 7; i++) {
        for (int a = 0; a < 3; a++) L->e[i][a] = e[i][a];
        L->w[i] = (i == 0) ? 0.25 : 0.125;
    }
}

static void finish_opp(lattice* L) {
    for (int i = 0; i < L->Q; i++)
        for (int j = 0; j < L->Q; j++)
            if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] &&
                L->e[j][2] == -L->e[i][2])
                L->opp[i] = j;
}

static void flow_lattice(const orc_problem* P, lattice* L) {
    if (P->stencil == 0) make_d2q9(L); else make_d3q19(L);
    finish_opp(L);
}

static void heat_lattice(lattice* L) {
    make_d3q7(L);
    finish_opp(L);
}

static int node_type(uint8_t fl) { return fl & 7; }

static void node_normal(uint8_t fl, int n[3]) {
    int code = (fl >> 3) & 7;
    n[0] = n[1] = n[2] = 0;
    n[code / 2] = (code % 2 == 0) ? 1 : -1;
}

static long nnodes(const orc_problem* P) { return (long)P->nx * P->ny * P->nz; }

/* flat index (node * Q + population) that streaming reads for population i
 * at node n: the node x + sgn e_i (sgn = -1: the forward pull of Eq. 37;
 * sgn = +1: the adjoint's reverse pull of Eq. 61), wrapped periodically,
 * except along an axis with symmetry planes: there the source is the image
 * of that node in the plane (half a node beyond the face) and the population
 * is e_i with that component reversed (specular reflection).  Streaming stays
 * a permutation, and the reverse pull is its transpose. */
static long stream_src(const orc_problem* P, const lattice* L, long n, int i, int sgn) {
    const long dim[3] = {P->nx, P->ny, P->nz};
    long c[3] = {n % P->nx, (n / P->nx) % P->ny, n / ((long)P->nx * P->ny)};
    int e[3] = {L->e[i][0], L->e[i][1], L->e[i][2]};
    for (int a = 0; a < 3; a++) {
        long v = c[a] + sgn * e[a];
        if (v < 0) {
            if (P->mirror & (1 << a)) {
                v = -1 - v;
                e[a] = ORC_MUTATION == 11 ? e[a] : -e[a];
            } else {
                v += dim[a];
            }
        } else if (v >= dim[a]) {
            if (P->mirror & (1 << a)) {
                v = 2 * dim[a] - 1 - v;
                e[a] = ORC_MUTATION == 11 ? e[a] : -e[a];
            } else {
                v -= dim[a];
            }
        }
        c[a] = v;
    }
    int j = 0;
    while (j < L->Q && !(L->e[j][0] == e[0] && L->e[j][1] == e[1] && L->e[j][2] == e[2])) j++;
    return (c[0] + (long)P->nx * (c[1] + (long)P->ny * c[2])) * L->Q + j;
}

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void evec(const lattice* L, int i, double v[3]) {
    for (int a = 0; a < 3; a++) v[a] = (double)L->e[i][a];
}

/* ---------------------------------------------------------------------- */
/* macroscopic moments, Eq. 6: rho = sum f, rho0 u = sum e f               */
/* ---------------------------------------------------------------------- */
static void moments(const lattice* L, const double* f, double rho0, double* rho, double u[3]) {
    double r = 0, m[3] = {0, 0, 0};
    for (int i = 0; i < L->Q; i++) {
        r += f[i];
        for (int a = 0; a < 3; a++) m[a] += L->e[i][a] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; a++) u[a] = m[a] / rho0;
}

/* equilibrium, Eq. 4 with the design coupling of Eq. 12 (model 0) or its
 * linear-in-gamma counterpart (model 1) */
static void equilibrium(const lattice* L, double rho, const double u[3], double gamma,
                        int model, double rho0, double* feq) {
    for (int i = 0; i < L->Q; i++) {
        double e[3];
        evec(L, i, e);
        if (model == 0) {
            double ua[3] = {gamma * u[0], gamma * u[1], gamma * u[2]};
            double eu = dot3(e, ua);
            feq[i] = L->w[i] * (rho + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * dot3(ua, ua)));
        } else {
            double eu = dot3(e, u);
            feq[i] = L->w[i] * (rho + gamma * rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * dot3(u, u)));
        }
    }
}

/* d f^eq_m / d f_i for all m, i: rho and u are linear in f (Eq. 6) */
static void equilibrium_jacobian(const lattice* L, const double u[3], double gamma, int model,
                                 double rho0, double J[QMAX][QMAX]) {
    for (int m = 0; m < L->Q; m++) {
        double em[3];
        evec(L, m, em);
        double emu = dot3(em, u);
        for (int i = 0; i < L->Q; i++) {
            double du[3];
            for (int a = 0; a < 3; a++) du[a] = L->e[i][a] / rho0; /* d u / d f_i */
            double drho = 1.0;                                     /* d rho / d f_i */
            double d;
            if (model == 0) {
                d = drho + rho0 * (3.0 * gamma * dot3(em, du) +
                                   9.0 * gamma * (ORC_MUTATION == 5 ? 1.0 : gamma) * emu * dot3(em, du) -
                                   3.0 * gamma * gamma * dot3(u, du));
            } else {
                d = drho + gamma * rho0 * (3.0 * dot3(em, du) + 9.0 * emu * dot3(em, du) -
                                           3.0 * dot3(u, du));
            }
            J[m][i] = L->w[m] * d;
        }
    }
}

/* d f^eq_i / d gamma (the bracket of Eq. 66 for model 1) */
static void equilibrium_dgamma(const lattice* L, const double u[3], double gamma, int model,
                               double rho0, double* out) {
    for (int i = 0; i < L->Q; i++) {
        double e[3];
        evec(L, i, e);
        double eu = dot3(e, u), uu = dot3(u, u);
        if (model == 0)
            out[i] = L->w[i] * rho0 * (3.0 * eu + 9.0 * gamma * eu * eu - 3.0 * gamma * uu);
        else
            out[i] = L->w[i] * rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* collision operator at one node, Eq. 36; wall nodes do not collide */
static void collide_node(const lattice* L, const orc_problem* P, uint8_t fl, double gamma,
                         const double* f, double* out) {
    if (node_type(fl) == T_WALL) {
        for (int i = 0; i < L->Q; i++) out[i] = f[i];
        return;
    }
    double rho, u[3], feq[QMAX];
    moments(L, f, P->rho0, &rho, u);
    equilibrium(L, rho, u, gamma, P->gamma_model, P->rho0, feq);
    for (int i = 0; i < L->Q; i++) out[i] = f[i] - (f[i] - feq[i]) / P->tau;
}

/* local collision Jacobian C_j, Eq. 63 */
static void collision_jacobian(const lattice* L, const orc_problem* P, uint8_t fl, double gamma,
                               const double* f, double C[QMAX][QMAX]) {
    for (int m = 0; m < L->Q; m++)
        for (int i = 0; i < L->Q; i++) C[m][i] = (m == i) ? 1.0 : 0.0;
    if (node_type(fl) == T_WALL) return;
    double rho, u[3], Jeq[QMAX][QMAX];
    moments(L, f, P->rho0, &rho, u);
    equilibrium_jacobian(L, u, gamma, P->gamma_model, P->rho0, Jeq);
    for (int m = 0; m < L->Q; m++)
        for (int i = 0; i < L->Q; i++)
            C[m][i] = ((m == i) ? 1.0 : 0.0) - (((m == i) ? 1.0 : 0.0) - Jeq[m][i]) / P->tau;
}

/* ---------------------------------------------------------------------- */
/* boundary operator B at one node                                          */
/* Zou-He in axis-aligned orientation with inward normal n:                 */
/*   unknowns are the populations with e_i.n > 0 (they arrive through the    */
/*   periodic wrap and are overwritten, Eq. 37 text);                        */
/*   rho = K0 + 2 K- + rho0 u.n            (Eq. 7 first line, Eq. 8 first)   */
/*   f_i = f_opp(i) + 6 w_i rho0 (e_i.u) - sum_t (e_i.t) N_t                  */
/*   N_t = 1/2 sum_{e_j.n=0} f_j (e_j.t) - 1/3 rho0 u.t                       */
/* which reproduces Eq. 7 (left inlet) and Eq. 8 (bottom outlet) in D2Q9.    */
/* A fixed-density node has u = u_n n with u_n from the density line.        */
/* Walls: full-way bounce-back, a symmetric index permutation (Eq. 9).      */
/* ---------------------------------------------------------------------- */
static void bc_node(const lattice* L, const orc_problem* P, uint8_t fl, const double* bcv,
                    const double* fs, double* out) {
    int t = node_type(fl);
    for (int i = 0; i < L->Q; i++) out[i] = fs[i];
    if (t == T_FLUID) return;
    if (t == T_WALL) {
        for (int i = 0; i < L->Q; i++) out[i] = fs[L->opp[i]];
        return;
    }
    int n[3];
    node_normal(fl, n);
    double K0 = 0, Km = 0;
    for (int i = 0; i < L->Q; i++) {
        int d = L->e[i][0] * n[0] + L->e[i][1] * n[1] + L->e[i][2] * n[2];
        if (d == 0) K0 += fs[i];
        if (d < 0) Km += fs[i];
    }
    double u[3];
    if (t == T_VEL) {
        u[0] = bcv[0]; u[1] = bcv[1]; u[2] = bcv[2];
    } else {
        double un = (bcv[0] - K0 - 2.0 * Km) / P->rho0;
        for (int a = 0; a < 3; a++) u[a] = un * n[a];
    }
    double N[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) {
        if (n[a] != 0) continue; /* tangential axes only */
        double s = 0;
        for (int j = 0; j < L->Q; j++) {
            int d = L->e[j][0] * n[0] + L->e[j][1] * n[1] + L->e[j][2] * n[2];
            if (d == 0) s += fs[j] * L->e[j][a];
        }
        N[a] = 0.5 * s - P->rho0 * u[a] / 3.0;
    }
    for (int i = 0; i < L->Q; i++) {
        int d = L->e[i][0] * n[0] + L->e[i][1] * n[1] + L->e[i][2] * n[2];
        if (d <= 0) continue;
        double e[3];
        evec(L, i, e);
        double v = fs[L->opp[i]] + 6.0 * L->w[i] * P->rho0 * dot3(e, u);
        for (int a = 0; a < 3; a++)
            if (n[a] == 0) v -= (ORC_MUTATION == 1 ? -1.0 : 1.0) * e[a] * N[a];
        out[i] = v;
    }
}

/* Jacobian of B at one node (B is affine, so this does not depend on f_S):
 * B[i][j] = d f_i / d f_S,j, written out from the same formulas. */
static void bc_jacobian(const lattice* L, const orc_problem* P, uint8_t fl,
                        double B[QMAX][QMAX]) {
    int t = node_type(fl);
    for (int i = 0; i < L->Q; i++)
        for (int j = 0; j < L->Q; j++) B[i][j] = 0.0;
    if (t == T_FLUID) {
        for (int i = 0; i < L->Q; i++) B[i][i] = 1.0;
        return;
    }
    if (t == T_WALL) {
        for (int i = 0; i < L->Q; i++) B[i][L->opp[i]] = 1.0;
        return;
    }
    int n[3];
    node_normal(fl, n);
    for (int i = 0; i < L->Q; i++) {
        int di = L->e[i][0] * n[0] + L->e[i][1] * n[1] + L->e[i][2] * n[2];
        if (di <= 0) {
            B[i][i] = 1.0;
            continue;
        }
        /* f_i = f_S,opp(i) + 6 w_i rho0 (e_i.u) - sum_t e_i,t N_t */
        B[i][L->opp[i]] += 1.0;
        for (int j = 0; j < L->Q; j++) {
            int dj = L->e[j][0] * n[0] + L->e[j][1] * n[1] + L->e[j][2] * n[2];
            /* dN_t / d f_S,j = 1/2 e_j,t for e_j.n = 0 (u.t is fixed or zero) */
            if (dj == 0)
                for (int a = 0; a < 3; a++)
                    if (n[a] == 0) B[i][j] -= L->e[i][a] * (ORC_MUTATION == 2 ? 1.0 : 0.5) * L->e[j][a];
            if (t == T_PRES) {
                /* e_i.u = u_n (e_i.n) with u_n = (rho_out - K0 - 2 K-)/rho0 */
                double dun = (dj == 0) ? -1.0 / P->rho0 : (dj < 0 ? -2.0 / P->rho0 : 0.0);
                B[i][j] += (ORC_MUTATION == 6 ? 3.0 : 6.0) * L->w[i] * P->rho0 * di * dun;
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* forward flow                                                             */
/* ---------------------------------------------------------------------- */
void orc_flow_init(const orc_problem* P, double* f) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    for (long n = 0; n < N; n++)
        for (int i = 0; i < L.Q; i++) f[n * L.Q + i] = L.w[i] * P->rho0;
}

/* one step f -> f_new: collision, periodic streaming, boundary operator */
void orc_flow_step(const orc_problem* P, const uint8_t* flags, const double* gamma,
                   const double* bcval, const double* f, double* fnew, double* work) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    int Q = L.Q;
    double* fc = work; /* N*Q */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) collide_node(&L, P, flags[n], gamma[n], f + n * Q, fc + n * Q);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double fs[QMAX];
        for (int i = 0; i < Q; i++) {
            fs[i] = fc[stream_src(P, &L, n, i, -1)];
        }
        bc_node(&L, P, flags[n], bcval + 4 * n, fs, fnew + n * Q);
    }
}

void orc_flow_run(const orc_problem* P, const uint8_t* flags, const double* gamma,
                  const double* bcval, double* f, long nsteps, double* work) {
    long N = nnodes(P);
    lattice L;
    flow_lattice(P, &L);
    double* tmp = (double*)malloc(sizeof(double) * N * L.Q);
    for (long s = 0; s < nsteps; s++) {
        orc_flow_step(P, flags, gamma, bcval, f, tmp, work);
        memcpy(f, tmp, sizeof(double) * N * L.Q);
    }
    free(tmp);
}

void orc_flow_macro(const orc_problem* P, const double* f, double* rho, double* u) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    for (long n = 0; n < N; n++) {
        double r, v[3];
        moments(&L, f + n * L.Q, P->rho0, &r, v);
        rho[n] = r;
        for (int a = 0; a < 3; a++) u[3 * n + a] = v[a];
    }
}

/* tangent of one step: dw -> B' S C' dw (B' and C' at the state f) */
void orc_flow_tangent(const orc_problem* P, const uint8_t* flags, const double* gamma,
                      const double* f, const double* dw, double* out) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    int Q = L.Q;
    double* dc = (double*)malloc(sizeof(double) * N * Q);
    for (long n = 0; n < N; n++) {
        double C[QMAX][QMAX];
        collision_jacobian(&L, P, flags[n], gamma[n], f + n * Q, C);
        for (int m = 0; m < Q; m++) {
            double s = 0;
            for (int i = 0; i < Q; i++) s += C[m][i] * dw[n * Q + i];
            dc[n * Q + m] = s;
        }
    }
    for (long n = 0; n < N; n++) {
        double ds[QMAX], B[QMAX][QMAX];
        for (int i = 0; i < Q; i++)
            ds[i] = dc[stream_src(P, &L, n, i, -1)];
        bc_jacobian(&L, P, flags[n], B);
        for (int i = 0; i < Q; i++) {
            double s = 0;
            for (int j = 0; j < Q; j++) s += B[i][j] * ds[j];
            out[n * Q + i] = s;
        }
    }
    free(dc);
}

/* ---------------------------------------------------------------------- */
/* discrete adjoint of the flow step, Eq. 53-56 / 59-61 / 64-65             */
/* ---------------------------------------------------------------------- */

/* f* = B^T f*_C at every node (Eq. 54) */
void orc_adjoint_bc(const orc_problem* P, const uint8_t* flags, const double* fsc, double* fs) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    int Q = L.Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double B[QMAX][QMAX];
        bc_jacobian(&L, P, flags[n], B);
        for (int j = 0; j < Q; j++) {
            double s = 0;
            for (int i = 0; i < Q; i++) s += B[i][j] * fsc[n * Q + i];
            fs[n * Q + j] = s;
        }
    }
}

/* f*_S = S^T f*: f*_S,i(x) = f*_i(x + e_i) (Eq. 61) */
static void adjoint_stream(const lattice* L, const orc_problem* P, const double* fs, double* fss) {
    long N = nnodes(P);
    int Q = L->Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++)
        for (int i = 0; i < Q; i++)
            fss[n * Q + i] = fs[stream_src(P, L, n, i, ORC_MUTATION == 4 ? -1 : 1)];
}

static long count_type(const orc_problem* P, const uint8_t* flags, int t) {
    long c = 0, N = nnodes(P);
    for (long n = 0; n < N; n++) c += node_type(flags[n]) == t;
    return c;
}

static long count_nonwall(const orc_problem* P, const uint8_t* flags) {
    return nnodes(P) - count_type(P, flags, T_WALL);
}

/* one adjoint iteration f*_C -> f*_C_new.
 * f is the converged forward state (post-B).  with_source adds -dJ/df of
 * the inlet-pressure objective (steady form of Eq. 34): 1/(3 N_in) per
 * population at each inlet node.  coupling (N*Q, may be NULL) is added as is
 * (thermal-to-flow term). */
void orc_flow_adjoint_step(const orc_problem* P, const uint8_t* flags, const double* gamma,
                           const double* f, const double* fsc, const double* coupling,
                           int with_source, double* fsc_new) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    int Q = L.Q;
    double* fs = (double*)malloc(sizeof(double) * N * Q);
    double* fss = (double*)malloc(sizeof(double) * N * Q);
    orc_adjoint_bc(P, flags, fsc, fs);
    adjoint_stream(&L, P, fs, fss);
    long nin = count_type(P, flags, T_VEL);
    double src = (nin > 0) ? P->w_pin / (3.0 * (double)nin) : 0.0;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double C[QMAX][QMAX];
        collision_jacobian(&L, P, flags[n], gamma[n], f + n * Q, C);
        for (int i = 0; i < Q; i++) {
            double s = 0;
            for (int m = 0; m < Q; m++) s += (ORC_MUTATION == 3 ? C[i][m] : C[m][i]) * fss[n * Q + m]; /* C^T */
            if (with_source && node_type(flags[n]) == T_VEL) s -= (ORC_MUTATION == 7 ? -src : src);
            if (coupling) s += coupling[n * Q + i];
            fsc_new[n * Q + i] = s;
        }
    }
    free(fs);
    free(fss);
}

void orc_flow_adjoint_run(const orc_problem* P, const uint8_t* flags, const double* gamma,
                          const double* f, double* fsc, const double* coupling, long nsteps) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    double* tmp = (double*)malloc(sizeof(double) * N * L.Q);
    for (long s = 0; s < nsteps; s++) {
        orc_flow_adjoint_step(P, flags, gamma, f, fsc, coupling, 1, tmp);
        memcpy(fsc, tmp, sizeof(double) * N * L.Q);
    }
    free(tmp);
}

/* J'(x) = -(1/tau) sum_i f*_S,i df^eq_i/dgamma (Eq. 66 without lambda);
 * f*_S = S^T B^T f*_C of the converged adjoint.  Zero at wall nodes. */
void orc_flow_sensitivity(const orc_problem* P, const uint8_t* flags, const double* gamma,
                          const double* f, const double* fsc, double* sens) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    int Q = L.Q;
    double* fs = (double*)malloc(sizeof(double) * N * Q);
    double* fss = (double*)malloc(sizeof(double) * N * Q);
    orc_adjoint_bc(P, flags, fsc, fs);
    adjoint_stream(&L, P, fs, fss);
    for (long n = 0; n < N; n++) {
        if (node_type(flags[n]) == T_WALL) {
            sens[n] = 0.0;
            continue;
        }
        double rho, u[3], dg[QMAX];
        moments(&L, f + n * Q, P->rho0, &rho, u);
        equilibrium_dgamma(&L, u, gamma[n], P->gamma_model, P->rho0, dg);
        double s = 0;
        for (int i = 0; i < Q; i++) s += fss[n * Q + i] * dg[i];
        sens[n] = -s / P->tau;
    }
    free(fs);
    free(fss);
}

/* ---------------------------------------------------------------------- */
/* continuous adjoint LBM (Sec. 2.3), kept as the comparison the paper makes */
/*   one iteration: adjoint collision C^T and reverse streaming (Eq. 30),     */
/*   then the boundary conditions derived from the continuous Lagrangian     */
/*   (Eq. 25-29) and bounce-back walls.  At an open node with inward normal  */
/*   n the reverse-streamed values f*_k with e_k.n < 0 came through the      */
/*   periodic wrap (they point out of the domain) and are the unknowns:      */
/*     fixed-density outlet (Eq. 27): f*_k = f*_opp(k) - K,                   */
/*        K = 12 sum_{e_i.n > 0} w_i f*_i                                     */
/*     velocity inlet (Eq. 29):       f*_k = f*_opp(k) - 2 w_pin / (3 N_in)   */
/*   This is Eq. 27 for the bottom outlet (unknowns 4, 7, 8; K = 4/3 f*_2 +   */
/*   1/3 f*_5 + 1/3 f*_6) and Eq. 29 for the left inlet (unknowns 3, 6, 7),   */
/*   each derived from the vanishing boundary term of Eq. 25 with the Zou-He */
/*   map of Eq. 7-8 substituted, which is why the same rule holds on every  */
/*   face.  The rows of Eq. 26 and 28 for the tangential populations cannot  */
/*   be satisfied (the inconsistency the paper points out) and are dropped,  */
/*   as in the paper.  The objective's 1/(3 W_in t_f) is read as            */
/*   w_pin / (3 N_in) for the steady objective.  D2Q9 only (the 3D forms are */
/*   in the paper's unavailable Supplementary A); returns -1 otherwise.      */
/* ---------------------------------------------------------------------- */
static int cont_geometry_ok(const orc_problem* P, const uint8_t* flags) {
    (void)flags;
    return P->stencil == 0;
}

/* the continuous adjoint boundary condition at one node, in place on its
 * reverse-streamed values t (s_in = 2 w_pin / (3 N_in)) */
static void cont_bc_node(const lattice* L, uint8_t fl, double s_in, double* t) {
    int ty = node_type(fl);
    if (ty == T_FLUID) return;
    if (ty == T_WALL) {
        for (int i = 1; i < L->Q; i++)
            if (L->opp[i] > i) {
                double x = t[i];
                t[i] = t[L->opp[i]];
                t[L->opp[i]] = x;
            }
        return;
    }
    int n[3];
    node_normal(fl, n);
    if (ORC_MUTATION == 10) { /* the printed bottom-outlet / left-inlet indices on every face */
        n[0] = ty == T_VEL ? 1 : 0;
        n[1] = ty == T_VEL ? 0 : 1;
        n[2] = 0;
    }
    double K = 0;
    if (ty == T_PRES)
        for (int i = 0; i < L->Q; i++)
            if (L->e[i][0] * n[0] + L->e[i][1] * n[1] + L->e[i][2] * n[2] > 0) K += 12.0 * L->w[i] * t[i];
    double sub = ty == T_PRES ? K : s_in;
    double old[QMAX];
    for (int i = 0; i < L->Q; i++) old[i] = t[i];
    for (int k = 0; k < L->Q; k++)
        if (L->e[k][0] * n[0] + L->e[k][1] * n[1] + L->e[k][2] * n[2] < 0) t[k] = old[L->opp[k]] - sub;
}

int orc_cont_adjoint_step(const orc_problem* P, const uint8_t* flags, const double* gamma,
                          const double* f, const double* fs, double* fs_new) {
    if (!cont_geometry_ok(P, flags)) return -1;
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    const int Q = 9;
    double* c = (double*)malloc(sizeof(double) * N * Q);
    for (long n = 0; n < N; n++) {
        if (node_type(flags[n]) == T_WALL) {
            for (int i = 0; i < Q; i++) c[n * Q + i] = fs[n * Q + i];
            continue;
        }
        double C[QMAX][QMAX];
        collision_jacobian(&L, P, flags[n], gamma[n], f + n * Q, C);
        for (int i = 0; i < Q; i++) {
            double v = 0;
            for (int m = 0; m < Q; m++) v += C[m][i] * fs[n * Q + m]; /* C^T */
            c[n * Q + i] = v;
        }
    }
    long nin = count_type(P, flags, T_VEL);
    double s_in = (nin > 0) ? 2.0 * P->w_pin / (3.0 * (double)nin) : 0.0;
    for (long n = 0; n < N; n++) {
        double t[9];
        for (int i = 0; i < Q; i++)
            t[i] = c[stream_src(P, &L, n, i, 1)]; /* reverse stream */
        cont_bc_node(&L, flags[n], s_in, t);
        for (int i = 0; i < Q; i++) fs_new[n * Q + i] = t[i];
    }
    free(c);
    return 0;
}

/* the continuous adjoint boundary condition of one node applied to given
 * reverse-streamed values (for the pins); D2Q9 only, returns -1 otherwise */
int orc_cont_node_bc(const orc_problem* P, uint8_t fl, double s_in, const double* t_in,
                     double* t_out) {
    if (P->stencil != 0) return -1;
    lattice L;
    flow_lattice(P, &L);
    for (int i = 0; i < L.Q; i++) t_out[i] = t_in[i];
    cont_bc_node(&L, fl, s_in, t_out);
    return 0;
}

/* J'(x) = -(1/tau) sum_i f*_i df^eq_i/dgamma (Eq. 32 without lambda) with the
 * converged continuous adjoint f*; zero at wall nodes */
void orc_cont_sensitivity(const orc_problem* P, const uint8_t* flags, const double* gamma,
                          const double* f, const double* fs, double* sens) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    int Q = L.Q;
    for (long n = 0; n < N; n++) {
        if (node_type(flags[n]) == T_WALL) {
            sens[n] = 0.0;
            continue;
        }
        double rho, u[3], dg[QMAX];
        moments(&L, f + n * Q, P->rho0, &rho, u);
        equilibrium_dgamma(&L, u, gamma[n], P->gamma_model, P->rho0, dg);
        double v = 0;
        for (int i = 0; i < Q; i++) v += fs[n * Q + i] * dg[i];
        sens[n] = -v / P->tau;
    }
}

/* ---------------------------------------------------------------------- */
/* thermal lattice (D3Q7), u frozen from the converged flow                 */
/*   g_C = g - (g - g^eq)/tau_g,  g^eq_k = w_k T (1 + 4 e_k.(gamma u))         */
/*   tau_g = 1/2 + 4 kappa(gamma), kappa = kappa_f (gamma + (1-gamma) k_r)     */
/*   boundaries: VEL node = Dirichlet T_in on the unknown population;          */
/*               PRES node = unknown set to its equilibrium share of the node's */
/*               own T; WALL = bounce-back, HEAT wall adds q towards its normal */
/* ---------------------------------------------------------------------- */
static double tau_g(const orc_problem* P, double gamma) {
    return 0.5 + 4.0 * P->kappa_f * (gamma + (1.0 - gamma) * P->k_ratio);
}

static double dtau_g(const orc_problem* P) { return 4.0 * P->kappa_f * (1.0 - P->k_ratio); }

static void flow_u(const lattice* LF, const orc_problem* P, const double* fnode, double u[3]) {
    double rho;
    moments(LF, fnode, P->rho0, &rho, u);
}

static int unknown_dir(const lattice* LG, const int n[3]) {
    for (int k = 0; k < LG->Q; k++)
        if (LG->e[k][0] == n[0] && LG->e[k][1] == n[1] && LG->e[k][2] == n[2]) return k;
    return -1;
}

static void thermal_collide_node(const lattice* LG, const orc_problem* P, uint8_t fl,
                                 double gamma, const double u[3], const double* g, double* out) {
    if (node_type(fl) == T_WALL) {
        for (int k = 0; k < LG->Q; k++) out[k] = g[k];
        return;
    }
    double T = 0;
    for (int k = 0; k < LG->Q; k++) T += g[k];
    double tg = tau_g(P, gamma);
    double Qsrc = P->beta_max * (1.0 - gamma) * (1.0 - T); /* Eq. 69 in Eq. 71 */
    for (int k = 0; k < LG->Q; k++) {
        double e[3];
        evec(LG, k, e);
        double geq = LG->w[k] * T * (1.0 + 4.0 * gamma * dot3(e, u));
        out[k] = g[k] - (g[k] - geq) / tg + LG->w[k] * Qsrc;
    }
}

static void thermal_bc_node(const lattice* LG, const orc_problem* P, uint8_t fl, double gamma,
                            const double u[3], const double* bcv, const double* gs, double* out) {
    int t = node_type(fl);
    for (int k = 0; k < LG->Q; k++) out[k] = gs[k];
    if (t == T_FLUID) return;
    int n[3];
    node_normal(fl, n);
    if (t == T_WALL) {
        for (int k = 0; k < LG->Q; k++) out[k] = gs[LG->opp[k]];
        if (fl & 0x40) out[unknown_dir(LG, n)] += P->q_flux;
        return;
    }
    int kn = unknown_dir(LG, n);
    double K = 0;
    for (int k = 0; k < LG->Q; k++)
        if (k != kn) K += gs[k];
    if (t == T_VEL || (fl & 0x40)) { /* inlet: T held at T_in (a fixed-density node with
                                         bit 6 is a pressure-driven inlet, Eq. 70) */
        out[kn] = bcv[3] - K;
    } else {
        double e[3];
        evec(LG, kn, e);
        double a = 1.0 + 4.0 * gamma * dot3(e, u);
        out[kn] = LG->w[kn] * a * K / (1.0 - LG->w[kn] * a);
    }
}

void orc_thermal_init(const orc_problem* P, double T0, double* g) {
    lattice LG;
    heat_lattice(&LG);
    long N = nnodes(P);
    for (long n = 0; n < N; n++)
        for (int k = 0; k < 7; k++) g[n * 7 + k] = LG.w[k] * T0;
}

void orc_thermal_step(const orc_problem* P, const uint8_t* flags, const double* gamma,
                      const double* bcval, const double* f, const double* g, double* gnew,
                      double* work) {
    lattice LF, LG;
    flow_lattice(P, &LF);
    heat_lattice(&LG);
    long N = nnodes(P);
    double* gc = work; /* N*7 */
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double u[3];
        flow_u(&LF, P, f + n * LF.Q, u);
        thermal_collide_node(&LG, P, flags[n], gamma[n], u, g + n * 7, gc + n * 7);
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; n++) {
        double gs[7], u[3];
        for (int k = 0; k < 7; k++)
            gs[k] = gc[stream_src(P, &LG, n, k, -1)];
        flow_u(&LF, P, f + n * LF.Q, u);
        thermal_bc_node(&LG, P, flags[n], gamma[n], u, bcval + 4 * n, gs, gnew + n * 7);
    }
}

void orc_thermal_run(const orc_problem* P, const uint8_t* flags, const double* gamma,
                     const double* bcval, const double* f, double* g, long nsteps) {
    long N = nnodes(P);
    double* tmp = (double*)malloc(sizeof(double) * N * 7);
    double* work = (double*)malloc(sizeof(double) * N * 7);
    for (long s = 0; s < nsteps; s++) {
        orc_thermal_step(P, flags, gamma, bcval, f, g, tmp, work);
        memcpy(g, tmp, sizeof(double) * N * 7);
    }
    free(tmp);
    free(work);
}

void orc_thermal_macro(const orc_problem* P, const double* g, double* T) {
    long N = nnodes(P);
    for (long n = 0; n < N; n++) {
        double s = 0;
        for (int k = 0; k < 7; k++) s += g[n * 7 + k];
        T[n] = s;
    }
}

/* local Jacobians of the thermal step at node n.
 * Cg[k][l] = d g_C,k / d g_l;  Cf[k][i] = d g_C,k / d f_i (through u);
 * Cgam[k] = d g_C,k / d gamma.  g is the post-B thermal state at the node. */
static void thermal_collision_jacobians(const lattice* LF, const lattice* LG,
                                        const orc_problem* P, uint8_t fl, double gamma,
                                        const double u[3], const double* g, double Cg[7][7],
                                        double Cf[7][QMAX], double Cgam[7]) {
    for (int k = 0; k < 7; k++) {
        for (int l = 0; l < 7; l++) Cg[k][l] = (k == l) ? 1.0 : 0.0;
        for (int i = 0; i < LF->Q; i++) Cf[k][i] = 0.0;
        Cgam[k] = 0.0;
    }
    if (node_type(fl) == T_WALL) return;
    double T = 0;
    for (int k = 0; k < 7; k++) T += g[k];
    double tg = tau_g(P, gamma);
    double dinv = -dtau_g(P) / (tg * tg); /* d(1/tau_g)/dgamma */
    for (int k = 0; k < 7; k++) {
        double e[3];
        evec(LG, k, e);
        double a = 1.0 + 4.0 * gamma * dot3(e, u);
        double geq = LG->w[k] * T * a;
        /* the source w_k beta (1 - T) adds -w_k beta to every column */
        for (int l = 0; l < 7; l++)
            Cg[k][l] = ((k == l) ? 1.0 : 0.0) - (((k == l) ? 1.0 : 0.0) - LG->w[k] * a) / tg
                       - LG->w[k] * P->beta_max * (1.0 - gamma);
        for (int i = 0; i < LF->Q; i++) {
            double du[3];
            for (int b = 0; b < 3; b++) du[b] = LF->e[i][b] / P->rho0;
            Cf[k][i] = (ORC_MUTATION == 8 ? -1.0 : 1.0) * LG->w[k] * T * 4.0 * gamma * dot3(e, du) / tg;
        }
        Cgam[k] = -(g[k] - geq) * dinv + LG->w[k] * T * 4.0 * dot3(e, u) / tg
                  - LG->w[k] * P->beta_max * (1.0 - T);
    }
}

/* local Jacobians of the thermal boundary operator at node n.
 * Bg[k][l] = d g_k / d g_S,l;  Bf[k][i] = d g_k / d f_i;  Bgam[k] = d g_k / d gamma.
 * gs are the post-stream populations (needed by the outlet, which is not affine in u). */
static void thermal_bc_jacobians(const lattice* LF, const lattice* LG, const orc_problem* P,
                                 uint8_t fl, double gamma, const double u[3], const double* gs,
                                 double Bg[7][7], double Bf[7][QMAX], double Bgam[7]) {
    int t = node_type(fl);
    for (int k = 0; k < 7; k++) {
        for (int l = 0; l < 7; l++) Bg[k][l] = 0.0;
        for (int i = 0; i < LF->Q; i++) Bf[k][i] = 0.0;
        Bgam[k] = 0.0;
    }
    if (t == T_FLUID) {
        for (int k = 0; k < 7; k++) Bg[k][k] = 1.0;
        return;
    }
    if (t == T_WALL) {
        for (int k = 0; k < 7; k++) Bg[k][LG->opp[k]] = 1.0;
        return;
    }
    int n[3];
    node_normal(fl, n);
    int kn = unknown_dir(LG, n);
    for (int k = 0; k < 7; k++)
        if (k != kn) Bg[k][k] = 1.0;
    if (t == T_VEL || (fl & 0x40)) {
        for (int l = 0; l < 7; l++)
            if (l != kn) Bg[kn][l] = -1.0;
        return;
    }
    double e[3];
    evec(LG, kn, e);
    double a = 1.0 + 4.0 * gamma * dot3(e, u);
    double K = 0;
    for (int l = 0; l < 7; l++)
        if (l != kn) K += gs[l];
    double w = LG->w[kn];
    for (int l = 0; l < 7; l++)
        if (l != kn) Bg[kn][l] = w * a / (1.0 - w * a);
    double dgda = w * K / ((1.0 - w * a) * (1.0 - w * a));
    for (int i = 0; i < LF->Q; i++) {
        double du[3];
        for (int b = 0; b < 3; b++) du[b] = LF->e[i][b] / P->rho0;
        Bf[kn][i] = dgda * 4.0 * gamma * dot3(e, du);
    }
    Bgam[kn] = dgda * 4.0 * dot3(e, u);
}

/* post-stream thermal populations at every node from the post-B state g */
static void thermal_poststream(const lattice* LF, const lattice* LG, const orc_problem* P,
                               const uint8_t* flags, const double* gamma, const double* f,
                               const double* g, double* gs_all) {
    long N = nnodes(P);
    double* gc = (double*)malloc(sizeof(double) * N * 7);
    for (long n = 0; n < N; n++) {
        double u[3];
        flow_u(LF, P, f + n * LF->Q, u);
        thermal_collide_node(LG, P, flags[n], gamma[n], u, g + n * 7, gc + n * 7);
    }
    for (long n = 0; n < N; n++)
        for (int k = 0; k < 7; k++)
            gs_all[n * 7 + k] = gc[stream_src(P, LG, n, k, -1)];
    free(gc);
}

/* tangent of the thermal step at the state (f, g):
 * dg_new = Bg S (Cg dg + Cf df) + Bf df      (df applied at both levels) */
void orc_thermal_tangent(const orc_problem* P, const uint8_t* flags, const double* gamma,
                         const double* f, const double* g, const double* dg, const double* df,
                         double* out) {
    lattice LF, LG;
    flow_lattice(P, &LF);
    heat_lattice(&LG);
    long N = nnodes(P);
    int Q = LF.Q;
    double* dc = (double*)malloc(sizeof(double) * N * 7);
    double* gs_all = (double*)malloc(sizeof(double) * N * 7);
    thermal_poststream(&LF, &LG, P, flags, gamma, f, g, gs_all);
    for (long n = 0; n < N; n++) {
        double u[3], Cg[7][7], Cf[7][QMAX], Cgam[7];
        flow_u(&LF, P, f + n * Q, u);
        thermal_collision_jacobians(&LF, &LG, P, flags[n], gamma[n], u, g + n * 7, Cg, Cf, Cgam);
        for (int k = 0; k < 7; k++) {
            double s = 0;
            for (int l = 0; l < 7; l++) s += Cg[k][l] * dg[n * 7 + l];
            for (int i = 0; i < Q; i++) s += Cf[k][i] * df[n * Q + i];
            dc[n * 7 + k] = s;
        }
    }
    for (long n = 0; n < N; n++) {
        double ds[7], u[3], Bg[7][7], Bf[7][QMAX], Bgam[7];
        for (int k = 0; k < 7; k++)
            ds[k] = dc[stream_src(P, &LG, n, k, -1)];
        flow_u(&LF, P, f + n * Q, u);
        thermal_bc_jacobians(&LF, &LG, P, flags[n], gamma[n], u, gs_all + n * 7, Bg, Bf, Bgam);
        for (int k = 0; k < 7; k++) {
            double s = 0;
            for (int l = 0; l < 7; l++) s += Bg[k][l] * ds[l];
            for (int i = 0; i < Q; i++) s += Bf[k][i] * df[n * Q + i];
            out[n * 7 + k] = s;
        }
    }
    free(dc);
    free(gs_all);
}

/* g* = B_g^T g*_C at every node (thermal counterpart of Eq. 54) */
void orc_thermal_adjoint_bc(const orc_problem* P, const uint8_t* flags, const double* gamma,
                            const double* f, const double* g, const double* gsc, double* gs) {
    lattice LF, LG;
    flow_lattice(P, &LF);
    heat_lattice(&LG);
    long N = nnodes(P);
    int Q = LF.Q;
    double* gs_all = (double*)malloc(sizeof(double) * N * 7);
    thermal_poststream(&LF, &LG, P, flags, gamma, f, g, gs_all);
    for (long n = 0; n < N; n++) {
        double u[3], Bg[7][7], Bf[7][QMAX], Bgam[7];
        flow_u(&LF, P, f + n * Q, u);
        thermal_bc_jacobians(&LF, &LG, P, flags[n], gamma[n], u, gs_all + n * 7, Bg, Bf, Bgam);
        for (int l = 0; l < 7; l++) {
            double s = 0;
            for (int k = 0; k < 7; k++) s += Bg[k][l] * gsc[n * 7 + k];
            gs[n * 7 + l] = s;
        }
    }
    free(gs_all);
}

/* one thermal adjoint iteration g*_C -> g*_C_new:
 * g* = Bg^T g*_C;  g*_S = S^T g*;  g*_C = Cg^T g*_S - dJ/dg.
 * with_source adds -w_tmean/N_nonwall per population at non-wall nodes. */
void orc_thermal_adjoint_step(const orc_problem* P, const uint8_t* flags, const double* gamma,
                              const double* f, const double* g, const double* gsc,
                              int with_source, double* gsc_new) {
    lattice LF, LG;
    flow_lattice(P, &LF);
    heat_lattice(&LG);
    long N = nnodes(P);
    int Q = LF.Q;
    double* gs_all = (double*)malloc(sizeof(double) * N * 7);
    double* gst = (double*)malloc(sizeof(double) * N * 7);
    thermal_poststream(&LF, &LG, P, flags, gamma, f, g, gs_all);
    for (long n = 0; n < N; n++) {
        double u[3], Bg[7][7], Bf[7][QMAX], Bgam[7];
        flow_u(&LF, P, f + n * Q, u);
        thermal_bc_jacobians(&LF, &LG, P, flags[n], gamma[n], u, gs_all + n * 7, Bg, Bf, Bgam);
        for (int l = 0; l < 7; l++) {
            double s = 0;
            for (int k = 0; k < 7; k++) s += Bg[k][l] * gsc[n * 7 + k];
            gst[n * 7 + l] = s;
        }
    }
    long nnw = count_nonwall(P, flags);
    double src = (nnw > 0) ? P->w_tmean / (double)nnw : 0.0;
    for (long n = 0; n < N; n++) {
        double gss[7], u[3], Cg[7][7], Cf[7][QMAX], Cgam[7];
        for (int k = 0; k < 7; k++)
            gss[k] = gst[stream_src(P, &LG, n, k, 1)];
        flow_u(&LF, P, f + n * Q, u);
        thermal_collision_jacobians(&LF, &LG, P, flags[n], gamma[n], u, g + n * 7, Cg, Cf, Cgam);
        /* dJ_Q/dg_l = w_qgen beta_max (1 - gamma) at non-wall nodes (Eq. 72) */
        double srcq = (ORC_MUTATION == 9 ? -1.0 : 1.0) * P->w_qgen * P->beta_max * (1.0 - gamma[n]);
        for (int l = 0; l < 7; l++) {
            double s = 0;
            for (int k = 0; k < 7; k++) s += Cg[k][l] * gss[k];
            if (with_source && node_type(flags[n]) != T_WALL) s -= src + srcq;
            gsc_new[n * 7 + l] = s;
        }
    }
    free(gs_all);
    free(gst);
}

void orc_thermal_adjoint_run(const orc_problem* P, const uint8_t* flags, const double* gamma,
                             const double* f, const double* g, double* gsc, long nsteps) {
    long N = nnodes(P);
    double* tmp = (double*)malloc(sizeof(double) * N * 7);
    for (long s = 0; s < nsteps; s++) {
        orc_thermal_adjoint_step(P, flags, gamma, f, g, gsc, 1, tmp);
        memcpy(gsc, tmp, sizeof(double) * N * 7);
    }
    free(tmp);
}

/* thermal-to-flow coupling and the thermal part of the sensitivity, from
 * the converged thermal adjoint g*_C:
 *   coupling_i(x) = sum_k g*_S,k dg_C,k/df_i + sum_k g*_C,k dB_g,k/df_i
 *   sensT(x)      = -sum_k g*_S,k dg_C,k/dgamma - sum_k g*_C,k dB_g,k/dgamma */
void orc_thermal_coupling(const orc_problem* P, const uint8_t* flags, const double* gamma,
                          const double* f, const double* g, const double* gsc,
                          double* coupling, double* sensT) {
    lattice LF, LG;
    flow_lattice(P, &LF);
    heat_lattice(&LG);
    long N = nnodes(P);
    int Q = LF.Q;
    double* gs_all = (double*)malloc(sizeof(double) * N * 7);
    double* gst = (double*)malloc(sizeof(double) * N * 7);
    thermal_poststream(&LF, &LG, P, flags, gamma, f, g, gs_all);
    for (long n = 0; n < N; n++) {
        double u[3], Bg[7][7], Bf[7][QMAX], Bgam[7];
        flow_u(&LF, P, f + n * Q, u);
        thermal_bc_jacobians(&LF, &LG, P, flags[n], gamma[n], u, gs_all + n * 7, Bg, Bf, Bgam);
        for (int l = 0; l < 7; l++) {
            double s = 0;
            for (int k = 0; k < 7; k++) s += Bg[k][l] * gsc[n * 7 + k];
            gst[n * 7 + l] = s;
        }
        for (int i = 0; i < Q; i++) {
            double s = 0;
            for (int k = 0; k < 7; k++) s += gsc[n * 7 + k] * Bf[k][i];
            coupling[n * Q + i] = s;
        }
        double sg = 0;
        for (int k = 0; k < 7; k++) sg += gsc[n * 7 + k] * Bgam[k];
        sensT[n] = -sg;
    }
    for (long n = 0; n < N; n++) {
        double gss[7], u[3], Cg[7][7], Cf[7][QMAX], Cgam[7];
        for (int k = 0; k < 7; k++)
            gss[k] = gst[stream_src(P, &LG, n, k, 1)];
        flow_u(&LF, P, f + n * Q, u);
        thermal_collision_jacobians(&LF, &LG, P, flags[n], gamma[n], u, g + n * 7, Cg, Cf, Cgam);
        for (int i = 0; i < Q; i++) {
            double s = 0;
            for (int k = 0; k < 7; k++) s += gss[k] * Cf[k][i];
            coupling[n * Q + i] += s;
        }
        double sg = 0;
        for (int k = 0; k < 7; k++) sg += gss[k] * Cgam[k];
        sensT[n] -= sg;
        /* direct part of J_Q: dJ_Q/dgamma = w_qgen beta_max (1 - T) */
        if (node_type(flags[n]) != T_WALL) {
            double T = 0;
            for (int k = 0; k < 7; k++) T += g[n * 7 + k];
            sensT[n] += P->w_qgen * P->beta_max * (1.0 - T);
        }
    }
    free(gs_all);
    free(gst);
}

/* J_Q = -sum over non-wall nodes of beta_max (1 - gamma)(1 - T), T of the
 * post-B state g (Eq. 72), times w_qgen */
double orc_objective_qgen(const orc_problem* P, const uint8_t* flags, const double* gamma,
                          const double* g) {
    long N = nnodes(P);
    double s = 0;
    for (long n = 0; n < N; n++) {
        if (node_type(flags[n]) == T_WALL) continue;
        double T = 0;
        for (int k = 0; k < 7; k++) T += g[n * 7 + k];
        s -= P->beta_max * (1.0 - gamma[n]) * (1.0 - T);
    }
    return P->w_qgen * s;
}

/* objective J = w_pin/(3 N_in) sum_inlet rho + w_tmean/N_nonwall sum_nonwall T
 * evaluated on post-B states (steady form of Eq. 34; the temperature term is
 * the heat-sink objective of the workload, g may be NULL) */
double orc_objective(const orc_problem* P, const uint8_t* flags, const double* f,
                     const double* g) {
    lattice L;
    flow_lattice(P, &L);
    long N = nnodes(P);
    long nin = count_type(P, flags, T_VEL), nnw = count_nonwall(P, flags);
    double sp = 0, st = 0;
    for (long n = 0; n < N; n++) {
        int t = node_type(flags[n]);
        if (t == T_VEL) {
            double r = 0;
            for (int i = 0; i < L.Q; i++) r += f[n * L.Q + i];
            sp += r;
        }
        if (g && t != T_WALL) {
            double T = 0;
            for (int k = 0; k < 7; k++) T += g[n * 7 + k];
            st += T;
        }
    }
    double J = 0;
    if (nin > 0) J += P->w_pin * sp / (3.0 * (double)nin);
    if (g && nnw > 0) J += P->w_tmean * st / (double)nnw;
    return J;
}

/* ---------------------------------------------------------------------- */
/* single-node access for pins                                              */
/* ---------------------------------------------------------------------- */
void orc_node_bc(const orc_problem* P, uint8_t fl, const double* bcv, const double* fs,
                 double* out) {
    lattice L;
    flow_lattice(P, &L);
    bc_node(&L, P, fl, bcv, fs, out);
}

void orc_node_bc_jacobian(const orc_problem* P, uint8_t fl, double* Bflat) {
    lattice L;
    flow_lattice(P, &L);
    double B[QMAX][QMAX];
    bc_jacobian(&L, P, fl, B);
    for (int i = 0; i < L.Q; i++)
        for (int j = 0; j < L.Q; j++) Bflat[i * L.Q + j] = B[i][j];
}

void orc_node_collide(const orc_problem* P, uint8_t fl, double gamma, const double* f,
                      double* out) {
    lattice L;
    flow_lattice(P, &L);
    collide_node(&L, P, fl, gamma, f, out);
}

void orc_node_collision_jacobian(const orc_problem* P, uint8_t fl, double gamma,
                                 const double* f, double* Cflat) {
    lattice L;
    flow_lattice(P, &L);
    double C[QMAX][QMAX];
    collision_jacobian(&L, P, fl, gamma, f, C);
    for (int i = 0; i < L.Q; i++)
        for (int j = 0; j < L.Q; j++) Cflat[i * L.Q + j] = C[i][j];
}

void orc_node_equilibrium(const orc_problem* P, double rho, const double* u, double gamma,
                          double* feq) {
    lattice L;
    flow_lattice(P, &L);
    equilibrium(&L, rho, u, gamma, P->gamma_model, P->rho0, feq);
}

/* lattice tables, so tests can check the moments of the weights */
int orc_lattice(int which, int* e, double* w, int* opp) {
    lattice L;
    if (which == 0) make_d2q9(&L);
    else if (which == 1) make_d3q19(&L);
    else make_d3q7(&L);
    finish_opp(&L);
    for (int i = 0; i < L.Q; i++) {
        for (int a = 0; a < 3; a++) e[3 * i + a] = L.e[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return L.Q;
}
