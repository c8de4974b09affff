/*
 * FP64 CPU oracle for the D3Q19 lattice Boltzmann time step of Bauer & Ruede,
 * "An improved lattice Boltzmann D3Q19 method based on an alternative
 * equilibrium discretization" (arXiv:1803.04937).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * definition of what the GPU library computes.  It is used by the tests, by
 * the smoke check and by the CPU-baseline leg of the benchmark, never by the
 * library itself.  It shares no code, tables or headers with the CUDA path.
 *
 * Conventions (all lattice units, dx = dt = 1, c_s^2 = 1/3):
 *   - velocity sets (Sec. 2.3), built here by enumerating {-1,0,1}^3 in this
 *     file's own order: D3Q19 keeps |c|^2 <= 2 (rest, 6 faces, 12 edges;
 *     weights 1/3, 1/18, 1/36); D3Q27 keeps all 27 (weights 8/27, 2/27, 1/54,
 *     1/216).  On D3Q27 the moment-matching construction gives the standard
 *     equilibrium (Sec. 3.1), so both equilibrium choices are Eq. 14 there.
 *   - state: f[((z*ny + y)*nx + x)*Q + q] (Q = 19 or 27), the post-streaming,
 *     pre-collision populations f_q(x, t) of Eq. 15.
 *   - equilibria: standard D3Q19-S = Eq. 14 truncated at second order in u;
 *     improved D3Q19-I = Eq. 22.  rho0 = 1 (Sec. 2.3, used for all of the
 *     paper's analysis) or rho0 = rho (the compressible variant below Eq. 14).
 *   - update: Eq. 15 with the Buick-Greated force F_q = w_q c_q.a / c_s^2 and
 *     the velocity shift of Eq. 17: rho0 u = sum_q c_q f_q + a/2.
 *   - TRT (Sec. 3.3 names it; the paper gives no formula): symmetric and
 *     antisymmetric parts relax with omega+ = 1/tau and omega- = 1/tau-,
 *     (tau+ - 1/2)(tau- - 1/2) = Lambda; the force is odd in c and takes
 *     (1 - omega-/2).  With omega- = omega+ this is Eq. 15 exactly.
 *   - MRT (Sec. 3.2-3.3): the populations are mapped to the monomial moments
 *     xi_x^e0 xi_y^e1 xi_z^e2, e_i in {0,1,2} (on D3Q19 without the eight of
 *     Eq. 21), relaxed there against the moments of the Maxwellian truncated
 *     at second order in u (D3Q19-I; for D3Q19-S against the moments of the
 *     discrete equilibrium Eq. 14), and mapped back with the inverse moment
 *     matrix.  Rates: odd orders omega- (as TRT), the deviatoric part of the
 *     second-order block omega+, its trace omega_bulk, even orders >= 4
 *     omega_4; the force enters as (I - S/2) M F.  The paper fixes none of the
 *     rates; with omega_bulk = omega_4 = omega+ this is TRT exactly.
 *   - boundaries: periodic, or half-way bounce-back walls at both ends of an
 *     axis (Sec. 5.1): a population whose link leaves the domain through a
 *     wall returns to its own cell reversed, f_qbar(x, t+1) = f*_q(x, t).
 *   - streaming is done by PUSH after collision (the GPU library pulls).
 *
 * The adjoint (reverse-mode derivative of one step; not in the paper) is
 * written as the transpose of the explicitly assembled QxQ Jacobian of the
 * collision, composed with the transpose of the streaming permutation.  It
 * supports rho0 = 1 and SRT/TRT only.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 27

typedef struct {
    int nx, ny, nz;
    int equilibrium;   /* 0: standard D3Q19-S, 1: improved D3Q19-I */
    int collision;     /* 0: SRT, 1: TRT, 2: MRT */
    int rho0_is_rho;   /* 0: rho0 = 1, 1: rho0 = rho */
    int wall[3];       /* 1: half-way bounce-back walls at both ends of axis */
    int nthreads;      /* OpenMP threads (<= 0: library default) */
    double tau;        /* relaxation time, omega = 1/tau */
    double trt_magic;  /* Lambda = (tau+ - 1/2)(tau- - 1/2) */
    double accel[3];   /* body force a */
    int stencil;       /* 19 (D3Q19, default when 0) or 27 (D3Q27) */
    double omega_bulk; /* MRT: rate of the trace of the second-order moments */
    double omega_4;    /* MRT: rate of the even moments of order >= 4 */
} oracle_cfg;

/* A velocity set: Q velocities C, weights W, opposite index OPP. */
typedef struct {
    int Q;
    int C[QMAX][3];
    double W[QMAX];
    int OPP[QMAX];
} lattice;

static lattice D3Q19, D3Q27;
static int built = 0;

/* D3Q19 and D3Q27 velocities and weights (Sec. 2.3). */
static void build_one(lattice *L, int maxnorm)
{
    int q = 0;
    for (int cx = -1; cx <= 1; ++cx)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cz = -1; cz <= 1; ++cz) {
                int n = cx * cx + cy * cy + cz * cz;
                if (n > maxnorm) continue;
                L->C[q][0] = cx; L->C[q][1] = cy; L->C[q][2] = cz;
                if (maxnorm == 2)
                    L->W[q] = (n == 0) ? 1.0 / 3.0 : (n == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                else
                    L->W[q] = (n == 0) ? 8.0 / 27.0 : (n == 1) ? 2.0 / 27.0 : (n == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
                ++q;
            }
    L->Q = q;
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b)
            if (L->C[a][0] == -L->C[b][0] && L->C[a][1] == -L->C[b][1] && L->C[a][2] == -L->C[b][2])
                L->OPP[a] = b;
}

static void build_bases(void);

/* Built once, before any OpenMP region uses the tables. */
static void build_lattice(void)
{
    if (built) return;
    build_one(&D3Q19, 2);
    build_one(&D3Q27, 3);
    built = 1;
    build_bases();
}

static const lattice *lattice_of(int stencil)
{
    build_lattice();
    return stencil == 27 ? &D3Q27 : &D3Q19;
}

/* Velocities c[3q+i], weights w[q], opposites opp[q] of the stencil (19 or
 * 27); returns Q. */
int oracle_velocity_set_of(int stencil, int *c, double *w, int *opp)
{
    const lattice *L = lattice_of(stencil);
    for (int q = 0; q < L->Q; ++q) {
        for (int i = 0; i < 3; ++i) c[3 * q + i] = L->C[q][i];
        w[q] = L->W[q];
        opp[q] = L->OPP[q];
    }
    return L->Q;
}

void oracle_velocity_set(int *c, double *w, int *opp)
{
    oracle_velocity_set_of(19, c, w, opp);
}

/* Eq. 14 (second-order part) or Eq. 22 (D3Q19 only), for one cell. */
static void equilibrium(const lattice *L, int kind, double rho, double rho0, const double u[3], double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < L->Q; ++q) {
        const int *c = L->C[q];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        int n = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        double bracket;
        if (kind == 0 || L->Q == 27) {
            /* standard: 3 c.u + 9/2 u_a u_b (c_a c_b - delta_ab / 3) */
            bracket = 3.0 * cu + 4.5 * cu * cu - 1.5 * uu;
        } else if (n == 0) {
            /* D3Q19-I, rest */
            bracket = -uu;
        } else if (n == 1) {
            /* D3Q19-I, faces */
            bracket = 3.0 * cu - 3.0 * uu + 6.0 * cu * cu;
        } else {
            /* D3Q19-I, edges; sum over i of u_i^2 c_qi^2 */
            double s = 0.0;
            for (int i = 0; i < 3; ++i) s += u[i] * u[i] * c[i] * c[i];
            bracket = 3.0 * cu - 1.5 * s + 4.5 * cu * cu;
        }
        feq[q] = L->W[q] * rho + L->W[q] * rho0 * bracket;
    }
}

/* d feq_q / d u_i at fixed rho, for rho0 = 1 (the derivative of the closed
 * forms above, written out by hand). */
static void equilibrium_du(const lattice *L, int kind, const double u[3], double d[][3])
{
    for (int q = 0; q < L->Q; ++q) {
        const int *c = L->C[q];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        int n = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        for (int i = 0; i < 3; ++i) {
            double ci = c[i];
            double v;
            if (kind == 0 || L->Q == 27) v = 3.0 * ci + 9.0 * cu * ci - 3.0 * u[i];
            else if (n == 0) v = -2.0 * u[i];
            else if (n == 1) v = 3.0 * ci - 6.0 * u[i] + 12.0 * cu * ci;
            else v = 3.0 * ci - 3.0 * u[i] * ci * ci + 9.0 * cu * ci;
            d[q][i] = L->W[q] * v;
        }
    }
}

void oracle_equilibrium_field_of(int stencil, int kind, int rho0_is_rho, long n, const double *rho,
                                 const double *u, double *feq)
{
    const lattice *L = lattice_of(stencil);
    for (long k = 0; k < n; ++k) {
        double uk[3] = {u[k], u[n + k], u[2 * n + k]};
        double rho0 = rho0_is_rho ? rho[k] : 1.0;
        equilibrium(L, kind, rho[k], rho0, uk, feq + k * L->Q);
    }
}

void oracle_equilibrium_field(int kind, int rho0_is_rho, long n, const double *rho,
                              const double *u, double *feq)
{
    oracle_equilibrium_field_of(19, kind, rho0_is_rho, n, rho, u, feq);
}

static const lattice *cfg_lattice(const oracle_cfg *cfg) { return lattice_of(cfg->stencil); }

static void omegas(const oracle_cfg *cfg, double *wp, double *wm)
{
    *wp = 1.0 / cfg->tau;
    if (cfg->collision == 1 || cfg->collision == 2) {
        double tau_minus = 0.5 + cfg->trt_magic / (cfg->tau - 0.5);
        *wm = 1.0 / tau_minus;
    } else {
        *wm = *wp;
    }
}

/* Moments of Eq. 16 and Eq. 17 for one cell. */
static void cell_moments(const oracle_cfg *cfg, const lattice *L, const double *f, double *rho, double *rho0,
                         double u[3])
{
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < L->Q; ++q) {
        r += f[q];
        for (int i = 0; i < 3; ++i) j[i] += L->C[q][i] * f[q];
    }
    double r0 = cfg->rho0_is_rho ? r : 1.0;
    for (int i = 0; i < 3; ++i) u[i] = (j[i] + 0.5 * cfg->accel[i]) / r0;
    *rho = r;
    *rho0 = r0;
}

static double force_term(const oracle_cfg *cfg, const lattice *L, int q)
{
    const int *c = L->C[q];
    return 3.0 * L->W[q] * (c[0] * cfg->accel[0] + c[1] * cfg->accel[1] + c[2] * cfg->accel[2]);
}

/* ---------------- MRT in moment space (Sec. 3.2, 3.3) ---------------- */

/* The monomial moments of a stencil: exponents E[k] and the moment matrix
 * M[k][q] = prod_i c_qi^E[k][i], with its inverse (Gauss-Jordan elimination
 * with partial pivoting; the matrix is invertible by construction, Sec. 3.2). */
typedef struct {
    int K;
    int E[QMAX][3];
    double M[QMAX][QMAX], Minv[QMAX][QMAX];
} moment_basis;

static moment_basis BASIS19, BASIS27;

/* The eight moments Eq. 21 drops for D3Q19. */
static int dropped_on_d3q19(const int e[3])
{
    int n1 = 0, n2 = 0;
    for (int i = 0; i < 3; ++i) {
        n1 += e[i] == 1;
        n2 += e[i] == 2;
    }
    /* (1,2,2) and permutations, (1,1,2) and permutations, (1,1,1), (2,2,2) */
    return (n1 == 1 && n2 == 2) || (n1 == 2 && n2 == 1) || n1 == 3 || n2 == 3;
}

static double ipow(int c, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= c;
    return r;
}

static void invert(int n, double A[][QMAX], double X[][QMAX])
{
    double W[QMAX][2 * QMAX];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) W[r][c] = c < n ? A[r][c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(W[r][col]) > fabs(W[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = W[col][c]; W[col][c] = W[piv][c]; W[piv][c] = t;
            }
        double d = W[col][col];
        for (int c = 0; c < 2 * n; ++c) W[col][c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = W[r][col];
            if (m != 0.0)
                for (int c = 0; c < 2 * n; ++c) W[r][c] -= m * W[col][c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) X[r][c] = W[r][n + c];
}

static void build_basis(moment_basis *B, const lattice *L)
{
    int k = 0;
    for (int e0 = 0; e0 <= 2; ++e0)
        for (int e1 = 0; e1 <= 2; ++e1)
            for (int e2 = 0; e2 <= 2; ++e2) {
                int e[3] = {e0, e1, e2};
                if (L->Q == 19 && dropped_on_d3q19(e)) continue;
                for (int i = 0; i < 3; ++i) B->E[k][i] = e[i];
                for (int q = 0; q < L->Q; ++q)
                    B->M[k][q] = ipow(L->C[q][0], e0) * ipow(L->C[q][1], e1) * ipow(L->C[q][2], e2);
                ++k;
            }
    B->K = k;
    invert(k, B->M, B->Minv);
}

static void build_bases(void)
{
    build_basis(&BASIS19, &D3Q19);
    build_basis(&BASIS27, &D3Q27);
}

static const moment_basis *basis_of(const lattice *L)
{
    return L->Q == 27 ? &BASIS27 : &BASIS19;
}

/* Moment xi^e of the continuous Maxwellian (Eq. 6, c_s^2 = 1/3) truncated at
 * second order in u, with rho on the u-free part and rho0 on the rest (Table
 * 1).  The 1D factors are 1, u, u^2 + 1/3; their product is expanded by
 * degree in u and cut after degree 2. */
static double maxwellian_moment(const int e[3], double rho, double rho0, const double u[3])
{
    double P[7] = {1.0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 3; ++i) {
        double fac[3] = {0, 0, 0};
        if (e[i] == 0) fac[0] = 1.0;
        else if (e[i] == 1) fac[1] = u[i];
        else { fac[0] = 1.0 / 3.0; fac[2] = u[i] * u[i]; }
        double R[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 7; ++a)
            for (int b = 0; b < 3 && a + b < 7; ++b) R[a + b] += P[a] * fac[b];
        for (int a = 0; a < 7; ++a) P[a] = R[a];
    }
    return rho * P[0] + rho0 * (P[1] + P[2]);
}

/* Relaxation matrix S in moment space (rates as described at the top). */
static void mrt_rates(const oracle_cfg *cfg, const moment_basis *B, double S[][QMAX])
{
    double wp, wm;
    omegas(cfg, &wp, &wm);
    for (int k = 0; k < B->K; ++k)
        for (int l = 0; l < B->K; ++l) S[k][l] = 0.0;
    for (int k = 0; k < B->K; ++k) {
        const int *e = B->E[k];
        int order = e[0] + e[1] + e[2];
        int diag2 = order == 2 && (e[0] == 2 || e[1] == 2 || e[2] == 2);
        if (order % 2 == 1) S[k][k] = wm;
        else if (order == 0) S[k][k] = wp;
        else if (order == 2 && !diag2) S[k][k] = wp;
        else if (order == 2) {
            /* xi_a^2 block: deviator at omega+, trace at omega_bulk */
            for (int l = 0; l < B->K; ++l) {
                const int *g = B->E[l];
                if (g[0] + g[1] + g[2] == 2 && (g[0] == 2 || g[1] == 2 || g[2] == 2))
                    S[k][l] = wp * ((k == l ? 1.0 : 0.0) - 1.0 / 3.0) + cfg->omega_bulk / 3.0;
            }
        } else S[k][k] = cfg->omega_4;
    }
}

/* Post-collision populations of one cell, MRT:
 * fs = f - M^-1 [ S (M f - m_eq) - (I - S/2) M F ]. */
static void collide_mrt(const oracle_cfg *cfg, const lattice *L, const double *f, double *fs)
{
    const moment_basis *B = basis_of(L);
    const int K = B->K;
    double rho, rho0, u[3], S[QMAX][QMAX], m[QMAX], meq[QMAX], mF[QMAX], r[QMAX];
    cell_moments(cfg, L, f, &rho, &rho0, u);
    mrt_rates(cfg, B, S);
    double feq[QMAX], F[QMAX];
    equilibrium(L, 0, rho, rho0, u, feq);
    for (int q = 0; q < L->Q; ++q) F[q] = force_term(cfg, L, q);
    for (int k = 0; k < K; ++k) {
        m[k] = mF[k] = 0.0;
        double mS = 0.0;
        for (int q = 0; q < L->Q; ++q) {
            m[k] += B->M[k][q] * f[q];
            mF[k] += B->M[k][q] * F[q];
            mS += B->M[k][q] * feq[q];
        }
        /* improved: Maxwellian moments (Sec. 3.2); standard: moments of Eq. 14 */
        meq[k] = cfg->equilibrium == 1 ? maxwellian_moment(B->E[k], rho, rho0, u) : mS;
    }
    for (int k = 0; k < K; ++k) {
        double a = 0.0, b = 0.0;
        for (int l = 0; l < K; ++l) {
            a += S[k][l] * (m[l] - meq[l]);
            b += S[k][l] * mF[l];
        }
        r[k] = a - (mF[k] - 0.5 * b);
    }
    for (int q = 0; q < L->Q; ++q) {
        double d = 0.0;
        for (int k = 0; k < K; ++k) d += B->Minv[q][k] * r[k];
        fs[q] = f[q] - d;
    }
}

/* Post-collision populations of one cell (Eq. 15, its TRT split, or MRT). */
static void collide(const oracle_cfg *cfg, const lattice *L, const double *f, double *fs)
{
    if (cfg->collision == 2) {
        collide_mrt(cfg, L, f, fs);
        return;
    }
    double rho, rho0, u[3], feq[QMAX], wp, wm;
    cell_moments(cfg, L, f, &rho, &rho0, u);
    equilibrium(L, cfg->equilibrium, rho, rho0, u, feq);
    omegas(cfg, &wp, &wm);
    for (int q = 0; q < L->Q; ++q) {
        int o = L->OPP[q];
        double F = force_term(cfg, L, q);
        double fp = 0.5 * (f[q] + f[o]), fm = 0.5 * (f[q] - f[o]);
        double ep = 0.5 * (feq[q] + feq[o]), em = 0.5 * (feq[q] - feq[o]);
        if (cfg->collision == 0)
            fs[q] = f[q] - wp * (f[q] - feq[q]) + (1.0 - 0.5 * wp) * F;
        else
            fs[q] = f[q] - wp * (fp - ep) - wm * (fm - em) + (1.0 - 0.5 * wm) * F;
    }
}

static long cell_index(const oracle_cfg *cfg, int x, int y, int z)
{
    return ((long)z * cfg->ny + y) * (long)cfg->nx + x;
}

/* Target of the link from (x,y,z) along c_q.  Returns 0 and the wrapped
 * target cell for a periodic or interior link; returns 1 when the link
 * crosses a wall (half-way bounce-back). */
static int link_target(const oracle_cfg *cfg, const lattice *L, int x, int y, int z, int q, long *target)
{
    int p[3] = {x + L->C[q][0], y + L->C[q][1], z + L->C[q][2]};
    int n[3] = {cfg->nx, cfg->ny, cfg->nz};
    for (int i = 0; i < 3; ++i) {
        if (p[i] < 0 || p[i] >= n[i]) {
            if (cfg->wall[i]) return 1;
            p[i] = (p[i] + n[i]) % n[i];
        }
    }
    *target = cell_index(cfg, p[0], p[1], p[2]);
    return 0;
}

static void set_threads(const oracle_cfg *cfg)
{
#ifdef _OPENMP
    if (cfg->nthreads > 0) omp_set_num_threads(cfg->nthreads);
#else
    (void)cfg;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* f(t=0) = feq(rho, u0): the initialisation without non-equilibrium part. */
void oracle_init(const oracle_cfg *cfg, const double *rho, const double *u, double *f)
{
    const lattice *L = cfg_lattice(cfg);
    long n = (long)cfg->nx * cfg->ny * cfg->nz;
    for (long k = 0; k < n; ++k) {
        double uk[3] = {u[k], u[n + k], u[2 * n + k]};
        double rho0 = cfg->rho0_is_rho ? rho[k] : 1.0;
        equilibrium(L, cfg->equilibrium, rho[k], rho0, uk, f + k * L->Q);
    }
}

/* One time step of Eq. 15: collide every cell, then push along c_q. */
void oracle_step(const oracle_cfg *cfg, const double *f, double *fnew)
{
    const lattice *L = cfg_lattice(cfg);
    const int Q = L->Q;
    set_threads(cfg);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < cfg->nz; ++z)
        for (int y = 0; y < cfg->ny; ++y)
            for (int x = 0; x < cfg->nx; ++x) {
                long k = cell_index(cfg, x, y, z);
                double fs[QMAX];
                collide(cfg, L, f + k * Q, fs);
                for (int q = 0; q < Q; ++q) {
                    long t;
                    if (link_target(cfg, L, x, y, z, q, &t))
                        fnew[k * Q + L->OPP[q]] = fs[q];
                    else
                        fnew[t * Q + q] = fs[q];
                }
            }
}

/* rho = sum_q f_q (Eq. 16), u from Eq. 17. */
void oracle_moments(const oracle_cfg *cfg, const double *f, double *rho, double *u)
{
    const lattice *L = cfg_lattice(cfg);
    long n = (long)cfg->nx * cfg->ny * cfg->nz;
    for (long k = 0; k < n; ++k) {
        double r, r0, uk[3];
        cell_moments(cfg, L, f + k * L->Q, &r, &r0, uk);
        rho[k] = r;
        for (int i = 0; i < 3; ++i) u[i * n + k] = uk[i];
    }
}

/* nsteps steps from f = feq(rho, u); returns final rho, u.  Two grids. */
int oracle_run(const oracle_cfg *cfg, const double *rho_in, const double *u_in, int nsteps,
               double *rho_out, double *u_out)
{
    const lattice *L = cfg_lattice(cfg);
    long n = (long)cfg->nx * cfg->ny * cfg->nz;
    double *a = (double *)malloc(sizeof(double) * L->Q * n);
    double *b = (double *)malloc(sizeof(double) * L->Q * n);
    if (!a || !b) { free(a); free(b); return 1; }
    oracle_init(cfg, rho_in, u_in, a);
    for (int s = 0; s < nsteps; ++s) {
        oracle_step(cfg, a, b);
        double *t = a; a = b; b = t;
    }
    oracle_moments(cfg, a, rho_out, u_out);
    free(a);
    free(b);
    return 0;
}

/* ---------------- adjoint (rho0 = 1) ---------------- */

/* Jacobian J[q][p] = d fs_q / d f_p of the collision of one cell, and the
 * derivatives of fs with respect to omega+ and omega-. */
static void collide_jacobian(const oracle_cfg *cfg, const lattice *L, const double *f, double J[][QMAX],
                             double *dfs_dwp, double *dfs_dwm)
{
    const int Q = L->Q;
    double rho, rho0, u[3], feq[QMAX], du[QMAX][3], wp, wm, dfeq[QMAX][QMAX];
    cell_moments(cfg, L, f, &rho, &rho0, u);
    equilibrium(L, cfg->equilibrium, rho, rho0, u, feq);
    equilibrium_du(L, cfg->equilibrium, u, du);
    omegas(cfg, &wp, &wm);
    /* d feq_q / d f_p = w_q d rho/d f_p + sum_i d feq_q/d u_i d u_i/d f_p,
     * with d rho / d f_p = 1 and d u_i / d f_p = c_pi (rho0 = 1). */
    for (int q = 0; q < Q; ++q)
        for (int p = 0; p < Q; ++p)
            dfeq[q][p] = L->W[q] + du[q][0] * L->C[p][0] + du[q][1] * L->C[p][1] + du[q][2] * L->C[p][2];
    for (int q = 0; q < Q; ++q) {
        int o = L->OPP[q];
        double F = force_term(cfg, L, q);
        for (int p = 0; p < Q; ++p) {
            double dqp = (q == p) ? 1.0 : 0.0, dop = (o == p) ? 1.0 : 0.0;
            double dfp = 0.5 * (dqp + dop), dfm = 0.5 * (dqp - dop);
            double dep = 0.5 * (dfeq[q][p] + dfeq[o][p]), dem = 0.5 * (dfeq[q][p] - dfeq[o][p]);
            J[q][p] = dqp - wp * (dfp - dep) - wm * (dfm - dem);
        }
        dfs_dwp[q] = -(0.5 * (f[q] + f[o]) - 0.5 * (feq[q] + feq[o]));
        dfs_dwm[q] = -(0.5 * (f[q] - f[o]) - 0.5 * (feq[q] - feq[o])) - 0.5 * F;
    }
}

/* lam_t = (d state(t+1) / d state(t))^T lam_next, and the contributions of
 * this step to dL/d omega+ and dL/d omega- (added to grad_omega[0..1]).
 * For SRT both omegas are 1/tau and dL/d omega = grad_omega[0] + grad_omega[1]. */
int oracle_adjoint_step(const oracle_cfg *cfg, const double *f_t, const double *lam_next,
                        double *lam_t, double *grad_omega)
{
    const lattice *L = cfg_lattice(cfg);
    const int Q = L->Q;
    if (cfg->rho0_is_rho || cfg->collision == 2) return 1;
    double gp = 0.0, gm = 0.0;
    for (int z = 0; z < cfg->nz; ++z)
        for (int y = 0; y < cfg->ny; ++y)
            for (int x = 0; x < cfg->nx; ++x) {
                long k = cell_index(cfg, x, y, z);
                double J[QMAX][QMAX], dwp[QMAX], dwm[QMAX], mu[QMAX];
                collide_jacobian(cfg, L, f_t + k * Q, J, dwp, dwm);
                /* transpose of the push: fs_q(x) went to f_q(x + c_q) or,
                 * through a wall, to f_qbar(x). */
                for (int q = 0; q < Q; ++q) {
                    long t;
                    if (link_target(cfg, L, x, y, z, q, &t))
                        mu[q] = lam_next[k * Q + L->OPP[q]];
                    else
                        mu[q] = lam_next[t * Q + q];
                }
                for (int p = 0; p < Q; ++p) {
                    double s = 0.0;
                    for (int q = 0; q < Q; ++q) s += mu[q] * J[q][p];
                    lam_t[k * Q + p] = s;
                }
                for (int q = 0; q < Q; ++q) {
                    gp += mu[q] * dwp[q];
                    gm += mu[q] * dwm[q];
                }
            }
    grad_omega[0] += gp;
    grad_omega[1] += gm;
    return 0;
}

/* dL/df_q(T) for L = 1/2 sum_x |u(x,T) - u_target(x)|^2 (rho0 = 1):
 * lam_q = sum_i (u_i - target_i) c_qi.  Returns L in *loss. */
int oracle_loss_velocity_l2(const oracle_cfg *cfg, const double *f, const double *u_target,
                            double *lam, double *loss)
{
    const lattice *L = cfg_lattice(cfg);
    if (cfg->rho0_is_rho) return 1;
    long n = (long)cfg->nx * cfg->ny * cfg->nz;
    double Lsum = 0.0;
    for (long k = 0; k < n; ++k) {
        double r, r0, u[3], g[3];
        cell_moments(cfg, L, f + k * L->Q, &r, &r0, u);
        for (int i = 0; i < 3; ++i) {
            g[i] = u[i] - u_target[i * n + k];
            Lsum += 0.5 * g[i] * g[i];
        }
        for (int q = 0; q < L->Q; ++q)
            lam[k * L->Q + q] = g[0] * L->C[q][0] + g[1] * L->C[q][1] + g[2] * L->C[q][2];
    }
    *loss = Lsum;
    return 0;
}

/* dL/du0_i(x) = sum_q lam0_q(x) d feq_q / d u_i (rho(x), u0(x)), from
 * f(0) = feq(rho, u0). */
int oracle_adjoint_init_velocity(const oracle_cfg *cfg, const double *u0, const double *lam0,
                                 double *grad_u0)
{
    const lattice *L = cfg_lattice(cfg);
    if (cfg->rho0_is_rho) return 1;
    long n = (long)cfg->nx * cfg->ny * cfg->nz;
    for (long k = 0; k < n; ++k) {
        double uk[3] = {u0[k], u0[n + k], u0[2 * n + k]}, d[QMAX][3];
        equilibrium_du(L, cfg->equilibrium, uk, d);
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
            for (int q = 0; q < L->Q; ++q) s += lam0[k * L->Q + q] * d[q][i];
            grad_u0[i * n + k] = s;
        }
    }
    return 0;
}

/* d omega+/d tau and d omega-/d tau for the configured collision. */
void oracle_domega_dtau(const oracle_cfg *cfg, double *dwp, double *dwm)
{
    double tau = cfg->tau;
    *dwp = -1.0 / (tau * tau);
    if (cfg->collision == 1 || cfg->collision == 2) {
        double tm = 0.5 + cfg->trt_magic / (tau - 0.5);
        double dtm = -cfg->trt_magic / ((tau - 0.5) * (tau - 0.5));
        *dwm = -dtm / (tm * tm);
    } else {
        *dwm = *dwp;
    }
}
