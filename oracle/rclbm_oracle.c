/*
 * rclbm_oracle.c -- FP64 CPU oracle of the RC-LBM and RNR-LBM on a D2Q9
 * rectangular lattice (Yahia & Premnath, arXiv 2103.02119).
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA library and is never called by
 * the product path.
 *
 * This file is deliberately plain.  It follows the paper's algorithm in the
 * paper's order and notation, in its literal matrix form:
 *   - T is built by evaluating the monomials of Eq. 3 on the velocities of
 *     Eq. 2 (it is not typed in, so it does not inherit the misprint of
 *     Eq. 4 row 7).
 *   - T^-1 is obtained by Gauss-Jordan elimination (not typed in from
 *     App. A, which has one misprinted entry).
 *   - F(u) is built from its definition m^c = F m: the central monomials
 *     evaluated at e_i - u, times T^-1; F^-1 is F(-u) (App. B).
 *   - Equilibria, corrections and strain rates are Eq. 12, 23-27, 37-40 and
 *     49 written out term by term.
 *   - Streaming is an explicit gather loop; walls are a separate pass.
 * Parallelism is OpenMP over rows and nothing else.
 */
#include "rclbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Eq. 2: e_x and e_y / a for directions 0..8. */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Opposite direction: e_opp(i) = -e_i. */
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

struct orc {
    orc_params p;
    int N;
    double T[81], Ti[81];
    unsigned char* solid;
    double* f;    /* state f(x, t), plane-major 9*N          */
    double* ft;   /* post-collision f~(x, t)                 */
    double* rho;  /* rho(x, t)                               */
    double* dxr;  /* density gradient, central differences   */
    double* dyr;
};

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra                                                 */
/* ------------------------------------------------------------------------ */

/* Eq. 3: the non-orthogonal basis 1, x, y, x^2+y^2, x^2-y^2, xy, x^2 y,
 * x y^2, x^2 y^2. */
static double basis(int k, double x, double y)
{
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return x * x + y * y;
    case 4: return x * x - y * y;
    case 5: return x * y;
    case 6: return x * x * y;
    case 7: return x * y * y;
    default: return x * x * y * y;
    }
}

static void matmul9(const double* A, const double* B, double* C)
{
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            double s = 0.0;
            for (int k = 0; k < 9; ++k) s += A[i * 9 + k] * B[k * 9 + j];
            C[i * 9 + j] = s;
        }
}

static void matvec9(const double* A, const double* x, double* y)
{
    for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int k = 0; k < 9; ++k) s += A[i * 9 + k] * x[k];
        y[i] = s;
    }
}

/* Gauss-Jordan elimination with partial pivoting. */
static int invert9(const double* A, double* Ai)
{
    double M[9][18];
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            M[i][j] = A[i * 9 + j];
            M[i][9 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 9; ++c) {
        int piv = c;
        for (int r = c + 1; r < 9; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (fabs(M[piv][c]) < 1e-300) return -1;
        if (piv != c)
            for (int j = 0; j < 18; ++j) {
                double t = M[c][j];
                M[c][j] = M[piv][j];
                M[piv][j] = t;
            }
        double d = M[c][c];
        for (int j = 0; j < 18; ++j) M[c][j] /= d;
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            double g = M[r][c];
            if (g == 0.0) continue;
            for (int j = 0; j < 18; ++j) M[r][j] -= g * M[c][j];
        }
    }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) Ai[i * 9 + j] = M[i][9 + j];
    return 0;
}

/* T of Eq. 4: row k holds monomial k of Eq. 3 evaluated at e_i. */
static void build_T(double a, double* T)
{
    for (int k = 0; k < 9; ++k)
        for (int i = 0; i < 9; ++i) T[k * 9 + i] = basis(k, EX[i], a * EY[i]);
}

/* Frame transformation of App. B from its definition: m^c = Tc(u) f and
 * m = T f give F(u) = Tc(u) T^-1, where row k of Tc(u) holds monomial k
 * evaluated at e_i - u. */
static void build_F(double a, double ux, double uy, const double* Ti,
                    double* F)
{
    double Tc[81];
    for (int k = 0; k < 9; ++k)
        for (int i = 0; i < 9; ++i)
            Tc[k * 9 + i] = basis(k, EX[i] - ux, a * EY[i] - uy);
    matmul9(Tc, Ti, F);
}

int orc_matrices(double a, double ux, double uy, double T[81], double Ti[81],
                 double F[81], double Fi[81])
{
    if (!(a > 0.0) || !T || !Ti || !F || !Fi) return -1;
    build_T(a, T);
    if (invert9(T, Ti)) return -1;
    build_F(a, ux, uy, Ti, F);
    build_F(a, -ux, -uy, Ti, Fi); /* App. B: F^-1(u) = F(-u) */
    return 0;
}

int orc_central_moments(double a, const double f[9], double ux, double uy,
                        double kc[9])
{
    if (!f || !kc) return -1;
    /* Eq. 43 summed directly. */
    for (int k = 0; k < 9; ++k) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i)
            s += f[i] * basis(k, EX[i] - ux, a * EY[i] - uy);
        kc[k] = s;
    }
    return 0;
}

/* f^eq = T^-1 F(-u) m^{c,eqr} with the Maxwell-matched central moments of
 * the square lattice (rho, 0, 0, 2 rho cs2, 0, 0, 0, 0, rho cs2^2) written in
 * the basis of Eq. 46 (Sec. 4, first entries of Eq. 49). */
static void feq_with(const double* Ti, double a, double cs2, double rho,
                     double ux, double uy, double* feq)
{
    double Fi[81], kc[9] = {0}, m[9];
    kc[0] = rho;
    kc[3] = 2.0 * rho * cs2;
    kc[8] = rho * cs2 * cs2;
    build_F(a, -ux, -uy, Ti, Fi);
    matvec9(Fi, kc, m);
    matvec9(Ti, m, feq);
}

int orc_feq(double a, double cs2, double rho, double ux, double uy,
            double feq[9])
{
    double T[81], Ti[81];
    if (!(a > 0.0) || !feq) return -1;
    build_T(a, T);
    if (invert9(T, Ti)) return -1;
    feq_with(Ti, a, cs2, rho, ux, uy, feq);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Collision                                                                  */
/* ------------------------------------------------------------------------ */

/* The collision of one cell, RC-LBM (Sec. 4) or RNR-LBM (Sec. 3). */
static void collide(const orc_params* p, const double* T, const double* Ti,
                    const double* f, double dxr, double dyr, double* ft,
                    double* strain)
{
    const double a = p->a, cs2 = p->cs2;
    const double* w = p->omega;
    const double Fx = p->Fx, Fy = p->Fy;
    double m[9];

    /* Pre-collision raw moments m = T f (Sec. 3/4, first step). */
    matvec9(T, f, m);

    /* Hydrodynamic fields: rho = sum f, rho u = sum f e + F dt / 2. */
    const double rho = m[0];
    const double ux = (m[1] + 0.5 * Fx) / rho;
    const double uy = (m[2] + 0.5 * Fy) / rho;

    /* Eq. 12: raw equilibria of the square lattice, j = 3, 4 (the strain
     * rates use the literal non-equilibrium raw moments of Eq. 34-35). */
    const double meqr3 = 2.0 * rho * cs2 + rho * (ux * ux + uy * uy);
    const double meqr4 = rho * (ux * ux - uy * uy);

    /* Eq. 40: coefficients of the local strain-rate expressions. */
    const double w3 = w[3], w4 = w[4];
    const double B1 = rho * (-2.0 * cs2 / w3 - (-3.0 * cs2 + 1.0) / 2.0
                             + 3.0 * ux * ux / 2.0);
    const double B2 = rho * (-2.0 * cs2 / w3 - (-3.0 * cs2 + a * a) / 2.0
                             + 3.0 * uy * uy / 2.0);
    const double B3 = ((3.0 * cs2 - 1.0) / 2.0) * ux;
    const double B4 = ((3.0 * cs2 - a * a) / 2.0) * uy;
    const double C1 = rho * (-2.0 * cs2 / w4 - (-3.0 * cs2 + 1.0) / 2.0
                             + 3.0 * ux * ux / 2.0);
    const double C2 = rho * (2.0 * cs2 / w4 - (3.0 * cs2 - a * a) / 2.0
                             - 3.0 * uy * uy / 2.0);
    const double C3 = ((3.0 * cs2 - 1.0) / 2.0) * ux;
    const double C4 = ((-3.0 * cs2 + a * a) / 2.0) * uy;

    /* Eq. 37-38. */
    const double R3 = m[3] - meqr3 - B3 * dxr - B4 * dyr;
    const double R4 = m[4] - meqr4 - C3 * dxr - C4 * dyr;
    const double dxux = (C2 * R3 - B2 * R4) / (C2 * B1 - C1 * B2);
    const double dyuy = (C1 * R3 - B1 * R4) / (C1 * B2 - C2 * B1);
    if (strain) {
        strain[0] = dxux;
        strain[1] = dyuy;
    }

    /* Eq. 23-26 (Eq. 27: no correction on the off-diagonal moment). */
    const double l3 = 1.0 / w3 - 0.5, l4 = 1.0 / w4 - 0.5;
    double m3s = l3 * ((-3.0 * cs2 + 1.0) * rho * dxux
                       + (-3.0 * cs2 + a * a) * rho * dyuy
                       + (-3.0 * cs2 + 1.0) * ux * dxr
                       + (-3.0 * cs2 + a * a) * uy * dyr);
    double m4s = l4 * ((-3.0 * cs2 + 1.0) * rho * dxux
                       + (3.0 * cs2 - a * a) * rho * dyuy
                       + (-3.0 * cs2 + 1.0) * ux * dxr
                       + (3.0 * cs2 - a * a) * uy * dyr);
    double m3G = -3.0 * rho * l3 * (ux * ux * dxux + uy * uy * dyuy);
    double m4G = -3.0 * rho * l4 * (ux * ux * dxux - uy * uy * dyuy);
    if (!p->use_iso_corr) m3s = m4s = 0.0;
    if (!p->use_gi_corr) m3G = m4G = 0.0;

    double mt[9];
    if (p->scheme == 0) {
        /* RC-LBM, Sec. 4. */
        double F[81], Fi[81], mc[9], mceq[9], phic[9], mct[9];
        build_F(a, ux, uy, Ti, F);
        build_F(a, -ux, -uy, Ti, Fi);
        matvec9(F, m, mc); /* m^c = F m */
        /* Eq. 49 with dt = 1. */
        mceq[0] = rho;
        mceq[1] = 0.0;
        mceq[2] = 0.0;
        mceq[3] = 2.0 * rho * cs2 + m3s + m3G;
        mceq[4] = m4s + m4G;
        mceq[5] = 0.0;
        mceq[6] = 0.0;
        mceq[7] = 0.0;
        mceq[8] = rho * cs2 * cs2;
        /* Central moments of the source (Sec. 4). */
        for (int j = 0; j < 9; ++j) phic[j] = 0.0;
        phic[1] = Fx;
        phic[2] = Fy;
        for (int j = 0; j < 9; ++j)
            mct[j] = mc[j] + w[j] * (mceq[j] - mc[j])
                     + (1.0 - w[j] / 2.0) * phic[j];
        matvec9(Fi, mct, mt); /* m~ = F^-1 m~^c */
    } else {
        /* RNR-LBM, Sec. 3: Eq. 10-13 in raw-moment space.  m^{eq,r}_8 is the
         * binomial transform of the Maxwell-matched central moments,
         * rho cs2^2 + rho cs2 (ux^2 + uy^2) + rho ux^2 uy^2 (Eq. 12 prints the
         * middle coefficient as 3, which contradicts its own construction and
         * Eq. 55). */
        double meq[9], phi[9];
        meq[0] = rho;
        meq[1] = rho * ux;
        meq[2] = rho * uy;
        meq[3] = meqr3 + m3s + m3G;
        meq[4] = meqr4 + m4s + m4G;
        meq[5] = rho * ux * uy;
        meq[6] = cs2 * rho * uy + rho * ux * ux * uy;
        meq[7] = cs2 * rho * ux + rho * ux * uy * uy;
        meq[8] = rho * cs2 * cs2 + rho * cs2 * (ux * ux + uy * uy)
                 + rho * ux * ux * uy * uy;
        /* Eq. 13. */
        phi[0] = 0.0;
        phi[1] = Fx;
        phi[2] = Fy;
        phi[3] = 2.0 * (Fx * ux + Fy * uy);
        phi[4] = 2.0 * (Fx * ux - Fy * uy);
        phi[5] = Fx * uy + Fy * ux;
        phi[6] = Fy * ux * ux + 2.0 * Fx * ux * uy;
        phi[7] = Fx * uy * uy + 2.0 * Fy * uy * ux;
        phi[8] = 2.0 * (Fx * ux * uy * uy + Fy * uy * ux * ux);
        for (int j = 0; j < 9; ++j)
            mt[j] = m[j] + w[j] * (meq[j] - m[j]) + (1.0 - w[j] / 2.0) * phi[j];
    }
    matvec9(Ti, mt, ft); /* f~ = T^-1 m~ */
}

static int check_params(const orc_params* p)
{
    if (!p) return -1;
    if (p->nx < 3 || p->ny < 3) return -1;
    if (!(p->a > 0.0) || !isfinite(p->a)) return -1;
    if (!(p->cs2 > 0.0) || !(p->cs2 < 1.0) || !(p->cs2 < p->a * p->a))
        return -1;
    for (int j = 0; j < 9; ++j)
        if (!(p->omega[j] >= 0.0 && p->omega[j] <= 2.0)) return -1;
    if (!(p->omega[3] > 0.0) || !(p->omega[4] > 0.0)) return -1;
    if (p->scheme != 0 && p->scheme != 1) return -1;
    return 0;
}

int orc_collide_cell(const orc_params* p, const double f[9], double dxrho,
                     double dyrho, double ft[9], double strain[2])
{
    double T[81], Ti[81];
    if (!p || !f || !ft || !(p->a > 0.0) || !(p->omega[3] > 0.0) || !(p->omega[4] > 0.0))
        return -1;
    build_T(p->a, T);
    if (invert9(T, Ti)) return -1;
    collide(p, T, Ti, f, dxrho, dyrho, ft, strain);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lattice                                                                    */
/* ------------------------------------------------------------------------ */

/* Node (x+dx, y+dy) of the lattice.  Periodic axes wrap.  Returns 1 and its
 * index when the node is a fluid cell; returns 0 when it is a wall or solid
 * node, and then writes that node's velocity to uw (nullable). */
static int locate(const orc* o, int x, int y, int dx, int dy, int* idx,
                  double* uw)
{
    const int nx = o->p.nx, ny = o->p.ny;
    int X = x + dx, Y = y + dy, outx = 0, outy = 0;
    if (X < 0 || X >= nx) {
        if (o->p.periodic_x) X = (X + nx) % nx;
        else outx = (X < 0) ? -1 : 1;
    }
    if (Y < 0 || Y >= ny) {
        if (o->p.periodic_y) Y = (Y + ny) % ny;
        else outy = (Y < 0) ? -1 : 1;
    }
    if (outy) { /* bottom / top wall, corners included */
        const int k = outy < 0 ? 2 : 3;
        if (uw) { uw[0] = o->p.wall_u[k][0]; uw[1] = o->p.wall_u[k][1]; }
        return 0;
    }
    if (outx) {
        const int k = outx < 0 ? 0 : 1;
        if (uw) { uw[0] = o->p.wall_u[k][0]; uw[1] = o->p.wall_u[k][1]; }
        return 0;
    }
    const int id = Y * nx + X;
    if (o->solid[id]) {
        if (uw) uw[0] = uw[1] = 0.0;
        return 0;
    }
    if (idx) *idx = id;
    return 1;
}

static int nthreads_of(const orc* o)
{
#ifdef _OPENMP
    return o->p.nthreads > 0 ? o->p.nthreads : omp_get_max_threads();
#else
    (void)o;
    return 1;
#endif
}

orc* orc_create(const orc_params* p, const unsigned char* solid)
{
    if (check_params(p)) return NULL;
    orc* o = (orc*)calloc(1, sizeof(orc));
    if (!o) return NULL;
    o->p = *p;
    o->N = p->nx * p->ny;
    const size_t N = (size_t)o->N;
    o->solid = (unsigned char*)calloc(N, 1);
    o->f = (double*)calloc(9 * N, sizeof(double));
    o->ft = (double*)calloc(9 * N, sizeof(double));
    o->rho = (double*)calloc(N, sizeof(double));
    o->dxr = (double*)calloc(N, sizeof(double));
    o->dyr = (double*)calloc(N, sizeof(double));
    if (!o->solid || !o->f || !o->ft || !o->rho || !o->dxr || !o->dyr) {
        orc_destroy(o);
        return NULL;
    }
    build_T(p->a, o->T);
    if (invert9(o->T, o->Ti)) {
        orc_destroy(o);
        return NULL;
    }
    if (solid)
        for (size_t c = 0; c < N; ++c) o->solid[c] = solid[c] ? 1 : 0;
    /* A fluid cell whose 8 neighbours are all wall/solid nodes exchanges
     * nothing with the flow; it is made solid. */
    unsigned char* iso = (unsigned char*)calloc(N, 1);
    if (!iso) {
        orc_destroy(o);
        return NULL;
    }
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const int c = y * p->nx + x;
            if (o->solid[c]) continue;
            int open = 0;
            for (int i = 1; i < 9; ++i)
                open += locate(o, x, y, EX[i], EY[i], NULL, NULL);
            iso[c] = (open == 0);
        }
    for (size_t c = 0; c < N; ++c)
        if (iso[c]) o->solid[c] = 1;
    free(iso);
    orc_init_fields(o, NULL, NULL, NULL);
    return o;
}

void orc_destroy(orc* o)
{
    if (!o) return;
    free(o->solid);
    free(o->f);
    free(o->ft);
    free(o->rho);
    free(o->dxr);
    free(o->dyr);
    free(o);
}

int orc_init_fields(orc* o, const double* rho, const double* ux,
                    const double* uy)
{
    if (!o) return -1;
    const int N = o->N;
#pragma omp parallel for num_threads(nthreads_of(o)) schedule(static)
    for (int c = 0; c < N; ++c) {
        double feq[9] = {0};
        if (!o->solid[c])
            feq_with(o->Ti, o->p.a, o->p.cs2, rho ? rho[c] : 1.0,
                     ux ? ux[c] : 0.0, uy ? uy[c] : 0.0, feq);
        for (int i = 0; i < 9; ++i) o->f[(size_t)i * N + c] = feq[i];
    }
    return 0;
}

int orc_set_f(orc* o, const double* f)
{
    if (!o || !f) return -1;
    memcpy(o->f, f, sizeof(double) * 9 * (size_t)o->N);
    return 0;
}

int orc_get_f(const orc* o, double* f)
{
    if (!o || !f) return -1;
    memcpy(f, o->f, sizeof(double) * 9 * (size_t)o->N);
    return 0;
}

int orc_set_force(orc* o, double Fx, double Fy)
{
    if (!o) return -1;
    o->p.Fx = Fx;
    o->p.Fy = Fy;
    return 0;
}

/* rho = sum_i f_i at every fluid cell (solid cells: 0). */
static void density(orc* o)
{
    const int N = o->N;
#pragma omp parallel for num_threads(nthreads_of(o)) schedule(static)
    for (int c = 0; c < N; ++c) {
        double s = 0.0;
        if (!o->solid[c])
            for (int i = 0; i < 9; ++i) s += o->f[(size_t)i * N + c];
        o->rho[c] = s;
    }
}

/* Density gradient by central differences at the same time level: spacing
 * 2 dx = 2 along x and 2 dy = 2a along y; the density of a wall or solid
 * neighbour is taken equal to the cell's own (zero normal gradient). */
static void density_gradient(orc* o)
{
    const int nx = o->p.nx, ny = o->p.ny;
#pragma omp parallel for num_threads(nthreads_of(o)) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int c = y * nx + x;
            if (o->solid[c]) {
                o->dxr[c] = o->dyr[c] = 0.0;
                continue;
            }
            int n;
            const double r0 = o->rho[c];
            const double rE = locate(o, x, y, 1, 0, &n, NULL) ? o->rho[n] : r0;
            const double rW = locate(o, x, y, -1, 0, &n, NULL) ? o->rho[n] : r0;
            const double rN = locate(o, x, y, 0, 1, &n, NULL) ? o->rho[n] : r0;
            const double rS = locate(o, x, y, 0, -1, &n, NULL) ? o->rho[n] : r0;
            o->dxr[c] = (rE - rW) / 2.0;
            o->dyr[c] = (rN - rS) / (2.0 * o->p.a);
        }
}

static void one_step(orc* o)
{
    const int nx = o->p.nx, ny = o->p.ny, N = o->N;
    const size_t NN = (size_t)N;
    const int nt = nthreads_of(o);

    density(o);
    density_gradient(o);

    /* Collision at every fluid cell. */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int c = 0; c < N; ++c) {
        if (o->solid[c]) continue;
        double f[9], ft[9];
        for (int i = 0; i < 9; ++i) f[i] = o->f[i * NN + c];
        collide(&o->p, o->T, o->Ti, f, o->dxr[c], o->dyr[c], ft, NULL);
        for (int i = 0; i < 9; ++i) o->ft[i * NN + c] = ft[i];
    }

    /* Streaming, f_i(x, t+1) = f~_i(x - e_i, t), from fluid sources. */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int c = y * nx + x;
            if (o->solid[c]) continue;
            for (int i = 0; i < 9; ++i) {
                int s;
                if (locate(o, x, y, -EX[i], -EY[i], &s, NULL))
                    o->f[i * NN + c] = o->ft[i * NN + s];
            }
        }

    /* Half-way bounce-back for links whose source is a wall or solid node:
     * f_i(x_f, t+1) = f~_opp(x_f, t) - (f^eq_opp - f^eq_i)(rho_w, U_w) with
     * rho_w the density of the fluid cell x_f (Sec. 5.2; Eq. 57-59 are this
     * formula at the top wall).  A stationary node needs no correction. */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int c = y * nx + x;
            if (o->solid[c]) continue;
            for (int i = 1; i < 9; ++i) {
                double uw[2];
                if (locate(o, x, y, -EX[i], -EY[i], NULL, uw)) continue;
                double v = o->ft[OPP[i] * NN + c];
                if (uw[0] != 0.0 || uw[1] != 0.0) {
                    double feq[9];
                    feq_with(o->Ti, o->p.a, o->p.cs2, o->rho[c], uw[0], uw[1],
                             feq);
                    v -= feq[OPP[i]] - feq[i];
                }
                o->f[i * NN + c] = v;
            }
        }
}

int orc_step(orc* o, long n)
{
    if (!o || n < 0) return -1;
    for (long k = 0; k < n; ++k) one_step(o);
    return 0;
}

int orc_moments(const orc* o, double* rho, double* ux, double* uy)
{
    if (!o) return -1;
    const int N = o->N;
    const double a = o->p.a;
#pragma omp parallel for num_threads(nthreads_of(o)) schedule(static)
    for (int c = 0; c < N; ++c) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        if (!o->solid[c]) {
            for (int i = 0; i < 9; ++i) {
                const double fi = o->f[(size_t)i * N + c];
                r += fi;
                jx += fi * EX[i];
                jy += fi * (a * EY[i]);
            }
        }
        if (rho) rho[c] = r;
        if (ux) ux[c] = o->solid[c] ? 0.0 : (jx + 0.5 * o->p.Fx) / r;
        if (uy) uy[c] = o->solid[c] ? 0.0 : (jy + 0.5 * o->p.Fy) / r;
    }
    return 0;
}

int orc_strain(const orc* o, double* dxux, double* dyuy)
{
    if (!o) return -1;
    orc* w = (orc*)o; /* refreshes the rho / gradient scratch only */
    density(w);
    density_gradient(w);
    const int N = o->N;
#pragma omp parallel for num_threads(nthreads_of(o)) schedule(static)
    for (int c = 0; c < N; ++c) {
        double f[9], ft[9], st[2] = {0.0, 0.0};
        if (!o->solid[c]) {
            for (int i = 0; i < 9; ++i) f[i] = o->f[(size_t)i * N + c];
            collide(&o->p, o->T, o->Ti, f, o->dxr[c], o->dyr[c], ft, st);
        }
        if (dxux) dxux[c] = st[0];
        if (dyuy) dyuy[c] = st[1];
    }
    return 0;
}

int orc_stress(const orc* o, double* sxy, double* txx, double* tyy,
               double* txy)
{
    if (!o) return -1;
    orc* w = (orc*)o; /* refreshes the rho / gradient scratch only */
    density(w);
    density_gradient(w);
    const int N = o->N;
    const double cs2 = o->p.cs2;
    const double* om = o->p.omega;
    /* Eq. 32-33: shear viscosity from omega_4 (normal) and omega_5 (shear),
     * bulk viscosity from omega_3. */
    const double nu4 = cs2 * (1.0 / om[4] - 0.5);
    const double nu5 = cs2 * (1.0 / om[5] - 0.5);
    const double zeta = cs2 * (1.0 / om[3] - 0.5);
#pragma omp parallel for num_threads(nthreads_of(o)) schedule(static)
    for (int c = 0; c < N; ++c) {
        double f[9], ft[9], m[9], st[2] = {0.0, 0.0};
        double shear = 0.0, rho = 0.0;
        if (!o->solid[c]) {
            for (int i = 0; i < 9; ++i) f[i] = o->f[(size_t)i * N + c];
            collide(&o->p, o->T, o->Ti, f, o->dxr[c], o->dyr[c], ft, st);
            matvec9(o->T, f, m);
            rho = m[0];
            const double ux = (m[1] + 0.5 * o->p.Fx) / rho;
            const double uy = (m[2] + 0.5 * o->p.Fy) / rho;
            /* Eq. 39 with Eq. 36 and D1 of Eq. 40 (left side read as
             * d_y u_x + d_x u_y, as Eq. 21 gives it). */
            const double D1 = -rho * cs2 / om[5];
            shear = (m[5] - rho * ux * uy) / D1;
        }
        const double div = st[0] + st[1];
        if (sxy) sxy[c] = shear;
        if (txx) txx[c] = rho * (nu4 * (2.0 * st[0] - div) + zeta * div);
        if (tyy) tyy[c] = rho * (nu4 * (2.0 * st[1] - div) + zeta * div);
        if (txy) txy[c] = rho * nu5 * shear;
    }
    return 0;
}

int orc_solid(const orc* o, unsigned char* solid)
{
    if (!o || !solid) return -1;
    memcpy(solid, o->solid, (size_t)o->N);
    return 0;
}

int orc_threads(const orc* o)
{
    if (!o) return -1;
    return nthreads_of(o);
}
