/*
 * rclbm_oracle.h -- FP64 CPU oracle of the rectangular central-moment lattice
 * Boltzmann method (RC-LBM) and of its raw-moment special case (RNR-LBM),
 * Yahia & Premnath, "Central Moment Lattice Boltzmann Method on a Rectangular
 * Lattice" (arXiv 2103.02119).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA library
 * against the paper. Only the test suite, the smoke check and the timed CPU
 * baseline of the benchmark may load it; the product path never does.
 *
 * Conventions (shared by every entry point below):
 *   - D2Q9 velocities of Eq. 2, lattice units dx = dt = 1, dy = a, so the
 *     y component of e_i is +-a.  Direction order 0..8 is the order of Eq. 2.
 *   - Cell (x, y), 0 <= x < nx, 0 <= y < ny, has linear index y*nx + x.
 *   - Distribution arrays are plane-major: f[i*N + y*nx + x], N = nx*ny.
 *   - An axis that is not periodic is closed by half-way bounce-back walls
 *     on both of its ends (Sec. 5.1); wall_u gives each wall's velocity,
 *     index 0 = left (x = -1), 1 = right (x = nx), 2 = bottom (y = -1),
 *     3 = top (y = ny).  A node outside the domain in both x and y (a corner)
 *     belongs to the bottom/top wall.
 *   - solid[] (nullable) marks solid nodes (non-zero) inside the domain;
 *     they are stationary.  A fluid cell whose 8 neighbours are all wall or
 *     solid nodes is turned into a solid node when the oracle is created.
 *   - All functions return 0 on success and a negative value on invalid
 *     arguments.
 */
#ifndef RCLBM_ORACLE_H
#define RCLBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;                 /* cells along x and y, each >= 3            */
    double a;                   /* grid aspect ratio dy/dx (Sec. 2.1), > 0   */
    double cs2;                 /* c_s^2, 0 < cs2 < min(1, a^2)              */
    double omega[9];            /* relaxation rates w_0..w_8 (Eq. 5)         */
    double Fx, Fy;              /* uniform body-force density (Eq. 13)       */
    int periodic_x, periodic_y; /* 1 = periodic axis, 0 = walls on both ends */
    double wall_u[4][2];        /* wall velocities (Ux, Uy), see above       */
    int use_iso_corr;           /* 1: include m^{eq,s} (Eq. 23-24)           */
    int use_gi_corr;            /* 1: include m^{eq,G} (Eq. 25-26)           */
    int scheme;                 /* 0 = RC-LBM (Sec. 4), 1 = RNR-LBM (Sec. 3) */
    int nthreads;               /* OpenMP threads, 0 = runtime default       */
} orc_params;

typedef struct orc orc;

/* T (Eq. 4) from the monomials of Eq. 3, T^-1 by numerical inversion,
 * F(u) = frame transformation of App. B (raw -> central moments) built from
 * its definition, Fi = F(-u).  All 9x9 row-major. */
int orc_matrices(double a, double ux, double uy,
                 double T[81], double Ti[81], double F[81], double Fi[81]);

/* Central moments of one cell by the definition of Eq. 43, in the order of
 * Eq. 46. */
int orc_central_moments(double a, const double f[9], double ux, double uy,
                        double kc[9]);

/* Equilibrium f^eq = T^-1 F(-u) m^{c,eqr}(rho) (Sec. 4, central moment
 * equilibria of the square lattice mapped back to populations). */
int orc_feq(double a, double cs2, double rho, double ux, double uy,
            double feq[9]);

/* One-cell collision (pre-collision f -> post-collision ft) with the given
 * density gradient.  strain (nullable) receives (d_x u_x, d_y u_y) of
 * Eq. 37-38. */
int orc_collide_cell(const orc_params* p, const double f[9], double dxrho,
                     double dyrho, double ft[9], double strain[2]);

orc* orc_create(const orc_params* p, const unsigned char* solid);
void orc_destroy(orc* o);
/* f = f^eq(rho, u) everywhere (nullable arrays: rho = 1, u = 0). */
int orc_init_fields(orc* o, const double* rho, const double* ux,
                    const double* uy);
int orc_set_f(orc* o, const double* f);   /* copy in a 9*N state  */
int orc_get_f(const orc* o, double* f);   /* copy out a 9*N state */
int orc_set_force(orc* o, double Fx, double Fy);
/* Advance n time steps: collide, stream, update the macroscopic fields. */
int orc_step(orc* o, long n);
/* rho and u = (sum f e + F/2)/rho of the current state; solid cells -> 0. */
int orc_moments(const orc* o, double* rho, double* ux, double* uy);
/* Local strain rates (Eq. 37-38) the next collision would use; solid -> 0. */
int orc_strain(const orc* o, double* dxux, double* dyuy);
/* Off-diagonal strain rate d_y u_x + d_x u_y of Eq. 39 (its left side read
 * as the off-diagonal rate, as Eq. 21 gives it) and the viscous stress of the
 * Navier-Stokes equations the scheme recovers (Eq. 30-33):
 *   txx = rho [nu (2 d_x u_x - div u) + zeta div u], tyy likewise,
 *   txy = rho nu (d_y u_x + d_x u_y),
 * nu = cs2 (1/omega_4 - 1/2) for the normal and cs2 (1/omega_5 - 1/2) for
 * the shear stress, zeta = cs2 (1/omega_3 - 1/2), with the local rates of
 * Eq. 37-39 the next collision would use.  Nullable outputs; solid -> 0. */
int orc_stress(const orc* o, double* sxy, double* txx, double* tyy,
               double* txy);
/* The solid map in use (after the isolated-cell rule), N bytes. */
int orc_solid(const orc* o, unsigned char* solid);
int orc_threads(const orc* o);

#ifdef __cplusplus
}
#endif
#endif
