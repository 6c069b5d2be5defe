/* Drives every entry point of the FP64 oracle (test infrastructure) on tiny
 * and ragged lattices -- walls, moving walls, solid cells, a body force,
 * both schemes, a < 1 and a > 1 -- and its argument checks, for a build
 * under AddressSanitizer and UndefinedBehaviorSanitizer.  Exit status 0 and
 * "ok" mean no sanitizer report (they abort on the first one) and every
 * result finite. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "rclbm_oracle.h"

static int fails = 0;
#define CHECK(c)                                                          \
    do {                                                                  \
        if (!(c)) {                                                       \
            fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
            ++fails;                                                      \
        }                                                                 \
    } while (0)

static void set_omega(orc_params* p) {
    for (int i = 0; i < 9; ++i) p->omega[i] = 1.0;
    p->omega[4] = p->omega[5] = 1.6;
}

static void run_case(int nx, int ny, double a, double cs2, int px, int py, int scheme,
                     int with_solid, double Fx, double Fy, double lid) {
    orc_params p;
    memset(&p, 0, sizeof p);
    p.nx = nx;
    p.ny = ny;
    p.a = a;
    p.cs2 = cs2;
    set_omega(&p);
    p.Fx = Fx;
    p.Fy = Fy;
    p.periodic_x = px;
    p.periodic_y = py;
    p.wall_u[3][0] = lid;
    p.use_iso_corr = 1;
    p.use_gi_corr = 1;
    p.scheme = scheme;
    p.nthreads = 0;  /* the runtime default (OMP_NUM_THREADS) */
    const int N = nx * ny;
    unsigned char* solid = NULL;
    if (with_solid) {
        solid = (unsigned char*)calloc((size_t)N, 1);
        for (int c = 0; c < N; c += 7) solid[c] = 1;
    }
    orc* o = orc_create(&p, solid);
    CHECK(o != NULL);
    if (!o) {
        free(solid);
        return;
    }
    double* rho = (double*)malloc(sizeof(double) * N);
    double* ux = (double*)malloc(sizeof(double) * N);
    double* uy = (double*)malloc(sizeof(double) * N);
    double* f = (double*)malloc(sizeof(double) * 9 * N);
    double* w[4];
    for (int k = 0; k < 4; ++k) w[k] = (double*)malloc(sizeof(double) * N);
    for (int c = 0; c < N; ++c) {
        rho[c] = 1.0 + 1e-3 * sin(0.7 * c);
        ux[c] = 0.02 * cos(0.3 * c);
        uy[c] = -0.01 * sin(0.5 * c);
    }
    CHECK(orc_init_fields(o, rho, ux, uy) == 0);
    CHECK(orc_init_fields(o, NULL, NULL, NULL) == 0);
    CHECK(orc_init_fields(o, rho, ux, uy) == 0);
    CHECK(orc_step(o, 3) == 0);
    CHECK(orc_get_f(o, f) == 0);
    CHECK(orc_set_f(o, f) == 0);
    CHECK(orc_set_force(o, Fx * 0.5, Fy * 0.5) == 0);
    CHECK(orc_step(o, 4) == 0);
    CHECK(orc_moments(o, rho, ux, uy) == 0);
    CHECK(orc_strain(o, w[0], w[1]) == 0);
    CHECK(orc_stress(o, w[0], w[1], w[2], w[3]) == 0);
    CHECK(orc_stress(o, NULL, NULL, NULL, w[3]) == 0);
    unsigned char* s2 = (unsigned char*)malloc((size_t)N);
    CHECK(orc_solid(o, s2) == 0);
    CHECK(orc_threads(o) >= 1);
    CHECK(orc_get_f(o, f) == 0);
    for (int i = 0; i < 9 * N; ++i) CHECK(isfinite(f[i]));
    for (int c = 0; c < N; ++c) CHECK(isfinite(rho[c]) && isfinite(ux[c]) && isfinite(uy[c]));
    free(s2);
    for (int k = 0; k < 4; ++k) free(w[k]);
    free(f);
    free(uy);
    free(ux);
    free(rho);
    orc_destroy(o);
    free(solid);
}

int main(void) {
    /* one-cell entry points */
    double T[81], Ti[81], F[81], Fi[81], kc[9], feq[9], ft[9], st[2];
    CHECK(orc_matrices(0.5, 0.02, -0.01, T, Ti, F, Fi) == 0);
    CHECK(orc_feq(0.5, 0.075, 1.001, 0.02, -0.01, feq) == 0);
    CHECK(orc_central_moments(0.5, feq, 0.02, -0.01, kc) == 0);
    orc_params p;
    memset(&p, 0, sizeof p);
    p.nx = p.ny = 3;
    p.a = 0.5;
    p.cs2 = 0.075;
    set_omega(&p);
    p.use_iso_corr = p.use_gi_corr = 1;
    CHECK(orc_collide_cell(&p, feq, 1e-4, -2e-4, ft, st) == 0);
    CHECK(orc_collide_cell(&p, feq, 1e-4, -2e-4, ft, NULL) == 0);
    p.scheme = 1;
    CHECK(orc_collide_cell(&p, feq, 1e-4, -2e-4, ft, st) == 0);
    /* rejected arguments */
    orc_params bad = p;
    bad.nx = 2;
    CHECK(orc_create(&bad, NULL) == NULL);
    bad = p;
    bad.a = 0.0;
    CHECK(orc_create(&bad, NULL) == NULL);
    bad = p;
    bad.cs2 = 0.3;  /* >= a^2 */
    CHECK(orc_create(&bad, NULL) == NULL);
    CHECK(orc_create(NULL, NULL) == NULL);
    CHECK(orc_step(NULL, 1) < 0);
    CHECK(orc_get_f(NULL, ft) < 0);
    CHECK(orc_feq(0.5, 0.075, 1.0, 0.0, 0.0, NULL) < 0);
    CHECK(orc_matrices(0.5, 0.0, 0.0, T, NULL, F, Fi) < 0);
    CHECK(orc_central_moments(0.5, NULL, 0.0, 0.0, kc) < 0);
    CHECK(orc_collide_cell(&p, feq, 0.0, 0.0, NULL, st) < 0);
    /* lattices */
    run_case(3, 3, 1.0, 1.0 / 3.0, 1, 1, 0, 0, 0.0, 0.0, 0.0);
    run_case(5, 3, 0.5, 0.075, 0, 0, 0, 0, 0.0, 0.0, 0.03);
    run_case(5, 3, 0.5, 0.075, 0, 0, 1, 0, 0.0, 0.0, 0.03);
    run_case(7, 9, 2.0, 1.0 / 3.0, 1, 0, 0, 1, 1e-5, 0.0, 0.0);
    run_case(7, 9, 0.25, 0.01875, 0, 1, 1, 1, 0.0, 2e-5, 0.0);
    run_case(31, 17, 0.8, 0.19, 0, 0, 0, 1, 1e-5, -1e-5, 0.05);
    if (fails) {
        fprintf(stderr, "%d checks failed\n", fails);
        return 1;
    }
    printf("ok\n");
    return 0;
}
