// lbm_device.cuh -- device-side building blocks of the RC-LBM step
// (Yahia & Premnath, arXiv 2103.02119, Sec. 4), for FP32 and FP64.
//
// Storage: nine population planes of rows padded to `pitch` values (x
// fastest); population i of cell (x, y) sits at i * plane + y * rstride + x,
// so one layout keeps each plane contiguous (plane = pitch * ny,
// rstride = pitch) and the other interleaves the nine planes row by row
// (plane = pitch, rstride = 9 * pitch).  The values are deviations fhat_i = f_i - w_i rho0 from
// the rest equilibrium.  The stored state of a time step is the
// post-collision field f~ (pull scheme): the next step streams by gathering
// f_i(x) = f~_i(x - e_i) (Sec. 4, streaming step), and a link whose source
// is a wall or solid node reads back the cell's own outgoing population
// f~_opp(i)(x) (half-way bounce-back, Sec. 5.1).  The moving-wall term of
// Eq. 57-59 is added when that outgoing population is stored, with the
// density of the colliding cell.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

// Eq. 2, in cell units: e_x and e_y / a.
__host__ __device__ constexpr int ex(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}

// Kernel parameters, converted once on the host to the arithmetic type T.
template <typename T>
struct KParams {
    int nx, ny, pitch;        // pitch: padded row length (also of the link mask)
    long long plane;          // element stride between population planes
    int rstride;              // element stride between rows of a plane
    int px, py;               // periodic along x / y
    int moving;               // some wall moves
    int collide;              // 0: streaming and bounce-back only
    int raw;                  // 1: raw-moment collision (RNR-LBM, Sec. 3)
    T a, iah, ia2, iah2;      // a, 1/(2a), 1/a^2, 1/(2a^2)
    T a2, cs2, cs4, rho0;
    T w3, w4, w5, w6, w7, w8; // relaxation rates
    T lw3, lw4;               // w_j (1/w_j - 1/2) = 1 - w_j/2
    T lw5, lw6, lw7, lw8;     // 1 - w_j/2 (raw source moments, RNR-LBM)
    T g1i, g2i, g3;           // iso * (1 - 3cs2), iso * (a^2 - 3cs2), gi * 3
    T g1h, g2h;               // (1 - 3cs2)/2, (a^2 - 3cs2)/2 (strain solve)
    T b1c, b2c, c1c, c2c;     // rho-free, u-free parts of B1, B2, C1, C2 (Eq. 40)
    T Fx, Fy, hFx, hFy;       // force and half force
    T wall_u[4][2];
    const uint8_t* __restrict__ lmask;  // per-cell link mask (nullable)
    int* status;                        // bit 0: a bounded wait ran out
};

// Host/device double-precision parameters for the auxiliary kernels.
struct AuxParams {
    int nx, ny, pitch;
    long long plane;
    int rstride;
    int px, py;
    double a, cs2, rho0, Fx, Fy;
    double wrest[9];          // rest weights times rho0
    double w3, w4, w5;        // relaxation rates of the second-order moments
    const uint8_t* __restrict__ lmask;
};

// Bit i-1 (i = 1..8) is set when the source node x - e_i of direction i is a
// wall or solid node.  With a mask the bits are precomputed per cell (0xFF
// marks a solid cell); without one the walls are the non-periodic domain
// edges.
template <bool MASK, typename P>
__device__ __forceinline__ unsigned link_bits(const P& p, int x, int y) {
    if (MASK) return p.lmask[(long long)y * p.pitch + x];
    const unsigned W = (x == 0) & !p.px, E = (x == p.nx - 1) & !p.px;
    const unsigned S = (y == 0) & !p.py, N = (y == p.ny - 1) & !p.py;
    return W | (S << 1) | (E << 2) | (N << 3) | ((W | S) << 4) | ((E | S) << 5) |
           ((E | N) << 6) | ((W | N) << 7);
}

// Pull-stream the nine populations of cell (x, y) (Sec. 4, streaming step;
// half-way bounce-back for wall/solid sources).  `sb` are the link bits of
// the cell.
template <typename S, typename P>
__device__ __forceinline__ void pull(const S* __restrict__ fin, const P& p, int x,
                                     int y, unsigned sb, S f[9]) {
    const int xm = x == 0 ? p.nx - 1 : x - 1;
    const int xp = x == p.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? p.ny - 1 : y - 1;
    const int yp = y == p.ny - 1 ? 0 : y + 1;
    const long long pl = p.plane;
    const long long rc = (long long)y * p.rstride, rm = (long long)ym * p.rstride,
                    rp = (long long)yp * p.rstride;
    const long long c = rc + x;
    f[0] = __ldg(fin + c);
    f[1] = __ldg(fin + ((sb & 1u) ? 3 * pl + c : 1 * pl + rc + xm));
    f[2] = __ldg(fin + ((sb & 2u) ? 4 * pl + c : 2 * pl + rm + x));
    f[3] = __ldg(fin + ((sb & 4u) ? 1 * pl + c : 3 * pl + rc + xp));
    f[4] = __ldg(fin + ((sb & 8u) ? 2 * pl + c : 4 * pl + rp + x));
    f[5] = __ldg(fin + ((sb & 16u) ? 7 * pl + c : 5 * pl + rm + xm));
    f[6] = __ldg(fin + ((sb & 32u) ? 8 * pl + c : 6 * pl + rm + xp));
    f[7] = __ldg(fin + ((sb & 64u) ? 5 * pl + c : 7 * pl + rp + xp));
    f[8] = __ldg(fin + ((sb & 128u) ? 6 * pl + c : 8 * pl + rp + xm));
}

// Reciprocal used by the collision: FP32 takes the hardware approximation
// (at most 2 ulp off, below the FP32 storage rounding), FP64 an IEEE division.
__device__ __forceinline__ float rcp(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ double rcp(double v) { return 1.0 / v; }

// 1-D three-velocity Maxwell-matched factors of the equilibrium
// f_i^eq = rho phi_x(e_ix, u_x) phi_y(e_iy, u_y) (the tensor-product form of
// T^-1 F(-u) m^{c,eqr}).
template <typename T>
__device__ __forceinline__ T phi_x(int s, T u, T cs2) {
    return s == 0 ? T(1) - cs2 - u * u : T(0.5) * (cs2 + u * u + T(s) * u);
}
template <typename T>
__device__ __forceinline__ T phi_y(int s, T u, T cs2, T a, T iah2) {
    return s == 0 ? T(1) - (cs2 + u * u) * (T(2) * iah2)
                  : iah2 * (cs2 + u * u + T(s) * a * u);
}

// f^eq_k - f^eq_opp(k) at (rho, U): the moving-wall term of Sec. 5.2.
template <typename T>
__device__ __forceinline__ T eq_odd(int k, T rho, T Ux, T Uy, T cs2, T a, T iah2) {
    const int sx = ex(k), sy = ey(k);
    return rho * (phi_x<T>(sx, Ux, cs2) * phi_y<T>(sy, Uy, cs2, a, iah2) -
                  phi_x<T>(-sx, Ux, cs2) * phi_y<T>(-sy, Uy, cs2, a, iah2));
}

// Collision of one cell (Sec. 4) in increment form on deviations:
//   f~ = f + T^-1 F(-u) [ Lambda (m^{c,eq} - m^c) + (I - Lambda/2) Phi^c ].
// The D2Q9 basis of Eq. 3 is the tensor product {1, x, x^2} x {1, y, y^2},
// so T, F(u) and their inverses factor into 3x3 maps along x and along y:
// central moments are reduced column by column (over e_y, then e_x), and the
// increment is expanded back the same way.  The rest equilibrium rho0 w_i is
// carried analytically so that FP32 only ever adds small numbers.
//   f: deviations in, post-collision deviations out.  d = sum f (density
//   deviation).  dxr, dyr: density gradient.  Returns rho.
template <typename T>
__device__ __forceinline__ T collide(const KParams<T>& p, T f[9], T d, T dxr, T dyr) {
    const T rho = p.rho0 + d;
    const T jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
    const T jy = p.a * ((f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]));
    const T ir = rcp(rho);
    const T ux = (jx + p.hFx) * ir;
    const T uy = (jy + p.hFy) * ir;
    const T a = p.a, a2 = p.a2, cs2 = p.cs2;

    // Central moments along y of each column e_x = 0, +1, -1:
    // k0 = sum g, k1 = sum g (e_y - u_y), k2 = sum g (e_y - u_y)^2.
    T k0[3], k1[3], k2[3];
    {
        const T gz[3] = {f[0], f[1], f[3]}, gp[3] = {f[2], f[5], f[6]},
                gm[3] = {f[4], f[8], f[7]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T s = gp[c] + gm[c], dd = gp[c] - gm[c];
            k0[c] = gz[c] + s;
            k1[c] = a * dd - uy * k0[c];
            k2[c] = a2 * s - uy * (k1[c] + a * dd);
        }
    }
    // Along x: C[p][q] = sum_X (e_x - u_x)^p k_q(X).
    T C[3][3];
    {
        const T* kq[3] = {k0, k1, k2};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T S = kq[q][1] + kq[q][2], D = kq[q][1] - kq[q][2];
            C[0][q] = kq[q][0] + S;
            C[1][q] = D - ux * C[0][q];
            C[2][q] = S - ux * (C[1][q] + D);
        }
    }
    // Non-equilibrium central moments: subtract the Maxwell-matched values
    // (rho cs2 on xx and yy, rho cs2^2 on xxyy) and add back the central
    // moments of rho0 w about u.
    const T ux2 = ux * ux, uy2 = uy * uy;
    const T r0 = p.rho0;
    const T n20 = C[2][0] + r0 * ux2 - d * cs2;
    const T n02 = C[0][2] + r0 * uy2 - d * cs2;
    const T n11 = C[1][1] + r0 * ux * uy;
    const T n21 = C[2][1] - r0 * uy * (cs2 + ux2);
    const T n12 = C[1][2] - r0 * ux * (cs2 + uy2);
    const T n22 = C[2][2] + r0 * (cs2 * (ux2 + uy2) + ux2 * uy2) - d * p.cs4;
    const T k3 = n20 + n02, k4 = n20 - n02;

    // Local strain rates, Eq. 37-38, from the raw non-equilibrium moments of
    // Eq. 34-35 (central ones minus the force terms u.F).
    const T N3 = k3 - (ux * p.Fx + uy * p.Fy);
    const T N4 = k4 - (ux * p.Fx - uy * p.Fy);
    const T b1 = p.b1c + T(1.5) * ux2, b2 = p.b2c + T(1.5) * uy2;
    const T c1 = p.c1c + T(1.5) * ux2, c2 = p.c2c - T(1.5) * uy2;
    const T gx = p.g1h * ux * dxr, gy = p.g2h * uy * dyr;
    const T R3 = N3 + gx + gy;
    const T R4 = N4 + gx - gy;
    const T idet = rcp(rho * (b1 * c2 - b2 * c1));
    const T dxux = (c2 * R3 - b2 * R4) * idet;
    const T dyuy = (b1 * R4 - c1 * R3) * idet;

    // Corrections, Eq. 23-26: m3s + m3G = l3 (Px + Py), m4s + m4G = l4 (Px - Py).
    const T Px = p.g1i * (rho * dxux + ux * dxr) - p.g3 * rho * ux2 * dxux;
    const T Py = p.g2i * (rho * dyuy + uy * dyr) - p.g3 * rho * uy2 * dyuy;

    // Relaxation (Eq. 49 equilibria, Phi^c = (0, Fx, Fy, 0, ...)):
    // increments of the central moments.  kappa_1 = -Fx/2 before collision,
    // so its increment is Fx whatever omega_1 (same for y).
    const T dk3 = p.lw3 * (Px + Py) - p.w3 * k3;
    const T dk4 = p.lw4 * (Px - Py) - p.w4 * k4;
    const T D20 = T(0.5) * (dk3 + dk4), D02 = T(0.5) * (dk3 - dk4);
    const T D11 = -p.w5 * n11, D21 = -p.w6 * n21, D12 = -p.w7 * n12,
            D22 = -p.w8 * n22;

    // Back along x: central -> raw x-moments -> the three columns, for each q.
    T h[3][3];  // h[X][q], X = 0, +1, -1
    {
        const T Dq0[3] = {T(0), p.Fx, D20};
        const T Dq1[3] = {p.Fy, D11, D21};
        const T Dq2[3] = {D02, D12, D22};
        const T* Dq[3] = {Dq0, Dq1, Dq2};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T m0 = Dq[q][0];
            const T m1 = Dq[q][1] + ux * m0;
            const T m2 = Dq[q][2] + ux * (Dq[q][1] + m1);
            h[0][q] = m0 - m2;
            h[1][q] = T(0.5) * (m2 + m1);
            h[2][q] = T(0.5) * (m2 - m1);
        }
    }
    // Back along y for each column, and add the increment.
    {
        const int iz[3] = {0, 1, 3}, ip[3] = {2, 5, 6}, im[3] = {4, 8, 7};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T m0 = h[c][0];
            const T m1 = h[c][1] + uy * m0;
            const T m2 = h[c][2] + uy * (h[c][1] + m1);
            const T t2 = p.iah2 * m2, t1 = p.iah * m1;
            f[iz[c]] += m0 - p.ia2 * m2;
            f[ip[c]] += t2 + t1;
            f[im[c]] += t2 - t1;
        }
    }
    return rho;
}

// Collision of one cell of the raw-moment scheme (RNR-LBM, Sec. 3), in the
// increment form of collide():
//   f~ = f + T^-1 [ Lambda (m^eq - m) + (I - Lambda/2) Phi ]
// with the raw equilibria of Eq. 12 (m^eq_8 = rho cs2^2 + rho cs2 |u|^2 +
// rho ux^2 uy^2, the binomial transform of the central equilibria), the
// corrections of Eq. 23-26 on m3 and m4, and the raw source moments of
// Eq. 13.  The raw moments factor as R[p][q] = sum_i f_i e_ix^p e_iy^q, so
// the transforms are those of collide() at u = 0.  The strain rates
// (Eq. 37-38) and corrections are the same as in collide().
template <typename T>
__device__ __forceinline__ T collide_raw(const KParams<T>& p, T f[9], T d, T dxr, T dyr) {
    const T rho = p.rho0 + d;
    const T jx = (f[1] + f[5] + f[8]) - (f[3] + f[6] + f[7]);
    const T jy = p.a * ((f[2] + f[5] + f[6]) - (f[4] + f[7] + f[8]));
    const T ir = rcp(rho);
    const T ux = (jx + p.hFx) * ir;
    const T uy = (jy + p.hFy) * ir;
    const T a = p.a, a2 = p.a2, cs2 = p.cs2;

    // Raw moments along y of each column: k0 = sum g, k1 = sum g e_y,
    // k2 = sum g e_y^2; then along x: R[p][q] = sum_X e_x^p k_q(X).
    T k0[3], k1[3], k2[3];
    {
        const T gz[3] = {f[0], f[1], f[3]}, gp[3] = {f[2], f[5], f[6]},
                gm[3] = {f[4], f[8], f[7]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T sum = gp[c] + gm[c];
            k0[c] = gz[c] + sum;
            k1[c] = a * (gp[c] - gm[c]);
            k2[c] = a2 * sum;
        }
    }
    T R[3][3];
    {
        const T* kq[3] = {k0, k1, k2};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T S = kq[q][1] + kq[q][2];
            R[0][q] = kq[q][0] + S;
            R[1][q] = kq[q][1] - kq[q][2];
            R[2][q] = S;
        }
    }
    // Non-equilibrium raw moments m - m^{eq,r} (Eq. 12); the stored values
    // are deviations from rho0 w, whose raw moments are rho0 cs2 on xx and
    // yy and rho0 cs2^2 on xxyy.
    const T ux2 = ux * ux, uy2 = uy * uy;
    const T n20 = R[2][0] - d * cs2 - rho * ux2;
    const T n02 = R[0][2] - d * cs2 - rho * uy2;
    const T n11 = R[1][1] - rho * ux * uy;
    const T n21 = R[2][1] - rho * uy * (cs2 + ux2);
    const T n12 = R[1][2] - rho * ux * (cs2 + uy2);
    const T n22 = R[2][2] - d * p.cs4 - rho * (cs2 * (ux2 + uy2) + ux2 * uy2);
    const T N3 = n20 + n02, N4 = n20 - n02;

    // Local strain rates, Eq. 37-38, and corrections, Eq. 23-26.
    const T b1 = p.b1c + T(1.5) * ux2, b2 = p.b2c + T(1.5) * uy2;
    const T c1 = p.c1c + T(1.5) * ux2, c2 = p.c2c - T(1.5) * uy2;
    const T gx = p.g1h * ux * dxr, gy = p.g2h * uy * dyr;
    const T R3 = N3 + gx + gy;
    const T R4 = N4 + gx - gy;
    const T idet = rcp(rho * (b1 * c2 - b2 * c1));
    const T dxux = (c2 * R3 - b2 * R4) * idet;
    const T dyuy = (b1 * R4 - c1 * R3) * idet;
    const T Px = p.g1i * (rho * dxux + ux * dxr) - p.g3 * rho * ux2 * dxux;
    const T Py = p.g2i * (rho * dyuy + uy * dyr) - p.g3 * rho * uy2 * dyuy;

    // Relaxation with the raw source moments of Eq. 13: increments of the
    // raw moments.  m1 relaxes to rho ux = m1 + Fx/2, so its increment is Fx
    // whatever omega_1 (same for m2).
    const T Fx = p.Fx, Fy = p.Fy;
    const T dm3 = p.lw3 * (Px + Py + T(2) * (Fx * ux + Fy * uy)) - p.w3 * N3;
    const T dm4 = p.lw4 * (Px - Py + T(2) * (Fx * ux - Fy * uy)) - p.w4 * N4;
    const T D20 = T(0.5) * (dm3 + dm4), D02 = T(0.5) * (dm3 - dm4);
    const T D11 = p.lw5 * (Fx * uy + Fy * ux) - p.w5 * n11;
    const T D21 = p.lw6 * (Fy * ux2 + T(2) * Fx * ux * uy) - p.w6 * n21;
    const T D12 = p.lw7 * (Fx * uy2 + T(2) * Fy * ux * uy) - p.w7 * n12;
    const T D22 = p.lw8 * T(2) * (Fx * ux * uy2 + Fy * uy * ux2) - p.w8 * n22;

    // Back along x (raw x-moments -> columns), then along y.
    T h[3][3];
    {
        const T Dq0[3] = {T(0), Fx, D20};
        const T Dq1[3] = {Fy, D11, D21};
        const T Dq2[3] = {D02, D12, D22};
        const T* Dq[3] = {Dq0, Dq1, Dq2};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            h[0][q] = Dq[q][0] - Dq[q][2];
            h[1][q] = T(0.5) * (Dq[q][2] + Dq[q][1]);
            h[2][q] = T(0.5) * (Dq[q][2] - Dq[q][1]);
        }
    }
    {
        const int iz[3] = {0, 1, 3}, ip[3] = {2, 5, 6}, im[3] = {4, 8, 7};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T t2 = p.iah2 * h[c][2], t1 = p.iah * h[c][1];
            f[iz[c]] += h[c][0] - p.ia2 * h[c][2];
            f[ip[c]] += t2 + t1;
            f[im[c]] += t2 - t1;
        }
    }
    return rho;
}

// Moving-wall term (Sec. 5.2, Eq. 57-59) added to the outgoing populations
// of a boundary cell whose link k points into a moving wall node:
// f~_k -= (f^eq_k - f^eq_opp(k))(rho_w, U_w), rho_w the cell's density.
// Nodes outside the domain in both x and y belong to the bottom/top wall.
template <typename T>
__device__ __forceinline__ void moving_wall(const KParams<T>& p, int x, int y, T rho,
                                            T f[9]) {
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const int tx = x + ex(k), ty = y + ey(k);
        int w = -1;
        if (!p.py && (ty < 0 || ty >= p.ny)) w = ty < 0 ? 2 : 3;
        else if (!p.px && (tx < 0 || tx >= p.nx)) w = tx < 0 ? 0 : 1;
        if (w < 0) continue;
        const T Ux = p.wall_u[w][0], Uy = p.wall_u[w][1];
        if (Ux == T(0) && Uy == T(0)) continue;
        f[k] -= eq_odd<T>(k, rho, Ux, Uy, p.cs2, p.a, p.iah2);
    }
}

}  // namespace lbm
