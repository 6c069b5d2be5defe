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

template <typename T> struct Lane;
template <> struct Lane<float> { using V = float2; };
template <> struct Lane<double> { using V = double; };

// Constants of the collision (the field list, in storage order):
//   rho0, -rho0, a, a^2, cs2, cs2^2;
//   force, half force, twice the force (x and y);
//   1/2, 2, 3/2, -3/2;
//   the rho-free, u-free parts of B1, B2, C1, C2 (Eq. 40);
//   (1 - 3cs2)/2, (a^2 - 3cs2)/2 (strain solve);
//   iso (1 - 3cs2), iso (a^2 - 3cs2), -3 gi;
//   1 - w_j/2 and -w_j for j = 3..8;
//   1/(2a), -1/(2a), 1/(2a^2), -1/a^2 and the halves of the first three;
//   the halves of 1 - w_j/2 and -w_j for j = 3, 4.
#define LBM_COLL_FIELDS(X)                                                              \
    X(rho0) X(nrho0) X(a) X(a2) X(cs2) X(cs4)                                          \
    X(Fx) X(Fy) X(hFx) X(hFy) X(twoFx) X(twoFy)                                        \
    X(half) X(two) X(c15) X(nc15)                                                      \
    X(b1c) X(b2c) X(c1c) X(c2c)                                                        \
    X(g1h) X(g2h)                                                                      \
    X(g1i) X(g2i) X(ng3)                                                               \
    X(lw3) X(lw4) X(lw5) X(lw6) X(lw7) X(lw8)                                          \
    X(nw3) X(nw4) X(nw5) X(nw6) X(nw7) X(nw8)                                          \
    X(iah) X(niah) X(iah2) X(nia2)                                                     \
    X(qa) X(nqa) X(qa2)                                                                \
    X(lw3h) X(lw4h) X(nw3h) X(nw4h)

// The constants as lane values (FP32: the same value in both halves of a
// float2), computed once on the host; the form the collision takes.
template <typename T>
struct CollConst {
    using V = typename Lane<T>::V;
#define LBM_DECL_LANE(n) V n;
    LBM_COLL_FIELDS(LBM_DECL_LANE)
#undef LBM_DECL_LANE
};

// The same constants stored once each (FP32), half the size: the form a
// batch keeps in its constant-memory lattice table.
struct CollConstF {
#define LBM_DECL_ONE(n) float n;
    LBM_COLL_FIELDS(LBM_DECL_ONE)
#undef LBM_DECL_ONE
};

// Either form as lane values for the collision, as a copy (bound to the
// parameter block by reference, the FP32 step spills a word and ran 1.5 %
// slower).
template <typename T>
__host__ __device__ __forceinline__ CollConst<T> to_lanes(const CollConst<T>& c) {
    return c;
}
__host__ __device__ __forceinline__ CollConst<float> to_lanes(const CollConstF& c) {
    CollConst<float> l;
#define LBM_COPY_LANE(n) l.n = make_float2(c.n, c.n);
    LBM_COLL_FIELDS(LBM_COPY_LANE)
#undef LBM_COPY_LANE
    return l;
}
__host__ __device__ __forceinline__ CollConstF compact(const CollConst<float>& c) {
    CollConstF o;
#define LBM_COPY_ONE(n) o.n = c.n.x;
    LBM_COLL_FIELDS(LBM_COPY_ONE)
#undef LBM_COPY_ONE
    return o;
}

// Kernel parameters, converted once on the host to the arithmetic type T;
// CC: the form of the collision constants.
template <typename T, typename CC = CollConst<T>>
struct KParams {
    int nx, ny, pitch;        // pitch: padded row length (also of the link mask)
    long long plane;          // element stride between population planes
    int rstride;              // element stride between rows of a plane
    int px, py;               // periodic along x / y
    int moving;               // some wall moves
    int collide;              // 0: streaming and bounce-back only
    int raw;                  // 1: raw-moment collision (RNR-LBM, Sec. 3)
    int forced;               // a body force is set
    unsigned spin_limit;      // polls of a bounded wait for staged rows
    T a, iah, iah2, cs2, rho0;  // a, 1/(2a), 1/(2a^2), c_s^2, rho0
    T wall_u[4][2];
    const uint8_t* __restrict__ lmask;  // per-cell link mask (nullable)
    int* status;                        // bit 0: a bounded wait ran out
    CC cc;                              // constants of the collision
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

// Device bounds checks of the checked build (compiled with LBM_CHECKED):
// every computed population index is tested against the buffer's 9 * plane
// elements, every link-mask index against pitch * ny, every shared-memory
// index against its array.  A failed test sets the caller's `bad` flag and
// skips the access (a load gives 0); the kernel then records bit 1 of its
// status word and its block stops at the next point where it can, without
// a trap.  In the normal build the tests compile away.
#ifdef LBM_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
constexpr int kStatusTimeout = 1;  // status bit: a bounded wait ran out
constexpr int kStatusBounds = 2;   // status bit: a bounds check failed (checked build)

template <typename I>
__device__ __forceinline__ bool idx_ok(I i, long long n, int width = 1) {
    return (long long)i >= 0 && (long long)i + width <= n;
}
// Global read-only load of p[i], checked against n elements.
template <typename S, typename I>
__device__ __forceinline__ S ldg_chk(const S* __restrict__ p, I i, long long n, bool& bad) {
    if constexpr (kChecked) {
        if (!idx_ok(i, n)) {
            bad = true;
            return S(0);
        }
    }
    return __ldg(p + i);
}
// Link-mask byte of cell (x, y), checked.
template <typename P>
__device__ __forceinline__ unsigned mask_at(const P& p, long long i, bool& bad) {
    if constexpr (kChecked) {
        if (!idx_ok(i, (long long)p.pitch * p.ny)) {
            bad = true;
            return 0xFFu;
        }
    }
    return p.lmask[i];
}

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

// pull() with its nine indices checked in the checked build.
template <typename S, typename P>
__device__ __forceinline__ void pull(const S* __restrict__ fin, const P& p, int x, int y,
                                     unsigned sb, S f[9], bool& bad) {
    if constexpr (kChecked) {
        const int xm = x == 0 ? p.nx - 1 : x - 1;
        const int xp = x == p.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? p.ny - 1 : y - 1;
        const int yp = y == p.ny - 1 ? 0 : y + 1;
        const long long pl = p.plane, n = 9 * pl;
        const long long rc = (long long)y * p.rstride, rm = (long long)ym * p.rstride,
                        rp = (long long)yp * p.rstride;
        const long long c = rc + x;
        bool ok = x >= 0 && x < p.nx && y >= 0 && y < p.ny;
        const long long idx[9] = {c,
                                  (sb & 1u) ? 3 * pl + c : 1 * pl + rc + xm,
                                  (sb & 2u) ? 4 * pl + c : 2 * pl + rm + x,
                                  (sb & 4u) ? 1 * pl + c : 3 * pl + rc + xp,
                                  (sb & 8u) ? 2 * pl + c : 4 * pl + rp + x,
                                  (sb & 16u) ? 7 * pl + c : 5 * pl + rm + xm,
                                  (sb & 32u) ? 8 * pl + c : 6 * pl + rm + xp,
                                  (sb & 64u) ? 5 * pl + c : 7 * pl + rp + xp,
                                  (sb & 128u) ? 6 * pl + c : 8 * pl + rp + xm};
#pragma unroll
        for (int i = 0; i < 9; ++i) ok = ok && idx_ok(idx[i], n);
        if (!ok) {
            bad = true;
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = S(0);
            return;
        }
    }
    pull(fin, p, x, y, sb, f);
}

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

// Lane arithmetic of the collision.  FP32 collides the two cells a thread
// owns as one float2 through the packed FP32 instructions of sm_100 and
// later (add, multiply and fused multiply-add on both cells at once); FP64
// collides one cell per double.  Every operation is written out, so the
// rounding of a cell does not depend on how the compiler would have
// contracted an expression, nor on which lane or block computes it.
__device__ __forceinline__ double vadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ double vrcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// FP32: the hardware reciprocal approximation (at most 2 ulp off, below the
// FP32 storage rounding); FP64: an IEEE division.
__device__ __forceinline__ float2 vrcp(float2 a) {
    return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}

// Collision of one lane (Sec. 4) in increment form on deviations:
//   f~ = f + T^-1 F(-u) [ Lambda (m^{c,eq} - m^c) + (I - Lambda/2) Phi^c ].
// The D2Q9 basis of Eq. 3 is the tensor product {1, x, x^2} x {1, y, y^2},
// so T, F(u) and their inverses factor into 3x3 maps along x and along y:
// central moments are reduced column by column (over e_y, then e_x), and the
// increment is expanded back the same way.  The rest equilibrium rho0 w_i is
// carried analytically so that FP32 only ever adds small numbers.
//   f: deviations in, post-collision deviations out.  d = sum f (density
//   deviation).  dxr, dyr: density gradient.  Returns rho.
// A constant of the collision as an operand of both lanes: the stored pair
// holds the same value twice, and the collision reads its low half for both
// (which needs fewer registers than the pair itself: the FP32 step then
// spills nothing and ran 1.4 % faster, the batch 2 %).
__device__ __forceinline__ float2 bc(float2 v) { return make_float2(v.x, v.x); }
__device__ __forceinline__ double bc(double v) { return v; }

template <typename T, bool FORCE = true>
__device__ __forceinline__ typename Lane<T>::V collide(const CollConst<T>& c,
                                                       typename Lane<T>::V f[9],
                                                       typename Lane<T>::V d,
                                                       typename Lane<T>::V dxr,
                                                       typename Lane<T>::V dyr) {
    using V = typename Lane<T>::V;
    // Column sums of each column e_x = 0, +1, -1: sq = g(+a) + g(-a),
    // ad = a (g(+a) - g(-a)), k0 = g(0) + sq; the momentum is
    // j = (k0(+1) - k0(-1), ad(0) + ad(+1) + ad(-1)).
    V sq[3], ad[3], k0[3], k1[3], k2[3];
    {
        const V gz[3] = {f[0], f[1], f[3]}, gp[3] = {f[2], f[5], f[6]},
                gm[3] = {f[4], f[8], f[7]};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            sq[q] = vadd(gp[q], gm[q]);
            ad[q] = vmul(bc(c.a), vsub(gp[q], gm[q]));
            k0[q] = vadd(gz[q], sq[q]);
        }
    }
    const V rho = vadd(bc(c.rho0), d);
    const V jx = vsub(k0[1], k0[2]);
    const V jy = vadd(vadd(ad[0], ad[1]), ad[2]);
    const V ir = vrcp(rho);
    const V ux = FORCE ? vmul(vadd(jx, bc(c.hFx)), ir) : vmul(jx, ir);
    const V uy = FORCE ? vmul(vadd(jy, bc(c.hFy)), ir) : vmul(jy, ir);
    const V nux = vneg(ux), nuy = vneg(uy);

    // Central moments along y of each column:
    // k0 = sum g, k1 = sum g (e_y - u_y), k2 = sum g (e_y - u_y)^2.
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        k1[q] = vfma(nuy, k0[q], ad[q]);
        k2[q] = vfma(nuy, vadd(ad[q], k1[q]), vmul(bc(c.a2), sq[q]));
    }
    // Along x: C[p][q] = sum_X (e_x - u_x)^p k_q(X).
    V C[3][3];
    {
        const V* kq[3] = {k0, k1, k2};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const V S = vadd(kq[q][1], kq[q][2]), D = vsub(kq[q][1], kq[q][2]);
            C[0][q] = vadd(kq[q][0], S);
            C[1][q] = vfma(nux, C[0][q], D);
            C[2][q] = vfma(nux, vadd(C[1][q], D), S);
        }
    }
    // Non-equilibrium central moments: subtract the Maxwell-matched values
    // (rho cs2 on xx and yy, rho cs2^2 on xxyy) and add back the central
    // moments of rho0 w about u.
    const V ux2 = vmul(ux, ux), uy2 = vmul(uy, uy);
    const V nd = vneg(d);
    const V n20 = vfma(bc(c.rho0), ux2, vfma(nd, bc(c.cs2), C[2][0]));
    const V n02 = vfma(bc(c.rho0), uy2, vfma(nd, bc(c.cs2), C[0][2]));
    const V n11 = vfma(vmul(bc(c.rho0), ux), uy, C[1][1]);
    const V n21 = vfma(vmul(bc(c.nrho0), uy), vadd(bc(c.cs2), ux2), C[2][1]);
    const V n12 = vfma(vmul(bc(c.nrho0), ux), vadd(bc(c.cs2), uy2), C[1][2]);
    const V n22 = vfma(bc(c.rho0), vfma(bc(c.cs2), vadd(ux2, uy2), vmul(ux2, uy2)),
                       vfma(nd, bc(c.cs4), C[2][2]));
    const V k3 = vadd(n20, n02), k4 = vsub(n20, n02);

    // Local strain rates, Eq. 37-38, from the raw non-equilibrium moments of
    // Eq. 34-35 (central ones minus the force terms u.F).
    V N3 = k3, N4 = k4;
    if constexpr (FORCE) {
        const V uFy = vmul(uy, bc(c.Fy));
        N3 = vsub(k3, vfma(ux, bc(c.Fx), uFy));
        N4 = vsub(k4, vsub(vmul(ux, bc(c.Fx)), uFy));
    }
    const V b1 = vfma(bc(c.c15), ux2, bc(c.b1c)), b2 = vfma(bc(c.c15), uy2, bc(c.b2c));
    const V c1 = vfma(bc(c.c15), ux2, bc(c.c1c)), c2 = vfma(bc(c.nc15), uy2, bc(c.c2c));
    const V gx = vmul(vmul(bc(c.g1h), ux), dxr), gy = vmul(vmul(bc(c.g2h), uy), dyr);
    const V R3 = vadd(vadd(N3, gx), gy);
    const V R4 = vsub(vadd(N4, gx), gy);
    // the 2x2 solve gives rho d_x u_x and rho d_y u_y directly, which is all
    // the corrections use
    const V idet = vrcp(vfma(b1, c2, vmul(vneg(b2), c1)));

    // Corrections, Eq. 23-26: m3s + m3G = l3 (Px + Py), m4s + m4G = l4 (Px - Py).
    const V rdx = vmul(vfma(c2, R3, vmul(vneg(b2), R4)), idet);
    const V rdy = vmul(vfma(b1, R4, vmul(vneg(c1), R3)), idet);
    const V Px = vfma(bc(c.g1i), vfma(ux, dxr, rdx), vmul(vmul(bc(c.ng3), rdx), ux2));
    const V Py = vfma(bc(c.g2i), vfma(uy, dyr, rdy), vmul(vmul(bc(c.ng3), rdy), uy2));

    // Relaxation (Eq. 49 equilibria, Phi^c = (0, Fx, Fy, 0, ...)):
    // increments of the central moments.  kappa_1 = -Fx/2 before collision,
    // so its increment is Fx whatever omega_1 (same for y).
    // (dk3, dk4 are the halves of the increments of k3, k4: halving the
    // constants is exact, so D20 and D02 round as (dk3 +- dk4) / 2 would)
    const V dk3 = vfma(bc(c.lw3h), vadd(Px, Py), vmul(bc(c.nw3h), k3));
    const V dk4 = vfma(bc(c.lw4h), vsub(Px, Py), vmul(bc(c.nw4h), k4));
    const V D20 = vadd(dk3, dk4), D02 = vsub(dk3, dk4);
    const V D11 = vmul(bc(c.nw5), n11), D21 = vmul(bc(c.nw6), n21), D12 = vmul(bc(c.nw7), n12),
            D22 = vmul(bc(c.nw8), n22);

    // Back along x: central -> raw x-moments -> the three columns (h[X][q],
    // X = 0, +1, -1), for q = 0: (0, Fx, D20), q = 1: (Fy, D11, D21),
    // q = 2: (D02, D12, D22).  The columns X = +-1 are kept doubled (their
    // factor 1/2 goes into the constants of the expansion along y, exactly).
    V h[3][3];
    {
        const V m2 = FORCE ? vfma(ux, bc(c.twoFx), D20) : D20;  // m0 = 0, m1 = Fx
        h[0][0] = vneg(m2);
        h[1][0] = FORCE ? vadd(m2, bc(c.Fx)) : m2;
        h[2][0] = FORCE ? vsub(m2, bc(c.Fx)) : m2;
    }
    {
        const V m0[2] = {bc(c.Fy), D02}, m1in[2] = {D11, D12}, m2in[2] = {D21, D22};
#pragma unroll
        for (int q = 1; q < 3; ++q) {
            const bool zero_m0 = q == 1 && !FORCE;  // m0 = Fy = 0
            const V m1 = zero_m0 ? m1in[0] : vfma(ux, m0[q - 1], m1in[q - 1]);
            const V m2 = vfma(ux, vadd(m1in[q - 1], m1), m2in[q - 1]);
            h[0][q] = zero_m0 ? vneg(m2) : vsub(m0[q - 1], m2);
            h[1][q] = vadd(m2, m1);
            h[2][q] = vsub(m2, m1);
        }
    }
    // Back along y for each column, and add the increment.
    {
        const int iz[3] = {0, 1, 3}, ip[3] = {2, 5, 6}, im[3] = {4, 8, 7};
#pragma unroll
        for (int X = 0; X < 3; ++X) {
            const V m0 = h[X][0];
            const V m1 = vfma(uy, m0, h[X][1]);
            const V m2 = vfma(uy, vadd(h[X][1], m1), h[X][2]);
            if (X == 0) {
                f[0] = vadd(f[0], vfma(bc(c.nia2), m2, m0));
                f[2] = vfma(bc(c.iah2), m2, vfma(bc(c.iah), m1, f[2]));
                f[4] = vfma(bc(c.iah2), m2, vfma(bc(c.niah), m1, f[4]));
            } else {
                f[iz[X]] = vfma(bc(c.half), vfma(bc(c.nia2), m2, m0), f[iz[X]]);
                f[ip[X]] = vfma(bc(c.qa2), m2, vfma(bc(c.qa), m1, f[ip[X]]));
                f[im[X]] = vfma(bc(c.qa2), m2, vfma(bc(c.nqa), m1, f[im[X]]));
            }
        }
    }
    return rho;
}

// Collision of one lane of the raw-moment scheme (RNR-LBM, Sec. 3), in the
// increment form of collide():
//   f~ = f + T^-1 [ Lambda (m^eq - m) + (I - Lambda/2) Phi ]
// with the raw equilibria of Eq. 12 (m^eq_8 = rho cs2^2 + rho cs2 |u|^2 +
// rho ux^2 uy^2, the binomial transform of the central equilibria), the
// corrections of Eq. 23-26 on m3 and m4, and the raw source moments of
// Eq. 13.  The raw moments factor as R[p][q] = sum_i f_i e_ix^p e_iy^q, so
// the transforms are those of collide() at u = 0.  The strain rates
// (Eq. 37-38) and corrections are the same as in collide().
template <typename T>
__device__ __forceinline__ typename Lane<T>::V collide_raw(const CollConst<T>& c,
                                                           typename Lane<T>::V f[9],
                                                           typename Lane<T>::V d,
                                                           typename Lane<T>::V dxr,
                                                           typename Lane<T>::V dyr) {
    using V = typename Lane<T>::V;
    // Raw moments along y of each column: k0 = sum g, k1 = sum g e_y,
    // k2 = sum g e_y^2; then along x: R[p][q] = sum_X e_x^p k_q(X).  The
    // momentum is j = (k0(+1) - k0(-1), k1(0) + k1(+1) + k1(-1)).
    V k0[3], k1[3], k2[3];
    {
        const V gz[3] = {f[0], f[1], f[3]}, gp[3] = {f[2], f[5], f[6]},
                gm[3] = {f[4], f[8], f[7]};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const V s = vadd(gp[q], gm[q]);
            k0[q] = vadd(gz[q], s);
            k1[q] = vmul(c.a, vsub(gp[q], gm[q]));
            k2[q] = vmul(c.a2, s);
        }
    }
    const V rho = vadd(c.rho0, d);
    const V jx = vsub(k0[1], k0[2]);
    const V jy = vadd(vadd(k1[0], k1[1]), k1[2]);
    const V ir = vrcp(rho);
    const V ux = vmul(vadd(jx, c.hFx), ir);
    const V uy = vmul(vadd(jy, c.hFy), ir);
    V R[3][3];
    {
        const V* kq[3] = {k0, k1, k2};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const V S = vadd(kq[q][1], kq[q][2]);
            R[0][q] = vadd(kq[q][0], S);
            R[1][q] = vsub(kq[q][1], kq[q][2]);
            R[2][q] = S;
        }
    }
    // Non-equilibrium raw moments m - m^{eq,r} (Eq. 12); the stored values
    // are deviations from rho0 w, whose raw moments are rho0 cs2 on xx and
    // yy and rho0 cs2^2 on xxyy.
    const V ux2 = vmul(ux, ux), uy2 = vmul(uy, uy);
    const V nd = vneg(d), nrho = vneg(rho);
    const V n20 = vfma(nrho, ux2, vfma(nd, c.cs2, R[2][0]));
    const V n02 = vfma(nrho, uy2, vfma(nd, c.cs2, R[0][2]));
    const V n11 = vfma(vmul(nrho, ux), uy, R[1][1]);
    const V n21 = vfma(vmul(nrho, uy), vadd(c.cs2, ux2), R[2][1]);
    const V n12 = vfma(vmul(nrho, ux), vadd(c.cs2, uy2), R[1][2]);
    const V n22 = vfma(nrho, vfma(c.cs2, vadd(ux2, uy2), vmul(ux2, uy2)),
                       vfma(nd, c.cs4, R[2][2]));
    const V N3 = vadd(n20, n02), N4 = vsub(n20, n02);

    // Local strain rates, Eq. 37-38, and corrections, Eq. 23-26.
    const V b1 = vfma(c.c15, ux2, c.b1c), b2 = vfma(c.c15, uy2, c.b2c);
    const V c1 = vfma(c.c15, ux2, c.c1c), c2 = vfma(c.nc15, uy2, c.c2c);
    const V gx = vmul(vmul(c.g1h, ux), dxr), gy = vmul(vmul(c.g2h, uy), dyr);
    const V R3 = vadd(vadd(N3, gx), gy);
    const V R4 = vsub(vadd(N4, gx), gy);
    const V idet = vrcp(vmul(rho, vfma(b1, c2, vmul(vneg(b2), c1))));
    const V dxux = vmul(vfma(c2, R3, vmul(vneg(b2), R4)), idet);
    const V dyuy = vmul(vfma(b1, R4, vmul(vneg(c1), R3)), idet);
    const V rdx = vmul(rho, dxux), rdy = vmul(rho, dyuy);
    const V Px = vfma(c.g1i, vfma(ux, dxr, rdx), vmul(vmul(c.ng3, rdx), ux2));
    const V Py = vfma(c.g2i, vfma(uy, dyr, rdy), vmul(vmul(c.ng3, rdy), uy2));

    // Relaxation with the raw source moments of Eq. 13: increments of the
    // raw moments.  m1 relaxes to rho ux = m1 + Fx/2, so its increment is Fx
    // whatever omega_1 (same for m2).
    const V uFx = vmul(ux, c.Fx), uFy = vmul(uy, c.Fy);
    const V dm3 = vfma(c.lw3, vfma(c.two, vadd(uFx, uFy), vadd(Px, Py)), vmul(c.nw3, N3));
    const V dm4 = vfma(c.lw4, vfma(c.two, vsub(uFx, uFy), vsub(Px, Py)), vmul(c.nw4, N4));
    const V D20 = vmul(c.half, vadd(dm3, dm4)), D02 = vmul(c.half, vsub(dm3, dm4));
    const V D11 = vfma(c.lw5, vfma(c.Fx, uy, vmul(c.Fy, ux)), vmul(c.nw5, n11));
    const V D21 = vfma(c.lw6, vfma(c.Fy, ux2, vmul(vmul(c.twoFx, ux), uy)), vmul(c.nw6, n21));
    const V D12 = vfma(c.lw7, vfma(c.Fx, uy2, vmul(vmul(c.twoFy, ux), uy)), vmul(c.nw7, n12));
    const V D22 = vfma(c.lw8, vmul(c.two, vfma(uFx, uy2, vmul(uFy, ux2))), vmul(c.nw8, n22));

    // Back along x (raw x-moments -> columns), then along y.
    V h[3][3];
    h[0][0] = vneg(D20);
    h[1][0] = vmul(c.half, vadd(D20, c.Fx));
    h[2][0] = vmul(c.half, vsub(D20, c.Fx));
    h[0][1] = vsub(c.Fy, D21);
    h[1][1] = vmul(c.half, vadd(D21, D11));
    h[2][1] = vmul(c.half, vsub(D21, D11));
    h[0][2] = vsub(D02, D22);
    h[1][2] = vmul(c.half, vadd(D22, D12));
    h[2][2] = vmul(c.half, vsub(D22, D12));
    {
        const int iz[3] = {0, 1, 3}, ip[3] = {2, 5, 6}, im[3] = {4, 8, 7};
#pragma unroll
        for (int X = 0; X < 3; ++X) {
            f[iz[X]] = vadd(f[iz[X]], vfma(c.nia2, h[X][2], h[X][0]));
            f[ip[X]] = vfma(c.iah2, h[X][2], vfma(c.iah, h[X][1], f[ip[X]]));
            f[im[X]] = vfma(c.iah2, h[X][2], vfma(c.niah, h[X][1], f[im[X]]));
        }
    }
    return rho;
}

// Moving-wall term (Sec. 5.2, Eq. 57-59) added to the outgoing populations
// of a boundary cell whose link k points into a moving wall node:
// f~_k -= (f^eq_k - f^eq_opp(k))(rho_w, U_w), rho_w the cell's density.
// Nodes outside the domain in both x and y belong to the bottom/top wall.
template <typename T, typename P>
__device__ __forceinline__ void moving_wall(const P& p, int x, int y, T rho, T f[9]) {
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
