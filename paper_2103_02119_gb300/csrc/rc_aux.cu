// rc_aux.cu -- state set-up, read-out and FP64 diagnostics kernels of the
// RC-LBM library (arXiv 2103.02119, Sec. 4), for sm_103a.
//
// The stored state is post-collision and in pull form (see lbm_device.cuh):
// slot i of cell c is what the next step pulls into cell c + e_i, or, when
// c + e_i is a wall or solid node, what cell c pulls back as direction
// opp(i).  Setting a state scatters distributions into that form; reading it
// gathers them with the same pull the step kernel uses.
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double feq_d(int i, double rho, double ux, double uy,
                                        double cs2, double a) {
    const double iah2 = 0.5 / (a * a);
    return rho * phi_x<double>(ex(i), ux, cs2) * phi_y<double>(ey(i), uy, cs2, a, iah2);
}

// Target cell of direction i from (x, y), wrapped on periodic axes.  Only
// called when the target is a fluid cell (so inside the domain).
__device__ __forceinline__ long long target(const AuxParams& p, int x, int y, int i) {
    int tx = x + ex(i), ty = y + ey(i);
    if (tx < 0) tx += p.nx; else if (tx >= p.nx) tx -= p.nx;
    if (ty < 0) ty += p.ny; else if (ty >= p.ny) ty -= p.ny;
    return (long long)ty * p.nx + tx;
}

// f_i^eq(r, u, v) - w_i rho0, the stored deviation of an equilibrium.  FP64
// storage evaluates f^eq in FP64 and subtracts the rest part.
__device__ __forceinline__ double feq_dev64(int i, double r, double u, double v,
                                            const AuxParams& p) {
    return feq_d(i, r, u, v, p.cs2, p.a) - p.wrest[i];
}

// FP32 storage carries the rest part analytically, as the step does: with
// the 1-D factors X = X0 + dX (along x) and Y = Y0 + dY (along y), X0 Y0 =
// w_i,
//   r X Y - rho0 X0 Y0 = (r - rho0) X Y + rho0 (dX Y + X0 dY),
// where dX, dY vanish with the velocity, so FP32 only forms small numbers
// (and GB300's FP64 pipe, a small fraction of its FP32 rate, stays idle).
// The state comes in FP32 too: dr = r - rho0, (u, v).
struct Feq32 {
    float cs2, a, iah2, rho0;
    __device__ __forceinline__ float operator()(int i, float dr, float u, float v) const {
        const int sx = ex(i), sy = ey(i);
        const float X0 = sx == 0 ? 1.0f - cs2 : 0.5f * cs2;
        const float dX = sx == 0 ? -u * u : 0.5f * (u * u + (float)sx * u);
        const float Y0 = sy == 0 ? 1.0f - 2.0f * iah2 * cs2 : iah2 * cs2;
        const float dY = sy == 0 ? -2.0f * iah2 * v * v : iah2 * (v * v + (float)sy * a * v);
        const float X = X0 + dX, Y = Y0 + dY;
        return dr * X * Y + rho0 * (dX * Y + X0 * dY);
    }
};

// One row per block row of the grid, x across the block: no division of a
// cell index.
#define LBM_FOR_CELLS(p)                                                                 \
    for (int y = blockIdx.y; y < (p).ny; y += gridDim.y)                                 \
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < (p).nx;                  \
             x += gridDim.x * blockDim.x)

template <bool MASK>
__global__ void init_kernel(double* __restrict__ f, const AuxParams p, const double* rho,
                            const double* ux, const double* uy) {
    LBM_FOR_CELLS(p) {
        const long long c = (long long)y * p.nx + x;
        const long long o = (long long)y * p.rstride + x;
        const unsigned sb = link_bits<MASK>(p, x, y);
        if (sb == 0xFFu) {
            for (int i = 0; i < 9; ++i) f[i * p.plane + o] = 0.0;
            continue;
        }
        const double r0 = rho ? rho[c] : 1.0, u0 = ux ? ux[c] : 0.0,
                     v0 = uy ? uy[c] : 0.0;
        for (int i = 0; i < 9; ++i) {
            double v;
            if (i > 0 && ((sb >> (opp(i) - 1)) & 1u)) {
                v = feq_dev64(opp(i), r0, u0, v0, p);  // pulled back by c itself
            } else {
                const long long t = i == 0 ? c : target(p, x, y, i);
                v = feq_dev64(i, rho ? rho[t] : 1.0, ux ? ux[t] : 0.0, uy ? uy[t] : 0.0, p);
            }
            f[i * p.plane + o] = v;
        }
    }
}

// FP32 storage: a block owns up to kThreads columns and marches down a band
// of rows, keeping the FP32 state (r - rho0, u, v) of the rows y - 1, y,
// y + 1 and of one column either side in shared memory, so that each cell's
// FP64 input is converted once rather than once per population.
constexpr int kInitRows = 16;  // rows of a band (more when ny / 16 > 65535)

template <bool MASK>
__global__ void __launch_bounds__(kThreads)
init32_kernel(float* __restrict__ f, const AuxParams p, const double* rho, const double* ux,
              const double* uy, int rows) {
    constexpr int SW = kThreads + 2;
    __shared__ float st[3][3][SW];  // [component][ring row][column x - x0 + 1]
    const Feq32 feq{(float)p.cs2, (float)p.a, (float)(0.5 / (p.a * p.a)), (float)p.rho0};
    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * kThreads;
    const int w = min(kThreads, p.nx - x0);
    const int y0 = blockIdx.y * rows;
    const int y1 = min(p.ny, y0 + rows);
    // ring slot of row yy in [y0 - 1, y1]
    auto slot = [&](int yy) { return (yy - y0 + 1) % 3; };
    auto load_row = [&](int yy) {
        const int k = slot(yy);
        int gy = yy;
        if (gy < 0) gy = p.py ? gy + p.ny : -1;
        else if (gy >= p.ny) gy = p.py ? gy - p.ny : -1;
        for (int c = tx; c < w + 2; c += kThreads) {
            int gx = x0 - 1 + c;
            if (gx < 0) gx = p.px ? gx + p.nx : -1;
            else if (gx >= p.nx) gx = p.px ? gx - p.nx : -1;
            float dr = 0.0f, u = 0.0f, v = 0.0f;  // outside a wall: never read
            if (gx >= 0 && gy >= 0) {
                const long long t = (long long)gy * p.nx + gx;
                dr = (float)((rho ? rho[t] : 1.0) - p.rho0);
                u = ux ? (float)ux[t] : 0.0f;
                v = uy ? (float)uy[t] : 0.0f;
            }
            st[0][k][c] = dr;
            st[1][k][c] = u;
            st[2][k][c] = v;
        }
    };
    if (w <= 0 || y0 >= p.ny) return;
    load_row(y0 - 1);
    load_row(y0);
    for (int y = y0; y < y1; ++y) {
        load_row(y + 1);
        __syncthreads();
        if (tx < w) {
            const int x = x0 + tx;
            const long long o = (long long)y * p.rstride + x;
            const unsigned sb = link_bits<MASK>(p, x, y);
            if (sb == 0xFFu) {
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i * p.plane + o] = 0.0f;
            } else {
                const int k = slot(y), c = tx + 1;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    float v;
                    if (i > 0 && ((sb >> (opp(i) - 1)) & 1u)) {
                        // pulled back by the cell itself
                        v = feq(opp(i), st[0][k][c], st[1][k][c], st[2][k][c]);
                    } else {
                        const int kk = slot(y + ey(i)), cc = c + ex(i);
                        v = feq(i, st[0][kk][cc], st[1][kk][cc], st[2][kk][cc]);
                    }
                    f[i * p.plane + o] = v;
                }
            }
        }
        __syncthreads();  // row y - 1's slot is overwritten next
    }
}

template <typename T, bool MASK>
__global__ void set_f_kernel(T* __restrict__ f, const AuxParams p,
                             const double* __restrict__ fin) {
    const long long N = (long long)p.nx * p.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const long long o = (long long)y * p.rstride + x;
        const unsigned sb = link_bits<MASK>(p, x, y);
        if (sb == 0xFFu) {
            for (int i = 0; i < 9; ++i) f[i * p.plane + o] = T(0);
            continue;
        }
        for (int i = 0; i < 9; ++i) {
            double v;
            if (i > 0 && ((sb >> (opp(i) - 1)) & 1u)) v = fin[opp(i) * N + c];
            else v = fin[i * N + (i == 0 ? c : target(p, x, y, i))];
            f[i * p.plane + o] = T(v - p.wrest[i]);
        }
    }
}

template <typename T, bool MASK>
__global__ void get_f_kernel(const T* __restrict__ f, const AuxParams p,
                             double* __restrict__ fout) {
    const long long N = (long long)p.nx * p.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const unsigned sb = link_bits<MASK>(p, x, y);
        if (sb == 0xFFu) {
            for (int i = 0; i < 9; ++i) fout[i * N + c] = 0.0;
            continue;
        }
        T g[9];
        pull(f, p, x, y, sb, g);
        for (int i = 0; i < 9; ++i) fout[i * N + c] = (double)g[i] + p.wrest[i];
    }
}

// rho and u of one fluid cell from its pulled deviations, in FP64.
template <typename T>
__device__ __forceinline__ void macro(const AuxParams& p, const T g[9], double& rho,
                                      double& ux, double& uy) {
    double d = 0.0, jx = 0.0, jy = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double v = (double)g[i];
        d += v;
        jx += ex(i) * v;
        jy += ey(i) * v;
    }
    rho = p.rho0 + d;
    ux = (jx + 0.5 * p.Fx) / rho;
    uy = (p.a * jy + 0.5 * p.Fy) / rho;
}

// The read-out of FP32 storage (lbm_moments): the nine deviations summed in
// FP32 and rho = rho0 + d formed in FP64, u in FP32 (the accuracy the FP32
// state holds), so that the FP64 pipe only converts.  The diagnostics and
// residuals keep the FP64 macro().
__device__ __forceinline__ void macro_out(const AuxParams& p, const float g[9], double& rho,
                                          double& ux, double& uy) {
    float d = 0.0f, jx = 0.0f, jy = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        d += g[i];
        if (ex(i) != 0) jx += ex(i) > 0 ? g[i] : -g[i];
        if (ey(i) != 0) jy += ey(i) > 0 ? g[i] : -g[i];
    }
    rho = p.rho0 + (double)d;
    const float r = (float)p.rho0 + d;
    ux = (double)((jx + 0.5f * (float)p.Fx) / r);
    uy = (double)(((float)p.a * jy + 0.5f * (float)p.Fy) / r);
}
__device__ __forceinline__ void macro_out(const AuxParams& p, const double g[9], double& rho,
                                          double& ux, double& uy) {
    macro(p, g, rho, ux, uy);
}

template <typename T, bool MASK, bool EXACT64>
__global__ void moments_kernel(const T* __restrict__ f, const AuxParams p,
                               double* rho, double* ux, double* uy) {
    LBM_FOR_CELLS(p) {
        const long long c = (long long)y * p.nx + x;
        const unsigned sb = link_bits<MASK>(p, x, y);
        double r = 0.0, u = 0.0, v = 0.0;
        if (sb != 0xFFu) {
            T g[9];
            pull(f, p, x, y, sb, g);
            if constexpr (EXACT64) macro(p, g, r, u, v);
            else macro_out(p, g, r, u, v);
        }
        if (rho) rho[c] = r;
        if (ux) ux[c] = u;
        if (uy) uy[c] = v;
    }
}

// Local strain rates of one fluid cell from its raw non-equilibrium moments
// (Eq. 34-40; the left side of Eq. 39 read as d_y u_x + d_x u_y) and the
// viscous stress of the recovered Navier-Stokes equations (Eq. 30-33), all in
// FP64.  The density gradient is the central difference of the step (spacing
// 2 along x and 2a along y), a wall or solid neighbour counting with the
// cell's own density.
template <typename T, bool MASK>
__global__ void stress_kernel(const T* __restrict__ f, const AuxParams p,
                              const double* __restrict__ rho, double* dxux, double* dyuy,
                              double* sxy, double* txx, double* tyy, double* txy) {
    const long long N = (long long)p.nx * p.ny;
    const double a = p.a, a2 = a * a, cs2 = p.cs2;
    const double nu4 = cs2 * (1.0 / p.w4 - 0.5), nu5 = cs2 * (1.0 / p.w5 - 0.5);
    const double zeta = cs2 * (1.0 / p.w3 - 0.5);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const unsigned sb = link_bits<MASK>(p, x, y);
        double e_xx = 0.0, e_yy = 0.0, e_xy = 0.0, r = 0.0;
        if (sb != 0xFFu) {
            T g[9];
            pull(f, p, x, y, sb, g);
            double m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0, m5 = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double fi = (double)g[i] + p.wrest[i];
                const double ex_ = ex(i), ey_ = a * ey(i);
                m0 += fi;
                m1 += fi * ex_;
                m2 += fi * ey_;
                m3 += fi * (ex_ * ex_ + ey_ * ey_);
                m4 += fi * (ex_ * ex_ - ey_ * ey_);
                m5 += fi * ex_ * ey_;
            }
            r = m0;
            const double ux = (m1 + 0.5 * p.Fx) / r, uy = (m2 + 0.5 * p.Fy) / r;
            const double rc = rho[c];
            const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
            const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
            const long long row = (long long)y * p.nx;
            const double rW = (sb & 1u) ? rc : rho[row + xm];
            const double rS = (sb & 2u) ? rc : rho[(long long)ym * p.nx + x];
            const double rE = (sb & 4u) ? rc : rho[row + xp];
            const double rN = (sb & 8u) ? rc : rho[(long long)yp * p.nx + x];
            const double dxr = 0.5 * (rE - rW), dyr = (rN - rS) / (2.0 * a);
            const double ux2 = ux * ux, uy2 = uy * uy;
            const double B1 = r * (-2.0 * cs2 / p.w3 - 0.5 * (1.0 - 3.0 * cs2) + 1.5 * ux2);
            const double B2 = r * (-2.0 * cs2 / p.w3 - 0.5 * (a2 - 3.0 * cs2) + 1.5 * uy2);
            const double B3 = 0.5 * (3.0 * cs2 - 1.0) * ux, B4 = 0.5 * (3.0 * cs2 - a2) * uy;
            const double C1 = r * (-2.0 * cs2 / p.w4 - 0.5 * (1.0 - 3.0 * cs2) + 1.5 * ux2);
            const double C2 = r * (2.0 * cs2 / p.w4 - 0.5 * (3.0 * cs2 - a2) - 1.5 * uy2);
            const double C3 = B3, C4 = -B4;
            const double R3 = m3 - (2.0 * r * cs2 + r * (ux2 + uy2)) - B3 * dxr - B4 * dyr;
            const double R4 = m4 - r * (ux2 - uy2) - C3 * dxr - C4 * dyr;
            e_xx = (C2 * R3 - B2 * R4) / (C2 * B1 - C1 * B2);
            e_yy = (C1 * R3 - B1 * R4) / (C1 * B2 - C2 * B1);
            e_xy = (m5 - r * ux * uy) / (-r * cs2 / p.w5);
        }
        const double div = e_xx + e_yy;
        if (dxux) dxux[c] = e_xx;
        if (dyuy) dyuy[c] = e_yy;
        if (sxy) sxy[c] = e_xy;
        if (txx) txx[c] = r * (nu4 * (2.0 * e_xx - div) + zeta * div);
        if (tyy) tyy[c] = r * (nu4 * (2.0 * e_yy - div) + zeta * div);
        if (txy) txy[c] = r * nu5 * e_xy;
    }
}

// Adds v exactly (down to 2^-kMassShift) to a fixed-point number held as
// 24-bit limbs.  Returns false when v is too large for the accumulator.
__device__ __forceinline__ bool add_fixed(long long limb[kMassLimbs], double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((bits >> 52) & 0x7FF);
    unsigned long long M = bits & 0xFFFFFFFFFFFFFull;
    if (E == 0x7FF) return false;
    int e2;
    if (E == 0) e2 = -1074;
    else { M |= 1ull << 52; e2 = E - 1075; }
    if (M == 0) return true;
    int pos = e2 + kMassShift;
    if (pos < 0) {
        if (pos <= -64) return true;   // below the accumulator's resolution
        M >>= -pos;
        pos = 0;
    }
    if (pos > 24 * (kMassLimbs - 4)) return false;
    const int k0 = pos / 24, o = pos % 24;
    const unsigned __int128 t = (unsigned __int128)M << o;
    long long c[4] = {(long long)(t & 0xFFFFFF), (long long)((t >> 24) & 0xFFFFFF),
                      (long long)((t >> 48) & 0xFFFFFF), (long long)(t >> 72)};
    const bool neg = (bits >> 63) != 0;
#pragma unroll
    for (int k = 0; k < kMassLimbs; ++k) {
        const int j = k - k0;
        long long add = 0;
        if (j == 0) add = c[0];
        else if (j == 1) add = c[1];
        else if (j == 2) add = c[2];
        else if (j == 3) add = c[3];
        limb[k] += neg ? -add : add;
    }
    return true;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// Sums one DiagPartial per thread over the block in a fixed order.
__device__ void block_reduce(DiagPartial& d, DiagPartial* out) {
    __shared__ DiagPartial sh[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    d.mx = warp_sum(d.mx);
    d.my = warp_sum(d.my);
    d.en = warp_sum(d.en);
    d.dres = warp_sum(d.dres);
    d.ures = warp_sum(d.ures);
    d.sres = warp_sum(d.sres);
    d.nonfinite = warp_sum(d.nonfinite);
#pragma unroll
    for (int k = 0; k < kMassLimbs; ++k) d.limb[k] = warp_sum(d.limb[k]);
    if (lane == 0) sh[w] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        DiagPartial s = sh[0];
        for (int i = 1; i < (int)(blockDim.x / 32); ++i) {
            s.mx += sh[i].mx;
            s.my += sh[i].my;
            s.en += sh[i].en;
            s.dres += sh[i].dres;
            s.ures += sh[i].ures;
            s.sres += sh[i].sres;
            s.nonfinite += sh[i].nonfinite;
            for (int k = 0; k < kMassLimbs; ++k) s.limb[k] += sh[i].limb[k];
        }
        *out = s;
    }
}

// The steady residual is taken on the two-step mean velocity
// ubar(n) = (u(n) + u(n-1)) / 2 when the state one step earlier is at hand
// (fprev, the other buffer): the scheme carries exact invariants, the
// staggered momenta sum (-1)^(x+n) rho ux and sum (-1)^(y+n) rho uy, whose
// motion alternates sign every step; a residual between two states an even
// number of steps apart never sees it, and the mean cancels it.  The
// step-to-step change |u(n) - u(n-1)|^2 is summed beside it.
template <typename T, bool MASK>
__global__ void __launch_bounds__(kThreads)
diag_kernel(const T* __restrict__ f, const T* __restrict__ fprev, const AuxParams p,
            double* __restrict__ uprev, int have_prev, DiagPartial* part) {
    const long long N = (long long)p.nx * p.ny;
    DiagPartial d = {};
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const unsigned sb = link_bits<MASK>(p, x, y);
        if (sb == 0xFFu) continue;
        T g[9];
        pull(f, p, x, y, sb, g);
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) ok &= add_fixed(d.limb, (double)g[i]);
        double rho, ux, uy;
        macro(p, g, rho, ux, uy);
        if (!ok || !isfinite(rho) || !isfinite(ux) || !isfinite(uy)) {
            d.nonfinite += 1;
            continue;
        }
        d.mx += rho * ux;
        d.my += rho * uy;
        d.en += 0.5 * rho * (ux * ux + uy * uy);
        double mx = ux, my = uy;
        if (fprev) {
            T q[9];
            pull(fprev, p, x, y, sb, q);
            double r1, ux1, uy1;
            macro(p, q, r1, ux1, uy1);
            const double sx = ux - ux1, sy = uy - uy1;
            d.sres += sx * sx + sy * sy;
            mx = 0.5 * (ux + ux1);
            my = 0.5 * (uy + uy1);
        }
        d.ures += mx * mx + my * my;
        if (have_prev) {
            const double du = mx - uprev[c], dv = my - uprev[N + c];
            d.dres += du * du + dv * dv;
        }
        uprev[c] = mx;
        uprev[N + c] = my;
    }
    block_reduce(d, part + blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) diag_final(DiagPartial* part, int n) {
    DiagPartial d = {};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const DiagPartial& q = part[i];
        d.mx += q.mx;
        d.my += q.my;
        d.en += q.en;
        d.dres += q.dres;
        d.ures += q.ures;
        d.sres += q.sres;
        d.nonfinite += q.nonfinite;
        for (int k = 0; k < kMassLimbs; ++k) d.limb[k] += q.limb[k];
    }
    block_reduce(d, part + n);
}

// Residual sums of one thread summed over the block, in a fixed order.
__device__ void res_block_reduce(ResPartial& d, ResPartial* out) {
    __shared__ ResPartial sh[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    d.dres = warp_sum(d.dres);
    d.ures = warp_sum(d.ures);
    d.nonfinite = warp_sum(d.nonfinite);
    if (lane == 0) sh[w] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        ResPartial s = sh[0];
        for (int i = 1; i < (int)(blockDim.x / 32); ++i) {
            s.dres += sh[i].dres;
            s.ures += sh[i].ures;
            s.nonfinite += sh[i].nonfinite;
        }
        *out = s;
    }
}

// Block w sums reduction chunk w - rbegin[j] of active lattice j: cells
// chunk * kThreads + t + m * nchunk * kThreads.
__global__ void __launch_bounds__(kThreads)
batch_res_kernel(const BatchLattice<float>* __restrict__ lat, const BatchAux* __restrict__ aux,
                 const int* __restrict__ active, const int* __restrict__ rbegin,
                 const int* __restrict__ counts, const int* __restrict__ two, int parity,
                 ResPartial* part) {
    const int n = counts[0];
    const int w = blockIdx.x;
    if (w >= counts[1]) return;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rbegin[mid] <= w) lo = mid;
        else hi = mid - 1;
    }
    const int k = active[lo];
    const BatchAux& B = aux[k];
    const AuxParams& p = B.a;
    const float* f = lat[k].f[parity];
    const float* fp = two[k] ? lat[k].f[parity ^ 1] : nullptr;  // one step earlier
    const int chunk = w - rbegin[lo];
    const long long N = (long long)p.nx * p.ny;
    double* __restrict__ up = B.uprev;
    ResPartial d = {};
    for (long long c = (long long)chunk * kThreads + threadIdx.x; c < N;
         c += (long long)B.nchunk * kThreads) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const unsigned sb = link_bits<true>(p, x, y);
        if (sb == 0xFFu) continue;
        float g[9];
        pull(f, p, x, y, sb, g);
        double rho, ux, uy;
        macro(p, g, rho, ux, uy);
        if (!isfinite(rho) || !isfinite(ux) || !isfinite(uy)) {
            d.nonfinite += 1;
            continue;
        }
        double mx = ux, my = uy;  // the two-step mean velocity, as in diag_kernel
        if (fp) {
            float q[9];
            pull(fp, p, x, y, sb, q);
            double r1, ux1, uy1;
            macro(p, q, r1, ux1, uy1);
            mx = 0.5 * (ux + ux1);
            my = 0.5 * (uy + uy1);
        }
        const double du = mx - up[c], dv = my - up[N + c];
        d.dres += du * du + dv * dv;
        d.ures += mx * mx + my * my;
        up[c] = mx;
        up[N + c] = my;
    }
    res_block_reduce(d, part + B.pbegin + chunk);
}

// Block j sums the chunks of active lattice j in chunk order.
__global__ void __launch_bounds__(kThreads)
batch_res_final(const BatchAux* __restrict__ aux, const int* __restrict__ active,
                const int* __restrict__ counts, const ResPartial* __restrict__ part,
                ResPartial* out) {
    if ((int)blockIdx.x >= counts[0]) return;
    const int k = active[blockIdx.x];
    const BatchAux& B = aux[k];
    ResPartial d = {};
    for (int i = threadIdx.x; i < B.nchunk; i += blockDim.x) {
        const ResPartial& q = part[B.pbegin + i];
        d.dres += q.dres;
        d.ures += q.ures;
        d.nonfinite += q.nonfinite;
    }
    res_block_reduce(d, out + k);
}

int grid_for(long long N) {
    long long b = (N + kThreads - 1) / kThreads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// grid of LBM_FOR_CELLS: blocks across a row, rows down the grid, at most
// 16384 blocks
dim3 grid2_for(int nx, int ny) {
    const int gx = (nx + kThreads - 1) / kThreads;
    const int gy = ny < 16384 / gx ? ny : (16384 / gx > 0 ? 16384 / gx : 1);
    return dim3(gx > 0 ? gx : 1, gy > 0 ? gy : 1);
}

}  // namespace

template <typename T>
cudaError_t launch_init(T* f, const AuxParams& p, const double* rho, const double* ux,
                        const double* uy, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        const int rows = max(kInitRows, (p.ny + 65534) / 65535);  // grid.y limit
        const dim3 g((p.nx + kThreads - 1) / kThreads, (p.ny + rows - 1) / rows);
        if (p.lmask) init32_kernel<true><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy, rows);
        else init32_kernel<false><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy, rows);
    } else {
        const dim3 g = grid2_for(p.nx, p.ny);
        if (p.lmask) init_kernel<true><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
        else init_kernel<false><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_set_f(T* f, const AuxParams& p, const double* fin, cudaStream_t s) {
    const int g = grid_for((long long)p.nx * p.ny);
    if (p.lmask) set_f_kernel<T, true><<<g, kThreads, 0, s>>>(f, p, fin);
    else set_f_kernel<T, false><<<g, kThreads, 0, s>>>(f, p, fin);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_get_f(const T* f, const AuxParams& p, double* fout, cudaStream_t s) {
    const int g = grid_for((long long)p.nx * p.ny);
    if (p.lmask) get_f_kernel<T, true><<<g, kThreads, 0, s>>>(f, p, fout);
    else get_f_kernel<T, false><<<g, kThreads, 0, s>>>(f, p, fout);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_moments(const T* f, const AuxParams& p, double* rho, double* ux,
                           double* uy, cudaStream_t s, bool exact64) {
    const dim3 g = grid2_for(p.nx, p.ny);
    if (exact64) {
        if (p.lmask) moments_kernel<T, true, true><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
        else moments_kernel<T, false, true><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
    } else {
        if (p.lmask) moments_kernel<T, true, false><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
        else moments_kernel<T, false, false><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stress(const T* f, const AuxParams& p, const double* rho, double* dxux,
                          double* dyuy, double* sxy, double* txx, double* tyy, double* txy,
                          cudaStream_t s) {
    const int g = grid_for((long long)p.nx * p.ny);
    if (p.lmask)
        stress_kernel<T, true><<<g, kThreads, 0, s>>>(f, p, rho, dxux, dyuy, sxy, txx, tyy, txy);
    else
        stress_kernel<T, false><<<g, kThreads, 0, s>>>(f, p, rho, dxux, dyuy, sxy, txx, tyy, txy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag(const T* f, const T* fprev, const AuxParams& p, double* uprev,
                        int have_prev, DiagPartial* part, int nblocks, cudaStream_t s) {
    if (p.lmask)
        diag_kernel<T, true><<<nblocks, kThreads, 0, s>>>(f, fprev, p, uprev, have_prev, part);
    else
        diag_kernel<T, false><<<nblocks, kThreads, 0, s>>>(f, fprev, p, uprev, have_prev, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, kThreads, 0, s>>>(part, nblocks);
    return cudaGetLastError();
}

cudaError_t launch_batch_residual(const BatchLattice<float>* lat, const BatchAux* aux,
                                  const int* active, const int* rbegin, const int* counts,
                                  const int* two, int parity, ResPartial* part,
                                  ResPartial* out, int nactive, int nblocks, cudaStream_t s) {
    if (nactive <= 0 || nblocks <= 0) return cudaSuccess;
    batch_res_kernel<<<nblocks, kThreads, 0, s>>>(lat, aux, active, rbegin, counts, two, parity,
                                                  part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_res_final<<<nactive, kThreads, 0, s>>>(aux, active, counts, part, out);
    return cudaGetLastError();
}

#define LBM_AUX_INST(T)                                                                \
    template cudaError_t launch_init<T>(T*, const AuxParams&, const double*,          \
                                        const double*, const double*, cudaStream_t);  \
    template cudaError_t launch_set_f<T>(T*, const AuxParams&, const double*,         \
                                         cudaStream_t);                               \
    template cudaError_t launch_get_f<T>(const T*, const AuxParams&, double*,         \
                                         cudaStream_t);                               \
    template cudaError_t launch_moments<T>(const T*, const AuxParams&, double*,       \
                                           double*, double*, cudaStream_t, bool);     \
    template cudaError_t launch_stress<T>(const T*, const AuxParams&, const double*,  \
                                          double*, double*, double*, double*, double*, \
                                          double*, cudaStream_t);                     \
    template cudaError_t launch_diag<T>(const T*, const T*, const AuxParams&, double*, int, \
                                        DiagPartial*, int, cudaStream_t);
LBM_AUX_INST(float)
LBM_AUX_INST(double)

}  // namespace lbm
