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

template <typename T, bool MASK>
__global__ void init_kernel(T* __restrict__ f, const AuxParams p, const double* rho,
                            const double* ux, const double* uy) {
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
        const double r0 = rho ? rho[c] : 1.0, u0 = ux ? ux[c] : 0.0,
                     v0 = uy ? uy[c] : 0.0;
        for (int i = 0; i < 9; ++i) {
            double v;
            if (i > 0 && ((sb >> (opp(i) - 1)) & 1u)) {
                v = feq_d(opp(i), r0, u0, v0, p.cs2, p.a);  // pulled back by c itself
            } else {
                const long long t = i == 0 ? c : target(p, x, y, i);
                v = feq_d(i, rho ? rho[t] : 1.0, ux ? ux[t] : 0.0, uy ? uy[t] : 0.0,
                          p.cs2, p.a);
            }
            f[i * p.plane + o] = T(v - p.wrest[i]);
        }
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

template <typename T, bool MASK>
__global__ void moments_kernel(const T* __restrict__ f, const AuxParams p,
                               double* rho, double* ux, double* uy) {
    const long long N = (long long)p.nx * p.ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % p.nx), y = (int)(c / p.nx);
        const unsigned sb = link_bits<MASK>(p, x, y);
        double r = 0.0, u = 0.0, v = 0.0;
        if (sb != 0xFFu) {
            T g[9];
            pull(f, p, x, y, sb, g);
            macro(p, g, r, u, v);
        }
        if (rho) rho[c] = r;
        if (ux) ux[c] = u;
        if (uy) uy[c] = v;
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
            s.nonfinite += sh[i].nonfinite;
            for (int k = 0; k < kMassLimbs; ++k) s.limb[k] += sh[i].limb[k];
        }
        *out = s;
    }
}

template <typename T, bool MASK>
__global__ void __launch_bounds__(kThreads)
diag_kernel(const T* __restrict__ f, const AuxParams p, double* __restrict__ uprev,
            int have_prev, DiagPartial* part) {
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
        d.ures += ux * ux + uy * uy;
        if (have_prev) {
            const double du = ux - uprev[c], dv = uy - uprev[N + c];
            d.dres += du * du + dv * dv;
        }
        uprev[c] = ux;
        uprev[N + c] = uy;
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
        d.nonfinite += q.nonfinite;
        for (int k = 0; k < kMassLimbs; ++k) d.limb[k] += q.limb[k];
    }
    block_reduce(d, part + n);
}

int grid_for(long long N) {
    long long b = (N + kThreads - 1) / kThreads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

template <typename T>
cudaError_t launch_init(T* f, const AuxParams& p, const double* rho, const double* ux,
                        const double* uy, cudaStream_t s) {
    const int g = grid_for((long long)p.nx * p.ny);
    if (p.lmask) init_kernel<T, true><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
    else init_kernel<T, false><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
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
                           double* uy, cudaStream_t s) {
    const int g = grid_for((long long)p.nx * p.ny);
    if (p.lmask) moments_kernel<T, true><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
    else moments_kernel<T, false><<<g, kThreads, 0, s>>>(f, p, rho, ux, uy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag(const T* f, const AuxParams& p, double* uprev, int have_prev,
                        DiagPartial* part, int nblocks, cudaStream_t s) {
    if (p.lmask) diag_kernel<T, true><<<nblocks, kThreads, 0, s>>>(f, p, uprev, have_prev, part);
    else diag_kernel<T, false><<<nblocks, kThreads, 0, s>>>(f, p, uprev, have_prev, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final<<<1, kThreads, 0, s>>>(part, nblocks);
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
                                           double*, double*, cudaStream_t);           \
    template cudaError_t launch_diag<T>(const T*, const AuxParams&, double*, int,     \
                                        DiagPartial*, int, cudaStream_t);
LBM_AUX_INST(float)
LBM_AUX_INST(double)

}  // namespace lbm
