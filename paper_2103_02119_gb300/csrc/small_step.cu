// small_step.cu -- many steps of a small lattice in one launch (Sec. 4, the
// same fused step as step_block.cuh), for lattices whose step is bound by
// launch and synchronisation latency rather than by memory.
//
// One thread-block cluster of C CTAs (C <= 16) runs all the steps.  CTA b
// owns rows [b ny / C, (b+1) ny / C); its threads take the band's cells in
// turn.  Per step:
//   1. every cell pulls its populations (L2 loads that bypass L1, as the
//      other CTAs write them) and writes its density deviation to a small
//      density field;
//   2. cluster barrier (release / acquire);
//   3. every cell pulls again, takes its density gradient from the field
//      (central differences; a wall or solid neighbour mirrors the cell's
//      own density), collides, adds the moving-wall term and stores;
//   4. cluster barrier; the buffers swap.
// Every CTA runs the same number of steps and barriers, with no early exit
// (a checked build skips an access that fails its bounds test and records
// bit 1 of the status word at the end).
// The arithmetic is that of step_block in the same order (the FP32 collision
// on a float2 lane pair whose lanes are independent), so a lattice goes
// through the same states bit for bit on either path.
#include <cooperative_groups.h>

#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace cg = cooperative_groups;

namespace lbm {

namespace {

constexpr int kSmallThreads = 256;  // per CTA; a CTA loops over its band's cells

// pull() with loads that bypass L1 (the state is written by other CTAs of
// the cluster within the launch)
template <typename S, typename P>
__device__ __forceinline__ void pull_l2(const S* fin, const P& p, int x, int y, unsigned sb,
                                        S f[9], bool& bad) {
    const int xm = x == 0 ? p.nx - 1 : x - 1;
    const int xp = x == p.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? p.ny - 1 : y - 1;
    const int yp = y == p.ny - 1 ? 0 : y + 1;
    const long long pl = p.plane;
    const long long rc = (long long)y * p.rstride, rm = (long long)ym * p.rstride,
                    rp = (long long)yp * p.rstride;
    const long long c = rc + x;
    if constexpr (kChecked) {
        const long long n = 9 * pl;
        const long long idx[9] = {c,
                                  (sb & 1u) ? 3 * pl + c : 1 * pl + rc + xm,
                                  (sb & 2u) ? 4 * pl + c : 2 * pl + rm + x,
                                  (sb & 4u) ? 1 * pl + c : 3 * pl + rc + xp,
                                  (sb & 8u) ? 2 * pl + c : 4 * pl + rp + x,
                                  (sb & 16u) ? 7 * pl + c : 5 * pl + rm + xm,
                                  (sb & 32u) ? 8 * pl + c : 6 * pl + rm + xp,
                                  (sb & 64u) ? 5 * pl + c : 7 * pl + rp + xp,
                                  (sb & 128u) ? 6 * pl + c : 8 * pl + rp + xm};
        bool ok = true;
#pragma unroll
        for (int i = 0; i < 9; ++i) ok = ok && idx_ok(idx[i], n);
        if (!ok) {
            bad = true;
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = S(0);
            return;
        }
    }
    f[0] = __ldcg(fin + c);
    f[1] = __ldcg(fin + ((sb & 1u) ? 3 * pl + c : 1 * pl + rc + xm));
    f[2] = __ldcg(fin + ((sb & 2u) ? 4 * pl + c : 2 * pl + rm + x));
    f[3] = __ldcg(fin + ((sb & 4u) ? 1 * pl + c : 3 * pl + rc + xp));
    f[4] = __ldcg(fin + ((sb & 8u) ? 2 * pl + c : 4 * pl + rp + x));
    f[5] = __ldcg(fin + ((sb & 16u) ? 7 * pl + c : 5 * pl + rm + xm));
    f[6] = __ldcg(fin + ((sb & 32u) ? 8 * pl + c : 6 * pl + rm + xp));
    f[7] = __ldcg(fin + ((sb & 64u) ? 5 * pl + c : 7 * pl + rp + xp));
    f[8] = __ldcg(fin + ((sb & 128u) ? 6 * pl + c : 8 * pl + rp + xm));
}

// the density deviation, summed in step_block's order
template <typename T>
__device__ __forceinline__ T dens(const T g[9]) {
    return ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
}

template <typename T, bool MASK>
__global__ void __launch_bounds__(kSmallThreads) small_run_kernel(T* f0, T* f1, T* dfield,
                                                         const __grid_constant__ KParams<T> p,
                                                         int from, int nsteps) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)gridDim.x;
    const int b = (int)blockIdx.x;
    const int y0 = (int)((long long)b * p.ny / C), y1 = (int)((long long)(b + 1) * p.ny / C);
    const int ncell = (y1 - y0) * p.nx;
    const long long ncells = (long long)p.nx * p.ny;  // elements of the density field
    bool bad = false;  // checked build: a failed bounds check (the access is skipped)
    auto bits = [&](int x, int y) -> unsigned {
        if constexpr (MASK) return mask_at(p, (long long)y * p.pitch + x, bad);
        return link_bits<false>(p, x, y);
    };
    auto dload = [&](long long i) -> T {
        if (kChecked && !idx_ok(i, ncells)) {
            bad = true;
            return T(0);
        }
        return __ldcg(dfield + i);
    };
    for (int s = 0; s < nsteps; ++s) {
        const T* fin = ((from + s) & 1) ? f1 : f0;
        T* fout = ((from + s) & 1) ? f0 : f1;
        // 1. densities
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int y = y0 + c / p.nx, x = c % p.nx;
            const unsigned sb = bits(x, y);
            T d = T(0);
            if (sb != 0xFFu) {
                T g[9];
                pull_l2(fin, p, x, y, sb, g, bad);
                d = dens(g);
            }
            const long long di = (long long)y * p.nx + x;
            if (kChecked && !idx_ok(di, ncells))
                bad = true;
            else
                dfield[di] = d;
        }
        cluster.sync();
        // 3. collide and store
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            const int y = y0 + c / p.nx, x = c % p.nx;
            const unsigned sb = bits(x, y);
            const long long o = (long long)y * p.rstride + x;
            if (kChecked && !(y >= 0 && y < p.ny && x >= 0 && x < p.rstride)) {
                bad = true;
                continue;
            }
            T g[9];
            if (sb == 0xFFu) {
#pragma unroll
                for (int i = 0; i < 9; ++i) fout[i * p.plane + o] = T(0);
                continue;
            }
            pull_l2(fin, p, x, y, sb, g, bad);
            const T d = dens(g);
            const int xw = x == 0 ? p.nx - 1 : x - 1, xe = x == p.nx - 1 ? 0 : x + 1;
            const int ys = y == 0 ? p.ny - 1 : y - 1, yn = y == p.ny - 1 ? 0 : y + 1;
            const T dW = (sb & 1u) ? d : dload((long long)y * p.nx + xw);
            const T dS = (sb & 2u) ? d : dload((long long)ys * p.nx + x);
            const T dE = (sb & 4u) ? d : dload((long long)y * p.nx + xe);
            const T dN = (sb & 8u) ? d : dload((long long)yn * p.nx + x);
            const T dxr = T(0.5) * (dE - dW);
            const T dyr = p.iah * (dN - dS);
            T rho = p.rho0 + d;
            if (p.collide) {
                if constexpr (sizeof(T) == 4) {
                    float2 F[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) F[i] = make_float2(g[i], g[i]);
                    const float2 D = make_float2(d, d), Gx = make_float2(dxr, dxr),
                                 Gy = make_float2(dyr, dyr);
                    const float2 R = p.raw ? collide_raw<float>(CollConst<float>(p.cc), F, D, Gx, Gy)
                                           : (p.forced ? collide<float, true>(CollConst<float>(p.cc), F, D, Gx, Gy)
                                                       : collide<float, false>(CollConst<float>(p.cc), F, D, Gx, Gy));
                    rho = R.x;
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = F[i].x;
                } else {
                    rho = p.raw ? collide_raw<T>(CollConst<T>(p.cc), g, d, dxr, dyr)
                                : (p.forced ? collide<T, true>(CollConst<T>(p.cc), g, d, dxr, dyr)
                                            : collide<T, false>(CollConst<T>(p.cc), g, d, dxr, dyr));
                }
            }
            if (p.moving && (x == 0 || x == p.nx - 1 || y == 0 || y == p.ny - 1))
                moving_wall(p, x, y, rho, g);
#pragma unroll
            for (int i = 0; i < 9; ++i) fout[i * p.plane + o] = g[i];
        }
        cluster.sync();
    }
    if (kChecked && bad) atomicOr(p.status, kStatusBounds);
}

template <typename T, bool MASK>
cudaLaunchConfig_t small_config(const KParams<T>& p, int csize, cudaStream_t s,
                                cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize, 1, 1);
    const int per = (p.ny + csize - 1) / csize * p.nx;
    cfg.blockDim = dim3(per < kSmallThreads ? (per + 31) / 32 * 32 : kSmallThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <typename T, bool MASK>
cudaError_t configure_small() {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(small_run_kernel<T, MASK>,
                                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    return cudaSuccess;
}

template <typename T, bool MASK>
cudaError_t launch_small_mask(T* f0, T* f1, T* dfield, const KParams<T>& p, int from, int nsteps,
                              int csize, cudaStream_t s) {
    if (cudaError_t e = configure_small<T, MASK>(); e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = small_config<T, MASK>(p, csize, s, attr);
    return cudaLaunchKernelEx(&cfg, small_run_kernel<T, MASK>, f0, f1, dfield, p, from, nsteps);
}

template <typename T, bool MASK>
bool small_fits_mask(const KParams<T>& p, int csize) {
    if (configure_small<T, MASK>() != cudaSuccess) return false;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = small_config<T, MASK>(p, csize, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, small_run_kernel<T, MASK>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

int small_cluster_size(int ny) { return ny < kSmallCluster ? ny : kSmallCluster; }

}  // namespace

template <typename T>
cudaError_t launch_small_run(T* f0, T* f1, T* dfield, const KParams<T>& p, int from, int nsteps,
                             cudaStream_t s) {
    if (nsteps <= 0) return cudaSuccess;
    const int csize = small_cluster_size(p.ny);
    return p.lmask ? launch_small_mask<T, true>(f0, f1, dfield, p, from, nsteps, csize, s)
                   : launch_small_mask<T, false>(f0, f1, dfield, p, from, nsteps, csize, s);
}

template <typename T>
bool small_run_fits(const KParams<T>& p) {
    const int csize = small_cluster_size(p.ny);
    return p.lmask ? small_fits_mask<T, true>(p, csize) : small_fits_mask<T, false>(p, csize);
}
template bool small_run_fits<float>(const KParams<float>&);
template bool small_run_fits<double>(const KParams<double>&);

template cudaError_t launch_small_run<float>(float*, float*, float*, const KParams<float>&, int,
                                             int, cudaStream_t);
template cudaError_t launch_small_run<double>(double*, double*, double*,
                                              const KParams<double>&, int, int, cudaStream_t);

}  // namespace lbm
