// rc_step.cu -- the fused collide-and-stream step of the RC-LBM
// (arXiv 2103.02119, Sec. 4) for sm_103a, FP32 and FP64.
//
// One launch advances the whole lattice by one time step.  Each thread block
// owns a segment of BX columns and a band of rows, and marches through its
// band one row at a time:
//   1. pull-stream the nine populations of the next row (bounce-back at
//      walls and solids) into registers and put the row's density into a
//      four-row ring in shared memory (the block also computes the density of
//      the two columns just outside its segment, and the row before and after
//      its band, so that every cell has its four axial neighbours);
//   2. one __syncthreads;
//   3. collide the previous row: its density gradient comes from the ring by
//      central differences (spacing 2 along x, 2a along y, a wall or solid
//      neighbour mirrors the cell's own density), the collision runs in
//      registers, and the result goes to its own cell in the output buffer.
// Even bands march up, odd bands march down, so that the rows two
// neighbouring bands both read are read at about the same time.
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace lbm {

template <typename T, bool MASK, int BX>
__global__ void __launch_bounds__(BX)
rc_step_kernel(const T* __restrict__ fin, T* __restrict__ fout, const KParams<T> p,
               int nbands) {
    __shared__ T ring[4][BX + 2];
    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * BX;
    const int x = x0 + tx;
    const int nseg = min(BX, p.nx - x0);
    const bool active = tx < nseg;
    const int band = blockIdx.y;
    const int y0 = (int)(((long long)band * p.ny) / nbands);
    const int y1 = (int)(((long long)(band + 1) * p.ny) / nbands);
    const int dir = (band & 1) ? -1 : 1;
    const int rfirst = dir > 0 ? y0 - 1 : y1;
    const int nit = (y1 - y0) + 2;
    const long long pl = p.plane;

    T Pp[9];                 // populations of the previous row (to collide)
    unsigned bp = 0xFFu;     // its link bits (0xFF: nothing to collide)
    T dp = T(0);             // its density deviation

    for (int k = 0; k < nit; ++k) {
        const int r = rfirst + dir * k;
        const int slot = k & 3;
        const bool rin = r >= 0 && r < p.ny;
        const int rr = rin ? r : (r < 0 ? r + p.ny : r - p.ny);
        T Pc[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Pc[i] = T(0);
        unsigned bc = 0xFFu;
        T dc = T(0);
        if (rin || p.py) {
            if (active) {
                bc = link_bits<MASK>(p, x, rr);
                if (bc != 0xFFu) {
                    pull(fin, p, x, rr, bc, Pc);
                    dc = ((Pc[0] + Pc[1]) + (Pc[2] + Pc[3])) +
                         ((Pc[4] + Pc[5]) + (Pc[6] + Pc[7])) + Pc[8];
                }
                ring[slot][tx + 1] = dc;
            }
            if (tx < 2) {  // density of the columns just outside the segment
                int hx = tx == 0 ? x0 - 1 : x0 + nseg;
                const int si = tx == 0 ? 0 : nseg + 1;
                bool ok = true;
                if (hx < 0) { if (p.px) hx += p.nx; else ok = false; }
                else if (hx >= p.nx) { if (p.px) hx -= p.nx; else ok = false; }
                if (ok) {
                    const unsigned hb = link_bits<MASK>(p, hx, rr);
                    T hd = T(0);
                    if (hb != 0xFFu) {
                        T Ph[9];
                        pull(fin, p, hx, rr, hb, Ph);
                        hd = ((Ph[0] + Ph[1]) + (Ph[2] + Ph[3])) +
                             ((Ph[4] + Ph[5]) + (Ph[6] + Ph[7])) + Ph[8];
                    }
                    ring[slot][si] = hd;
                }
            }
        }
        __syncthreads();
        if (k >= 2 && bp != 0xFFu) {
            const int rc = r - dir;
            const int sC = (k - 1) & 3;
            const int sN = dir > 0 ? (k & 3) : ((k - 2) & 3);
            const int sS = dir > 0 ? ((k - 2) & 3) : (k & 3);
            const T dW = (bp & 1u) ? dp : ring[sC][tx];
            const T dS = (bp & 2u) ? dp : ring[sS][tx + 1];
            const T dE = (bp & 4u) ? dp : ring[sC][tx + 2];
            const T dN = (bp & 8u) ? dp : ring[sN][tx + 1];
            const T dxr = T(0.5) * (dE - dW);
            const T dyr = p.iah * (dN - dS);
            const T rho = p.collide ? collide(p, Pp, dp, dxr, dyr) : p.rho0 + dp;
            if (p.moving && (x == 0 || x == p.nx - 1 || rc == 0 || rc == p.ny - 1))
                moving_wall(p, x, rc, rho, Pp);
            const long long o = (long long)rc * p.pitch + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) fout[i * pl + o] = Pp[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) Pp[i] = Pc[i];
        bp = bc;
        dp = dc;
    }
}

template <typename T, bool MASK, int BX>
static cudaError_t launch_bx(const T* fin, T* fout, const KParams<T>& p, int nbands,
                             cudaStream_t s) {
    dim3 grid((p.nx + BX - 1) / BX, nbands);
    rc_step_kernel<T, MASK, BX><<<grid, BX, 0, s>>>(fin, fout, p, nbands);
    return cudaGetLastError();
}

template <typename T, bool MASK>
static cudaError_t launch_mask(const T* fin, T* fout, const KParams<T>& p, int bx,
                               int nbands, cudaStream_t s) {
    switch (bx) {
    case 32: return launch_bx<T, MASK, 32>(fin, fout, p, nbands, s);
    case 64: return launch_bx<T, MASK, 64>(fin, fout, p, nbands, s);
    case 128: return launch_bx<T, MASK, 128>(fin, fout, p, nbands, s);
    case 256: return launch_bx<T, MASK, 256>(fin, fout, p, nbands, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_step(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                        cudaStream_t s) {
    return p.lmask ? launch_mask<T, true>(fin, fout, p, bx, nbands, s)
                   : launch_mask<T, false>(fin, fout, p, bx, nbands, s);
}
template cudaError_t launch_step<float>(const float*, float*, const KParams<float>&,
                                        int, int, cudaStream_t);
template cudaError_t launch_step<double>(const double*, double*,
                                         const KParams<double>&, int, int,
                                         cudaStream_t);

template <typename T, bool MASK, int BX>
static int occ_bx() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rc_step_kernel<T, MASK, BX>,
                                                      BX, 0) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <typename T>
int step_occupancy(int bx, bool mask) {
    switch (bx) {
    case 32: return mask ? occ_bx<T, true, 32>() : occ_bx<T, false, 32>();
    case 64: return mask ? occ_bx<T, true, 64>() : occ_bx<T, false, 64>();
    case 128: return mask ? occ_bx<T, true, 128>() : occ_bx<T, false, 128>();
    default: return mask ? occ_bx<T, true, 256>() : occ_bx<T, false, 256>();
    }
}
template int step_occupancy<float>(int, bool);
template int step_occupancy<double>(int, bool);

}  // namespace lbm
