// rc_step.cu -- kernels of the fused step with the RC-LBM collision
// (Sec. 4), the persistent batch kernel, and the launch dispatch.  The
// block's work is in step_block.cuh.
#include "step_block.cuh"

namespace lbm {

// Persistent kernel over many lattices of one scheme (SCH: 0 RC-LBM or no
// collision, 1 RNR-LBM): block b takes work items b,
// b + gridDim.x, ... of a device work list; item w belongs to the active
// lattice whose block range [begin, begin + nseg * nbands) holds w.  The
// lattice's parameters are copied from the (read-only) lattice table into
// shared memory for the item, so the collision reads its constants there.
// Bounded to 128 registers (four 128-thread blocks per SM): the parameters
// read from shared memory need more registers than the single-lattice
// step's constant-bank operands; at 96 registers the kernel spills, and
// unbounded (168 registers, three blocks) it ran 18 % slower.
template <typename T, int BXT, int SCH>
__global__ void __launch_bounds__(BXT, 512 / BXT)
rc_batch_kernel(const BatchLattice<T>* __restrict__ lat, const int* __restrict__ active,
                const int* __restrict__ begin, const int* __restrict__ counts, int parity) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(16) int kwords[sizeof(KParams<T>) / 4];
    static_assert(sizeof(KParams<T>) % 4 == 0, "lattice parameters copy as words");
    const int n = counts[0], total = counts[1];
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(begin + mid) <= w) lo = mid;
            else hi = mid - 1;
        }
        const BatchLattice<T>* L = lat + __ldg(active + lo);
        const int local = w - __ldg(begin + lo);
        __syncthreads();  // the previous item is done with kwords
        for (int i = threadIdx.x; i < (int)(sizeof(KParams<T>) / 4); i += BXT)
            kwords[i] = __ldg(reinterpret_cast<const int*>(&L->kp) + i);
        __syncthreads();
        const KParams<T>& kp = *reinterpret_cast<const KParams<T>*>(kwords);
        const int nseg = L->nseg;
        const T* fin = L->f[parity];
        T* fout = L->f[parity ^ 1];
        // lattices of a batch stay below 2^31 elements (checked on the host)
        if (!step_block<T, true, BXT, int, SCH, const KParams<T>&>(fin, fout, kp, L->nbands,
                                                              local % nseg, local / nseg, smem))
            return;
    }
}

template <typename T, int BXT, int SCH>
static cudaError_t launch_batch_bx(const BatchLattice<T>* lat, const int* active,
                                   const int* begin, const int* counts, int parity, int grid,
                                   cudaStream_t s) {
    constexpr size_t smem = step_smem_bytes<T, BXT>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(rc_batch_kernel<T, BXT, SCH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    rc_batch_kernel<T, BXT, SCH><<<grid, BXT, smem, s>>>(lat, active, begin, counts, parity);
    return cudaGetLastError();
}

template <typename T, int SCH>
static cudaError_t launch_batch_sch(const BatchLattice<T>* lat, const int* active,
                                    const int* begin, const int* counts, int parity, int bx,
                                    int grid, cudaStream_t s) {
    switch (bx) {
    case 32: return launch_batch_bx<T, 32, SCH>(lat, active, begin, counts, parity, grid, s);
    case 64: return launch_batch_bx<T, 64, SCH>(lat, active, begin, counts, parity, grid, s);
    case 128: return launch_batch_bx<T, 128, SCH>(lat, active, begin, counts, parity, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_batch_step(const BatchLattice<T>* lat, const int* active, const int* begin,
                              const int* counts, int parity, int bx, int grid, int raw,
                              cudaStream_t s) {
    return raw ? launch_batch_sch<T, 1>(lat, active, begin, counts, parity, bx, grid, s)
               : launch_batch_sch<T, 0>(lat, active, begin, counts, parity, bx, grid, s);
}
template cudaError_t launch_batch_step<float>(const BatchLattice<float>*, const int*,
                                              const int*, const int*, int, int, int, int,
                                              cudaStream_t);

template <typename T, int BXT>
static int batch_occ_bx() {
    constexpr size_t smem = step_smem_bytes<T, BXT>();
    cudaFuncSetAttribute(rc_batch_kernel<T, BXT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rc_batch_kernel<T, BXT, 0>, BXT, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <typename T>
int batch_occupancy(int bx) {
    return bx == 32 ? batch_occ_bx<T, 32>() : bx == 64 ? batch_occ_bx<T, 64>()
                                                       : batch_occ_bx<T, 128>();
}
template int batch_occupancy<float>(int);

template <typename T>
cudaError_t launch_step(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                        cudaStream_t s) {
    if (p.collide && p.raw) return launch_step_rnr<T>(fin, fout, p, bx, nbands, s);
    // flows without a body force take the collision with the force terms
    // compiled out
    if (p.collide && !p.forced) return launch_step_free<T>(fin, fout, p, bx, nbands, s);
    return launch_step_scheme<T, 0>(fin, fout, p, bx, nbands, s);
}
template cudaError_t launch_step<float>(const float*, float*, const KParams<float>&,
                                        int, int, cudaStream_t);
template cudaError_t launch_step<double>(const double*, double*,
                                         const KParams<double>&, int, int,
                                         cudaStream_t);

template <typename T, bool MASK, int BXT>
static int occ_bx() {
    constexpr size_t smem = step_smem_bytes<T, BXT>();
    cudaFuncSetAttribute(rc_step_kernel<T, MASK, BXT, int, 0>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rc_step_kernel<T, MASK, BXT, int, 0>,
                                                      BXT, smem) != cudaSuccess)
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

template <typename T>
int step_segment_width(int bx) { return bx * step_cells_per_thread<T>(); }
template int step_segment_width<float>(int);
template int step_segment_width<double>(int);

}  // namespace lbm
