// batch_table.cuh -- the persistent batch kernel with its lattice table in
// constant memory.  Included once by each of rc_batch_t0.cu .. rc_batch_t3.cu,
// which define LBM_BATCH_SLOT (0 .. 3): every translation unit is a module
// with a constant bank of its own, so each holds the table of one group of
// lattices; the groups' kernels run one after another.
//
// Why constant memory: block b takes work items b, b + gridDim.x, ... and
// finds an item's lattice by a binary search over the table; with the table
// in constant memory the search and the lattice's parameters depend only on
// blockIdx and constant data, so the compiler keeps them in uniform
// registers, as in the single-lattice kernel whose parameters are a kernel
// argument (96 registers, 20 warps per SM with 64-thread blocks).  Read from
// a table in global or shared memory, the same parameters take vector
// registers (127, 16 warps per SM).  Measured on the uneven sweep recipe,
// 64-thread blocks, bands of 32 rows: 38.9k against 36.1k MLUPS for 128
// lattices (one table); 39.6k against 38.6k for 512 (four tables, best
// shapes), where each step pays four kernel tails.
//
// The block's work is step_block's, so a lattice goes through the same states
// bit for bit as with the single-lattice kernel.
#pragma once
#include "step_block.cuh"

#ifndef LBM_BATCH_SLOT
#error "define LBM_BATCH_SLOT (0 .. kBatchTables - 1) before including batch_table.cuh"
#endif

#define LBM_PASTE2(a, b) a##b
#define LBM_PASTE(a, b) LBM_PASTE2(a, b)
#define LBM_SLOT_NAME(n) LBM_PASTE(n, LBM_BATCH_SLOT)

namespace lbm {

namespace {

__constant__ BatchTableLattice c_table[kBatchTableCap];
// first work item of each lattice; c_table_begin[c_table_n] = the group's
// number of work items
__constant__ int c_table_begin[kBatchTableCap + 1];
__constant__ int c_table_n;

template <int BXT, int SCH>
__global__ void __launch_bounds__(BXT, step_min_blocks<float>(BXT))
batch_table_kernel(int parity) {
    extern __shared__ __align__(128) unsigned char smem[];
    // the counts are read from the constant bank where they are used: held
    // in locals across the loop they cost registers and the kernel spilled
    for (int w = blockIdx.x; w < c_table_begin[c_table_n]; w += gridDim.x) {
        int lo = 0, hi = c_table_n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (c_table_begin[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const BatchTableLattice& L = c_table[lo];
        const int local = w - c_table_begin[lo];
        // lattices of a batch stay below 2^31 elements (checked on the host)
        if (!step_block<float, true, BXT, int, SCH, const KParams<float, CollConstF>&>(
                L.f[parity], L.f[parity ^ 1], L.kp, L.nbands, local % L.nseg, local / L.nseg,
                smem))
            return;
    }
}

template <int BXT, int SCH>
cudaError_t launch_table_bx(int parity, int grid, cudaStream_t s) {
    constexpr size_t smem = step_smem_bytes<float, BXT>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(batch_table_kernel<BXT, SCH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    batch_table_kernel<BXT, SCH><<<grid, BXT, smem, s>>>(parity);
    return cudaGetLastError();
}

template <int SCH>
cudaError_t launch_table_sch(int parity, int bx, int grid, cudaStream_t s) {
    switch (bx) {
    case 32: return launch_table_bx<32, SCH>(parity, grid, s);
    case 64: return launch_table_bx<64, SCH>(parity, grid, s);
    case 128: return launch_table_bx<128, SCH>(parity, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int BXT>
int table_occ_bx() {
    constexpr size_t smem = step_smem_bytes<float, BXT>();
    cudaFuncSetAttribute(batch_table_kernel<BXT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_table_kernel<BXT, 0>, BXT, smem) !=
        cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

}  // namespace

cudaError_t LBM_SLOT_NAME(batch_table_upload_)(const BatchTableLattice* lat, const int* begin,
                                               int n, cudaStream_t s) {
    if (n < 1 || n > kBatchTableCap) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyToSymbolAsync(c_table, lat, sizeof(BatchTableLattice) * (size_t)n, 0,
                                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbolAsync(c_table_begin, begin, sizeof(int) * (size_t)(n + 1), 0,
                                cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_table_n, &n, sizeof(int), 0, cudaMemcpyHostToDevice, s);
}

cudaError_t LBM_SLOT_NAME(batch_table_launch_)(int parity, int bx, int grid, int raw,
                                               cudaStream_t s) {
    return raw ? launch_table_sch<1>(parity, bx, grid, s) : launch_table_sch<0>(parity, bx, grid, s);
}

int LBM_SLOT_NAME(batch_table_occupancy_)(int bx) {
    return bx == 32 ? table_occ_bx<32>() : bx == 64 ? table_occ_bx<64>() : table_occ_bx<128>();
}

}  // namespace lbm

#undef LBM_SLOT_NAME
#undef LBM_PASTE
#undef LBM_PASTE2
