// lbm_launch.h -- host-side entry points of the kernels (internal to the
// library; the public interface is include/lbm.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "lbm_device.cuh"

namespace lbm {

// Polls of the step kernels' bounded mbarrier waits (the default of
// KParams::spin_limit and the bound of the drain after a wait ran out).
constexpr unsigned kWaitPolls = 1u << 22;

// Fixed-point accumulator of the exact mass: value = sum_k limb[k] 2^(24k - 144).
constexpr int kMassLimbs = 8;
constexpr int kMassShift = 144;
// Per-block partial results of the diagnostics reduction.
struct DiagPartial {
    // sum rho ux, rho uy, rho |u|^2 / 2 over the current state; |ubar - uref|^2,
    // |ubar|^2 of the two-step mean ubar = (u(n) + u(n-1)) / 2; |u(n) - u(n-1)|^2
    double mx, my, en, dres, ures, sres;
    long long nonfinite;
    long long limb[kMassLimbs];
};

template <typename T>
cudaError_t launch_step(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                        cudaStream_t s);
// the same with the raw-moment collision (RNR-LBM); launch_step calls it
// when p.raw is set
template <typename T>
cudaError_t launch_step_rnr(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                            cudaStream_t s);
// The RC-LBM step of a lattice without a body force (the force terms of the
// collision compiled out).
template <typename T>
cudaError_t launch_step_free(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                             cudaStream_t s);
template <typename T>
int step_occupancy(int bx, bool mask);

// Small lattices (at most kSmallCells cells): nsteps steps in one launch of
// one thread-block cluster of min(ny, kSmallCluster) CTAs, from buffer
// `from` (f0 or f1); dfield: nx*ny values of T (the density field of a step).
constexpr long long kSmallCells = 4096;
constexpr int kSmallCluster = 16;
template <typename T>
cudaError_t launch_small_run(T* f0, T* f1, T* dfield, const KParams<T>& p, int from, int nsteps,
                             cudaStream_t s);
// whether such a cluster launch fits this device (queried, no launch)
template <typename T>
bool small_run_fits(const KParams<T>& p);
// columns of lattice one block of bx threads of the step kernel covers
template <typename T>
int step_segment_width(int bx);

// One lattice of a batch, as the persistent batch kernel sees it.
template <typename T>
struct BatchLattice {
    KParams<T> kp;        // its parameters (kp.lmask always set)
    T* f[2];              // its two population buffers
    int nseg, nbands;     // its work items: nseg * nbands blocks
};
// One step of every lattice of a work list (all of one scheme: raw = 1 for
// RNR-LBM, else RC-LBM or no collision): counts = {number of lattices, total
// work items}, begin[k] = first work item of active[k].
template <typename T>
cudaError_t launch_batch_step(const BatchLattice<T>* lat, const int* active, const int* begin,
                              const int* counts, int parity, int bx, int grid, int raw,
                              cudaStream_t s);
template <typename T>
int batch_occupancy(int bx);

// One lattice of a group of a batch, in a constant-memory table
// (batch_table.cuh): its parameters with the collision constants stored once
// each, its buffers and its work items (nseg * nbands; where they start in
// the group's list the table keeps in an array of its own).
struct BatchTableLattice {
    KParams<float, CollConstF> kp;
    float* f[2];
    int nseg, nbands;
};
// Tables (translation units rc_batch_t0.cu ..), and lattices per table: a
// module's constant bank holds 64 KiB.
constexpr int kBatchTables = 4;
constexpr int kBatchTableCap = 62000 / (int)sizeof(BatchTableLattice);
#define LBM_DECLARE_BATCH_TABLE(S)                                                         \
    cudaError_t batch_table_upload_##S(const BatchTableLattice* lat, const int* begin, int n, \
                                       cudaStream_t s);                                     \
    cudaError_t batch_table_launch_##S(int parity, int bx, int grid, int raw, cudaStream_t s); \
    int batch_table_occupancy_##S(int bx);
LBM_DECLARE_BATCH_TABLE(0)
LBM_DECLARE_BATCH_TABLE(1)
LBM_DECLARE_BATCH_TABLE(2)
LBM_DECLARE_BATCH_TABLE(3)
#undef LBM_DECLARE_BATCH_TABLE
// Table `slot`: copy n lattices (host array) and their first work items
// begin[0 .. n] (begin[n]: the group's number of work items) into it,
// asynchronously on s (after the kernels of the slot that were issued before
// on s; the caller orders them).
inline cudaError_t batch_table_upload(int slot, const BatchTableLattice* lat, const int* begin,
                                      int n, cudaStream_t s) {
    return slot == 0   ? batch_table_upload_0(lat, begin, n, s)
           : slot == 1 ? batch_table_upload_1(lat, begin, n, s)
           : slot == 2 ? batch_table_upload_2(lat, begin, n, s)
                       : batch_table_upload_3(lat, begin, n, s);
}
// One step of every lattice of table `slot` (all of one scheme: raw = 1 for
// RNR-LBM), from buffer f[parity], on a persistent grid of `grid` blocks.
inline cudaError_t batch_table_launch(int slot, int parity, int bx, int grid, int raw,
                                      cudaStream_t s) {
    return slot == 0   ? batch_table_launch_0(parity, bx, grid, raw, s)
           : slot == 1 ? batch_table_launch_1(parity, bx, grid, raw, s)
           : slot == 2 ? batch_table_launch_2(parity, bx, grid, raw, s)
                       : batch_table_launch_3(parity, bx, grid, raw, s);
}
inline int batch_table_occupancy(int slot, int bx) {
    return slot == 0   ? batch_table_occupancy_0(bx)
           : slot == 1 ? batch_table_occupancy_1(bx)
           : slot == 2 ? batch_table_occupancy_2(bx)
                       : batch_table_occupancy_3(bx);
}

// One lattice of a batch, as the batch residual kernels see it.
struct BatchAux {
    AuxParams a;      // a.lmask always set
    double* uprev;    // 2 * nx * ny doubles: the velocity at the last check
    int nchunk;       // reduction blocks of this lattice
    int pbegin;       // index of its first partial sum
};
// Sums of the steady-state residual of one lattice: sum |u - uprev|^2,
// sum |u|^2 over its fluid cells, and the number of non-finite cells.
struct ResPartial {
    double dres, ures;
    long long nonfinite;
};
// Residual sums of every active lattice from its FP32 state lat[k].f[parity]
// and, where two[k] != 0, its state one step earlier lat[k].f[parity ^ 1]
// (the residual is then on the two-step mean velocity): counts = {active
// lattices, total reduction blocks}, rbegin[j] = first block of active[j];
// writes out[active[j]] and overwrites uprev.  The host passes the same two
// counts as nactive / nblocks (launch sizes).
cudaError_t launch_batch_residual(const BatchLattice<float>* lat, const BatchAux* aux,
                                  const int* active, const int* rbegin, const int* counts,
                                  const int* two, int parity, ResPartial* part,
                                  ResPartial* out, int nactive, int nblocks, cudaStream_t s);

// f = f^eq(rho, u) (device inputs, nullable), written in pull-scheme form.
template <typename T>
cudaError_t launch_init(T* f, const AuxParams& p, const double* rho, const double* ux,
                        const double* uy, cudaStream_t s);
// state from post-stream distributions (device, 9 planes of nx*ny doubles)
template <typename T>
cudaError_t launch_set_f(T* f, const AuxParams& p, const double* fin, cudaStream_t s);
// post-stream distributions / moments of the state (device outputs)
template <typename T>
cudaError_t launch_get_f(const T* f, const AuxParams& p, double* fout, cudaStream_t s);
// exact64: rho and u in FP64 arithmetic (diagnostics, stress); otherwise FP32
// storage is read out in FP32 (rho = rho0 + d still in FP64).
template <typename T>
cudaError_t launch_moments(const T* f, const AuxParams& p, double* rho, double* ux,
                           double* uy, cudaStream_t s, bool exact64 = false);
// Local strain rates and viscous stress (FP64, nullable outputs of nx*ny
// doubles) of the state; rho: the density field of the same state (from
// launch_moments).
template <typename T>
cudaError_t launch_stress(const T* f, const AuxParams& p, const double* rho, double* dxux,
                          double* dyuy, double* sxy, double* txx, double* tyy, double* txy,
                          cudaStream_t s);
// diagnostics: per-block partials into `part` (nblocks entries) then a final
// reduction into part[nblocks]; fprev: the state one step earlier (nullable:
// the residual then uses u(n) alone); uprev (2*nx*ny doubles) is read (if
// have_prev) and overwritten with the two-step mean velocity.
template <typename T>
cudaError_t launch_diag(const T* f, const T* fprev, const AuxParams& p, double* uprev,
                        int have_prev, DiagPartial* part, int nblocks, cudaStream_t s);

}  // namespace lbm
