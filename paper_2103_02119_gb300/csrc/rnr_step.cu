// rnr_step.cu -- kernels of the fused step with the raw-moment collision
// (RNR-LBM, Sec. 3).  The block's work is in step_block.cuh.
#include "step_block.cuh"

namespace lbm {

template <typename T>
cudaError_t launch_step_rnr(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                            cudaStream_t s) {
    return launch_step_scheme<T, 1>(fin, fout, p, bx, nbands, s);
}
template cudaError_t launch_step_rnr<float>(const float*, float*, const KParams<float>&, int,
                                            int, cudaStream_t);
template cudaError_t launch_step_rnr<double>(const double*, double*, const KParams<double>&,
                                             int, int, cudaStream_t);

}  // namespace lbm
