// rc_free_step.cu -- kernels of the fused RC-LBM step (Sec. 4) for lattices
// without a body force: the collision's force terms (Phi^c, the u.F parts of
// Eq. 34-35, the force shift of u) are compiled out.  The block's work is in
// step_block.cuh; a translation unit of its own so that the library's
// kernels compile in parallel.
#include "step_block.cuh"

namespace lbm {

template <typename T>
cudaError_t launch_step_free(const T* fin, T* fout, const KParams<T>& p, int bx, int nbands,
                             cudaStream_t s) {
    return launch_step_scheme<T, 3>(fin, fout, p, bx, nbands, s);
}
template cudaError_t launch_step_free<float>(const float*, float*, const KParams<float>&, int,
                                             int, cudaStream_t);
template cudaError_t launch_step_free<double>(const double*, double*, const KParams<double>&,
                                              int, int, cudaStream_t);

}  // namespace lbm
