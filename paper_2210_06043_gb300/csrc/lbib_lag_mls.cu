// lbib_lag_mls.cu -- instantiations of the Lagrangian kernel
// (lbib_lag_kernel.cuh) for the moving-least-squares transfer, in a
// translation unit of their own so that the two flavours compile in parallel.
#include "lbib_lag_kernel.cuh"

namespace lbib {

cudaError_t configure_kernels_mls(int prec, int bytes) { return configure_transfer<true>(prec, bytes); }

cudaError_t launch_lagrangian_mls(const Dev& d, int prec, int parity, size_t bytes, cudaStream_t s)
{
    return launch_transfer<true>(d, prec, parity, bytes, s);
}

}  // namespace lbib
