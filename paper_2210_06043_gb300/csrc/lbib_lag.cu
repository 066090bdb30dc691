// lbib_lag.cu -- host side of the Lagrangian update and the instantiations
// of its kernel (lbib_lag_kernel.cuh) for the Peskin transfer.
#include "lbib_lag_kernel.cuh"

namespace lbib {

size_t lagrangian_smem_bytes(int prec, int nv_max)
{
    size_t r = (prec == PREC_F64) ? sizeof(double) : sizeof(float);
    return (size_t)nv_max * 33 * r;
}

cudaError_t configure_kernels(int prec, int nv_max)
{
    const int bytes = (int)lagrangian_smem_bytes(prec, nv_max);
    cudaError_t e = configure_transfer<false>(prec, bytes);
    return (e == cudaSuccess) ? configure_kernels_mls(prec, bytes) : e;
}

cudaError_t launch_lagrangian(const Dev& d, int prec, int parity, cudaStream_t s)
{
    const size_t bytes = lagrangian_smem_bytes(prec, d.nv_max);
    if (d.L.transfer == LBIB_TRANSFER_MLS) return launch_lagrangian_mls(d, prec, parity, bytes, s);
    return launch_transfer<false>(d, prec, parity, bytes, s);
}

}  // namespace lbib
