// lbib_noalloc.cu -- a lattice time stepper that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they want to
// step the fluid: code running under an external memory manager that owns
// every byte of the device (a pre-sized arena, a serving process with a fixed
// budget), or code on a path where a cudaMalloc would synchronise the device
// or fail.  lbib_lattice_advance_noalloc serves them: it advances a channel
// without membranes by running the library's bulk lattice kernel, with every
// buffer beyond the caller's populations (the two padded deviation buffers
// the kernel ping-pongs between, the per-tile flags and per-tile-column
// instance table it reads and the status word it sets) carved out of one
// file-scope device array of fixed size.
//
// The array exists once per device for the life of the process (every GPU
// that loads the library holds it until exit).  All calls on a device share
// it and it keeps the previous call's contents; each call clears the parts
// that must start at zero.  Calls whose GPU work overlaps (different host
// threads, or different streams) race on the array.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "lbib_internal.cuh"

using namespace lbib;

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

size_t up256(size_t n) { return (n + 255) & ~size_t(255); }

// Device address of g_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up,
// with the device current, on every call: the lookup allocates nothing, and a
// cached address would go stale if the caller reset the device (the module is
// then loaded again, possibly elsewhere).
cudaError_t scratch_address(void** out)
{
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

template <typename S>
__global__ void k_absolute_to_deviation(const double* __restrict__ f, S* __restrict__ g, Lattice L)
{
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    for (int q = 0; q < 9; ++q) {
        const double w = q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        g[q * L.qstride + y * L.nxp + x] = (S)(f[((size_t)q * L.ny + y) * L.nx + x] - w);
    }
}

template <typename S>
__global__ void k_deviation_to_absolute(const S* __restrict__ g, double* __restrict__ f, Lattice L)
{
    const int x = blockIdx.x * TX + threadIdx.x, y = blockIdx.y * TY + threadIdx.y;
    if (x >= L.nx || y >= L.ny) return;
    for (int q = 0; q < 9; ++q) {
        const double w = q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        f[((size_t)q * L.ny + y) * L.nx + x] = (double)g[q * L.qstride + y * L.nxp + x] + w;
    }
}

// one instance over every tile column: origin 0, width nx
__global__ void k_single_instance_columns(int4* ci, int ntx, int nx)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntx) ci[t] = make_int4(0, nx, 0, 0);
}

lbib_status fail_noalloc(lbib_status s, const std::string& msg)
{
    set_global_error(msg.c_str());
    return s;
}

}  // namespace

extern "C" lbib_status lbib_lattice_advance_noalloc(const lbib_fluid_params* P, double* f, int64_t nsteps)
{
    if (!P || !f) return fail_noalloc(LBIB_ERR_INVALID_ARG, "null argument");
    if (P->nx < 3 || P->ny < 2) return fail_noalloc(LBIB_ERR_INVALID_ARG, "need nx >= 3 and ny >= 2");
    if (!(P->tau > 0.5)) return fail_noalloc(LBIB_ERR_INVALID_ARG, "tau must exceed 1/2");
    if (!(P->re >= 0.0) || !(P->rho_out > 0.0)) return fail_noalloc(LBIB_ERR_INVALID_ARG, "re >= 0 and rho_out > 0");
    if (P->bc_mode != LBIB_BC_INLET_OUTLET && P->bc_mode != LBIB_BC_PERIODIC_FORCE)
        return fail_noalloc(LBIB_ERR_INVALID_ARG, "unknown bc_mode");
    if (P->storage != LBIB_STORE_FP64 && P->storage != LBIB_STORE_FP32)
        return fail_noalloc(LBIB_ERR_UNSUPPORTED, "only FP64 and FP32 storage");
    if (nsteps < 0) return fail_noalloc(LBIB_ERR_INVALID_ARG, "nsteps < 0");
    if (P->device < 0) return fail_noalloc(LBIB_ERR_INVALID_ARG, "device ordinal");

    Lattice L{};
    L.nx = P->nx;
    L.ny = P->ny;
    L.ntx = (P->nx + TX - 1) / TX;
    L.nty = (P->ny + TY - 1) / TY;
    L.nxp = L.ntx * TX;
    L.ntiles = L.ntx * L.nty;
    L.bc = P->bc_mode;
    L.qstride = L.nxp * L.ny;
    L.tau = P->tau;
    L.omega = 1.0 / P->tau;
    L.nu = (P->tau - 0.5) / 3.0;
    L.umax = P->re * L.nu / P->ny;
    L.rho_out = P->rho_out;
    L.gx = P->gx;
    L.gy = P->gy;
    set_float_params(L);
    const int prec = (P->storage == LBIB_STORE_FP64) ? PREC_F64 : PREC_F32;
    const size_t s = (prec == PREC_F64) ? 8 : 4;
    const size_t need_flags = up256((size_t)L.ntiles * 4);
    const size_t need_cols = up256((size_t)L.ntx * sizeof(int4));
    const size_t need_f = up256((size_t)9 * L.qstride * s);
    const size_t need = 256 + need_flags + need_cols + 2 * need_f;
    if ((double)L.nxp * L.ny * 9 >= 2147483648.0 || need > kScratchBytes)
        return fail_noalloc(LBIB_ERR_UNSUPPORTED,
                            "lattice needs " + std::to_string(need) + " bytes of scratch; the fixed array holds " +
                                std::to_string(kScratchBytes) + " (at most ~" +
                                std::to_string(kScratchBytes / (2 * 9 * s)) + " nodes in this precision)");

    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(P->device);
    lbib_status st = LBIB_OK;
    std::string msg;
    unsigned char* base = nullptr;
    cudaStream_t stream = static_cast<cudaStream_t>(P->cuda_stream);
    if (e == cudaSuccess) e = scratch_address(reinterpret_cast<void**>(&base));
    if (e == cudaSuccess) {
        Dev d{};
        d.L = L;
        d.store = (prec == PREC_F64) ? STORE_F64 : STORE_F32;
        d.status = reinterpret_cast<uint32_t*>(base);
#ifdef LBIB_CHECKED
        d.L.chk_status = d.status;
#endif
        d.nearflag[0] = d.nearflag[1] = d.nearflag[2] = reinterpret_cast<uint32_t*>(base + 256);
        int4* cols = reinterpret_cast<int4*>(base + 256 + need_flags);
        d.colinfo = cols;
        d.ninst = 1;
        d.f[0] = base + 256 + need_flags + need_cols;
        d.f[1] = base + 256 + need_flags + need_cols + need_f;
        const dim3 grid(L.ntx, L.nty), block(TX, TY);
        // status and tile flags must start at zero (the array keeps the last call's contents)
        e = cudaMemsetAsync(base, 0, 256 + need_flags, stream);
        if (e == cudaSuccess) {
            k_single_instance_columns<<<(L.ntx + 127) / 128, 128, 0, stream>>>(cols, L.ntx, L.nx);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            if (prec == PREC_F64)
                k_absolute_to_deviation<double><<<grid, block, 0, stream>>>(f, static_cast<double*>(d.f[0]), L);
            else
                k_absolute_to_deviation<float><<<grid, block, 0, stream>>>(f, static_cast<float*>(d.f[0]), L);
            e = cudaGetLastError();
        }
        for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k)
            e = launch_lbm_bulk(d, prec, (int)(k & 1), (int)(k % 3), stream);
        if (e == cudaSuccess) {
            const int last = (int)(nsteps & 1);
            if (prec == PREC_F64)
                k_deviation_to_absolute<double><<<grid, block, 0, stream>>>(static_cast<double*>(d.f[last]), f, L);
            else
                k_deviation_to_absolute<float><<<grid, block, 0, stream>>>(static_cast<float*>(d.f[last]), f, L);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        uint32_t status = 0;
        if (e == cudaSuccess) e = cudaMemcpy(&status, base, sizeof(status), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && (status & ST_DIVERGED)) {
            st = LBIB_ERR_DIVERGED;
            msg = "non-finite or non-positive state on the device";
        }
        if (e == cudaSuccess && (status & ST_BOUNDS)) {
            st = LBIB_ERR_STATE;
            msg = "an index left its array (bounds-checked build)";
        }
    }
    if (e != cudaSuccess) {
        st = LBIB_ERR_CUDA;
        msg = std::string("lbib_lattice_advance_noalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st != LBIB_OK) return fail_noalloc(st, msg);
    return LBIB_OK;
}
