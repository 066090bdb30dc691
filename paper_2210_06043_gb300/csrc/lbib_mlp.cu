// lbib_mlp.cu -- the learned surrogate (include/lbib_mlp.h): a multilayer
// perceptron with BF16 weights and activations, FP32 accumulation, trained
// with Adam, every step on the GPU in the kernels below.
//
// The dense products run on the tensor cores: one GEMM kernel computes
// C[M][N] = A[M][K] B[N][K]^T with A and B read either K-major or M/N-major
// from global memory (cp.async into padded shared tiles, ldmatrix / ldmatrix
// .trans into mma.sync m16n8k16 BF16 fragments, FP32 accumulators), with the
// layer's epilogue fused: bias + GELU (forward), bias (output layer), GELU'
// (backward), or an FP32 partial of a deterministic split-K (weight
// gradients).  Reductions (bias gradients, split-K sums, the loss) run in a
// fixed order, so a step is reproducible bit for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbib_internal.cuh"
#include "lbib_trace.h"
#include "../../include/lbib_mlp.h"

using namespace lbib;

namespace {

constexpr int BM = 64, BN = 64, BK = 32;  // block tile; 4 warps, each 32 x 32
constexpr int GEMM_THREADS = 128;
constexpr int PAD = 8;  // bf16 elements of row padding (ldmatrix rows stay 16-byte aligned, banks spread)
constexpr int MAX_SPLITS = 64;

enum Epi { EPI_FWD_GELU = 0, EPI_FWD_LIN = 1, EPI_BWD_GELU = 2, EPI_PARTIAL = 3 };

struct GemmArgs {
    const __nv_bfloat16* A;  // K-major: [M][lda]; M-major (TA): [K][lda]
    const __nv_bfloat16* B;  // K-major: [N][ldb]; N-major (TB): [K][ldb]
    int lda, ldb;
    int M, N, K;              // M rows valid (ragged), N multiple of BN, K valid (ragged allowed on trans operands)
    int k_tiles_per_split;
    const float* bias;        // [N] (forward epilogues)
    const float* Zin;         // [M][ldc] pre-activations (backward epilogue)
    float* Zout;              // [M][ldc] pre-activations (forward GELU) or output (forward linear)
    __nv_bfloat16* Aout;      // [M][ldc] bf16 activations (forward GELU) or gradients (backward)
    float* part;              // [splits][M][ldc] (split-K partials)
    int ldc;
    uint32_t* status;         // error word: bit 0 set when a bounded wait gave up
};

// The fused forward pass stores pre-activations tile by tile, so that each
// warp store is 512 contiguous bytes: for row m, column n of an N-column layer,
// 128-row tile m / 128, 16-column block n / 16, 4-column group (n / 4) % 4,
// then the tile's 128 rows of 4 values.
__host__ __device__ __forceinline__ size_t zt_index(int m, int n, int N)
{
    return ((((size_t)(m >> 7) * (N >> 4) + (n >> 4)) * 4 + ((n >> 2) & 3)) * 128 + (m & 127)) * 4 + (n & 3);
}
// The activations (and their gradients) likewise, in 16-byte groups of 8 BF16
// columns over 64-row blocks: block m / 64, 16-column block, 8-column group
// (n / 8) % 2, then the block's 64 rows of 8 values.  A 64-row block of every
// column is one contiguous range (N * 128 bytes).
__host__ __device__ __forceinline__ size_t at_index(int m, int n, int N)
{
    return ((((size_t)(m >> 6) * (N >> 4) + (n >> 4)) * 2 + ((n >> 3) & 1)) * 64 + (m & 63)) * 8 + (n & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid)
{
    const int n = valid ? 16 : 0;  // 0 source bytes: the 16 destination bytes are zero-filled
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// GELU in the tanh form of Hendrycks & Gimpel (Gaussian Error Linear Units,
// 2016): GELU(z) = z/2 (1 + tanh(u)), u = sqrt(2/pi) (z + 0.044715 z^3).  The
// tanh is the hardware approximation (tanh.approx.f32, relative error about
// 2^-11; its packed FP16 form gives no more results per clock); every other
// step is an explicitly rounded FP32 operation in a fixed order, so the packed
// two-lane form (gelu2_bf16, f32x2 arithmetic) returns the same bits as the
// scalar one.
constexpr float GELU_K0 = 0.7978845608028654f;     // sqrt(2/pi)
constexpr float GELU_K1 = 0.035677408136300125f;   // 0.044715 sqrt(2/pi)
constexpr float GELU_K1X3 = 0.10703222440890037f;  // 3 * 0.044715 sqrt(2/pi)

__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu(float z)
{
    const float u = __fmul_rn(z, __fmaf_rn(__fmul_rn(z, z), GELU_K1, GELU_K0));
    const float h = __fmul_rn(0.5f, z);
    return __fmaf_rn(h, tanh_hw(u), h);
}
// d GELU / dz = (1 + tanh u)/2 + z/2 (1 - tanh^2 u) sqrt(2/pi) (1 + 3 * 0.044715 z^2)
__device__ __forceinline__ float gelu_d(float z)
{
    const float zz = __fmul_rn(z, z);
    const float th = tanh_hw(__fmul_rn(z, __fmaf_rn(zz, GELU_K1, GELU_K0)));
    const float s = __fmaf_rn(-th, th, 1.0f);
    return __fmaf_rn(__fmul_rn(__fmul_rn(0.5f, z), s), __fmaf_rn(zz, GELU_K1X3, GELU_K0), __fmaf_rn(0.5f, th, 0.5f));
}

// Two-lane FP32 arithmetic (add/mul/fma .rn .f32x2): one instruction for two
// values, each lane rounded like the scalar operation.
__device__ __forceinline__ uint64_t f2(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(uint64_t v, float& a, float& b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// GELU(v0 + b0), GELU(v1 + b1) rounded to a BF16 pair: gelu() on two lanes;
// the pre-activations z = v + b in z0, z1.
__device__ __forceinline__ uint32_t gelu2_bf16(float v0, float v1, float b0, float b1, float& z0, float& z1)
{
    const uint64_t z = f2_add(f2(v0, v1), f2(b0, b1));
    f2_split(z, z0, z1);
    const uint64_t u = f2_mul(z, f2_fma(f2_mul(z, z), f2(GELU_K1, GELU_K1), f2(GELU_K0, GELU_K0)));
    const uint64_t h = f2_mul(f2(0.5f, 0.5f), z);
    float u0, u1, g0, g1;
    f2_split(u, u0, u1);
    f2_split(f2_fma(h, f2(tanh_hw(u0), tanh_hw(u1)), h), g0, g1);
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(g0, g1);
    return *reinterpret_cast<const uint32_t*>(&b2);
}

// Tensor memory -> registers: 32 lanes x 16 consecutive 32-bit columns
// (tcgen05.ld 32x32b.x16), and the wait for the loads issued so far.  The wait
// names the destination registers as operands, so no use of them can be
// scheduled above it.
__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr));
}
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15])
                 :
                 : "memory");
}

// Shared tiles: A as [BM][BK+PAD] (K-major) or [BK][BM+PAD] (M-major), B likewise.
template <bool TA, bool TB>
struct Tiles {
    __nv_bfloat16 a[2][TA ? BK : BM][(TA ? BM : BK) + PAD];
    __nv_bfloat16 b[2][TB ? BK : BN][(TB ? BN : BK) + PAD];
};

template <bool TA, bool TB>
__device__ __forceinline__ void load_tiles(Tiles<TA, TB>& s, int buf, const GemmArgs& g, int m0, int n0, int k0)
{
    const int tid = threadIdx.x;
    // 256 chunks of 8 bf16 per operand tile, two per thread
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int ch = tid + c * GEMM_THREADS;
        if (!TA) {  // rows m, 4 chunks of k
            const int r = ch >> 2, kc = (ch & 3) * 8;
            const int m = m0 + r;
            const bool v = m < g.M;
            cp_async16(&s.a[buf][r][kc], g.A + (size_t)(v ? m : 0) * g.lda + k0 + kc, v);
        } else {    // rows k, 8 chunks of m
            const int r = ch >> 3, mc = (ch & 7) * 8;
            const int k = k0 + r;
            const bool v = k < g.K;
            cp_async16(&s.a[buf][r][mc], g.A + (size_t)(v ? k : 0) * g.lda + m0 + mc, v);
        }
        if (!TB) {
            const int r = ch >> 2, kc = (ch & 3) * 8;
            cp_async16(&s.b[buf][r][kc], g.B + (size_t)(n0 + r) * g.ldb + k0 + kc, true);
        } else {
            const int r = ch >> 3, nc = (ch & 7) * 8;
            const int k = k0 + r;
            const bool v = k < g.K;
            cp_async16(&s.b[buf][r][nc], g.B + (size_t)(v ? k : 0) * g.ldb + n0 + nc, v);
        }
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm(GemmArgs g)
{
    __shared__ __align__(16) Tiles<TA, TB> s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kt_total = (g.K + BK - 1) / BK;
    const int kt0 = blockIdx.z * g.k_tiles_per_split;
    const int kt1 = min(kt_total, kt0 + g.k_tiles_per_split);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    if (kt0 < kt1) {
        load_tiles<TA, TB>(s, 0, g, m0, n0, kt0 * BK);
        cp_async_commit();
    }
    for (int kt = kt0; kt < kt1; ++kt) {
        const int buf = (kt - kt0) & 1;
        cp_async_wait_all();
        __syncthreads();
        if (kt + 1 < kt1) {  // prefetch the next tile into the other buffer
            load_tiles<TA, TB>(s, buf ^ 1, g, m0, n0, (kt + 1) * BK);
            cp_async_commit();
        }
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mb = wm + i * 16;
                if (!TA) ldsm_x4(af[i], &s.a[buf][mb + (lane & 7) + 8 * ((lane >> 3) & 1)][kk + 8 * (lane >> 4)]);
                else ldsm_x4_t(af[i], &s.a[buf][kk + (lane & 7) + 8 * (lane >> 4)][mb + 8 * ((lane >> 3) & 1)]);
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int nb = wn + p * 16;
                if (!TB) ldsm_x4(bf[p], &s.b[buf][nb + (lane & 7) + 8 * (lane >> 4)][kk + 8 * ((lane >> 3) & 1)]);
                else ldsm_x4_t(bf[p], &s.b[buf][kk + (lane & 7) + 8 * ((lane >> 3) & 1)][nb + 8 * (lane >> 4)]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j >> 1][2 * (j & 1)], bf[j >> 1][2 * (j & 1) + 1]);
        }
        __syncthreads();
    }
    // epilogue: c0, c1 at (row g, cols 2t, 2t + 1), c2, c3 at row g + 8
    const int gr = lane >> 2, tc = (lane & 3) * 2;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm + i * 16 + gr + 8 * h;
                const int n = n0 + wn + j * 8 + tc;
                if (m >= g.M) continue;
                const float v0 = acc[i][j][2 * h], v1 = acc[i][j][2 * h + 1];
                const size_t o = (size_t)m * g.ldc + n;
                if (EPI == EPI_FWD_GELU) {
                    const float z0 = v0 + g.bias[n], z1 = v1 + g.bias[n + 1];
                    g.Zout[o] = z0;
                    g.Zout[o + 1] = z1;
                    g.Aout[o] = __float2bfloat16_rn(gelu(z0));
                    g.Aout[o + 1] = __float2bfloat16_rn(gelu(z1));
                } else if (EPI == EPI_FWD_LIN) {
                    g.Zout[o] = v0 + g.bias[n];
                    g.Zout[o + 1] = v1 + g.bias[n + 1];
                } else if (EPI == EPI_BWD_GELU) {
                    g.Aout[o] = __float2bfloat16_rn(v0 * gelu_d(g.Zin[o]));
                    g.Aout[o + 1] = __float2bfloat16_rn(v1 * gelu_d(g.Zin[o + 1]));
                } else {
                    float* pp = g.part + (size_t)blockIdx.z * g.M * g.ldc;
                    pp[o] = v0;
                    pp[o + 1] = v1;
                }
            }
}

// ---------------------------------------------------------------- tcgen05 path
// C[M][N] = A[M][K] B[N][K]^T with both operands K-major: one CTA of 128
// threads per 128 x N tile (N <= 256, a multiple of 16), K in blocks of 64.
// Operand tiles are staged (cp.async) in the canonical no-swizzle K-major
// layout of 8 x 8 core matrices (element (r, k) at (r / 8) * 1024 + (k / 8) *
// 128 + (r % 8) * 16 + (k % 8) * 2 bytes: 128 B between core matrices along K,
// 1024 B between 8-row groups); one elected thread issues tcgen05.mma (M 128,
// N, K 16 per instruction, BF16 x BF16 -> FP32) into a tensor-memory
// accumulator of N columns and commits to an mbarrier; the epilogue reads the
// accumulator with tcgen05.ld (warp w owns rows 32 w .. 32 w + 31).
constexpr int TC_BM = 128, TC_BK = 64, TC_THREADS = 128;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 26;  // mbarrier polls before giving up

__host__ __device__ constexpr size_t tc_smem_bytes(int n) { return (size_t)(TC_BM + n) * TC_BK * 2 + 64; }
// shared memory requested per CTA: at most two CTAs per SM, so their tensor-memory
// allocations (<= 256 columns each) never exceed the SM's 512 columns
constexpr size_t TC_SMEM_REQUEST = 96 * 1024;

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;     // leading byte offset: next core matrix along K
    d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;    // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version (sm_100 family)
    // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
    return d;
}

__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    uint32_t d = 0;
    d |= 1u << 4;                     // D format FP32
    d |= 1u << 7;                     // A format BF16
    d |= 1u << 10;                    // B format BF16
    // A, B K-major (bits 15, 16 zero), no negation
    d |= (uint32_t)(n >> 3) << 17;    // N / 8
    d |= (uint32_t)(TC_BM >> 4) << 24; // M / 16
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase)
{
    for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sa = tc_smem;                                   // 128 x 64 bf16, 16 KB
    unsigned char* sb = tc_smem + TC_BM * TC_BK * 2;               // N x 64 bf16
    // barrier and tensor-memory address at the end of the region (the epilogue
    // reuses the front for staging)
    uint64_t* bar = reinterpret_cast<uint64_t*>(tc_smem + TC_SMEM_REQUEST - 64);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_BM, N = g.N;
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;  // power of two >= 32
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc_idesc(N);
    uint32_t phase = 0;
    bool ok = true;
    const int kblocks = g.K / TC_BK;
    for (int kb = 0; kb < kblocks && ok; ++kb) {
        const int k0 = kb * TC_BK;
        // stage A (128 rows) and B (N rows), 16-byte chunks, rows beyond M zero
        for (int c = tid; c < TC_BM * 8; c += TC_THREADS) {
            const int r = c >> 3, kc = c & 7;
            const int m = m0 + r;
            const bool v = m < g.M;
            cp_async16(sa + (r >> 3) * 1024 + kc * 128 + (r & 7) * 16, g.A + (size_t)(v ? m : 0) * g.lda + k0 + kc * 8,
                       v);
        }
        for (int c = tid; c < N * 8; c += TC_THREADS) {
            const int r = c >> 3, kc = c & 7;
            cp_async16(sb + (r >> 3) * 1024 + kc * 128 + (r & 7) * 16, g.B + (size_t)r * g.ldb + k0 + kc * 8, true);
        }
        cp_async_commit();
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {  // K 16 per instruction: two core matrices along K
                const uint64_t da = tc_desc(smem_u32(sa) + kk * 256);
                const uint64_t db = tc_desc(smem_u32(sb) + kk * 256);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(bar)));
        }
        ok = mbar_wait(bar, phase);  // the tiles are free again once the MMAs completed
        phase ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) atomicOr(g.status, 1u);
    } else {
        // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (its tile rows) in
        // blocks of 64 columns and stages them in shared memory (the operand
        // tiles are free once the last MMA completed), then writes whole row
        // segments: consecutive lanes, consecutive columns (coalesced)
        constexpr int SC = 64, ZP = SC + 1, AP = SC + 2;  // 12.5 KB per warp, 50 KB in all
        static_assert(4 * (32 * ZP + 16 * AP) * 4 <= TC_SMEM_REQUEST - 64, "staging below the barrier");
        float* zst = reinterpret_cast<float*>(tc_smem) + warp * (32 * ZP + 16 * AP);
        __nv_bfloat16* ast = reinterpret_cast<__nv_bfloat16*>(zst + 32 * ZP);
        for (int c0 = 0; c0 < N; c0 += SC) {
#pragma unroll
            for (int sub = 0; sub < SC / 16; ++sub) {
                uint32_t r[16];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + 16 * sub);
                tmem_ld16(ta, r);
                tmem_wait(r);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = 16 * sub + j;
                    const float z = __uint_as_float(r[j]) + g.bias[c0 + col];
                    zst[lane * ZP + col] = z;
                    if (EPI == EPI_FWD_GELU) ast[lane * AP + col] = __float2bfloat16_rn(gelu(z));
                }
            }
            __syncwarp();
            for (int rr = 0; rr < 32; ++rr) {
                const int m = m0 + warp * 32 + rr;
                if (m >= g.M) break;
                const size_t o = (size_t)m * g.ldc + c0;
                if (g.Zout) {
                    g.Zout[o + lane] = zst[rr * ZP + lane];
                    g.Zout[o + 32 + lane] = zst[rr * ZP + 32 + lane];
                }
                if (EPI == EPI_FWD_GELU) {
                    const __nv_bfloat162 v = __halves2bfloat162(ast[rr * AP + 2 * lane], ast[rr * AP + 2 * lane + 1]);
                    reinterpret_cast<__nv_bfloat162*>(g.Aout + o)[lane] = v;
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ------------------------------------------- fused inference (all layers)
// One persistent CTA per SM evaluates the whole network on 128-row tiles,
// two tiles in flight (slots 0 and 1).  A tile's activations stay in shared
// memory between layers, as the next layer's A operand (K-major core-matrix
// layout in 64-wide K chunks: element (r, k) at (k / 64) * 16384 + (r / 8) *
// 1024 + (k % 64 / 8) * 128 + (r % 8) * 16 + (k % 8) * 2 bytes); its
// accumulator lives in tensor-memory columns [256 s, 256 s + 256).  Roles:
//   warp 0, lane 0: issues the MMAs of each layer, slot by slot, and commits
//     them to the stage's "empty" barrier and then to the slot's "accumulator
//     full" barrier;
//   warp 1, lane 0: streams the pre-packed weight chunks (a layer's N x 64
//     K slice in the same core-matrix layout, contiguous in global memory)
//     through FZ_STAGES shared-memory stages with cp.async.bulk, each chunk
//     completing a "full" barrier by its byte count;
//   warps 4 .. 19: the epilogue.  Warp w reads tensor-memory lanes
//     32 (w % 4) .. + 31 (its tile rows) over a quarter of the columns, adds
//     the bias, applies GELU (f32x2 arithmetic, hardware tanh) and writes the
//     BF16 operand of the next layer in place, or writes the output rows;
//     they also load the inputs of the next tile of the slot.  Each step ends
//     with an arrival on the slot's "epilogue done" barrier, which the MMA
//     issuer waits for.  Four epilogue warps per SM sub-partition keep the
//     tanh unit (16 results per clock per SM, the epilogue's floor: 2048
//     cycles per 128 x 256 layer, as long as the layer's MMAs) busy.
// While the MMAs of one slot's layer run, the epilogue of the other slot's
// previous layer runs.  Both then share the SM's shared-memory bandwidth with
// the weight stream: per 128 x 256 x 256 layer the MMAs read 192 KB of
// operands, the stream writes 128 KB of weights and the epilogue 64 KB of
// activations, about 3000 cycles at 128 B per clock against 2048 for the
// MMAs alone.  Every wait is bounded: on timeout the CTA sets the status
// word, the other roles leave their loops, the copies and MMAs still in
// flight are waited for (bounded) and the tensor memory is freed.
constexpr int FZ_STAGES = 3, FZ_MAXW = 256, FZ_MAXL = 9, FZ_EW = 16, FZ_THREADS = 128 + 32 * FZ_EW;
constexpr size_t FZ_ACT = (size_t)TC_BM * FZ_MAXW * 2;        // 64 KB per slot
constexpr size_t FZ_STAGE = (size_t)FZ_MAXW * TC_BK * 2;      // 32 KB per weight chunk
constexpr size_t FZ_BAR = 2 * FZ_ACT + FZ_STAGES * FZ_STAGE;  // barriers after the buffers
constexpr size_t FZ_SMEM = FZ_BAR + 256;
static_assert(FZ_SMEM <= 227 * 1024, "fused kernel shared memory");

// Epilogue of one hidden layer for 16 accumulator columns cb .. cb + 15 of
// one tile row: bias, GELU, BF16, written as the next layer's A operand
// (K-major core matrices: 64-column chunks of 16 KB, 8-row groups of 1 KB,
// 8-column blocks of 128 B, one 16-byte row per block).  For a training
// forward pass (zg, ag non-null: the entries of this row and column cb in the
// tiled layouts of zt_index and at_index) the pre-activations (FP32) and
// activations (BF16) also go to global memory, each warp store 512 contiguous
// bytes.
__device__ __forceinline__ void fz_gelu16(const uint32_t (&v)[16], const float4 (&b)[4], int cb, unsigned char* arow,
                                          float* zg, __nv_bfloat16* ag)
{
    uint32_t pk[8];
    float z[16];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        pk[2 * i] = gelu2_bf16(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]), b[i].x, b[i].y, z[4 * i],
                               z[4 * i + 1]);
        pk[2 * i + 1] = gelu2_bf16(__uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3]), b[i].z, b[i].w,
                                   z[4 * i + 2], z[4 * i + 3]);
    }
    unsigned char* dst = arow + (cb >> 6) * 16384 + ((cb & 63) >> 3) * 128;
    *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    *reinterpret_cast<uint4*>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    if (zg) {
        // zg: the row's entry of column cb's 16-column block, tiled (zt_index): the
        // four 4-column groups are 128 rows of 16 bytes apart
        float4* zd = reinterpret_cast<float4*>(zg);
#pragma unroll
        for (int i = 0; i < 4; ++i) zd[i * 128] = make_float4(z[4 * i], z[4 * i + 1], z[4 * i + 2], z[4 * i + 3]);
    }
    if (ag) {
        // ag: the row's entry of column cb, tiled (at_index): the second 8-column group
        // is 64 rows of 16 bytes further; zero for a row past the batch (zg null)
        uint4* ad = reinterpret_cast<uint4*>(ag);
        ad[0] = zg ? make_uint4(pk[0], pk[1], pk[2], pk[3]) : make_uint4(0u, 0u, 0u, 0u);
        ad[64] = zg ? make_uint4(pk[4], pk[5], pk[6], pk[7]) : make_uint4(0u, 0u, 0u, 0u);
    }
}
__device__ __forceinline__ void ld_bias16(float4 (&b)[4], const float4* p)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = __ldg(p + i);
}

struct FusedArgs {
    const float* x;
    float* y;
    int M, n_in, n_out, L;
    const unsigned char* w;    // packed weight chunks
    const float* bias;         // FP32 parameters (biases at boff)
    int K[FZ_MAXL], N[FZ_MAXL], boff[FZ_MAXL];
    long long woff[FZ_MAXL];   // byte offset of layer l's first chunk in w
    const float *cin, *sin, *cout, *sout;
    uint32_t* status;
    // a training forward pass (k_mlp_fused<FZ_TRAIN>): layer l's pre-activations and
    // activations to zout[l], aout[l] (tiled: zt_index, at_index); the output
    // layer's raw values y_raw = W a + b go only into the loss gradient and the
    // squared errors below (nothing is written to y).  The backward chain (k_mlp_fused<FZ_BWD>): step s reads the
    // pre-activations zout[s] of its output width N[s] and writes the gradient
    // aout[s] = bf16(acc * GELU'(z)) (tiled), starting from dy ([M][K[0]] BF16).
    float* zout[FZ_MAXL];
    __nv_bfloat16* aout[FZ_MAXL];
    const __nv_bfloat16* dy;
    // training forward pass: the inputs a0 (tiled, 64 columns), and from the output
    // layer the loss gradient dY = bf16(2 d / (M n_out)), d = y_raw - (t - c_out) /
    // s_out (tiled, 64 columns), and per tile the sum of d^2 (loss_rows[tile], in a
    // fixed order)
    __nv_bfloat16 *a0_out, *dy_out;
    const float* t;
    float* loss_rows;
};

__device__ __forceinline__ bool fz_wait(uint64_t* bar, uint32_t parity, volatile uint32_t* abort_flag,
                                        uint32_t* status, bool honour_abort = true)
{
    for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (honour_abort && (it & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1u;
    atomicOr(status, 1u);
    return false;
}

__device__ __forceinline__ void fz_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// inputs of a tile into the slot's first K chunk: a0 = bf16(s_in (x - c_in)),
// zero beyond n_in and beyond the last row; 32 FZ_EW epilogue threads, warp w
// taking rows 8 w .. 8 w + 7 (lane % 8) and a quarter of the 64 columns
// (lane / 8) each, so the eight lanes of a 16-byte store phase fill one
// 128-byte row of core matrices (no bank conflicts)
// what an instantiation of k_mlp_fused computes (compile-time, so that the
// inference kernel carries none of the training code)
enum FzMode { FZ_INFER = 0, FZ_TRAIN = 1, FZ_BWD = 2 };

template <int MODE>
__device__ __forceinline__ void fz_prep(const FusedArgs& a, int tile, unsigned char* act, int e)
{
    static_assert(FZ_EW * 8 == TC_BM, "one warp per 8 rows");
    constexpr int COLS = 16;
    const int r = (e >> 5) * 8 + (e & 7), part = (e >> 3) & 3, row = tile * TC_BM + r;
    if (MODE == FZ_BWD) {
        // the output gradient rows (BF16, K[0] = 64 columns, tiled: at_index)
#pragma unroll
        for (int g8 = 0; g8 < COLS / 8; ++g8) {
            const int c0 = part * COLS + g8 * 8;
            const uint4 v = (row < a.M) ? __ldg(reinterpret_cast<const uint4*>(a.dy + at_index(row, c0, a.K[0])))
                                        : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(act + (r >> 3) * 1024 + (c0 >> 3) * 128 + (r & 7) * 16) = v;
        }
    } else {
#pragma unroll
        for (int g8 = 0; g8 < COLS / 8; ++g8) {
            const int c0 = part * COLS + g8 * 8;
            uint32_t pk[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = c0 + 2 * i + h;
                    v[h] = (row < a.M && j < a.n_in) ? a.sin[j] * (a.x[(size_t)row * a.n_in + j] - a.cin[j]) : 0.f;
                }
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
                pk[i] = *reinterpret_cast<const uint32_t*>(&b2);
            }
            *reinterpret_cast<uint4*>(act + (r >> 3) * 1024 + (c0 >> 3) * 128 + (r & 7) * 16) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
            if (MODE == FZ_TRAIN)  // the backward pass's copy (zeros past the batch)
                *reinterpret_cast<uint4*>(a.a0_out + at_index(row, c0, 64)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

// Epilogue of a backward step for one tile row (its columns of group cg):
// the accumulator (gradient before the activation) times GELU'(z), z the
// forward pass's pre-activations, rounded to BF16; written as the next step's
// A operand (except after the last step) and to the step's gradient output.
__device__ __forceinline__ void fz_bwd_step(const FusedArgs& a, int l, int tile, uint32_t trow, unsigned char* arow,
                                            int r, int cg)
{
    constexpr int NCG = FZ_EW / 4;
    const int N = a.N[l], cbeg = cg * (N / NCG), cend = cbeg + N / NCG;
    const bool last = (l + 1 == a.L);
    const int grow = tile * TC_BM + r;
    const bool st = grow < a.M;
    for (int cb = cbeg; cb < cend; cb += 16) {
        uint32_t v[16];
        tmem_ld16(trow + (uint32_t)cb, v);
        float4 z[4];
        const float4* zp = reinterpret_cast<const float4*>(a.zout[l] + zt_index(st ? grow : 0, cb, N));
#pragma unroll
        for (int i = 0; i < 4; ++i) z[i] = st ? __ldg(zp + i * 128) : make_float4(0.f, 0.f, 0.f, 0.f);
        tmem_wait(v);
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const __nv_bfloat162 p0 = __floats2bfloat162_rn(__uint_as_float(v[4 * i]) * gelu_d(z[i].x),
                                                            __uint_as_float(v[4 * i + 1]) * gelu_d(z[i].y));
            const __nv_bfloat162 p1 = __floats2bfloat162_rn(__uint_as_float(v[4 * i + 2]) * gelu_d(z[i].z),
                                                            __uint_as_float(v[4 * i + 3]) * gelu_d(z[i].w));
            pk[2 * i] = *reinterpret_cast<const uint32_t*>(&p0);
            pk[2 * i + 1] = *reinterpret_cast<const uint32_t*>(&p1);
        }
        if (!last) {
            unsigned char* dst = arow + (cb >> 6) * 16384 + ((cb & 63) >> 3) * 128;
            *reinterpret_cast<uint4*>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(dst + 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        }
        // (a row past the batch is written as zeros: the tiles are read whole)
        uint4* ad = reinterpret_cast<uint4*>(a.aout[l] + at_index(grow, cb, N));
        ad[0] = st ? make_uint4(pk[0], pk[1], pk[2], pk[3]) : make_uint4(0u, 0u, 0u, 0u);
        ad[64] = st ? make_uint4(pk[4], pk[5], pk[6], pk[7]) : make_uint4(0u, 0u, 0u, 0u);
    }
}

template <int MODE>
__global__ void __launch_bounds__(FZ_THREADS, 1) k_mlp_fused(FusedArgs a)
{
    extern __shared__ __align__(1024) unsigned char fz[];
    unsigned char* act[2] = {fz, fz + FZ_ACT};
    unsigned char* stages = fz + 2 * FZ_ACT;
    uint64_t* bar = reinterpret_cast<uint64_t*>(fz + FZ_BAR);
    uint64_t* full = bar;                    // [FZ_STAGES]
    uint64_t* empty = bar + FZ_STAGES;       // [FZ_STAGES]
    uint64_t* accf = bar + 2 * FZ_STAGES;    // [2]
    uint64_t* epid = accf + 2;               // [2]
    uint64_t* fin = epid + 2;                // MMAs drained on an abort
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(fin + 1);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1) + 1;
    uint64_t* lossb = fin + 2;                                 // [2] a tile's warp loss sums written
    float* lsum = reinterpret_cast<float*>(lossb + 2);          // [2][FZ_EW]
    static_assert(8 * 13 + 4 * 2 * FZ_EW <= 256, "barrier block");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (a.M + TC_BM - 1) / TC_BM;
    // this CTA's tiles: blockIdx.x + k gridDim.x, k < nk; tile k uses slot k & 1
    const int nk = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto tile_of = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
    if (tid == 0) {
        for (int i = 0; i < FZ_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
        }
        for (int sl = 0; sl < 2; ++sl) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&accf[sl])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&epid[sl])), "r"(32 * FZ_EW));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(fin)), "r"(1));
        for (int sl = 0; sl < 2; ++sl)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&lossb[sl])), "r"(FZ_EW));
        *abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        // ---------------------------------------------------- MMA issuer
        uint32_t q = 0, epar[2] = {0u, 0u};
        bool ok = true;
        for (int k0 = 0; k0 < nk && ok; k0 += 2)
            for (int l = 0; l < a.L && ok; ++l)
                for (int sl = 0; sl < 2 && ok; ++sl) {
                    if (k0 + sl >= nk) break;
                    ok = fz_wait(&epid[sl], epar[sl], abort_flag, a.status);
                    epar[sl] ^= 1u;
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t idesc = tc_idesc(a.N[l]);
                    const uint32_t dcol = tmem + (uint32_t)(sl * 256);
                    const int nch = a.K[l] / TC_BK;
                    for (int c = 0; c < nch && ok; ++c, ++q) {
                        const int st = (int)(q % FZ_STAGES);
                        ok = fz_wait(&full[st], (q / FZ_STAGES) & 1u, abort_flag, a.status);
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk) {
                            const uint64_t da = tc_desc(smem_u32(act[sl]) + c * 16384 + kk * 256);
                            const uint64_t db = tc_desc(smem_u32(stages + st * FZ_STAGE) + kk * 256);
                            const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
                            asm volatile(
                                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                                "l"(da), "l"(db), "r"(idesc), "r"(acc));
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                smem_u32(&empty[st])));
                    }
                    if (ok)
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                smem_u32(&accf[sl])));
                }
        if (!ok) {
            // let every MMA already issued finish before the memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(fin)));
            fz_wait(fin, 0u, abort_flag, a.status, false);
        }
    } else if (tid == 32) {
        // ---------------------------------------------------- weight producer
        uint32_t qi = 0;
        bool ok = true;
        for (int k0 = 0; k0 < nk && ok; k0 += 2)
            for (int l = 0; l < a.L && ok; ++l)
                for (int sl = 0; sl < 2 && ok; ++sl) {
                    if (k0 + sl >= nk) break;
                    const uint32_t bytes = (uint32_t)a.N[l] * TC_BK * 2;
                    const int nch = a.K[l] / TC_BK;
                    for (int c = 0; c < nch && ok; ++c, ++qi) {
                        const int st = (int)(qi % FZ_STAGES);
                        ok = fz_wait(&empty[st], ((qi / FZ_STAGES) & 1u) ^ 1u, abort_flag, a.status);
                        if (!ok) break;
                        const unsigned char* src = a.w + a.woff[l] + (long long)c * bytes;
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                         smem_u32(&full[st])),
                                     "r"(bytes)
                                     : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                smem_u32(stages + st * FZ_STAGE)),
                            "l"(src), "r"(bytes), "r"(smem_u32(&full[st]))
                            : "memory");
                    }
                }
        if (!ok) {
            // copies still in flight land before the CTA leaves
            for (uint32_t qq = (qi > FZ_STAGES ? qi - FZ_STAGES : 0u); qq < qi; ++qq)
                fz_wait(&full[qq % FZ_STAGES], (qq / FZ_STAGES) & 1u, abort_flag, a.status, false);
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------- epilogue
        constexpr int NCG = FZ_EW / 4;  // column groups per tile row
        const int e = tid - 128, q4 = warp & 3, cg = (warp - 4) >> 2, r = q4 * 32 + lane;
        for (int sl = 0; sl < 2 && sl < nk; ++sl) {
            fz_prep<MODE>(a, tile_of(sl), act[sl], e);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fz_arrive(&epid[sl]);
        }
        uint32_t apar[2] = {0u, 0u}, lpar[2] = {0u, 0u};
        bool ok = true;
        for (int k0 = 0; k0 < nk && ok; k0 += 2)
            for (int l = 0; l < a.L && ok; ++l)
                for (int sl = 0; sl < 2 && ok; ++sl) {
                    const int k = k0 + sl;
                    if (k >= nk) break;
                    ok = fz_wait(&accf[sl], apar[sl], abort_flag, a.status);
                    apar[sl] ^= 1u;
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int tile = tile_of(k);
                    const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(sl * 256);
                    if (MODE == FZ_BWD) {
                        fz_bwd_step(a, l, tile, trow, act[sl] + (r >> 3) * 1024 + (r & 7) * 16, r, cg);
                        // the slot's next tile once its last step is done (that step wrote
                        // nothing to the slot's shared memory)
                        if (l + 1 == a.L && k + 2 < nk) fz_prep<MODE>(a, tile_of(k + 2), act[sl], e);
                    } else if (l + 1 < a.L) {
                        // N is a multiple of 64: each column group is whole 16-column blocks
                        const int N = a.N[l], cbeg = cg * (N / NCG), cend = cbeg + N / NCG;
                        const float4* bias4 = reinterpret_cast<const float4*>(a.bias + a.boff[l]);
                        unsigned char* arow = act[sl] + (r >> 3) * 1024 + (r & 7) * 16;
                        const int grow = tile * TC_BM + r;
                        const bool st = MODE == FZ_TRAIN && grow < a.M;
                        for (int cb = cbeg; cb < cend; cb += 16) {
                            uint32_t v[16];
                            float4 b[4];
                            tmem_ld16(trow + (uint32_t)cb, v);
                            ld_bias16(b, bias4 + (cb >> 2));
                            tmem_wait(v);
                            fz_gelu16(v, b, cb, arow, st ? a.zout[l] + zt_index(grow, cb, N) : nullptr,
                                      MODE == FZ_TRAIN ? a.aout[l] + at_index(grow, cb, N) : nullptr);
                        }
                    } else if (MODE == FZ_TRAIN) {
                        // the loss gradient and squared errors of the row over its 16 of the
                        // 64 (padded) output columns, straight from the accumulator
                        static_assert(64 / NCG == 16, "one 16-column block per group");
                        const float* bias = a.bias + a.boff[l];
                        const int row = tile * TC_BM + r, cb = cg * 16;
                        uint32_t v[16];
                        tmem_ld16(trow + (uint32_t)cb, v);
                        tmem_wait(v);
                        float d2 = 0.f;
                        uint32_t pk[8];
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            float gv[2] = {0.f, 0.f};
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int col = cb + j + h;
                                if (row < a.M && col < a.n_out) {
                                    const float ts = (a.t[(size_t)row * a.n_out + col] - a.cout[col]) / a.sout[col];
                                    const float d = (__uint_as_float(v[j + h]) + bias[col]) - ts;
                                    d2 += d * d;
                                    gv[h] = 2.0f * d / ((float)a.M * (float)a.n_out);
                                }
                            }
                            const __nv_bfloat162 b2 = __floats2bfloat162_rn(gv[0], gv[1]);
                            pk[j / 2] = *reinterpret_cast<const uint32_t*>(&b2);
                        }
                        uint4* ad = reinterpret_cast<uint4*>(a.dy_out + at_index(row, cb, 64));
                        ad[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        ad[64] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                        // the tile's sum of d^2: a shuffle tree per warp, the warps' sums in
                        // shared memory (one array and barrier per slot), added in warp order by
                        // the first epilogue warp after a bounded wait
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
                        if (lane == 0) {
                            lsum[sl * FZ_EW + (warp - 4)] = d2;
                            fz_arrive(&lossb[sl]);
                        }
                        if (warp == 4) {
                            const bool lok = fz_wait(&lossb[sl], lpar[sl], abort_flag, a.status);
                            lpar[sl] ^= 1u;
                            if (lok && lane == 0) {
                                float ssum = 0.f;
                                for (int i = 0; i < FZ_EW; ++i) ssum += lsum[sl * FZ_EW + i];
                                a.loss_rows[tile] = ssum;
                            }
                        }
                        if (k + 2 < nk) fz_prep<MODE>(a, tile_of(k + 2), act[sl], e);
                    } else {
                        const float* bias = a.bias + a.boff[l];
                        const int row = tile * TC_BM + r;
                        for (int cb = cg * (64 / NCG); cb < (cg + 1) * (64 / NCG); cb += 16) {
                            if (cb >= a.n_out) break;  // uniform across the warp
                            uint32_t v[16];
                            tmem_ld16(trow + (uint32_t)cb, v);
                            tmem_wait(v);
                            if (row < a.M) {
#pragma unroll
                                for (int j = 0; j < 16; ++j) {
                                    const int col = cb + j;
                                    if (col < a.n_out)
                                        a.y[(size_t)row * a.n_out + col] =
                                            a.sout[col] * (__uint_as_float(v[j]) + bias[col]) + a.cout[col];
                                }
                            }
                        }
                        // the slot's next tile: the MMAs of this one have all completed
                        if (k + 2 < nk) fz_prep<MODE>(a, tile_of(k + 2), act[sl], e);
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    fz_arrive(&epid[sl]);
                }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ------------------------------------------- weight gradients on tcgen05
// dW_l = dZ_l^T A_l over a slice of the batch for every layer l in one launch:
// M = out (64 or 256), N = in (64 or 256), K = batch rows.  Both operands come
// from the tiled layout (at_index), which holds, per 64-row block and 8-column
// group, 64 rows of 16 bytes, a block of all columns contiguous: copied whole
// into shared memory (one bulk copy per operand and K block) it is the MN-major
// no-swizzle core-matrix layout (core matrix = 8 K-rows x 8 M/N elements;
// K-neighbours LBO = 128 B apart, M/N-neighbours SBO = 1024 B apart; measured on
// GB300 against exact small-integer products).  A CTA owns one 128 x 64 output
// tile (64 x 64 where M is 64) of one layer and one slice of the batch: it
// streams the slice in 64-row K blocks through DW_STAGES stages, accumulates in
// 64 tensor-memory columns (M 128, N 64, K 16 per instruction), and writes its
// FP32 partial (in the order k_reduce_dw reads) for a fixed-order reduction.
// Rows past the batch in the last block are zero in both layouts.
// Roles: warp 0 lane 0 issues the MMAs, warp 1 streams the operands, warps 2
// and 3 sum the dZ blocks of the layer's first column tile (the bias gradient),
// warps 4 .. 7 write the partial (warp w: the lanes of quadrant w % 4).
constexpr int DW_STAGES = 4, DW_THREADS = 256, DW_KB = 64, DW_TN = 64;
constexpr size_t DW_OPA = (size_t)TC_BM * DW_KB * 2;        // 16 KB of A (128 rows of M) per stage
constexpr size_t DW_OPB = (size_t)DW_TN * DW_KB * 2;        // 8 KB of B (64 columns of N) per stage
constexpr size_t DW_ST = DW_OPA + DW_OPB;
constexpr size_t DW_BAR = (size_t)DW_STAGES * DW_ST;        // barriers after the stages
constexpr size_t DW_SMEM = DW_BAR + 128;
static_assert(2 * (DW_SMEM + 1024) <= 228 * 1024, "two weight-gradient CTAs per SM");

// one layer's share of the launch: its CTAs are cta0 .. cta0 + tiles * splits - 1,
// CTA cta0 + s * tiles + t taking output tile t (row tile t / (N / 64), column
// tile t % (N / 64)) over batch slice s
struct DwLayer {
    const __nv_bfloat16* dz;   // tiled, width M
    const __nv_bfloat16* act;  // tiled, width N
    long long part_off;        // [split][M x N] partials at part + part_off
    int M, N, tiles, cta0, bpart_off;  // bias partials [split][M] at bias_part + bpart_off
};
struct DwArgs {
    DwLayer ly[FZ_MAXL];
    int nl, batch, rows_per_split;
    float* part;
    float* bias_part;
    uint32_t* status;
};

__device__ __forceinline__ uint32_t dw_idesc(int n)
{
    uint32_t d = 0;
    d |= 1u << 4;                      // D format FP32
    d |= 1u << 7;                      // A format BF16
    d |= 1u << 10;                     // B format BF16
    d |= 1u << 15;                     // A MN-major
    d |= 1u << 16;                     // B MN-major
    d |= (uint32_t)(n >> 3) << 17;     // N / 8
    d |= (uint32_t)(TC_BM >> 4) << 24; // M / 16
    return d;
}
__device__ __forceinline__ uint64_t dw_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);        // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;   // leading byte offset: next core matrix along K
    d |= (uint64_t)((1024u >> 4) & 0x3FFF) << 32;  // stride byte offset: next 8 elements along M / N
    d |= (uint64_t)1 << 46;                        // descriptor version (sm_100 family)
    return d;                                      // no swizzle
}

// one CTA per (layer, output tile, batch slice); see DwLayer
__global__ void __launch_bounds__(DW_THREADS, 2) k_dw_tc(DwArgs a)
{
    extern __shared__ __align__(1024) unsigned char dws[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(dws + DW_BAR);
    uint64_t* full = bar;                  // [DW_STAGES]
    uint64_t* empty = bar + DW_STAGES;     // [DW_STAGES]
    uint64_t* accf = bar + 2 * DW_STAGES;  // the last MMA done
    uint64_t* fin = accf + 1;              // MMAs drained on an abort
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(fin + 1);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1) + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this CTA's layer (constant indices only: the table stays in parameter space)
    const __nv_bfloat16 *dz = nullptr, *act = nullptr;
    long long part_off = 0;
    int M = 0, N = 0, tiles = 1, cta0 = 0, bpart_off = 0;
#pragma unroll
    for (int i = 0; i < FZ_MAXL; ++i)
        if (i < a.nl && (int)blockIdx.x >= a.ly[i].cta0) {
            dz = a.ly[i].dz;
            act = a.ly[i].act;
            part_off = a.ly[i].part_off;
            M = a.ly[i].M;
            N = a.ly[i].N;
            tiles = a.ly[i].tiles;
            cta0 = a.ly[i].cta0;
            bpart_off = a.ly[i].bpart_off;
        }
    const int idx = (int)blockIdx.x - cta0, tile = idx % tiles, split = idx / tiles;
    const int tn = N / DW_TN, mt = tile / tn, nt = tile % tn;
    const int mcols = min(TC_BM, M - mt * TC_BM);  // columns of M in this tile (64 or 128)
    const int b0 = split * a.rows_per_split, b1 = min(a.batch, b0 + a.rows_per_split);
    const int nkb = (b1 > b0) ? (b1 - b0 + DW_KB - 1) / DW_KB : 0;
    // the CTAs of the first column tile also sum dz over their rows (warps 2, 3):
    // a stage is then free once the MMAs and those 64 threads are done with it
    const bool bsum = nt == 0 && a.bias_part != nullptr;
    if (tid == 0) {
        for (int i = 0; i < DW_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(bsum ? 65 : 1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(accf)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(fin)), "r"(1));
        *abort_flag = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(DW_TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (tid == 0) {
        // ---------------------------------------------------- MMA issuer
        const uint32_t idesc = dw_idesc(DW_TN);
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int st = kb % DW_STAGES;
            ok = fz_wait(&full[st], (uint32_t)(kb / DW_STAGES) & 1u, abort_flag, a.status);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = smem_u32(dws + (size_t)st * DW_ST), sB = sA + (uint32_t)DW_OPA;
#pragma unroll
            for (int kk = 0; kk < DW_KB / 16; ++kk) {
                const uint64_t da = dw_desc(sA + (uint32_t)(kk * 256));
                const uint64_t db = dw_desc(sB + (uint32_t)(kk * 256));
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[st])));
        }
        if (ok)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(accf)));
        else {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(fin)));
            fz_wait(fin, 0u, abort_flag, a.status, false);
        }
    } else if (tid == 32) {
        // ---------------------------------------------------- operand stream
        // a 64-row block of the tile's columns is one contiguous range of either
        // operand (at_index): 128 (or 64) columns of M, 64 of N
        const uint32_t ba = (uint32_t)mcols * DW_KB * 2, bb = (uint32_t)DW_OPB;
        bool ok = true;
        int issued = 0;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int st = kb % DW_STAGES;
            ok = fz_wait(&empty[st], ((uint32_t)(kb / DW_STAGES) & 1u) ^ 1u, abort_flag, a.status);
            if (!ok) break;
            const int kr = b0 + kb * DW_KB;  // first row of the block, a multiple of 64
            const uint32_t sA = smem_u32(dws + (size_t)st * DW_ST), sB = sA + (uint32_t)DW_OPA;
            const uint32_t fb = smem_u32(&full[st]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(ba + bb) : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sA),
                "l"(dz + at_index(kr, mt * TC_BM, M)), "r"(ba), "r"(fb)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sB),
                "l"(act + at_index(kr, nt * DW_TN, N)), "r"(bb), "r"(fb)
                : "memory");
            issued = kb + 1;
        }
        if (!ok) {
            // copies still in flight land before the CTA leaves
            for (int qq = (issued > DW_STAGES ? issued - DW_STAGES : 0); qq < issued; ++qq)
                fz_wait(&full[qq % DW_STAGES], (uint32_t)(qq / DW_STAGES) & 1u, abort_flag, a.status, false);
        }
    } else if (warp == 2 || warp == 3) {
        // ---------------------------------------------------- bias-gradient partial
        // thread t sums columns 2t, 2t + 1 of the tile's dz block, rows in an order
        // rotated by the column group (conflict-free shared-memory reads)
        if (bsum) {
            const int t = tid - 64, c = 2 * t, g = c >> 3;
            float s0 = 0.f, s1 = 0.f;
            for (int kb = 0; kb < nkb; ++kb) {
                const int st = kb % DW_STAGES;
                if (!fz_wait(&full[st], (uint32_t)(kb / DW_STAGES) & 1u, abort_flag, a.status)) break;
                if (c < mcols) {
                    const unsigned char* A = dws + (size_t)st * DW_ST + g * 1024 + (c & 7) * 2;
                    for (int i = 0; i < DW_KB; ++i) {
                        const int k = (i + g) & (DW_KB - 1);
                        const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(A + k * 16));
                        s0 += v.x;
                        s1 += v.y;
                    }
                }
                fz_arrive(&empty[st]);
            }
            if (c < mcols) {
                float* bp = a.bias_part + bpart_off + (size_t)split * M + mt * TC_BM + c;
                bp[0] = s0;
                bp[1] = s1;
            }
        }
    } else if (warp >= 4) {
        // ---------------------------------------------------- partial out
        const int q4 = warp & 3, rl = q4 * 32 + lane, r = mt * TC_BM + rl;
        bool ok = true;
        if (nkb > 0) ok = fz_wait(accf, 0u, abort_flag, a.status);
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // the partial in k_reduce_dw's order: a warp's 32 rows of 4 columns
            // are 512 contiguous bytes
            float4* dst = reinterpret_cast<float4*>(a.part + part_off + (size_t)split * M * N) +
                          (size_t)(r >> 5) * (N >> 2) * 32 + (r & 31);
            for (int cb = 0; cb < DW_TN; cb += 16) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)cb, v);
                tmem_wait(v);
                if (rl < mcols)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        dst[(size_t)((nt * DW_TN + cb) / 4 + i) * 32] =
                            nkb > 0 ? make_float4(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]),
                                                  __uint_as_float(v[4 * i + 2]), __uint_as_float(v[4 * i + 3]))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(DW_TN));
}

// weights of every layer into the fused kernel's chunks: layer l, K chunk c
// (columns 64 c .. 64 c + 63) as an N_l x 64 core-matrix image of N_l * 128
// bytes, element (n, k) at (n / 8) * 1024 + (k % 64 / 8) * 128 + (n % 8) * 16 +
// (k % 8) * 2 within it; one thread per element
__device__ __forceinline__ size_t fz_chunk_offset(int n, int k, int N)
{
    return (size_t)(k >> 6) * N * 128 + (n >> 3) * 1024 + ((k & 63) >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}
// (out x in weights W: the forward pass's B has N = out, K = in; the backward
// chain's B is the transpose, N = in, K = out, in the same layout)
__global__ void k_pack_fused(const __nv_bfloat16* __restrict__ pb, size_t wsrc, int out, int in,
                             unsigned char* __restrict__ dst, unsigned char* __restrict__ dstT)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)out * in) return;
    const int o = (int)(i / in), j = (int)(i % in);
    const __nv_bfloat16 w = pb[wsrc + i];
    *reinterpret_cast<__nv_bfloat16*>(dst + fz_chunk_offset(o, j, out)) = w;
    *reinterpret_cast<__nv_bfloat16*>(dstT + fz_chunk_offset(j, o, in)) = w;
}

// a0 = bf16(s_in (x - c_in)), zero beyond n_in (blockDim.x = the padded width ldo)
__global__ void k_prep_input(const float* __restrict__ x, int batch, int n_in, int ldo, const float* __restrict__ c,
                             const float* __restrict__ sc, __nv_bfloat16* __restrict__ a0)
{
    const int b = blockIdx.x * blockDim.y + threadIdx.y, j = threadIdx.x;
    if (b >= batch || j >= ldo) return;
    const float v = (j < n_in) ? sc[j] * (x[(size_t)b * n_in + j] - c[j]) : 0.f;
    a0[(size_t)b * ldo + j] = __float2bfloat16_rn(v);
}

// loss terms and output gradient: d = y_raw - (t - c_out) / s_out over the first
// n_out columns; dY = bf16(2 d / (batch n_out)); per-block partial sums of d^2
__global__ void k_loss_grad(const float* __restrict__ yraw, int ldy, const float* __restrict__ t, int batch, int n_out,
                            const float* __restrict__ c, const float* __restrict__ sc, __nv_bfloat16* __restrict__ dY,
                            float* __restrict__ partial)
{
    __shared__ float red[256];
    const int b = blockIdx.x * blockDim.y + threadIdx.y, j = threadIdx.x;  // blockDim (64, 4)
    float d2 = 0.f;
    if (b < batch) {
        float gval = 0.f;
        if (j < n_out) {
            const float ts = (t[(size_t)b * n_out + j] - c[j]) / sc[j];
            const float d = yraw[(size_t)b * ldy + j] - ts;
            d2 = d * d;
            gval = 2.0f * d / ((float)batch * (float)n_out);
        }
        dY[(size_t)b * ldy + j] = __float2bfloat16_rn(gval);
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    red[tid] = d2;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (tid < s2) red[tid] += red[tid + s2];
        __syncthreads();
    }
    if (tid == 0) partial[blockIdx.x] = red[0];
}

// sum of n partials in a fixed order, divided by `div`, into *out
__global__ void k_sum_partials(const float* __restrict__ partial, int n, float div, float* __restrict__ out)
{
    __shared__ float red[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int s2 = 128; s2 > 0; s2 >>= 1) {
        if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / div;
}

// bias gradient: partial column sums of the bf16 gradients over chunks of
// BIAS_ROWS rows.  Block (32, 8): a warp reads 64 consecutive columns of a row
// as bf16 pairs (coalesced); the 8 warps take every 8th row of the chunk and
// their sums are added in warp order, so the result does not depend on timing.
constexpr int BIAS_ROWS = 64;
__global__ void k_bias_partial(const __nv_bfloat16* __restrict__ dZ, int ld, int batch, float* __restrict__ part)
{
    __shared__ float2 red[8][32];
    const int c = blockIdx.x * 64 + 2 * threadIdx.x, ch = blockIdx.y, w = threadIdx.y;
    const int b0 = ch * BIAS_ROWS, b1 = min(batch, b0 + BIAS_ROWS);
    float2 s = make_float2(0.f, 0.f);
    if (c < ld)
        for (int b = b0 + w; b < b1; b += 8) {
            const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(dZ + (size_t)b * ld + c));
            s.x += v.x;
            s.y += v.y;
        }
    red[w][threadIdx.x] = s;
    __syncthreads();
    if (w == 0 && c < ld) {
        float2 t = red[0][threadIdx.x];
        for (int k = 1; k < 8; ++k) {
            t.x += red[k][threadIdx.x].x;
            t.y += red[k][threadIdx.x].y;
        }
        part[(size_t)ch * ld + c] = t.x;
        part[(size_t)ch * ld + c + 1] = t.y;
    }
}

// out[i] = sum over s < splits of part[s][i] in a fixed order: block (32, 8),
// warp w adds s = w, w + 8, w + 16, ... for 32 consecutive i, then the eight
// warp sums are added in warp order
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, size_t count, float* __restrict__ out)
{
    __shared__ float red[8][32];
    const size_t i = (size_t)blockIdx.x * 32 + threadIdx.x;
    const int w = threadIdx.y;
    float s = 0.f;
    if (i < count)
        for (int k = w; k < splits; k += 8) s += part[(size_t)k * count + i];
    red[w][threadIdx.x] = s;
    __syncthreads();
    if (w == 0 && i < count) {
        float t = red[0][threadIdx.x];
        for (int k = 1; k < 8; ++k) t += red[k][threadIdx.x];
        out[i] = t;
    }
}
// the weight and bias gradients of every layer from k_dw_tc's partials, in one
// launch of 256-thread blocks.  A layer's weight partial j (of M N, per split) is
// element (m, n) of its gradient, m = (j / (128 N/4)) * 32 + (j / 4) % 32,
// n = ((j / 128) % (N / 4)) * 4 + j % 4 (32-row groups of 4-column groups, 32
// rows x 4 values each); its bias partials are [split][M].  Thread j adds the
// splits s = 0, 1, 2, ... in order (consecutive threads read consecutive
// partials), so the result does not depend on timing.  With loss_n > 0 the last
// block also sums the per-tile squared errors of the training forward pass into
// the loss (in k_sum_partials' order).
// one Adam step (bias-corrected, beta 0.9 / 0.999, eps 1e-8) of parameter i on the
// FP32 masters with gradient g, every operation explicitly rounded so that every
// kernel that applies it gives the same bits; returns the new BF16 copy
__device__ __forceinline__ __nv_bfloat16 adam_update(float* __restrict__ p, float* __restrict__ m,
                                                     float* __restrict__ v, __nv_bfloat16* __restrict__ pb, size_t i,
                                                     float g, float lr, float c1, float c2)
{
    const float mi = __fmaf_rn(0.9f, m[i], __fmul_rn(0.1f, g));
    const float vi = __fmaf_rn(0.999f, v[i], __fmul_rn(__fmul_rn(0.001f, g), g));
    m[i] = mi;
    v[i] = vi;
    const float upd =
        __fdiv_rn(__fmul_rn(lr, __fdiv_rn(mi, c1)), __fadd_rn(__fsqrt_rn(__fdiv_rn(vi, c2)), 1e-8f));
    const float pn = __fsub_rn(p[i], upd);
    p[i] = pn;
    const __nv_bfloat16 q = __float2bfloat16_rn(pn);
    pb[i] = q;
    return q;
}

constexpr int RED_THREADS = 256;
struct RedLayer {
    long long part_off;       // weight partials at part + part_off, [split][M x N]
    long long woff, boff;     // the layer's weights ([M][N]) and biases in the flat parameters
    long long pwoff;          // its chunks in the packed copies
    int M, N, blk0, bpart_off;  // blocks blk0 .. : weights, then bias
};
struct RedArgs {
    RedLayer ly[FZ_MAXL];
    int nl, splits, nblk;
    const float* part;
    const float* bpart;
    float* g;                // gradients (flat parameter layout)
    const float* loss_part;  // per-tile sums of squares, or null
    int loss_n;
    float loss_div;
    float* loss_out;
    // with p set, the Adam step of every parameter follows its gradient
    // (adam_update), and with pw set the packed weight copies (forward pw,
    // transposed pwT, layout of k_pack_fused) get the new BF16 values too
    float *p, *m, *v;
    __nv_bfloat16* pb;
    float lr, c1, c2;
    unsigned char *pw, *pwT;
};

__global__ void __launch_bounds__(RED_THREADS) k_reduce_dw(RedArgs a)
{
    const int t = threadIdx.x;
    if ((int)blockIdx.x >= a.nblk) {
        // the loss: the same strided sums and tree as k_sum_partials
        __shared__ float r[RED_THREADS];
        float s = 0.f;
        for (int i = t; i < a.loss_n; i += RED_THREADS) s += a.loss_part[i];
        r[t] = s;
        __syncthreads();
        for (int s2 = RED_THREADS / 2; s2 > 0; s2 >>= 1) {
            if (t < s2) r[t] += r[t + s2];
            __syncthreads();
        }
        if (t == 0) *a.loss_out = r[0] / a.loss_div;
        return;
    }
    long long part_off = 0, woff = 0, boff = 0, pwoff = 0;
    int M = 0, N = 64, blk0 = 0, bpart_off = 0;
#pragma unroll
    for (int i = 0; i < FZ_MAXL; ++i)
        if (i < a.nl && (int)blockIdx.x >= a.ly[i].blk0) {
            part_off = a.ly[i].part_off;
            woff = a.ly[i].woff;
            boff = a.ly[i].boff;
            pwoff = a.ly[i].pwoff;
            M = a.ly[i].M;
            N = a.ly[i].N;
            blk0 = a.ly[i].blk0;
            bpart_off = a.ly[i].bpart_off;
        }
    const size_t count = (size_t)M * N;
    const size_t wblocks = (count + RED_THREADS - 1) / RED_THREADS;
    const size_t b = (size_t)blockIdx.x - blk0;
    if (b >= wblocks) {
        const int i = (int)(b - wblocks) * RED_THREADS + t;
        if (i < M) {
            const float* q = a.bpart + bpart_off + i;
            float s = 0.f;
            for (int k = 0; k < a.splits; ++k) s += q[(size_t)k * M];
            a.g[boff + i] = s;
            if (a.p) adam_update(a.p, a.m, a.v, a.pb, (size_t)(boff + i), s, a.lr, a.c1, a.c2);
        }
        return;
    }
    const size_t j = b * RED_THREADS + t;
    if (j < count) {
        const float* q = a.part + part_off + j;
        float s = 0.f;
#pragma unroll 8
        for (int k = 0; k < a.splits; ++k) s += q[(size_t)k * count];
        const size_t grp = j / 128;  // (32-row group, 4-column group)
        const int m = (int)(grp / (N / 4)) * 32 + (int)((j / 4) % 32), n = (int)(grp % (N / 4)) * 4 + (int)(j % 4);
        const size_t i = (size_t)woff + (size_t)m * N + n;
        a.g[i] = s;
        if (a.p) {
            const __nv_bfloat16 q = adam_update(a.p, a.m, a.v, a.pb, i, s, a.lr, a.c1, a.c2);
            if (a.pw) {
                *reinterpret_cast<__nv_bfloat16*>(a.pw + pwoff + fz_chunk_offset(m, n, M)) = q;
                *reinterpret_cast<__nv_bfloat16*>(a.pwT + pwoff + fz_chunk_offset(n, m, N)) = q;
            }
        }
    }
}

cudaError_t reduce_splits(const float* part, int splits, size_t count, float* out, cudaStream_t s)
{
    k_reduce_splits<<<(unsigned)((count + 31) / 32), dim3(32, 8), 0, s>>>(part, splits, count, out);
    return cudaGetLastError();
}

// where the weights of each layer sit in the flat parameters and in the fused
// kernel's packed chunks (pw null: no packed copy to refresh)
struct PackTab {
    unsigned char *pw, *pwT;  // forward chunks and the transposed (backward) ones, same offsets
    int L;
    int in[FZ_MAXL], out[FZ_MAXL];
    long long woff[FZ_MAXL], pwoff[FZ_MAXL];
};

// Adam (bias-corrected) on the FP32 masters; refreshes the BF16 copies
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, size_t n, float lr, float c1, float c2, PackTab pk)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const __nv_bfloat16 q = adam_update(p, m, v, pb, i, gr[i], lr, c1, c2);
    // the same value into the fused kernel's packed weight chunks (layout of k_pack_fused)
    if (pk.pw)
        for (int l = 0; l < pk.L; ++l) {
            const long long j = (long long)i - pk.woff[l];
            if (j >= 0 && j < (long long)pk.out[l] * pk.in[l]) {
                const int nn = (int)(j / pk.in[l]), k = (int)(j % pk.in[l]);
                *reinterpret_cast<__nv_bfloat16*>(pk.pw + pk.pwoff[l] + fz_chunk_offset(nn, k, pk.out[l])) = q;
                *reinterpret_cast<__nv_bfloat16*>(pk.pwT + pk.pwoff[l] + fz_chunk_offset(k, nn, pk.in[l])) = q;
                break;
            }
        }
}

// y = s_out y_raw + c_out over the first n_out columns
__global__ void k_output(const float* __restrict__ yraw, int ldy, int batch, int n_out, const float* __restrict__ c,
                         const float* __restrict__ sc, float* __restrict__ y)
{
    const int b = blockIdx.x * blockDim.y + threadIdx.y, j = threadIdx.x;
    if (b >= batch || j >= n_out) return;
    y[(size_t)b * n_out + j] = sc[j] * yraw[(size_t)b * ldy + j] + c[j];
}

// public (unpadded) gradient layout <-> the padded device layout, through the
// index map pidx[k] = padded position of public parameter k
__global__ void k_pack(const float* __restrict__ g, const int* __restrict__ pidx, size_t n, float* __restrict__ out)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = g[pidx[k]];
}

__global__ void k_unpack_scaled(const float* __restrict__ in, const int* __restrict__ pidx, size_t n, float scale,
                                float* __restrict__ g)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) g[pidx[k]] = scale * in[k];
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, size_t n)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

thread_local std::string g_mlp_error;

lbib_status mlp_fail(lbib_status s, const std::string& m)
{
    g_mlp_error = m;
    set_global_error(m.c_str());
    return s;
}

__global__ void k_or_word(uint32_t* w, uint32_t bits) { atomicOr(w, bits); }

}  // namespace

struct lbib_mlp {
    lbib_mlp_desc desc{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int L = 0;                      // weight layers
    std::vector<int> in, out;       // padded dims per layer
    std::vector<int> in_true, out_true;
    std::vector<size_t> woff, boff; // offsets into the flat parameter arrays
    size_t nparam = 0;              // padded flat size
    size_t ntrue = 0;               // host (unpadded) size
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* pb = nullptr;
    float *cin = nullptr, *sin = nullptr, *cout = nullptr, *sout = nullptr;
    int max_batch = 0;
    __nv_bfloat16* a0 = nullptr;            // [B][in0]
    std::vector<__nv_bfloat16*> act;        // per hidden layer [B][width]
    std::vector<float*> z;                  // per hidden layer [B][width]
    float* yraw = nullptr;                  // [B][outL]
    __nv_bfloat16 *dY = nullptr, *dZa = nullptr, *dZb = nullptr;
    float* part = nullptr;                  // split-K / bias partials
    size_t part_floats = 0;
    float* loss_part = nullptr;
    float* loss_dev = nullptr;
    int* pidx = nullptr;                    // padded position of each public parameter
    int64_t t = 0;                          // Adam steps
    uint32_t* status = nullptr;             // bounded-wait error word of the tensor-core kernels
    // set when a sync found that a bounded wait gave up: the products of that
    // call were not completed, so the network refuses work until its
    // parameters are set again
    lbib_status fault = LBIB_OK;
    bool tc = true;                         // forward products on tcgen05
    // fused inference (k_mlp_fused): packed weight chunks, refreshed after every update
    unsigned char* pw = nullptr;
    unsigned char* pwT = nullptr;           // transposed chunks (backward chain), offsets pwoff
    long long pwoff[FZ_MAXL] = {};
    std::vector<__nv_bfloat16*> dzs;        // dZ_l of the hidden layers (tiled), fused backward
    float* bpart = nullptr;                 // [split][out] bias-gradient partials of k_dw_tc, every layer
    size_t bpart_floats = 0;
    bool pw_dirty = true;
    bool z_tiled = false;  // pre-activations stored tiled (zt_index) by the last forward pass
    bool fused = false;                     // network shape fits the fused kernel
    int nsm = 148;
    std::vector<void*> allocs;
};

namespace {

// status word of the finished work: a bounded wait that gave up makes the
// network refuse work (sticky) until lbib_mlp_set_params
lbib_status mlp_check_status(lbib_mlp* net)
{
    uint32_t st = 0;
    const cudaError_t e = cudaMemcpy(&st, net->status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("status read: ") + cudaGetErrorString(e));
    if (st & 1u) {
        net->fault = LBIB_ERR_TIMEOUT;
        return mlp_fail(LBIB_ERR_TIMEOUT, "a tensor-core kernel gave up a bounded wait (its products are incomplete)");
    }
    return LBIB_OK;
}

template <typename T>
cudaError_t mlp_alloc(lbib_mlp* net, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = device_malloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) {
        net->allocs.push_back(q);
        *p = static_cast<T*>(q);
    }
    return e;
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const GemmArgs& a0, int splits, cudaStream_t s)
{
    GemmArgs a = a0;
    const int kt = (a.K + BK - 1) / BK;
    splits = std::max(1, std::min(splits, kt));
    a.k_tiles_per_split = (kt + splits - 1) / splits;
    splits = (kt + a.k_tiles_per_split - 1) / a.k_tiles_per_split;
    dim3 grid((a.M + BM - 1) / BM, a.N / BN, splits);
    k_gemm<TA, TB, EPI><<<grid, GEMM_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t gemm_tc(const GemmArgs& a, cudaStream_t s)
{
    static_assert(tc_smem_bytes(256) <= TC_SMEM_REQUEST, "tiles fit the request");
    const size_t smem = TC_SMEM_REQUEST;
    dim3 grid((a.M + TC_BM - 1) / TC_BM);
    k_gemm_tc<EPI><<<grid, TC_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

// forward pass of `batch` rows already in net->a0; leaves y_raw
cudaError_t forward_core(lbib_mlp* net, int batch, bool store_z = true)
{
    cudaError_t e = cudaSuccess;
    const __nv_bfloat16* a = net->a0;
    int lda = net->in[0];
    for (int l = 0; l < net->L && e == cudaSuccess; ++l) {
        GemmArgs g{};
        g.A = a;
        g.lda = lda;
        g.B = net->pb + net->woff[l];
        g.ldb = net->in[l];
        g.M = batch;
        g.N = net->out[l];
        g.K = net->in[l];
        g.bias = net->p + net->boff[l];
        g.ldc = net->out[l];
        g.status = net->status;
        const bool tc = net->tc && g.K % TC_BK == 0 && g.N % 16 == 0 && g.N <= 256;
        if (l + 1 < net->L) {
            // pre-activations are kept for the backward pass only (the tensor-core path may skip them)
            g.Zout = (store_z || !tc) ? net->z[l] : nullptr;
            g.Aout = net->act[l];
            e = tc ? gemm_tc<EPI_FWD_GELU>(g, net->stream) : gemm<false, false, EPI_FWD_GELU>(g, 1, net->stream);
            a = net->act[l];
            lda = net->out[l];
        } else {
            g.Zout = net->yraw;
            e = tc ? gemm_tc<EPI_FWD_LIN>(g, net->stream) : gemm<false, false, EPI_FWD_LIN>(g, 1, net->stream);
        }
    }
    return e;
}

// inference through k_mlp_fused: weight chunks re-packed after an update,
// one persistent CTA per SM (at most one per 128-row tile)
cudaError_t forward_fused(lbib_mlp* net, const float* x, int batch, float* y, const float* t = nullptr)
{
    const bool train = t != nullptr;
    if (net->pw_dirty) {
        for (int l = 0; l < net->L; ++l) {
            const size_t n = (size_t)net->out[l] * net->in[l];
            k_pack_fused<<<(unsigned)((n + 255) / 256), 256, 0, net->stream>>>(net->pb, net->woff[l], net->out[l],
                                                                               net->in[l], net->pw + net->pwoff[l],
                                                                               net->pwT + net->pwoff[l]);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        net->pw_dirty = false;
    }
    FusedArgs a{};
    a.x = x;
    a.y = y;
    a.M = batch;
    a.n_in = net->desc.n_in;
    a.n_out = net->desc.n_out;
    a.L = net->L;
    a.w = net->pw;
    a.bias = net->p;
    for (int l = 0; l < net->L; ++l) {
        a.K[l] = net->in[l];
        a.N[l] = net->out[l];
        a.boff[l] = (int)net->boff[l];
        a.woff[l] = net->pwoff[l];
    }
    a.cin = net->cin;
    a.sin = net->sin;
    a.cout = net->cout;
    a.sout = net->sout;
    a.status = net->status;
    if (train) {
        for (int l = 0; l + 1 < net->L; ++l) {
            a.zout[l] = net->z[l];
            a.aout[l] = net->act[l];
        }
        a.a0_out = net->a0;
        a.dy_out = net->dY;
        a.t = t;
        a.loss_rows = net->loss_part;
    }
    const int ntiles = (batch + TC_BM - 1) / TC_BM;
    if (train)
        k_mlp_fused<FZ_TRAIN><<<std::min(ntiles, net->nsm), FZ_THREADS, FZ_SMEM, net->stream>>>(a);
    else
        k_mlp_fused<FZ_INFER><<<std::min(ntiles, net->nsm), FZ_THREADS, FZ_SMEM, net->stream>>>(a);
    return cudaGetLastError();
}

int splits_for(int batch)
{
    // enough blocks for the weight-gradient GEMMs (K = batch) to fill the GPU
    return std::max(1, std::min(MAX_SPLITS, (batch + 255) / 256));
}

// backward pass after forward_core and the loss gradient in dY; gradients into net->g
// the backward chain on tcgen05 (k_mlp_fused<FZ_BWD>): for l = L-1 .. 1,
// dZ_{l-1} = bf16((dZ_l W_l) * GELU'(z_{l-1})), tile by tile through every layer,
// from the output gradient dY; each dZ_{l-1} into dzs[l-1] (tiled)
cudaError_t backward_chain(lbib_mlp* net, int batch)
{
    if (net->dzs.size() + 1 < (size_t)net->L || !net->pwT) return cudaErrorInvalidValue;
    FusedArgs a{};
    a.M = batch;
    a.L = net->L - 1;
    a.w = net->pwT;
    a.status = net->status;
    a.dy = net->dY;
    for (int s = 0; s < a.L; ++s) {
        const int l = net->L - 1 - s;
        a.K[s] = net->out[l];
        a.N[s] = net->in[l];
        a.woff[s] = net->pwoff[l];
        a.zout[s] = net->z[l - 1];
        a.aout[s] = net->dzs[l - 1];
    }
    const int ntiles = (batch + TC_BM - 1) / TC_BM;
    k_mlp_fused<FZ_BWD><<<std::min(ntiles, net->nsm), FZ_THREADS, FZ_SMEM, net->stream>>>(a);
    return cudaGetLastError();
}

// an optimiser step to apply with the gradients (lr, bias corrections)
struct AdamStep {
    float lr, c1, c2;
};

// every layer's weight and bias gradients on tcgen05 after the gradient chain,
// with the loss of the fused forward pass: one k_dw_tc launch (all layers' 128 x
// 64 output tiles times batch slices of whole 64-row blocks, about two CTAs per
// SM) and one k_reduce_dw launch (the partials summed in a fixed order, and the
// Adam step when st is given)
cudaError_t gradients_tc(lbib_mlp* net, int batch, const AdamStep* st)
{
    int T = 0;  // output tiles over all layers
    for (int l = 0; l < net->L; ++l) T += (net->out[l] + TC_BM - 1) / TC_BM * (net->in[l] / DW_TN);
    const int nsplit =
        std::max(1, std::min(std::min(MAX_SPLITS, 2 * net->nsm / T), (batch + DW_KB - 1) / DW_KB));
    const int rps = ((batch + nsplit - 1) / nsplit + DW_KB - 1) / DW_KB * DW_KB;
    const int used = (batch + rps - 1) / rps;
    DwArgs da{};
    RedArgs ra{};
    da.nl = ra.nl = net->L;
    da.batch = batch;
    da.rows_per_split = rps;
    da.part = net->part;
    da.bias_part = net->bpart;
    da.status = net->status;
    long long poff = 0;
    int cta = 0, boff = 0, blk = 0;
    for (int l = 0; l < net->L; ++l) {
        const int M = net->out[l], N = net->in[l], tiles = (M + TC_BM - 1) / TC_BM * (N / DW_TN);
        // dZ of the layer's pre-activation: the loss gradient for the output layer,
        // the chain's result for the hidden ones
        da.ly[l] = DwLayer{l + 1 == net->L ? net->dY : net->dzs[l], l == 0 ? net->a0 : net->act[l - 1], poff, M, N,
                           tiles, cta, boff};
        ra.ly[l] = RedLayer{poff, (long long)net->woff[l], (long long)net->boff[l], net->pwoff[l], M, N, blk, boff};
        poff += (long long)used * M * N;
        boff += used * M;
        cta += tiles * used;
        blk += (int)(((size_t)M * N + RED_THREADS - 1) / RED_THREADS + (M + RED_THREADS - 1) / RED_THREADS);
    }
    if ((size_t)poff > net->part_floats || (size_t)boff > net->bpart_floats) return cudaErrorInvalidValue;
    k_dw_tc<<<cta, DW_THREADS, DW_SMEM, net->stream>>>(da);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ra.splits = used;
    ra.nblk = blk;
    ra.part = net->part;
    ra.bpart = net->bpart;
    ra.loss_part = net->loss_part;
    ra.loss_n = (batch + TC_BM - 1) / TC_BM;
    ra.loss_div = (float)batch * (float)net->desc.n_out;
    ra.loss_out = net->loss_dev;
    ra.g = net->g;
    if (st) {
        ra.p = net->p;
        ra.m = net->m;
        ra.v = net->v;
        ra.pb = net->pb;
        ra.lr = st->lr;
        ra.c1 = st->c1;
        ra.c2 = st->c2;
        // a packed copy that is current stays current: the update writes it too
        ra.pw = (net->fused && !net->pw_dirty) ? net->pw : nullptr;
        ra.pwT = net->pwT;
    }
    k_reduce_dw<<<blk + 1, RED_THREADS, 0, net->stream>>>(ra);
    return cudaGetLastError();
}

PackTab pack_tab(const lbib_mlp* net);

// the gradients of the loss of the last prep_and_loss into net->g, then, with
// st, the Adam step
cudaError_t backward_core(lbib_mlp* net, int batch, const AdamStep* st = nullptr)
{
    cudaError_t e = cudaSuccess;
    // after the fused forward pass (tiled pre-activations) the gradients of the
    // pre-activations come from the tcgen05 chain, stored tiled, and the weight
    // gradients from tensor-core products over batch slices
    if (net->z_tiled) {
        if (net->L > 1 && (e = backward_chain(net, batch)) != cudaSuccess) return e;
        return gradients_tc(net, batch, st);
    }
    const __nv_bfloat16* dcur = net->dY;  // gradient w.r.t. the current layer's output (pre-activation)
    int ldd = net->out[net->L - 1];
    const int splits = splits_for(batch);
    for (int l = net->L - 1; l >= 0 && e == cudaSuccess; --l) {
        const __nv_bfloat16* ain = (l == 0) ? net->a0 : net->act[l - 1];
        const int ldin = net->in[l];
        // dW_l = dcur^T ain: M = out, N = in, K = batch; both operands batch-major
        GemmArgs gw{};
        gw.A = dcur;
        gw.lda = ldd;
        gw.B = ain;
        gw.ldb = ldin;
        gw.M = net->out[l];
        gw.N = net->in[l];
        gw.K = batch;
        gw.part = net->part;
        gw.ldc = net->in[l];
        e = gemm<true, true, EPI_PARTIAL>(gw, splits, net->stream);
        if (e != cudaSuccess) break;
        {
            const int kt = (batch + BK - 1) / BK;
            const int tps = (kt + std::min(splits, kt) - 1) / std::min(splits, kt);
            const int used = (kt + tps - 1) / tps;
            const size_t cnt = (size_t)net->out[l] * net->in[l];
            e = reduce_splits(net->part, used, cnt, net->g + net->woff[l], net->stream);
            if (e != cudaSuccess) break;
        }
        // db_l = column sums of dcur
        {
            const int chunks = (batch + BIAS_ROWS - 1) / BIAS_ROWS;
            dim3 grid((ldd + 63) / 64, chunks);
            k_bias_partial<<<grid, dim3(32, 8), 0, net->stream>>>(dcur, ldd, batch, net->part);
            e = reduce_splits(net->part, chunks, (size_t)ldd, net->g + net->boff[l], net->stream);
            if (e != cudaSuccess) break;
        }
        e = cudaGetLastError();
        if (l == 0 || e != cudaSuccess) break;
        // d pre-activation of layer l-1 = (dcur W_l) * GELU'(z_{l-1}): M = batch, N = in_l, K = out_l
        __nv_bfloat16* dnext = (dcur == net->dZa) ? net->dZb : net->dZa;
        GemmArgs gx{};
        gx.A = dcur;
        gx.lda = ldd;
        gx.B = net->pb + net->woff[l];  // W_l stored [out][in] = [K][N]
        gx.ldb = net->in[l];
        gx.M = batch;
        gx.N = net->in[l];
        gx.K = net->out[l];
        gx.Zin = net->z[l - 1];
        gx.Aout = dnext;
        gx.ldc = net->in[l];
        e = gemm<false, true, EPI_BWD_GELU>(gx, 1, net->stream);
        dcur = dnext;
        ldd = net->in[l];
    }
    if (e == cudaSuccess && st) {
        k_adam<<<(unsigned)((net->nparam + 255) / 256), 256, 0, net->stream>>>(
            net->p, net->g, net->m, net->v, net->pb, net->nparam, st->lr, st->c1, st->c2, pack_tab(net));
        e = cudaGetLastError();
    }
    return e;
}

// the packed weight chunks of the fused kernel, for the optimiser to keep
// current (null when there are none, or when they are stale anyway)
PackTab pack_tab(const lbib_mlp* net)
{
    PackTab t{};
    t.pw = (net->fused && !net->pw_dirty) ? net->pw : nullptr;
    t.pwT = net->pwT;
    t.L = net->L;
    for (int l = 0; l < net->L; ++l) {
        t.in[l] = net->in[l];
        t.out[l] = net->out[l];
        t.woff[l] = (long long)net->woff[l];
        t.pwoff[l] = net->pwoff[l];
    }
    return t;
}

cudaError_t prep_and_loss(lbib_mlp* net, const float* x, const float* t, int batch)
{
    net->z_tiled = net->fused;  // the fused kernel stores what the backward pass reads tiled
    if (net->fused) {
        // one fused kernel: the inputs, every layer's pre-activations and activations,
        // the loss gradient and the squared errors per tile (every caller runs
        // backward_core next: its reduction launch sums the loss)
        return forward_fused(net, x, batch, net->yraw, t);
    }
    dim3 blk(64, 4);
    k_prep_input<<<(batch + blk.y - 1) / blk.y, blk, 0, net->stream>>>(x, batch, net->desc.n_in, net->in[0],
                                                                       net->cin, net->sin, net->a0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_core(net, batch);
    if (e != cudaSuccess) return e;
    const int ldy = net->out[net->L - 1];
    dim3 lb(64, 4);
    const int nblk = (batch + 3) / 4;
    // the output layer is padded to 64 columns: blockDim.x covers it
    k_loss_grad<<<nblk, lb, 0, net->stream>>>(net->yraw, ldy, t, batch, net->desc.n_out, net->cout, net->sout,
                                              net->dY, net->loss_part);
    k_sum_partials<<<1, 256, 0, net->stream>>>(net->loss_part, nblk, (float)batch * (float)net->desc.n_out,
                                               net->loss_dev);
    return cudaGetLastError();
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~Guard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" {

lbib_status lbib_mlp_create(const lbib_mlp_desc* d, lbib_mlp** out)
{
    LBIB_TRACE("lbib_mlp_create");
    if (!d || !out) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (d->n_in < 1 || d->n_in > 32 || d->width < 64 || d->width % 64 || d->width > 1024 || d->n_hidden < 1 ||
        d->n_hidden > 8 || d->n_out < 1 || d->n_out > 64 || d->max_batch < 1)
        return mlp_fail(LBIB_ERR_INVALID_ARG, "need 1 <= n_in <= 32, width a multiple of 64 up to 1024, "
                                              "1 <= n_hidden <= 8, 1 <= n_out <= 64, max_batch >= 1");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || d->device < 0 || d->device >= ndev) {
        cudaGetLastError();
        return mlp_fail(LBIB_ERR_CUDA, "no CUDA device with that ordinal");
    }
    lbib_mlp* net = new (std::nothrow) lbib_mlp();
    if (!net) return mlp_fail(LBIB_ERR_OOM, "host allocation failed");
    net->desc = *d;
    net->desc.in_shift = net->desc.in_scale = net->desc.out_shift = net->desc.out_scale = nullptr;
    net->device = d->device;
    Guard guard(net->device);
    auto bail = [&](cudaError_t e, const char* what) {
        lbib_mlp_destroy(net);
        cudaGetLastError();
        return mlp_fail(e == cudaErrorMemoryAllocation ? LBIB_ERR_OOM : LBIB_ERR_CUDA,
                        std::string(what) + ": " + cudaGetErrorString(e));
    };
    net->L = d->n_hidden + 1;
    for (int l = 0; l < net->L; ++l) {
        const int it = (l == 0) ? d->n_in : d->width, ot = (l + 1 < net->L) ? d->width : d->n_out;
        net->in_true.push_back(it);
        net->out_true.push_back(ot);
        net->in.push_back(l == 0 ? 64 : d->width);  // every GEMM dimension a multiple of the 64 tile
        net->out.push_back(l + 1 < net->L ? d->width : 64);
    }
    size_t off = 0;
    for (int l = 0; l < net->L; ++l) {
        net->woff.push_back(off);
        off += (size_t)net->out[l] * net->in[l];
        net->boff.push_back(off);
        off += (size_t)net->out[l];
        net->ntrue += (size_t)net->out_true[l] * net->in_true[l] + net->out_true[l];
    }
    net->nparam = off;
    net->max_batch = d->max_batch;
    const size_t B = (size_t)d->max_batch;
    cudaError_t e = cudaSuccess;
#define MA(p, n)                                     \
    do {                                             \
        e = mlp_alloc(net, &(p), (n));               \
        if (e != cudaSuccess) return bail(e, #p);    \
    } while (0)
    MA(net->p, net->nparam);
    MA(net->g, net->nparam);
    MA(net->m, net->nparam);
    MA(net->v, net->nparam);
    MA(net->pb, net->nparam);
    MA(net->cin, 32);
    MA(net->sin, 32);
    MA(net->cout, 64);
    MA(net->sout, 64);
    const size_t BT = (B + TC_BM - 1) / TC_BM * TC_BM;  // whole 128-row tiles (the tiled layouts)
    MA(net->a0, BT * 64);
    for (int l = 0; l + 1 < net->L; ++l) {
        __nv_bfloat16* a = nullptr;
        float* z = nullptr;
        MA(a, (B + TC_BM - 1) / TC_BM * TC_BM * d->width);  // whole 128-row tiles (the tiled layouts)
        MA(z, (B + TC_BM - 1) / TC_BM * TC_BM * d->width);
        net->act.push_back(a);
        net->z.push_back(z);
    }
    MA(net->yraw, B * 64);
    MA(net->dY, BT * 64);
    MA(net->dZa, B * d->width);
    MA(net->dZb, B * d->width);
    const size_t wmax = (size_t)d->width * d->width;
    const int chunks = (int)((B + BIAS_ROWS - 1) / BIAS_ROWS);  // bias-gradient partials
    net->part_floats = std::max((size_t)MAX_SPLITS * wmax, (size_t)chunks * d->width);
    cudaDeviceGetAttribute(&net->nsm, cudaDevAttrMultiProcessorCount, net->device);
    {
        // gradients_tc: at most max(2 SMs, output tiles) CTAs' 128 x 64 partials
        size_t tiles = 0, outs = 0;
        for (int l = 0; l < net->L; ++l) {
            tiles += (size_t)(net->out[l] + TC_BM - 1) / TC_BM * (net->in[l] / DW_TN);
            outs += (size_t)net->out[l];
        }
        net->part_floats = std::max(net->part_floats, std::max((size_t)2 * net->nsm, tiles) * TC_BM * DW_TN);
        net->bpart_floats = (size_t)MAX_SPLITS * outs;
    }
    MA(net->part, net->part_floats);
    MA(net->loss_part, BT * 4);  // per tile (fused), per block of 4 rows otherwise
    MA(net->loss_dev, 1);
    MA(net->status, 1);
    MA(net->pidx, net->ntrue);
    net->fused = d->width <= FZ_MAXW && net->L <= FZ_MAXL;
    if (net->fused) {
        for (int l = 0; l + 1 < net->L; ++l) {
            __nv_bfloat16* dz = nullptr;
            MA(dz, (B + TC_BM - 1) / TC_BM * TC_BM * d->width);
            net->dzs.push_back(dz);
        }
        MA(net->bpart, net->bpart_floats);
    }
    if (net->fused) {
        size_t bytes = 0;
        for (int l = 0; l < net->L; ++l) {
            net->pwoff[l] = (long long)bytes;
            bytes += (size_t)net->out[l] * net->in[l] * 2;
        }
        MA(net->pw, bytes);
        MA(net->pwT, bytes);
    }
#undef MA
    // shared-memory opt-ins are per device: set them here, with the net's device current
    if ((e = cudaFuncSetAttribute(k_gemm_tc<EPI_FWD_GELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TC_SMEM_REQUEST)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_gemm_tc<EPI_FWD_LIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TC_SMEM_REQUEST)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_fused<FZ_INFER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FZ_SMEM)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_fused<FZ_TRAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FZ_SMEM)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(k_dw_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DW_SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_mlp_fused<FZ_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FZ_SMEM)) !=
            cudaSuccess)
        return bail(e, "cudaFuncSetAttribute");
    if (d->cuda_stream) {
        net->stream = static_cast<cudaStream_t>(d->cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(e, "cudaStreamCreate");
        net->own_stream = true;
    }
    // normalisation constants
    std::vector<float> cin(32, 0.f), sin(32, 1.f), cout(64, 0.f), sout(64, 1.f);
    for (int j = 0; j < d->n_in; ++j) {
        if (d->in_shift) cin[j] = d->in_shift[j];
        if (d->in_scale) sin[j] = d->in_scale[j];
    }
    for (int j = 0; j < d->n_out; ++j) {
        if (d->out_shift) cout[j] = d->out_shift[j];
        if (d->out_scale) sout[j] = d->out_scale[j];
    }
    for (int j = 0; j < d->n_out; ++j)
        if (!(sout[j] != 0.f) || !std::isfinite(sout[j])) {
            lbib_mlp_destroy(net);
            return mlp_fail(LBIB_ERR_INVALID_ARG, "out_scale must be finite and non-zero");
        }
    {
        std::vector<int> idx;
        idx.reserve(net->ntrue);
        for (int l = 0; l < net->L; ++l) {
            for (int o = 0; o < net->out_true[l]; ++o)
                for (int i = 0; i < net->in_true[l]; ++i) idx.push_back((int)(net->woff[l] + (size_t)o * net->in[l] + i));
            for (int o = 0; o < net->out_true[l]; ++o) idx.push_back((int)(net->boff[l] + o));
        }
        if ((e = cudaMemcpyAsync(net->pidx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice,
                                 net->stream)) != cudaSuccess)
            return bail(e, "cudaMemcpy");
    }
    if ((e = cudaMemcpyAsync(net->cin, cin.data(), 32 * 4, cudaMemcpyHostToDevice, net->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(net->sin, sin.data(), 32 * 4, cudaMemcpyHostToDevice, net->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(net->cout, cout.data(), 64 * 4, cudaMemcpyHostToDevice, net->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(net->sout, sout.data(), 64 * 4, cudaMemcpyHostToDevice, net->stream)) != cudaSuccess)
        return bail(e, "cudaMemcpy");
    // Glorot-uniform weights from a host generator (splitmix64), zero biases and padding
    std::vector<float> h(net->nparam, 0.f);
    uint64_t st = d->seed ^ 0x9e3779b97f4a7c15ULL;
    auto next = [&]() {
        st += 0x9e3779b97f4a7c15ULL;
        uint64_t zz = st;
        zz = (zz ^ (zz >> 30)) * 0xbf58476d1ce4e5b9ULL;
        zz = (zz ^ (zz >> 27)) * 0x94d049bb133111ebULL;
        zz ^= zz >> 31;
        return (double)(zz >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < net->L; ++l) {
        const double lim = std::sqrt(6.0 / (net->in_true[l] + net->out_true[l]));
        for (int o = 0; o < net->out_true[l]; ++o)
            for (int i = 0; i < net->in_true[l]; ++i)
                h[net->woff[l] + (size_t)o * net->in[l] + i] = (float)((2.0 * next() - 1.0) * lim);
    }
    if ((e = cudaMemcpyAsync(net->p, h.data(), net->nparam * 4, cudaMemcpyHostToDevice, net->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(net->m, 0, net->nparam * 4, net->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(net->v, 0, net->nparam * 4, net->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(net->g, 0, net->nparam * 4, net->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(net->status, 0, 4, net->stream)) != cudaSuccess)
        return bail(e, "initialisation");
    k_to_bf16<<<(unsigned)((net->nparam + 255) / 256), 256, 0, net->stream>>>(net->p, net->pb, net->nparam);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(net->stream)) != cudaSuccess)
        return bail(e, "initialisation");
    *out = net;
    return LBIB_OK;
}

lbib_status lbib_mlp_forward(lbib_mlp* net, const float* x, int32_t batch, float* y)
{
    LBIB_TRACE("lbib_mlp_forward");
    if (!net || !x || !y) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (net->fault != LBIB_OK) return mlp_fail(net->fault, "a bounded device wait gave up earlier: set the parameters again");
    if (batch < 1 || batch > net->max_batch) return mlp_fail(LBIB_ERR_INVALID_ARG, "batch outside 1 .. max_batch");
    Guard guard(net->device);
    if (net->tc && net->fused) {
        cudaError_t e = forward_fused(net, x, batch, y);
        if (e != cudaSuccess)
            return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_forward: ") + cudaGetErrorString(e));
        return LBIB_OK;
    }
    dim3 blk(64, 4);
    k_prep_input<<<(batch + 3) / 4, blk, 0, net->stream>>>(x, batch, net->desc.n_in, net->in[0], net->cin, net->sin,
                                                           net->a0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward_core(net, batch, false);
    if (e == cudaSuccess) {
        dim3 ob(64, 4);
        k_output<<<(batch + 3) / 4, ob, 0, net->stream>>>(net->yraw, net->out[net->L - 1], batch, net->desc.n_out,
                                                          net->cout, net->sout, y);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_forward: ") + cudaGetErrorString(e));
    return LBIB_OK;
}

lbib_status lbib_mlp_train_step(lbib_mlp* net, const float* x, const float* t, int32_t batch, float lr, float* loss)
{
    LBIB_TRACE("lbib_mlp_train_step");
    if (!net || !x || !t) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (net->fault != LBIB_OK) return mlp_fail(net->fault, "a bounded device wait gave up earlier: set the parameters again");
    if (batch < 1 || batch > net->max_batch) return mlp_fail(LBIB_ERR_INVALID_ARG, "batch outside 1 .. max_batch");
    if (!(lr > 0.f) || !std::isfinite(lr)) return mlp_fail(LBIB_ERR_INVALID_ARG, "lr must be positive");
    Guard guard(net->device);
    cudaError_t e = prep_and_loss(net, x, t, batch);
    const int64_t step = net->t + 1;
    const AdamStep st{lr, 1.0f - (float)std::pow(0.9, (double)step), 1.0f - (float)std::pow(0.999, (double)step)};
    if (e == cudaSuccess) e = backward_core(net, batch, &st);
    if (e == cudaSuccess) net->t = step;
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net->loss_dev, 4, cudaMemcpyDeviceToDevice, net->stream);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_train_step: ") + cudaGetErrorString(e));
    return LBIB_OK;
}

lbib_status lbib_mlp_backward(lbib_mlp* net, const float* x, const float* t, int32_t batch, float* grad, size_t n,
                              float* loss)
{
    LBIB_TRACE("lbib_mlp_backward");
    if (!net || !x || !t || !grad) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (net->fault != LBIB_OK) return mlp_fail(net->fault, "a bounded device wait gave up earlier: set the parameters again");
    if (n < net->ntrue) return mlp_fail(LBIB_ERR_INVALID_ARG, "buffer smaller than the parameter count");
    if (batch < 1 || batch > net->max_batch) return mlp_fail(LBIB_ERR_INVALID_ARG, "batch outside 1 .. max_batch");
    Guard guard(net->device);
    cudaError_t e = prep_and_loss(net, x, t, batch);
    if (e == cudaSuccess) e = backward_core(net, batch);
    if (e == cudaSuccess) {
        k_pack<<<(unsigned)((net->ntrue + 255) / 256), 256, 0, net->stream>>>(net->g, net->pidx, net->ntrue, grad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, net->loss_dev, 4, cudaMemcpyDeviceToDevice, net->stream);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_backward: ") + cudaGetErrorString(e));
    return LBIB_OK;
}

lbib_status lbib_mlp_apply_gradient(lbib_mlp* net, const float* grad, size_t n, float scale, float lr)
{
    LBIB_TRACE("lbib_mlp_apply_gradient");
    if (!net || !grad) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (net->fault != LBIB_OK) return mlp_fail(net->fault, "a bounded device wait gave up earlier: set the parameters again");
    if (n < net->ntrue) return mlp_fail(LBIB_ERR_INVALID_ARG, "buffer smaller than the parameter count");
    if (!std::isfinite(scale)) return mlp_fail(LBIB_ERR_INVALID_ARG, "scale must be finite");
    if (!(lr > 0.f) || !std::isfinite(lr)) return mlp_fail(LBIB_ERR_INVALID_ARG, "lr must be positive");
    Guard guard(net->device);
    // padding entries of the gradient stay zero, so Adam leaves the padded weights at zero
    cudaError_t e = cudaMemsetAsync(net->g, 0, net->nparam * 4, net->stream);
    if (e == cudaSuccess) {
        k_unpack_scaled<<<(unsigned)((net->ntrue + 255) / 256), 256, 0, net->stream>>>(grad, net->pidx, net->ntrue,
                                                                                       scale, net->g);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        net->t += 1;
        const float c1 = 1.0f - (float)std::pow(0.9, (double)net->t);
        const float c2 = 1.0f - (float)std::pow(0.999, (double)net->t);
        // a packed copy that is current stays current: the update writes it too
        k_adam<<<(unsigned)((net->nparam + 255) / 256), 256, 0, net->stream>>>(net->p, net->g, net->m, net->v, net->pb,
                                                                               net->nparam, lr, c1, c2, pack_tab(net));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_apply_gradient: ") + cudaGetErrorString(e));
    return LBIB_OK;
}

lbib_status lbib_mlp_param_count(lbib_mlp* net, size_t* n)
{
    if (!net || !n) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    *n = net->ntrue;
    return LBIB_OK;
}

static void padded_to_host(const lbib_mlp* net, const std::vector<float>& pad, float* out)
{
    size_t k = 0;
    for (int l = 0; l < net->L; ++l) {
        for (int o = 0; o < net->out_true[l]; ++o)
            for (int i = 0; i < net->in_true[l]; ++i) out[k++] = pad[net->woff[l] + (size_t)o * net->in[l] + i];
        for (int o = 0; o < net->out_true[l]; ++o) out[k++] = pad[net->boff[l] + o];
    }
}

lbib_status lbib_mlp_gradients(lbib_mlp* net, const float* x, const float* t, int32_t batch, float* grad, size_t n,
                               float* loss)
{
    LBIB_TRACE("lbib_mlp_gradients");
    if (!net || !x || !t || !grad) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (net->fault != LBIB_OK) return mlp_fail(net->fault, "a bounded device wait gave up earlier: set the parameters again");
    if (n < net->ntrue) return mlp_fail(LBIB_ERR_INVALID_ARG, "buffer smaller than the parameter count");
    if (batch < 1 || batch > net->max_batch) return mlp_fail(LBIB_ERR_INVALID_ARG, "batch outside 1 .. max_batch");
    Guard guard(net->device);
    cudaError_t e = prep_and_loss(net, x, t, batch);
    if (e == cudaSuccess) e = backward_core(net, batch);
    std::vector<float> h(net->nparam);
    float lh = 0.f;
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), net->g, net->nparam * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&lh, net->loss_dev, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_gradients: ") + cudaGetErrorString(e));
    const lbib_status st = mlp_check_status(net);
    if (st != LBIB_OK) return st;
    padded_to_host(net, h, grad);
    if (loss) *loss = lh;
    return LBIB_OK;
}

lbib_status lbib_mlp_get_params(lbib_mlp* net, float* params, size_t n)
{
    LBIB_TRACE("lbib_mlp_get_params");
    if (!net || !params) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (n < net->ntrue) return mlp_fail(LBIB_ERR_INVALID_ARG, "buffer smaller than the parameter count");
    Guard guard(net->device);
    std::vector<float> h(net->nparam);
    cudaError_t e = cudaStreamSynchronize(net->stream);
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), net->p, net->nparam * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_get_params: ") + cudaGetErrorString(e));
    const lbib_status st = mlp_check_status(net);
    if (st != LBIB_OK) return st;
    padded_to_host(net, h, params);
    return LBIB_OK;
}

lbib_status lbib_mlp_set_params(lbib_mlp* net, const float* params, size_t n)
{
    LBIB_TRACE("lbib_mlp_set_params");
    if (!net || !params) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (n < net->ntrue) return mlp_fail(LBIB_ERR_INVALID_ARG, "buffer smaller than the parameter count");
    for (size_t i = 0; i < net->ntrue; ++i)
        if (!std::isfinite(params[i])) return mlp_fail(LBIB_ERR_INVALID_ARG, "non-finite parameter");
    Guard guard(net->device);
    std::vector<float> h(net->nparam, 0.f);
    size_t k = 0;
    for (int l = 0; l < net->L; ++l) {
        for (int o = 0; o < net->out_true[l]; ++o)
            for (int i = 0; i < net->in_true[l]; ++i) h[net->woff[l] + (size_t)o * net->in[l] + i] = params[k++];
        for (int o = 0; o < net->out_true[l]; ++o) h[net->boff[l] + o] = params[k++];
    }
    cudaError_t e = cudaStreamSynchronize(net->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(net->p, h.data(), net->nparam * 4, cudaMemcpyHostToDevice, net->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->m, 0, net->nparam * 4, net->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->v, 0, net->nparam * 4, net->stream);
    if (e == cudaSuccess) {
        k_to_bf16<<<(unsigned)((net->nparam + 255) / 256), 256, 0, net->stream>>>(net->p, net->pb, net->nparam);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(net->status, 0, 4, net->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_set_params: ") + cudaGetErrorString(e));
    net->t = 0;
    net->pw_dirty = true;
    net->fault = LBIB_OK;
    return LBIB_OK;
}

lbib_status lbib_mlp_sync(lbib_mlp* net)
{
    if (!net) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    Guard guard(net->device);
    cudaError_t e = cudaStreamSynchronize(net->stream);
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_sync: ") + cudaGetErrorString(e));
    return mlp_check_status(net);
}

lbib_status lbib_mlp_inject_fault(lbib_mlp* net, int32_t kind)
{
    if (!net) return mlp_fail(LBIB_ERR_INVALID_ARG, "null argument");
    if (kind != LBIB_FAULT_WAIT_TIMEOUT) return mlp_fail(LBIB_ERR_INVALID_ARG, "unknown fault kind");
    Guard guard(net->device);
    // the bit the tensor-core kernels set when a bounded wait gives up, in stream order
    k_or_word<<<1, 1, 0, net->stream>>>(net->status, 1u);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(LBIB_ERR_CUDA, std::string("lbib_mlp_inject_fault: ") + cudaGetErrorString(e));
    return LBIB_OK;
}

void lbib_mlp_destroy(lbib_mlp* net)
{
    if (!net) return;
    Guard guard(net->device);
    if (net->stream) cudaStreamSynchronize(net->stream);
    for (void* p : net->allocs) cudaFree(p);
    if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
    cudaGetLastError();
    delete net;
}

}  // extern "C"
