// Dense BF16 contraction on the 5th-generation tensor cores (tcgen05) for
// the learned surrogate: C = A B^T with A (M x K) and B (N x K) row-major
// BF16, FP32 accumulation in tensor memory (TMEM), fused epilogue.
//
// Per CTA: one 128-row tile of C and all N <= 256 columns.  K is consumed in
// chunks of up to 64; each chunk of A and B is copied to shared memory with
// 16-byte cp.async in the tensor core's K-major layout without swizzle
// (8-row x 16-byte core matrices: [row group][k group][row][16 B]), double
// buffered, and contracted by one elected thread issuing tcgen05.mma
// (M = 128, N, K = 16) into a TMEM accumulator of N columns.  Completion of
// each chunk's MMAs is signalled through an mbarrier (tcgen05.commit); every
// wait gives up after one second, raising an error flag, and the CTA still
// releases its TMEM.  The epilogue reads the accumulator with tcgen05.ld
// (each warp its 32-lane quarter), adds a column bias and an optional
// row-scaled bias, stores the pre-activation, applies SiLU, adds a residual
// and writes FP32 and/or BF16 (or FP16) outputs, or adds into FP32 with
// atomics when K is split across CTAs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace umma {

constexpr int BM = 128;       // rows of a tile (MMA M)
constexpr int BK = 64;        // K of a staged chunk
constexpr int THREADS = 256;  // 8 warps: loads and epilogue (warps w and w+4 share a lane quarter)
constexpr unsigned ERR_TIMEOUT = 1u;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle:
// start address, leading-dimension byte offset (between core matrices
// adjacent in K), stride-dimension byte offset (between 8-row groups), the
// descriptor version bit of tcgen05 (bit 46); base offset, offset mode and
// swizzle mode 0.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A
// and B BF16 (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the completion of the mbarrier phase with the given parity; false
// after one second without it.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    if (mbar_try_wait(mbar, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (!mbar_try_wait(mbar, parity))
        if (now_ns() - t0 > 1000000000ull) return false;
    return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }

__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Arguments of one contraction C = A B^T (+ epilogue).
struct GemmArgs {
    const __nv_bfloat16 *A;
    int lda;                    // M x K, row-major, lda % 8 == 0
    const __nv_bfloat16 *B;
    int ldb;                    // N x K, row-major, ldb % 8 == 0
    int M, N, K;                // N in {16, 32, 64, 128, 256}; K % 16 == 0
    int k_split;                // K range of one CTA (multiple of 64); >= K: no split
    float *Cf;                  // FP32 output (or NULL)
    int ldcf;
    __nv_bfloat16 *Cb;          // BF16 output (or NULL)
    int ldcb;
    const float *bias;          // per column (or NULL)
    const float *row_scale;     // C[r][c] += row_scale[r] * row_bias[c] (or NULL)
    const float *row_bias;
    float *Z;                   // pre-activation output, FP32 (or NULL)
    int ldz;
    const float *residual;      // added after the activation (or NULL)
    int ldr;
    int act;                    // 0 none, 1 SiLU, 2 multiply by SiLU'(dact) (backward)
    const float *dact;          // pre-activation for act == 2
    int lddact;
    int atomic;                 // 1: atomicAdd the raw accumulator into Cf (split K)
    int n_store;                // columns stored (0: N)
    int cb_half;                // 1: Cb holds FP16 (__half) instead of BF16
    unsigned *err;              // error word (ERR_TIMEOUT)
};

// Copies chunk rows [row0, row0 + R) x k-groups [0, KG) of X (ld elements,
// columns k0...) into shared memory at dst in the core-matrix layout; rows at
// or beyond `rows` are zero-filled.
template <int R>
__device__ __forceinline__ void load_chunk(uint8_t *dst, const __nv_bfloat16 *X, int ld, int row0, int rows, int k0,
                                           int KG)
{
    const int pieces = R * KG;
    for (int p = threadIdx.x; p < pieces; p += THREADS) {
        const int r_lo = p & 7;
        const int kg = (p >> 3) % KG;
        const int rg = (p >> 3) / KG;
        const int row = row0 + rg * 8 + r_lo;
        const bool ok = row < rows;
        const __nv_bfloat16 *src = X + (size_t)(ok ? row : 0) * ld + k0 + kg * 8;
        cp_async16(dst + (size_t)p * 16, src, ok);
    }
}

__device__ __forceinline__ bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// 16 consecutive FP32 values: four 16-byte accesses when the chunk is whole
// and aligned, else element by element (the first `count` values).
__device__ __forceinline__ void store16(float *p, const float (&v)[16], bool full, int count)
{
    if (full && aligned16(p)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) ((float4 *)p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < count) p[j] = v[j];
    }
}

__device__ __forceinline__ void load16(const float *p, float (&v)[16], bool full, int count)
{
    if (full && aligned16(p)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t = ((const float4 *)p)[q];
            v[4 * q] = t.x;
            v[4 * q + 1] = t.y;
            v[4 * q + 2] = t.z;
            v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = j < count ? p[j] : 0.f;
    }
}

__device__ __forceinline__ void store16_half(__half *p, const float (&v)[16], bool full, int count)
{
    if (full && aligned16(p)) {
        uint4 w[2];
        uint32_t *u = (uint32_t *)w;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const __half2 b = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
            u[q] = *(const uint32_t *)&b;
        }
        ((uint4 *)p)[0] = w[0];
        ((uint4 *)p)[1] = w[1];
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < count) p[j] = __float2half_rn(v[j]);
    }
}

__device__ __forceinline__ void store16_bf16(__nv_bfloat16 *p, const float (&v)[16], bool full, int count)
{
    if (full && aligned16(p)) {
        uint4 w[2];
        uint32_t *u = (uint32_t *)w;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            u[q] = *(const uint32_t *)&b;
        }
        ((uint4 *)p)[0] = w[0];
        ((uint4 *)p)[1] = w[1];
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < count) p[j] = __float2bfloat16_rn(v[j]);
    }
}

template <int BN>
__global__ void __launch_bounds__(THREADS, 1) k_gemm(GemmArgs g)
{
    constexpr int NCOLS = BN < 32 ? 32 : BN;
    constexpr int A_BYTES = BM * BK * 2;
    constexpr int B_BYTES = BN * BK * 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // buffer b: A at smem + b * (A_BYTES + B_BYTES), B right after it
    auto bufA = [&](int b) { return smem + b * (A_BYTES + B_BYTES); };
    auto bufB = [&](int b) { return smem + b * (A_BYTES + B_BYTES) + A_BYTES; };
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * BM;
    const int k_begin = blockIdx.y * g.k_split;
    const int k_end = min(g.K, k_begin + g.k_split);
    const int nchunks = (k_end - k_begin + BK - 1) / BK;

    if (warp == 0) {
        tmem_alloc(&tmem_base, NCOLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    const uint32_t idesc = idesc_bf16(BM, BN);

    bool failed = false;
    if (nchunks > 0) {
        {
            const int kc = min(BK, k_end - k_begin);
            load_chunk<BM>(bufA(0), g.A, g.lda, row0, g.M, k_begin, kc / 8);
            load_chunk<BN>(bufB(0), g.B, g.ldb, 0, g.N, k_begin, kc / 8);
            cp_async_commit();
        }
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            if (c + 1 < nchunks) {
                // buffer b^1 held chunk c-1: its MMAs must be complete before it is overwritten
                if (c >= 1) failed |= !mbar_wait(&mbar[b ^ 1], ((c - 1) >> 1) & 1);
                if (__syncthreads_or(failed)) {
                    failed = true;
                    break;
                }
                const int k0 = k_begin + (c + 1) * BK;
                const int kc = min(BK, k_end - k0);
                load_chunk<BM>(bufA(b ^ 1), g.A, g.lda, row0, g.M, k0, kc / 8);
                load_chunk<BN>(bufB(b ^ 1), g.B, g.ldb, 0, g.N, k0, kc / 8);
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            fence_proxy_async();
            __syncthreads();
            if (threadIdx.x == 0) {
                tc_fence_after();
                const int k0 = k_begin + c * BK;
                const int kc = min(BK, k_end - k0);
                const int KG = kc / 8;
                const uint32_t a0 = smem_u32(bufA(b)), b0 = smem_u32(bufB(b));
                for (int kk = 0; kk < kc / 16; ++kk) {
                    const uint64_t ad = desc_kmajor(a0 + kk * 256, 128, KG * 128);
                    const uint64_t bd = desc_kmajor(b0 + kk * 256, 128, KG * 128);
                    mma_bf16(taddr, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&mbar[b]);
            }
        }
        if (!failed) {
            const int last = nchunks - 1;
            failed |= !mbar_wait(&mbar[last & 1], (last >> 1) & 1);
        }
        failed = __syncthreads_or(failed);
    }
    if (failed) {
        cp_async_wait<0>();
        if (threadIdx.x == 0) atomicOr(g.err, ERR_TIMEOUT);
    } else {
        tc_fence_after();
        const int quarter = warp & 3;
        const int half = warp >> 2;
        const int row = row0 + quarter * 32 + lane;
        constexpr int COLS_PER_HALF = BN >= 32 ? BN / 2 : BN;
        const bool active = BN >= 32 || half == 0;
        if (active) {
            for (int cc = 0; cc < COLS_PER_HALF; cc += 16) {
                const int c0 = half * COLS_PER_HALF + cc;
                float v[16];
                if (nchunks > 0) {
                    tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
                }
                if (row >= g.M) continue;
                const int nst = g.n_store > 0 ? g.n_store : BN;
                // whole 16-column chunks go through 16-byte vector accesses
                const bool full = c0 + 16 <= nst;
                if (g.atomic) {
                    float *dst = g.Cf + (size_t)row * g.ldcf + c0;
                    if (full && aligned16(dst)) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            atomicAdd((float4 *)dst + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < nst) atomicAdd(dst + j, v[j]);
                    }
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (g.bias) v[j] += g.bias[c0 + j];
                    if (g.row_scale) v[j] += g.row_scale[row] * g.row_bias[c0 + j];
                }
                if (g.Z) store16(g.Z + (size_t)row * g.ldz + c0, v, full, nst - c0);
                if (g.act == 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = silu(v[j]);
                } else if (g.act == 2) {
                    float a[16];
                    load16(g.dact + (size_t)row * g.lddact + c0, a, full, nst - c0);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] *= dsilu(a[j]);
                }
                if (g.residual) {
                    float r[16];
                    load16(g.residual + (size_t)row * g.ldr + c0, r, full, nst - c0);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += r[j];
                }
                if (g.Cf) store16(g.Cf + (size_t)row * g.ldcf + c0, v, full, nst - c0);
                if (g.Cb) {
                    if (g.cb_half) store16_half((__half *)g.Cb + (size_t)row * g.ldcb + c0, v, full, nst - c0);
                    else store16_bf16(g.Cb + (size_t)row * g.ldcb + c0, v, full, nst - c0);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, NCOLS);
}

inline size_t gemm_smem_bytes(int BN) { return 2 * (size_t)(BM * BK * 2 + BN * BK * 2) + 1024; }

// Launches C = A B^T (+ epilogue) on `stream`; returns a cudaError_t.
inline cudaError_t gemm(const GemmArgs &g, cudaStream_t stream)
{
    if (g.M <= 0) return cudaSuccess;
    if (g.K % 16 != 0 || g.lda % 8 != 0 || g.ldb % 8 != 0 || g.k_split % BK != 0 || g.k_split <= 0)
        return cudaErrorInvalidValue;
    const dim3 grid((g.M + BM - 1) / BM, (g.K + g.k_split - 1) / g.k_split);
    const size_t smem = gemm_smem_bytes(g.N);
    cudaError_t e = cudaSuccess;
    switch (g.N) {
#define SPH_GEMM_CASE(BN)                                                                                  \
    case BN:                                                                                              \
        e = cudaFuncSetAttribute(k_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
        if (e != cudaSuccess) return e;                                                                   \
        k_gemm<BN><<<grid, THREADS, smem, stream>>>(g);                                                   \
        break;
        SPH_GEMM_CASE(16)
        SPH_GEMM_CASE(32)
        SPH_GEMM_CASE(64)
        SPH_GEMM_CASE(128)
        SPH_GEMM_CASE(256)
#undef SPH_GEMM_CASE
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace umma
