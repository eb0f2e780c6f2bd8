// Dense BF16 contraction on the 5th-generation tensor cores (tcgen05) for
// the learned surrogate: C = A B^T with A (M x K) and B (N x K) row-major
// BF16, FP32 accumulation in tensor memory (TMEM), fused epilogue.
//
// Per CTA: one 128-row tile of C and all N <= 256 columns.  K is consumed in
// chunks of up to 64; each chunk of A and B is brought to shared memory by the
// tensor memory accelerator (cp.async.bulk.tensor, one 2-D box of rows x 8
// elements per 8-wide k group) in the tensor core's K-major layout without
// swizzle ([k group][row][16 B]: core matrices of 8 rows x 16 bytes, 128 B
// apart along M and rows x 16 B apart along K), double buffered, and contracted by one thread issuing tcgen05.mma (M = 128, N,
// K = 16) into a TMEM accumulator of N columns.  The same thread issues the
// copies: a chunk's arrival and the completion of its MMAs (tcgen05.commit)
// are each signalled through an mbarrier; every wait gives up after one
// second, raising an error flag, and the CTA waits (again bounded) for its
// copies in flight and still releases its TMEM.  The epilogue reads the accumulator with tcgen05.ld
// (each warp its 32-lane quarter), adds a column bias and an optional
// row-scaled bias, stores the pre-activation, applies SiLU, adds a residual
// and writes FP32 and/or BF16 (or FP16) outputs, or adds into FP32 with
// atomics when K is split across CTAs.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

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

// Expects `bytes` more transaction bytes on the mbarrier and arrives once.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// 2-D tensor copy global -> shared of the box at (x, y) = (k, row) of the
// tensor map; completion counted in bytes on the mbarrier.  x is a multiple
// of 8 elements (16 bytes) and dst 128-byte aligned.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}

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

// Issues the copies of K chunk [k0, k0 + kc) of A (rows row0...) and B into
// one buffer pair: kc / 8 boxes each, [k group][row][16 B].
template <int BN>
__device__ __forceinline__ void tma_chunk(uint8_t *a, uint8_t *b, const CUtensorMap *mA, const CUtensorMap *mB,
                                          int row0, int k0, int kc, uint64_t *bar)
{
    const int KG = kc / 8;
    mbar_arrive_expect_tx(bar, (uint32_t)(KG * (BM + BN) * 16));
    for (int kg = 0; kg < KG; ++kg) {
        tma_load_2d(a + kg * BM * 16, mA, k0 + kg * 8, row0, bar);
        tma_load_2d(b + kg * BN * 16, mB, k0 + kg * 8, 0, bar);
    }
}

template <int BN>
__global__ void __launch_bounds__(THREADS, 1)
    k_gemm(const __grid_constant__ GemmArgs g, const __grid_constant__ CUtensorMap mapA,
           const __grid_constant__ CUtensorMap mapB)
{
    constexpr int NCOLS = BN < 32 ? 32 : BN;
    constexpr int A_BYTES = BM * BK * 2;
    constexpr int B_BYTES = BN * BK * 2;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // buffer b: A at smem + b * (A_BYTES + B_BYTES), B right after it
    auto bufA = [&](int b) { return smem + b * (A_BYTES + B_BYTES); };
    auto bufB = [&](int b) { return smem + b * (A_BYTES + B_BYTES) + A_BYTES; };
    __shared__ __align__(8) uint64_t mbar[2];   // MMAs of the chunk in buffer b complete
    __shared__ __align__(8) uint64_t lbar[2];   // copies into buffer b complete
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
        mbar_init(&lbar[0], 1);
        mbar_init(&lbar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = tmem_base;
    const uint32_t idesc = idesc_bf16(BM, BN);

    bool failed = false;
    if (nchunks > 0) {
        if (threadIdx.x == 0) {
            // copies issued into each buffer (their arrivals are waited on by
            // phase parity (uses - 1) & 1)
            int issued[2] = {0, 0}, landed[2] = {0, 0};
            int committed = -1;  // last chunk whose MMAs were committed
            tma_chunk<BN>(bufA(0), bufB(0), &mapA, &mapB, row0, k_begin, min(BK, k_end - k_begin), &lbar[0]);
            issued[0] = 1;
            for (int c = 0; c < nchunks; ++c) {
                const int b = c & 1;
                if (c + 1 < nchunks) {
                    // buffer b^1 held chunk c-1: its MMAs must be complete before it is overwritten
                    if (c >= 1 && !mbar_wait(&mbar[b ^ 1], ((c - 1) >> 1) & 1)) {
                        failed = true;
                        break;
                    }
                    const int k0 = k_begin + (c + 1) * BK;
                    tma_chunk<BN>(bufA(b ^ 1), bufB(b ^ 1), &mapA, &mapB, row0, k0, min(BK, k_end - k0), &lbar[b ^ 1]);
                    issued[b ^ 1] += 1;
                }
                if (!mbar_wait(&lbar[b], (c >> 1) & 1)) {
                    failed = true;
                    break;
                }
                landed[b] += 1;
                tc_fence_after();
                const int k0 = k_begin + c * BK;
                const int kc = min(BK, k_end - k0);
                const uint32_t a0 = smem_u32(bufA(b)), b0 = smem_u32(bufB(b));
                for (int kk = 0; kk < kc / 16; ++kk) {
                    const uint64_t ad = desc_kmajor(a0 + kk * 2 * BM * 16, BM * 16, 128);
                    const uint64_t bd = desc_kmajor(b0 + kk * 2 * BN * 16, BN * 16, 128);
                    mma_bf16(taddr, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&mbar[b]);
                committed = c;
            }
            if (failed) {
                // copies still in flight write this CTA's shared memory and
                // MMAs in flight its TMEM: wait for them (bounded) before the
                // CTA releases either (the last commit covers every MMA)
                for (int bb = 0; bb < 2; ++bb)
                    for (int u = landed[bb]; u < issued[bb]; ++u) mbar_wait(&lbar[bb], u & 1);
                if (committed >= 0) mbar_wait(&mbar[committed & 1], (committed >> 1) & 1);
            }
        }
        if (!__syncthreads_or(failed)) {
            const int last = nchunks - 1;
            failed = !mbar_wait(&mbar[last & 1], (last >> 1) & 1);
        }
        failed = __syncthreads_or(failed);
    }
    if (failed) {
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

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime.
inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// Tensor map of a row-major BF16 matrix (rows x cols, ld elements between
// rows) read in boxes of box_rows rows x 8 elements; rows beyond `rows` and
// columns beyond `cols` read as zero.  False when the base is not 16-byte
// aligned, ld not a multiple of 8, or the driver refuses the map.
inline bool make_map(CUtensorMap *m, const __nv_bfloat16 *base, int rows, int cols, int ld, int box_rows)
{
    const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
    if (!fn || ((uintptr_t)base & 15u) || ld % 8 != 0 || rows <= 0 || cols <= 0) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {8, (cuuint32_t)box_rows};
    const cuuint32_t step[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box, step,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Launches C = A B^T (+ epilogue) on `stream`; returns a cudaError_t.
inline cudaError_t gemm(const GemmArgs &g, cudaStream_t stream)
{
    if (g.M <= 0) return cudaSuccess;
    if (g.K % 16 != 0 || g.lda % 8 != 0 || g.ldb % 8 != 0 || g.k_split % BK != 0 || g.k_split <= 0)
        return cudaErrorInvalidValue;
    const dim3 grid((g.M + BM - 1) / BM, (g.K + g.k_split - 1) / g.k_split);
    const size_t smem = gemm_smem_bytes(g.N);
    CUtensorMap mapA{}, mapB{};
    if (g.K > 0 && (!make_map(&mapA, g.A, g.M, g.K, g.lda, BM) || !make_map(&mapB, g.B, g.N, g.K, g.ldb, g.N)))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    switch (g.N) {
#define SPH_GEMM_CASE(BN)                                                                                  \
    case BN:                                                                                              \
        e = cudaFuncSetAttribute(k_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
        if (e != cudaSuccess) return e;                                                                   \
        k_gemm<BN><<<grid, THREADS, smem, stream>>>(g, mapA, mapB);                                       \
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
