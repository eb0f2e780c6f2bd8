// Learned k-step surrogate of the particle loop: a message-passing network
// over the SPH neighbour graph (edges |r_ij| < 2h), BF16 operands on the
// tensor cores (umma.cuh) with FP32 accumulation, hand-written forward and
// backward kernels, Adam, and the C ABI declared in include/sph_surrogate.h.
#include "sph_surrogate.h"
#include "sph_kernels.cuh"
#include "umma.cuh"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

namespace sphgb {
int set_error(int code, const std::string &msg);
}

extern "C" int sph_mm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K,
                           int k_split, int accumulate, void *stream, unsigned *err_dev)
{
    if (!A || !B || !C || !err_dev) return sphgb::set_error(SPH_EINVAL, "NULL argument");
    if (M < 0 || K < 0 || (N != 16 && N != 32 && N != 64 && N != 128 && N != 256))
        return sphgb::set_error(SPH_EINVAL, "N must be 16, 32, 64, 128 or 256 and M, K >= 0");
    if (K % 16 != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K || ldc < N)
        return sphgb::set_error(SPH_EINVAL, "K must be a multiple of 16, lda and ldb multiples of 8 and >= K");
    if (k_split <= 0) k_split = ((K + umma::BK - 1) / umma::BK) * umma::BK;
    if (k_split % umma::BK != 0) return sphgb::set_error(SPH_EINVAL, "k_split must be a multiple of 64");
    if (K > k_split && !accumulate) return sphgb::set_error(SPH_EINVAL, "a split K needs accumulate");
    if ((uintptr_t)A % 16 || (uintptr_t)B % 16) return sphgb::set_error(SPH_EINVAL, "A and B must be 16-byte aligned");
    umma::GemmArgs g{};
    g.A = (const __nv_bfloat16 *)A;
    g.lda = lda;
    g.B = (const __nv_bfloat16 *)B;
    g.ldb = ldb;
    g.M = M;
    g.N = N;
    g.K = K;
    g.k_split = k_split;
    g.Cf = C;
    g.ldcf = ldc;
    g.atomic = accumulate ? 1 : 0;
    g.err = err_dev;
    cudaError_t e = umma::gemm(g, (cudaStream_t)stream);
    if (e != cudaSuccess) return sphgb::set_error(SPH_ECUDA, std::string("gemm launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}
