/*
 * sph_surrogate.h -- C ABI of the learned k-step surrogate and of its dense
 * BF16 contraction on the tensor cores.
 *
 * The paper has no learned component; this library adds one: a
 * message-passing network over the SPH neighbour graph that advances the
 * particle state by k plain steps at once, trained on trajectories of the
 * plain method, with the plain method as its fallback and judge.  Return
 * values and error messages follow sph.h (SPH_OK or a negative SPH_E* code,
 * message from sph_last_error()).
 */
#ifndef SPH_SURROGATE_H
#define SPH_SURROGATE_H

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Dense contraction C = A B^T on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation).  A: M x K BF16, row-major with leading dimension lda;
 * B: N x K BF16, row-major, ldb; C: M x N FP32, row-major, ldc.  All three are
 * device pointers owned by the caller; A and B 16-byte aligned, lda and ldb
 * multiples of 8.  N in {16, 32, 64, 128, 256}; K a multiple of 16.  With
 * accumulate = 0, C is overwritten; with accumulate = 1, the products are
 * added to C with atomics, and K may be split across CTAs in ranges of
 * k_split (a multiple of 64; 0 = no split).  The call only queues the work on
 * `stream`; a tensor-core wait that exceeded one second sets bit 0 of the
 * device word *err_dev, which the caller reads. */
int sph_mm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K,
                int k_split, int accumulate, void *stream, unsigned *err_dev);

#ifdef __cplusplus
}
#endif

#endif /* SPH_SURROGATE_H */
