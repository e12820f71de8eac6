/*
 * Test hooks of libgf2.  These have no counterpart in the paper: they expose
 * single building blocks of the tensor-core path so that tests can check the
 * operand layouts in isolation.  Not part of the GF2 API proper.
 */
#ifndef GF2_TESTING_H
#define GF2_TESTING_H

#include "gf2.h"

#ifdef __cplusplus
extern "C" {
#endif

/* One 128 x 64 x 64 BF16 tile D = A B^T through TMA loads (128-byte swizzle),
 * four tcgen05.mma (K = 16 each, FP32 accumulation in TMEM) and tcgen05.ld.
 *   d_A: bf16, [128][64] row-major (M x K) if a_mn_major == 0,
 *        [64][128] row-major (K x M) if a_mn_major == 1,
 *        [128][64] row-major (M x K) written to TMEM by the threads and used as
 *        the TMEM-resident A operand if a_mn_major == 2;
 *   d_B: bf16 [64][64] row-major (N x K);
 *   d_D: fp32 [128][64] row-major output;  d_err: device int, set non-zero
 *        if a pipeline wait timed out.
 * Device pointers owned by the caller; synchronizes `stream`.
 * GF2_ERR_ARG for NULL pointers or a_mn_major outside 0..2, GF2_ERR_UNSUPPORTED
 * without tensor maps. */
gf2_status gf2_test_umma_tile(int a_mn_major, const void *d_A, const void *d_B, float *d_D, int *d_err,
                              void *stream);

/* Failure detection without a fault: one thread waits on an mbarrier that
 * nothing arrives at, through the same bounded wait the tensor-core pipelines
 * use.  After the wait limit (2 s of GPU wall time) it gives up, sets *d_err to
 * the timeout code 1, and the kernel returns normally, leaving the CUDA context
 * usable.  Synchronizes `stream`; GF2_ERR_ARG for a NULL d_err, GF2_ERR_CUDA if
 * the launch fails. */
gf2_status gf2_test_wait_timeout(int *d_err, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GF2_TESTING_H */
