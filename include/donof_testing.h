/*
 * donof_testing.h -- test hooks of libdonof (not needed to use the library).
 *
 * They expose the tensor-core building block of the mixed-precision build so that its
 * arithmetic can be checked in isolation against exact products on the host, and the
 * bounded device wait so that its time-out path can be exercised.  The paper has no
 * counterpart; these hooks exist for verification only.
 */
#ifndef DONOF_TESTING_H
#define DONOF_TESTING_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* D[m*N + n] = sum_k A_hi[m][k] B_hi[n][k] + A_hi[m][k] B_lo[n][k] + A_lo[m][k] B_hi[n][k]
 * on the tensor cores (fp16 operands given as raw IEEE half bits, fp32 accumulation).
 * All pointers are device pointers; A_* are [M][K], B_* are [N][K] (row-major, K
 * contiguous), D is [M][N] fp32.  K must be a multiple of 8; N a multiple of 16 in
 * [16, 256]; M >= 1.  Returns DONOF_OK or a DONOF_ERR_* code; the call is asynchronous on
 * `stream` and device wait time-outs are reported by the return of the next call's
 * status word (see donof_testing_status). */
int donof_testing_tc_gemm(const uint16_t* A_hi, const uint16_t* A_lo, const uint16_t* B_hi,
                          const uint16_t* B_lo, float* D, int32_t M, int32_t N, int32_t K,
                          void* stream);

/* The same product with A given MN-major, A_*[K][M] (M contiguous), loaded as two 64-wide
 * M boxes per 64-deep K step and read through MN-major shared-memory descriptors (leading
 * byte offset = the distance between the 64-wide M chunks, stride byte offset = the
 * distance between groups of 8 K rows, 128-byte swizzle).  M must be a multiple of 64. */
int donof_testing_tc_gemm_mn(const uint16_t* A_hi, const uint16_t* A_lo, const uint16_t* B_hi,
                             const uint16_t* B_lo, float* D, int32_t M, int32_t N, int32_t K,
                             void* stream);

/* The same product with A interleaved by 8 along K, A_*[K/8][M][8] (element (m, k) at
 * ((k / 8) * M + m) * 8 + k % 8), loaded without swizzle as 8-row x 16-byte core matrices.
 * K and M must be multiples of 8. */
int donof_testing_tc_gemm_il8(const uint16_t* A_hi, const uint16_t* A_lo, const uint16_t* B_hi,
                              const uint16_t* B_lo, float* D, int32_t M, int32_t N, int32_t K,
                              void* stream);

/* Any of the three A layouts above (layout 0: K-major, 1: MN-major, 2: interleaved by 8;
 * the same constraints), on one SM per 128-row tile (pair = 0) or with the 256-row tiles of
 * a CTA pair (pair = 1: a cluster of two CTAs, cta_group::2 MMAs issued by the even CTA, each
 * CTA staging its 128 rows of A and half of the N rows of B). */
int donof_testing_tc_gemm_ex(const uint16_t* A_hi, const uint16_t* A_lo, const uint16_t* B_hi,
                             const uint16_t* B_lo, float* D, int32_t M, int32_t N, int32_t K,
                             int32_t layout, int32_t pair, void* stream);

/* The bounded device wait of the tensor-core kernel, run out on purpose: one CTA whose two
 * roles wait on mbarriers that nothing completes, the first with a limit of limit_a_ns
 * (at most 2 s), the second with limit_b_ns (at most 20 s).  The first wait's time-out
 * sets the status word to DONOF_ERR_TIMEOUT and raises the abort flag, which must end the
 * second wait well before its own limit; the kernel then returns normally and the context
 * stays usable.  Read the outcome with donof_testing_status. */
int donof_testing_wait_timeout(int64_t limit_a_ns, int64_t limit_b_ns, void* stream);

/* Synchronises `stream` and returns (then clears) the status word of the test hooks. */
int donof_testing_status(void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DONOF_TESTING_H */
