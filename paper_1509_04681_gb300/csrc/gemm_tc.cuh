// Tensor-core contraction C = alpha A B^T + beta C (tcgen05, kind::tf32); see gemm_tc.cu.
#pragma once

#include "common.cuh"

namespace cggm {

// A: M x K, B: N x K, row-major float with row strides lda, ldb (multiples of 4 floats,
// 16-byte aligned bases); C: M x N row-major float (ldc).  With split, A_lo / B_lo (same
// layout) hold the low parts of A and B (see split_tf32) and A, B their TF32 high parts.
// err: device status word (DEV_TIMEOUT if a wait expired).  Returns CGGM_EINVAL for
// operands the tensor memory accessor cannot address.
cggm_status gemm_tc_nt(int64_t M, int64_t N, int64_t K, float alpha, const float *A, int64_t lda,
                       const float *B, int64_t ldb, float beta, float *C, int64_t ldc, bool split,
                       const float *A_lo, const float *B_lo, int *err, cudaStream_t st);

// hi = x truncated to TF32 (10 explicit mantissa bits), lo = x - hi, elementwise over a
// rows x ld array.
void split_tf32(int64_t rows, int64_t cols, int64_t ld, const float *x, float *hi, float *lo,
                cudaStream_t st);

bool tc_operand_ok(const void *ptr, int64_t ld);

}  // namespace cggm
