// Tensor-core contraction C = alpha A B^T + beta C on sm_103a (5th-generation tensor
// cores): A is M x K and B is N x K, both row-major float (K contiguous); C is M x N
// row-major float.  The products of the Newton iteration that are dense contractions from
// X (R = X Theta, P = R Sigma, Psi = P^T P / n, X^T (Y + P)) all take this form once their
// operands are laid out with the contracted index contiguous.
//
// One CTA computes a 128 x 128 tile of C.  Tiles of A and B (128 rows x 32 floats = 128 B,
// 128-byte swizzle) are brought to shared memory by TMA into a 4-stage (3 in split mode) ring guarded by
// mbarriers; one thread issues tcgen05.mma (kind::tf32, 128 x 128 x 8 per instruction)
// into an FP32 accumulator in tensor memory (128 lanes x 128 columns); after the last
// k-step a tcgen05.commit releases the 4-warp epilogue, which reads the accumulator with
// tcgen05.ld (32 lanes x 32 columns per instruction) and writes C.
//
// Split mode (3xTF32): A = A_hi + A_lo, B = B_hi + B_lo with A_hi the float truncated to
// the 19 bits a TF32 operand keeps; the product is accumulated as A_hi B_hi + A_hi B_lo +
// A_lo B_hi, which restores close to single-precision accuracy (the dropped A_lo B_lo term
// is below 2^-22 relative).
//
// Every wait on an mbarrier has a wall-clock deadline; a wait that expires records
// DEV_TIMEOUT, the CTA stops issuing work, waits (bounded) for the copies it has in flight,
// frees its tensor memory and returns.
#include <cuda.h>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "mbar.cuh"

namespace cggm {

namespace {

constexpr int TM = 128, TN = 128, TK = 32;  // TK floats = 128 B = one swizzle row
constexpr int STAGES_PLAIN = 4;  // 4 x 2 tiles x 16 KB = 128 KB of shared memory
constexpr int STAGES_SPLIT = 3;  // 3 x 4 tiles x 16 KB = 192 KB
constexpr int THREADS = 128;
constexpr int kGroupM = 8;     // tile rows per band of the launch order
constexpr int TILE_BYTES = TM * TK * 4;     // 16 KB (A tile; B tile is the same size)
constexpr uint64_t WAIT_NS = kMbarWaitNs;

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(mbar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout: rows of
// 128 B, groups of 8 rows 1024 B apart (stride byte offset), version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                    // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
    d |= (uint64_t)1 << 46;                    // descriptor version
    d |= (uint64_t)2 << 61;                    // 128-byte swizzle
    return d;
}

// Instruction descriptor: D f32, A and B tf32, both K-major, N = 128, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1)
gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapB2,
               int M, int N, int K, float alpha, float beta, float *C, int64_t ldc, int *err) {
    // operand tiles per stage: A_hi, B_hi (+ A_lo, B_lo in split mode), 1024-byte aligned
    constexpr int NT = SPLIT ? 4 : 2;
    constexpr int STAGES = SPLIT ? STAGES_SPLIT : STAGES_PLAIN;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[STAGES_PLAIN], empty[STAGES_PLAIN], done;
    __shared__ uint32_t s_tmem;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Tile order: CTAs that run at the same time (consecutive linear indices) take tiles from
    // a band of kGroupM tile rows, column by column, so that a wave reads kGroupM row blocks
    // of A and a few column blocks of B, which stay in L2, instead of every column block.
    int m0, n0;
    {
        const int gn = (int)gridDim.x, gm = (int)gridDim.y;
        const int lin = (int)(blockIdx.y * gridDim.x + blockIdx.x);
        const int per_group = kGroupM * gn;
        const int first_m = (lin / per_group) * kGroupM;
        const int rows = (gm - first_m) < kGroupM ? (gm - first_m) : kGroupM;
        const int in_group = lin % per_group;
        m0 = (first_m + in_group % rows) * TM;
        n0 = (in_group / rows) * TN;
    }
    const int nk = (K + TK - 1) / TK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        mbar_init_fence();
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mapB)) : "memory");
    }
    if (warp == 0) {  // tensor memory: 128 columns of 128 lanes (FP32 accumulator)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    int issued = 0;  // TMA stages issued (producer thread)
    if (warp == 0 && lane == 0) {
        // ---- producer: TMA loads into the ring ----
        for (int kt = 0; kt < nk; kt++) {
            const int s = kt % STAGES;
            if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) - 1) & 1, err)) break;
            unsigned char *st = smem + (size_t)s * NT * TILE_BYTES;
            mbar_expect_tx(&full[s], NT * TILE_BYTES);
            tma_load_2d(st, &mapA, kt * TK, m0, &full[s]);
            tma_load_2d(st + TILE_BYTES, &mapB, kt * TK, n0, &full[s]);
            if (SPLIT) {
                tma_load_2d(st + 2 * TILE_BYTES, &mapA2, kt * TK, m0, &full[s]);
                tma_load_2d(st + 3 * TILE_BYTES, &mapB2, kt * TK, n0, &full[s]);
            }
            issued = kt + 1;
        }
        // leave no copy in flight: wait (bounded) until every issued stage has landed
        for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; kt++) {
            const int s = kt % STAGES;
            if (!mbar_try(&full[s], (kt / STAGES) & 1)) {
                const uint64_t t0 = global_ns();
                while (!mbar_try(&full[s], (kt / STAGES) & 1))
                    if (global_ns() - t0 > WAIT_NS) break;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer ----
        bool ok = true;
        for (int kt = 0; kt < nk && ok; kt++) {
            const int s = kt % STAGES;
            if (!mbar_wait(&full[s], (kt / STAGES) & 1, err)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + (size_t)s * NT * TILE_BYTES);
            const uint32_t sb = sa + TILE_BYTES;
#pragma unroll
            for (int kk = 0; kk < TK / 8; kk++) {  // 8 tf32 = 32 B per instruction
                const uint64_t da = smem_desc_sw128(sa + kk * 32);
                const uint64_t db = smem_desc_sw128(sb + kk * 32);
                mma_tf32(tmem, da, db, (kt > 0 || kk > 0) ? 1u : 0u);
                if (SPLIT) {
                    const uint64_t da2 = smem_desc_sw128(sa + 2 * TILE_BYTES + kk * 32);
                    const uint64_t db2 = smem_desc_sw128(sb + 2 * TILE_BYTES + kk * 32);
                    mma_tf32(tmem, da, db2, 1u);   // A_hi B_lo
                    mma_tf32(tmem, da2, db, 1u);   // A_lo B_hi
                }
            }
            mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
        }
        mma_commit(&done);  // accumulator complete (or abandoned on error)
    }
    __syncwarp();

    // ---- epilogue: all four warps; warp w owns accumulator lanes (rows) 32w .. 32w+31 ----
    const bool good = mbar_wait(&done, 0, err) && (*(volatile int *)err == 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < TN; c0 += 32) {
        uint32_t r[32];
        tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        if (good && row < M) {
            float *crow = C + (int64_t)row * ldc + n0 + c0;
#pragma unroll
            for (int k = 0; k < 32; k++) {
                if (n0 + c0 + k < N) {
                    const float v = alpha * __uint_as_float(r[k]);
                    crow[k] = (beta == 0.0f) ? v : v + beta * crow[k];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                 const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                 const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map of a rows x K float matrix with row stride ld (floats), tiles of 128 x 32.
bool make_map(CUtensorMap *map, const float *ptr, int64_t rows, int64_t K, int64_t ld) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)TM};
    cuuint32_t estride[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), gdim,
                          gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

__global__ void split_tf32_kernel(int64_t rows, int64_t cols, int64_t ld, const float *x,
                                  float *hi, float *lo) {
    const int64_t len = rows * ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[e];
        const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);  // keep 10 mantissa bits
        hi[e] = h;
        lo[e] = v - h;
    }
}

}  // namespace

bool tc_operand_ok(const void *ptr, int64_t ld) {
    return ptr && (reinterpret_cast<uintptr_t>(ptr) % 16 == 0) && (ld % 4 == 0) && ld > 0;
}

cggm_status gemm_tc_nt(int64_t M, int64_t N, int64_t K, float alpha, const float *A, int64_t lda,
                       const float *B, int64_t ldb, float beta, float *C, int64_t ldc, bool split,
                       const float *A_lo, const float *B_lo, int *err, cudaStream_t st) {
    if (M <= 0 || N <= 0) return CGGM_OK;
    if (K <= 0 || M > 2147483647LL || N > 2147483647LL || K > 2147483647LL) return CGGM_EINVAL;
    if (!tc_operand_ok(A, lda) || !tc_operand_ok(B, ldb)) return CGGM_EINVAL;
    if (split && (!tc_operand_ok(A_lo, lda) || !tc_operand_ok(B_lo, ldb))) return CGGM_EINVAL;
    CUtensorMap ma, mb, ma2, mb2;
    if (!make_map(&ma, A, M, K, lda) || !make_map(&mb, B, N, K, ldb)) return CGGM_ECUDA;
    if (split) {
        if (!make_map(&ma2, A_lo, M, K, lda) || !make_map(&mb2, B_lo, N, K, ldb)) return CGGM_ECUDA;
    } else {
        ma2 = ma;
        mb2 = mb;
    }
    const int NT = split ? 4 : 2;
    const size_t smem = (size_t)(split ? STAGES_SPLIT : STAGES_PLAIN) * NT * TILE_BYTES + 1024;
    dim3 grid((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM));
    if (split) {
        CGGM_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        note_launch();
        gemm_tc_kernel<true><<<grid, THREADS, smem, st>>>(ma, mb, ma2, mb2, (int)M, (int)N, (int)K,
                                                          alpha, beta, C, ldc, err);
    } else {
        CGGM_CUDA_TRY(cudaFuncSetAttribute(gemm_tc_kernel<false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        note_launch();
        gemm_tc_kernel<false><<<grid, THREADS, smem, st>>>(ma, mb, ma2, mb2, (int)M, (int)N, (int)K,
                                                           alpha, beta, C, ldc, err);
    }
    CGGM_CUDA_TRY(cudaGetLastError());
    return CGGM_OK;
}

void split_tf32(int64_t rows, int64_t cols, int64_t ld, const float *x, float *hi, float *lo,
                cudaStream_t st) {
    const int64_t len = rows * ld;
    if (len <= 0) return;
    int64_t g = (len + 255) / 256, cap = (int64_t)sm_count() * 16;
    note_launch();
    split_tf32_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, st>>>(rows, cols, ld, x, hi, lo);
}

}  // namespace cggm
