// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (sm_103a):
// tcgen05.mma with the accumulator in tensor memory (TMEM), operands staged
// in shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle) through a
// 4-stage mbarrier pipeline.  Used for the dense input and recurrent
// projections of the differentiable HH layer and their weight gradients
// (the current into the HH neurons is produced by the preceding layer's
// parameters, Methods "Analysis of C_m").
//
// C_s[m][n] = sum_{k in split s} A[a_row0 + m][k] * Bt[b_row0 + n][k]
//   A  : bf16, row-major [rows][lda], K contiguous (K-major)
//   Bt : bf16, row-major [rows][ldb], K contiguous (the transpose of B)
//   C  : fp32, [splits][M][N] (one partial product per K split; the reader
//        sums the splits, so the result does not depend on timing)
// One CTA computes a 128 x 256 tile of one split with 4 warps: warp 0 lane 0
// issues TMA loads, warp 1 lane 0 issues the MMAs (M=128, N=256, K=16 per
// instruction), all four warps drain TMEM (tcgen05.ld 32x32b) to global
// memory.  Every mbarrier wait is bounded: on expiry the CTA records the
// failure in *err and leaves through the common teardown, which frees TMEM.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "hh_internal.h"
#include "hh_tc.cuh"

namespace hh {
namespace {

using namespace tc;

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 4;
constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = kBN * kBK * 2;
constexpr uint32_t kStageBytes = kBytesA + kBytesB;
constexpr uint32_t kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kIdesc = idesc_bf16(kBM, kBN);

__global__ void __launch_bounds__(128, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            float* __restrict__ C, int M, int N, int k_blocks, int kb_per_split, int a_row0,
            int b_row0, int32_t* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * kBN, m0 = blockIdx.y * kBM;
    const int split = blockIdx.z;
    const int kb0 = split * kb_per_split;
    const int kb1 = min(k_blocks, kb0 + kb_per_split);
    const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (nkb > 0) {
        if (warp == 0 && lane == 0) {
            // TMA producer
            for (int i = 0; i < nkb; ++i) {
                const int s = i % kStages;
                const uint32_t ph = (uint32_t)(i / kStages) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, err, 1))
                    break;
                uint8_t* sa = smem + s * kStageBytes;
                uint8_t* sb = sa + kBytesA;
                mbar_expect_tx(&full[s], kStageBytes);
                const int kx = (kb0 + i) * kBK;
                tma_load_2d(sa, &mapA, kx, a_row0 + m0, &full[s]);
                tma_load_2d(sb, &mapB, kx, b_row0 + n0, &full[s]);
                ++issued;
            }
        } else if (warp == 1 && lane == 0) {
            // MMA issuer
            bool ok = true;
            for (int i = 0; i < nkb; ++i) {
                const int s = i % kStages;
                const uint32_t ph = (uint32_t)(i / kStages) & 1u;
                if (!mbar_wait(&full[s], ph, err, 2)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_u32(smem + s * kStageBytes);
                const uint32_t sb = sa + kBytesA;
                const uint64_t da = sdesc(sa), db = sdesc(sb);
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)  // 16 bf16 = 32 bytes = 2 descriptor units
                    mma_bf16(tmem, da + 2 * k, db + 2 * k, kIdesc, (i > 0 || k > 0) ? 1u : 0u);
                mma_commit(&empty[s]);
            }
            if (ok)
                mma_commit(done);
            else
                mbar_expect_tx(done, 0);  // release the epilogue; the result is flagged bad
        }
        __syncwarp();
        // epilogue: wait for the accumulator
        mbar_wait(done, 0, err, 4);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    const int row = m0 + warp * 32 + lane;
    float* crow = C + ((size_t)split * M + (size_t)(row < M ? row : 0)) * N;
#pragma unroll 1
    for (int c = 0; c < kBN; c += 32) {
        float v[32];
        if (nkb > 0) {
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                v[j] = 0.0f;
        }
        const int col = n0 + c;
        if (row < M && col < N) {
            float4* dst = reinterpret_cast<float4*>(crow + col);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
    }
    // no TMA copy may still be landing in shared memory when the CTA exits:
    // the producer waits (bounded) for the last phase of every stage it used
    if (warp == 0 && lane == 0) {
        for (int i = issued - 1; i >= 0 && i >= issued - kStages; --i)
            mbar_wait(&full[i % kStages], (uint32_t)(i / kStages) & 1u, err, 8);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

bool make_map(CUtensorMap* map, const void* base, int rows, int cols, int ld, int box_rows)
{
    EncodeTiled enc = encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

const char* gemm_check(const GemmArgs& g)
{
    if (g.M < 1 || g.N < 32 || g.K < 1 || g.splits < 1)
        return "GEMM sizes must be M >= 1, N >= 32, K >= 1, splits >= 1";
    if (g.N % 32 != 0)
        return "GEMM N must be a multiple of 32";
    if (g.lda % 8 != 0 || g.ldb % 8 != 0 || g.lda < g.K || g.ldb < g.K)
        return "GEMM leading dimensions must be >= K and multiples of 8 elements (16 bytes)";
    if ((reinterpret_cast<uintptr_t>(g.A) & 15) || (reinterpret_cast<uintptr_t>(g.Bt) & 15) ||
        (reinterpret_cast<uintptr_t>(g.C) & 15))
        return "GEMM operands must be 16-byte aligned";
    if (g.a_row0 < 0 || g.b_row0 < 0)
        return "GEMM row offsets must be >= 0";
    return nullptr;
}

cudaError_t launch_gemm_bf16(const GemmArgs& g, int32_t* err, cudaStream_t st)
{
    CUtensorMap ma, mb;
    if (!make_map(&ma, g.A, g.a_rows, g.K, g.lda, kBM) || !make_map(&mb, g.Bt, g.b_rows, g.K, g.ldb, kBN))
        return cudaErrorInvalidValue;
    static std::once_flag attr;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr, [] {
        attr_err = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    });
    if (attr_err != cudaSuccess)
        return attr_err;
    const int k_blocks = (g.K + kBK - 1) / kBK;
    const int per = (k_blocks + g.splits - 1) / g.splits;
    const dim3 grid((unsigned)((g.N + kBN - 1) / kBN), (unsigned)((g.M + kBM - 1) / kBM), (unsigned)g.splits);
    k_gemm_bf16<<<grid, 128, kSmemBytes, st>>>(ma, mb, g.C, g.M, g.N, k_blocks, per, g.a_row0, g.b_row0, err);
    return cudaGetLastError();
}

}  // namespace hh
