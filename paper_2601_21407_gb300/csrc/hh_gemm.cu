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
//
// Persistent and warp-specialised: one CTA per SM walks the 128 x 256 tiles
// of all splits (tile index n-fastest, stride gridDim.x).  Warp 0 lane 0
// issues the TMA loads, warp 1 lane 0 the MMAs (M=128, N=256, K=16 per
// instruction) into one of two 256-column TMEM accumulators, and warps 2-5
// drain the other accumulator meanwhile: tcgen05.ld (each warp its 32-lane
// quarter of TMEM), a 128-byte-swizzled 32 x 32 staging box in shared memory
// per warp (double-buffered), and a TMA store into the 3-D [splits][M][N]
// view of C, which drops the rows past M of the last tile of a split.  So one
// tile's epilogue overlaps the next tile's main loop and C is written as
// whole lines.  Every mbarrier wait is bounded: on expiry the thread records
// the failure in *err and its role stops, the others stop at their own
// bounded waits, and the common teardown waits for the copies in flight and
// frees TMEM.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda.h>

#include "hh_internal.h"
#include "hh_tc.cuh"

namespace hh {
namespace {

using namespace tc;
static_assert(kWaitLimit == kWaitLimitPolls, "one default bound of the mbarrier waits");

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 4;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = kBN * kBK * 2;
constexpr uint32_t kStageBytes = kBytesA + kBytesB;
constexpr uint32_t kEpiBoxBytes = 32 * 32 * 4;                 // 32 rows x 32 fp32 columns
constexpr uint32_t kEpiBytes = kEpiWarps * 2 * kEpiBoxBytes;   // double-buffered per warp
constexpr uint32_t kSmemBytes = kStages * kStageBytes + kEpiBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr uint32_t kTmemCols = 2 * kBN;                        // two accumulators
constexpr uint32_t kIdesc = idesc_bf16(kBM, kBN);

struct TileGrid {
    int M, N;
    int tiles_n, tiles_m, splits;
    int k_blocks, kb_per_split;
    int a_row0, b_row0;
    long long polls;  // limit of the pipeline's mbarrier waits
};

__device__ __forceinline__ void tile_of(const TileGrid& g, int tile, int& m0, int& n0, int& split, int& kb0,
                                        int& nkb)
{
    const int nt = tile % g.tiles_n;
    const int rest = tile / g.tiles_n;
    m0 = (rest % g.tiles_m) * kBM;
    n0 = nt * kBN;
    split = rest / g.tiles_m;
    kb0 = split * g.kb_per_split;
    const int kb1 = min(g.k_blocks, kb0 + g.kb_per_split);
    nkb = kb1 > kb0 ? kb1 - kb0 : 0;
}

__global__ void __launch_bounds__(kThreads, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
            const __grid_constant__ CUtensorMap mapC, const __grid_constant__ TileGrid g, int32_t* err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* epi = smem + kStages * kStageBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(epi + kEpiBytes);
    uint64_t* empty = full + kStages;
    uint64_t* tfull = empty + kStages;  // [2] accumulator ready for the epilogue
    uint64_t* tempty = tfull + 2;       // [2] accumulator drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = g.tiles_n * g.tiles_m * g.splits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], kEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0)
        tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    uint32_t issued = 0;  // TMA stage loads issued by the producer (for the drain)
    if (warp == 0) {
        if (lane == 0) {
            bool ok = true;
            for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
                int m0, n0, split, kb0, nkb;
                tile_of(g, tile, m0, n0, split, kb0, nkb);
                for (int i = 0; i < nkb; ++i) {
                    const int s = issued % kStages;
                    const uint32_t ph = (issued / kStages) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, err, 1, g.polls)) {
                        ok = false;
                        break;
                    }
                    uint8_t* sa = smem + s * kStageBytes;
                    mbar_expect_tx(&full[s], kStageBytes);
                    const int kx = (kb0 + i) * kBK;
                    tma_load_2d(sa, &mapA, kx, g.a_row0 + m0, &full[s]);
                    tma_load_2d(sa + kBytesA, &mapB, kx, g.b_row0 + n0, &full[s]);
                    ++issued;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t used = 0;  // stage loads consumed
            int it = 0;
            for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
                const int acc = it & 1;
                const uint32_t aph = (uint32_t)(it >> 1) & 1u;
                if (!mbar_wait(&tempty[acc], aph ^ 1u, err, 2, g.polls))
                    break;
                tc_fence_after();
                int m0, n0, split, kb0, nkb;
                tile_of(g, tile, m0, n0, split, kb0, nkb);
                const uint32_t d = tmem + (uint32_t)(acc * kBN);
                bool ok = true;
                for (int i = 0; i < nkb; ++i) {
                    const int s = used % kStages;
                    const uint32_t ph = (used / kStages) & 1u;
                    if (!mbar_wait(&full[s], ph, err, 4, g.polls)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * kStageBytes);
                    const uint64_t da = sdesc(sa), db = sdesc(sa + kBytesA);
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)  // 16 bf16 = 32 bytes = 2 descriptor units
                        mma_bf16(d, da + 2 * k, db + 2 * k, kIdesc, (i > 0 || k > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                    ++used;
                }
                if (!ok)
                    break;
                if (nkb > 0)
                    mma_commit(&tfull[acc]);
                else
                    mbar_arrive(&tfull[acc]);  // empty K range: the epilogue writes zeros
            }
        }
    } else {
        // epilogue: this warp reads TMEM lanes 32q..32q+31 (= tile rows)
        const int q = warp & 3;
        uint32_t box = 0;
        int it = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
            const int acc = it & 1;
            const uint32_t aph = (uint32_t)(it >> 1) & 1u;
            int got = 1;
            if (lane == 0)
                got = mbar_wait(&tfull[acc], aph, err, 8, g.polls) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, got, 0))
                break;
            tc_fence_after();
            int m0, n0, split, kb0, nkb;
            tile_of(g, tile, m0, n0, split, kb0, nkb);
            for (int c = 0; c < kBN && n0 + c < g.N; c += 32, ++box) {
                float v[32];
                if (nkb > 0) {
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kBN + c), v);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        v[j] = 0.0f;
                }
                uint8_t* buf = epi + (q * 2 + (box & 1)) * kEpiBoxBytes;
                if (lane == 0)
                    bulk_wait_read1();  // the store issued from this buffer two boxes ago has read it
                __syncwarp();
                // row `lane`, 16-byte piece j at piece j ^ (lane & 7): the
                // 128-byte swizzle of the store's tensor map
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    *reinterpret_cast<float4*>(buf + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                fence_async_smem();
                __syncwarp();
                if (lane == 0) {
                    tma_store_3d(buf, &mapC, n0 + c, m0 + 32 * q, split);
                    bulk_commit();
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&tempty[acc]);
        }
        if (lane == 0)
            bulk_wait_all();
        __syncwarp();
    }
    // no TMA load may still be landing in shared memory when the CTA exits:
    // the producer waits (bounded by the default limit, whatever the
    // pipeline's) for the last phase of every stage it used
    if (warp == 0 && lane == 0) {
        for (int i = (int)issued - 1; i >= 0 && i >= (int)issued - kStages; --i)
            mbar_wait(&full[i % kStages], (uint32_t)(i / kStages) & 1u, err, 16);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tmem_dealloc(tmem, kTmemCols);
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

// C as [splits][M][N] fp32 for the epilogue's TMA stores: 32 x 32 boxes with
// the 128-byte swizzle (a box row is 32 floats = 128 bytes); rows past M of
// a split fall outside the tensor and are not written.
bool make_map_c(CUtensorMap* map, void* base, int M, int N, int splits)
{
    EncodeTiled enc = encoder();
    if (!enc)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)M, (cuuint64_t)splits};
    const cuuint64_t strides[2] = {(cuuint64_t)N * 4, (cuuint64_t)M * N * 4};
    const cuuint32_t box[3] = {32, 32, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
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
    CUtensorMap ma, mb, mc;
    if (!make_map(&ma, g.A, g.a_rows, g.K, g.lda, kBM) || !make_map(&mb, g.Bt, g.b_rows, g.K, g.ldb, kBN) ||
        !make_map_c(&mc, g.C, g.M, g.N, g.splits))
        return cudaErrorInvalidValue;
    static std::once_flag attr;
    static cudaError_t attr_err = cudaSuccess;
    static int n_sm = 0;
    std::call_once(attr, [] {
        attr_err = cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        int dev = 0;
        if (attr_err == cudaSuccess && (attr_err = cudaGetDevice(&dev)) == cudaSuccess)
            attr_err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    });
    if (attr_err != cudaSuccess)
        return attr_err;
    TileGrid tg{};
    tg.M = g.M;
    tg.N = g.N;
    tg.tiles_n = (g.N + kBN - 1) / kBN;
    tg.tiles_m = (g.M + kBM - 1) / kBM;
    tg.splits = g.splits;
    tg.k_blocks = (g.K + kBK - 1) / kBK;
    tg.kb_per_split = (tg.k_blocks + g.splits - 1) / g.splits;
    tg.a_row0 = g.a_row0;
    tg.b_row0 = g.b_row0;
    tg.polls = wait_polls();
    const int n_tiles = tg.tiles_n * tg.tiles_m * tg.splits;
    const int grid = n_tiles < n_sm ? n_tiles : n_sm;
    k_gemm_bf16<<<grid, kThreads, kSmemBytes, st>>>(ma, mb, mc, tg, err);
    return cudaGetLastError();
}

}  // namespace hh
