// Internal declarations shared by the C-ABI layer (hh_abi.cu) and the
// kernels (hh_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/hh.h"
#include "hh_device.cuh"

namespace hh {


// Limits of the bounded device-side waits (hh_set_wait_limits; hh_abi.cu):
// the persistent kernel's progress waits in ns of the global timer, the
// tensor-core pipelines' mbarrier waits in polls.
unsigned long long wait_limit_ns();
long long wait_polls();

// error reporting into the thread-local hh_last_error() message (hh_abi.cu)
hh_status fail(hh_status s, const char* fmt, ...);
// validate a user model and prepare it for the device (hh_abi.cu)
hh_status prep_model(const hh_model_desc* m, double dt, DevModel* out);

// launchers (hh_kernels.cu); all asynchronous on `st`
cudaError_t launch_init_state(const DevModels& M, const NeuronParams& P, const float* V0,
                              int32_t model_index, int precision, cudaStream_t st);
cudaError_t launch_independent(const DevModels& M, const NeuronParams& P, int precision,
                               int64_t t0, int32_t n_steps, const float* I_steps,
                               const RecordParams& R, cudaStream_t st);
cudaError_t launch_net_window(const DevModels& M, const NeuronParams& P, int precision,
                              int64_t t0, int32_t W, int32_t window_parity,
                              const float* I_steps, const RecordParams& R,
                              const SpikeList& L, cudaStream_t st);
// the table-interpreting kernels of one precision each (hh_table.cu)
#define HH_TABLE_DECL(suffix)                                                                              \
    cudaError_t table_independent_##suffix(const DevModels& M, const NeuronParams& P, int64_t t0,          \
                                           int32_t n_steps, const float* I_steps, const RecordParams& R, \
                                           int grid, int block, cudaStream_t st);                          \
    cudaError_t table_net_window_##suffix(const DevModels& M, const NeuronParams& P, int64_t t0, int32_t W, \
                                          int32_t parity, const float* I_steps, const RecordParams& R,    \
                                          const SpikeList& L, int grid, int block, cudaStream_t st);
HH_TABLE_DECL(fast)
HH_TABLE_DECL(accurate)
HH_TABLE_DECL(compensated)
#undef HH_TABLE_DECL
cudaError_t launch_route_window(const RouteParams& RP, const SpikeList& L, int32_t parity, int64_t t0,
                                int32_t W, int32_t blocks, cudaStream_t st);
cudaError_t route_pull_prepare();
cudaError_t launch_route_list(const RouteParams& RP, const int32_t* step, const int32_t* idx,
                              int64_t n, cudaStream_t st);
cudaError_t launch_csr_check(const int32_t* col, const float* w, int64_t S, int64_t N,
                             int32_t* flag, cudaStream_t st);
cudaError_t launch_count_pre(const int32_t* col, int64_t S, int32_t* cnt, cudaStream_t st);
cudaError_t launch_pull_records(const int32_t* col, const float* w, int64_t S, uint2* out, cudaStream_t st);
cudaError_t launch_fill_out(const int64_t* row_ptr, const int32_t* col, const float* w,
                            int64_t N, unsigned long long* cursor, int32_t* out_post,
                            float* out_w, cudaStream_t st);
// gbar[c][i] = src[c][i] (src != nullptr) or the model default, for every
// neuron i of model `model_index` (all installed models when < 0).
cudaError_t launch_fill_gbar(const DevModels& M, int64_t N, const uint8_t* model_id,
                             int32_t model_index, const float* src, float* gbar, cudaStream_t st);
cudaError_t launch_trace_slots(const int32_t* trace_idx, int32_t n_trace, int64_t N,
                               int32_t* slot, cudaStream_t st);

// BF16 GEMM on tcgen05 (hh_gemm.cu): C[s][m][n] = sum_{k in split s}
// A[a_row0+m][k] Bt[b_row0+n][k]; A, Bt K-major bf16 with leading dimensions
// lda, ldb (elements, multiples of 8); C fp32 [splits][M][N].
struct GemmArgs {
    const void* A;
    int a_rows, lda, a_row0;
    const void* Bt;
    int b_rows, ldb, b_row0;
    float* C;
    int M, N, K, splits;
};
const char* gemm_check(const GemmArgs& g);
cudaError_t launch_gemm_bf16(const GemmArgs& g, int32_t* err, cudaStream_t st);

// learned surrogate (hh_surrogate.cu)
struct Surrogate;
hh_status surrogate_train(const DevModels& Ms, int precision, double dt, int64_t N_net,
                          const hh_surrogate_desc* d, cudaStream_t st, Surrogate** out, hh_surrogate_report* rep);
void surrogate_free(Surrogate* s);
cudaError_t surrogate_window(const DevModels& Ms, Surrogate* S, const NeuronParams& P, int precision,
                             cudaStream_t st);
int surrogate_window_steps(const Surrogate* S);
const int32_t* surrogate_fb_list(const Surrogate* S);
const int32_t* surrogate_fb_count(const Surrogate* S);
cudaError_t surrogate_stats(const Surrogate* S, unsigned long long* host2, int32_t* err);
cudaError_t surrogate_reset_stats(Surrogate* S, cudaStream_t st);

// Neuron kernels specialised for a model set, compiled with NVRTC (hh_jit.cu).
// The differentiable layer's kernels compiled for its model (hh_jit.cu).
struct LayerKernels {
    cudaKernel_t fwd = nullptr;
    cudaKernel_t recompute = nullptr;
    cudaKernel_t bwd = nullptr;
};
struct LayerParams;
bool jit_get_layer(const DevModels& M, int precision, LayerKernels* out, std::string* err);
// Launch k(L, arg) with one thread per neuron-sample (n of them), blocks of
// 128, `smem` bytes of dynamic shared memory.
cudaError_t jit_launch_layer(cudaKernel_t k, const LayerParams& L, int arg, int64_t n, size_t smem,
                             cudaStream_t st);

// FP32 FMA, ex2.approx and rcp.approx results per second on the current device.
cudaError_t measure_peaks(double* ffma, double* ex2, double* rcp, cudaStream_t st);

struct JitKernels {
    cudaKernel_t independent = nullptr;
    cudaKernel_t window = nullptr;
    cudaKernel_t indexed = nullptr;
    cudaKernel_t persistent = nullptr;
};
int jit_persistent_capacity(const JitKernels& K, const NeuronParams& P);
cudaError_t jit_launch_persistent(const JitKernels& K, const NeuronParams& P, const RouteParams& RP, int64_t t0,
                                  int32_t n_steps, int32_t W, int64_t w_index0, const float* I_steps,
                                  const RecordParams& R, const SpikeList& L, const PhaseCounters& pc,
                                  cudaStream_t st);
// Compile (or take from the process-wide cache) the kernels for the installed
// models; false with a message in *err on failure.
// What the run-time compiled neuron kernels of a network carry besides the
// models: its V update and the optional per-step inputs.
struct JitFlags {
    int v_update = HH_V_EXP_EULER;
    bool drive = false, cable = false, syn_current = false, compound = false;
};
bool jit_get(const DevModels& M, const bool* installed, int precision, const JitFlags& f, JitKernels* out,
             std::string* err);
cudaError_t jit_launch_independent(const JitKernels& K, const NeuronParams& P, int64_t t0,
                                   int32_t n_steps, const float* I_steps, const RecordParams& R,
                                   cudaStream_t st);
cudaError_t jit_launch_indexed(const JitKernels& K, const NeuronParams& P, const int32_t* list,
                               const int32_t* n_list, int64_t max_list, int64_t t0, int32_t n_steps,
                               const RecordParams& R, cudaStream_t st);
cudaError_t jit_launch_window(const JitKernels& K, const NeuronParams& P, int64_t t0, int32_t W,
                              int32_t parity, const float* I_steps, const RecordParams& R,
                              const SpikeList& L, int32_t early, int32_t block, cudaStream_t st);

}  // namespace hh
