// Internal declarations shared by the C-ABI layer (hh_abi.cu) and the
// kernels (hh_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hh.h"

namespace hh {

constexpr int kMaxModels = HH_MAX_MODELS;
constexpr int kMaxGates = HH_MAX_GATES;
constexpr int kMaxChannels = HH_MAX_CHANNELS;
constexpr int kMaxPoisson = 64;
constexpr float kLog2e = 1.4426950408889634f;

// A rate function prepared for the device.  For the SFU path the exponent
// (V - vh)/k is evaluated as V*s + b in base 2 (s = log2(e)/k, b = -vh*s);
// the accurate paths use (V - vh)*ik with ik = 1/k.
struct DevFn {
    int32_t form;
    float a, c;
    float vh, k, ik, s, b;     // first exponential
    float vh2, ik2, s2, b2;    // second exponential (bell)
};

struct DevGate {
    int32_t kind;
    int32_t power;
    DevFn f1, f2;
};

struct DevModel {
    float C_m, inv_C;
    int32_t n_ch, n_gates, ca_ch;
    float ca_tau, ca_k, ca_rest, ca_decay;  // ca_decay = exp(-dt/ca_tau)
    float E[kMaxChannels];
    float gbar[kMaxChannels];
    int32_t ch_first[kMaxChannels];
    int32_t ch_ng[kMaxChannels];
    // per gate: the channel it belongs to, whether it is that channel's last
    // gate (eta complete), the channel's reversal potential, and whether the
    // channel feeds the calcium pool
    int32_t gate_ch[kMaxGates];
    int32_t gate_last[kMaxGates];
    float gate_E[kMaxGates];
    int32_t gate_ca[kMaxGates];
    DevGate g[kMaxGates];
};

struct DevModels {
    int32_t n;
    int32_t max_gates, max_channels;
    DevModel m[kMaxModels];
};

// Everything a neuron kernel reads besides its own state.
struct NeuronParams {
    int64_t N;
    float dt, theta;
    int32_t v_update;
    // state (SoA, library-owned)
    float* V;
    float* Vlo;      // compensated low parts (precision 2)
    float* P;        // [kMaxGates][N]
    float* Plo;      // [kMaxGates][N] (precision 2)
    float* Ca;
    float* gE;       // nS
    float* gI;       // nS
    const uint8_t* model_id;
    const float* gbar;     // [kMaxChannels][N] or nullptr
    const float* I_const;  // [N] or nullptr
    const int32_t* trace_slot;  // [N] or nullptr (slot = i for i < n_trace)
    int32_t* status;
    // synapses
    int64_t* ringE;   // [R][N] fixed point 2^-32 nS
    int64_t* ringI;
    int32_t R;        // ring slots (= delay steps)
    float E_E, E_I, decE, decI, to_mS;
    // background
    int32_t bg_n;     // number of thresholds (0 = off)
    float bg_w;
    uint64_t seed;
    unsigned long long bg_thr[kMaxPoisson];
};

struct RecordParams {
    float* V_trace;
    int32_t n_trace;
    hh_spike* spikes;
    int64_t spike_cap;
    unsigned long long* n_spikes;
    int32_t* counts;
};

// Window spike list used between the neuron and the routing kernels.
struct SpikeList {
    int32_t* step;
    int32_t* idx;
    int32_t* counter;   // [2] alternating per window
    int64_t cap;
};

struct RouteParams {
    int64_t N;
    const int64_t* out_ptr;
    const int32_t* out_post;
    const float* out_w;
    const uint8_t* inh;
    int64_t* ringE;
    int64_t* ringI;
    int32_t R;         // slots in the destination (ring: R = D; open loop: unused)
    int32_t D;
    int32_t open_loop; // 1: destination is [n_window][N] linear, drop >= n_window
    int32_t n_window;
};

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
cudaError_t launch_route_window(const RouteParams& RP, const SpikeList& L,
                                int32_t window_parity, cudaStream_t st);
cudaError_t launch_route_list(const RouteParams& RP, const int32_t* step, const int32_t* idx,
                              int64_t n, cudaStream_t st);
cudaError_t launch_csr_check(const int32_t* col, const float* w, int64_t S, int64_t N,
                             int32_t* flag, cudaStream_t st);
cudaError_t launch_count_pre(const int32_t* col, int64_t S, int32_t* cnt, cudaStream_t st);
cudaError_t launch_fill_out(const int64_t* row_ptr, const int32_t* col, const float* w,
                            int64_t N, unsigned long long* cursor, int32_t* out_post,
                            float* out_w, cudaStream_t st);
// gbar[c][i] = src[c][i] (src != nullptr) or the model default, for every
// neuron i of model `model_index` (all installed models when < 0).
cudaError_t launch_fill_gbar(const DevModels& M, int64_t N, const uint8_t* model_id,
                             int32_t model_index, const float* src, float* gbar, cudaStream_t st);
cudaError_t launch_trace_slots(const int32_t* trace_idx, int32_t n_trace, int64_t N,
                               int32_t* slot, cudaStream_t st);

}  // namespace hh
