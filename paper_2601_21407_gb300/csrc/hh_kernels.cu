// CUDA kernels of the Hodgkin-Huxley hot path compiled into libhh.so (sm_103a).
//
//   launchers of the table-interpreting neuron kernels (k_independent,
//                  k_net_window in hh_table.cu, one translation unit per
//                  precision)
//   k_route        spike propagation over the out-CSR: one warp per
//                  (spike, 256-synapse segment) item, or per spike for
//                  large windows; 128-bit reads of (target, weight), 64-bit
//                  fixed-point atomic adds into the delay ring (order
//                  independent)
//   transpose/check/init/trace helpers.
// The neuron bodies live in hh_device.cuh and are shared with the per-model
// kernels compiled at run time (hh_jit.cu).
#include <cstdint>

#include "hh_internal.h"

namespace hh {
namespace {

// Spike routing of a list whose length is read on the device.  A window of
// the window schedule (W > 0: steps t0 .. t0 + W - 1, list slot lslot) with
// at least RP.pull_min spikes is pulled over the in-CSR when the network
// keeps one (dynamic shared memory: pull_smem_bytes(N)).
__global__ void __launch_bounds__(256) k_route(const __grid_constant__ RouteParams RP,
                                               const int32_t* __restrict__ st,
                                               const int32_t* __restrict__ ix,
                                               const int32_t* __restrict__ n_dev, int64_t n_host,
                                               int64_t cap, int64_t t0, int32_t W, int32_t lslot)
{
    int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    if (n > cap)
        n = cap;
    if (RP.in_rec && RP.last_spk && W > 0 && W <= RP.pull_w && RP.pull_min >= 0 && n > 0 && n >= RP.pull_min &&
        blockDim.x == 32 * kPullWarps) {
        extern __shared__ __align__(16) unsigned char pull_smem[];
        route_pull(RP, st, ix, n, t0, W, lslot, pull_smem);
        return;
    }
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // Up to 16 segments per warp, every (spike, 256-synapse segment) item is
    // taken by its own warp, so a spike's fan-out is not a chain of dependent
    // row reads on one warp (a window of a few hundred spikes would wait for
    // ten DRAM round trips per spike); beyond, one warp streams each spike's
    // row with two chunks in flight (bursts, bound by the L2 atomics).
    if (n * RP.segs <= 16 * nw)
        route_items(RP, st, ix, n, warp, nw);
    else
        route_spikes(RP, st, ix, n, warp, nw);
}

// -------------------------------------------------------------------------
// Helpers
// -------------------------------------------------------------------------
template <int MAXG>
__global__ void k_init_state(const __grid_constant__ DevModels Ms, const __grid_constant__ NeuronParams P, const float* __restrict__ V0,
                             int32_t model_index)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N)
        return;
    const int mid = P.model_id ? P.model_id[i] : 0;
    if (model_index >= 0 && mid != model_index)
        return;
    const DevModel& M = Ms.m[mid];
    const float V = V0 ? V0[i] : P.V[i];
    P.V[i] = V;
    if (P.Vlo)
        P.Vlo[i] = 0.0f;
    const float Ca = M.ca_ch >= 0 ? M.ca_rest : 0.0f;
    P.Ca[i] = Ca;
    for (int q = 0; q < kMaxGates; ++q) {
        float inf = 0.0f, z;
        if (q < M.n_gates)
            gate_inf_z<false>(M.g[q], V, Ca, 1.0f, inf, z);
        P.P[(int64_t)q * P.N + i] = inf;
        if (P.Plo)
            P.Plo[(int64_t)q * P.N + i] = 0.0f;
    }
}

__global__ void k_csr_check(const int32_t* __restrict__ col, const float* __restrict__ w, int64_t S,
                            int64_t N, int32_t* flag)
{
    int32_t bad = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < S;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = col[e];
        const float x = w[e];
        if (c < 0 || c >= N)
            bad |= 1;
        if (!(x >= 0.0f && x < 65536.0f))
            bad |= 2;
    }
    if (bad)
        atomicOr(flag, bad);
}

__global__ void k_count_pre(const int32_t* __restrict__ col, int64_t S, int32_t* cnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < S;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[e], 1);
}

__global__ void k_fill_out(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                           const float* __restrict__ w, int64_t N, unsigned long long* cursor,
                           int32_t* out_post, float* out_w)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < N; r += nw) {
        const int64_t e1 = row_ptr[r + 1];
        for (int64_t e = row_ptr[r] + lane; e < e1; e += 32) {
            const unsigned long long pos = atomicAdd(cursor + col[e], 1ull);
            out_post[pos] = (int32_t)r;
            out_w[pos] = w[e];
        }
    }
}

// pull-routing records of the in-CSR: presynaptic index (checked to lie in
// [0, N), N <= 65536) and the three 16-bit parts of the weight's fixed-point
// value (the value the push adds)
__global__ void k_pull_records(const int32_t* __restrict__ col, const float* __restrict__ w, int64_t S,
                               uint2* out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < S; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long f = nS_to_fixed(w[e]);
        out[e] = make_uint2((uint32_t)col[e] | ((uint32_t)(f & 0xffffu) << 16),
                            (uint32_t)((f >> 16) & 0xffffu) | ((uint32_t)(f >> 32) << 16));
    }
}

__global__ void k_fill_gbar(const __grid_constant__ DevModels Ms, int64_t N, const uint8_t* __restrict__ model_id,
                            int32_t model_index, const float* __restrict__ src, float* gbar)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N)
        return;
    const int mid = model_id ? model_id[i] : 0;
    if (model_index >= 0 && mid != model_index)
        return;
    const DevModel& M = Ms.m[mid];
    for (int c = 0; c < kMaxChannels; ++c)
        gbar[(int64_t)c * N + i] = c < M.n_ch ? (src ? src[(int64_t)c * N + i] : M.gbar[c]) : 0.0f;
}

__global__ void k_trace_slots(const int32_t* __restrict__ idx, int32_t n, int64_t N, int32_t* slot)
{
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        const int32_t i = idx[r];
        // a neuron listed more than once takes its last row (the largest r),
        // whatever order the threads run in
        if (i >= 0 && i < N)
            atomicMax(slot + i, r);
    }
}

int block_for(int64_t N)
{
    // spread small populations over all SMs: at least ~2 blocks per SM
    if (N <= 152 * 2 * 32)
        return 32;
    if (N <= 152 * 2 * 64)
        return 64;
    return 128;
}

int grid_for(int64_t N, int bs)
{
    return (int)((N + bs - 1) / bs);
}

}  // namespace

cudaError_t launch_init_state(const DevModels& M, const NeuronParams& P, const float* V0,
                              int32_t model_index, int precision, cudaStream_t st)
{
    (void)precision;
    const int bs = 128;
    k_init_state<kMaxGates><<<grid_for(P.N, bs), bs, 0, st>>>(M, P, V0, model_index);
    return cudaGetLastError();
}

// The table-interpreting neuron kernels, one translation unit per
// precision (hh_table.cu); COMPENSATED also serves any other mode.
cudaError_t launch_independent(const DevModels& M, const NeuronParams& P, int precision, int64_t t0,
                               int32_t n_steps, const float* I_steps, const RecordParams& R,
                               cudaStream_t st)
{
    const int bs = block_for(P.N);
    const int grid = grid_for(P.N, bs);
    if (precision == HH_PREC_FAST)
        return table_independent_fast(M, P, t0, n_steps, I_steps, R, grid, bs, st);
    if (precision == HH_PREC_ACCURATE)
        return table_independent_accurate(M, P, t0, n_steps, I_steps, R, grid, bs, st);
    return table_independent_compensated(M, P, t0, n_steps, I_steps, R, grid, bs, st);
}

cudaError_t launch_net_window(const DevModels& M, const NeuronParams& P, int precision, int64_t t0,
                              int32_t W, int32_t parity, const float* I_steps,
                              const RecordParams& R, const SpikeList& L, cudaStream_t st)
{
    const int bs = block_for(P.N);
    const int grid = grid_for(P.N, bs);
    if (precision == HH_PREC_FAST)
        return table_net_window_fast(M, P, t0, W, parity, I_steps, R, L, grid, bs, st);
    if (precision == HH_PREC_ACCURATE)
        return table_net_window_accurate(M, P, t0, W, parity, I_steps, R, L, grid, bs, st);
    return table_net_window_compensated(M, P, t0, W, parity, I_steps, R, L, grid, bs, st);
}

// the shared memory a pulling routing block may take, and the largest
// shared-memory carveout, which the window kernels it co-runs with prefer as
// well (blocks of kernels with different carveouts do not share an SM); set
// on the current device where a network that may pull is created
cudaError_t route_pull_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_route, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pull_smem_bytes(kPullMaxN, kPullMaxW));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_route, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t launch_route_window(const RouteParams& RP, const SpikeList& L, int32_t parity, int64_t t0,
                                int32_t W, int32_t blocks, cudaStream_t st)
{
    // by default two resident blocks per SM whose warps loop over the
    // window's spikes: routing overlaps the next window's neuron kernel,
    // whose blocks must still find registers on every SM
    const size_t smem = RP.in_rec && RP.pull_min >= 0 ? pull_smem_bytes(RP.N, RP.pull_w) : 0;
    k_route<<<blocks > 0 ? blocks : 152 * 2, 32 * kPullWarps, smem, st>>>(RP, L.step + parity * L.cap, L.idx + parity * L.cap,
                                                   L.counter + parity, 0, L.cap, t0, W, parity);
    return cudaGetLastError();
}

cudaError_t launch_route_list(const RouteParams& RP, const int32_t* step, const int32_t* idx,
                              int64_t n, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_route<<<152 * 8, 256, 0, st>>>(RP, step, idx, nullptr, n, n, 0, 0, 0);
    return cudaGetLastError();
}

cudaError_t launch_csr_check(const int32_t* col, const float* w, int64_t S, int64_t N, int32_t* flag,
                             cudaStream_t st)
{
    if (S <= 0)
        return cudaSuccess;
    k_csr_check<<<152 * 8, 256, 0, st>>>(col, w, S, N, flag);
    return cudaGetLastError();
}

cudaError_t launch_count_pre(const int32_t* col, int64_t S, int32_t* cnt, cudaStream_t st)
{
    if (S <= 0)
        return cudaSuccess;
    k_count_pre<<<152 * 8, 256, 0, st>>>(col, S, cnt);
    return cudaGetLastError();
}

cudaError_t launch_fill_out(const int64_t* row_ptr, const int32_t* col, const float* w, int64_t N,
                            unsigned long long* cursor, int32_t* out_post, float* out_w,
                            cudaStream_t st)
{
    k_fill_out<<<152 * 8, 256, 0, st>>>(row_ptr, col, w, N, cursor, out_post, out_w);
    return cudaGetLastError();
}

cudaError_t launch_pull_records(const int32_t* col, const float* w, int64_t S, uint2* out, cudaStream_t st)
{
    if (S <= 0)
        return cudaSuccess;
    k_pull_records<<<152 * 8, 256, 0, st>>>(col, w, S, out);
    return cudaGetLastError();
}

cudaError_t launch_fill_gbar(const DevModels& M, int64_t N, const uint8_t* model_id,
                             int32_t model_index, const float* src, float* gbar, cudaStream_t st)
{
    k_fill_gbar<<<grid_for(N, 256), 256, 0, st>>>(M, N, model_id, model_index, src, gbar);
    return cudaGetLastError();
}

cudaError_t launch_trace_slots(const int32_t* trace_idx, int32_t n_trace, int64_t N, int32_t* slot,
                               cudaStream_t st)
{
    if (n_trace <= 0)
        return cudaSuccess;
    k_trace_slots<<<(n_trace + 255) / 256, 256, 0, st>>>(trace_idx, n_trace, N, slot);
    return cudaGetLastError();
}

}  // namespace hh
