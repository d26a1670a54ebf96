// Table-interpreting neuron kernels (the model read from a table in the
// kernel parameters; the kernels specialised per model at run time are in
// hh_jit.cu).  This file is compiled once per precision, with
// HH_TABLE_PREC set to HH_PREC_FAST, HH_PREC_ACCURATE or
// HH_PREC_COMPENSATED, so the instantiations build in parallel.
//
//   k_independent  many time steps of independent neurons in one launch,
//                  state in registers (Methods, Eq. hh_eq_full with
//                  exponential-Euler gates and V)
//   k_net_window   up to D steps of a network per launch: delivery from the
//                  delay ring + Poisson background, rates, gates, V, Ca,
//                  threshold, warp-aggregated spike compaction, synaptic
//                  decay
// The neuron bodies live in hh_device.cuh.
#include <cstdint>

#include "hh_internal.h"

#ifndef HH_TABLE_PREC
#error "compile with -DHH_TABLE_PREC=<precision>"
#endif

namespace hh {
namespace {

// Dynamics read from a model table in the kernel parameters.
struct TableDyn {
    static constexpr bool kDrive = true, kCable = true, kSynCurrent = true, kCompound = true;
    const DevModels& Ms;
    template <int MAXG, int PREC>
    __device__ __forceinline__ void load(int mid, const NeuronParams& P, int64_t i,
                                         State<MAXG, PREC>& s) const
    {
        load_conductances(Ms.m[mid], P.gbar, P.N, i, s);
    }
    template <int MAXG, int PREC>
    __device__ __forceinline__ void step(int mid, float dt, int v_update, float I, float gsE, float EE,
                                         float gsI, float EI, State<MAXG, PREC>& s) const
    {
        neuron_step<MAXG, PREC>(Ms.m[mid], dt, v_update, I, gsE, EE, gsI, EI, s);
    }
};

template <int MAXG, int PREC>
__global__ void __launch_bounds__(128) k_independent(const __grid_constant__ DevModels Ms,
                                                     const __grid_constant__ NeuronParams P,
                                                     int64_t t0, int32_t n_steps,
                                                     const float* __restrict__ I_steps,
                                                     const __grid_constant__ RecordParams R)
{
    independent_body<MAXG, PREC>(TableDyn{Ms}, P, t0, n_steps, I_steps, R);
}

template <int MAXG, int PREC>
__global__ void __launch_bounds__(128) k_net_window(const __grid_constant__ DevModels Ms,
                                                    const __grid_constant__ NeuronParams P,
                                                    int64_t t0, int32_t W,
                                                    const float* __restrict__ I_steps,
                                                    const __grid_constant__ RecordParams R,
                                                    const __grid_constant__ SpikeList L,
                                                    int32_t parity)
{
    window_body<MAXG, PREC, 1>(TableDyn{Ms}, P, t0, W, I_steps, R, L, parity, 0);
}

}  // namespace

#if HH_TABLE_PREC == 0
#define HH_TABLE_FN(name) name##_fast
#elif HH_TABLE_PREC == 1
#define HH_TABLE_FN(name) name##_accurate
#else
#define HH_TABLE_FN(name) name##_compensated
#endif

// gate arrays of 4 (classic models) or 8 entries
cudaError_t HH_TABLE_FN(table_independent)(const DevModels& M, const NeuronParams& P, int64_t t0, int32_t n_steps,
                                          const float* I_steps, const RecordParams& R, int grid, int block,
                                          cudaStream_t st)
{
    if (M.max_gates <= 4)
        k_independent<4, HH_TABLE_PREC><<<grid, block, 0, st>>>(M, P, t0, n_steps, I_steps, R);
    else
        k_independent<8, HH_TABLE_PREC><<<grid, block, 0, st>>>(M, P, t0, n_steps, I_steps, R);
    return cudaGetLastError();
}

cudaError_t HH_TABLE_FN(table_net_window)(const DevModels& M, const NeuronParams& P, int64_t t0, int32_t W,
                                         int32_t parity, const float* I_steps, const RecordParams& R,
                                         const SpikeList& L, int grid, int block, cudaStream_t st)
{
    if (M.max_gates <= 4)
        k_net_window<4, HH_TABLE_PREC><<<grid, block, 0, st>>>(M, P, t0, W, I_steps, R, L, parity);
    else
        k_net_window<8, HH_TABLE_PREC><<<grid, block, 0, st>>>(M, P, t0, W, I_steps, R, L, parity);
    return cudaGetLastError();
}

}  // namespace hh
