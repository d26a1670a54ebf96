// CUDA kernels of the Hodgkin-Huxley hot path (sm_103a).
//
//   k_independent  many time steps of independent neurons in one launch, the
//                  neuron state held in registers across steps (Methods,
//                  Eq. hh_eq_full with exponential-Euler gates and V).
//   k_net_window   up to D (synaptic delay) steps of a network: the input of
//                  every step in the window was produced by spikes at least D
//                  steps earlier, so neurons stay independent inside the
//                  window and only the window boundary needs a grid-wide
//                  ordering (the routing launch).  Per step: delivery from the
//                  delay ring + Poisson background, rates, gates, V, Ca,
//                  threshold, warp-aggregated spike compaction, synaptic decay.
//   k_route        spike propagation over the out-CSR: one warp per spike,
//                  coalesced reads of (target, weight), 64-bit fixed-point
//                  atomic adds into the delay ring (order independent).
//   transpose/check/init/trace helpers.
#include <cstdint>

#include "hh_internal.h"

namespace hh {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float ex2a(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcpa(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Arithmetic policies: SFU approximations or IEEE-accurate FP32.
template <bool FAST>
struct Mth;

template <>
struct Mth<true> {
    static __device__ __forceinline__ float expv(const DevFn& f, float V) { return ex2a(fmaf(V, f.s, f.b)); }
    static __device__ __forceinline__ float expv2(const DevFn& f, float V) { return ex2a(fmaf(V, f.s2, f.b2)); }
    static __device__ __forceinline__ float div(float a, float b) { return a * rcpa(b); }
};

template <>
struct Mth<false> {
    static __device__ __forceinline__ float expv(const DevFn& f, float V) { return expf((V - f.vh) * f.ik); }
    static __device__ __forceinline__ float expv2(const DevFn& f, float V) { return expf((V - f.vh2) * f.ik2); }
    static __device__ __forceinline__ float div(float a, float b) { return a / b; }
};

// c + form(V) for the closed forms of the ABI (HH_FN_*).
template <bool FAST>
__device__ __forceinline__ float rate(const DevFn& f, float V)
{
    using M = Mth<FAST>;
    float r;
    switch (f.form) {
    case HH_FN_CONST:
        r = f.a;
        break;
    case HH_FN_EXP:
        r = f.a * M::expv(f, V);
        break;
    case HH_FN_SIGMOID:
        r = M::div(f.a, 1.0f + M::expv(f, V));
        break;
    case HH_FN_LINOID: {
        // a x / (1 - e^{-x/k}) = a k * y/(1 - e^{-y}), y = x/k.  Near y = 0 the
        // SFU path uses the Bernoulli series 1 + y/2 + y^2/12 - y^4/720
        // (truncation < 1e-10 for |y| < 0.1); the accurate path uses expm1f.
        const float x = V - f.vh;
        if (FAST) {
            const float y = x * f.ik;
            if (fabsf(y) < 0.1f) {
                const float y2 = y * y;
                r = f.a * f.k * (1.0f + 0.5f * y + y2 * (1.0f / 12.0f - y2 * (1.0f / 720.0f)));
            } else {
                r = f.a * x * rcpa(1.0f - ex2a(-y * kLog2e));
            }
        } else {
            r = (x == 0.0f) ? f.a * f.k : f.a * x / (-expm1f(-x * f.ik));
        }
        break;
    }
    default:  // HH_FN_BELL
        r = M::div(f.a, M::expv(f, V) + M::expv2(f, V));
        break;
    }
    return r + f.c;
}

// Steady-state value and dt/tau of one gate at (V, Ca).
template <bool FAST>
__device__ __forceinline__ void gate_inf_z(const DevGate& g, float V, float Ca, float dt, float& inf,
                                           float& z)
{
    using M = Mth<FAST>;
    if (g.kind == HH_GATE_AB) {
        const float al = rate<FAST>(g.f1, V), be = rate<FAST>(g.f2, V);
        const float s = al + be;
        inf = M::div(al, s);
        z = dt * s;
    } else if (g.kind == HH_GATE_INFTAU) {
        inf = rate<FAST>(g.f1, V);
        z = M::div(dt, rate<FAST>(g.f2, V));
    } else {
        inf = M::div(Ca, Ca + g.f1.a);
        z = M::div(dt, rate<FAST>(g.f2, V));
    }
}

// 1 - e^{-z} for z >= 0 with a small relative error.  The SFU path uses the
// Taylor polynomial of -expm1(-z) up to z^8 below z = 0.5 (truncation
// < 1.2e-8 relative) and 1 - 2^{-z log2 e} above; the accurate path expm1f.
// Forming the update as an increment (p_inf - p)(1 - e^{-z}) keeps the
// relaxation rate exact to rounding even when z is small, where
// p_inf + (p - p_inf) e^{-z} would turn the absolute error of e^{-z} near 1
// into a relative error of order ulp/z on every step.
template <bool FAST>
__device__ __forceinline__ float em1(float z)
{
    if (FAST) {
        if (z < 0.5f) {
            float c = fmaf(z, -1.0f / 40320.0f, 1.0f / 5040.0f);
            c = fmaf(z, c, -1.0f / 720.0f);
            c = fmaf(z, c, 1.0f / 120.0f);
            c = fmaf(z, c, -1.0f / 24.0f);
            c = fmaf(z, c, 1.0f / 6.0f);
            c = fmaf(z, c, -0.5f);
            c = fmaf(z, c, 1.0f);
            return z * c;
        }
        return 1.0f - ex2a(-z * kLog2e);
    }
    return -expm1f(-z);
}

__device__ __forceinline__ float powi(float p, int n)
{
    switch (n) {
    case 1: return p;
    case 2: return p * p;
    case 3: return p * p * p;
    default: {
        const float q = p * p;
        return q * q;
    }
    }
}

// hi + lo += d with an error-free two-sum and renormalisation.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float d)
{
    const float s = __fadd_rn(hi, d);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float lo2 = __fadd_rn(lo, err);
    const float h2 = __fadd_rn(s, lo2);
    lo = __fsub_rn(lo2, __fsub_rn(h2, s));
    hi = h2;
}

template <int MAXG, int PREC>
struct State {
    float V, Vlo, Ca;
    float p[MAXG];
    float plo[MAXG];
    // per-neuron conductance layout: gate q closes channel ch_last[q]
    float gq[MAXG];   // maximal conductance of the channel closed at gate q
    float gconst, gconstE;  // gate-less channels: sum gbar, sum gbar*E
};

template <int MAXG, int PREC>
__device__ __forceinline__ void load_conductances(const DevModel& M, const float* __restrict__ gbar,
                                                  int64_t N, int64_t i, State<MAXG, PREC>& s)
{
    s.gconst = 0.0f;
    s.gconstE = 0.0f;
#pragma unroll
    for (int c = 0; c < kMaxChannels; ++c) {
        if (c < M.n_ch && M.ch_ng[c] == 0) {
            const float g = gbar ? gbar[(int64_t)c * N + i] : M.gbar[c];
            s.gconst += g;
            s.gconstE += g * M.E[c];
        }
    }
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        s.gq[q] = 0.0f;
        if (q < M.n_gates && M.gate_last[q]) {
            const int c = M.gate_ch[q];
            s.gq[q] = gbar ? gbar[(int64_t)c * N + i] : M.gbar[c];
        }
    }
}

// One exponential-Euler step of one neuron (order: rates at V_t, gates,
// conductances with the new gates, V, Ca).  gsE/gsI in mS/cm^2.
template <int MAXG, int PREC>
__device__ __forceinline__ void neuron_step(const DevModel& M, float dt, int v_update, float I,
                                            float gsE, float EE, float gsI, float EI,
                                            State<MAXG, PREC>& s)
{
    constexpr bool FAST = PREC == HH_PREC_FAST;
    using Mt = Mth<FAST>;
    const float V = s.V;
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        if (q < M.n_gates) {
            float inf, z;
            gate_inf_z<FAST>(M.g[q], V, s.Ca, dt, inf, z);
            if (PREC == HH_PREC_COMPENSATED) {
                const float d = ((inf - s.p[q]) - s.plo[q]) * em1<false>(z);
                two_sum_add(s.p[q], s.plo[q], d);
            } else {
                s.p[q] = fmaf(inf - s.p[q], em1<FAST>(z), s.p[q]);
            }
        }
    }
    float G = gsE + gsI + s.gconst;
    float Ip = gsE * (V - EE) + gsI * (V - EI) + (s.gconst * V - s.gconstE);
    float gCa = 0.0f, ECa = 0.0f;
    float eta = 1.0f;
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        if (q < M.n_gates) {
            eta *= powi(s.p[q], M.g[q].power);
            if (M.gate_last[q]) {
                const float gx = s.gq[q] * eta;
                const float Ex = M.gate_E[q];
                G += gx;
                Ip += gx * (V - Ex);
                if (M.gate_ca[q]) {
                    gCa = gx;
                    ECa = Ex;
                }
                eta = 1.0f;
            }
        }
    }
    // V: exponential Euler with frozen conductances, as an increment
    //   dV = (V_inf - V)(1 - e^{-dt G/C}) = (I - I_ion)/G (1 - e^{-dt G/C}),
    // I_ion = sum g (V - E) formed term by term (no cancellation near rest);
    // or explicit Euler dV = dt/C (I - I_ion).
    const float Iion = PREC == HH_PREC_COMPENSATED ? Ip + G * s.Vlo : Ip;
    float dV;
    if (v_update == HH_V_EXP_EULER)
        dV = Mt::div(I - Iion, G) * em1<FAST>(dt * G * M.inv_C);
    else
        dV = dt * M.inv_C * (I - Iion);
    if (PREC == HH_PREC_COMPENSATED)
        two_sum_add(s.V, s.Vlo, dV);
    else
        s.V = V + dV;
    if (M.ca_ch >= 0) {
        const float ICa = gCa * (V - ECa);
        const float Cainf = M.ca_rest - M.ca_k * M.ca_tau * ICa;
        s.Ca = fmaf(s.Ca - Cainf, M.ca_decay, Cainf);
    }
}

template <int MAXG, int PREC>
__device__ __forceinline__ void load_state(const NeuronParams& P, int64_t i, State<MAXG, PREC>& s)
{
    s.V = P.V[i];
    s.Vlo = PREC == HH_PREC_COMPENSATED ? P.Vlo[i] : 0.0f;
    s.Ca = P.Ca[i];
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        s.p[q] = P.P[(int64_t)q * P.N + i];
        s.plo[q] = PREC == HH_PREC_COMPENSATED ? P.Plo[(int64_t)q * P.N + i] : 0.0f;
    }
}

template <int MAXG, int PREC>
__device__ __forceinline__ void store_state(const NeuronParams& P, int64_t i, const State<MAXG, PREC>& s)
{
    P.V[i] = s.V;
    if (PREC == HH_PREC_COMPENSATED)
        P.Vlo[i] = s.Vlo;
    P.Ca[i] = s.Ca;
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        P.P[(int64_t)q * P.N + i] = s.p[q];
        if (PREC == HH_PREC_COMPENSATED)
            P.Plo[(int64_t)q * P.N + i] = s.plo[q];
    }
}

// Warp-aggregated append of this step's spikes to the caller's record:
// one atomic per warp (ballot + popc), each spiking lane writes its slot.
__device__ __forceinline__ void record_spikes(bool spk, int32_t step, int32_t idx, float frac,
                                              const RecordParams& R, int32_t* status)
{
    const unsigned b = __ballot_sync(kFull, spk);
    if (b == 0u || R.n_spikes == nullptr)
        return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(b) - 1;
    unsigned long long base = 0;
    if (lane == leader)
        base = atomicAdd(R.n_spikes, (unsigned long long)__popc(b));
    base = __shfl_sync(kFull, base, leader);
    if (spk) {
        const unsigned long long pos = base + __popc(b & ((1u << lane) - 1u));
        if (pos < (unsigned long long)R.spike_cap) {
            hh_spike e;
            e.step = step;
            e.neuron = idx;
            e.frac = frac;
            R.spikes[pos] = e;
        } else {
            atomicOr(status, HH_STATUS_SPIKE_OVERFLOW);
        }
    }
}

__device__ __forceinline__ void list_append(bool spk, int32_t step, int32_t idx, int32_t* counter,
                                            int32_t* lstep, int32_t* lidx, int64_t cap)
{
    const unsigned b = __ballot_sync(kFull, spk);
    if (b == 0u)
        return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(b) - 1;
    int base = 0;
    if (lane == leader)
        base = atomicAdd(counter, __popc(b));
    base = __shfl_sync(kFull, base, leader);
    if (spk) {
        const int pos = base + __popc(b & ((1u << lane) - 1u));
        if (pos < cap) {
            lstep[pos] = step;
            lidx[pos] = idx;
        }
    }
}

// Philox-4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t pick(const uint4& v, int w)
{
    return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// -------------------------------------------------------------------------
// Independent neurons: n_steps in one launch, state in registers.
// -------------------------------------------------------------------------
template <int MAXG, int PREC>
__global__ void __launch_bounds__(128) k_independent(const DevModels Ms, const NeuronParams P,
                                                     int64_t t0, int32_t n_steps,
                                                     const float* __restrict__ I_steps,
                                                     const RecordParams R)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < P.N;
    const int64_t i = valid ? gi : 0;
    const DevModel& M = Ms.m[P.model_id ? P.model_id[i] : 0];
    State<MAXG, PREC> s;
    load_state(P, i, s);
    load_conductances(M, P.gbar, P.N, i, s);
    const float Ic = P.I_const ? P.I_const[i] : 0.0f;
    int32_t slot = -1;
    if (R.V_trace)
        slot = P.trace_slot ? P.trace_slot[i] : (i < R.n_trace ? (int32_t)i : -1);
    if (!valid)
        slot = -1;
    int32_t cnt = 0;
    for (int32_t k = 0; k < n_steps; ++k) {
        const float I = Ic + (I_steps ? I_steps[(int64_t)k * P.N + i] : 0.0f);
        const float Vt = s.V;
        neuron_step<MAXG, PREC>(M, P.dt, P.v_update, I, 0.0f, 0.0f, 0.0f, 0.0f, s);
        const bool spk = valid && Vt < P.theta && s.V >= P.theta;
        cnt += spk;
        const float frac = spk ? (P.theta - Vt) / (s.V - Vt) : 0.0f;
        record_spikes(spk, (int32_t)(t0 + k), (int32_t)i, frac, R, P.status);
        if (slot >= 0)
            R.V_trace[(int64_t)k * R.n_trace + slot] = s.V;
    }
    if (valid) {
        store_state(P, i, s);
        if (R.counts && cnt)
            R.counts[i] += cnt;
        if (!isfinite(s.V))
            atomicOr(P.status, HH_STATUS_NONFINITE);
    }
}

// -------------------------------------------------------------------------
// Network window: W <= D steps; spikes go to the window list for routing.
// -------------------------------------------------------------------------
template <int MAXG, int PREC>
__global__ void __launch_bounds__(128) k_net_window(const DevModels Ms, const NeuronParams P,
                                                    int64_t t0, int32_t W,
                                                    const float* __restrict__ I_steps,
                                                    const RecordParams R, const SpikeList L,
                                                    int32_t parity)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi == 0)
        L.counter[parity ^ 1] = 0;  // the next window's list (its reader has finished)
    const bool valid = gi < P.N;
    const int64_t i = valid ? gi : 0;
    const DevModel& M = Ms.m[P.model_id ? P.model_id[i] : 0];
    State<MAXG, PREC> s;
    load_state(P, i, s);
    load_conductances(M, P.gbar, P.N, i, s);
    float gE = P.gE[i], gI = P.gI[i];
    const float Ic = P.I_const ? P.I_const[i] : 0.0f;
    int32_t slot = -1;
    if (R.V_trace)
        slot = P.trace_slot ? P.trace_slot[i] : (i < R.n_trace ? (int32_t)i : -1);
    if (!valid)
        slot = -1;
    const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    uint4 rnd = make_uint4(0, 0, 0, 0);
    int32_t cnt = 0;
    int32_t ring_slot = (int32_t)(t0 % P.R);
    // The delay-line slots of this window were completed by earlier routing
    // launches: prefetch one step ahead so the L2 latency overlaps compute.
    long long nE = 0, nI = 0;
    if (valid && W > 0) {
        nE = P.ringE[(int64_t)ring_slot * P.N + i];
        nI = P.ringI[(int64_t)ring_slot * P.N + i];
    }
    for (int32_t k = 0; k < W; ++k) {
        const int64_t t = t0 + k;
        const long long e = nE, h = nI;
        const int32_t next_slot = ring_slot + 1 == P.R ? 0 : ring_slot + 1;
        if (valid && k + 1 < W) {
            nE = P.ringE[(int64_t)next_slot * P.N + i];
            nI = P.ringI[(int64_t)next_slot * P.N + i];
        }
        // a. delayed synaptic input (fixed point 2^-32 nS) and background
        if (valid) {
            const int64_t o = (int64_t)ring_slot * P.N + i;
            if (e) {
                gE += __ll2float_rn(e) * 2.3283064365386963e-10f;
                P.ringE[o] = 0;
            }
            if (h) {
                gI += __ll2float_rn(h) * 2.3283064365386963e-10f;
                P.ringI[o] = 0;
            }
        }
        if (P.bg_n > 0) {
            if (k == 0 || (t & 3) == 0) {
                const uint64_t q = (uint64_t)t >> 2;
                rnd = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)i, 1u, (uint32_t)(q >> 32)), key);
            }
            const unsigned long long u = pick(rnd, (int)(t & 3));
            int32_t c = 0;
            while (c < P.bg_n && u >= P.bg_thr[c])
                ++c;
            gE += (float)c * P.bg_w;
        }
        const float I = Ic + (I_steps ? I_steps[(int64_t)k * P.N + i] : 0.0f);
        const float Vt = s.V;
        neuron_step<MAXG, PREC>(M, P.dt, P.v_update, I, gE * P.to_mS, P.E_E, gI * P.to_mS, P.E_I, s);
        const bool spk = valid && Vt < P.theta && s.V >= P.theta;
        cnt += spk;
        list_append(spk, (int32_t)t, (int32_t)i, L.counter + parity, L.step, L.idx, L.cap);
        if (R.n_spikes) {
            const float frac = spk ? (P.theta - Vt) / (s.V - Vt) : 0.0f;
            record_spikes(spk, (int32_t)t, (int32_t)i, frac, R, P.status);
        }
        if (slot >= 0)
            R.V_trace[(int64_t)k * R.n_trace + slot] = s.V;
        gE *= P.decE;
        gI *= P.decI;
        ring_slot = next_slot;
    }
    if (valid) {
        store_state(P, i, s);
        P.gE[i] = gE;
        P.gI[i] = gI;
        if (R.counts && cnt)
            R.counts[i] += cnt;
        if (!isfinite(s.V))
            atomicOr(P.status, HH_STATUS_NONFINITE);
    }
}

// -------------------------------------------------------------------------
// Spike routing: one warp per spike; the spike count is read on the device.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_route(const RouteParams RP, const int32_t* __restrict__ st,
                                               const int32_t* __restrict__ ix,
                                               const int32_t* __restrict__ n_dev, int64_t n_host,
                                               int64_t cap)
{
    int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    if (n > cap)
        n = cap;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sp = warp; sp < n; sp += nw) {
        const int32_t j = ix[sp];
        const int32_t t = st[sp];
        if (j < 0 || j >= RP.N || t < 0)
            continue;
        int64_t row;
        if (RP.open_loop) {
            row = (int64_t)t + RP.D;
            if (row >= RP.n_window)
                continue;
        } else {
            row = ((int64_t)t + RP.D) % RP.R;
        }
        unsigned long long* dst =
            reinterpret_cast<unsigned long long*>((RP.inh && RP.inh[j] ? RP.ringI : RP.ringE) + row * RP.N);
        const int64_t e1 = RP.out_ptr[j + 1];
        for (int64_t e = RP.out_ptr[j] + lane; e < e1; e += 32) {
            const long long q = __float2ll_rn(RP.out_w[e] * 4294967296.0f);
            atomicAdd(dst + RP.out_post[e], (unsigned long long)q);
        }
    }
}

// -------------------------------------------------------------------------
// Helpers
// -------------------------------------------------------------------------
template <int MAXG>
__global__ void k_init_state(const DevModels Ms, const NeuronParams P, const float* __restrict__ V0,
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

__global__ void k_fill_gbar(const DevModels Ms, int64_t N, const uint8_t* __restrict__ model_id,
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
        if (i >= 0 && i < N)
            slot[i] = r;
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

#define HH_DISPATCH(MAXG_, PREC_, CALL)                                            \
    do {                                                                           \
        if ((MAXG_) <= 4) {                                                        \
            if ((PREC_) == HH_PREC_FAST) { constexpr int G = 4, Q = HH_PREC_FAST; CALL; }             \
            else if ((PREC_) == HH_PREC_ACCURATE) { constexpr int G = 4, Q = HH_PREC_ACCURATE; CALL; } \
            else { constexpr int G = 4, Q = HH_PREC_COMPENSATED; CALL; }            \
        } else {                                                                   \
            if ((PREC_) == HH_PREC_FAST) { constexpr int G = 8, Q = HH_PREC_FAST; CALL; }             \
            else if ((PREC_) == HH_PREC_ACCURATE) { constexpr int G = 8, Q = HH_PREC_ACCURATE; CALL; } \
            else { constexpr int G = 8, Q = HH_PREC_COMPENSATED; CALL; }            \
        }                                                                          \
    } while (0)

cudaError_t launch_init_state(const DevModels& M, const NeuronParams& P, const float* V0,
                              int32_t model_index, int precision, cudaStream_t st)
{
    (void)precision;
    const int bs = 128;
    k_init_state<kMaxGates><<<grid_for(P.N, bs), bs, 0, st>>>(M, P, V0, model_index);
    return cudaGetLastError();
}

cudaError_t launch_independent(const DevModels& M, const NeuronParams& P, int precision, int64_t t0,
                               int32_t n_steps, const float* I_steps, const RecordParams& R,
                               cudaStream_t st)
{
    const int bs = block_for(P.N);
    HH_DISPATCH(M.max_gates, precision,
                (k_independent<G, Q><<<grid_for(P.N, bs), bs, 0, st>>>(M, P, t0, n_steps, I_steps, R)));
    return cudaGetLastError();
}

cudaError_t launch_net_window(const DevModels& M, const NeuronParams& P, int precision, int64_t t0,
                              int32_t W, int32_t parity, const float* I_steps,
                              const RecordParams& R, const SpikeList& L, cudaStream_t st)
{
    const int bs = block_for(P.N);
    HH_DISPATCH(M.max_gates, precision,
                (k_net_window<G, Q><<<grid_for(P.N, bs), bs, 0, st>>>(M, P, t0, W, I_steps, R, L, parity)));
    return cudaGetLastError();
}

cudaError_t launch_route_window(const RouteParams& RP, const SpikeList& L, int32_t parity,
                                cudaStream_t st)
{
    k_route<<<152 * 4, 256, 0, st>>>(RP, L.step, L.idx, L.counter + parity, 0, L.cap);
    return cudaGetLastError();
}

cudaError_t launch_route_list(const RouteParams& RP, const int32_t* step, const int32_t* idx,
                              int64_t n, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_route<<<152 * 4, 256, 0, st>>>(RP, step, idx, nullptr, n, n);
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
