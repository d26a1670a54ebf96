// Device code of the Hodgkin-Huxley neuron update, shared by the kernels
// compiled into libhh.so (table interpreter, hh_kernels.cu) and the
// per-model kernels compiled at run time with NVRTC (hh_jit.cu embeds this
// file verbatim).  It therefore includes nothing and relies only on builtin
// types; under NVRTC the few public ABI names it uses (HH_* constants and
// hh_spike) are emitted in front of it by the JIT generator.
//
// Method (Methods, Eq. hh_eq_full, exponential Euler of "Simplified
// discretization"): per step, rates at V_t, gates
//   p += (p_inf - p)(1 - e^{-dt/tau}),
// conductances with the new gates, then V with the conductances frozen:
//   V += (I - I_ion)/G (1 - e^{-dt G/C}),  I_ion = sum_X g_X (V - E_X),
// or explicit Euler V += dt/C (I - I_ion) (Eq. hh_dyn_simplified), and a
// first-order Ca pool.
#pragma once

#ifdef __CUDACC_RTC__
typedef long long int64_t;
typedef unsigned long long uint64_t;
typedef int int32_t;
typedef unsigned int uint32_t;
typedef unsigned char uint8_t;
#else
#include <cstdint>
#endif

namespace hh {

constexpr int kMaxModels = HH_MAX_MODELS;
constexpr int kMaxGates = HH_MAX_GATES;
constexpr int kMaxChannels = HH_MAX_CHANNELS;
constexpr int kMaxPoisson = 64;
constexpr float kLog2e = 1.4426950408889634f;
constexpr unsigned kFull = 0xffffffffu;

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

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)

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

__device__ __forceinline__ bool finite(float x) { return (x - x) == 0.0f; }

// A 64-bit fixed-point sum in units of 2^-32 nS as a float in nS, with two
// 32-bit conversions (the 64-bit integer conversion runs on the FP64 unit).
__device__ __forceinline__ float fixed_to_nS(long long e)
{
    const int hi = (int)(e >> 32);
    const unsigned lo = (unsigned)(e & 0xffffffffll);
    return fmaf((float)lo, 2.3283064365386963e-10f, (float)hi);
}

template <int MAXG, int PREC>
struct State {
    float V, Vlo, Ca;
    float p[MAXG];
    float plo[MAXG];
    float gq[MAXG];         // maximal conductance of the channel whose last gate is q
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
// Kernel bodies.  `Dyn` supplies the neuron model(s):
//   dyn.template load<MAXG, PREC>(mid, P, i, s)  per-neuron conductances
//   dyn.template step<MAXG, PREC>(mid, dt, v_update, I, gsE, EE, gsI, EI, s)
// The table interpreter reads a DevModel from the kernel parameters; the
// run-time compiled kernels build it as a compile-time constant so that the
// forms, gate counts and parameters fold into the instruction stream.
// -------------------------------------------------------------------------

// Independent neurons: n_steps in one launch, state in registers.
template <int MAXG, int PREC, class Dyn>
__device__ __forceinline__ void independent_body(const Dyn& dyn, const NeuronParams& P, int64_t t0,
                                                 int32_t n_steps, const float* __restrict__ I_steps,
                                                 const RecordParams& R)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < P.N;
    const int64_t i = valid ? gi : 0;
    const int mid = P.model_id ? P.model_id[i] : 0;
    State<MAXG, PREC> s;
    load_state(P, i, s);
    dyn.template load<MAXG, PREC>(mid, P, i, s);
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
        dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, I, 0.0f, 0.0f, 0.0f, 0.0f, s);
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
        if (!finite(s.V))
            atomicOr(P.status, HH_STATUS_NONFINITE);
    }
}

// Independent neurons named by a device list (the windows the learned
// surrogate declined): n_steps plain steps for each listed neuron.
template <int MAXG, int PREC, class Dyn>
__device__ __forceinline__ void indexed_body(const Dyn& dyn, const NeuronParams& P, const int32_t* __restrict__ list,
                                             const int32_t* __restrict__ n_list, int64_t t0, int32_t n_steps,
                                             const RecordParams& R)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nl = *n_list;
    if ((int64_t)blockIdx.x * blockDim.x >= nl)
        return;  // whole block past the list (uniform per block)
    const bool valid = gi < nl;
    const int64_t i = valid ? list[gi] : list[0];
    const int mid = P.model_id ? P.model_id[i] : 0;
    State<MAXG, PREC> s;
    load_state(P, i, s);
    dyn.template load<MAXG, PREC>(mid, P, i, s);
    const float Ic = P.I_const ? P.I_const[i] : 0.0f;
    int32_t cnt = 0;
    for (int32_t k = 0; k < n_steps; ++k) {
        const float Vt = s.V;
        dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, Ic, 0.0f, 0.0f, 0.0f, 0.0f, s);
        const bool spk = valid && Vt < P.theta && s.V >= P.theta;
        cnt += spk;
        const float frac = spk ? (P.theta - Vt) / (s.V - Vt) : 0.0f;
        record_spikes(spk, (int32_t)(t0 + k), (int32_t)i, frac, R, P.status);
    }
    if (valid) {
        store_state(P, i, s);
        if (R.counts && cnt)
            R.counts[i] += cnt;
        if (!finite(s.V))
            atomicOr(P.status, HH_STATUS_NONFINITE);
    }
}

// Network window: W <= D steps; spikes go to the window list for routing.
// The input of every step in the window comes from spikes at least D steps
// earlier, already routed by previous launches, so neurons are independent
// inside the window.
template <int MAXG, int PREC, class Dyn>
__device__ __forceinline__ void window_body(const Dyn& dyn, const NeuronParams& P, int64_t t0,
                                            int32_t W, const float* __restrict__ I_steps,
                                            const RecordParams& R, const SpikeList& L, int32_t parity)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi == 0)
        L.counter[parity ^ 1] = 0;  // the next window's list (its reader has finished)
    const bool valid = gi < P.N;
    const int64_t i = valid ? gi : 0;
    const int mid = P.model_id ? P.model_id[i] : 0;
    State<MAXG, PREC> s;
    load_state(P, i, s);
    dyn.template load<MAXG, PREC>(mid, P, i, s);
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
                gE += fixed_to_nS(e);
                P.ringE[o] = 0;
            }
            if (h) {
                gI += fixed_to_nS(h);
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
        dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, I, gE * P.to_mS, P.E_E, gI * P.to_mS,
                                      P.E_I, s);
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
        if (!finite(s.V))
            atomicOr(P.status, HH_STATUS_NONFINITE);
    }
}

#endif  // __CUDACC__ || __CUDACC_RTC__

}  // namespace hh
