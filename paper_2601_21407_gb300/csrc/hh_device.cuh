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
typedef unsigned short uint16_t;
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
    float ia;                  // 1/a (0 when a = 0)
    float irate;               // 1/(a + c) (0 when a + c = 0): a constant rate's reciprocal
    // the linoid's series a k (1 + y/2 + y^2/12 - y^4/720) on the SFU path
    // as n0 + n1 y + y^2 (n2 + n4 y^2)
    float n0, n1, n2, n4;
};

struct DevGate {
    int32_t kind;
    int32_t power;
    DevFn f1, f2;
};

struct DevModel {
    float C_m, inv_C;
    int32_t n_ch, n_gates, ca_ch;
    // piecewise-cubic rate tables (HH_PREC_POLY): poly_n intervals of 1/poly_ih
    // mV from poly_vlo; interval j of gate q holds p_inf and 1 - e^{-dt/tau}
    // as float4 coefficients (c0, c1, c2, c3) of c0 + x (c1 + x (c2 + x c3)),
    // x in [0, 1), at NeuronParams::poly[poly_base + j poly_stride + 2 q + f].
    // poly_stride = 2 n_gates + 1 is odd, so that the rows of the lanes of a
    // warp start in different shared-memory bank groups.
    int32_t poly_n, poly_base, poly_stride;
    float poly_vlo, poly_ih;
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
    const float4* poly;    // rate tables of the installed models (HH_PREC_POLY) or nullptr
    int32_t poly_rows;     // float4 rows of poly (staged in shared memory when at most kPolySmemRows)
    const uint8_t* model_id;
    const float* gbar;     // [kMaxChannels][N] or nullptr
    const float* I_const;  // [N] or nullptr
    // sinusoidal drive (or nullptr): I += amp sin(2 pi u 2^-32), u = step F + Ph (mod 2^32)
    const float* sin_amp;     // [N] uA/cm^2
    const uint32_t* sin_F;    // [N] phase advance per step, 2^-32 cycles
    const uint32_t* sin_Ph;   // [N] phase at step 0, 2^-32 cycles
    // multi-compartment cells: one cell per warp (0: point neurons)
    int32_t cable_nd, cable_np;   // dendrites, compartments per dendrite
    float cable_g, cable_gs;      // axial conductance, and divided by the soma area ratio
    const int32_t* trace_slot;  // [N] or nullptr (slot = i for i < n_trace)
    int32_t* status;
    // synapses: the delay line, [R][N] entries of {E, I} (16 bytes, one
    // load per neuron-step), fixed point 2^-32 nS; R N < 2^32
    int64_t* ring;
    int32_t R;        // ring slots (= delay steps)
    // [kListSlots][pull_stride(N)] or nullptr: per window list slot, the
    // window-relative step of each neuron's last spike in the window
    // (kPullNone: none), read by the pull routing of dense windows
    uint8_t* last_spk;
    float E_E, E_I, decE, decI, to_mS;
    // background
    int32_t bg_n;     // thresholds below 2^32 (0 = off); the count of a step is
                      // #{j < bg_n : word >= bg_thr[j]} (nondecreasing table)
    float bg_w;
    float bg_sd;      // > 0: compound background N(k bg_w, k bg_sd^2)
    int32_t syn_current;  // 1: synapses inject gE - gI as a current (uA/cm^2)
    uint64_t seed;
    // Philox-4x32-10 round keys of the seed: (k0, k1) of round r at 2r, 2r + 1
    uint32_t rk[20];
    uint32_t bg_thr[kMaxPoisson];
};
// thresholds compared without a loop on every step (the rest only after a
// word that passes all of them)
constexpr int kPoissonUnroll = 4;
// steps of delay-line reads kept in flight by the window kernels
constexpr int kRingAhead = 2;

struct RecordParams {
    float* V_trace;
    int32_t n_trace;
    hh_spike* spikes;
    int64_t spike_cap;
    unsigned long long* n_spikes;
    int32_t* counts;
};

// Synaptic routing over the out-CSR (rows = presynaptic neuron).
struct RouteParams {
    int64_t N;
    const int64_t* out_ptr;
    const int32_t* out_post;
    const float* out_w;
    const uint8_t* inh;
    int64_t* ringE;    // destination of excitatory spikes (ring: the E words)
    int64_t* ringI;    // of inhibitory spikes (ring: the I words, ringE + 1)
    int32_t stride;    // words between neighbouring neurons: 2 in the ring, 1 open loop
    int32_t R;         // slots in the destination (ring: R = D; open loop: unused)
    int32_t D;
    int32_t open_loop; // 1: destination is [n_window][N] linear, drop >= n_window
    int32_t n_window;
    int32_t segs;      // most 256-synapse segments of a row (route_items)
    // pull routing of dense windows (nullptr in_rec: off): the in-CSR (rows =
    // postsynaptic neuron) as one 8-byte record per synapse, {presynaptic
    // index | p0 << 16, p1 | p2 << 16} with p0 + p1 2^16 + p2 2^32 the
    // weight in fixed point (nS_to_fixed), padded by 8 zero records; and the
    // neurons' last-spike tables of the window lists
    const int64_t* in_ptr;
    const uint2* in_rec;
    const uint8_t* last_spk;
    int64_t pull_min;  // windows of at least this many spikes are pulled (< 0: never)
    int32_t pull_w;    // the network's window steps (<= kPullMaxW): sums per replica 2 pull_w + 1
};
// Pull routing limits: 16-bit presynaptic indices, and the window-relative
// step of a spike in 6 bits of its table entry (bit 7: inhibitory)
constexpr int64_t kPullMaxN = 65536;
constexpr int kPullMaxW = 64;
constexpr uint8_t kPullNone = 0xff;
constexpr int kPullWarps = 8;  // warps per routing block (256 threads)
// A warp's (step, E/I) sums are kept as three 32-bit words of 16-bit parts
// of the 48-bit fixed-point weights (a row of at most 32,767 synapses puts
// at most ~4,100 parts below 2^16 into a word: below 2^29, no overflow), so
// that a synapse adds with native 32-bit shared-
// memory atomics; lane l adds into copy l mod kPullRep of the sums, so that
// the lanes of a burst, whose synapses hit a few sums, do not serialise.
constexpr int kPullRep = 8;
// entries per list slot of the last-spike tables (16-byte rows)
__host__ __device__ constexpr int64_t pull_stride(int64_t N) { return (N + 15) & ~(int64_t)15; }
// 32-bit words of one copy of the sums: 3 per (step, E/I), plus one (odd:
// the copies of a word fall in different banks)
__host__ __device__ constexpr int32_t pull_copy_words(int32_t W) { return 6 * W + 1; }
// dynamic shared memory of a routing block that may pull: the staged table
// and the warps' copies of the sums
__host__ __device__ constexpr size_t pull_smem_bytes(int64_t N, int32_t W)
{
    return (size_t)pull_stride(N) + (size_t)kPullWarps * kPullRep * pull_copy_words(W) * sizeof(uint32_t);
}
// Window spike lists used between the neuron and the routing kernels: three
// slots (window index mod 3) so that a window's list can be routed while the
// next window's neurons append to another slot.
constexpr int kListSlots = 3;
struct SpikeList {
    int32_t* step;      // [kListSlots][cap]
    int32_t* idx;       // [kListSlots][cap]
    int32_t* counter;   // [kListSlots]
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
        // Both branches are evaluated and one selected (no divergent branch).
        // x = V - vh is formed first: near vh the difference is exact, and
        // both y and a x keep their relative accuracy there
        const float x = V - f.vh;
        if (FAST) {
            const float y = x * f.ik;
            const float y2 = y * y;
            const float near0 = fmaf(y2, fmaf(y2, f.n4, f.n2), fmaf(y, f.n1, f.n0));
            const float far = f.a * x * rcpa(1.0f - ex2a(-y * kLog2e));
            r = fabsf(y) < 0.1f ? near0 : far;
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

// dt/tau for a time constant tau = c + form(V).  The SFU path takes a
// constant tau's reciprocal from the model table, and writes a bell-shaped
// tau = a/(e1 + e2) + c as dt (e1 + e2)/(a + c (e1 + e2)): one division
// instead of two, none when c = 0.
template <bool FAST>
__device__ __forceinline__ float dt_over_tau(const DevFn& f, float V, float dt)
{
    using M = Mth<FAST>;
    if (FAST && f.form == HH_FN_CONST)
        return dt * f.irate;
    if (FAST && f.form == HH_FN_BELL) {
        const float e = M::expv(f, V) + M::expv2(f, V);
        return f.c == 0.0f ? (dt * f.ia) * e : M::div(dt * e, fmaf(f.c, e, f.a));
    }
    return M::div(dt, rate<FAST>(f, V));
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
        z = dt_over_tau<FAST>(g.f2, V, dt);
    } else {
        inf = M::div(Ca, Ca + g.f1.a);
        z = dt_over_tau<FAST>(g.f2, V, dt);
    }
}

// 1 - e^{-z} for z >= 0 with a small relative error.  The SFU path uses the
// Taylor polynomial of -expm1(-z) up to z^5 below z = 0.125 (truncation
// < 4.3e-8 relative) and 1 - 2^{-z log2 e} above (relative error of order
// 1e-6 just above the switch, where the SFU exponential's rounding of
// e^{-z} <= 0.883 is divided by 1 - e^{-z} >= 0.117); the accurate path
// expm1f.
// Forming the update as an increment (p_inf - p)(1 - e^{-z}) keeps the
// relaxation rate exact to rounding even when z is small, where
// p_inf + (p - p_inf) e^{-z} would turn the absolute error of e^{-z} near 1
// into a relative error of order ulp/z on every step.
// The SFU path evaluates both forms and selects one (no divergent branch).
template <bool FAST>
__device__ __forceinline__ float em1(float z)
{
    if (FAST) {
        // c(z) = sum_{j<5} (-z)^j/(j+1)! by Estrin's scheme (dependency depth 3)
        const float z2 = z * z;
        const float a0 = fmaf(z, -0.5f, 1.0f);
        const float a1 = fmaf(z, -1.0f / 24.0f, 1.0f / 6.0f);
        const float c = fmaf(z2, fmaf(z2, 1.0f / 120.0f, a1), a0);
        const float far = 1.0f - ex2a(-z * kLog2e);
        return z < 0.125f ? z * c : far;
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
    const float4* poly;     // rate tables (HH_PREC_POLY), in shared or global memory
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

// SFU arithmetic: the FAST mode, and the POLY mode outside its tables.
template <int PREC>
__host__ __device__ constexpr bool sfu_math()
{
    return PREC == HH_PREC_FAST || PREC == HH_PREC_POLY;
}

// Gate part of one exponential-Euler step: the gates q with q % 2 == ROLE
// (ROLE < 0: every gate) from the rates at V_t = s.V.
template <int MAXG, int PREC, int ROLE>
__device__ __forceinline__ void neuron_gates(const DevModel& M, float dt, State<MAXG, PREC>& s)
{
    constexpr bool FAST = sfu_math<PREC>();
    const float V = s.V;
    if (PREC == HH_PREC_POLY && M.poly_n > 0) {
        // polynomial approximation of the rates (Results, "BrainFuse": the
        // operators' polynomial approximation): p_inf and 1 - e^{-dt/tau} of
        // every gate from the cubic of V's interval, when every active lane
        // of the warp lies inside the tables (else the SFU path below)
        const float u = (V - M.poly_vlo) * M.poly_ih;
        const bool in = u >= 0.0f && u < (float)M.poly_n;  // false for NaN
        if (__all_sync(__activemask(), in)) {
            const float jf = floorf(u);
            const float x = u - jf;
            const float4* b = s.poly + M.poly_base + (int)jf * M.poly_stride;
#pragma unroll
            for (int q = 0; q < MAXG; ++q) {
                if (q < M.n_gates && (ROLE < 0 || (q & 1) == ROLE)) {
                    const float4 ci = b[2 * q], ce = b[2 * q + 1];
                    float inf = fmaf(x, fmaf(x, fmaf(x, ci.w, ci.z), ci.y), ci.x);
                    const float E = fmaf(x, fmaf(x, fmaf(x, ce.w, ce.z), ce.y), ce.x);
                    if (M.g[q].kind == HH_GATE_CA)
                        inf = Mth<true>::div(s.Ca, s.Ca + M.g[q].f1.a);
                    s.p[q] = fmaf(inf - s.p[q], E, s.p[q]);
                }
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        if (q < M.n_gates && (ROLE < 0 || (q & 1) == ROLE)) {
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
}

// Membrane part: conductances with the new gates, V, Ca.  gsE/gsI in
// mS/cm^2.
template <int MAXG, int PREC>
__device__ __forceinline__ void neuron_vstep(const DevModel& M, float dt, int v_update, float I, float gsE,
                                             float EE, float gsI, float EI, State<MAXG, PREC>& s)
{
    constexpr bool FAST = sfu_math<PREC>();
    using Mt = Mth<FAST>;
    const float V = s.V;
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
    // (both forms evaluated, one selected: no branch inside the step)
    const float dV_exp = Mt::div(I - Iion, G) * em1<FAST>(dt * G * M.inv_C);
    const float dV_euler = dt * M.inv_C * (I - Iion);
    const float dV = v_update == HH_V_EXP_EULER ? dV_exp : dV_euler;
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

// One exponential-Euler step of one neuron (order: rates at V_t, gates,
// conductances with the new gates, V, Ca).  gsE/gsI in mS/cm^2.
template <int MAXG, int PREC>
__device__ __forceinline__ void neuron_step(const DevModel& M, float dt, int v_update, float I,
                                            float gsE, float EE, float gsI, float EI,
                                            State<MAXG, PREC>& s)
{
    neuron_gates<MAXG, PREC, -1>(M, dt, s);
    neuron_vstep<MAXG, PREC>(M, dt, v_update, I, gsE, EE, gsI, EI, s);
}

// Rate tables of HH_PREC_POLY: a launch whose table has at most
// kPolySmemRows rows gets them as dynamic shared memory (poly_smem_bytes),
// copied by the block at its start; larger tables are read from global
// memory.  Every thread of the block calls stage_poly before any other
// barrier.
constexpr int kPolySmemRows = 4096;  // 64 KB
__host__ __device__ constexpr size_t poly_smem_bytes(int rows)
{
    return rows > 0 && rows <= kPolySmemRows ? (size_t)rows * 16 : 0;
}
extern __shared__ float4 hh_poly_smem[];

template <int PREC>
__device__ __forceinline__ const float4* stage_poly(const NeuronParams& P)
{
    if (PREC != HH_PREC_POLY || P.poly_rows <= 0)
        return nullptr;
    if (P.poly_rows > kPolySmemRows)
        return P.poly;
    for (int k = threadIdx.x; k < P.poly_rows; k += blockDim.x)
        hh_poly_smem[k] = __ldg(P.poly + k);
    __syncthreads();
    return hh_poly_smem;
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

// Per-neuron sinusoidal drive of frequency-response sweeps: amp
// sin(2 pi (F t + Ph) 2^-32) at absolute step t, the phase kept exactly as a
// 32-bit fraction of a cycle (wrapping modulo one cycle).
struct Drive {
    float amp;
    uint32_t F, Ph;
};

__device__ __forceinline__ Drive load_drive(const NeuronParams& P, int64_t i)
{
    Drive d{0.0f, 0u, 0u};
    if (P.sin_amp) {
        d.amp = P.sin_amp[i];
        d.F = P.sin_F[i];
        d.Ph = P.sin_Ph[i];
    }
    return d;
}

template <bool FAST>
__device__ __forceinline__ float drive_at(const Drive& d, int64_t t)
{
    const uint32_t u = (uint32_t)t * d.F + d.Ph;
    const float x = (float)u * 2.3283064365386963e-10f;  // cycles in [0, 1]
    return d.amp * (FAST ? __sinf(6.283185307179586f * x) : sinpif(2.0f * x));
}

// Axial coupling of a multi-compartment cell laid out on one warp: lane 0 the
// soma, lane 1 + d n_per + j compartment j of dendrite d.  Each lane has up
// to three neighbour lanes and conductances (self and 0 when absent); the
// current from V_t is the explicit second difference of the cable term.
struct Axial {
    int nb0, nb1, nb2;
    float g0, g1, g2;
};

__device__ __forceinline__ Axial axial_setup(const NeuronParams& P)
{
    const int lane = threadIdx.x & 31;
    Axial a{lane, lane, lane, 0.0f, 0.0f, 0.0f};
    const int nd = P.cable_nd, np = P.cable_np;
    if (nd <= 0)
        return a;
    if (lane == 0) {
        a.nb0 = 1;
        a.g0 = P.cable_gs;
        if (nd > 1) {
            a.nb1 = 1 + np;
            a.g1 = P.cable_gs;
        }
        if (nd > 2) {
            a.nb2 = 1 + 2 * np;
            a.g2 = P.cable_gs;
        }
    } else if (lane < 1 + nd * np) {
        const int j = (lane - 1) % np;
        a.nb0 = j == 0 ? 0 : lane - 1;
        a.g0 = P.cable_g;
        if (j + 1 < np) {
            a.nb1 = lane + 1;
            a.g1 = P.cable_g;
        }
    }
    return a;
}

// Called by every lane of the warp.
__device__ __forceinline__ float axial_current(const Axial& a, float V)
{
    const float v0 = __shfl_sync(kFull, V, a.nb0);
    const float v1 = __shfl_sync(kFull, V, a.nb1);
    const float v2 = __shfl_sync(kFull, V, a.nb2);
    return fmaf(a.g0, v0 - V, fmaf(a.g1, v1 - V, a.g2 * (v2 - V)));
}

// Warp-aggregated append of this step's spikes to the caller's record:
// one atomic per warp (ballot + popc), each spiking lane writes its slot.
// frac = (theta - Vt)/(V - Vt) is formed only by lanes that spiked.  `b` is
// the warp's ballot of spk.
__device__ __forceinline__ void record_spikes_b(unsigned b, bool spk, int32_t step, int32_t idx, float theta,
                                                float Vt, float V, const RecordParams& R, int32_t* status)
{
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
            e.frac = (theta - Vt) / (V - Vt);
            R.spikes[pos] = e;
        } else {
            atomicOr(status, HH_STATUS_SPIKE_OVERFLOW);
        }
    }
}

__device__ __forceinline__ void record_spikes(bool spk, int32_t step, int32_t idx, float theta, float Vt,
                                              float V, const RecordParams& R, int32_t* status)
{
    record_spikes_b(__ballot_sync(kFull, spk), spk, step, idx, theta, Vt, V, R, status);
}

__device__ __forceinline__ void list_append_b(unsigned b, bool spk, int32_t step, int32_t idx, int32_t* counter,
                                              int32_t* lstep, int32_t* lidx, int64_t cap)
{
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

// The same with the ten round keys precomputed (rk[2r], rk[2r + 1] =
// k + r (0x9E3779B9, 0xBB67AE85)): no key additions per draw.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t* rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

// The four standard normals of steps 4q..4q+3 of the compound background
// from the Philox block of counter (q, i, 2, q >> 32): Box-Muller on words
// (0, 1) and (2, 3), cos then sin.
template <bool FAST>
__device__ __forceinline__ float4 bg_normals(uint64_t q, int64_t i, const uint32_t* rk)
{
    const uint4 w = philox4x32_10_rk(make_uint4((uint32_t)q, (uint32_t)i, 2u, (uint32_t)(q >> 32)), rk);
    const float s = 2.3283064365386963e-10f;
    const float u1 = fmaf((float)w.x, s, 0.5f * s), u2 = fmaf((float)w.y, s, 0.5f * s);
    const float u3 = fmaf((float)w.z, s, 0.5f * s), u4 = fmaf((float)w.w, s, 0.5f * s);
    float r0, r1, s0, c0, s1, c1;
    if (FAST) {
        r0 = sqrtf(-2.0f * __logf(u1));
        r1 = sqrtf(-2.0f * __logf(u3));
        __sincosf(6.283185307179586f * u2, &s0, &c0);
        __sincosf(6.283185307179586f * u4, &s1, &c1);
    } else {
        r0 = sqrtf(-2.0f * logf(u1));
        r1 = sqrtf(-2.0f * logf(u3));
        sincospif(2.0f * u2, &s0, &c0);
        sincospif(2.0f * u4, &s1, &c1);
    }
    return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

__device__ __forceinline__ float pickf(const float4& v, int w)
{
    return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

__device__ __forceinline__ uint32_t pick(const uint4& v, int w)
{
    return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// Inverse-CDF Poisson count of a uniform 32-bit word: #{j < n : u >= thr[j]}
// for a nondecreasing table (the first kPoissonUnroll compares without a
// loop, the rest only after a word that passed all of them).
__device__ __forceinline__ int32_t poisson_count(uint32_t u, const uint32_t* thr, int32_t n)
{
    int32_t c = 0;
#pragma unroll
    for (int j = 0; j < kPoissonUnroll; ++j)
        c += (j < n && u >= thr[j]) ? 1 : 0;
    if (c == kPoissonUnroll)
        for (int j = kPoissonUnroll; j < n && u >= thr[j]; ++j)
            ++c;
    return c;
}

// w (nS, finite, 0 <= w < 65536) as a 64-bit fixed-point count of 2^-32 nS,
// from the float's bits with integer operations only (the 64-bit float ->
// integer conversion executes on the FP64 unit).  Exact for w >= 2^-9 nS;
// below, rounded to nearest with ties up.
__device__ __forceinline__ unsigned long long nS_to_fixed(float w)
{
    const unsigned b = __float_as_uint(w);
    const int e = (int)(b >> 23);
    const unsigned m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int sh = (e ? e : 1) - 118;  // w 2^32 = m 2^(e - 150 + 32)
    if (sh >= 0)
        return (unsigned long long)m << sh;
    if (sh < -40)
        return 0ull;
    return ((unsigned long long)m + (1ull << (-sh - 1))) >> (-sh);
}

// Spike routing: one warp per spike.  The out-row is walked in 128-edge
// chunks aligned to 4 edges: lane l reads the int4 of targets and the float4
// of weights at chunk + 4l (the arrays carry 4 entries of padding), masks the
// entries outside the row and issues one RED.ADD.64 per edge.  Two chunks
// are in flight per iteration.  Warps `warp`, `warp + nw`, ... take spikes
// `warp`, `warp + nw`, ... of the list.
// Lane part of one 256-synapse chunk of an out-row: entries ea..ea+3 and
// ea+128..ea+131 (zeros past e1; rows are padded by 4 entries).
__device__ __forceinline__ void load_chunk(const RouteParams& RP, int64_t ea, int64_t e1, int4& pa, int4& pb,
                                           float4& wa, float4& wb)
{
    const int64_t eb = ea + 128;
    pa = make_int4(0, 0, 0, 0);
    pb = pa;
    wa = make_float4(0.f, 0.f, 0.f, 0.f);
    wb = wa;
    if (ea < e1) {
        pa = __ldcs(reinterpret_cast<const int4*>(RP.out_post + ea));
        wa = __ldcs(reinterpret_cast<const float4*>(RP.out_w + ea));
    }
    if (eb < e1) {
        pb = __ldcs(reinterpret_cast<const int4*>(RP.out_post + eb));
        wb = __ldcs(reinterpret_cast<const float4*>(RP.out_w + eb));
    }
}

// The atomics of one loaded chunk (entries outside [e0, e1) skipped); the
// destination word of target p is dst[p * stride].
__device__ __forceinline__ void deliver_chunk(unsigned long long* dst, int32_t stride, int64_t ea, int64_t e0,
                                              int64_t e1, const int4& pa, const int4& pb, const float4& wa,
                                              const float4& wb)
{
    const int64_t eb = ea + 128;
    const int pp[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
    const float ww[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int64_t e = (q < 4 ? ea : eb) + (q & 3);
        if (e >= e0 && e < e1)
            atomicAdd(dst + (int64_t)pp[q] * stride, nS_to_fixed(ww[q]));
    }
}

// Destination of presynaptic neuron j's spikes arriving in row `row`.
__device__ __forceinline__ unsigned long long* route_dst(const RouteParams& RP, int32_t j, int64_t row)
{
    return reinterpret_cast<unsigned long long*>((RP.inh && RP.inh[j] ? RP.ringI : RP.ringE) +
                                                 row * RP.N * RP.stride);
}

// One spike (presynaptic j at step t) delivered by the calling warp (j and
// t uniform over it).
__device__ __forceinline__ void route_one(const RouteParams& RP, int32_t j, int32_t t, int lane)
{
    if (j < 0 || j >= RP.N || t < 0)
        return;
    int64_t row;
    if (RP.open_loop) {
        row = (int64_t)t + RP.D;
        if (row >= RP.n_window)
            return;
    } else {
        row = ((int64_t)t + RP.D) % RP.R;
    }
    unsigned long long* dst = route_dst(RP, j, row);
    const int64_t e0 = RP.out_ptr[j], e1 = RP.out_ptr[j + 1];
    // 256 synapses per warp iteration, software-pipelined: the next chunk's
    // (target, weight) loads are issued before this chunk's atomics, so two
    // chunks are in flight per warp (the loop is latency-bound otherwise).
    // Streaming (evict-first) loads: the rows are read once per spike and
    // must not push the delay line out of L2.
    int64_t base = e0 & ~(int64_t)3;
    if (base >= e1)
        return;
    int4 pa, pb;
    float4 wa, wb;
    load_chunk(RP, base + 4 * lane, e1, pa, pb, wa, wb);
    for (; base < e1; base += 256) {
        int4 qa, qb;
        float4 va, vb;
        load_chunk(RP, base + 256 + 4 * lane, e1, qa, qb, va, vb);
        deliver_chunk(dst, RP.stride, base + 4 * lane, e0, e1, pa, pb, wa, wb);
        pa = qa;
        pb = qb;
        wa = va;
        wb = vb;
    }
}

__device__ __forceinline__ void route_spikes(const RouteParams& RP, const int32_t* __restrict__ st,
                                             const int32_t* __restrict__ ix, int64_t n, int64_t warp, int64_t nw)
{
    const int lane = threadIdx.x & 31;
    for (int64_t sp = warp; sp < n; sp += nw)
        route_one(RP, __ldcg(ix + sp), __ldcg(st + sp), lane);
}

// The same delivery split into items of (spike, 256-synapse segment): item
// x is segment x mod segs of spike x / segs (segments past the row's end are
// empty).  Warp r of nR takes items r, r + nR, ...; the split keeps one
// spike's fan-out from serialising on a single warp.
__device__ __forceinline__ void route_items(const RouteParams& RP, const int32_t* __restrict__ st,
                                            const int32_t* __restrict__ ix, int64_t n, int64_t r, int64_t nR)
{
    const int lane = threadIdx.x & 31;
    const int32_t S = RP.segs;
    if (S < 1 || r >= n * S)
        return;
    int64_t sp = r / S;
    int32_t q = (int32_t)(r - sp * S);
    const int64_t dsp = nR / S;
    const int32_t dq = (int32_t)(nR - dsp * S);
    for (; sp < n;) {
        const int32_t j = __ldcg(ix + sp);
        const int32_t t = __ldcg(st + sp);
        if (j >= 0 && j < RP.N && t >= 0) {
            const int64_t e0 = RP.out_ptr[j], e1 = RP.out_ptr[j + 1];
            const int64_t base = (e0 & ~(int64_t)3) + 256 * (int64_t)q;
            const int64_t row = RP.open_loop ? (int64_t)t + RP.D : ((int64_t)t + RP.D) % RP.R;
            if (base < e1 && (!RP.open_loop || row < RP.n_window)) {
                unsigned long long* dst = route_dst(RP, j, row);
                int4 pa, pb;
                float4 wa, wb;
                load_chunk(RP, base + 4 * lane, e1, pa, pb, wa, wb);
                deliver_chunk(dst, RP.stride, base + 4 * lane, e0, e1, pa, pb, wa, wb);
            }
        }
        sp += dsp;
        q += dq;
        if (q >= S) {
            q -= S;
            ++sp;
        }
    }
}

// Pull routing of a dense window: the same sums as the push above (fixed-
// point addition is exact, so the order does not matter).  Every row of the
// in-CSR (rows = postsynaptic neuron) is read once.  When a good part of the
// network spikes in one window, streaming the in-CSR (8 bytes a synapse)
// costs less than one L2 atomic per synaptic event.
//   a. every block stages the window's last-spike table, with the
//      presynaptic type in bit 7, in shared memory;
//   b. warp per target row: the row's records (presynaptic index and
//      weight) are streamed (8 synapses a lane, 256-synapse chunks, two
//      chunks ahead, across row ends);
//      a synapse whose source spiked adds its fixed-point weight to the
//      warp's shared-memory sum for (spike step, E/I) (in the lane's copy),
//      and the row's nonzero sums go to the delay line, one 64-bit atomic
//      each;
//   c. spikes that are not the last of their neuron in the window (a neuron
//      that fired twice) are pushed.
// Entered by whole blocks (the condition is uniform over the grid).

// bit 7 of every byte of x that is nonzero
__device__ __forceinline__ uint32_t nonzero_bytes_b7(uint32_t x)
{
    return (((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;
}

// One 256-synapse chunk of a row in flight: the lane's 8 records from ea =
// base + 8 lane (zeros past the row; the records are padded by 8).  The
// loads are volatile so that they are issued here, two chunks ahead of
// their use, and not moved to the uses behind the spike test.
struct PullChunk {
    uint4 r[4];               // records ea .. ea + 7, two per vector
    int64_t i, e0, e1, base;  // row, its bounds, chunk start (i < 0: none)
};

__device__ __forceinline__ void pull_issue(const RouteParams& RP, int64_t i, int64_t e0, int64_t e1, int64_t base,
                                           int lane, PullChunk& c)
{
    c.i = i;
    c.e0 = e0;
    c.e1 = e1;
    c.base = base;
    const int64_t ea = base + 8 * lane;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c.r[q] = make_uint4(0, 0, 0, 0);
        if (ea < e1) {
            const uint2* pr = RP.in_rec + ea + 2 * q;
            asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(c.r[q].x), "=r"(c.r[q].y), "=r"(c.r[q].z), "=r"(c.r[q].w)
                         : "l"(pr));
        }
    }
}

// The chunk cursor of a warp over its rows i0, i0 + nw, ... (empty rows
// skipped), with the bounds of the row after the current one read ahead.
struct PullCursor {
    int64_t i, e0, e1, base;  // next chunk to issue (i >= N: done)
    int64_t ni, ne0, ne1;     // the row after i
};

__device__ __forceinline__ void pull_row_bounds(const RouteParams& RP, int64_t i, int64_t& e0, int64_t& e1)
{
    e0 = 0;
    e1 = 0;
    if (i < RP.N) {
        e0 = __ldg(RP.in_ptr + i);
        e1 = __ldg(RP.in_ptr + i + 1);
    }
}

__device__ __forceinline__ void pull_advance_row(const RouteParams& RP, int64_t nw, PullCursor& k)
{
    for (;;) {
        k.i = k.ni;
        k.e0 = k.ne0;
        k.e1 = k.ne1;
        k.base = k.e0 & ~(int64_t)7;
        k.ni = k.i + nw;
        pull_row_bounds(RP, k.ni, k.ne0, k.ne1);
        if (k.i >= RP.N || k.base < k.e1)
            return;
    }
}

// issue the cursor's chunk into c and advance the cursor
__device__ __forceinline__ void pull_next(const RouteParams& RP, int64_t nw, int lane, PullCursor& k, PullChunk& c)
{
    if (k.i >= RP.N) {
        c.i = -1;
        return;
    }
    pull_issue(RP, k.i, k.e0, k.e1, k.base, lane, c);
    k.base += 256;
    if (k.base >= k.e1)
        pull_advance_row(RP, nw, k);
}

// records lo .. hi - 1 of a lane's 8 belong to the row
__device__ __forceinline__ void pull_chunk(const uint8_t* tab, uint32_t* mine, int32_t lo, int32_t hi,
                                           const uint4 (&r)[4])
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t x = (q & 1) ? r[q >> 1].z : r[q >> 1].x;
        const uint32_t y = (q & 1) ? r[q >> 1].w : r[q >> 1].y;
        const uint32_t v = tab[x & 0xffffu];  // index < N: another row's record or padding 0
        if (q >= lo && q < hi && v != kPullNone) {
            uint32_t* a = mine + 3 * (2 * (v & 63u) + (v >> 7));
            atomicAdd(a, x >> 16);
            atomicAdd(a + 1, y & 0xffffu);
            atomicAdd(a + 2, y >> 16);
        }
    }
}

__device__ __forceinline__ void route_pull(const RouteParams& RP, const int32_t* __restrict__ st,
                                           const int32_t* __restrict__ ix, int64_t n, int64_t t0, int32_t W,
                                           int32_t lslot, unsigned char* smem)
{
    const int64_t N = RP.N;
    const int64_t Np = pull_stride(N);
    const int lane = threadIdx.x & 31;
    const int32_t rs = pull_copy_words(RP.pull_w);
    uint8_t* tab = smem;
    uint32_t* acc = reinterpret_cast<uint32_t*>(smem + Np) + (threadIdx.x >> 5) * kPullRep * rs;
    uint32_t* mine = acc + (lane % kPullRep) * rs;
    // a. 16 entries per load (tables and inh hold Np entries)
    const uint4* last = reinterpret_cast<const uint4*>(RP.last_spk + (int64_t)lslot * Np);
    const uint4* inh = reinterpret_cast<const uint4*>(RP.inh);
    for (int64_t q = threadIdx.x; q < Np / 16; q += blockDim.x) {
        uint4 v = __ldcg(last + q);
        if (inh) {  // sets bit 7 of an inhibitory neuron's entry; kPullNone stays
            const uint4 h = __ldg(inh + q);
            v.x |= nonzero_bytes_b7(h.x);
            v.y |= nonzero_bytes_b7(h.y);
            v.z |= nonzero_bytes_b7(h.z);
            v.w |= nonzero_bytes_b7(h.w);
        }
        reinterpret_cast<uint4*>(tab)[q] = v;
    }
    for (int q = lane; q < kPullRep * rs; q += 32)
        acc[q] = 0u;
    __syncthreads();
    // b.
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the row's sums (all copies) to the delay line, then cleared
    auto flush = [&](int64_t i) {
        __syncwarp();
        for (int q = lane; q < 2 * W; q += 32) {
            unsigned long long a = 0ull;
#pragma unroll
            for (int r = 0; r < kPullRep; ++r) {
                uint32_t* c = acc + r * rs + 3 * q;
                a += (unsigned long long)c[0] + ((unsigned long long)c[1] << 16) + ((unsigned long long)c[2] << 32);
                c[0] = 0u;
                c[1] = 0u;
                c[2] = 0u;
            }
            if (a) {
                const int64_t row = (t0 + (q >> 1) + RP.D) % RP.R;
                atomicAdd(reinterpret_cast<unsigned long long*>((q & 1) ? RP.ringI : RP.ringE) +
                              (row * N + i) * RP.stride,
                          a);
            }
        }
        __syncwarp();
    };
    auto use = [&](const PullChunk& c) {
        const int64_t ea = c.base + 8 * lane;
        const int32_t lo = (int32_t)max(min(c.e0 - ea, (int64_t)8), (int64_t)0);
        const int32_t hi = (int32_t)max(min(c.e1 - ea, (int64_t)8), (int64_t)0);
        pull_chunk(tab, mine, lo, hi, c.r);
        if (c.base + 256 >= c.e1)  // the row's last chunk
            flush(c.i);
    };
    // a stream of chunks over the warp's rows, two chunks in flight (also
    // across row ends)
    PullCursor k;
    k.ni = warp;
    pull_row_bounds(RP, k.ni, k.ne0, k.ne1);
    pull_advance_row(RP, nw, k);
    PullChunk A, B;
    pull_next(RP, nw, lane, k, A);
    pull_next(RP, nw, lane, k, B);
    while (A.i >= 0) {
        use(A);
        pull_next(RP, nw, lane, k, A);
        if (B.i < 0)
            break;
        use(B);
        pull_next(RP, nw, lane, k, B);
    }
    // c. 32 list entries per warp and round
    for (int64_t b0 = warp * 32; b0 < n; b0 += nw * 32) {
        const int64_t sp = b0 + lane;
        int32_t j = -1, t = -1;
        bool extra = false;
        if (sp < n) {
            j = __ldcg(ix + sp);
            t = __ldcg(st + sp);
            if (j >= 0 && j < N && t >= 0) {
                const uint32_t v = tab[j];
                extra = t < t0 || t >= t0 + W || v == kPullNone || (int64_t)(v & 63u) != t - t0;
            }
        }
        unsigned m = __ballot_sync(kFull, extra);
        while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1;
            route_one(RP, __shfl_sync(kFull, j, l), __shfl_sync(kFull, t, l), lane);
        }
    }
}

// -------------------------------------------------------------------------
// Kernel bodies.  `Dyn` supplies the neuron model(s):
//   dyn.template load<MAXG, PREC>(mid, P, i, s)  per-neuron conductances
//   dyn.template step<MAXG, PREC>(mid, dt, v_update, I, gsE, EE, gsI, EI, s)
//   Dyn::kDrive, Dyn::kCable, Dyn::kSynCurrent, Dyn::kCompound  whether the
//       kernel carries the sinusoidal drive, the axial coupling, current-based
//       synapses and the compound background (the run-time compiled kernels
//       only for networks that use them)
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
    const float4* tab = stage_poly<PREC>(P);
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < P.N;
    const int64_t i = valid ? gi : 0;
    const int mid = P.model_id ? P.model_id[i] : 0;
    State<MAXG, PREC> s;
    s.poly = tab;
    load_state(P, i, s);
    dyn.template load<MAXG, PREC>(mid, P, i, s);
    const float Ic = P.I_const ? P.I_const[i] : 0.0f;
    int32_t slot = -1;
    if (R.V_trace)
        slot = P.trace_slot ? P.trace_slot[i] : (i < R.n_trace ? (int32_t)i : -1);
    if (!valid)
        slot = -1;
    const Drive dr = Dyn::kDrive ? load_drive(P, i) : Drive{0.0f, 0u, 0u};
    const Axial ax = axial_setup(P);
    int32_t cnt = 0;
    for (int32_t k = 0; k < n_steps; ++k) {
        float I = Ic + (I_steps ? I_steps[(int64_t)k * P.N + i] : 0.0f);
        if (Dyn::kDrive && P.sin_amp)
            I += drive_at<sfu_math<PREC>()>(dr, t0 + k);
        if (Dyn::kCable && P.cable_nd > 0)
            I += axial_current(ax, s.V);
        const float Vt = s.V;
        dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, I, 0.0f, 0.0f, 0.0f, 0.0f, s);
        const bool spk = valid && Vt < P.theta && s.V >= P.theta;
        cnt += spk;
        record_spikes(spk, (int32_t)(t0 + k), (int32_t)i, P.theta, Vt, s.V, R, P.status);
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
    s.poly = P.poly;  // (the surrogate's networks do not use HH_PREC_POLY)
    load_state(P, i, s);
    dyn.template load<MAXG, PREC>(mid, P, i, s);
    const float Ic = P.I_const ? P.I_const[i] : 0.0f;
    int32_t cnt = 0;
    for (int32_t k = 0; k < n_steps; ++k) {
        const float Vt = s.V;
        dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, Ic, 0.0f, 0.0f, 0.0f, 0.0f, s);
        const bool spk = valid && Vt < P.theta && s.V >= P.theta;
        cnt += spk;
        record_spikes(spk, (int32_t)(t0 + k), (int32_t)i, P.theta, Vt, s.V, R, P.status);
    }
    if (valid) {
        store_state(P, i, s);
        if (R.counts && cnt)
            R.counts[i] += cnt;
        if (!finite(s.V))
            atomicOr(P.status, HH_STATUS_NONFINITE);
    }
}

// The delay-line entries of the next kRingAhead steps of one neuron, in
// flight in registers ({E, I} per step: one 16-byte load each).  Slots past
// the window are read and discarded; inside it the slots are distinct (W <=
// R) and only cleared after their own step.
struct RingQueue {
    longlong2 q[kRingAhead];
    uint32_t ring_slot;  // slot of the next step
    uint32_t far_slot;   // slot of the next load
};

__device__ __forceinline__ longlong2* ring_entry(const NeuronParams& P, uint32_t slot, int64_t i)
{
    return reinterpret_cast<longlong2*>(P.ring) + (slot * (uint32_t)P.N + (uint32_t)i);
}

__device__ __forceinline__ void ring_preload(const NeuronParams& P, int64_t i, int64_t t0, RingQueue& rq)
{
    rq.ring_slot = (uint32_t)(t0 % P.R);
    rq.far_slot = rq.ring_slot;
#pragma unroll
    for (int a = 0; a < kRingAhead; ++a) {
        rq.q[a] = __ldcg(ring_entry(P, rq.far_slot, i));
        rq.far_slot = rq.far_slot + 1 == (uint32_t)P.R ? 0u : rq.far_slot + 1;
    }
}

// W <= D time steps of one network neuron with its state in registers.
// The delay-line slots of the window were completed by earlier routing;
// they are read through L2 (.cg: they were written by atomics from other
// blocks) kRingAhead steps ahead (rq, preloaded by the caller), and cleared
// after use.  Spikes go to list slot `lslot` (and to the caller's record).
// `between(k)` runs after step k with the whole warp (all lanes, valid or
// not): the persistent kernel routes part of the previous window there.
struct NoWork {
    __device__ __forceinline__ void operator()(int32_t) const {}
};
template <int MAXG, int PREC, bool BG, bool CB, int GROUP, class Dyn, class Between>
__device__ __forceinline__ void window_steps_bg(const Dyn& dyn, int mid, const NeuronParams& P, bool valid,
                                                int64_t i, int64_t t0, int32_t W,
                                                const float* __restrict__ I_steps, const RecordParams& R,
                                                float* V_trace, int32_t slot, const SpikeList& L, int32_t lslot,
                                                State<MAXG, PREC>& s, float& gE, float& gI, float Ic,
                                                const Drive& dr, int32_t& cnt, RingQueue& rq,
                                                const Between& between)
{
    const Axial ax = axial_setup(P);
    int32_t* lstep = L.step + lslot * L.cap;
    int32_t* lidx = L.idx + lslot * L.cap;
    // one step; `word` is the background word of step t0 + k and `z` its
    // standard normal (compound background)
    auto step = [&](int32_t k, uint32_t word, float z) {
        const int64_t t = t0 + k;
        const long long e = rq.q[0].x, h = rq.q[0].y;
#pragma unroll
        for (int a = 0; a + 1 < kRingAhead; ++a)
            rq.q[a] = rq.q[a + 1];
        rq.q[kRingAhead - 1] = __ldcg(ring_entry(P, rq.far_slot, i));
        rq.far_slot = rq.far_slot + 1 == (uint32_t)P.R ? 0u : rq.far_slot + 1;
        // a. delayed synaptic input (fixed point 2^-32 nS) and background
        // (added unconditionally: + 0 changes no bit, and the step stays
        // free of branches the scheduler cannot look across).  The
        // conductance arithmetic that crosses steps is written with explicit
        // rounding, so that no copy of the step fuses the previous step's
        // decay into this addition: every copy gives the same bits.
        gE = __fadd_rn(gE, fixed_to_nS(e));
        gI = __fadd_rn(gI, fixed_to_nS(h));
        if (valid && (e | h))
            *ring_entry(P, rq.ring_slot, i) = make_longlong2(0, 0);
        rq.ring_slot = rq.ring_slot + 1 == (uint32_t)P.R ? 0u : rq.ring_slot + 1;
        if (BG) {
            const float kb = (float)poisson_count(word, P.bg_thr, P.bg_n);
            if (CB)  // the sum of k Gaussian amplitudes: N(k w, k sd^2)
                gE = __fadd_rn(gE, fmaf(sqrtf(kb) * P.bg_sd, z, kb * P.bg_w));
            else
                gE = fmaf(kb, P.bg_w, gE);
        }
        float I = Ic + (I_steps ? I_steps[(int64_t)k * P.N + i] : 0.0f);
        if (Dyn::kDrive && P.sin_amp)
            I += drive_at<sfu_math<PREC>()>(dr, t);
        if (Dyn::kCable && P.cable_nd > 0)
            I += axial_current(ax, s.V);
        const float Vt = s.V;
        if (Dyn::kSynCurrent && P.syn_current)
            dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, __fadd_rn(I, __fsub_rn(gE, gI)), 0.0f, 0.0f, 0.0f,
                                          0.0f, s);
        else
            dyn.template step<MAXG, PREC>(mid, P.dt, P.v_update, I, __fmul_rn(gE, P.to_mS), P.E_E,
                                          __fmul_rn(gI, P.to_mS), P.E_I, s);
        const bool spk = valid && Vt < P.theta && s.V >= P.theta;
        cnt += spk;
        // one ballot for the window list and the caller's record
        const unsigned b = __ballot_sync(kFull, spk);
        if (b) {
            list_append_b(b, spk, (int32_t)t, (int32_t)i, L.counter + lslot, lstep, lidx, L.cap);
            record_spikes_b(b, spk, (int32_t)t, (int32_t)i, P.theta, Vt, s.V, R, P.status);
            if (spk && P.last_spk)
                P.last_spk[lslot * pull_stride(P.N) + i] = (uint8_t)k;
        }
        if (slot >= 0)
            V_trace[(int64_t)k * R.n_trace + slot] = s.V;
        gE = __fmul_rn(gE, P.decE);
        gI = __fmul_rn(gI, P.decI);
        between(k);
    };
    // The background words of steps 4q..4q+3 come from one Philox block
    // (counter q).
    auto draw = [&](int64_t t) {
        uint4 r = make_uint4(0, 0, 0, 0);
        if (BG) {
            const uint64_t q = (uint64_t)t >> 2;
            r = philox4x32_10_rk(make_uint4((uint32_t)q, (uint32_t)i, 1u, (uint32_t)(q >> 32)), P.rk);
        }
        return r;
    };
    // the block of normals of steps 4q..4q+3 (compound background)
    auto normals = [&](int64_t t) {
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (CB)
            z = bg_normals<sfu_math<PREC>()>((uint64_t)t >> 2, i, P.rk);
        return z;
    };
    if (GROUP != 4) {
        // one step per iteration, the block drawn at its first step (the
        // smaller loop body, for models whose step is long)
        uint4 r = make_uint4(0, 0, 0, 0);
        float4 zz = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll kRingAhead
        for (int32_t k = 0; k < W; ++k) {
            const int64_t t = t0 + k;
            if (BG && (k == 0 || (t & 3) == 0)) {
                r = draw(t);
                zz = normals(t);
            }
            step(k, pick(r, (int)(t & 3)), pickf(zz, (int)(t & 3)));
        }
        return;
    }
    // GROUP == 4: steps grouped by Philox block, so inside a group the draw
    // is not behind a branch and overlaps the first step's gates.  (Drawing
    // the next group's block one group ahead was measured slower: 10.4 ->
    // 10.8 us per 20-step window.)
    int32_t k = 0;
    const int32_t head = min(W, (int32_t)((4 - (t0 & 3)) & 3));
    if (head > 0) {
        const uint4 r = draw(t0);
        const float4 zz = normals(t0);
        for (; k < head; ++k)
            step(k, pick(r, (int)((t0 + k) & 3)), pickf(zz, (int)((t0 + k) & 3)));
    }
    // unrolled by four steps, a multiple of the queue depth, so that the
    // queue rotates by renaming registers instead of moving values whose
    // loads are still in flight
    static_assert(4 % kRingAhead == 0, "group of four steps");
#pragma unroll 1
    for (; k + 4 <= W; k += 4) {
        const uint4 r = draw(t0 + k);
        const float4 zz = normals(t0 + k);
        step(k, r.x, zz.x);
        step(k + 1, r.y, zz.y);
        step(k + 2, r.z, zz.z);
        step(k + 3, r.w, zz.w);
    }
    if (k < W) {
        const uint4 r = draw(t0 + k);
        const float4 zz = normals(t0 + k);
        for (; k < W; ++k)
            step(k, pick(r, (int)((t0 + k) & 3)), pickf(zz, (int)((t0 + k) & 3)));
    }
}

// GROUP: 4 = steps grouped by background block (short model steps), 1 = one
// step per iteration (long model steps: the four-step body would not stay in
// the instruction cache).  Both run the same step arithmetic.
template <int MAXG, int PREC, int GROUP, class Dyn, class Between>
__device__ __forceinline__ void window_steps(const Dyn& dyn, int mid, const NeuronParams& P, bool valid,
                                             int64_t i, int64_t t0, int32_t W, const float* __restrict__ I_steps,
                                             const RecordParams& R, float* V_trace, int32_t slot,
                                             const SpikeList& L, int32_t lslot, State<MAXG, PREC>& s,
                                             float& gE, float& gI, float Ic, const Drive& dr, int32_t& cnt,
                                             RingQueue& rq, const Between& between)
{
    if (P.bg_n > 0 && Dyn::kCompound && P.bg_sd > 0.0f)
        window_steps_bg<MAXG, PREC, true, Dyn::kCompound, GROUP>(dyn, mid, P, valid, i, t0, W, I_steps, R,
                                                                 V_trace, slot, L, lslot, s, gE, gI, Ic, dr, cnt,
                                                                 rq, between);
    else if (P.bg_n > 0)
        window_steps_bg<MAXG, PREC, true, false, GROUP>(dyn, mid, P, valid, i, t0, W, I_steps, R, V_trace, slot,
                                                        L, lslot, s, gE, gI, Ic, dr, cnt, rq, between);
    else
        window_steps_bg<MAXG, PREC, false, false, GROUP>(dyn, mid, P, valid, i, t0, W, I_steps, R, V_trace, slot,
                                                         L, lslot, s, gE, gI, Ic, dr, cnt, rq, between);
}

// Network window: W <= D steps; spikes go to the window list for routing.
// The input of every step in the window comes from spikes at least D steps
// earlier, already routed by previous launches, so neurons are independent
// inside the window.
// early != 0: the launch follows the pipelined schedule, in which the
// delay-line slots of this window were completed by routing launches that
// the stream waited for with full event dependencies, and no kernel that
// may still be running writes them; the first slots are then read before
// the programmatic wait, overlapping their latency with the previous
// window's tail.
template <int MAXG, int PREC, int GROUP, class Dyn>
__device__ __forceinline__ void window_body(const Dyn& dyn, const NeuronParams& P, int64_t t0,
                                            int32_t W, const float* __restrict__ I_steps,
                                            const RecordParams& R, const SpikeList& L, int32_t parity,
                                            int32_t early)
{
    const float4* tab = stage_poly<PREC>(P);  // constant tables: before the programmatic wait
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < P.N;
    const int64_t i = valid ? gi : 0;
    RingQueue rq;
    if (early)
        ring_preload(P, i, t0, rq);
    // Programmatic dependent launch (when the launch asks for it; no-ops
    // otherwise): the next window's blocks may be scheduled now, and this
    // window waits for the previous kernel of the stream to complete before
    // it touches the state that kernel wrote.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (!early)
        ring_preload(P, i, t0, rq);
    if (gi == 0)
        L.counter[parity + 1 == kListSlots ? 0 : parity + 1] = 0;  // next window's slot (its reader has finished)
    if (valid && P.last_spk)
        P.last_spk[parity * pull_stride(P.N) + i] = kPullNone;  // its reader finished before this launch
    const int mid = P.model_id ? P.model_id[i] : 0;
    State<MAXG, PREC> s;
    s.poly = tab;
    load_state(P, i, s);
    dyn.template load<MAXG, PREC>(mid, P, i, s);
    float gE = P.gE[i], gI = P.gI[i];
    const float Ic = P.I_const ? P.I_const[i] : 0.0f;
    int32_t slot = -1;
    if (R.V_trace)
        slot = P.trace_slot ? P.trace_slot[i] : (i < R.n_trace ? (int32_t)i : -1);
    if (!valid)
        slot = -1;
    const Drive dr = Dyn::kDrive ? load_drive(P, i) : Drive{0.0f, 0u, 0u};
    int32_t cnt = 0;
    window_steps<MAXG, PREC, GROUP>(dyn, mid, P, valid, i, t0, W, I_steps, R, R.V_trace, slot, L, parity, s, gE, gI,
                                    Ic, dr, cnt, rq, NoWork{});
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

// Progress counters of the persistent kernel (zeroed before each launch).
// Window w counts in slot w mod kPhaseSlots of `done` once per neuron block
// that finished it and of `routed` once per block whose routing warps
// delivered their share of it;
// window w is complete when its slot reaches (w / kPhaseSlots + 1) x the
// number of blocks or warps.  This is exact because no block or warp gets
// more than two windows ahead of the slowest one (see persistent_body), so
// a slot never holds a contribution from a later window than the one
// waited for.  Waits are bounded by the global timer (pc.limit_ns,
// kWaitLimitNs by default); on expiry the waiter records
// HH_STATUS_BARRIER_TIMEOUT and gives up.
constexpr int kPhaseSlots = 4;
struct PhaseCounters {
    unsigned long long* done;    // [kPhaseSlots], one count per neuron block
    unsigned long long* routed;  // [kPhaseSlots], one count per block's routing warps (own 128-B line)
    unsigned long long limit_ns; // bound of every wait (kWaitLimitNs by default)
};
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
// default bound of a tensor-core pipeline's mbarrier wait, in polls
constexpr long long kWaitLimitPolls = 1ll << 24;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool wait_at_least(const unsigned long long* c, unsigned long long target,
                                              int32_t* status, unsigned long long limit_ns)
{
    const volatile unsigned long long* p = c;
    if (*p < target) {
        const unsigned long long t0 = global_ns();
        unsigned ns = 32;  // back-off: few pollers on a line every other SM reads
        while (*p < target) {
            if (global_ns() - t0 > limit_ns) {
                atomicOr(status, HH_STATUS_BARRIER_TIMEOUT);
                return false;
            }
            __nanosleep(ns);
            ns = ns < 1024 ? 2 * ns : ns;
        }
    }
    __threadfence();
    return true;
}

__device__ __forceinline__ unsigned long long signal_done(unsigned long long* c)
{
    __threadfence();
    return atomicAdd(c, 1ull);
}

// The persistent kernel's block: kPersistNeurons neuron threads (warps 0-3)
// and kPersistRouters routing warps.  Barrier 1 spans the neuron threads
// only (the routing warps never wait on it).
constexpr int kPersistNeurons = 128;
constexpr int kPersistRouters = 4;
constexpr int kPersistThreads = kPersistNeurons + 32 * kPersistRouters;
constexpr int kPersistWarps = kPersistThreads / 32;

__device__ __forceinline__ void neuron_bar()
{
    asm volatile("barrier.sync 1, %0;" ::"n"(kPersistNeurons) : "memory");
}
// Barrier 2 spans the block's routing warps.
__device__ __forceinline__ void router_bar()
{
    asm volatile("barrier.sync 2, %0;" ::"n"(32 * kPersistRouters) : "memory");
}
__device__ __forceinline__ bool router_all(bool p)
{
    int r;
    asm volatile("{\n\t.reg .pred a, b;\n\tsetp.ne.s32 a, %1, 0;\n\tbarrier.red.and.pred b, 2, %2, a;\n\t"
                 "selp.s32 %0, 1, 0, b;\n\t}"
                 : "=r"(r)
                 : "r"((int)p), "n"(32 * kPersistRouters)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ bool neuron_all(bool p)
{
    int r;
    asm volatile("{\n\t.reg .pred a, b;\n\tsetp.ne.s32 a, %1, 0;\n\tbarrier.red.and.pred b, 1, %2, a;\n\t"
                 "selp.s32 %0, 1, 0, b;\n\t}"
                 : "=r"(r)
                 : "r"((int)p), "n"(kPersistNeurons)
                 : "memory");
    return r != 0;
}

// The whole n_steps of a network in one cooperative launch (windows of
// W <= D/2 steps, call-local window w in list slot (w_index0 + w) mod 3).
// Dataflow instead of a grid barrier:
//  - a neuron block integrates window w once the routing warps of every
//    block have routed window w - 2 (the input of window w comes from spikes
//    at least D >= 2W steps earlier, i.e. from windows <= w - 2; routing
//    goes in window order), then counts itself done with w;
//  - a block's routing warps deliver their share of window w once every
//    neuron block is done with it, then the block counts itself.  The
//    targets lie in windows >= w + 2, whose delay-line slots are disjoint
//    from those of the windows integrated meanwhile (w + 1 at most: a block
//    in w + 2 waits for w to be routed);
//  - the last window is routed by every warp of the grid once all blocks
//    are done with it.
// So a block in window k implies all blocks done with k - 2, and routing of
// window k implies all blocks done routing k - 2: nothing runs more than two
// windows ahead of the slowest block.
// The three list counters are zero at launch; the last block to finish
// routing window w clears its slot, which window w + 3 reuses: a block
// starting w + 3 has waited for window w + 1 to be routed, which that block
// signals after the clear.
template <int MAXG, int PREC, int GROUP, class Dyn>
__device__ __forceinline__ void persistent_body(const Dyn& dyn, const NeuronParams& P, const RouteParams& RP,
                                                int64_t t0, int32_t n_steps, int32_t W, int64_t w_index0,
                                                const float* __restrict__ I_steps, const RecordParams& R,
                                                const SpikeList& L, const PhaseCounters& pc)
{
    const float4* tab = stage_poly<PREC>(P);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int32_t n_win = (n_steps + W - 1) / W;
    const unsigned long long n_blocks = gridDim.x;
    const unsigned long long nR = (unsigned long long)gridDim.x * kPersistRouters;
    auto list_count = [&](int32_t w) -> int64_t {
        const int64_t n = __ldcg(L.counter + (int32_t)((w_index0 + w) % kListSlots));
        return n > L.cap ? L.cap : n;
    };
    auto list_step = [&](int32_t w) { return L.step + (int32_t)((w_index0 + w) % kListSlots) * L.cap; };
    auto list_idx = [&](int32_t w) { return L.idx + (int32_t)((w_index0 + w) % kListSlots) * L.cap; };
    auto window_done = [&](int32_t w, unsigned long long* c, unsigned long long per) {
        return wait_at_least(c + w % kPhaseSlots, (unsigned long long)(w / kPhaseSlots + 1) * per, P.status,
                             pc.limit_ns);
    };
    bool ok = true;
    if (threadIdx.x >= kPersistNeurons) {
        // the block's routing warps wait and signal together: one poller and
        // one count per block
        const bool lead = threadIdx.x == kPersistNeurons;
        const int64_t r = (int64_t)blockIdx.x * kPersistRouters + (warp - kPersistNeurons / 32);
        for (int32_t w = 0; w + 1 < n_win; ++w) {
            bool go = true;
            if (lead)
                go = window_done(w, pc.done, n_blocks);
            if (!router_all(go))
                return;
            route_items(RP, list_step(w), list_idx(w), list_count(w), r, (int64_t)nR);
            router_bar();
            // the last block to finish window w frees its list slot for window w + 3
            if (lead && signal_done(pc.routed + w % kPhaseSlots) + 1 ==
                            (unsigned long long)(w / kPhaseSlots + 1) * n_blocks)
                L.counter[(int32_t)((w_index0 + w) % kListSlots)] = 0;
        }
        bool go = true;
        if (lead && n_win >= 1)
            go = window_done(n_win - 1, pc.done, n_blocks);
        ok = router_all(go);
    } else {
        const int64_t gi = (int64_t)blockIdx.x * kPersistNeurons + threadIdx.x;
        const bool valid = gi < P.N;
        const int64_t i = valid ? gi : 0;
        const int mid = P.model_id ? P.model_id[i] : 0;
        State<MAXG, PREC> s;
        s.poly = tab;
        load_state(P, i, s);
        dyn.template load<MAXG, PREC>(mid, P, i, s);
        float gE = P.gE[i], gI = P.gI[i];
        const float Ic = P.I_const ? P.I_const[i] : 0.0f;
        int32_t slot = -1;
        if (R.V_trace && valid)
            slot = P.trace_slot ? P.trace_slot[i] : (i < R.n_trace ? (int32_t)i : -1);
        const Drive dr = Dyn::kDrive ? load_drive(P, i) : Drive{0.0f, 0u, 0u};
        int32_t cnt = 0;
        for (int32_t w = 0; w < n_win; ++w) {
            if (w >= 2) {
                bool go = true;
                if (threadIdx.x == 0)
                    go = window_done(w - 2, pc.routed, n_blocks);
                if (!neuron_all(go)) {
                    ok = false;
                    break;
                }
            }
            const int32_t Ww = min(W, n_steps - w * W);
            RingQueue rq;
            ring_preload(P, i, t0 + (int64_t)w * W, rq);
            window_steps<MAXG, PREC, GROUP>(dyn, mid, P, valid, i, t0 + (int64_t)w * W, Ww,
                                            I_steps ? I_steps + (int64_t)w * W * P.N : nullptr, R,
                                            R.V_trace ? R.V_trace + (int64_t)w * W * R.n_trace : nullptr, slot, L,
                                            (int32_t)((w_index0 + w) % kListSlots), s, gE, gI, Ic, dr, cnt, rq,
                                            NoWork{});
            neuron_bar();
            if (threadIdx.x == 0)
                signal_done(pc.done + w % kPhaseSlots);
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
        if (!ok)
            return;
        bool go = true;
        if (threadIdx.x == 0 && n_win >= 1)
            go = window_done(n_win - 1, pc.done, n_blocks);
        ok = neuron_all(go);
    }
    if (!ok || n_win < 1)
        return;
    // the last window, with every warp of the grid
    route_items(RP, list_step(n_win - 1), list_idx(n_win - 1), list_count(n_win - 1),
                (int64_t)blockIdx.x * kPersistWarps + warp, (int64_t)gridDim.x * kPersistWarps);
}

#endif  // __CUDACC__ || __CUDACC_RTC__

}  // namespace hh
