/*
 * hh.h -- C ABI of libhh, the GB300 (sm_103a) Hodgkin-Huxley hot path.
 *
 * The library advances populations and networks of conductance-based
 * Hodgkin-Huxley point neurons with hand-written CUDA kernels:
 *   - voltage-dependent alpha/beta (or p_inf/tau) rate functions and the
 *     exponential-Euler gate update of every channel gate
 *     (Methods, Eq. hh_eq_full, second line; "Simplified discretization");
 *   - membrane integration C_m dV/dt = I - sum_X gbar_X eta_X(p)(V - E_X)
 *     - g_E (V - E_E) - g_I (V - E_I) with the conductances frozen over the
 *     step (exponential Euler), or explicit Euler (Eq. hh_dyn_simplified);
 *   - upward threshold crossing (spike) detection with linear interpolation
 *     of the crossing time;
 *   - exponential synaptic conductances (E/IPSP filters) fed through a
 *     fixed synaptic delay by spike propagation over a CSR graph, plus a
 *     Poisson background drive (Methods, "Cerebral cortex network").
 *
 * Conventions shared by every call
 *   Units: V and E in mV, time in ms, currents in uA/cm^2, membrane
 *   conductances in mS/cm^2, capacitance in uF/cm^2, synaptic weights and
 *   g_E/g_I in nS (1 nS = 1e-6 mS / area_cm2), Ca in uM.
 *   Memory: pointers marked "any memory" may be host (pageable or pinned) or
 *   device pointers; the library copies them during the call (CUDA unified
 *   addressing decides the direction).  Pointers marked "device" must be
 *   device memory that the caller owns and keeps alive until the work queued
 *   on the network's stream has finished.  The library owns all network
 *   state; nothing it allocates is visible to the caller except through
 *   hh_readout.
 *   Streams: every call that launches work enqueues it on the stream given
 *   at creation and returns without waiting, unless stated otherwise.
 *   Errors: every call returns an hh_status; no exception or signal crosses
 *   the ABI.  hh_last_error() gives a thread-local message for the last
 *   failure of the calling thread.  Asynchronous CUDA errors and device-side
 *   status bits (spike-buffer overflow, non-finite V) are reported by the
 *   next call that synchronises, and by hh_readout(HH_READ_STATUS).
 *   Determinism: results depend only on the inputs and the seed.  Synaptic
 *   input is accumulated in 64-bit fixed point (units of 2^-32 nS), so the
 *   order in which spikes are delivered does not change any bit.
 */
#ifndef HH_H
#define HH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hh_net hh_net; /* opaque; created by hh_create_network */

typedef enum {
    HH_OK = 0,
    HH_EINVAL = 1,       /* an argument is out of range or inconsistent */
    HH_ENOMEM = 2,       /* a device or host allocation failed */
    HH_ECUDA = 3,        /* a CUDA call failed (message in hh_last_error) */
    HH_ETIMEOUT = 4,     /* a bounded device-side wait gave up */
    HH_ESTATE = 5,       /* the call is not valid in the network's state */
    HH_EUNSUPPORTED = 6, /* the request is valid but not implemented */
    HH_EOVERFLOW = 7     /* a caller buffer was too small (data truncated) */
} hh_status;

/* ------------------------------------------------------------------ */
/* Neuron models (user-defined ion channels)                            */
/* ------------------------------------------------------------------ */

/* Closed forms of a rate function r(V) = c + form(V)   (Methods, Eq.
 * hh_eq_full: "the specific form of eta_X, alpha_p and beta_p depends on
 * the ion X and sub-unit p"):
 *   HH_FN_CONST   a
 *   HH_FN_EXP     a * exp((V - vh)/k)
 *   HH_FN_SIGMOID a / (1 + exp((V - vh)/k))
 *   HH_FN_LINOID  a (V - vh) / (1 - exp(-(V - vh)/k)), equal to a k at V = vh
 *   HH_FN_BELL    a / (exp((V - vh)/k) + exp((V - vh2)/k2))            */
enum { HH_FN_CONST = 0, HH_FN_EXP = 1, HH_FN_SIGMOID = 2, HH_FN_LINOID = 3, HH_FN_BELL = 4 };

/* Gate kinds:
 *   HH_GATE_AB     f1 = alpha(V), f2 = beta(V) in 1/ms;
 *                  p_inf = alpha/(alpha+beta), tau = 1/(alpha+beta)
 *   HH_GATE_INFTAU f1 = p_inf(V), f2 = tau(V) in ms
 *   HH_GATE_CA     p_inf = Ca/(Ca + f1.a), tau = f2(V)  (Ca-dependent) */
enum { HH_GATE_AB = 0, HH_GATE_INFTAU = 1, HH_GATE_CA = 2 };

#define HH_MAX_CHANNELS 8        /* channels per model (leak counts)      */
#define HH_MAX_GATES_PER_CHANNEL 3
#define HH_MAX_GATES 8           /* gates per model, all channels          */
#define HH_MAX_MODELS 4          /* models per network                     */

typedef struct {
    int32_t form; /* HH_FN_* */
    float a, vh, k, vh2, k2, c;
} hh_fn;

typedef struct {
    int32_t kind;  /* HH_GATE_* */
    int32_t power; /* exponent of the gate in eta_X, 1..4 */
    hh_fn f1, f2;
} hh_gate;

typedef struct {
    float E_rev;   /* reversal potential E_X (mV) */
    float gbar;    /* default maximal conductance (mS/cm^2) */
    int32_t n_gates;
    hh_gate gates[HH_MAX_GATES_PER_CHANNEL];
} hh_channel;

/* A point-neuron model: eta_X = prod_g p_g^power_g for each channel, and an
 * optional first-order calcium pool fed by one channel:
 *   d[Ca]/dt = -ca_k I_Ca - ([Ca] - ca_rest)/ca_tau,
 * advanced by exponential Euler with I_Ca evaluated at V_t and the updated
 * gates.  ca_channel = -1 disables the pool. */
typedef struct {
    float C_m; /* uF/cm^2 */
    int32_t n_channels;
    hh_channel channels[HH_MAX_CHANNELS];
    int32_t ca_channel;
    float ca_tau, ca_k, ca_rest;
} hh_model_desc;

/* ------------------------------------------------------------------ */
/* Network creation                                                     */
/* ------------------------------------------------------------------ */

/* Arithmetic of the neuron update.  Every mode forms each update as an
 * increment, p += (p_inf - p)(1 - e^{-z}) and V += (I - I_ion)/G (1 -
 * e^{-dt G/C_m}) with I_ion = sum_X g_X (V - E_X), which is the exponential-
 * Euler map itself; the modes differ in how 1 - e^{-z}, the rates and the
 * divisions are evaluated:
 *   HH_PREC_FAST        FP32 on the SFU: ex2.approx for the exponentials of
 *                       the rate functions, rcp.approx for divisions, and a
 *                       degree-5 Taylor polynomial of 1 - e^{-z} for z < 0.125;
 *   HH_PREC_ACCURATE    FP32 with IEEE division, expf and expm1f;
 *   HH_PREC_COMPENSATED as ACCURATE, on a two-float (hi + lo) state: each
 *                       increment is added by an error-free two-sum, so the
 *                       state keeps the low bits of small increments over
 *                       many steps;
 *   HH_PREC_POLY        polynomial approximation of the rates (Results,
 *                       "BrainFuse": the operators' polynomial
 *                       approximation): hh_set_channels fits, per model and
 *                       gate, p_inf(V) and 1 - e^{-dt/tau(V)} by cubics on
 *                       uniform intervals of [HH_POLY_V_LO, HH_POLY_V_HI)
 *                       mV (Chebyshev interpolation in FP64), halving the
 *                       interval from 1 mV down to 1/8 mV until every
 *                       function's relative error, measured at 64 points
 *                       per interval, is at most HH_POLY_REL_ERR; each step
 *                       then takes one table row per gate instead of the
 *                       rate functions, their division and the exponential
 *                       (HH_READ_POLY gives the interval and the error
 *                       reached).  A warp with any lane outside the range
 *                       takes the FAST arithmetic for that step; V and Ca
 *                       are as in FAST.  Needs HH_KERNELS_SPECIALISED or
 *                       HH_KERNELS_PERSISTENT.                             */
enum { HH_PREC_FAST = 0, HH_PREC_ACCURATE = 1, HH_PREC_COMPENSATED = 2, HH_PREC_POLY = 3 };
#define HH_POLY_V_LO (-120.0f)
#define HH_POLY_V_HI 80.0f
#define HH_POLY_REL_ERR 5e-7f
enum { HH_V_EXP_EULER = 0, HH_V_FWD_EULER = 1 };

/* Neuron kernels:
 *   HH_KERNELS_SPECIALISED  compiled with NVRTC for the installed models at
 *                           the first hh_step_n after hh_set_channels (the
 *                           model table becomes compile-time constants;
 *                           about a second per new model set, cached for the
 *                           life of the process).  A network runs one neuron
 *                           launch per window of delay_steps/2 steps (D >= 2)
 *                           and routes each window on a second stream while
 *                           the next one integrates;
 *   HH_KERNELS_TABLE        precompiled kernels that read the model table at
 *                           run time (no compilation; slower per step), one
 *                           window of delay_steps steps per launch;
 *   HH_KERNELS_PERSISTENT   the compiled kernels of HH_KERNELS_SPECIALISED,
 *                           but a network with synapses and delay_steps >= 2
 *                           whose neurons fit on the GPU at once (128 per
 *                           block, with 4 routing warps each) runs a whole
 *                           hh_step_n call as ONE cooperative launch: the
 *                           routing warps deliver window w - 1 while the
 *                           neuron threads integrate window w, ordered by
 *                           device-side progress counters instead of launch
 *                           boundaries.  Otherwise as HH_KERNELS_SPECIALISED.
 * All run the same device code and give the same results up to the
 * compiler's instruction selection (FMA contraction); SPECIALISED and
 * PERSISTENT give bit-identical results.                                  */
enum { HH_KERNELS_SPECIALISED = 0, HH_KERNELS_TABLE = 1, HH_KERNELS_PERSISTENT = 2 };

typedef struct {
    int64_t n_neurons;          /* N >= 1 (all networks together)            */
    int32_t n_nets;             /* >= 1 independent networks, concatenated     */
    const int64_t* net_offsets; /* host [n_nets+1] neuron offsets, or NULL
                                   when n_nets == 1 (informational: networks
                                   are independent because the CSR graph is
                                   block-diagonal)                            */
    double dt_ms;               /* time step (> 0)                            */
    float v_threshold;          /* spike threshold theta (mV)                 */
    int32_t v_update;           /* HH_V_*                                     */
    int32_t precision;          /* HH_PREC_*                                  */
    int32_t kernels;            /* HH_KERNELS_*                               */
    const float* V0;            /* [N] initial V, any memory (copied)        */
    const float* I_const;       /* [N] constant injected current, any memory,
                                   or NULL for none                            */
    const uint8_t* model_id;    /* [N] model index per neuron (< n models),
                                   any memory, or NULL for model 0             */
    /* synapses: in-CSR by postsynaptic neuron (n_synapses = 0: none) */
    int64_t n_synapses;
    const int64_t* row_ptr;     /* [N+1], any memory; row_ptr[0] = 0,
                                   nondecreasing, row_ptr[N] = n_synapses     */
    const int32_t* col_idx;     /* [n_synapses] presynaptic index in [0, N)   */
    const float* weight;        /* [n_synapses] nS, finite, 0 <= w < 65536    */
    const uint8_t* is_inhibitory; /* [N] presynaptic type (selects tau_I and
                                   E_I), any memory, or NULL: all excitatory  */
    float tau_E, tau_I;         /* ms (> 0)                                   */
    float E_E, E_I;             /* mV                                         */
    int32_t delay_steps;        /* synaptic delay D in steps, 1..1024         */
    float area_cm2;             /* membrane area converting nS to mS/cm^2     */
    /* Poisson background: bg_sources independent sources per neuron, each at
     * bg_rate_hz, every event adding bg_weight_nS to g_E */
    float bg_rate_hz;
    int32_t bg_sources;
    float bg_weight_nS;
    uint64_t seed;              /* Philox key for the background counts       */
    void* stream;               /* cudaStream_t for all work, NULL = legacy   */
    /* sinusoidal drive of frequency-response sweeps (Results, the HH filter
     * bank's response to periodic input): at step t every neuron i gets
     * I_inj += sin_amp[i] sin(2 pi u_i(t) 2^-32) with the phase, a 32-bit
     * fraction of a cycle, u_i(t) = t F_i + P_i (mod 2^32),
     * F_i = round(sin_freq_hz[i] dt_ms 2^32 / 1000), P_i = round(sin_phase[i]
     * 2^32) mod 2^32 (so the phase is exact over any run length).  Any
     * memory, [N]; sin_amp NULL = no drive; sin_phase NULL = 0. */
    const float* sin_amp;       /* uA/cm^2                                     */
    const float* sin_freq_hz;   /* Hz, >= 0 (required with sin_amp)           */
    const float* sin_phase;     /* cycles                                      */
    const struct hh_morphology* morph; /* multi-compartment cells, or NULL   */
    /* synapse model (Methods, "Cerebral cortex network"): HH_SYN_CONDUCTANCE
     * (g_E (V - E_E) + g_I (V - E_I), weights in nS) or HH_SYN_CURRENT (the
     * synapses inject their filtered currents, I_E - I_I, weights in
     * uA/cm^2; E_E, E_I and area_cm2 unused); tau_E, tau_I filter both */
    int32_t syn_mode;
    /* compound background: with bg_weight_sd > 0 each step's background is
     * N(k bg_weight_nS, k bg_weight_sd^2) for its Poisson count k (the sum of
     * k Gaussian event amplitudes), the normal by Box-Muller on the
     * Philox-4x32-10 block of counter (t/4, i, 2, (t/4) >> 32): steps 4q,
     * 4q + 1 take r cos and r sin of words 0, 1, steps 4q + 2, 4q + 3 of words
     * 2, 3 (r = sqrt(-2 ln u1), angle 2 pi u2, u = (word + 1/2) 2^-32) */
    float bg_weight_sd;
} hh_net_desc;
enum { HH_SYN_CONDUCTANCE = 0, HH_SYN_CURRENT = 1 };

/* Multi-compartment cells (Methods, Eq. hh_eq_full with the cable term,
 * "Simplified discretization": exponential Euler for the ion channels, the
 * second-order explicit difference for the spatial term; Results,
 * "neuronal morphology modeling": three dendrites and a soma).  With
 * hh_net_desc.morph set, every HH_CABLE_LANES consecutive neurons are the
 * compartments of one cell (n_neurons a multiple of HH_CABLE_LANES): index
 * 32 k is cell k's soma, 32 k + 1 + d n_per_dendrite + j compartment j
 * (counted from the soma outward) of dendrite d, and the remaining indices
 * are ordinary uncoupled point neurons.  Compartments keep every per-neuron
 * property (model, gbar, currents, synapses, spike records).  At every step
 * each compartment's injected current gains, from V at the start of the
 * step, g_axial (V_neighbour - V) for each neighbour -- the compartment
 * towards the soma and the one further out; the soma's terms towards the
 * dendrites' first compartments are divided by soma_area_ratio (its
 * membrane area over a dendritic compartment's).  The explicit coupling is
 * stable for dt g_axial (2 + 1/soma_area_ratio) / C_m below about 2. */
#define HH_CABLE_LANES 32
typedef struct hh_morphology {
    int32_t n_dendrites;      /* 1..3                                         */
    int32_t n_per_dendrite;   /* >= 1, 1 + n_dendrites n_per_dendrite <= 32   */
    float g_axial;            /* mS/cm^2 of membrane (1/(r_l dx^2)), >= 0     */
    float soma_area_ratio;    /* > 0                                          */
} hh_morphology;

/* Create a network (Methods, Eq. hh_eq_full; "Cerebral cortex network").
 * Copies every array of *d into library-owned device memory, transposes the
 * in-CSR into an out-CSR (rows = presynaptic neuron) on the GPU, and sets
 * V = V0, g_E = g_I = 0, t = 0.  No neuron model is installed yet:
 * hh_set_channels must install every model index that model_id uses (it
 * also sets those neurons' gates to p_inf(V) and Ca to ca_rest) before
 * hh_step_n runs.
 * Synchronous.  Errors: HH_EINVAL for a NULL/out-of-range argument or an
 * invalid CSR (checked on the device for col_idx and weight), HH_ENOMEM,
 * HH_ECUDA.  On error *out is NULL and nothing is leaked. */
hh_status hh_create_network(const hh_net_desc* d, hh_net** out);

/* Install neuron model `model_index` (Methods, "Flexibility and
 * extensibility": users define the ion-channel dynamics; Eq. hh_eq_full).
 *   m     : the model, host memory (copied).
 *   gbar  : [m->n_channels][N] per-neuron maximal conductances (mS/cm^2),
 *           any memory, or NULL to use m->channels[c].gbar for every neuron.
 *           Only the entries of neurons whose model_id equals model_index
 *           are used.
 * Re-initialises the gates (and Ca) of every neuron of this model to their
 * steady state at its current V.  Synchronous.
 * Errors: HH_EINVAL (index >= HH_MAX_MODELS, a count above the HH_MAX_*
 * limits, a power outside 1..4, an unknown form or kind, C_m <= 0),
 * HH_ECUDA. */
hh_status hh_set_channels(hh_net* net, int32_t model_index, const hh_model_desc* m,
                          const float* gbar);

/* ------------------------------------------------------------------ */
/* Issue-rate peaks (the denominators of the neuron kernels' roofline)   */
/* ------------------------------------------------------------------ */

typedef struct {
    double ffma_per_s;  /* FP32 fused multiply-adds per second, whole GPU   */
    double ex2_per_s;   /* ex2.approx.ftz.f32 results per second            */
    double rcp_per_s;   /* rcp.approx.ftz.f32 results per second            */
} hh_peaks;

/* Measure the three rates on the current device: 8 blocks of 256 threads
 * per SM, 8 independent unrolled dependency chains per thread, one warm-up
 * launch, CUDA events on `stream` (cudaStream_t, NULL = legacy).  Takes a
 * few milliseconds; allocates and frees a small scratch buffer on the
 * stream.  Synchronous.  Errors: HH_EINVAL (out NULL), HH_ECUDA. */
hh_status hh_measure_peaks(hh_peaks* out, void* stream);

/* ------------------------------------------------------------------ */
/* Stepping                                                             */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t step;   /* absolute step index: V crossed theta between t = step*dt
                       and (step+1)*dt */
    int32_t neuron; /* neuron index */
    float frac;     /* (theta - V_t)/(V_{t+1} - V_t) in [0, 1): the crossing
                       time is (step + frac)*dt */
} hh_spike;

/* Caller-owned device buffers that hh_step_n fills.  Any field may be NULL
 * (or zero) to skip that output. */
typedef struct {
    float* V_trace;           /* device [n_steps][n_trace]: V after each step */
    const int32_t* trace_idx; /* device [n_trace] neuron indices, or NULL for
                                 neurons 0..n_trace-1.  A neuron listed more
                                 than once is recorded in the last of its
                                 rows; its earlier rows are left unwritten    */
    int32_t n_trace;
    hh_spike* spikes;         /* device [spike_cap], unordered                */
    int64_t spike_cap;
    int64_t* n_spikes;        /* device counter the library adds the number of
                                 spikes to (caller initialises it); spikes
                                 beyond spike_cap are counted but not stored
                                 and set HH_STATUS_SPIKE_OVERFLOW             */
    int32_t* counts;          /* device [N] per-neuron spike counts, added to */
} hh_record;

/* Advance the network by n_steps time steps (Methods, Eq. hh_eq_full with
 * the exponential-Euler discretisation; order per step: synaptic delivery
 * and background into g_E/g_I, rates at V_t, gates, conductances, V, Ca,
 * threshold test, spike propagation into the delay line, decay of g_E/g_I).
 *   I_steps: device [n_steps][N] extra injected current per step, or NULL.
 *   rec    : outputs, or NULL.
 * Asynchronous on the network's stream.  Errors: HH_EINVAL (n_steps < 0,
 * trace_idx out of range is not checked: the caller guarantees it),
 * HH_ESTATE (a model index used by model_id was never installed), HH_ECUDA
 * (also when the specialised kernels fail to compile: the message holds the
 * compiler log). */
hh_status hh_step_n(hh_net* net, int32_t n_steps, const float* I_steps,
                    const hh_record* rec);

/* Reset time to 0, V to V0 (any memory, [N]; NULL = the V0 given at
 * creation), gates and Ca to steady state, g_E = g_I = 0, and clear the
 * delay line and the status word.  Asynchronous. */
hh_status hh_reset(hh_net* net, const float* V0);

/* Checkpoint and resume of the whole dynamic state of the integrator of
 * Methods, Eq. hh_eq_full after a completed step (the paper describes no
 * checkpoint format; this one is the library's own): the step index, V,
 * every gate, Ca, g_E and g_I, the
 * compensated low parts (HH_PREC_COMPENSATED), the delay line with the
 * spikes still in flight, and the status word.  The background and the
 * sinusoidal drive are functions of (seed, step, neuron), so a network
 * restored at step t continues bit for bit as the saved one did, provided
 * it was created from the same descriptor and given the same channels.
 * The model tables, maximal conductances and currents are parameters, not
 * state, and are not saved.
 *
 * The image is a 256-byte header followed by the arrays, each starting on
 * a 256-byte boundary.  hh_state_size gives its size in bytes. */
hh_status hh_state_size(const hh_net* net, size_t* bytes);

/* Write the state image into dst (any memory the device can address:
 * device, pinned or pageable host; cap bytes).  Synchronous: it returns
 * once the image is complete.  Errors: HH_EINVAL (NULL, cap too small),
 * HH_ECUDA. */
hh_status hh_save_state(hh_net* net, void* dst, size_t cap);

/* Replace the network's state by an image written by hh_save_state (any
 * memory, n bytes).  The image must come from a network with the same
 * neuron count, delay slots, precision and synapse / background layout
 * (HH_EINVAL otherwise, with the mismatch in hh_last_error()).  The copy is
 * asynchronous on the network's stream; src must stay valid until the
 * stream reaches it.  Errors: HH_EINVAL, HH_ECUDA. */
hh_status hh_load_state(hh_net* net, const void* src, size_t n);

/* Launch shape of the specialised window schedule: threads per block of the
 * neuron-window kernel (32, 64 or 128; 0 = the library's choice from N) and
 * blocks per routing launch (1 .. 4,096; 0 = the default 304).  Results do
 * not depend on it (delivery is order independent), only the speed.
 * Errors: HH_EINVAL. */
hh_status hh_set_launch_shape(hh_net* net, int32_t neuron_block, int32_t route_blocks);

/* Autotuning of the launch shape for this network's size and activity (no
 * counterpart in the paper, whose batched simulations run on its own
 * operators; Results, large-scale and batched simulation): each
 * candidate -- the library's default shape, reported as (0, 0), then
 * neuron blocks 32, 64, 128 x routing grids of 152, 304, 608 blocks (one
 * grid when the network has no synapses) -- advances the network by
 * trial_steps from its current state four times (the first run compiles
 * and captures, the other three are timed with CUDA events and their
 * median kept), the state is restored before every run, and the fastest
 * shape is installed if it beats the default by at least 3 % (else the
 * default stays).  On return the
 * network's state is the one it had on entry.
 * Needs a network with synapses or background on the specialised kernels
 * (HH_EUNSUPPORTED otherwise).  Synchronous.  rep may be NULL. */
#define HH_TUNE_MAX 16
typedef struct {
    int32_t n;                          /* candidates tried */
    int32_t best;                       /* index of the installed one */
    int32_t neuron_block[HH_TUNE_MAX];
    int32_t route_blocks[HH_TUNE_MAX];
    float ms[HH_TUNE_MAX];              /* median timed run of trial_steps steps */
} hh_tune_report;
hh_status hh_autotune(hh_net* net, int32_t trial_steps, hh_tune_report* rep);

/* Open-loop spike routing (Methods, "Cerebral cortex network": synaptic
 * delays and E/IPSP filters; the spike-delivery step of the network):
 * for every spike (step s, neuron j) of the given list and every synapse
 * j -> i of weight w, add round(w * 2^32) to
 *   sum_E[s + D][i]  (j excitatory)  or  sum_I[s + D][i]  (j inhibitory),
 * dropping arrivals at or after n_window.  This is the same routing kernel
 * hh_step_n uses, run on a caller-given raster without neuron dynamics.
 *   spk_step, spk_idx: device [n_spk]; spk_step >= 0, spk_idx in [0, N)
 *                      (entries outside are skipped).
 *   sum_E, sum_I     : device int64 [n_window][N], accumulated into (the
 *                      caller zeroes them).
 * Asynchronous.  Errors: HH_EINVAL, HH_ESTATE (network has no synapses). */
hh_status hh_route_spikes(hh_net* net, const int32_t* spk_step, const int32_t* spk_idx,
                          int64_t n_spk, int32_t n_window, int64_t* sum_E, int64_t* sum_I);

/* Pull routing of dense windows (Methods, "Cerebral cortex network": the
 * delayed delivery of spikes over the synapse graph).  A window of the
 * window schedule in which at least min_spikes spikes occurred is routed by
 * a pull over the in-CSR (every postsynaptic row read once, one 64-bit
 * atomic per nonzero (step, E/I) sum of a row) instead of the push over the
 * out-CSR (one atomic per synaptic event); both give the same delay-line
 * bits, since the fixed-point sums are exact.  Possible for networks with
 * synapses, at most 65,536 neurons and windows of at most 64 steps
 * (delay_steps <= 129).  Off by default (on GB300 the pull costs about as
 * much as the push even for windows in which half the network spikes).
 *   min_spikes: >= 0 the threshold (0: every window with a spike), < 0 off.
 * The first call with min_spikes >= 0 builds the in-CSR (8 bytes per
 * synapse, from the out-CSR) and the last-spike tables; it is synchronous.
 * Takes effect at the next hh_step_n; the persistent schedule and
 * hh_route_spikes always push.  Errors: HH_EINVAL (net NULL),
 * HH_EUNSUPPORTED (min_spikes >= 0 for a network that cannot pull),
 * HH_ENOMEM, HH_ECUDA. */
hh_status hh_set_route_pull(hh_net* net, int64_t min_spikes);

/* ------------------------------------------------------------------ */
/* Learned multi-step surrogate                                         */
/* ------------------------------------------------------------------ */

/* A small MLP (features -> 64 -> 64 -> state corrections, tanh, bf16
 * weights with fp32 accumulation on the tensor cores) that advances V, the
 * gates and Ca of an independent neuron by `window` steps at once while the
 * neuron is inside the sub-threshold envelope it was trained on.  Its
 * prediction is one exponential-Euler step over the whole window (rates at
 * the window's first V, step dt window) plus the MLP's learned correction.  It has no
 * counterpart in the paper (whose operators use polynomial approximations of
 * the rates, Methods "Engineering optimization"); the plain exponential-
 * Euler integrator generates its training data, integrates every window the
 * surrogate declines, and judges its error.
 * Features: (V + 65)/20, 2p - 1 per gate, log(Ca/Ca_rest)/2, I/10,
 * log(gbar_c / default gbar_c)/0.3 per channel.  Targets: the plain
 * integrator's state after the window minus the coarse step's, scaled to
 * unit variance.  A window is taken from the MLP
 * when V < v_envelope at its start, every feature lies within the range seen
 * in training (widened by 2 %), and the prediction keeps V below the
 * envelope, the gates in [0, 1] and Ca positive, and -- the per-neuron
 * error estimate, when err_V > 0 -- the MLP's correction to the coarse step
 * is at most err_V mV in V and err_p in every gate; otherwise the plain
 * kernel integrates it (so every spike comes from the plain integrator).
 * The coarse step is exact for a neuron at rest; the correction grows where
 * V and the fast gates move within the window, and the MLP's error is a
 * fraction of the correction it predicts. */
typedef struct {
    int32_t window;          /* steps per MLP evaluation, 1..1000           */
    float v_envelope;        /* mV                                          */
    int32_t train_neurons;   /* training trajectories (>= 128)              */
    int32_t train_windows;   /* windows recorded for training (>= 1024)     */
    int32_t epochs;          /* >= 1                                        */
    int32_t batch;           /* >= 128 (rounded down to a multiple of 128)  */
    float lr;                /* Adam learning rate, cosine decay            */
    uint64_t seed;
    float I_min, I_max;      /* uA/cm^2 range of the training neurons       */
    float gbar_sigma;        /* lognormal spread of their maximal conductances */
    float V0_min, V0_max;    /* initial V range (gates at steady state)     */
    float err_V;             /* error-estimate tolerance in V (mV); 0: off  */
    float err_p;             /* error-estimate tolerance of the gates (used
                                when err_V > 0)                            */
} hh_surrogate_desc;

typedef struct {
    int64_t train_windows;   /* windows used                                  */
    float train_loss;        /* mean squared error of the scaled increments   */
    float val_loss;          /* same on 5 % held-out windows                  */
    float out_scale_V;       /* std of the V increment over a window (mV)     */
} hh_surrogate_report;

/* Train a surrogate for model 0 of `net` (its dt and precision) and keep it
 * in the network.  Requires a network of independent neurons (no synapses,
 * no background) with a single model and HH_KERNELS_SPECIALISED, precision
 * FAST or ACCURATE.  Synchronous.  Errors: HH_EINVAL, HH_EUNSUPPORTED,
 * HH_ESTATE (model 0 not installed), HH_ENOMEM, HH_ECUDA. */
hh_status hh_surrogate_train(hh_net* net, const hh_surrogate_desc* d, hh_surrogate_report* rep);

/* Use (1) or stop using (0) the trained surrogate in hh_step_n: whole
 * windows go through the MLP or the plain kernel as described above; the
 * steps left over after the last whole window are plain.  V traces and
 * per-step currents are not supported while it is enabled (HH_EUNSUPPORTED).  HH_READ_SURROGATE reads
 * the counts of accepted and declined neuron-windows. */
hh_status hh_surrogate_enable(hh_net* net, int32_t enable);

/* ------------------------------------------------------------------ */
/* Dense projections on the tensor cores                                */
/* ------------------------------------------------------------------ */

/* C[s][m][n] = sum over the K range of split s of A[m][k] * Bt[n][k]
 * The BF16 x BF16 -> FP32 product on the tcgen05 tensor cores that the
 * differentiable layer uses for its input and recurrent projections and
 * their weight gradients (the input current of an HH layer is produced by
 * the previous layer's weights, Methods "Analysis of C_m").
 *   A : device bf16 [M][lda], row-major (K contiguous), lda >= K, lda % 8 == 0
 *   Bt: device bf16 [N][ldb], row-major (K contiguous: the transpose of the
 *       K x N matrix B), ldb >= K, ldb % 8 == 0
 *   C : device fp32 [splits][M][N]; split s holds the partial product over
 *       K blocks [s*P, (s+1)*P) of 64, P = ceil(ceil(K/64)/splits); the
 *       caller sums the splits (splits = 1 gives C = A B)
 *   N % 32 == 0; A, Bt, C 16-byte aligned; status: device int32 that bounded
 *       device waits OR a nonzero code into on failure (caller zeroes it).
 * Asynchronous on `stream`.  Errors: HH_EINVAL, HH_ECUDA. */
hh_status hh_gemm_bf16(const void* A, int32_t lda, const void* Bt, int32_t ldb, float* C, int32_t M,
                       int32_t N, int32_t K, int32_t splits, int32_t* status, void* stream);

/* ------------------------------------------------------------------ */
/* Differentiable recurrent HH layer (BPTT)                             */
/* ------------------------------------------------------------------ */

/* A recurrent layer of n_hidden HH point neurons trained by
 * back-propagation through time (Methods, "Gradient learning support":
 * gradients of the discretised state update derived by hand; "Engineering
 * optimization": re-computation).  Per outer step t (substeps x dt_ms):
 *   I_t = bias + X_t W_in + S_{t-1} W_rec     (bf16 tensor-core products,
 *                                               fp32 accumulation)
 *   K = substeps exponential-Euler steps with I_t held;
 *   S_t = sum_k H(V_k - theta)(1 - H(V_{k-1} - theta))  (smooth = 0), or
 *         the same with H replaced by 0.5 + 0.5 b x/(1 + b|x|) (smooth = 1)
 *   r = mean_t S_t,  logits = r W_out^T,  loss = mean_b CE(logits_b, y_b).
 * The backward pass replaces dH/dx by 1/(1 + b|x|)^2 (b = surrogate_beta)
 * and treats the (1 - H(V_{k-1} - theta)) factor as a constant.  W_in and
 * W_rec are rounded to bf16 when set; S is rounded to bf16 for the
 * recurrent product (exact for 0/1 spikes).  Neurons start at v_init with
 * gates at steady state; checkpoints every checkpoint_every outer steps. */
typedef struct hh_layer hh_layer;

typedef struct {
    int32_t batch;            /* B >= 1                                       */
    int32_t n_in;             /* input channels                               */
    int32_t n_hidden;         /* N, a multiple of 32                          */
    int32_t n_out;            /* classes                                      */
    int32_t n_steps;          /* T outer steps                                */
    int32_t substeps;         /* K in 1..16                                   */
    double dt_ms;             /* substep                                      */
    float v_threshold, v_init, surrogate_beta;
    int32_t precision;        /* HH_PREC_FAST or HH_PREC_ACCURATE            */
    int32_t smooth;           /* 0 Heaviside + surrogate, 1 smooth spikes     */
    int32_t checkpoint_every; /* outer steps between state checkpoints        */
    void* stream;
} hh_layer_desc;

/* Gradient outputs of a backward pass, caller-owned device buffers,
 * overwritten (not accumulated).  hh_backward needs the first four;
 * hh_backward_from skips every NULL field. */
typedef struct {
    float* dW_in;   /* device [n_in][N]                                    */
    float* dW_rec;  /* device [N][N]                                       */
    float* dW_out;  /* device [n_out][N]                                   */
    float* dbias;   /* device [N]                                          */
    float* dI;      /* device [T][B][N]: dL/dI_t, the gradient of each outer
                       step's input current (the hand-derived adjoint)     */
    float* dX;      /* device [T][B][n_in]: dL/dX_t = dI_t W_in^T (tensor
                       cores: dI split into bf16 hi + lo parts, fp32
                       accumulation), for a preceding layer                */
} hh_grads;

enum { HH_LAYER_SPIKES = 0, /* float [T][B][N] spikes of the last forward  */
       HH_LAYER_V = 1,      /* float [B][N] V after the last forward       */
       HH_LAYER_STATUS = 2  /* int32: nonzero if a bounded device wait failed */ };

/* Create a layer for one model (alpha/beta or inf/tau gates, no calcium pool)
 * and allocate every buffer it needs.  Synchronous.  Errors: HH_EINVAL,
 * HH_EUNSUPPORTED (model or precision), HH_ENOMEM, HH_ECUDA. */
hh_status hh_layer_create(const hh_layer_desc* d, const hh_model_desc* model, hh_layer** out);

/* W_in [n_in][N], W_rec [N][N], W_out [n_out][N], bias [N]: fp32, any memory
 * (copied; W_in and W_rec rounded to bf16).  Synchronous. */
hh_status hh_layer_set_weights(hh_layer* layer, const float* W_in, const float* W_rec,
                               const float* W_out, const float* bias);

/* Forward pass.  X: device fp32 [T][B][n_in] inputs (0/1 spikes, or any
 * values, which the input projection rounds to bf16); labels: device int32
 * [B], or NULL for no built-in loss; loss: device fp32 [1] (needed with
 * labels, else ignored); logits: device [B][n_out] or NULL.  Asynchronous.
 * Errors: HH_EINVAL, HH_ECUDA. */
hh_status hh_layer_forward(hh_layer* layer, const float* X, const int32_t* labels, float* loss,
                           float* logits);

/* Backward pass of the last forward for its built-in loss (the mean
 * cross-entropy; the forward must have had labels): fills dW_in, dW_rec,
 * dW_out and dbias (all required), and dI / dX when given.  The same as
 * hh_backward_from(layer, 1, NULL, NULL, NULL, g).  Asynchronous.
 * Errors: HH_EINVAL, HH_ESTATE (no forward yet, or one without labels),
 * HH_ECUDA. */
hh_status hh_backward(hh_layer* layer, const hh_grads* g);

/* Backward pass of the last forward for any loss of its outputs (Methods,
 * "Gradient learning support": the hand-derived gradient of the discretised
 * update, so that HH layers train inside larger models end to end):
 *   L = ce_weight * CE + sum dL_dlogits * logits + sum dL_dS * S + sum dL_dV * V_T
 * where CE is the built-in mean cross-entropy of the forward (ce_weight = 0
 * drops it; nonzero needs a forward with labels), S the [T][B][N] spike
 * outputs (HH_LAYER_SPIKES) and V_T the [B][N] membrane potentials after the
 * last step (HH_LAYER_V).  Each cotangent is a device fp32 array or NULL:
 *   dL_dlogits [B][n_out], dL_dS [T][B][N], dL_dV [B][N].
 * Every non-NULL field of g is filled.  Asynchronous.  Errors: HH_EINVAL,
 * HH_ESTATE (no forward yet; ce_weight != 0 after a forward without
 * labels), HH_ENOMEM (the first request of dX allocates its operands),
 * HH_ECUDA. */
hh_status hh_backward_from(hh_layer* layer, float ce_weight, const float* dL_dlogits,
                           const float* dL_dS, const float* dL_dV, const hh_grads* g);

/* Copy HH_LAYER_* into dst (any memory); synchronous. */
hh_status hh_layer_readout(hh_layer* layer, int32_t what, void* dst, size_t cap_bytes,
                           size_t* n_bytes);

void hh_layer_destroy(hh_layer* layer);

/* ------------------------------------------------------------------ */
/* Readout                                                              */
/* ------------------------------------------------------------------ */

enum {
    HH_READ_V = 0,       /* float [N] membrane potential (hi part)         */
    HH_READ_GATES = 1,   /* float [HH_MAX_GATES][N] gate values            */
    HH_READ_CA = 2,      /* float [N]                                       */
    HH_READ_G_SYN = 3,   /* float [2][N] g_E then g_I (nS)                  */
    HH_READ_STATUS = 4,  /* int32: OR of HH_STATUS_* bits since the last reset */
    HH_READ_TIME = 5,    /* int64: steps advanced since creation / reset    */
    HH_READ_N_OUT = 6,   /* int64 [N+1] out-CSR row pointer (rows = pre)    */
    HH_READ_PROFILE = 7, /* hh_kernel_time [HH_KERNEL_COUNT] since hh_profile(net, 1) */
    HH_READ_SURROGATE = 8, /* uint64 [2]: neuron-windows taken from the surrogate, declined */
    HH_READ_POLY = 9       /* float [HH_MAX_MODELS][3]: interval (mV), first V (mV) and largest
                              relative error of the rate tables per model (zeros: none) */
};
enum { HH_STATUS_SPIKE_OVERFLOW = 1, HH_STATUS_NONFINITE = 2, HH_STATUS_BARRIER_TIMEOUT = 4 };

/* Copy a quantity into dst (any memory) of cap_bytes bytes; *n_bytes (if
 * not NULL) receives the bytes written.  Synchronous: waits for the work
 * queued on the network's stream.  Errors: HH_EINVAL (unknown `what`),
 * HH_EOVERFLOW (cap_bytes too small: nothing is written), HH_ECUDA (also for
 * an asynchronous error of earlier queued work). */
hh_status hh_readout(hh_net* net, int32_t what, void* dst, size_t cap_bytes, size_t* n_bytes);

/* Kernel timing (a tracing aid for benchmarks).  While enabled, hh_step_n
 * brackets every neuron-update launch and every routing launch with CUDA
 * events on the network's stream; HH_READ_PROFILE returns, per kernel class,
 * the number of launches and the summed event-to-event time.  Enabling
 * clears the totals; disabling keeps them for readout.  Timing adds a few
 * microseconds of event records per launch, so time throughput with it off.
 * Errors: HH_EINVAL, HH_ECUDA. */
typedef struct {
    int64_t launches;
    double total_ms;
} hh_kernel_time;
enum { HH_KERNEL_NEURON = 0, HH_KERNEL_ROUTE = 1, HH_KERNEL_COUNT = 2 };
hh_status hh_profile(hh_net* net, int32_t enable);

/* ------------------------------------------------------------------ */
/* Allocation-free stepping of independent neurons                      */
/* ------------------------------------------------------------------ */

/* Some callers cannot call cudaMalloc: code running inside another
 * framework's memory pool or arena, a host process that must not grow its
 * device footprint after start-up, or a runtime that hands out device memory
 * only from its own allocator.  hh_step_neurons_noalloc lets them step a
 * population of independent neurons (no synapses) in buffers they already
 * own.  It has no counterpart in the paper: it is the same neuron kernel as
 * hh_step_n, with its only scratch space -- the map from neuron to
 * V-trace slot used when rec->trace_idx is given -- held in a file-scope
 * device array of the library instead of library-allocated memory.
 *
 * Limits and behaviour:
 *   - n_neurons <= HH_NOALLOC_MAX_NEURONS (larger sizes return HH_EINVAL);
 *     the static scratch (4 MiB of slot map plus one status word that takes
 *     the status bits when s->status is NULL) stays resident on every GPU
 *     that loads the library until the process exits.
 *   - The first call on a device looks up the scratch array's device
 *     address (cudaGetSymbolAddress with that device current) and caches
 *     it; make that first call before any stream capture.
 *   - Every call shares the one scratch array and overwrites the part it
 *     uses (it resets the slot map at the start of each call that records
 *     a trace with trace_idx).  Calls whose work overlaps on the GPU -- on
 *     different streams, or from several threads -- race on it.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.  The
 *     very first launch of the library's kernels in a process may still make
 *     the CUDA driver load their module (lazy loading), which reserves device
 *     memory once; later calls leave the free device memory unchanged.
 * All state and I/O pointers are device memory owned by the caller; the
 * state arrays are updated in place. */
#define HH_NOALLOC_MAX_NEURONS (1 << 20)

typedef struct {
    int64_t n_neurons;       /* 1 .. HH_NOALLOC_MAX_NEURONS                   */
    double dt_ms;            /* > 0                                            */
    float v_threshold;       /* mV                                             */
    int32_t v_update;        /* HH_V_*                                         */
    int32_t precision;       /* HH_PREC_*; COMPENSATED needs V_lo, gates_lo    */
    float* V;                /* device [N], updated in place                  */
    float* V_lo;             /* device [N] or NULL                            */
    float* gates;            /* device [HH_MAX_GATES][N], updated in place    */
    float* gates_lo;         /* device [HH_MAX_GATES][N] or NULL              */
    float* Ca;               /* device [N]                                    */
    const float* I_const;    /* device [N] constant current, or NULL          */
    const float* gbar;       /* device [HH_MAX_CHANNELS][N] per-neuron maximal
                                conductances, or NULL for the model's         */
    int32_t* status;         /* device int32 the call ORs HH_STATUS_* bits
                                into, or NULL to discard them                 */
    int32_t init_state;      /* 1: first set gates to p_inf(V), Ca to rest    */
    void* stream;            /* cudaStream_t, NULL = legacy default stream    */
} hh_neurons_noalloc;

/* Advance the population by n_steps: the same step as hh_step_n for a
 * network without synapses; t0 is the absolute index of the first step
 * (spike records).
 * m: the neuron model, host memory.  I_steps: device [n_steps][N] or NULL.
 * rec: as for hh_step_n, or NULL.  Asynchronous on s->stream.
 * Errors: HH_EINVAL (sizes beyond the limits, NULL state pointers, an
 * invalid model, COMPENSATED without lo arrays), HH_ECUDA. */
hh_status hh_step_neurons_noalloc(const hh_model_desc* m, const hh_neurons_noalloc* s,
                                  int64_t t0, int32_t n_steps, const float* I_steps,
                                  const hh_record* rec);

/* Release everything the network owns (waits for its queued work). NULL ok. */
void hh_destroy(hh_net* net);

/* Thread-local description of the last error of the calling thread. */
const char* hh_last_error(void);

/* Bounds of the device-side waits, for every later launch in the process
 * (failure detection: a wait that runs out records a status and the kernel
 * returns, so that the context stays usable).  progress_ns bounds each wait
 * of the persistent kernel on another block's progress counter (global
 * timer; default 2e9 = 2 s; on expiry HH_STATUS_BARRIER_TIMEOUT is set);
 * mbarrier_polls bounds each wait of the tensor-core GEMM's pipeline on its
 * TMA / MMA / epilogue mbarriers (default 2^24 polls; on expiry a nonzero
 * code is ORed into the GEMM's status word).  0 gives up at the first wait
 * that has not completed; a negative value restores the default.  The
 * GEMM's final wait for its own TMA loads in flight always uses the
 * default, so no copy lands after its block exits.  Errors: none. */
hh_status hh_set_wait_limits(int64_t progress_ns, int64_t mbarrier_polls);

/* The rate tables HH_PREC_POLY installs for model m at time step dt_ms,
 * computed on the host (no device work; the same fit hh_set_channels runs).
 *   info       : host float [3]: interval (mV), first V (mV), largest relative
 *                error measured
 *   n_intervals: host, or NULL: intervals of the table
 *   coeffs     : host float [n_intervals][n_gates][2][4], or NULL: per
 *                interval j (V in [v_lo + j h, v_lo + (j + 1) h)) and gate (in
 *                channel order), the coefficients c0..c3 of c0 + x (c1 + x (c2
 *                + x c3)), x = (V - v_lo)/h - j, for p_inf (zeros for a
 *                Ca-dependent gate) and for 1 - e^{-dt/tau}
 *   n_floats   : host, or NULL: floats the table holds
 * Errors: HH_EINVAL (invalid model or dt), HH_EOVERFLOW (cap_floats too
 * small; info, n_intervals and n_floats are filled). */
hh_status hh_poly_fit(const hh_model_desc* m, double dt_ms, float* info, int32_t* n_intervals, float* coeffs,
                      int64_t cap_floats, int64_t* n_floats);

/* Library version, e.g. 0x000100 for 0.1.0. */
int32_t hh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HH_H */
