/*
 * FP64 CPU oracle for the Hodgkin-Huxley hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source,
 * header, table or constant generator with the CUDA path: every structure and
 * routine below is defined here, from the paper's statement of the method.
 *
 * What it computes, step by step, in double precision:
 *   - Membrane and gating equations (Methods, Eq. hh_eq_full, point-neuron
 *     case: the cable term d2V/dx2 is absent):
 *         C_m dV/dt = I - sum_X gbar_X eta_X(p) (V - E_X) - g_E (V-E_E) - g_I (V-E_I)
 *         dp/dt     = alpha_p(V) (1 - p) - beta_p(V) p
 *     The sign of the ionic term follows the first line of Eq. hh_eq_full;
 *     the '+' printed in Eq. hh_dyn_simplified is read as f(V,t) absorbing
 *     the sign.
 *   - Exponential-Euler discretisation of the ion-channel terms (Methods,
 *     "Simplified discretization"):
 *         p <- p_inf + (p - p_inf) exp(-dt / tau_p),
 *         p_inf = alpha/(alpha+beta), tau_p = 1/(alpha+beta)
 *     and of V with the conductances frozen over the step:
 *         V <- V_inf + (V - V_inf) exp(-dt G / C_m),  V_inf = (I + sum g E)/G.
 *     The explicit-Euler variant of Eq. hh_dyn_simplified is selectable.
 *   - Order inside one step: synaptic delivery + background into g_E/g_I,
 *     rates at V_t, gates, conductances with the new gates, V, calcium pool,
 *     upward threshold test on (V_t, V_{t+1}), push of this step's spikes
 *     into the delay ring, decay of g_E/g_I (E/IPSP filters and synaptic
 *     delays of the cortex model, Methods "Cerebral cortex network").
 *   - Background input: per neuron and step a Poisson count drawn from a
 *     Philox-4x32-10 counter (Salmon et al., SC'11) by inversion against the
 *     Poisson CDF scaled to 2^32; each count adds bg_w nS to g_E.
 *
 * Conventions: V in mV, t in ms, currents in uA/cm^2, membrane conductances
 * in mS/cm^2, synaptic weights and g_E/g_I in nS (converted with the
 * membrane area: 1 nS = 1e-6 mS / area_cm2), Ca in uM.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_CH 8
#define OR_MAX_GATES 12

enum { OR_CONST = 0, OR_EXP = 1, OR_SIGMOID = 2, OR_LINOID = 3, OR_BELL = 4 };
enum { OR_AB = 0, OR_INFTAU = 1, OR_CA = 2 };

typedef struct { int32_t form; int32_t pad; double a, vh, k, vh2, k2, c; } or_fn;
typedef struct { int32_t kind; int32_t power; or_fn f1; or_fn f2; } or_gate;
typedef struct { double E; double gbar; int32_t n_gates; int32_t first_gate; } or_channel;
typedef struct {
    double C_m;
    int32_t n_channels;
    int32_t n_gates;
    or_channel ch[OR_MAX_CH];
    or_gate g[OR_MAX_GATES];
    int32_t ca_channel; /* -1: no calcium pool */
    int32_t pad;
    double ca_tau, ca_k, ca_rest;
} or_model;

/* sizes the Python side checks its mirrors against */
int32_t or_sizeof_model(void) { return (int32_t)sizeof(or_model); }
int32_t or_sizeof_gate(void) { return (int32_t)sizeof(or_gate); }

/* ---------------------------------------------------------------------------
 * Rate functions: the closed forms a user channel can take (alpha, beta,
 * p_inf or tau as functions of V).
 * ------------------------------------------------------------------------- */
double or_rate(const or_fn* f, double V)
{
    double r;
    switch (f->form) {
    case OR_CONST:
        r = f->a;
        break;
    case OR_EXP:
        r = f->a * exp((V - f->vh) / f->k);
        break;
    case OR_SIGMOID:
        r = f->a / (1.0 + exp((V - f->vh) / f->k));
        break;
    case OR_LINOID: {
        /* a x / (1 - exp(-x/k)); its limit at x = 0 is a k */
        double x = V - f->vh;
        if (x == 0.0)
            r = f->a * f->k;
        else
            r = f->a * x / (-expm1(-x / f->k));
        break;
    }
    case OR_BELL:
        r = f->a / (exp((V - f->vh) / f->k) + exp((V - f->vh2) / f->k2));
        break;
    default:
        r = NAN;
    }
    return r + f->c;
}

/* p_inf and tau of one gate at (V, Ca) */
void or_gate_inf_tau(const or_gate* g, double V, double Ca, double* inf, double* tau)
{
    if (g->kind == OR_AB) {
        double al = or_rate(&g->f1, V), be = or_rate(&g->f2, V);
        *inf = al / (al + be);
        *tau = 1.0 / (al + be);
    } else if (g->kind == OR_INFTAU) {
        *inf = or_rate(&g->f1, V);
        *tau = or_rate(&g->f2, V);
    } else { /* OR_CA */
        *inf = Ca / (Ca + g->f1.a);
        *tau = or_rate(&g->f2, V);
    }
}

/* Resting gate values p_inf(V0) (and Ca at rest). */
void or_init_neuron(const or_model* M, double V0, double* p, double* Ca)
{
    *Ca = M->ca_channel >= 0 ? M->ca_rest : 0.0;
    for (int q = 0; q < M->n_gates; ++q) {
        double inf, tau;
        or_gate_inf_tau(&M->g[q], V0, *Ca, &inf, &tau);
        p[q] = inf;
    }
}

/* Total ionic current sum_X gbar_X eta_X (V - E_X) at (V, p) (for the
 * resting-potential pin). */
double or_ionic_current(const or_model* M, const double* gbar, double V, const double* p)
{
    double Iion = 0.0;
    for (int c = 0; c < M->n_channels; ++c) {
        double eta = 1.0;
        for (int q = 0; q < M->ch[c].n_gates; ++q) {
            const or_gate* g = &M->g[M->ch[c].first_gate + q];
            eta *= pow(p[M->ch[c].first_gate + q], (double)g->power);
        }
        Iion += gbar[c] * eta * (V - M->ch[c].E);
    }
    return Iion;
}

/* One step of one neuron.  gE/gI are synaptic conductances in mS/cm^2.
 * Returns V_{t+1}; updates p and Ca in place. */
double or_step_neuron(const or_model* M, const double* gbar, double dt, double I,
                      double gE, double EE, double gI, double EI, int32_t v_mode,
                      double V, double* p, double* Ca)
{
    /* gates: rates at V_t, exponential Euler */
    for (int q = 0; q < M->n_gates; ++q) {
        double inf, tau;
        or_gate_inf_tau(&M->g[q], V, *Ca, &inf, &tau);
        p[q] = inf + (p[q] - inf) * exp(-dt / tau);
    }
    /* conductances with the new gates */
    double G = gE + gI;
    double GE = gE * EE + gI * EI;
    double gCa = 0.0, ECa = 0.0;
    for (int c = 0; c < M->n_channels; ++c) {
        double eta = 1.0;
        for (int q = 0; q < M->ch[c].n_gates; ++q) {
            const or_gate* g = &M->g[M->ch[c].first_gate + q];
            eta *= pow(p[M->ch[c].first_gate + q], (double)g->power);
        }
        double gx = gbar[c] * eta;
        G += gx;
        GE += gx * M->ch[c].E;
        if (c == M->ca_channel) {
            gCa = gx;
            ECa = M->ch[c].E;
        }
    }
    double Vn;
    if (v_mode == 0) {
        double Vinf = (I + GE) / G;
        Vn = Vinf + (V - Vinf) * exp(-dt * G / M->C_m);
    } else {
        Vn = V + dt / M->C_m * (I - (G * V - GE));
    }
    if (M->ca_channel >= 0) {
        double ICa = gCa * (V - ECa);
        double Cainf = M->ca_rest - M->ca_k * M->ca_tau * ICa;
        *Ca = Cainf + (*Ca - Cainf) * exp(-dt / M->ca_tau);
    }
    return Vn;
}

/* ---------------------------------------------------------------------------
 * Independent neurons (no synapses).
 *   gbar: [OR_MAX_CH][N] per-neuron maximal conductances, or NULL for the
 *         model's defaults.
 *   I_const [N] or NULL; I_steps [T][N] or NULL (added together).
 *   V_trace [T][N] or NULL: V after each step.
 *   spikes: per neuron up to spk_cap (step, frac) pairs at [i*spk_cap + s].
 * ------------------------------------------------------------------------- */
int or_simulate(const or_model* models, int32_t n_models, const uint8_t* model_id,
                const double* gbar, int64_t N, int64_t T, double dt, double theta,
                int32_t v_mode, const double* I_const, const double* I_steps,
                const double* V0, double* V_trace, int32_t* counts, int32_t spk_cap,
                int32_t* spk_step, double* spk_frac, int32_t n_threads)
{
    if (n_models < 1 || N < 0 || T < 0 || !(dt > 0.0))
        return 1;
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < N; ++i) {
        const or_model* M = &models[model_id ? model_id[i] : 0];
        double gb[OR_MAX_CH];
        for (int c = 0; c < M->n_channels; ++c)
            gb[c] = gbar ? gbar[(int64_t)c * N + i] : M->ch[c].gbar;
        double p[OR_MAX_GATES], Ca;
        double V = V0[i];
        or_init_neuron(M, V, p, &Ca);
        int32_t cnt = 0;
        for (int64_t t = 0; t < T; ++t) {
            double I = (I_const ? I_const[i] : 0.0) + (I_steps ? I_steps[t * N + i] : 0.0);
            double Vn = or_step_neuron(M, gb, dt, I, 0.0, 0.0, 0.0, 0.0, v_mode, V, p, &Ca);
            if (V < theta && Vn >= theta) {
                if (cnt < spk_cap && spk_step) {
                    spk_step[i * spk_cap + cnt] = (int32_t)t;
                    spk_frac[i * spk_cap + cnt] = (theta - V) / (Vn - V);
                }
                ++cnt;
            }
            V = Vn;
            if (V_trace)
                V_trace[t * N + i] = V;
        }
        if (counts)
            counts[i] = cnt;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Multi-compartment neurons (Methods, Eq. hh_eq_full with the cable term;
 * "Simplified discretization": exponential Euler for the ion-channel terms,
 * the second-order explicit difference for the spatial term).  Compartments
 * form a tree: compartment c with parent[c] >= 0 is joined to it by the
 * axial conductance g_ax per unit membrane area of c.  Per step, from V_t:
 *   I_ax[c] += g_ax (V_p - V_c),   I_ax[p] += g_ax (area[c]/area[p]) (V_c - V_p)
 * (the second difference of the cable, explicit), then every compartment
 * takes the point-neuron step with I = I_const + I_steps + I_ax held.
 * ------------------------------------------------------------------------- */
int or_simulate_cable(const or_model* M, const double* gbar, int64_t N, const int64_t* parent,
                      const double* area, double g_ax, int64_t T, double dt, double theta,
                      const double* I_const, const double* I_steps, const double* V0, double* V_trace,
                      int32_t* counts, int32_t spk_cap, int32_t* spk_step, double* spk_frac)
{
    if (N < 0 || T < 0 || !(dt > 0.0) || !(g_ax >= 0.0))
        return 1;
    for (int64_t c = 0; c < N; ++c)
        if (parent[c] >= N || parent[c] == c || !(area[c] > 0.0))
            return 1;
    double* V = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* P = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1) * OR_MAX_GATES);
    double* Ca = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    double* Iax = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t c = 0; c < N; ++c) {
        V[c] = V0[c];
        or_init_neuron(M, V[c], &P[c * OR_MAX_GATES], &Ca[c]);
        if (counts)
            counts[c] = 0;
    }
    for (int64_t t = 0; t < T; ++t) {
        for (int64_t c = 0; c < N; ++c)
            Iax[c] = 0.0;
        for (int64_t c = 0; c < N; ++c) {
            const int64_t p = parent[c];
            if (p < 0)
                continue;
            Iax[c] += g_ax * (V[p] - V[c]);
            Iax[p] += g_ax * (area[c] / area[p]) * (V[c] - V[p]);
        }
        for (int64_t c = 0; c < N; ++c) {
            double gb[OR_MAX_CH];
            for (int k = 0; k < M->n_channels; ++k)
                gb[k] = gbar ? gbar[(int64_t)k * N + c] : M->ch[k].gbar;
            const double I = (I_const ? I_const[c] : 0.0) + (I_steps ? I_steps[t * N + c] : 0.0) + Iax[c];
            const double Vt = V[c];
            const double Vn = or_step_neuron(M, gb, dt, I, 0.0, 0.0, 0.0, 0.0, 0, Vt, &P[c * OR_MAX_GATES], &Ca[c]);
            if (Vt < theta && Vn >= theta) {
                int32_t k = counts ? counts[c] : 0;
                if (spk_step && k < spk_cap) {
                    spk_step[c * spk_cap + k] = (int32_t)t;
                    spk_frac[c * spk_cap + k] = (theta - Vt) / (Vn - Vt);
                }
                if (counts)
                    counts[c] = k + 1;
            }
            V[c] = Vn;
        }
        if (V_trace)
            for (int64_t c = 0; c < N; ++c)
                V_trace[t * N + c] = V[c];
    }
    free(V); free(P); free(Ca); free(Iax);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies on a
 * 4-word counter with a 2-word Weyl-incremented key.
 * ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The uniform word used for the background count of neuron i at step t:
 * one Philox block serves four consecutive steps.  Counter = (q, i, 1, q>>32)
 * with q = t / 4, key = (seed, seed >> 32); the word is output[t mod 4]. */
uint32_t or_background_word(uint64_t seed, int64_t t, int64_t i)
{
    uint64_t q = (uint64_t)t >> 2;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)i, 1u, (uint32_t)(q >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return out[(uint64_t)t & 3u];
}

/* Standard normal of the compound background (Methods, "Cerebral cortex
 * network": the background after integration is sum_i Poisson(lambda)_i
 * Gaussian(mu, sigma)_i, sampled directly as N(k mu, k sigma^2) for the
 * Poisson count k): Box-Muller on the Philox-4x32-10 block of counter
 * (t/4, i, 2, (t/4) >> 32), key = seed.  Steps 4q, 4q+1 use words 0, 1 and
 * steps 4q+2, 4q+3 words 2, 3, as r cos(2 pi u2) and r sin(2 pi u2) with
 * r = sqrt(-2 ln u1), u = (word + 1/2) 2^-32. */
double or_background_normal(uint64_t seed, int64_t t, int64_t i)
{
    uint64_t q = (uint64_t)t >> 2;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)i, 2u, (uint32_t)(q >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    const int pair = (int)(((uint64_t)t & 3u) >> 1);
    const double u1 = ((double)out[2 * pair] + 0.5) / 4294967296.0;
    const double u2 = ((double)out[2 * pair + 1] + 0.5) / 4294967296.0;
    const double r = sqrt(-2.0 * log(u1));
    const double a = 2.0 * 3.14159265358979323846 * u2;
    return ((uint64_t)t & 1u) ? r * sin(a) : r * cos(a);
}

/* Poisson CDF thresholds on the 2^32 grid: thr[j] = min(2^32, floor(F(j) 2^32))
 * with F(j) = sum_{i<=j} e^-lambda lambda^i / i!, accumulated as
 * pmf_0 = exp(-lambda), pmf_j = (pmf_{j-1} * lambda) / j, F_j = F_{j-1} + pmf_j.
 * The last entry (or entry cap-1) is forced to 2^32.  Returns the count. */
int32_t or_poisson_table(double lambda, uint64_t* thr, int32_t cap)
{
    const double two32 = 4294967296.0;
    double pmf = exp(-lambda), F = pmf;
    for (int32_t j = 0; j < cap; ++j) {
        if (j > 0) {
            pmf = (pmf * lambda) / (double)j;
            F = F + pmf;
        }
        double t = floor(F * two32);
        uint64_t v = t >= two32 ? (uint64_t)1 << 32 : (uint64_t)t;
        if (j == cap - 1)
            v = (uint64_t)1 << 32;
        thr[j] = v;
        if (v == ((uint64_t)1 << 32))
            return j + 1;
    }
    return cap;
}

/* k = #{ j : thr[j] <= u } */
int32_t or_poisson_sample(uint32_t u, const uint64_t* thr, int32_t n)
{
    int32_t k = 0;
    while (k < n && (uint64_t)u >= thr[k])
        ++k;
    return k;
}

/* Background count lambda = K * rate_hz * dt_ms / 1000, left to right. */
double or_background_lambda(int32_t K, double rate_hz, double dt_ms)
{
    return (((double)K * rate_hz) * dt_ms) / 1000.0;
}

/* Background input of neuron i at step t: k w for the Poisson count k of
 * the step, plus sqrt(k) sd z with z the step's standard normal when sd > 0
 * (the compound Poisson x Gaussian sum of the k event amplitudes). */
double or_background_input(uint64_t seed, int64_t t, int64_t i, const uint64_t* thr, int32_t n_thr, double w,
                           double sd)
{
    const int32_t k = or_poisson_sample(or_background_word(seed, t, i), thr, n_thr);
    double amp = (double)k * w;
    if (sd > 0.0 && k > 0)
        amp += sqrt((double)k) * sd * or_background_normal(seed, t, i);
    return amp;
}

/* ---------------------------------------------------------------------------
 * In-CSR (rows = postsynaptic neuron) -> out-CSR (rows = presynaptic neuron).
 * Entries within an out-row are in ascending postsynaptic order.
 * ------------------------------------------------------------------------- */
static void or_transpose(int64_t N, const int64_t* row_ptr, const int32_t* col,
                         const double* w, int64_t* out_ptr, int32_t* out_post,
                         double* out_w)
{
    int64_t S = row_ptr[N];
    memset(out_ptr, 0, sizeof(int64_t) * (size_t)(N + 1));
    for (int64_t e = 0; e < S; ++e)
        out_ptr[col[e] + 1]++;
    for (int64_t j = 0; j < N; ++j)
        out_ptr[j + 1] += out_ptr[j];
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    memcpy(cur, out_ptr, sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            int64_t pos = cur[col[e]]++;
            out_post[pos] = (int32_t)i;
            out_w[pos] = w[e];
        }
    free(cur);
}

/* ---------------------------------------------------------------------------
 * Open-loop routing: given a spike list (step, pre), the conductance delivered
 * to every target at every step, separately for excitatory and inhibitory
 * presynaptic neurons:
 *     sumE[t][i] = sum over spikes (s, j), s + D = t, j excitatory,
 *                  of sum over edges j -> i of w.
 * Steps t >= T are dropped.  sumE/sumI: [T][N], zeroed here.
 * ------------------------------------------------------------------------- */
int or_route(int64_t N, int64_t T, int32_t D, const int64_t* row_ptr, const int32_t* col,
             const double* w, const uint8_t* inh, const int32_t* spk_step,
             const int32_t* spk_idx, int64_t n_spk, double* sumE, double* sumI)
{
    if (D < 1)
        return 1;
    int64_t S = row_ptr[N];
    int64_t* out_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int32_t* out_post = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S > 0 ? S : 1));
    double* out_w = (double*)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
    or_transpose(N, row_ptr, col, w, out_ptr, out_post, out_w);
    memset(sumE, 0, sizeof(double) * (size_t)(N * T));
    memset(sumI, 0, sizeof(double) * (size_t)(N * T));
    for (int64_t s = 0; s < n_spk; ++s) {
        int64_t t = (int64_t)spk_step[s] + D;
        int32_t j = spk_idx[s];
        if (t >= T || j < 0 || j >= N)
            continue;
        double* dst = (inh[j] ? sumI : sumE) + t * N;
        for (int64_t e = out_ptr[j]; e < out_ptr[j + 1]; ++e)
            dst[out_post[e]] += out_w[e];
    }
    free(out_ptr);
    free(out_post);
    free(out_w);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Conductance-based network, closed loop (or open loop when a forced spike
 * list is given: then the forced spikes, not the network's own, are routed).
 *   row_ptr/col/w: in-CSR by postsynaptic neuron, w in nS.
 *   inh[N]: 1 for inhibitory presynaptic neurons.
 *   D: delay in steps (>= 1).  area_cm2: membrane area.
 *   bg_*: K sources per neuron at rate_hz each, weight bg_w nS; seed for Philox.
 *   trace_idx[n_trace]: neurons whose V is recorded into V_trace[T][n_trace].
 * ------------------------------------------------------------------------- */
int or_simulate_network(const or_model* models, int32_t n_models, const uint8_t* model_id,
                        const double* gbar, int64_t N, int64_t T, double dt,
                        double theta, int32_t v_mode, const double* I_const,
                        const double* I_steps, const double* V0, const int64_t* row_ptr,
                        const int32_t* col,
                        const double* w, const uint8_t* inh, double tau_E, double tau_I,
                        double E_E, double E_I, int32_t D, double area_cm2,
                        double bg_rate_hz, int32_t bg_K, double bg_w, uint64_t seed,
                        double bg_sd, int32_t syn_current,
                        const int32_t* forced_step, const int32_t* forced_idx,
                        int64_t n_forced, const int64_t* trace_idx, int64_t n_trace,
                        double* V_trace, int32_t* counts, int32_t spk_cap,
                        int32_t* spk_step, double* spk_frac, int32_t n_threads)
{
    if (n_models < 1 || N < 0 || T < 0 || !(dt > 0.0) || D < 1 || !(area_cm2 > 0.0))
        return 1;
    int64_t S = row_ptr ? row_ptr[N] : 0;
    int64_t* out_ptr = (int64_t*)calloc((size_t)(N + 1), sizeof(int64_t));
    int32_t* out_post = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S > 0 ? S : 1));
    double* out_w = (double*)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1));
    if (S > 0)
        or_transpose(N, row_ptr, col, w, out_ptr, out_post, out_w);
    double* ringE = (double*)calloc((size_t)(D * N), sizeof(double));
    double* ringI = (double*)calloc((size_t)(D * N), sizeof(double));
    double* V = (double*)malloc(sizeof(double) * (size_t)N);
    double* P = (double*)malloc(sizeof(double) * (size_t)N * OR_MAX_GATES);
    double* Ca = (double*)malloc(sizeof(double) * (size_t)N);
    double* gE = (double*)calloc((size_t)N, sizeof(double));
    double* gI = (double*)calloc((size_t)N, sizeof(double));
    uint8_t* spiked = (uint8_t*)calloc((size_t)N, 1);
    uint64_t thr[64];
    int32_t n_thr = 0;
    if (bg_K > 0 && bg_rate_hz > 0.0)
        n_thr = or_poisson_table(or_background_lambda(bg_K, bg_rate_hz, dt), thr, 64);
    const double dE = exp(-dt / tau_E), dI = exp(-dt / tau_I);
    const double to_mS = 1e-6 / area_cm2;
    int64_t fpos = 0;

    for (int64_t i = 0; i < N; ++i) {
        const or_model* M = &models[model_id ? model_id[i] : 0];
        V[i] = V0[i];
        or_init_neuron(M, V[i], &P[i * OR_MAX_GATES], &Ca[i]);
        if (counts)
            counts[i] = 0;
    }
#ifdef _OPENMP
    if (n_threads > 0)
        omp_set_num_threads(n_threads);
#endif
    for (int64_t t = 0; t < T; ++t) {
        const int64_t slot = t % D;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < N; ++i) {
            const or_model* M = &models[model_id ? model_id[i] : 0];
            double gb[OR_MAX_CH];
            for (int c = 0; c < M->n_channels; ++c)
                gb[c] = gbar ? gbar[(int64_t)c * N + i] : M->ch[c].gbar;
            /* a. delivery of delayed spikes and background */
            gE[i] += ringE[slot * N + i];
            gI[i] += ringI[slot * N + i];
            ringE[slot * N + i] = 0.0;
            ringI[slot * N + i] = 0.0;
            if (n_thr > 0)
                gE[i] += or_background_input(seed, t, i, thr, n_thr, bg_w, bg_sd);
            /* b-e. rates, gates, conductances, V, Ca */
            double Vt = V[i];
            /* injected current: constant part plus the per-step part (e.g. a
               sinusoidal drive), held over the step; current-based synapses
               add their filtered currents (excitatory minus inhibitory) */
            double Ii = (I_const ? I_const[i] : 0.0) + (I_steps ? I_steps[t * N + i] : 0.0);
            double gEs = gE[i] * to_mS, gIs = gI[i] * to_mS;
            if (syn_current) {
                Ii += gE[i] - gI[i];
                gEs = gIs = 0.0;
            }
            double Vn = or_step_neuron(M, gb, dt, Ii, gEs, E_E, gIs, E_I, v_mode, Vt,
                                       &P[i * OR_MAX_GATES], &Ca[i]);
            /* f. threshold */
            spiked[i] = 0;
            if (Vt < theta && Vn >= theta) {
                spiked[i] = 1;
                int32_t c = counts ? counts[i] : 0;
                if (spk_step && c < spk_cap) {
                    spk_step[i * spk_cap + c] = (int32_t)t;
                    spk_frac[i * spk_cap + c] = (theta - Vt) / (Vn - Vt);
                }
                if (counts)
                    counts[i] = c + 1;
            }
            V[i] = Vn;
            /* h. synaptic decay */
            gE[i] *= dE;
            gI[i] *= dI;
        }
        if (V_trace)
            for (int64_t r = 0; r < n_trace; ++r)
                V_trace[t * n_trace + r] = V[trace_idx[r]];
        /* g. push this step's spikes into ring slot t + D */
        const int64_t dst = (t + D) % D;
        if (n_forced < 0) {
            for (int64_t j = 0; j < N; ++j) {
                if (!spiked[j])
                    continue;
                double* ring = (inh[j] ? ringI : ringE) + dst * N;
                for (int64_t e = out_ptr[j]; e < out_ptr[j + 1]; ++e)
                    ring[out_post[e]] += out_w[e];
            }
        } else {
            while (fpos < n_forced && forced_step[fpos] < t)
                ++fpos;
            while (fpos < n_forced && forced_step[fpos] == t) {
                int32_t j = forced_idx[fpos++];
                if (j < 0 || j >= N)
                    continue;
                double* ring = (inh[j] ? ringI : ringE) + dst * N;
                for (int64_t e = out_ptr[j]; e < out_ptr[j + 1]; ++e)
                    ring[out_post[e]] += out_w[e];
            }
        }
    }
    free(out_ptr); free(out_post); free(out_w); free(ringE); free(ringI);
    free(V); free(P); free(Ca); free(gE); free(gI); free(spiked);
    return 0;
}
