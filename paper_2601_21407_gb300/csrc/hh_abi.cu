// C ABI of libhh (see include/hh.h): argument validation, ownership of the
// network's device memory, model preparation and the launch schedule.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "hh_internal.h"

namespace {
thread_local std::string g_err;
// bounds of the device-side waits, process-wide (hh_set_wait_limits)
std::atomic<unsigned long long> g_wait_ns{hh::kWaitLimitNs};
std::atomic<long long> g_wait_polls{hh::kWaitLimitPolls};
}  // namespace

namespace hh {
unsigned long long wait_limit_ns() { return g_wait_ns.load(); }
long long wait_polls() { return g_wait_polls.load(); }

hh_status fail(hh_status s, const char* fmt, ...)
{
    char buf[2048];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}
}  // namespace hh

namespace {
using hh::fail;

#define HH_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA,          \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

}  // namespace

struct hh_net {
    int64_t N = 0;
    int32_t n_nets = 1;
    double dt = 0.0;
    float theta = 0.0f;
    int32_t v_update = 0, precision = 0;
    int32_t kernels = HH_KERNELS_SPECIALISED;
    hh::JitKernels jit{};
    bool jit_ready = false;
    cudaStream_t st = nullptr;
    int64_t t = 0;
    int64_t window_index = 0;

    hh::DevModels models{};
    bool installed[HH_MAX_MODELS] = {false, false, false, false};
    // rate tables of HH_PREC_POLY: per model its fitted rows, and all of
    // them in one device array (model k at models.m[k].poly_base)
    std::vector<float> poly_host[HH_MAX_MODELS];
    float poly_info[HH_MAX_MODELS][3] = {};  // interval, first V, largest relative error
    float4* poly = nullptr;
    size_t poly_cap = 0, poly_rows = 0;
    int32_t max_model_used = 0;

    // state and per-neuron inputs (device)
    float *V = nullptr, *Vlo = nullptr, *P = nullptr, *Plo = nullptr, *Ca = nullptr;
    float *gE = nullptr, *gI = nullptr, *V0 = nullptr, *I_const = nullptr, *gbar = nullptr;
    float* sin_amp = nullptr;
    uint32_t *sin_F = nullptr, *sin_Ph = nullptr;
    hh_morphology morph{};  // n_dendrites 0: point neurons
    int32_t syn_mode = HH_SYN_CONDUCTANCE;
    float bg_sd = 0.0f;

    hh::JitFlags jit_flags() const
    {
        hh::JitFlags f;
        f.v_update = v_update;
        f.drive = sin_amp != nullptr;
        f.cable = morph.n_dendrites > 0;
        f.syn_current = syn_mode == HH_SYN_CURRENT;
        f.compound = has_bg && bg_sd > 0.0f;
        return f;
    }
    uint8_t *model_id = nullptr, *inh = nullptr;
    int32_t *trace_slot = nullptr, *status = nullptr;

    // synapses
    bool has_syn = false;
    int64_t S = 0;
    int64_t* out_ptr = nullptr;
    int32_t* out_post = nullptr;
    float* out_w = nullptr;
    int64_t* ring = nullptr;  // [R][N][2]: {E, I} per neuron and slot
    int32_t D = 1, R = 1;
    int32_t route_segs = 1;  // most 256-synapse segments in one out-CSR row
    // pull routing of dense windows (networks of at most 65,536 neurons whose
    // windows have at most 64 steps): the in-CSR as 8-byte records (16-bit
    // presynaptic index, fixed-point weight in 16-bit parts) and the
    // last-spike tables the window kernels write
    std::vector<int64_t> in_ptr_host;  // the caller's row_ptr where pull routing is possible
    int64_t* in_ptr = nullptr;
    uint2* in_rec = nullptr;
    uint8_t* last_spk = nullptr;
    int64_t pull_min = -1;
    float tau_E = 1.0f, tau_I = 1.0f, E_E = 0.0f, E_I = 0.0f, area = 1.0f;

    // background
    bool has_bg = false;
    float bg_w = 0.0f;
    uint64_t seed = 0;
    int32_t n_thr = 0;
    unsigned long long thr[hh::kMaxPoisson] = {};

    hh::SpikeList list{};
    // routing stream and events of the pipelined window schedule
    cudaStream_t st_route = nullptr;
    cudaEvent_t ev_neuron[hh::kListSlots] = {};
    cudaEvent_t ev_route[hh::kListSlots] = {};
    int32_t W_pipe = 0;  // window length when routing overlaps the next window (0: serial)
    unsigned long long* progress = nullptr;  // persistent kernel: done[4] at 0, routed[4] at 16 (own lines)
    // the window schedule of a call as a CUDA graph: two executables used in
    // turn (each updated in place when the next call has the same shape)
    cudaGraphExec_t gexec[2] = {};
    cudaEvent_t gdone[2] = {};
    int gnext = 0;
    // the call each executable was captured from (its kernel arguments and
    // launch shape); a call identical to the last one relaunches it as is
    std::string gsig[2];
    int glast = -1;
    cudaStream_t st_own = nullptr;  // capture stream when the caller's is the legacy default stream
    cudaEvent_t ev_enter = nullptr, ev_leave = nullptr;
    int persistent_cap = -1;      // co-resident blocks of the persistent kernel (-1: not queried)
    // launch shape of the specialised window schedule (hh_set_launch_shape,
    // hh_autotune): neuron-window block size and routing grid, 0 = default
    int32_t shape_block = 0, shape_route = 0;

    // learned surrogate
    hh::Surrogate* sur = nullptr;
    bool sur_on = false;

    // kernel timing
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    hh_kernel_time ktime[HH_KERNEL_COUNT] = {};

    cudaEvent_t take_event()
    {
        cudaEvent_t e = nullptr;
        if (!ev_pool.empty()) {
            e = ev_pool.back();
            ev_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    }

    cudaError_t harvest()
    {
        for (auto& u : ev_used) {
            float ms = 0.0f;
            cudaError_t e = cudaEventElapsedTime(&ms, u.second.first, u.second.second);
            if (e != cudaSuccess)
                return e;
            ktime[u.first].launches += 1;
            ktime[u.first].total_ms += ms;
            ev_pool.push_back(u.second.first);
            ev_pool.push_back(u.second.second);
        }
        ev_used.clear();
        return cudaSuccess;
    }

    std::vector<void*> allocs;

    template <class T>
    cudaError_t alloc(T** p, size_t count)
    {
        *p = nullptr;
        if (count == 0)
            count = 1;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
        if (e == cudaSuccess)
            allocs.push_back(*p);
        return e;
    }

    // free one tracked allocation now (nullptr: nothing)
    void free_tracked(void* p)
    {
        if (!p)
            return;
        for (size_t k = 0; k < allocs.size(); ++k)
            if (allocs[k] == p) {
                cudaFree(p);
                allocs.erase(allocs.begin() + (long)k);
                return;
            }
    }

    void release()
    {
        if (st)
            cudaStreamSynchronize(st);
        else
            cudaDeviceSynchronize();
        if (sur) {
            hh::surrogate_free(sur);
            sur = nullptr;
        }
        for (void* p : allocs)
            cudaFree(p);
        allocs.clear();
        for (auto& u : ev_used) {
            cudaEventDestroy(u.second.first);
            cudaEventDestroy(u.second.second);
        }
        ev_used.clear();
        for (cudaEvent_t e : ev_pool)
            cudaEventDestroy(e);
        ev_pool.clear();
        for (int k = 0; k < hh::kListSlots; ++k) {
            if (ev_neuron[k])
                cudaEventDestroy(ev_neuron[k]);
            if (ev_route[k])
                cudaEventDestroy(ev_route[k]);
            ev_neuron[k] = ev_route[k] = nullptr;
        }
        if (st_route) {
            cudaStreamDestroy(st_route);
            st_route = nullptr;
        }
        if (st_own) {
            cudaStreamDestroy(st_own);
            st_own = nullptr;
        }
        if (ev_enter)
            cudaEventDestroy(ev_enter);
        if (ev_leave)
            cudaEventDestroy(ev_leave);
        ev_enter = ev_leave = nullptr;
        for (int k = 0; k < 2; ++k) {
            if (gexec[k])
                cudaGraphExecDestroy(gexec[k]);
            if (gdone[k])
                cudaEventDestroy(gdone[k]);
            gexec[k] = nullptr;
            gdone[k] = nullptr;
        }
    }

    // Launch a captured window schedule on stream s: update the executable
    // used two calls ago in place when the shape matches (after its launch
    // has finished), else instantiate it anew.
    cudaError_t launch_graph(cudaGraph_t g, cudaStream_t s, const std::string& sig)
    {
        const int k = gnext;
        gnext ^= 1;
        gsig[k].clear();
        glast = -1;
        cudaError_t e = cudaSuccess;
        if (!gdone[k] && (e = cudaEventCreateWithFlags(&gdone[k], cudaEventDisableTiming)) != cudaSuccess)
            return e;
        if (gexec[k]) {
            if ((e = cudaEventSynchronize(gdone[k])) != cudaSuccess)
                return e;
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(gexec[k], g, &info) != cudaSuccess) {
                cudaGetLastError();  // the failed update is not sticky; instantiate instead
                cudaGraphExecDestroy(gexec[k]);
                gexec[k] = nullptr;
            }
        }
        if (!gexec[k] && (e = cudaGraphInstantiate(&gexec[k], g, 0)) != cudaSuccess) {
            gexec[k] = nullptr;
            return e;
        }
        if ((e = cudaGraphLaunch(gexec[k], s)) != cudaSuccess)
            return e;
        gsig[k] = sig;
        glast = k;
        return cudaEventRecord(gdone[k], s);
    }

    // Launch the last executable again when this call's schedule is the one
    // it was captured from (false: capture anew).  Launches of one
    // executable on one stream run in order.
    bool relaunch_graph(const std::string& sig, cudaStream_t s, cudaError_t* e)
    {
        if (glast < 0 || !gexec[glast] || gsig[glast] != sig)
            return false;
        if ((*e = cudaGraphLaunch(gexec[glast], s)) == cudaSuccess)
            *e = cudaEventRecord(gdone[glast], s);
        return true;
    }

    hh::NeuronParams neuron_params() const
    {
        hh::NeuronParams p{};
        p.N = N;
        p.dt = (float)dt;
        p.theta = theta;
        p.v_update = v_update;
        p.V = V;
        p.Vlo = Vlo;
        p.P = P;
        p.Plo = Plo;
        p.Ca = Ca;
        p.gE = gE;
        p.gI = gI;
        p.poly = poly;
        p.poly_rows = (int32_t)poly_rows;
        p.model_id = model_id;
        p.gbar = gbar;
        p.I_const = I_const;
        p.sin_amp = sin_amp;
        p.sin_F = sin_F;
        p.sin_Ph = sin_Ph;
        p.cable_nd = morph.n_dendrites;
        p.cable_np = morph.n_per_dendrite;
        p.cable_g = morph.g_axial;
        p.cable_gs = morph.n_dendrites > 0 ? (float)((double)morph.g_axial / (double)morph.soma_area_ratio) : 0.0f;
        p.trace_slot = nullptr;
        p.status = status;
        p.ring = ring;
        p.R = R;
        p.last_spk = in_rec && pull_min >= 0 ? last_spk : nullptr;
        p.E_E = E_E;
        p.E_I = E_I;
        p.decE = (float)std::exp(-dt / (double)tau_E);
        p.decI = (float)std::exp(-dt / (double)tau_I);
        p.to_mS = (float)(1e-6 / (double)area);
        // the table ends with 2^32, which no 32-bit word reaches: keep the
        // entries below it
        int32_t nb = 0;
        while (has_bg && nb < n_thr && thr[nb] < (1ull << 32))
            ++nb;
        p.bg_n = nb;
        p.bg_w = bg_w;
        p.bg_sd = bg_sd;
        p.syn_current = syn_mode == HH_SYN_CURRENT ? 1 : 0;
        p.seed = seed;
        // Philox-4x32-10 key schedule (Salmon et al.): the key is bumped by
        // the Weyl constants after every round
        for (uint32_t r = 0; r < 10; ++r) {
            p.rk[2 * r] = (uint32_t)seed + r * 0x9E3779B9u;
            p.rk[2 * r + 1] = (uint32_t)(seed >> 32) + r * 0xBB67AE85u;
        }
        for (int j = 0; j < hh::kMaxPoisson; ++j)
            p.bg_thr[j] = thr[j] < (1ull << 32) ? (uint32_t)thr[j] : 0xffffffffu;
        return p;
    }

    hh::RouteParams route_params() const
    {
        hh::RouteParams r{};
        r.N = N;
        r.out_ptr = out_ptr;
        r.out_post = out_post;
        r.out_w = out_w;
        r.inh = inh;
        r.ringE = ring;
        r.ringI = ring ? ring + 1 : nullptr;
        r.stride = 2;
        r.R = R;
        r.D = D;
        r.open_loop = 0;
        r.n_window = 0;
        r.segs = route_segs;
        r.in_ptr = in_ptr;
        r.in_rec = in_rec;
        r.last_spk = last_spk;
        r.pull_min = in_rec ? pull_min : -1;
        r.pull_w = D >= 2 ? D / 2 : D;
        return r;
    }
};

namespace {

// Poisson CDF thresholds on the 2^32 grid (inversion sampling of the
// background count): thr[j] = min(2^32, floor(F(j) 2^32)), F accumulated as
// pmf_0 = e^-lambda, pmf_j = (pmf_{j-1} lambda)/j; the last entry is 2^32.
int32_t poisson_thresholds(double lambda, unsigned long long* thr, int32_t cap)
{
    const double two32 = 4294967296.0;
    double pmf = std::exp(-lambda), F = pmf;
    for (int32_t j = 0; j < cap; ++j) {
        if (j > 0) {
            pmf = (pmf * lambda) / (double)j;
            F = F + pmf;
        }
        const double x = std::floor(F * two32);
        unsigned long long v = x >= two32 ? (1ull << 32) : (unsigned long long)x;
        if (j == cap - 1)
            v = 1ull << 32;
        thr[j] = v;
        if (v == (1ull << 32))
            return j + 1;
    }
    return cap;
}

bool finite_f(float x) { return std::isfinite(x); }

hh_status check_fn(const hh_fn& f, const char* where)
{
    if (f.form < HH_FN_CONST || f.form > HH_FN_BELL)
        return fail(HH_EINVAL, "%s: unknown rate form %d", where, f.form);
    if (!finite_f(f.a) || !finite_f(f.c) || !finite_f(f.vh) || !finite_f(f.k) || !finite_f(f.vh2) ||
        !finite_f(f.k2))
        return fail(HH_EINVAL, "%s: non-finite rate parameter", where);
    if (f.form != HH_FN_CONST && f.k == 0.0f)
        return fail(HH_EINVAL, "%s: k must be non-zero", where);
    if (f.form == HH_FN_BELL && f.k2 == 0.0f)
        return fail(HH_EINVAL, "%s: k2 must be non-zero", where);
    return HH_OK;
}

hh::DevFn prep_fn(const hh_fn& f)
{
    hh::DevFn d{};
    d.form = f.form;
    d.a = f.a;
    d.c = f.c;
    d.vh = f.vh;
    d.k = f.k;
    const double k = f.k != 0.0f ? (double)f.k : 1.0;
    const double k2 = f.k2 != 0.0f ? (double)f.k2 : 1.0;
    d.ik = (float)(1.0 / k);
    d.s = (float)(1.4426950408889634 / k);
    d.b = (float)(-(double)f.vh * 1.4426950408889634 / k);
    d.vh2 = f.vh2;
    d.ik2 = (float)(1.0 / k2);
    d.s2 = (float)(1.4426950408889634 / k2);
    d.b2 = (float)(-(double)f.vh2 * 1.4426950408889634 / k2);
    d.ia = f.a != 0.0f ? (float)(1.0 / (double)f.a) : 0.0f;
    const double ac = (double)f.a + (double)f.c;
    d.irate = ac != 0.0 ? (float)(1.0 / ac) : 0.0f;
    const double ak = (double)f.a * k;
    d.n0 = (float)ak;
    d.n1 = (float)(ak / 2.0);
    d.n2 = (float)(ak / 12.0);
    d.n4 = (float)(-ak / 720.0);
    return d;
}

// ---------------------------------------------------------------------------
// Polynomial rate tables (HH_PREC_POLY)
// ---------------------------------------------------------------------------

// r(V) = c + form(V) in FP64 (the closed forms of hh_fn; the linoid's
// removable point by its series)
double host_rate(const hh_fn& f, double V)
{
    const double a = f.a, vh = f.vh, k = f.k != 0.0f ? (double)f.k : 1.0;
    double r;
    switch (f.form) {
    case HH_FN_CONST: r = a; break;
    case HH_FN_EXP: r = a * std::exp((V - vh) / k); break;
    case HH_FN_SIGMOID: r = a / (1.0 + std::exp((V - vh) / k)); break;
    case HH_FN_LINOID: {
        const double y = (V - vh) / k;
        r = std::fabs(y) < 1e-8 ? a * k * (1.0 + 0.5 * y) : a * (V - vh) / (-std::expm1(-y));
        break;
    }
    default: {
        const double k2 = f.k2 != 0.0f ? (double)f.k2 : 1.0;
        r = a / (std::exp((V - vh) / k) + std::exp((V - (double)f.vh2) / k2));
        break;
    }
    }
    return r + (double)f.c;
}

// The two tabulated functions of a gate at V: p_inf (0 for a Ca-dependent
// gate, whose p_inf depends on Ca) and 1 - e^{-dt/tau}.
void host_gate(const hh_gate& g, double V, double dt, double* inf, double* E)
{
    double z;
    if (g.kind == HH_GATE_AB) {
        const double al = host_rate(g.f1, V), be = host_rate(g.f2, V);
        *inf = al / (al + be);
        z = dt * (al + be);
    } else {
        *inf = g.kind == HH_GATE_INFTAU ? host_rate(g.f1, V) : 0.0;
        z = dt / host_rate(g.f2, V);
    }
    *E = -std::expm1(-z);
}

struct PolyTable {
    float h = 0.0f, v_lo = 0.0f, err = 0.0f;
    int32_t n = 0, n_gates = 0;
    std::vector<float> c;  // [n][n_gates][2][4]
};

// Cubic interpolation at the four Chebyshev points of [0, 1) for every
// interval of h mV and every function; the interval is halved from 1 mV to
// 1/8 mV until the largest relative error (FP32 Horner, 64 points per
// interval) is at most HH_POLY_REL_ERR.
hh_status poly_fit(const hh_model_desc* m, double dt, PolyTable* out)
{
    std::vector<const hh_gate*> gates;
    for (int c = 0; c < m->n_channels; ++c)
        for (int g = 0; g < m->channels[c].n_gates; ++g)
            gates.push_back(&m->channels[c].gates[g]);
    const int ng = (int)gates.size();
    // monomial coefficients of the interpolant from the values at the nodes:
    // invert the 4 x 4 Vandermonde matrix of the nodes once
    double t[4], Vi[4][8];
    for (int i = 0; i < 4; ++i) {
        t[i] = 0.5 - 0.5 * std::cos((2 * i + 1) * 3.14159265358979323846 / 8.0);
        for (int k = 0; k < 4; ++k) {
            Vi[i][k] = std::pow(t[i], k);
            Vi[i][4 + k] = (i == k) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(Vi[r][col]) > std::fabs(Vi[piv][col]))
                piv = r;
        for (int k = 0; k < 8; ++k)
            std::swap(Vi[col][k], Vi[piv][k]);
        const double d = Vi[col][col];
        for (int k = 0; k < 8; ++k)
            Vi[col][k] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != col) {
                const double f = Vi[r][col];
                for (int k = 0; k < 8; ++k)
                    Vi[r][k] -= f * Vi[col][k];
            }
    }
    // inverse: coefficient k = sum_i inv[k][i] f(t_i)
    double inv[4][4];
    for (int k = 0; k < 4; ++k)
        for (int i = 0; i < 4; ++i)
            inv[k][i] = Vi[k][4 + i];
    const double lo = HH_POLY_V_LO, hi = HH_POLY_V_HI;
    PolyTable T;
    for (double h = 1.0; h >= 0.125; h *= 0.5) {
        T.h = (float)h;
        T.v_lo = (float)lo;
        T.n = (int32_t)std::lround((hi - lo) / h);
        T.n_gates = ng;
        T.c.assign((size_t)T.n * ng * 8, 0.0f);
        double worst = 0.0;
        for (int j = 0; j < T.n; ++j) {
            const double v0 = lo + j * h;
            for (int q = 0; q < ng; ++q) {
                double fv[2][4];
                for (int i = 0; i < 4; ++i)
                    host_gate(*gates[q], v0 + t[i] * h, dt, &fv[0][i], &fv[1][i]);
                for (int f = 0; f < 2; ++f) {
                    float* c = &T.c[(((size_t)j * ng + q) * 2 + f) * 4];
                    for (int k = 0; k < 4; ++k) {
                        double acc = 0.0;
                        for (int i = 0; i < 4; ++i)
                            acc += inv[k][i] * fv[f][i];
                        c[k] = (float)acc;
                    }
                    if (f == 0 && gates[q]->kind == HH_GATE_CA)
                        continue;  // not used
                    for (int u = 0; u < 64; ++u) {
                        const float x = ((float)u + 0.5f) / 64.0f;
                        double ex[2];
                        host_gate(*gates[q], v0 + (double)x * h, dt, &ex[0], &ex[1]);
                        const float pv = std::fma(x, std::fma(x, std::fma(x, c[3], c[2]), c[1]), c[0]);
                        const double e = std::fabs((double)pv - ex[f]) / std::max(std::fabs(ex[f]), 1e-7);
                        if (!(e <= worst))  // NaN counts as the worst
                            worst = std::isfinite(e) ? e : 1e30;
                    }
                }
            }
        }
        T.err = (float)worst;
        if (worst <= HH_POLY_REL_ERR)
            break;
    }
    *out = std::move(T);
    return HH_OK;
}

}  // namespace

namespace hh {
hh_status prep_model(const hh_model_desc* m, double dt, hh::DevModel* out)
{
    if (!(m->C_m > 0.0f) || !finite_f(m->C_m))
        return fail(HH_EINVAL, "model: C_m must be > 0");
    if (m->n_channels < 1 || m->n_channels > HH_MAX_CHANNELS)
        return fail(HH_EINVAL, "model: n_channels %d outside 1..%d", m->n_channels, HH_MAX_CHANNELS);
    hh::DevModel d{};
    d.C_m = m->C_m;
    d.inv_C = (float)(1.0 / (double)m->C_m);
    d.n_ch = m->n_channels;
    d.ca_ch = -1;
    int q = 0;
    for (int c = 0; c < m->n_channels; ++c) {
        const hh_channel& ch = m->channels[c];
        if (ch.n_gates < 0 || ch.n_gates > HH_MAX_GATES_PER_CHANNEL)
            return fail(HH_EINVAL, "channel %d: n_gates %d outside 0..%d", c, ch.n_gates,
                        HH_MAX_GATES_PER_CHANNEL);
        if (!finite_f(ch.E_rev) || !finite_f(ch.gbar) || ch.gbar < 0.0f)
            return fail(HH_EINVAL, "channel %d: E_rev and gbar must be finite, gbar >= 0", c);
        d.E[c] = ch.E_rev;
        d.gbar[c] = ch.gbar;
        d.ch_first[c] = q;
        d.ch_ng[c] = ch.n_gates;
        for (int g = 0; g < ch.n_gates; ++g) {
            if (q >= HH_MAX_GATES)
                return fail(HH_EINVAL, "model: more than %d gates", HH_MAX_GATES);
            const hh_gate& gt = ch.gates[g];
            if (gt.kind < HH_GATE_AB || gt.kind > HH_GATE_CA)
                return fail(HH_EINVAL, "channel %d gate %d: unknown kind %d", c, g, gt.kind);
            if (gt.power < 1 || gt.power > 4)
                return fail(HH_EINVAL, "channel %d gate %d: power %d outside 1..4", c, g, gt.power);
            hh_status s = check_fn(gt.f1, "f1");
            if (s != HH_OK)
                return s;
            if ((s = check_fn(gt.f2, "f2")) != HH_OK)
                return s;
            if (gt.kind == HH_GATE_CA && !(gt.f1.a > 0.0f))
                return fail(HH_EINVAL, "channel %d gate %d: Ca half-activation must be > 0", c, g);
            d.g[q].kind = gt.kind;
            d.g[q].power = gt.power;
            d.g[q].f1 = prep_fn(gt.f1);
            d.g[q].f2 = prep_fn(gt.f2);
            d.gate_ch[q] = c;
            d.gate_last[q] = (g == ch.n_gates - 1);
            d.gate_E[q] = ch.E_rev;
            d.gate_ca[q] = 0;
            ++q;
        }
    }
    d.n_gates = q;
    if (m->ca_channel >= 0) {
        if (m->ca_channel >= m->n_channels)
            return fail(HH_EINVAL, "model: ca_channel %d out of range", m->ca_channel);
        if (m->channels[m->ca_channel].n_gates < 1)
            return fail(HH_EINVAL, "model: the calcium channel needs at least one gate");
        if (!(m->ca_tau > 0.0f) || !finite_f(m->ca_k) || !finite_f(m->ca_rest) || m->ca_rest < 0.0f)
            return fail(HH_EINVAL, "model: calcium pool needs ca_tau > 0, finite ca_k, ca_rest >= 0");
        d.ca_ch = m->ca_channel;
        d.ca_tau = m->ca_tau;
        d.ca_k = m->ca_k;
        d.ca_rest = m->ca_rest;
        d.ca_decay = (float)std::exp(-dt / (double)m->ca_tau);
        const int last = d.ch_first[m->ca_channel] + d.ch_ng[m->ca_channel] - 1;
        d.gate_ca[last] = 1;
    } else if (m->ca_channel != -1) {
        return fail(HH_EINVAL, "model: ca_channel must be -1 or a channel index");
    }
    for (int g = 0; g < d.n_gates; ++g)
        if (d.g[g].kind == HH_GATE_CA && d.ca_ch < 0)
            return fail(HH_EINVAL, "model: a Ca-dependent gate needs a calcium pool");
    *out = d;
    return HH_OK;
}
}  // namespace hh

namespace {
using hh::prep_model;

template <class T>
cudaError_t copy_in(T* dst, const T* src, size_t count, cudaStream_t st)
{
    if (count == 0)
        return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDefault, st);
    if (e != cudaSuccess)
        return e;
    return cudaStreamSynchronize(st);
}

hh_status build_network(const hh_net_desc* d, hh_net* n)
{
    const int64_t N = d->n_neurons;
    n->N = N;
    n->n_nets = d->n_nets;
    n->dt = d->dt_ms;
    n->theta = d->v_threshold;
    n->v_update = d->v_update;
    n->precision = d->precision;
    n->kernels = d->kernels;
    n->st = (cudaStream_t)d->stream;
    cudaStream_t st = n->st;

    HH_CUDA(n->alloc(&n->V, N));
    HH_CUDA(n->alloc(&n->V0, N));
    HH_CUDA(n->alloc(&n->Ca, N));
    HH_CUDA(n->alloc(&n->gE, N));
    HH_CUDA(n->alloc(&n->gI, N));
    HH_CUDA(n->alloc(&n->P, (size_t)N * hh::kMaxGates));
    HH_CUDA(n->alloc(&n->status, 1));
    HH_CUDA(n->alloc(&n->trace_slot, N));
    if (n->precision == HH_PREC_COMPENSATED) {
        HH_CUDA(n->alloc(&n->Vlo, N));
        HH_CUDA(n->alloc(&n->Plo, (size_t)N * hh::kMaxGates));
    }
    HH_CUDA(copy_in(n->V0, d->V0, (size_t)N, st));
    HH_CUDA(cudaMemcpyAsync(n->V, n->V0, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    HH_CUDA(cudaMemsetAsync(n->P, 0, (size_t)N * hh::kMaxGates * sizeof(float), st));
    HH_CUDA(cudaMemsetAsync(n->Ca, 0, N * sizeof(float), st));
    HH_CUDA(cudaMemsetAsync(n->gE, 0, N * sizeof(float), st));
    HH_CUDA(cudaMemsetAsync(n->gI, 0, N * sizeof(float), st));
    HH_CUDA(cudaMemsetAsync(n->status, 0, sizeof(int32_t), st));
    if (n->Vlo) {
        HH_CUDA(cudaMemsetAsync(n->Vlo, 0, N * sizeof(float), st));
        HH_CUDA(cudaMemsetAsync(n->Plo, 0, (size_t)N * hh::kMaxGates * sizeof(float), st));
    }
    if (d->I_const) {
        HH_CUDA(n->alloc(&n->I_const, N));
        HH_CUDA(copy_in(n->I_const, d->I_const, (size_t)N, st));
    }
    if (d->morph) {
        const hh_morphology& m = *d->morph;
        if (m.n_dendrites < 1 || m.n_dendrites > 3 || m.n_per_dendrite < 1 ||
            1 + m.n_dendrites * m.n_per_dendrite > HH_CABLE_LANES)
            return fail(HH_EINVAL, "morphology: 1..3 dendrites, and 1 + n_dendrites n_per_dendrite <= %d",
                        HH_CABLE_LANES);
        if (!finite_f(m.g_axial) || m.g_axial < 0.0f || !finite_f(m.soma_area_ratio) || !(m.soma_area_ratio > 0.0f))
            return fail(HH_EINVAL, "morphology: g_axial >= 0 and soma_area_ratio > 0, finite");
        if (N % HH_CABLE_LANES != 0)
            return fail(HH_EINVAL, "with a morphology n_neurons must be a multiple of %d", HH_CABLE_LANES);
        n->morph = m;
    }
    if (d->sin_amp) {
        // phase advance per step and initial phase as 32-bit fractions of a cycle
        if (!d->sin_freq_hz)
            return fail(HH_EINVAL, "sin_amp needs sin_freq_hz");
        std::vector<float> a(N), f(N), ph(N, 0.0f);
        HH_CUDA(cudaMemcpy(a.data(), d->sin_amp, N * sizeof(float), cudaMemcpyDefault));
        HH_CUDA(cudaMemcpy(f.data(), d->sin_freq_hz, N * sizeof(float), cudaMemcpyDefault));
        if (d->sin_phase)
            HH_CUDA(cudaMemcpy(ph.data(), d->sin_phase, N * sizeof(float), cudaMemcpyDefault));
        std::vector<uint32_t> F(N), P(N);
        const double two32 = 4294967296.0;
        for (int64_t i = 0; i < N; ++i) {
            if (!finite_f(a[i]) || !finite_f(f[i]) || !(f[i] >= 0.0f) || !finite_f(ph[i]))
                return fail(HH_EINVAL, "sinusoidal drive of neuron %lld: finite amp, phase and freq >= 0 needed",
                            (long long)i);
            const double adv = std::nearbyint((double)f[i] * d->dt_ms * two32 / 1000.0);
            F[i] = (uint32_t)(uint64_t)std::fmod(adv, two32);
            double pc = std::nearbyint((double)ph[i] * two32);
            pc = std::fmod(pc, two32);
            if (pc < 0.0)
                pc += two32;
            P[i] = (uint32_t)(uint64_t)pc;
        }
        HH_CUDA(n->alloc(&n->sin_amp, N));
        HH_CUDA(n->alloc(&n->sin_F, N));
        HH_CUDA(n->alloc(&n->sin_Ph, N));
        HH_CUDA(cudaMemcpy(n->sin_amp, a.data(), N * sizeof(float), cudaMemcpyHostToDevice));
        HH_CUDA(cudaMemcpy(n->sin_F, F.data(), N * sizeof(uint32_t), cudaMemcpyHostToDevice));
        HH_CUDA(cudaMemcpy(n->sin_Ph, P.data(), N * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    if (d->model_id) {
        std::vector<uint8_t> h(N);
        HH_CUDA(cudaMemcpy(h.data(), d->model_id, N, cudaMemcpyDefault));
        int32_t mx = 0;
        for (int64_t i = 0; i < N; ++i)
            mx = h[i] > mx ? h[i] : mx;
        if (mx >= HH_MAX_MODELS)
            return fail(HH_EINVAL, "model_id %d >= HH_MAX_MODELS", mx);
        n->max_model_used = mx;
        HH_CUDA(n->alloc(&n->model_id, N));
        HH_CUDA(copy_in(n->model_id, h.data(), (size_t)N, st));
    }

    // synapses: in-CSR -> out-CSR on the device
    n->has_syn = d->n_synapses > 0;
    if (d->n_synapses < 0)
        return fail(HH_EINVAL, "n_synapses < 0");
    n->tau_E = d->tau_E;
    n->tau_I = d->tau_I;
    n->E_E = d->E_E;
    n->E_I = d->E_I;
    n->area = d->area_cm2;
    n->D = d->delay_steps;
    if (n->has_syn || d->bg_sources > 0) {
        if (!(d->tau_E > 0.0f) || !(d->tau_I > 0.0f) || !(d->area_cm2 > 0.0f) ||
            !finite_f(d->E_E) || !finite_f(d->E_I))
            return fail(HH_EINVAL, "synapses need tau_E, tau_I, area_cm2 > 0 and finite E_E, E_I");
    }
    if (n->has_syn) {
        if (d->delay_steps < 1 || d->delay_steps > 1024)
            return fail(HH_EINVAL, "delay_steps %d outside 1..1024", d->delay_steps);
        if (!d->row_ptr || !d->col_idx || !d->weight)
            return fail(HH_EINVAL, "row_ptr, col_idx and weight are required when n_synapses > 0");
        const int64_t S = d->n_synapses;
        n->S = S;
        std::vector<int64_t> rp(N + 1);
        HH_CUDA(cudaMemcpy(rp.data(), d->row_ptr, (N + 1) * sizeof(int64_t), cudaMemcpyDefault));
        if (rp[0] != 0 || rp[N] != S)
            return fail(HH_EINVAL, "row_ptr[0] must be 0 and row_ptr[N] = n_synapses");
        for (int64_t i = 0; i < N; ++i) {
            if (rp[i + 1] < rp[i])
                return fail(HH_EINVAL, "row_ptr decreases at row %lld", (long long)i);
            if (rp[i + 1] - rp[i] > 32767)
                return fail(HH_EINVAL, "in-degree of neuron %lld exceeds 32767", (long long)i);
        }
        int32_t* col = nullptr;
        float* w = nullptr;
        int64_t* drp = nullptr;
        int32_t* cnt = nullptr;
        unsigned long long* cursor = nullptr;
        hh_status rc = HH_OK;
        auto cleanup = [&]() {
            cudaStreamSynchronize(st);
            for (void* p : {(void*)col, (void*)w, (void*)drp, (void*)cnt, (void*)cursor})
                if (p)
                    cudaFree(p);
        };
        do {
            cudaError_t e;
            if ((e = cudaMalloc(&col, S * sizeof(int32_t))) != cudaSuccess ||
                (e = cudaMalloc(&w, S * sizeof(float))) != cudaSuccess ||
                (e = cudaMalloc(&drp, (N + 1) * sizeof(int64_t))) != cudaSuccess ||
                (e = cudaMalloc(&cnt, (N + 1) * sizeof(int32_t))) != cudaSuccess ||
                (e = cudaMalloc(&cursor, (N + 1) * sizeof(unsigned long long))) != cudaSuccess) {
                rc = fail(HH_ENOMEM, "allocating the CSR staging buffers: %s", cudaGetErrorString(e));
                break;
            }
            if ((e = copy_in(col, d->col_idx, (size_t)S, st)) != cudaSuccess ||
                (e = copy_in(w, d->weight, (size_t)S, st)) != cudaSuccess ||
                (e = copy_in(drp, rp.data(), (size_t)N + 1, st)) != cudaSuccess ||
                (e = cudaMemsetAsync(cnt, 0, (N + 1) * sizeof(int32_t), st)) != cudaSuccess ||
                (e = hh::launch_csr_check(col, w, S, N, cnt + N, st)) != cudaSuccess) {
                rc = fail(HH_ECUDA, "copying the CSR: %s", cudaGetErrorString(e));
                break;
            }
            int32_t flag = 0;
            if ((e = cudaMemcpyAsync(&flag, cnt + N, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rc = fail(HH_ECUDA, "checking the CSR: %s", cudaGetErrorString(e));
                break;
            }
            if (flag & 1) {
                rc = fail(HH_EINVAL, "col_idx holds an index outside [0, N)");
                break;
            }
            if (flag & 2) {
                rc = fail(HH_EINVAL, "weight holds a value that is not finite or outside [0, 65536) nS");
                break;
            }
            std::vector<int32_t> hc(N);
            std::vector<int64_t> op(N + 1);
            if ((e = hh::launch_count_pre(col, S, cnt, st)) != cudaSuccess ||
                (e = cudaMemcpyAsync(hc.data(), cnt, N * sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rc = fail(HH_ECUDA, "counting out-degrees: %s", cudaGetErrorString(e));
                break;
            }
            op[0] = 0;
            int32_t max_out = 0;
            for (int64_t j = 0; j < N; ++j) {
                op[j + 1] = op[j] + hc[j];
                max_out = hc[j] > max_out ? hc[j] : max_out;
            }
            // 256-synapse segments per row, counted from the row start rounded down to 4
            n->route_segs = (max_out + 3 + 255) / 256;
            // 4 entries of padding: the routing kernel reads rows as aligned int4/float4
            if ((e = n->alloc(&n->out_ptr, N + 1)) != cudaSuccess ||
                (e = n->alloc(&n->out_post, S + 4)) != cudaSuccess ||
                (e = n->alloc(&n->out_w, S + 4)) != cudaSuccess ||
                (e = cudaMemsetAsync(n->out_post + S, 0, 4 * sizeof(int32_t), st)) != cudaSuccess ||
                (e = cudaMemsetAsync(n->out_w + S, 0, 4 * sizeof(float), st)) != cudaSuccess) {
                rc = fail(HH_ENOMEM, "allocating the out-CSR: %s", cudaGetErrorString(e));
                break;
            }
            if ((e = copy_in(n->out_ptr, op.data(), (size_t)N + 1, st)) != cudaSuccess ||
                (e = copy_in(reinterpret_cast<int64_t*>(cursor), op.data(), (size_t)N, st)) != cudaSuccess ||
                (e = hh::launch_fill_out(drp, col, w, N, cursor, n->out_post, n->out_w, st)) !=
                    cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rc = fail(HH_ECUDA, "filling the out-CSR: %s", cudaGetErrorString(e));
                break;
            }
            // pull routing is possible for windows of D/2 steps (1 step when
            // D = 1) of at most kPullMaxW steps; its in-CSR is built from the
            // out-CSR when it is first asked for (hh_set_route_pull)
            const int32_t Wnet = n->D >= 2 ? n->D / 2 : n->D;
            if (N <= hh::kPullMaxN && Wnet <= hh::kPullMaxW)
                n->in_ptr_host = rp;
        } while (0);
        cleanup();
        if (rc != HH_OK)
            return rc;
        if (d->is_inhibitory) {
            // padded to the last-spike tables' row (zeros), read 16 at a time
            const size_t Np = (size_t)hh::pull_stride(N);
            HH_CUDA(n->alloc(&n->inh, Np));
            HH_CUDA(cudaMemsetAsync(n->inh, 0, Np, st));
            HH_CUDA(copy_in(n->inh, d->is_inhibitory, (size_t)N, st));
        }
    }
    // background
    if (d->bg_sources < 0 || !(d->bg_rate_hz >= 0.0f) || !(d->bg_weight_nS >= 0.0f) ||
        !finite_f(d->bg_rate_hz) || !finite_f(d->bg_weight_nS))
        return fail(HH_EINVAL, "background needs bg_sources >= 0, finite bg_rate_hz >= 0, bg_weight_nS >= 0");
    n->has_bg = d->bg_sources > 0 && d->bg_rate_hz > 0.0f;
    n->seed = d->seed;
    n->bg_w = d->bg_weight_nS;
    if (!finite_f(d->bg_weight_sd) || d->bg_weight_sd < 0.0f)
        return fail(HH_EINVAL, "bg_weight_sd must be finite and >= 0");
    n->bg_sd = d->bg_weight_sd;
    if (d->syn_mode != HH_SYN_CONDUCTANCE && d->syn_mode != HH_SYN_CURRENT)
        return fail(HH_EINVAL, "unknown syn_mode %d", d->syn_mode);
    n->syn_mode = d->syn_mode;
    if (n->has_bg) {
        const double lambda = (((double)d->bg_sources * (double)d->bg_rate_hz) * d->dt_ms) / 1000.0;
        n->n_thr = poisson_thresholds(lambda, n->thr, hh::kMaxPoisson);
    }
    // delay ring and window spike lists
    if (n->has_syn || n->has_bg) {
        n->R = n->has_syn ? n->D : 1;
        if ((uint64_t)n->R * (uint64_t)N >= (1ull << 32))
            return fail(HH_EINVAL, "delay_steps x n_neurons must stay below 2^32 (delay-line index)");
        HH_CUDA(n->alloc(&n->ring, (size_t)n->R * N * 2));
        HH_CUDA(cudaMemsetAsync(n->ring, 0, (size_t)n->R * N * 2 * sizeof(int64_t), st));
        const int64_t W = n->has_syn ? n->D : 1;
        n->list.cap = N * ((W + 1) / 2) + 32;
        HH_CUDA(n->alloc(&n->list.step, (size_t)hh::kListSlots * n->list.cap));
        HH_CUDA(n->alloc(&n->list.idx, (size_t)hh::kListSlots * n->list.cap));
        HH_CUDA(n->alloc(&n->list.counter, hh::kListSlots));
        HH_CUDA(cudaMemsetAsync(n->list.counter, 0, hh::kListSlots * sizeof(int32_t), st));
        if (n->has_syn && n->D >= 2) {
            // windows of W <= D/2 steps: the spikes of window w arrive in window
            // w + 2 at the earliest, so routing window w may overlap window w + 1
            n->W_pipe = n->D / 2;
            int lo = 0, hi = 0;
            HH_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            HH_CUDA(cudaStreamCreateWithPriority(&n->st_route, cudaStreamNonBlocking, lo));
            if (!n->st) {
                // the legacy default stream cannot be captured: calls on it run
                // their schedule on a stream of the library, ordered by events
                HH_CUDA(cudaStreamCreateWithFlags(&n->st_own, cudaStreamNonBlocking));
                HH_CUDA(cudaEventCreateWithFlags(&n->ev_enter, cudaEventDisableTiming));
                HH_CUDA(cudaEventCreateWithFlags(&n->ev_leave, cudaEventDisableTiming));
            }
            for (int k = 0; k < hh::kListSlots; ++k) {
                HH_CUDA(cudaEventCreateWithFlags(&n->ev_neuron[k], cudaEventDisableTiming));
                HH_CUDA(cudaEventCreateWithFlags(&n->ev_route[k], cudaEventDisableTiming));
            }
            HH_CUDA(n->alloc(&n->progress, 32));
        }
    }
    HH_CUDA(cudaStreamSynchronize(st));
    return HH_OK;
}

// Blocks of the persistent kernel that fit on the GPU at once (queried once
// per compiled kernel set).
int persistent_capacity(hh_net* n)
{
    if (n->persistent_cap < 0)
        n->persistent_cap = hh::jit_persistent_capacity(n->jit, n->neuron_params());
    return n->persistent_cap;
}

int max_gates_installed(const hh_net* n)
{
    int g = 1;
    for (int m = 0; m < HH_MAX_MODELS; ++m)
        if (n->installed[m] && n->models.m[m].n_gates > g)
            g = n->models.m[m].n_gates;
    return g;
}

}  // namespace

extern "C" {

hh_status hh_create_network(const hh_net_desc* d, hh_net** out)
{
    if (!out)
        return fail(HH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d)
        return fail(HH_EINVAL, "descriptor is NULL");
    if (d->n_neurons < 1 || d->n_neurons > ((int64_t)1 << 31) - 1)
        return fail(HH_EINVAL, "n_neurons %lld outside 1..2^31-1", (long long)d->n_neurons);
    if (d->n_nets < 1)
        return fail(HH_EINVAL, "n_nets must be >= 1");
    if (d->n_nets > 1 && d->net_offsets) {
        if (d->net_offsets[0] != 0 || d->net_offsets[d->n_nets] != d->n_neurons)
            return fail(HH_EINVAL, "net_offsets must run from 0 to n_neurons");
        for (int32_t k = 0; k < d->n_nets; ++k)
            if (d->net_offsets[k + 1] < d->net_offsets[k])
                return fail(HH_EINVAL, "net_offsets decrease at %d", k);
    }
    if (!(d->dt_ms > 0.0) || !std::isfinite(d->dt_ms))
        return fail(HH_EINVAL, "dt_ms must be > 0");
    if (!finite_f(d->v_threshold))
        return fail(HH_EINVAL, "v_threshold must be finite");
    if (d->v_update != HH_V_EXP_EULER && d->v_update != HH_V_FWD_EULER)
        return fail(HH_EINVAL, "unknown v_update %d", d->v_update);
    if (d->precision < HH_PREC_FAST || d->precision > HH_PREC_POLY)
        return fail(HH_EINVAL, "unknown precision %d", d->precision);
    if (d->precision == HH_PREC_POLY && d->kernels == HH_KERNELS_TABLE)
        return fail(HH_EUNSUPPORTED, "HH_PREC_POLY needs HH_KERNELS_SPECIALISED or HH_KERNELS_PERSISTENT");
    if (d->kernels != HH_KERNELS_SPECIALISED && d->kernels != HH_KERNELS_TABLE &&
        d->kernels != HH_KERNELS_PERSISTENT)
        return fail(HH_EINVAL, "unknown kernels %d", d->kernels);
    if (!d->V0)
        return fail(HH_EINVAL, "V0 is required");
    hh_net* n = new (std::nothrow) hh_net();
    if (!n)
        return fail(HH_ENOMEM, "host allocation failed");
    hh_status s = build_network(d, n);
    if (s != HH_OK) {
        std::string keep = g_err;
        n->release();
        delete n;
        g_err = keep;
        return s;
    }
    *out = n;
    return HH_OK;
}

hh_status hh_set_channels(hh_net* net, int32_t model_index, const hh_model_desc* m, const float* gbar)
{
    if (!net || !m)
        return fail(HH_EINVAL, "net and model must not be NULL");
    if (model_index < 0 || model_index >= HH_MAX_MODELS)
        return fail(HH_EINVAL, "model_index %d outside 0..%d", model_index, HH_MAX_MODELS - 1);
    hh::DevModel dm{};
    hh_status s = prep_model(m, net->dt, &dm);
    if (s != HH_OK)
        return s;
    net->models.m[model_index] = dm;
    net->installed[model_index] = true;
    net->jit_ready = false;
    net->models.max_gates = max_gates_installed(net);
    net->models.n = HH_MAX_MODELS;
    if (net->precision == HH_PREC_POLY) {
        PolyTable T;
        if ((s = poly_fit(m, net->dt, &T)) != HH_OK)
            return s;
        net->poly_host[model_index] = std::move(T.c);
        net->poly_info[model_index][0] = T.h;
        net->poly_info[model_index][1] = T.v_lo;
        net->poly_info[model_index][2] = T.err;
        // every installed model's rows in one device array, each row padded
        // to 2 n_gates + 1 coefficient vectors (an odd stride)
        auto rows_of = [&](int k) {
            const hh::DevModel& M = net->models.m[k];
            const size_t n = net->poly_host[k].size() / (8 * (size_t)(M.n_gates > 0 ? M.n_gates : 1));
            return n * (size_t)(2 * M.n_gates + 1);
        };
        size_t total = 0;
        for (int k = 0; k < HH_MAX_MODELS; ++k)
            if (net->installed[k] && !net->poly_host[k].empty())
                total += rows_of(k);
        if (total > net->poly_cap) {
            net->free_tracked(net->poly);
            net->poly = nullptr;
            net->poly_cap = 0;
            HH_CUDA(net->alloc(&net->poly, total));
            net->poly_cap = total;
        }
        size_t off = 0;
        for (int k = 0; k < HH_MAX_MODELS; ++k) {
            hh::DevModel& M = net->models.m[k];
            M.poly_n = 0;
            if (!net->installed[k] || net->poly_host[k].empty())
                continue;
            const int ng = M.n_gates, stride = 2 * ng + 1;
            const size_t n = net->poly_host[k].size() / (8 * (size_t)ng);
            std::vector<float4> padded(n * stride, make_float4(0.f, 0.f, 0.f, 0.f));
            for (size_t j = 0; j < n; ++j)
                for (int v = 0; v < 2 * ng; ++v) {
                    const float* c = &net->poly_host[k][(j * 2 * ng + v) * 4];
                    padded[j * stride + v] = make_float4(c[0], c[1], c[2], c[3]);
                }
            HH_CUDA(cudaMemcpy(net->poly + off, padded.data(), padded.size() * sizeof(float4),
                               cudaMemcpyHostToDevice));
            M.poly_base = (int32_t)off;
            M.poly_stride = stride;
            M.poly_n = (int32_t)n;
            M.poly_vlo = net->poly_info[k][1];
            M.poly_ih = 1.0f / net->poly_info[k][0];
            off += padded.size();
        }
        net->poly_rows = off;
        if (off > (size_t)INT32_MAX)
            return fail(HH_EINVAL, "rate tables too large");
    }
    if (gbar || net->gbar) {
        if (!net->gbar) {
            // first per-neuron table: every other model's neurons take their defaults
            HH_CUDA(net->alloc(&net->gbar, (size_t)hh::kMaxChannels * net->N));
            HH_CUDA(hh::launch_fill_gbar(net->models, net->N, net->model_id, -1, nullptr, net->gbar,
                                         net->st));
        }
        float* staged = nullptr;
        if (gbar) {
            const size_t cnt = (size_t)m->n_channels * net->N;
            HH_CUDA(cudaMalloc(&staged, cnt * sizeof(float)));
            cudaError_t e = copy_in(staged, gbar, cnt, net->st);
            if (e != cudaSuccess) {
                cudaFree(staged);
                return fail(HH_ECUDA, "copying gbar: %s", cudaGetErrorString(e));
            }
        }
        cudaError_t e = hh::launch_fill_gbar(net->models, net->N, net->model_id, model_index, staged,
                                             net->gbar, net->st);
        cudaError_t e2 = cudaStreamSynchronize(net->st);
        if (staged)
            cudaFree(staged);
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(HH_ECUDA, "filling gbar: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    hh::NeuronParams p = net->neuron_params();
    HH_CUDA(hh::launch_init_state(net->models, p, nullptr, model_index, net->precision, net->st));
    HH_CUDA(cudaStreamSynchronize(net->st));
    return HH_OK;
}

hh_status hh_step_n(hh_net* net, int32_t n_steps, const float* I_steps, const hh_record* rec)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (n_steps < 0)
        return fail(HH_EINVAL, "n_steps < 0");
    for (int m = 0; m <= net->max_model_used; ++m)
        if (!net->installed[m])
            return fail(HH_ESTATE, "model %d is used but was not installed with hh_set_channels", m);
    if (net->t + n_steps > (int64_t)INT32_MAX)
        return fail(HH_EINVAL, "step index would exceed 2^31-1");
    hh::RecordParams R{};
    if (rec) {
        if (rec->n_trace < 0 || (rec->V_trace && rec->n_trace == 0))
            return fail(HH_EINVAL, "n_trace must be > 0 when V_trace is given");
        if (rec->spikes && !rec->n_spikes)
            return fail(HH_EINVAL, "spikes needs an n_spikes counter");
        if (rec->spike_cap < 0)
            return fail(HH_EINVAL, "spike_cap < 0");
        if (!rec->trace_idx && rec->n_trace > net->N)
            return fail(HH_EINVAL, "n_trace > N without trace_idx");
        R.V_trace = rec->V_trace;
        R.n_trace = rec->V_trace ? rec->n_trace : 0;
        R.spikes = rec->spikes;
        R.spike_cap = rec->spikes ? rec->spike_cap : 0;
        R.n_spikes = reinterpret_cast<unsigned long long*>(rec->n_spikes);
        R.counts = rec->counts;
    }
    if (n_steps == 0)
        return HH_OK;
    hh::NeuronParams p = net->neuron_params();
    if (R.V_trace && rec->trace_idx) {
        HH_CUDA(cudaMemsetAsync(net->trace_slot, 0xff, net->N * sizeof(int32_t), net->st));
        HH_CUDA(hh::launch_trace_slots(rec->trace_idx, rec->n_trace, net->N, net->trace_slot, net->st));
        p.trace_slot = net->trace_slot;
    }
    // optional event bracketing of each launch (hh_profile)
    auto timed_on = [&](cudaStream_t s, int kind, auto&& launch) -> cudaError_t {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (net->profiling) {
            e0 = net->take_event();
            e1 = net->take_event();
            if (!e0 || !e1)
                return cudaErrorMemoryAllocation;
            cudaError_t e = cudaEventRecord(e0, s);
            if (e != cudaSuccess)
                return e;
        }
        cudaError_t e = launch();
        if (e != cudaSuccess || !net->profiling)
            return e;
        e = cudaEventRecord(e1, s);
        net->ev_used.push_back({kind, {e0, e1}});
        return e;
    };
    auto timed = [&](int kind, auto&& launch) -> cudaError_t { return timed_on(net->st, kind, launch); };
    const bool spec = net->kernels != HH_KERNELS_TABLE;
    if (spec && !net->jit_ready) {
        std::string err;
        if (!hh::jit_get(net->models, net->installed, net->precision, net->jit_flags(), &net->jit, &err))
            return fail(HH_ECUDA, "%s", err.c_str());
        net->jit_ready = true;
        net->persistent_cap = -1;
    }
    if (net->sur_on) {
        if (R.V_trace)
            return fail(HH_EUNSUPPORTED, "V traces are not recorded while the surrogate is enabled");
        if (I_steps)
            return fail(HH_EUNSUPPORTED, "per-step currents are not supported while the surrogate is enabled");
        const int W = hh::surrogate_window_steps(net->sur);
        const int n_win = n_steps / W, rem = n_steps % W;
        for (int w = 0; w < n_win; ++w) {
            const int64_t t0 = net->t + (int64_t)w * W;
            HH_CUDA(timed(HH_KERNEL_NEURON, [&] {
                return hh::surrogate_window(net->models, net->sur, p, net->precision, net->st);
            }));
            HH_CUDA(timed(HH_KERNEL_NEURON, [&] {
                return hh::jit_launch_indexed(net->jit, p, hh::surrogate_fb_list(net->sur),
                                              hh::surrogate_fb_count(net->sur), net->N, t0, W, R, net->st);
            }));
        }
        if (rem)
            HH_CUDA(timed(HH_KERNEL_NEURON, [&] {
                return hh::jit_launch_independent(net->jit, p, net->t + (int64_t)n_win * W, rem, I_steps, R,
                                                  net->st);
            }));
        net->t += n_steps;
        return HH_OK;
    }
    if (!net->has_syn && !net->has_bg) {
        if (spec)
            HH_CUDA(timed(HH_KERNEL_NEURON, [&] {
                return hh::jit_launch_independent(net->jit, p, net->t, n_steps, I_steps, R, net->st);
            }));
        else
        HH_CUDA(timed(HH_KERNEL_NEURON, [&] { return hh::launch_independent(net->models, p, net->precision, net->t, n_steps, I_steps, R,
                                       net->st); }));
    } else if (net->kernels == HH_KERNELS_PERSISTENT && net->W_pipe > 0 &&
               (int64_t)persistent_capacity(net) * hh::kPersistNeurons >= net->N) {
        // one cooperative launch for the whole call
        const hh::RouteParams rp = net->route_params();
        const int32_t W = net->W_pipe;
        const int64_t n_win = (n_steps + W - 1) / W;
        HH_CUDA(cudaMemsetAsync(net->progress, 0, 32 * sizeof(unsigned long long), net->st));
        HH_CUDA(cudaMemsetAsync(net->list.counter, 0, hh::kListSlots * sizeof(int32_t), net->st));
        const hh::PhaseCounters pc{net->progress, net->progress + 16, hh::wait_limit_ns()};
        HH_CUDA(timed(HH_KERNEL_NEURON, [&] {
            return hh::jit_launch_persistent(net->jit, p, rp, net->t, n_steps, W, net->window_index, I_steps, R,
                                             net->list, pc, net->st);
        }));
        net->window_index += n_win;
    } else {
        const hh::RouteParams rp = net->route_params();
        const bool pipe = net->W_pipe > 0;
        const int32_t Wmax = net->has_syn ? (pipe ? net->W_pipe : net->D) : (1 << 30);
        // Window schedule.  Waits on routing events of the previous call are
        // not needed: the caller's stream waited for its last routing launch.
        const int64_t gw_first = net->window_index;
        auto enqueue = [&]() -> cudaError_t {
            cudaError_t e = cudaSuccess;
            int64_t last_route = -1;
            for (int32_t w0 = 0; w0 < n_steps; w0 += Wmax) {
                const int32_t W = (n_steps - w0) < Wmax ? (n_steps - w0) : Wmax;
                const int64_t gw = net->window_index;
                const int32_t slot = (int32_t)(gw % hh::kListSlots);
                hh::RecordParams Rw = R;
                if (Rw.V_trace)
                    Rw.V_trace += (int64_t)w0 * Rw.n_trace;
                const float* Iw = I_steps ? I_steps + (int64_t)w0 * net->N : nullptr;
                // the input of this window was routed by window gw - 2
                if (pipe && gw - 2 >= gw_first &&
                    (e = cudaStreamWaitEvent(net->st, net->ev_route[(gw - 2) % hh::kListSlots], 0)) != cudaSuccess)
                    return e;
                e = timed(HH_KERNEL_NEURON, [&] {
                    // in the pipelined schedule the window's delay-line slots
                    // depend only on routing launches the stream waited for
                    if (spec)
                        return hh::jit_launch_window(net->jit, p, net->t + w0, W, slot, Iw, Rw, net->list,
                                                     pipe && net->has_syn ? 1 : 0, net->shape_block, net->st);
                    return hh::launch_net_window(net->models, p, net->precision, net->t + w0, W, slot, Iw, Rw,
                                                 net->list, net->st);
                });
                if (e != cudaSuccess)
                    return e;
                if (net->has_syn && pipe) {
                    if ((e = cudaEventRecord(net->ev_neuron[slot], net->st)) != cudaSuccess ||
                        (e = cudaStreamWaitEvent(net->st_route, net->ev_neuron[slot], 0)) != cudaSuccess ||
                        (e = timed_on(net->st_route, HH_KERNEL_ROUTE, [&] {
                             return hh::launch_route_window(rp, net->list, slot, net->t + w0, W, net->shape_route,
                                                            net->st_route);
                         })) != cudaSuccess ||
                        (e = cudaEventRecord(net->ev_route[slot], net->st_route)) != cudaSuccess)
                        return e;
                    last_route = gw;
                } else if (net->has_syn) {
                    e = timed(HH_KERNEL_ROUTE, [&] {
                        return hh::launch_route_window(rp, net->list, slot, net->t + w0, W, net->shape_route,
                                                       net->st);
                    });
                } else {
                    e = cudaMemsetAsync(net->list.counter + slot, 0, sizeof(int32_t), net->st);
                }
                if (e != cudaSuccess)
                    return e;
                net->window_index++;
            }
            // the caller's stream sees every routing launch of this call complete
            if (last_route >= 0)
                e = cudaStreamWaitEvent(net->st, net->ev_route[last_route % hh::kListSlots], 0);
            return e;
        };
        // With routing on a second stream the schedule is captured into a CUDA
        // graph and launched as one (dependencies resolved on the device,
        // without per-launch stream and event work); not while profiling.  On
        // the legacy default stream, which cannot be captured, the capture and
        // the graph use the library's own stream, entered and left through
        // events so that the call stays ordered on the caller's stream.
        if (pipe && net->has_syn && !net->profiling) {
            const cudaStream_t user = net->st;
            if (!user) {
                HH_CUDA(cudaEventRecord(net->ev_enter, user));
                HH_CUDA(cudaStreamWaitEvent(net->st_own, net->ev_enter, 0));
                net->st = net->st_own;
            }
            // everything the captured schedule depends on: repeated calls
            // with the same arguments from the same state (a reset, then
            // the same run) skip the capture and the executable update
            std::string sig;
            auto put = [&sig](const void* x, size_t n) { sig.append(static_cast<const char*>(x), n); };
            const int64_t wmod = net->window_index % hh::kListSlots;
            const void* kw = spec ? (const void*)net->jit.window : nullptr;
            const cudaStream_t cs = net->st;
            put(&n_steps, sizeof n_steps);
            put(&net->t, sizeof net->t);
            put(&wmod, sizeof wmod);
            put(&p, sizeof p);
            put(&R, sizeof R);
            put(&rp, sizeof rp);
            put(&I_steps, sizeof I_steps);
            put(&kw, sizeof kw);
            put(&cs, sizeof cs);
            put(&net->precision, sizeof net->precision);
            put(&net->models, sizeof net->models);
            put(&net->shape_block, sizeof net->shape_block);
            put(&net->shape_route, sizeof net->shape_route);
            cudaError_t e = cudaSuccess;
            if (!net->relaunch_graph(sig, net->st, &e)) {
                e = cudaStreamBeginCapture(net->st, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    e = enqueue();
                    cudaGraph_t g = nullptr;
                    const cudaError_t e_end = cudaStreamEndCapture(net->st, &g);
                    if (e == cudaSuccess)
                        e = e_end;
                    if (e == cudaSuccess)
                        e = net->launch_graph(g, net->st, sig);
                    if (g)
                        cudaGraphDestroy(g);
                }
            } else {
                net->window_index += (n_steps + Wmax - 1) / Wmax;
            }
            if (!user) {
                if (e == cudaSuccess)
                    e = cudaEventRecord(net->ev_leave, net->st);
                if (e == cudaSuccess)
                    e = cudaStreamWaitEvent(user, net->ev_leave, 0);
                net->st = user;
            }
            HH_CUDA(e);
        } else {
            HH_CUDA(enqueue());
        }
    }
    net->t += n_steps;
    return HH_OK;
}

hh_status hh_measure_peaks(hh_peaks* out, void* stream)
{
    if (!out)
        return fail(HH_EINVAL, "out is NULL");
    *out = hh_peaks{};
    HH_CUDA(hh::measure_peaks(&out->ffma_per_s, &out->ex2_per_s, &out->rcp_per_s, (cudaStream_t)stream));
    return HH_OK;
}

hh_status hh_reset(hh_net* net, const float* V0)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    cudaStream_t st = net->st;
    if (V0)
        HH_CUDA(cudaMemcpyAsync(net->V0, V0, net->N * sizeof(float), cudaMemcpyDefault, st));
    hh::NeuronParams p = net->neuron_params();
    HH_CUDA(hh::launch_init_state(net->models, p, net->V0, -1, net->precision, st));
    HH_CUDA(cudaMemsetAsync(net->gE, 0, net->N * sizeof(float), st));
    HH_CUDA(cudaMemsetAsync(net->gI, 0, net->N * sizeof(float), st));
    HH_CUDA(cudaMemsetAsync(net->status, 0, sizeof(int32_t), st));
    if (net->ring) {
        HH_CUDA(cudaMemsetAsync(net->ring, 0, (size_t)net->R * net->N * 2 * sizeof(int64_t), st));
        HH_CUDA(cudaMemsetAsync(net->list.counter, 0, hh::kListSlots * sizeof(int32_t), st));
    }
    net->t = 0;
    net->window_index = 0;
    return HH_OK;
}

namespace {

// The state image: a 256-byte header, then the arrays in the order of
// state_arrays(), each at a 256-byte boundary.
constexpr uint64_t kStateMagic = 0x3145544154534848ull;  // "HHSTATE1"
struct StateHeader {
    uint64_t magic;
    uint64_t bytes;
    int64_t N, t, window_index;
    int32_t R, max_gates, precision, has_lo, has_ring, has_syn;
    uint8_t pad[256 - 8 * 5 - 4 * 6];
};
static_assert(sizeof(StateHeader) == 256, "state header");

struct StateArray {
    void* dev;
    size_t bytes;
};

std::vector<StateArray> state_arrays(const hh_net* n)
{
    const size_t N = (size_t)n->N, G = (size_t)hh::kMaxGates;
    std::vector<StateArray> a = {{n->V, N * 4}, {n->Ca, N * 4}, {n->gE, N * 4}, {n->gI, N * 4},
                                 {n->P, G * N * 4}, {n->status, 4}};
    if (n->Vlo) {
        a.push_back({n->Vlo, N * 4});
        a.push_back({n->Plo, G * N * 4});
    }
    if (n->ring) {
        a.push_back({n->ring, (size_t)n->R * N * 2 * sizeof(int64_t)});
        a.push_back({n->list.counter, hh::kListSlots * sizeof(int32_t)});
    }
    return a;
}

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t state_bytes(const hh_net* n)
{
    size_t b = sizeof(StateHeader);
    for (const StateArray& x : state_arrays(n))
        b += round256(x.bytes);
    return b;
}

StateHeader state_header(const hh_net* n)
{
    StateHeader h{};
    h.magic = kStateMagic;
    h.bytes = state_bytes(n);
    h.N = n->N;
    h.t = n->t;
    h.window_index = n->window_index;
    h.R = n->ring ? n->R : 0;
    h.max_gates = hh::kMaxGates;
    h.precision = n->precision;
    h.has_lo = n->Vlo != nullptr;
    h.has_ring = n->ring != nullptr;
    h.has_syn = n->has_syn;
    return h;
}

}  // namespace

hh_status hh_state_size(const hh_net* net, size_t* bytes)
{
    if (!net || !bytes)
        return fail(HH_EINVAL, "net and bytes must not be NULL");
    *bytes = state_bytes(net);
    return HH_OK;
}

hh_status hh_save_state(hh_net* net, void* dst, size_t cap)
{
    if (!net || !dst)
        return fail(HH_EINVAL, "net and dst must not be NULL");
    const StateHeader h = state_header(net);
    if (cap < h.bytes)
        return fail(HH_EINVAL, "the state image needs %zu bytes, cap is %zu", (size_t)h.bytes, cap);
    uint8_t* out = static_cast<uint8_t*>(dst);
    HH_CUDA(cudaMemcpyAsync(out, &h, sizeof h, cudaMemcpyDefault, net->st));
    size_t off = sizeof h;
    for (const StateArray& x : state_arrays(net)) {
        HH_CUDA(cudaMemcpyAsync(out + off, x.dev, x.bytes, cudaMemcpyDefault, net->st));
        off += round256(x.bytes);
    }
    // h lives on this stack frame: the copies complete before returning
    HH_CUDA(cudaStreamSynchronize(net->st));
    return HH_OK;
}

hh_status hh_load_state(hh_net* net, const void* src, size_t n)
{
    if (!net || !src)
        return fail(HH_EINVAL, "net and src must not be NULL");
    if (n < sizeof(StateHeader))
        return fail(HH_EINVAL, "a state image has at least %zu bytes", sizeof(StateHeader));
    StateHeader h{};
    HH_CUDA(cudaMemcpyAsync(&h, src, sizeof h, cudaMemcpyDefault, net->st));
    HH_CUDA(cudaStreamSynchronize(net->st));
    const StateHeader mine = state_header(net);
    if (h.magic != kStateMagic)
        return fail(HH_EINVAL, "not a state image of this library");
    if (h.bytes > n)
        return fail(HH_EINVAL, "the image has %zu bytes, %zu given", (size_t)h.bytes, n);
    if (h.N != mine.N || h.R != mine.R || h.max_gates != mine.max_gates || h.precision != mine.precision ||
        h.has_lo != mine.has_lo || h.has_ring != mine.has_ring || h.has_syn != mine.has_syn ||
        h.bytes != mine.bytes)
        return fail(HH_EINVAL,
                    "the image does not fit this network: N %lld vs %lld, delay slots %d vs %d, precision %d vs "
                    "%d, synapses %d vs %d",
                    (long long)h.N, (long long)mine.N, h.R, mine.R, h.precision, mine.precision, h.has_syn,
                    mine.has_syn);
    if (h.t < 0 || h.t > (int64_t)INT32_MAX || h.window_index < 0)
        return fail(HH_EINVAL, "the image's step index is out of range");
    const uint8_t* in = static_cast<const uint8_t*>(src);
    size_t off = sizeof h;
    for (const StateArray& x : state_arrays(net)) {
        HH_CUDA(cudaMemcpyAsync(x.dev, in + off, x.bytes, cudaMemcpyDefault, net->st));
        off += round256(x.bytes);
    }
    net->t = h.t;
    net->window_index = h.window_index;
    return HH_OK;
}

hh_status hh_set_launch_shape(hh_net* net, int32_t neuron_block, int32_t route_blocks)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (neuron_block != 0 && neuron_block != 32 && neuron_block != 64 && neuron_block != 128)
        return fail(HH_EINVAL, "neuron_block must be 0, 32, 64 or 128");
    if (route_blocks < 0 || route_blocks > 4096)
        return fail(HH_EINVAL, "route_blocks must be in 0 .. 4096");
    if (net->morph.n_dendrites > 0 && neuron_block != 0 && neuron_block < 32)
        return fail(HH_EINVAL, "multi-compartment cells need whole warps");
    net->shape_block = neuron_block;
    net->shape_route = route_blocks;
    return HH_OK;
}

hh_status hh_autotune(hh_net* net, int32_t trial_steps, hh_tune_report* rep)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (trial_steps < 1 || trial_steps > 1000000)
        return fail(HH_EINVAL, "trial_steps must be in 1 .. 1e6");
    if (net->kernels != HH_KERNELS_SPECIALISED || !(net->has_syn || net->has_bg) || net->sur_on)
        return fail(HH_EUNSUPPORTED,
                    "autotuning covers the specialised window schedule (a network with synapses or background)");
    if (net->t + 2 * (int64_t)trial_steps > (int64_t)INT32_MAX)
        return fail(HH_EINVAL, "step index would exceed 2^31-1");
    const int32_t blocks[] = {32, 64, 128};
    const int32_t routes[] = {152, 304, 608};
    static_assert(1 + 3 * 3 <= HH_TUNE_MAX, "tune report size");
    const size_t bytes = state_bytes(net);
    void* saved = nullptr;
    if (cudaMalloc(&saved, bytes) != cudaSuccess)
        return fail(HH_ENOMEM, "autotune: %zu bytes for the saved state", bytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    hh_tune_report r{};
    hh_status s = HH_OK;
    const int32_t old_block = net->shape_block, old_route = net->shape_route;
    auto run = [&](float* ms) -> hh_status {
        hh_status q = hh_load_state(net, saved, bytes);
        if (q != HH_OK)
            return q;
        if (ms && cudaEventRecord(e0, net->st) != cudaSuccess)
            return fail(HH_ECUDA, "autotune: event record failed");
        if ((q = hh_step_n(net, trial_steps, nullptr, nullptr)) != HH_OK)
            return q;
        if (ms) {
            if (cudaEventRecord(e1, net->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
                return fail(HH_ECUDA, "autotune: timing failed");
        }
        return HH_OK;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        s = fail(HH_ECUDA, "autotune: event creation failed");
    if (s == HH_OK)
        s = hh_save_state(net, saved, bytes);
    // candidate 0 is the library's default shape (0, 0); another one is
    // installed only when the median of its three timed runs beats the
    // default's by at least 3 %, so that timing noise between near-equal
    // shapes does not move the choice
    std::vector<std::pair<int32_t, int32_t>> cand = {{0, 0}};
    for (int32_t b : blocks)
        for (int32_t g : routes)
            if (net->has_syn || g == routes[1])  // no routing launches: the grid does not matter
                cand.push_back({b, g});
    for (const auto& c : cand) {
        if (s != HH_OK)
            break;
        if ((s = hh_set_launch_shape(net, c.first, c.second)) != HH_OK || (s = run(nullptr)) != HH_OK)
            break;
        float t[3] = {0.0f, 0.0f, 0.0f};
        for (int k = 0; k < 3 && s == HH_OK; ++k)
            s = run(&t[k]);
        if (s != HH_OK)
            break;
        std::sort(t, t + 3);
        r.neuron_block[r.n] = c.first;
        r.route_blocks[r.n] = c.second;
        r.ms[r.n] = t[1];  // median of three timed runs
        ++r.n;
    }
    r.best = -1;
    if (s == HH_OK && r.n > 0) {
        int32_t k = 0;
        for (int32_t j = 1; j < r.n; ++j)
            if (r.ms[j] < r.ms[k])
                k = j;
        r.best = r.ms[k] <= 0.97f * r.ms[0] ? k : 0;
    }
    if (s == HH_OK && r.best >= 0) {
        s = hh_set_launch_shape(net, r.neuron_block[r.best], r.route_blocks[r.best]);
    } else {
        net->shape_block = old_block;
        net->shape_route = old_route;
    }
    // the network leaves with the state it came in with
    const hh_status s_restore = hh_load_state(net, saved, bytes);
    if (s == HH_OK)
        s = s_restore;
    if (cudaStreamSynchronize(net->st) != cudaSuccess && s == HH_OK)
        s = fail(HH_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(saved);
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (s == HH_OK && rep)
        *rep = r;
    return s;
}

hh_status hh_route_spikes(hh_net* net, const int32_t* spk_step, const int32_t* spk_idx, int64_t n_spk,
                          int32_t n_window, int64_t* sum_E, int64_t* sum_I)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (!net->has_syn)
        return fail(HH_ESTATE, "the network has no synapses");
    if (n_spk < 0 || n_window < 0)
        return fail(HH_EINVAL, "n_spk and n_window must be >= 0");
    if (n_spk > 0 && (!spk_step || !spk_idx))
        return fail(HH_EINVAL, "spike arrays are NULL");
    if (n_window > 0 && (!sum_E || !sum_I))
        return fail(HH_EINVAL, "sum_E and sum_I are required");
    if (n_spk == 0 || n_window == 0)
        return HH_OK;
    hh::RouteParams rp = net->route_params();
    rp.open_loop = 1;
    rp.n_window = n_window;
    rp.ringE = sum_E;
    rp.ringI = sum_I;
    rp.stride = 1;
    HH_CUDA(hh::launch_route_list(rp, spk_step, spk_idx, n_spk, net->st));
    return HH_OK;
}

hh_status hh_readout(hh_net* net, int32_t what, void* dst, size_t cap, size_t* n_bytes)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (n_bytes)
        *n_bytes = 0;
    HH_CUDA(cudaStreamSynchronize(net->st));
    const size_t N = (size_t)net->N;
    size_t need = 0;
    switch (what) {
    case HH_READ_V: need = N * sizeof(float); break;
    case HH_READ_GATES: need = N * hh::kMaxGates * sizeof(float); break;
    case HH_READ_CA: need = N * sizeof(float); break;
    case HH_READ_G_SYN: need = 2 * N * sizeof(float); break;
    case HH_READ_STATUS: need = sizeof(int32_t); break;
    case HH_READ_TIME: need = sizeof(int64_t); break;
    case HH_READ_N_OUT:
        if (!net->has_syn)
            return fail(HH_ESTATE, "the network has no synapses");
        need = (N + 1) * sizeof(int64_t);
        break;
    case HH_READ_PROFILE: need = sizeof(net->ktime); break;
    case HH_READ_SURROGATE:
        if (!net->sur)
            return fail(HH_ESTATE, "no surrogate trained");
        need = 2 * sizeof(uint64_t);
        break;
    case HH_READ_POLY: need = sizeof(net->poly_info); break;
    default: return fail(HH_EINVAL, "unknown readout %d", what);
    }
    if (!dst)
        return fail(HH_EINVAL, "dst is NULL");
    if (cap < need)
        return fail(HH_EOVERFLOW, "readout %d needs %zu bytes, got %zu", what, need, cap);
    switch (what) {
    case HH_READ_V: HH_CUDA(cudaMemcpy(dst, net->V, need, cudaMemcpyDefault)); break;
    case HH_READ_GATES: HH_CUDA(cudaMemcpy(dst, net->P, need, cudaMemcpyDefault)); break;
    case HH_READ_CA: HH_CUDA(cudaMemcpy(dst, net->Ca, need, cudaMemcpyDefault)); break;
    case HH_READ_G_SYN:
        HH_CUDA(cudaMemcpy(dst, net->gE, N * sizeof(float), cudaMemcpyDefault));
        HH_CUDA(cudaMemcpy((char*)dst + N * sizeof(float), net->gI, N * sizeof(float), cudaMemcpyDefault));
        break;
    case HH_READ_STATUS: HH_CUDA(cudaMemcpy(dst, net->status, need, cudaMemcpyDefault)); break;
    case HH_READ_TIME: {
        int64_t t = net->t;
        HH_CUDA(cudaMemcpy(dst, &t, need, cudaMemcpyDefault));
        break;
    }
    case HH_READ_N_OUT: HH_CUDA(cudaMemcpy(dst, net->out_ptr, need, cudaMemcpyDefault)); break;
    case HH_READ_SURROGATE: {
        unsigned long long s2[2];
        int32_t err = 0;
        HH_CUDA(hh::surrogate_stats(net->sur, s2, &err));
        if (err)
            return fail(HH_ETIMEOUT, "a bounded wait in the surrogate kernel expired (code %d)", err);
        HH_CUDA(cudaMemcpy(dst, s2, need, cudaMemcpyDefault));
        break;
    }
    case HH_READ_PROFILE:
        HH_CUDA(net->harvest());
        HH_CUDA(cudaMemcpy(dst, net->ktime, need, cudaMemcpyDefault));
        break;
    case HH_READ_POLY: HH_CUDA(cudaMemcpy(dst, net->poly_info, need, cudaMemcpyDefault)); break;
    }
    if (n_bytes)
        *n_bytes = need;
    return HH_OK;
}

hh_status hh_gemm_bf16(const void* A, int32_t lda, const void* Bt, int32_t ldb, float* C, int32_t M,
                       int32_t N, int32_t K, int32_t splits, int32_t* status, void* stream)
{
    if (!A || !Bt || !C || !status)
        return fail(HH_EINVAL, "A, Bt, C and status must not be NULL");
    hh::GemmArgs g{};
    g.A = A;
    g.a_rows = M;
    g.lda = lda;
    g.Bt = Bt;
    g.b_rows = N;
    g.ldb = ldb;
    g.C = C;
    g.M = M;
    g.N = N;
    g.K = K;
    g.splits = splits;
    if (const char* why = hh::gemm_check(g))
        return fail(HH_EINVAL, "%s", why);
    HH_CUDA(hh::launch_gemm_bf16(g, status, (cudaStream_t)stream));
    return HH_OK;
}

hh_status hh_surrogate_train(hh_net* net, const hh_surrogate_desc* d, hh_surrogate_report* rep)
{
    if (!net || !d)
        return fail(HH_EINVAL, "net and descriptor must not be NULL");
    if (net->has_syn || net->has_bg)
        return fail(HH_EUNSUPPORTED, "the surrogate is for networks of independent neurons");
    if (net->model_id)
        return fail(HH_EUNSUPPORTED, "the surrogate supports a single model (model_id must be NULL)");
    if (net->kernels != HH_KERNELS_SPECIALISED)
        return fail(HH_EUNSUPPORTED, "the surrogate needs HH_KERNELS_SPECIALISED");
    if (net->precision != HH_PREC_FAST && net->precision != HH_PREC_ACCURATE)
        return fail(HH_EUNSUPPORTED, "the surrogate supports HH_PREC_FAST and HH_PREC_ACCURATE");
    if (net->sin_amp || net->morph.n_dendrites > 0)
        return fail(HH_EUNSUPPORTED, "the surrogate supports point neurons without a sinusoidal drive");
    if (!net->installed[0])
        return fail(HH_ESTATE, "model 0 is not installed");
    if (!net->jit_ready) {
        std::string err;
        if (!hh::jit_get(net->models, net->installed, net->precision, net->jit_flags(), &net->jit, &err))
            return fail(HH_ECUDA, "%s", err.c_str());
        net->jit_ready = true;
    }
    hh::Surrogate* s = nullptr;
    hh_status rc = hh::surrogate_train(net->models, net->precision, net->dt, net->N, d, net->st, &s, rep);
    if (rc != HH_OK)
        return rc;
    if (net->sur)
        hh::surrogate_free(net->sur);
    net->sur = s;
    return HH_OK;
}

hh_status hh_surrogate_enable(hh_net* net, int32_t enable)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (enable && !net->sur)
        return fail(HH_ESTATE, "no surrogate trained");
    net->sur_on = enable != 0;
    if (net->sur)
        HH_CUDA(hh::surrogate_reset_stats(net->sur, net->st));
    return HH_OK;
}

hh_status hh_set_route_pull(hh_net* net, int64_t min_spikes)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (min_spikes < 0) {
        net->pull_min = -1;
        return HH_OK;
    }
    if (!net->has_syn || net->in_ptr_host.empty())
        return fail(HH_EUNSUPPORTED, "pull routing needs synapses, at most %lld neurons and windows of at most %d "
                    "steps", (long long)hh::kPullMaxN, hh::kPullMaxW);
    if (!net->in_rec) {
        // the in-CSR from the out-CSR (k_fill_out run on the out-CSR
        // transposes it back; the order inside a row is free), then its
        // records; the last-spike tables
        const int64_t N = net->N, S = net->S;
        const cudaStream_t st = net->st;
        const size_t Np = (size_t)hh::pull_stride(N);
        int32_t* col = nullptr;
        float* w = nullptr;
        unsigned long long* cursor = nullptr;
        cudaError_t e;
        hh_status rc = HH_OK;
        if ((e = net->alloc(&net->in_ptr, N + 1)) != cudaSuccess ||
            (e = net->alloc(&net->in_rec, S + 8)) != cudaSuccess ||
            (e = net->alloc(&net->last_spk, hh::kListSlots * Np)) != cudaSuccess ||
            (e = cudaMalloc(&col, S * sizeof(int32_t))) != cudaSuccess ||
            (e = cudaMalloc(&w, S * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&cursor, N * sizeof(unsigned long long))) != cudaSuccess)
            rc = fail(HH_ENOMEM, "allocating the in-CSR of pull routing: %s", cudaGetErrorString(e));
        else if ((e = copy_in(net->in_ptr, net->in_ptr_host.data(), (size_t)N + 1, st)) != cudaSuccess ||
                 (e = copy_in(reinterpret_cast<int64_t*>(cursor), net->in_ptr_host.data(), (size_t)N, st)) !=
                     cudaSuccess ||
                 (e = hh::launch_fill_out(net->out_ptr, net->out_post, net->out_w, N, cursor, col, w, st)) !=
                     cudaSuccess ||
                 (e = hh::launch_pull_records(col, w, S, net->in_rec, st)) != cudaSuccess ||
                 (e = cudaMemsetAsync(net->in_rec + S, 0, 8 * sizeof(uint2), st)) != cudaSuccess ||
                 (e = cudaMemsetAsync(net->last_spk, hh::kPullNone, hh::kListSlots * Np, st)) != cudaSuccess ||
                 (e = hh::route_pull_prepare()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
            rc = fail(HH_ECUDA, "building the in-CSR of pull routing: %s", cudaGetErrorString(e));
        cudaStreamSynchronize(st);
        for (void* q : {(void*)col, (void*)w, (void*)cursor})
            if (q)
                cudaFree(q);
        if (rc != HH_OK) {
            net->free_tracked(net->in_ptr);
            net->free_tracked(net->in_rec);
            net->free_tracked(net->last_spk);
            net->in_ptr = nullptr;
            net->in_rec = nullptr;
            net->last_spk = nullptr;
            return rc;
        }
    }
    net->pull_min = min_spikes;
    return HH_OK;
}

hh_status hh_profile(hh_net* net, int32_t enable)
{
    if (!net)
        return fail(HH_EINVAL, "net is NULL");
    if (enable) {
        HH_CUDA(cudaStreamSynchronize(net->st));
        HH_CUDA(net->harvest());
        for (auto& k : net->ktime)
            k = hh_kernel_time{0, 0.0};
    }
    net->profiling = enable != 0;
    return HH_OK;
}

void hh_destroy(hh_net* net)
{
    if (!net)
        return;
    net->release();
    delete net;
}

const char* hh_last_error(void) { return g_err.c_str(); }

int32_t hh_version(void) { return 0x000100; }

hh_status hh_poly_fit(const hh_model_desc* m, double dt_ms, float* info, int32_t* n_intervals, float* coeffs,
                      int64_t cap_floats, int64_t* n_floats)
{
    if (!m || !info)
        return fail(HH_EINVAL, "model and info must not be NULL");
    if (!(dt_ms > 0.0))
        return fail(HH_EINVAL, "dt_ms must be > 0");
    hh::DevModel dm{};
    hh_status s = prep_model(m, dt_ms, &dm);
    if (s != HH_OK)
        return s;
    PolyTable T;
    if ((s = poly_fit(m, dt_ms, &T)) != HH_OK)
        return s;
    info[0] = T.h;
    info[1] = T.v_lo;
    info[2] = T.err;
    if (n_intervals)
        *n_intervals = T.n;
    if (n_floats)
        *n_floats = (int64_t)T.c.size();
    if (coeffs) {
        if (cap_floats < (int64_t)T.c.size())
            return fail(HH_EOVERFLOW, "the table needs %zu floats", T.c.size());
        std::memcpy(coeffs, T.c.data(), T.c.size() * sizeof(float));
    }
    return HH_OK;
}

hh_status hh_set_wait_limits(int64_t progress_ns, int64_t mbarrier_polls)
{
    g_wait_ns.store(progress_ns < 0 ? hh::kWaitLimitNs : (unsigned long long)progress_ns);
    g_wait_polls.store(mbarrier_polls < 0 ? hh::kWaitLimitPolls : (long long)mbarrier_polls);
    return HH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free stepping of independent neurons.  The neuron kernel's only
// scratch (the neuron -> V-trace-slot map, and one word that receives the
// status bits when the caller passes no status pointer) lives in this
// file-scope array; host code reaches it through the device address
// cudaGetSymbolAddress returns for each device, looked up once per device
// and cached.
// ---------------------------------------------------------------------------
static __device__ __align__(256) int32_t g_noalloc_trace_slot[HH_NOALLOC_MAX_NEURONS + 64];

namespace {

std::mutex g_noalloc_mu;
int32_t* g_noalloc_addr[64] = {};

hh_status noalloc_scratch(int32_t** out)
{
    int dev = 0;
    HH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64)
        return fail(HH_EUNSUPPORTED, "device index %d outside 0..63", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_trace_slot);
        if (e != cudaSuccess || !p)
            return fail(HH_ECUDA, "cudaGetSymbolAddress of the scratch array failed on device %d: %s",
                        dev, cudaGetErrorString(e));
        g_noalloc_addr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_noalloc_addr[dev];
    return HH_OK;
}

}  // namespace

extern "C" hh_status hh_step_neurons_noalloc(const hh_model_desc* m, const hh_neurons_noalloc* s,
                                             int64_t t0, int32_t n_steps, const float* I_steps,
                                             const hh_record* rec)
{
    if (!m || !s)
        return fail(HH_EINVAL, "model and state descriptor must not be NULL");
    const int64_t N = s->n_neurons;
    if (N < 1 || N > HH_NOALLOC_MAX_NEURONS)
        return fail(HH_EINVAL, "n_neurons %lld outside 1..%d (the static scratch holds %d neurons)",
                    (long long)N, HH_NOALLOC_MAX_NEURONS, HH_NOALLOC_MAX_NEURONS);
    if (n_steps < 0 || t0 < 0 || t0 + n_steps > (int64_t)INT32_MAX)
        return fail(HH_EINVAL, "n_steps/t0 out of range");
    if (!(s->dt_ms > 0.0) || !std::isfinite(s->dt_ms) || !finite_f(s->v_threshold))
        return fail(HH_EINVAL, "dt_ms must be > 0 and v_threshold finite");
    if (s->v_update != HH_V_EXP_EULER && s->v_update != HH_V_FWD_EULER)
        return fail(HH_EINVAL, "unknown v_update %d", s->v_update);
    if (s->precision < HH_PREC_FAST || s->precision > HH_PREC_COMPENSATED)
        return fail(HH_EINVAL, "unknown precision %d", s->precision);
    if (!s->V || !s->gates || !s->Ca)
        return fail(HH_EINVAL, "V, gates and Ca are required");
    if (s->precision == HH_PREC_COMPENSATED && (!s->V_lo || !s->gates_lo))
        return fail(HH_EINVAL, "HH_PREC_COMPENSATED needs V_lo and gates_lo");
    hh::RecordParams R{};
    if (rec) {
        if (rec->n_trace < 0 || (rec->V_trace && rec->n_trace == 0))
            return fail(HH_EINVAL, "n_trace must be > 0 when V_trace is given");
        if (rec->spikes && !rec->n_spikes)
            return fail(HH_EINVAL, "spikes needs an n_spikes counter");
        if (rec->spike_cap < 0)
            return fail(HH_EINVAL, "spike_cap < 0");
        if (!rec->trace_idx && rec->n_trace > N)
            return fail(HH_EINVAL, "n_trace > N without trace_idx");
        R.V_trace = rec->V_trace;
        R.n_trace = rec->V_trace ? rec->n_trace : 0;
        R.spikes = rec->spikes;
        R.spike_cap = rec->spikes ? rec->spike_cap : 0;
        R.n_spikes = reinterpret_cast<unsigned long long*>(rec->n_spikes);
        R.counts = rec->counts;
    }
    hh::DevModels models{};
    hh_status st = prep_model(m, s->dt_ms, &models.m[0]);
    if (st != HH_OK)
        return st;
    models.n = 1;
    models.max_gates = models.m[0].n_gates > 0 ? models.m[0].n_gates : 1;
    int32_t* scratch = nullptr;
    if ((st = noalloc_scratch(&scratch)) != HH_OK)
        return st;
    cudaStream_t stream = (cudaStream_t)s->stream;

    hh::NeuronParams p{};
    p.N = N;
    p.dt = (float)s->dt_ms;
    p.theta = s->v_threshold;
    p.v_update = s->v_update;
    p.V = s->V;
    p.Vlo = s->V_lo;
    p.P = s->gates;
    p.Plo = s->gates_lo;
    p.Ca = s->Ca;
    p.gbar = s->gbar;
    p.I_const = s->I_const;
    p.status = s->status ? s->status : scratch + HH_NOALLOC_MAX_NEURONS;
    p.R = 1;
    if (s->init_state)
        HH_CUDA(hh::launch_init_state(models, p, nullptr, -1, s->precision, stream));
    if (n_steps == 0)
        return HH_OK;
    if (R.V_trace && rec->trace_idx) {
        HH_CUDA(cudaMemsetAsync(scratch, 0xff, (size_t)N * sizeof(int32_t), stream));
        HH_CUDA(hh::launch_trace_slots(rec->trace_idx, rec->n_trace, N, scratch, stream));
        p.trace_slot = scratch;
    }
    HH_CUDA(hh::launch_independent(models, p, s->precision, t0, n_steps, I_steps, R, stream));
    return HH_OK;
}
