// Neuron kernels specialised per model table, compiled at run time with
// NVRTC for sm_103a (Methods, "Flexibility and extensibility": users define
// the channel dynamics, the platform supplies the fused, parallel update).
//
// The generated translation unit is: the ABI constants it needs, the shared
// device code (hh_device.cuh, embedded verbatim at build time), one function
// per installed model that returns its DevModel built from literal
// constants, and two extern "C" kernels that run the same bodies as the
// table interpreter.  Because the model is a compile-time constant inside
// the kernel, the rate forms, gate counts, exponents and parameters fold into
// the instruction stream: no constant-bank loads, no branches on forms.
// Compiled modules are cached for the life of the process, keyed by source.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvrtc.h>

#include "hh_internal.h"
#include "hh_layer_device.cuh"

namespace {

const char kDeviceSrc[] =
#include "hh_device_src.inc"
    ;
const char kLayerDeviceSrc[] =
#include "hh_layer_device_src.inc"
    ;

std::string flt(float x)
{
    char b[64];
    snprintf(b, sizeof(b), "%af", (double)x);
    return b;
}

void emit_fn(std::string& s, const char* path, const hh::DevFn& f)
{
    char b[96];
    snprintf(b, sizeof(b), "    %s.form = %d;\n", path, f.form);
    s += b;
    const struct { const char* n; float v; } fields[] = {
        {"a", f.a}, {"c", f.c}, {"vh", f.vh}, {"k", f.k}, {"ik", f.ik}, {"s", f.s}, {"b", f.b},
        {"vh2", f.vh2}, {"ik2", f.ik2}, {"s2", f.s2}, {"b2", f.b2}, {"ia", f.ia}, {"irate", f.irate},
        {"n0", f.n0}, {"n1", f.n1}, {"n2", f.n2}, {"n4", f.n4}};
    for (const auto& fl : fields)
        s += std::string("    ") + path + "." + fl.n + " = " + flt(fl.v) + ";\n";
}

std::string model_function(const hh::DevModel& m, int idx)
{
    std::string s;
    char b[160];
    snprintf(b, sizeof(b), "__device__ __forceinline__ DevModel jit_model_%d()\n{\n    DevModel m{};\n", idx);
    s += b;
    auto F = [&](const char* n, float v) { s += std::string("    m.") + n + " = " + flt(v) + ";\n"; };
    auto I = [&](const char* n, int v) {
        snprintf(b, sizeof(b), "    m.%s = %d;\n", n, v);
        s += b;
    };
    F("C_m", m.C_m);
    F("inv_C", m.inv_C);
    I("n_ch", m.n_ch);
    I("n_gates", m.n_gates);
    I("ca_ch", m.ca_ch);
    I("poly_n", m.poly_n);
    I("poly_base", m.poly_base);
    I("poly_stride", m.poly_stride);
    F("poly_vlo", m.poly_vlo);
    F("poly_ih", m.poly_ih);
    F("ca_tau", m.ca_tau);
    F("ca_k", m.ca_k);
    F("ca_rest", m.ca_rest);
    F("ca_decay", m.ca_decay);
    for (int c = 0; c < hh::kMaxChannels; ++c) {
        snprintf(b, sizeof(b), "    m.E[%d] = %s; m.gbar[%d] = %s; m.ch_first[%d] = %d; m.ch_ng[%d] = %d;\n",
                 c, flt(m.E[c]).c_str(), c, flt(m.gbar[c]).c_str(), c, m.ch_first[c], c, m.ch_ng[c]);
        s += b;
    }
    for (int q = 0; q < hh::kMaxGates; ++q) {
        snprintf(b, sizeof(b),
                 "    m.gate_ch[%d] = %d; m.gate_last[%d] = %d; m.gate_E[%d] = %s; m.gate_ca[%d] = %d;\n",
                 q, m.gate_ch[q], q, m.gate_last[q], q, flt(m.gate_E[q]).c_str(), q, m.gate_ca[q]);
        s += b;
        snprintf(b, sizeof(b), "    m.g[%d].kind = %d; m.g[%d].power = %d;\n", q, m.g[q].kind, q,
                 m.g[q].power);
        s += b;
        char p1[32], p2[32];
        snprintf(p1, sizeof(p1), "m.g[%d].f1", q);
        snprintf(p2, sizeof(p2), "m.g[%d].f2", q);
        emit_fn(s, p1, m.g[q].f1);
        emit_fn(s, p2, m.g[q].f2);
    }
    s += "    return m;\n}\n\n";
    return s;
}

std::string abi_constants()
{
    std::string s;
    char b[96];
    const struct { const char* n; int v; } c[] = {
        {"HH_MAX_CHANNELS", HH_MAX_CHANNELS}, {"HH_MAX_GATES_PER_CHANNEL", HH_MAX_GATES_PER_CHANNEL},
        {"HH_MAX_GATES", HH_MAX_GATES}, {"HH_MAX_MODELS", HH_MAX_MODELS},
        {"HH_FN_CONST", HH_FN_CONST}, {"HH_FN_EXP", HH_FN_EXP}, {"HH_FN_SIGMOID", HH_FN_SIGMOID},
        {"HH_FN_LINOID", HH_FN_LINOID}, {"HH_FN_BELL", HH_FN_BELL}, {"HH_GATE_AB", HH_GATE_AB},
        {"HH_GATE_INFTAU", HH_GATE_INFTAU}, {"HH_GATE_CA", HH_GATE_CA},
        {"HH_PREC_FAST", HH_PREC_FAST}, {"HH_PREC_ACCURATE", HH_PREC_ACCURATE},
        {"HH_PREC_COMPENSATED", HH_PREC_COMPENSATED}, {"HH_PREC_POLY", HH_PREC_POLY},
        {"HH_V_EXP_EULER", HH_V_EXP_EULER},
        {"HH_V_FWD_EULER", HH_V_FWD_EULER}, {"HH_STATUS_SPIKE_OVERFLOW", HH_STATUS_SPIKE_OVERFLOW},
        {"HH_STATUS_NONFINITE", HH_STATUS_NONFINITE}, {"HH_STATUS_BARRIER_TIMEOUT", HH_STATUS_BARRIER_TIMEOUT}};
    for (const auto& x : c) {
        snprintf(b, sizeof(b), "#define %s %d\n", x.n, x.v);
        s += b;
    }
    s += "struct hh_spike { int step; int neuron; float frac; };\n";
    return s;
}

std::string generate(const hh::DevModels& M, const bool* installed, int precision, int max_gates,
                     const hh::JitFlags& f)
{
    std::string s = "// generated by libhh: neuron kernels specialised for one model set\n";
    s += abi_constants();
    s += kDeviceSrc;
    s += "\nnamespace hh {\n\n";
    int n_inst = 0, only = 0;
    for (int k = 0; k < hh::kMaxModels; ++k)
        if (installed[k]) {
            s += model_function(M.m[k], k);
            ++n_inst;
            only = k;
        }
    auto dispatch = [&](const char* call) {
        std::string d;
        char b[256];
        if (n_inst == 1) {
            snprintf(b, sizeof(b), "        const DevModel M = jit_model_%d();\n        %s;\n", only, call);
            return std::string(b);
        }
        d += "        switch (mid) {\n";
        for (int k = 0; k < hh::kMaxModels; ++k)
            if (installed[k]) {
                snprintf(b, sizeof(b), "        case %d: { const DevModel M = jit_model_%d(); %s; } break;\n", k, k,
                         call);
                d += b;
            }
        d += "        default: break;\n        }\n";
        return d;
    };
    {
        // the network's V update (exponential or explicit Euler) as a constant
        char vb[96];
        snprintf(vb, sizeof(vb), "constexpr int kJitVUpdate = %d;\n\n", f.v_update);
        s += vb;
    }
    s += "struct JitDyn {\n";
    auto tf = [](bool x) { return x ? "true" : "false"; };
    s += std::string("    static constexpr bool kDrive = ") + tf(f.drive) + ", kCable = " + tf(f.cable) +
         ", kSynCurrent = " + tf(f.syn_current) + ", kCompound = " + tf(f.compound) + ";\n";
    s += "    template <int MAXG, int PREC>\n";
    s += "    __device__ __forceinline__ void load(int mid, const NeuronParams& P, int64_t i, State<MAXG, PREC>& s) const\n    {\n";
    s += dispatch("load_conductances(M, P.gbar, P.N, i, s)");
    s += "    }\n";
    s += "    template <int MAXG, int PREC>\n";
    s += "    __device__ __forceinline__ void step(int mid, float dt, int v_update, float I, float gsE, float EE,\n"
         "                                         float gsI, float EI, State<MAXG, PREC>& s) const\n    {\n";
    s += dispatch("neuron_step<MAXG, PREC>(M, dt, kJitVUpdate, I, gsE, EE, gsI, EI, s)");
    s += "    }\n};\n\n}  // namespace hh\n\n";
    // Window steps grouped by background block (four steps unrolled) for one
    // installed model with a short step; one step per iteration otherwise,
    // where four unrolled copies of the dispatch would leave the
    // instruction cache.
    const int group = (n_inst == 1 && max_gates <= 4) ? 4 : 1;
    // With long model steps the window kernel is held to 64 registers (8
    // blocks of 128 per SM): their networks are large and throughput-bound,
    // and need the resident warps.
    const char* window_bounds = group == 4 ? "128" : "128, 8";
    char b[4096];
    snprintf(b, sizeof(b),
             "constexpr int kJitMaxG = %d;\nconstexpr int kJitPrec = %d;\nconstexpr int kJitGroup = %d;\n\n"
             "extern \"C\" __global__ void __launch_bounds__(128)\n"
             "hh_jit_independent(const __grid_constant__ hh::NeuronParams P, long long t0, int n_steps,\n"
             "                   const float* __restrict__ I_steps, const __grid_constant__ hh::RecordParams R)\n"
             "{\n    hh::independent_body<kJitMaxG, kJitPrec>(hh::JitDyn{}, P, t0, n_steps, I_steps, R);\n}\n\n"
             "extern \"C\" __global__ void __launch_bounds__(%s)\n"
             "hh_jit_window(const __grid_constant__ hh::NeuronParams P, long long t0, int W,\n"
             "              const float* __restrict__ I_steps, const __grid_constant__ hh::RecordParams R,\n"
             "              const __grid_constant__ hh::SpikeList L, int parity, int early)\n"
             "{\n    hh::window_body<kJitMaxG, kJitPrec, kJitGroup>(hh::JitDyn{}, P, t0, W, I_steps, R, L, parity, early);\n}\n\n"
             "extern \"C\" __global__ void __launch_bounds__(128)\n"
             "hh_jit_indexed(const __grid_constant__ hh::NeuronParams P, const int* __restrict__ list,\n"
             "               const int* __restrict__ n_list, long long t0, int n_steps,\n"
             "               const __grid_constant__ hh::RecordParams R)\n"
             "{\n    hh::indexed_body<kJitMaxG, kJitPrec>(hh::JitDyn{}, P, list, n_list, t0, n_steps, R);\n}\n\n"
             "extern \"C\" __global__ void __launch_bounds__(hh::kPersistThreads)\n"
             "hh_jit_persistent(const __grid_constant__ hh::NeuronParams P, const __grid_constant__ hh::RouteParams RP,\n"
             "                  long long t0, int n_steps, int W, long long w_index0, const float* __restrict__ I_steps,\n"
             "                  const __grid_constant__ hh::RecordParams R, const __grid_constant__ hh::SpikeList L,\n"
             "                  const __grid_constant__ hh::PhaseCounters pc)\n"
             "{\n    hh::persistent_body<kJitMaxG, kJitPrec, kJitGroup>(hh::JitDyn{}, P, RP, t0, n_steps, W, w_index0, I_steps, R, L, pc);\n}\n",
             max_gates, precision, group, window_bounds);
    s += b;
    return s;
}

struct Entry {
    cudaLibrary_t lib = nullptr;
    std::vector<cudaKernel_t> kernels;  // in the order of the names compiled
    std::string log;
};

std::mutex g_mu;
std::map<std::string, Entry>* g_cache = nullptr;

bool compile(const std::string& src, const std::vector<const char*>& names, Entry* e, std::string* err)
{
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "hh_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *err = "nvrtcCreateProgram failed";
        return false;
    }
    const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo",
                          "--ptxas-options=-v", "-DHH_JIT=1"};
    nvrtcResult rc = nvrtcCompileProgram(prog, (int)(sizeof(opts) / sizeof(opts[0])), opts);
    size_t log_size = 0;
    nvrtcGetProgramLogSize(prog, &log_size);
    std::string log(log_size, '\0');
    if (log_size)
        nvrtcGetProgramLog(prog, &log[0]);
    e->log = log;
    if (rc != NVRTC_SUCCESS) {
        *err = std::string("NVRTC compilation of the specialised neuron kernels failed: ") +
               nvrtcGetErrorString(rc) + "\n" + log.substr(0, 2000);
        nvrtcDestroyProgram(&prog);
        return false;
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    std::vector<char> cubin(n);
    nvrtcGetCUBIN(prog, cubin.data());
    nvrtcDestroyProgram(&prog);
    if (getenv("HH_JIT_VERBOSE"))
        fprintf(stderr, "[libhh jit] %zu-byte cubin\n%s\n", n, log.c_str());
    cudaError_t ce = cudaLibraryLoadData(&e->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    for (const char* name : names) {
        cudaKernel_t k = nullptr;
        if (ce == cudaSuccess)
            ce = cudaLibraryGetKernel(&k, e->lib, name);
        e->kernels.push_back(k);
    }
    if (ce != cudaSuccess) {
        *err = std::string("loading the specialised kernels failed: ") + cudaGetErrorString(ce);
        return false;
    }
    return true;
}

// Compile (once per distinct source, for the life of the process) and look
// up the named kernels.
bool cached_compile(const std::string& src, const std::vector<const char*>& names, const Entry** out,
                    std::string* err)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_cache)
        g_cache = new std::map<std::string, Entry>();
    auto it = g_cache->find(src);
    if (it == g_cache->end()) {
        Entry e;
        if (!compile(src, names, &e, err))
            return false;
        it = g_cache->emplace(src, e).first;
    }
    *out = &it->second;
    return true;
}

int block_for(int64_t N)
{
    if (N <= 152 * 2 * 32)
        return 32;
    if (N <= 152 * 2 * 64)
        return 64;
    return 128;
}

}  // namespace

namespace hh {

bool jit_get(const DevModels& M, const bool* installed, int precision, const JitFlags& f, JitKernels* out,
             std::string* err)
{
    int max_gates = 1;
    for (int k = 0; k < kMaxModels; ++k)
        if (installed[k] && M.m[k].n_gates > max_gates)
            max_gates = M.m[k].n_gates;
    const std::string src = generate(M, installed, precision, max_gates, f);
    if (const char* path = getenv("HH_JIT_DUMP")) {
        if (FILE* f = fopen(path, "w")) {
            fwrite(src.data(), 1, src.size(), f);
            fclose(f);
        }
    }
    const Entry* e = nullptr;
    if (!cached_compile(src, {"hh_jit_independent", "hh_jit_window", "hh_jit_indexed", "hh_jit_persistent"}, &e,
                        err))
        return false;
    out->independent = e->kernels[0];
    out->window = e->kernels[1];
    out->indexed = e->kernels[2];
    out->persistent = e->kernels[3];
    // the routing kernel co-running with the window kernel may hold shared
    // memory (pull routing); the same carveout lets their blocks share SMs
    const cudaError_t ce = cudaFuncSetAttribute((const void*)out->window,
                                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                                cudaSharedmemCarveoutMaxShared);
    if (ce != cudaSuccess) {
        *err = std::string("setting the window kernel's carveout: ") + cudaGetErrorString(ce);
        return false;
    }
    return true;
}

// The layer kernels for one model (model index 0 of M), compiled in as
// constants like the network kernels.
bool jit_get_layer(const DevModels& M, int precision, LayerKernels* out, std::string* err)
{
    std::string s = "// generated by libhh: differentiable-layer kernels specialised for one model\n";
    s += abi_constants();
    s += kDeviceSrc;
    s += kLayerDeviceSrc;
    s += "\nnamespace hh {\n\n";
    s += model_function(M.m[0], 0);
    s += "}  // namespace hh\n\n";
    char b[2048];
    snprintf(b, sizeof(b),
             "constexpr int kJitMaxG = %d;\nconstexpr int kJitPrec = %d;\n\n"
             "extern \"C\" __global__ void __launch_bounds__(128)\n"
             "hh_jit_layer_fwd(const __grid_constant__ hh::LayerParams L, int t)\n"
             "{\n    const hh::DevModel M = hh::jit_model_0();\n"
             "    hh::layer_fwd_body<kJitMaxG, kJitPrec>(M, L, t);\n}\n\n"
             "extern \"C\" __global__ void __launch_bounds__(128)\n"
             "hh_jit_layer_recompute(const __grid_constant__ hh::LayerParams L, int g)\n"
             "{\n    const hh::DevModel M = hh::jit_model_0();\n"
             "    hh::layer_recompute_body<kJitMaxG, kJitPrec>(M, L, g);\n}\n\n"
             "extern \"C\" __global__ void __launch_bounds__(128)\n"
             "hh_jit_layer_bwd(const __grid_constant__ hh::LayerParams L, int t)\n"
             "{\n    const hh::DevModel M = hh::jit_model_0();\n"
             "    hh::layer_bwd_body<kJitMaxG, kJitPrec>(M, L, t);\n}\n",
             M.m[0].n_gates > 0 ? M.m[0].n_gates : 1, precision);
    s += b;
    if (const char* path = getenv("HH_JIT_DUMP_LAYER")) {
        if (FILE* f = fopen(path, "w")) {
            fwrite(s.data(), 1, s.size(), f);
            fclose(f);
        }
    }
    const Entry* e = nullptr;
    if (!cached_compile(s, {"hh_jit_layer_fwd", "hh_jit_layer_recompute", "hh_jit_layer_bwd"}, &e, err))
        return false;
    out->fwd = e->kernels[0];
    out->recompute = e->kernels[1];
    out->bwd = e->kernels[2];
    return true;
}

cudaError_t jit_launch_layer(cudaKernel_t k, const LayerParams& L, int arg, int64_t n, size_t smem,
                             cudaStream_t st)
{
    LayerParams l = L;
    int a = arg;
    void* args[] = {&l, &a};
    return cudaLaunchKernel((const void*)k, dim3((unsigned)((n + 127) / 128)), dim3(128), args, smem, st);
}

// Dynamic shared memory of a neuron launch: the staged rate tables of
// HH_PREC_POLY (poly_smem_bytes), with the kernel's limit raised when they
// exceed the default 48 KB.
cudaError_t poly_smem(cudaKernel_t k, const NeuronParams& P, size_t* bytes)
{
    *bytes = poly_smem_bytes(P.poly_rows);
    if (*bytes > 48 * 1024)
        return cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes);
    return cudaSuccess;
}

cudaError_t jit_launch_independent(const JitKernels& K, const NeuronParams& P, int64_t t0,
                                   int32_t n_steps, const float* I_steps, const RecordParams& R,
                                   cudaStream_t st)
{
    const int bs = block_for(P.N);
    const dim3 grid((unsigned)((P.N + bs - 1) / bs)), block(bs);
    long long t = t0;
    int n = n_steps;
    NeuronParams p = P;
    RecordParams r = R;
    void* args[] = {&p, &t, &n, &I_steps, &r};
    size_t smem = 0;
    cudaError_t e = poly_smem(K.independent, P, &smem);
    if (e != cudaSuccess)
        return e;
    return cudaLaunchKernel((const void*)K.independent, grid, block, args, smem, st);
}

cudaError_t jit_launch_window(const JitKernels& K, const NeuronParams& P, int64_t t0, int32_t W,
                              int32_t parity, const float* I_steps, const RecordParams& R,
                              const SpikeList& L, int32_t early, int32_t block_size, cudaStream_t st)
{
    const int bs = block_size > 0 ? block_size : block_for(P.N);
    const dim3 grid((unsigned)((P.N + bs - 1) / bs)), block(bs);
    long long t = t0;
    int w = W, par = parity, ea = early;
    NeuronParams p = P;
    RecordParams r = R;
    SpikeList l = L;
    void* args[] = {&p, &t, &w, &I_steps, &r, &l, &par, &ea};
    // programmatic dependent launch: scheduled while the previous window
    // runs, released by its completion (griddepcontrol in the kernel)
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = st;
    cudaError_t e = poly_smem(K.window, P, &cfg.dynamicSmemBytes);
    if (e != cudaSuccess)
        return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)K.window, args);
}

// Blocks of the persistent kernel (kPersistNeurons neurons each) that can
// be resident at once (0 if the query fails).
int jit_persistent_capacity(const JitKernels& K, const NeuronParams& P)
{
    int per_sm = 0, dev = 0, sms = 0;
    size_t smem = 0;
    if (poly_smem(K.persistent, P, &smem) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)K.persistent, kPersistThreads, smem) !=
            cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t jit_launch_persistent(const JitKernels& K, const NeuronParams& P, const RouteParams& RP, int64_t t0,
                                  int32_t n_steps, int32_t W, int64_t w_index0, const float* I_steps,
                                  const RecordParams& R, const SpikeList& L, const PhaseCounters& pc,
                                  cudaStream_t st)
{
    NeuronParams p = P;
    RouteParams rp = RP;
    RecordParams r = R;
    SpikeList l = L;
    PhaseCounters g = pc;
    long long t = t0, wi = w_index0;
    int n = n_steps, w = W;
    void* args[] = {&p, &rp, &t, &n, &w, &wi, &I_steps, &r, &l, &g};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((P.N + kPersistNeurons - 1) / kPersistNeurons));
    cfg.blockDim = dim3(kPersistThreads);
    cfg.stream = st;
    cudaError_t e = poly_smem(K.persistent, P, &cfg.dynamicSmemBytes);
    if (e != cudaSuccess)
        return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)K.persistent, args);
}

cudaError_t jit_launch_indexed(const JitKernels& K, const NeuronParams& P, const int32_t* list,
                               const int32_t* n_list, int64_t max_list, int64_t t0, int32_t n_steps,
                               const RecordParams& R, cudaStream_t st)
{
    const int bs = 128;
    const dim3 grid((unsigned)((max_list + bs - 1) / bs)), block(bs);
    long long t = t0;
    int n = n_steps;
    NeuronParams p = P;
    RecordParams r = R;
    void* args[] = {&p, &list, &n_list, &t, &n, &r};
    return cudaLaunchKernel((const void*)K.indexed, grid, block, args, 0, st);
}

}  // namespace hh
