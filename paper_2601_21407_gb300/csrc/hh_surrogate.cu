// Learned multi-step gating surrogate for independent neurons.
//
// A small MLP (features 32 -> 64 -> 64 -> 16, tanh) advances the neuron
// state (V, gates, Ca) by W time steps at once inside the sub-threshold
// envelope it was trained on, as a learned correction to one
// exponential-Euler step over the whole window; everything else -- and
// every window that leaves the envelope or needs a larger correction than
// the error estimate allows -- is integrated by the plain exponential-Euler
// kernel, which also generated the training data and judges the error.
// (The paper accelerates its ion-channel operators with polynomial
// approximations of the rates, Methods "Engineering optimization"; this
// surrogate replaces several steps instead, a design the paper does not
// describe.)
//
//   data      k_sur_gen: the plain integrator on random training neurons
//             records (features(state_t), state_{t+W} - coarse(state_t))
//             for windows whose V stays below v_env;
//   training  k_sur_train / k_sur_adam: FP32 forward + backward of a
//             128-sample block, deterministic reduction of block partials,
//             Adam;
//   inference k_sur_infer: per CTA 128 neurons, three tcgen05.mma layers
//             (M=128, bf16 operands in 128-byte-swizzled shared memory, fp32
//             accumulators in TMEM, tanh epilogues written back to shared
//             memory); predictions inside the envelope are accepted, the
//             other neurons are appended to a list that the plain kernel
//             integrates for the same window.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <random>
#include <vector>

#include "hh_internal.h"
#include "hh_tc.cuh"

namespace hh {
namespace {

using namespace tc;

constexpr int kSF = 32;          // feature slots (layer-1 K used; rows padded to 64)
constexpr int kSH = 64;          // hidden width
constexpr int kSO = 16;          // output slots
constexpr int kRow = 64;         // bf16 per operand row (128 bytes, one swizzle row)
constexpr int kNP = kSH * kRow + kSH + kSH * kRow + kSH + kSO * kRow + kSO;  // parameter count

// offsets into the parameter vector [W1 | b1 | W2 | b2 | W3 | b3], W row-major [out][64]
constexpr int oW1 = 0, ob1 = oW1 + kSH * kRow, oW2 = ob1 + kSH, ob2 = oW2 + kSH * kRow,
              oW3 = ob2 + kSH, ob3 = oW3 + kSO * kRow;

struct SurNorm {
    float out_scale[kSO];
    float lo[kSF], hi[kSF];   // trained envelope of the features, widened by the margin
    float v_env;
    int32_t n_feat, n_out, G, has_ca;
    float gbar_ref[kMaxChannels];
};

// Features of one neuron (see the header comment of hh_surrogate_train).
__device__ __forceinline__ void sur_features(const DevModel& M, const SurNorm& S, float V, const float* p,
                                             float Ca, float I, const float* gch, float* f)
{
#pragma unroll
    for (int k = 0; k < kSF; ++k)
        f[k] = 0.0f;
    f[0] = (V + 65.0f) * 0.05f;
#pragma unroll
    for (int q = 0; q < kMaxGates; ++q)
        if (q < M.n_gates)
            f[1 + q] = 2.0f * p[q] - 1.0f;
    const int G = M.n_gates;
    // (fast logarithms and divisions: the features feed a bf16 network, and
    // training and inference evaluate them alike)
    f[1 + G] = S.has_ca ? 0.5f * __logf(__fdividef(fmaxf(Ca, 1e-6f), M.ca_rest)) : 0.0f;
    f[2 + G] = I * 0.1f;
#pragma unroll
    for (int c = 0; c < kMaxChannels; ++c)
        if (c < M.n_ch && 3 + G + c < kSF)
            f[3 + G + c] = S.gbar_ref[c] > 0.0f
                               ? __logf(__fdividef(fmaxf(gch[c], 1e-12f), S.gbar_ref[c])) * (1.0f / 0.3f)
                               : 0.0f;
}

// One exponential-Euler step over a whole window (rates at its first V,
// step dt W; Mc is the model with the calcium decay of dt W) from a
// neuron's state: the coarse prediction the MLP corrects.
template <int PREC>
__device__ __forceinline__ void coarse_step(const DevModel& Mc, float dt_w, float V, const float* p, float Ca,
                                            float I, const float* gch, State<kMaxGates, PREC>& c)
{
    c.poly = nullptr;
    c.V = V;
    c.Vlo = 0.0f;
    c.Ca = Ca;
    c.gconst = 0.0f;
    c.gconstE = 0.0f;
#pragma unroll
    for (int ch = 0; ch < kMaxChannels; ++ch)
        if (ch < Mc.n_ch && Mc.ch_ng[ch] == 0) {
            c.gconst += gch[ch];
            c.gconstE += gch[ch] * Mc.E[ch];
        }
#pragma unroll
    for (int q = 0; q < kMaxGates; ++q) {
        c.p[q] = p[q];
        c.plo[q] = 0.0f;
        c.gq[q] = (q < Mc.n_gates && Mc.gate_last[q]) ? gch[Mc.gate_ch[q]] : 0.0f;
    }
    neuron_step<kMaxGates, PREC>(Mc, dt_w, HH_V_EXP_EULER, I, 0.0f, 0.0f, 0.0f, 0.0f, c);
}

// ---------------------------------------------------------------------------
// training data
// ---------------------------------------------------------------------------
struct GenParams {
    int32_t n_neurons, windows, W, precision;
    float dt, v_env;
    const float* I;        // [n]
    const float* V0;       // [n]
    const float* gch;      // [kMaxChannels][n]
    float* X;              // [cap][kSF]
    float* Y;              // [cap][kSO]  (raw increments)
    unsigned long long* count;
    int64_t cap;
};

template <int PREC>
__global__ void __launch_bounds__(128) k_sur_gen(const __grid_constant__ DevModels Ms,
                                                 const __grid_constant__ DevModels Mc,
                                                 const __grid_constant__ SurNorm S,
                                                 const __grid_constant__ GenParams g)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_neurons)
        return;
    const DevModel& M = Ms.m[0];
    State<kMaxGates, PREC> s;
    float gch[kMaxChannels];
    for (int c = 0; c < kMaxChannels; ++c)
        gch[c] = c < M.n_ch ? g.gch[(int64_t)c * g.n_neurons + i] : 0.0f;
    // per-neuron conductances: the channel's gbar at its last gate / gate-less channels
    s.gconst = 0.0f;
    s.gconstE = 0.0f;
    for (int c = 0; c < kMaxChannels; ++c)
        if (c < M.n_ch && M.ch_ng[c] == 0) {
            s.gconst += gch[c];
            s.gconstE += gch[c] * M.E[c];
        }
#pragma unroll
    for (int q = 0; q < kMaxGates; ++q)
        s.gq[q] = (q < M.n_gates && M.gate_last[q]) ? gch[M.gate_ch[q]] : 0.0f;
    s.V = g.V0[i];
    s.Vlo = 0.0f;
    s.Ca = M.ca_ch >= 0 ? M.ca_rest : 0.0f;
#pragma unroll
    for (int q = 0; q < kMaxGates; ++q) {
        float inf = 0.0f, z;
        if (q < M.n_gates)
            gate_inf_z<false>(M.g[q], s.V, s.Ca, 1.0f, inf, z);
        s.p[q] = inf;
        s.plo[q] = 0.0f;
    }
    const float I = g.I[i];
    for (int w = 0; w < g.windows; ++w) {
        const float V0 = s.V, Ca0 = s.Ca;
        float p0[kMaxGates];
#pragma unroll
        for (int q = 0; q < kMaxGates; ++q)
            p0[q] = s.p[q];
        State<kMaxGates, PREC> c;
        coarse_step<PREC>(Mc.m[0], g.dt * (float)g.W, V0, p0, Ca0, I, gch, c);
        float vmax = s.V;
        for (int k = 0; k < g.W; ++k) {
            neuron_step<kMaxGates, PREC>(M, g.dt, HH_V_EXP_EULER, I, 0.0f, 0.0f, 0.0f, 0.0f, s);
            vmax = fmaxf(vmax, s.V);
        }
        if (V0 < g.v_env && vmax < g.v_env && finite(s.V)) {
            const unsigned long long slot = atomicAdd(g.count, 1ull);
            if ((int64_t)slot < g.cap) {
                float f[kSF];
                sur_features(M, S, V0, p0, Ca0, I, gch, f);
                float* x = g.X + slot * kSF;
                for (int k = 0; k < kSF; ++k)
                    x[k] = f[k];
                float* y = g.Y + slot * kSO;
                for (int k = 0; k < kSO; ++k)
                    y[k] = 0.0f;
                // the target is the plain integrator's window minus the
                // coarse step: what the MLP has to add to the coarse step
                y[0] = s.V - c.V;
                for (int q = 0; q < M.n_gates; ++q)
                    y[1 + q] = s.p[q] - c.p[q];
                if (S.has_ca)
                    y[1 + M.n_gates] = s.Ca - c.Ca;
            }
        }
    }
}

// column statistics (deterministic two-pass): part[c][col] over row chunks
constexpr int kStatChunks = 256;
__global__ void k_col_stats(const float* __restrict__ A, int64_t rows, int cols, float* psum, float* psq,
                            float* pmin, float* pmax)
{
    const int col = threadIdx.x;
    const int c = blockIdx.x;
    if (col >= cols)
        return;
    const int64_t r0 = rows * c / kStatChunks, r1 = rows * (c + 1) / kStatChunks;
    double s = 0.0, q = 0.0;
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t r = r0; r < r1; ++r) {
        const float v = A[r * cols + col];
        s += v;
        q += (double)v * v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    psum[c * cols + col] = (float)s;
    psq[c * cols + col] = (float)q;
    pmin[c * cols + col] = mn;
    pmax[c * cols + col] = mx;
}

__global__ void k_scale_targets(float* Y, int64_t rows, const float* __restrict__ inv_scale)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < rows * kSO)
        Y[i] *= inv_scale[i % kSO];
}

// ---------------------------------------------------------------------------
// training: one block = 128 samples; writes its gradient partials
// ---------------------------------------------------------------------------
constexpr int kTB = 128;
constexpr int kTS = 65;  // smem row stride for 64-wide activations
constexpr size_t kTrainSmem =
    sizeof(float) * (kNP + kTB * (kSF + 1) + 4 * kTB * kTS + kTB * (kSO + 1));

__global__ void __launch_bounds__(kTB, 1) k_sur_train(const float* __restrict__ params, const float* __restrict__ X,
                                                      const float* __restrict__ Y, const int32_t* __restrict__ idx,
                                                      int64_t n_rows, int n_out, float* __restrict__ partial,
                                                      float* __restrict__ loss_part)
{
    extern __shared__ float sm[];
    float* W = sm;                                   // kNP
    float* xs = W + kNP;                             // [128][33]
    float* h1 = xs + kTB * (kSF + 1);                // [128][65]
    float* h2 = h1 + kTB * kTS;
    float* g2 = h2 + kTB * kTS;
    float* g1 = g2 + kTB * kTS;
    float* dout = g1 + kTB * kTS;                    // [128][17]
    const int t = threadIdx.x;
    for (int k = t; k < kNP; k += kTB)
        W[k] = params[k];
    const int64_t r = (int64_t)blockIdx.x * kTB + t;
    const bool valid = r < n_rows;
    const int64_t row = valid ? idx[r] : 0;
    for (int k = 0; k < kSF; ++k)
        xs[t * (kSF + 1) + k] = valid ? X[row * kSF + k] : 0.0f;
    __syncthreads();
    // forward
    for (int j = 0; j < kSH; ++j) {
        float a = W[ob1 + j];
        for (int k = 0; k < kSF; ++k)
            a = fmaf(W[oW1 + j * kRow + k], xs[t * (kSF + 1) + k], a);
        h1[t * kTS + j] = tanhf(a);
    }
    for (int j = 0; j < kSH; ++j) {
        float a = W[ob2 + j];
        for (int k = 0; k < kSH; ++k)
            a = fmaf(W[oW2 + j * kRow + k], h1[t * kTS + k], a);
        h2[t * kTS + j] = tanhf(a);
    }
    float lsum = 0.0f;
    for (int j = 0; j < kSO; ++j) {
        float a = W[ob3 + j];
        for (int k = 0; k < kSH; ++k)
            a = fmaf(W[oW3 + j * kRow + k], h2[t * kTS + k], a);
        float e = 0.0f;
        if (valid && j < n_out) {
            e = a - Y[row * kSO + j];
            lsum += e * e;
        }
        dout[t * (kSO + 1) + j] = 2.0f * e;
    }
    // backward to the hidden layers
    for (int k = 0; k < kSH; ++k) {
        float a = 0.0f;
        for (int j = 0; j < kSO; ++j)
            a = fmaf(dout[t * (kSO + 1) + j], W[oW3 + j * kRow + k], a);
        const float h = h2[t * kTS + k];
        g2[t * kTS + k] = a * (1.0f - h * h);
    }
    for (int k = 0; k < kSH; ++k) {
        float a = 0.0f;
        for (int j = 0; j < kSH; ++j)
            a = fmaf(g2[t * kTS + j], W[oW2 + j * kRow + k], a);
        const float h = h1[t * kTS + k];
        g1[t * kTS + k] = a * (1.0f - h * h);
    }
    __syncthreads();
    // weight gradients of this block: thread t covers entries t, t+128, ...
    float* out = partial + (int64_t)blockIdx.x * kNP;
    for (int e = t; e < kNP; e += kTB) {
        float s = 0.0f;
        if (e < ob1) {
            const int j = (e - oW1) / kRow, k = (e - oW1) % kRow;
            if (k < kSF)
                for (int b = 0; b < kTB; ++b)
                    s = fmaf(g1[b * kTS + j], xs[b * (kSF + 1) + k], s);
        } else if (e < oW2) {
            const int j = e - ob1;
            for (int b = 0; b < kTB; ++b)
                s += g1[b * kTS + j];
        } else if (e < ob2) {
            const int j = (e - oW2) / kRow, k = (e - oW2) % kRow;
            for (int b = 0; b < kTB; ++b)
                s = fmaf(g2[b * kTS + j], h1[b * kTS + k], s);
        } else if (e < oW3) {
            const int j = e - ob2;
            for (int b = 0; b < kTB; ++b)
                s += g2[b * kTS + j];
        } else if (e < ob3) {
            const int j = (e - oW3) / kRow, k = (e - oW3) % kRow;
            for (int b = 0; b < kTB; ++b)
                s = fmaf(dout[b * (kSO + 1) + j], h2[b * kTS + k], s);
        } else {
            const int j = e - ob3;
            for (int b = 0; b < kTB; ++b)
                s += dout[b * (kSO + 1) + j];
        }
        out[e] = s;
    }
    // block loss (sum of squared errors) for reporting
    __shared__ float red[kTB];
    red[t] = lsum;
    __syncthreads();
    if (t == 0) {
        float s = 0.0f;
        for (int b = 0; b < kTB; ++b)
            s += red[b];
        loss_part[blockIdx.x] = s;
    }
}

__global__ void k_sur_adam(float* params, float* m, float* v, const float* __restrict__ partial, int n_blocks,
                           float scale, float lr, float b1t, float b2t)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kNP)
        return;
    float g = 0.0f;
    for (int b = 0; b < n_blocks; ++b)
        g += partial[(int64_t)b * kNP + e];
    g *= scale;
    const float mm = 0.9f * m[e] + 0.1f * g;
    const float vv = 0.999f * v[e] + 0.001f * g * g;
    m[e] = mm;
    v[e] = vv;
    params[e] -= lr * (mm / (1.0f - b1t)) / (sqrtf(vv / (1.0f - b2t)) + 1e-8f);
}

__global__ void k_to_bf16(const float* __restrict__ a, int n, uint16_t* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint32_t u = __float_as_uint(a[i]);
        out[i] = (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
    }
}

// ---------------------------------------------------------------------------
// inference
// ---------------------------------------------------------------------------
struct InferParams {
    const uint16_t* W1;   // bf16 [64][64]
    const uint16_t* W2;   // bf16 [64][64]
    const uint16_t* W3;   // bf16 [16][64]
    const float* b;       // [64 | 64 | 16]
    int32_t* fb_list;     // [N] neurons the plain kernel integrates this window
    int32_t* fb_count;
    unsigned long long* stats;  // [0] accepted windows, [1] fallbacks
    int32_t* err;
    int32_t W;            // steps per window
    float err_V, err_p;   // error-estimate tolerances (err_V <= 0: off)
};

constexpr uint32_t kTile = 128 * kRow * 2;  // 16 KB per 128-row bf16 tile
// one activation tile (features, then each hidden layer's output in turn),
// the three weight tiles and the biases: five CTAs per SM
constexpr size_t kInferSmem = 1024 + kTile + (kSH + kSH + kSO) * kRow * 2 + (2 * kSH + kSO) * 4 + 64;
constexpr int kInferCtasPerSm = 5;
constexpr uint32_t kInferTmemCols = 64;

// two floats as a packed bf16 pair (lo in the low half), rounded to nearest
// even by the hardware conversion
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// columns 32 h .. 32 h + 31 of row r of a 128-byte-swizzled bf16 tile
// (16-byte chunk j of row r at chunk j ^ (r & 7); here j = 4 h .. 4 h + 3);
// v == nullptr writes zeros
__device__ __forceinline__ void put_half(uint8_t* tile, int r, int h, const float* v)
{
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        uint4 c = make_uint4(0u, 0u, 0u, 0u);
        if (v) {
            c.x = bf16x2_rn(v[8 * jj + 0], v[8 * jj + 1]);
            c.y = bf16x2_rn(v[8 * jj + 2], v[8 * jj + 3]);
            c.z = bf16x2_rn(v[8 * jj + 4], v[8 * jj + 5]);
            c.w = bf16x2_rn(v[8 * jj + 6], v[8 * jj + 7]);
        }
        const int j = 4 * h + jj;
        *reinterpret_cast<uint4*>(tile + r * 128 + ((j ^ (r & 7)) << 4)) = c;
    }
}

template <int PREC>
__global__ void __launch_bounds__(128, kInferCtasPerSm) k_sur_infer(const __grid_constant__ DevModels Ms,
                                                                    const __grid_constant__ DevModels Mcoarse,
                                                                    const __grid_constant__ SurNorm S,
                                                                    const __grid_constant__ NeuronParams P,
                                                                    const __grid_constant__ InferParams Q)
{
    // Persistent: each CTA stages the weights and biases once, allocates its
    // TMEM columns once and takes 128-neuron tiles tile = blockIdx.x,
    // blockIdx.x + gridDim.x, ...  Per tile: features -> A; three
    // tcgen05.mma layers, each epilogue reading its accumulator from TMEM
    // (columns 0..63, reused by every layer) and writing its activations
    // back into A once the layer's MMA has completed.
    extern __shared__ uint8_t raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* A = sm;
    uint8_t* B1 = A + kTile;
    uint8_t* B2 = B1 + kSH * 128;
    uint8_t* B3 = B2 + kSH * 128;
    float* sb = reinterpret_cast<float*>(B3 + kSO * 128);   // [64 | 64 | 16]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sb + 2 * kSH + kSO);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const DevModel& M = Ms.m[0];

    // weights -> swizzled tiles (row r chunk j at j ^ (r & 7)); biases
    for (int c = t; c < (kSH + kSH + kSO) * 8; c += 128) {
        const int r = c >> 3, j = c & 7;
        const uint16_t* src;
        uint8_t* dst;
        int rr;
        if (r < kSH) {
            src = Q.W1; dst = B1; rr = r;
        } else if (r < 2 * kSH) {
            src = Q.W2; dst = B2; rr = r - kSH;
        } else {
            src = Q.W3; dst = B3; rr = r - 2 * kSH;
        }
        *reinterpret_cast<uint4*>(dst + rr * 128 + ((j ^ (rr & 7)) << 4)) =
            *reinterpret_cast<const uint4*>(src + rr * kRow + 8 * j);
    }
    for (int k = t; k < 2 * kSH + kSO; k += 128)
        sb[k] = Q.b[k];
    if (t == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0)
        tmem_alloc(tslot, kInferTmemCols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    const int64_t n_tiles = (P.N + 127) / 128;
    unsigned long long n_acc = 0, n_dec = 0;
    // false once a wait of this CTA has run out (status bit set): the phase
    // bookkeeping can no longer be trusted, so every later window of the
    // CTA goes to the plain kernel
    bool ok = true;

    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // neuron state and features
        const int64_t gi = tile * 128 + t;
        const bool valid = gi < P.N;
        const int64_t i = valid ? gi : 0;
        const float V = P.V[i], Ca = P.Ca[i];
        float p[kMaxGates];
#pragma unroll
        for (int q = 0; q < kMaxGates; ++q)
            p[q] = P.P[(int64_t)q * P.N + i];
        float gch[kMaxChannels];
#pragma unroll
        for (int c = 0; c < kMaxChannels; ++c)
            gch[c] = c < M.n_ch ? (P.gbar ? P.gbar[(int64_t)c * P.N + i] : M.gbar[c]) : 0.0f;
        const float I = P.I_const ? P.I_const[i] : 0.0f;
        bool cand = valid && V < S.v_env && finite(V);
        {
            float f[kSF];
            sur_features(M, S, V, p, Ca, I, gch, f);
#pragma unroll
            for (int k = 0; k < kSF; ++k) {
                if (k < S.n_feat)
                    cand = cand && f[k] >= S.lo[k] && f[k] <= S.hi[k];
            }
            put_half(A, t, 0, cand ? f : nullptr);
            put_half(A, t, 1, nullptr);
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // two hidden layers: A x W^T -> TMEM columns 0..63, tanh(. + b) -> A
#pragma unroll 1
        for (int layer = 0; layer < 2; ++layer) {
            if (t == 0) {
                const uint64_t da = sdesc(smem_u32(A)), db = sdesc(smem_u32(layer == 0 ? B1 : B2));
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc_bf16(128, kSH), k > 0 ? 1u : 0u);
                mma_commit(bar);
            }
            ok = mbar_wait(bar, phase, Q.err, 16) && ok;
            phase ^= 1u;
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float v[32];
                tmem_ld32(tmem + lane_base + 32 * h, v);
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    v[k] = tanh_approx(v[k] + sb[layer * kSH + 32 * h + k]);
                put_half(A, t, h, v);
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
        }
        // output layer: A x W3^T -> columns 0..15
        if (t == 0) {
            const uint64_t da = sdesc(smem_u32(A)), db = sdesc(smem_u32(B3));
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc_bf16(128, kSO), k > 0 ? 1u : 0u);
            mma_commit(bar);
        }
        ok = mbar_wait(bar, phase, Q.err, 16) && ok;
        phase ^= 1u;
        tc_fence_after();
        float o[kSO];
        tmem_ld16(tmem + lane_base, o);

        // the prediction: the coarse step plus the learned correction;
        // accepted inside the envelope (and, with the error estimate on,
        // when the correction is small: the MLP's error is a fraction of
        // it), otherwise the window goes to the plain kernel
        const int G = M.n_gates;
        State<kMaxGates, PREC> c;
        coarse_step<PREC>(Mcoarse.m[0], P.dt * (float)Q.W, V, p, Ca, I, gch, c);
        const float Vn = c.V + (o[0] + sb[2 * kSH + 0]) * S.out_scale[0];
        bool acc = cand && ok && Vn < S.v_env && finite(Vn);
        if (Q.err_V > 0.0f)
            acc = acc && fabsf(Vn - c.V) <= Q.err_V;
        float pn[kMaxGates];
#pragma unroll
        for (int q = 0; q < kMaxGates; ++q) {
            pn[q] = p[q];
            if (q < G) {
                pn[q] = c.p[q] + (o[1 + q] + sb[2 * kSH + 1 + q]) * S.out_scale[1 + q];
                acc = acc && pn[q] >= 0.0f && pn[q] <= 1.0f;
                if (Q.err_V > 0.0f)
                    acc = acc && fabsf(pn[q] - c.p[q]) <= Q.err_p;
            }
        }
        float Can = Ca;
        if (S.has_ca) {
            Can = c.Ca + (o[1 + G] + sb[2 * kSH + 1 + G]) * S.out_scale[1 + G];
            acc = acc && Can > 0.0f;
        }
        if (valid && acc) {
            P.V[i] = Vn;
            P.Ca[i] = Can;
#pragma unroll
            for (int q = 0; q < kMaxGates; ++q)
                if (q < G)
                    P.P[(int64_t)q * P.N + i] = pn[q];
        }
        // warp-aggregated append of the declined neurons
        const bool fb = valid && !acc;
        const unsigned bm = __ballot_sync(0xffffffffu, fb);
        const unsigned am = __ballot_sync(0xffffffffu, valid && acc);
        if (bm) {
            int base = 0;
            if (lane == __ffs(bm) - 1)
                base = atomicAdd(Q.fb_count, __popc(bm));
            base = __shfl_sync(0xffffffffu, base, __ffs(bm) - 1);
            if (fb)
                Q.fb_list[base + __popc(bm & ((1u << lane) - 1u))] = (int32_t)i;
        }
        n_acc += __popc(am);
        n_dec += __popc(bm);
        // every thread's TMEM reads are complete before the next tile's
        // first MMA (the barrier after the next features) overwrites them
    }
    if (lane == 0) {
        if (n_acc)
            atomicAdd(&Q.stats[0], n_acc);
        if (n_dec)
            atomicAdd(&Q.stats[1], n_dec);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        tmem_dealloc(tmem, kInferTmemCols);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Surrogate {
    int W = 10;
    int n_out = 0;
    SurNorm norm{};
    float err_V = 0.0f, err_p = 0.0f;
    DevModels coarse{};          // the network's models with the calcium decay of dt W
    float* params = nullptr;     // fp32 master parameters
    uint16_t* wb = nullptr;      // bf16 copies of W1 | W2 | W3
    float* bias = nullptr;       // [64 | 64 | 16]
    int32_t* fb_list = nullptr;
    int32_t* fb_count = nullptr;
    unsigned long long* stats = nullptr;
    int32_t* err = nullptr;
    int64_t N = 0;
    float margin = 0.0f;         // fractional widening of the feature envelope
    std::vector<void*> allocs;
    template <class T>
    cudaError_t alloc(T** p, size_t n)
    {
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
        if (e == cudaSuccess) {
            allocs.push_back(*p);
            e = cudaMemset(*p, 0, (n ? n : 1) * sizeof(T));
        }
        return e;
    }
    ~Surrogate()
    {
        for (void* p : allocs)
            cudaFree(p);
    }
};

void surrogate_free(Surrogate* s) { delete s; }

hh_status surrogate_train(const DevModels& Ms, int precision, double dt, int64_t N_net,
                          const hh_surrogate_desc* d, cudaStream_t st, Surrogate** out, hh_surrogate_report* rep)
{
    const DevModel& M = Ms.m[0];
    if (d->window < 1 || d->window > 1000 || d->train_neurons < 128 || d->train_windows < 1024 ||
        d->epochs < 1 || d->batch < 128 || !(d->lr > 0.0f) || !(d->I_max >= d->I_min) ||
        !(d->V0_max >= d->V0_min) || d->gbar_sigma < 0.0f)
        return fail(HH_EINVAL, "surrogate descriptor out of range");
    const int G = M.n_gates, has_ca = M.ca_ch >= 0 ? 1 : 0;
    const int n_feat = 3 + G + M.n_ch, n_out = 1 + G + has_ca;
    if (n_feat > kSF || n_out > kSO)
        return fail(HH_EUNSUPPORTED, "model too large for the surrogate (%d features, %d outputs)", n_feat, n_out);
    if (!(d->err_V >= 0.0f) || !(d->err_p >= 0.0f) || !std::isfinite(d->err_V) || !std::isfinite(d->err_p) ||
        (d->err_V > 0.0f && !(d->err_p > 0.0f)))
        return fail(HH_EINVAL, "surrogate error-estimate tolerances: err_V >= 0, and err_p > 0 when err_V > 0");
    Surrogate* S = new Surrogate();
    S->W = d->window;
    S->err_V = d->err_V;
    S->err_p = d->err_p;
    S->coarse = Ms;
    for (int k = 0; k < kMaxModels; ++k)
        if (S->coarse.m[k].ca_tau > 0.0f)
            S->coarse.m[k].ca_decay = (float)std::exp(-(double)d->window * dt / (double)S->coarse.m[k].ca_tau);
    S->n_out = n_out;
    S->N = N_net;
    S->margin = 0.02f;
    SurNorm& nm = S->norm;
    nm.v_env = d->v_envelope;
    nm.n_feat = n_feat;
    nm.n_out = n_out;
    nm.G = G;
    nm.has_ca = has_ca;
    for (int c = 0; c < kMaxChannels; ++c)
        nm.gbar_ref[c] = c < M.n_ch ? M.gbar[c] : 0.0f;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess)
            e = S->alloc(p, n);
    };
    // training population
    const int ntr = d->train_neurons;
    std::mt19937_64 rng(d->seed);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::normal_distribution<double> Z(0.0, 1.0);
    std::vector<float> hI(ntr), hV(ntr), hg((size_t)kMaxChannels * ntr, 0.0f);
    for (int k = 0; k < ntr; ++k) {
        hI[k] = (float)(d->I_min + (d->I_max - d->I_min) * U(rng));
        hV[k] = (float)(d->V0_min + (d->V0_max - d->V0_min) * U(rng));
        for (int c = 0; c < M.n_ch; ++c)
            hg[(size_t)c * ntr + k] = (float)(M.gbar[c] * std::exp(d->gbar_sigma * Z(rng)));
    }
    float *dI = nullptr, *dV = nullptr, *dg = nullptr, *X = nullptr, *Y = nullptr;
    unsigned long long* cnt = nullptr;
    const int64_t cap = d->train_windows;
    A(&dI, ntr);
    A(&dV, ntr);
    A(&dg, (size_t)kMaxChannels * ntr);
    A(&X, (size_t)cap * kSF);
    A(&Y, (size_t)cap * kSO);
    A(&cnt, 1);
    A(&S->params, kNP);
    A(&S->wb, (size_t)(2 * kSH + kSO) * kRow);
    A(&S->bias, 2 * kSH + kSO);
    A(&S->fb_list, (size_t)std::max<int64_t>(N_net, 1));
    A(&S->fb_count, 1);
    A(&S->stats, 2);
    A(&S->err, 1);
    float *m = nullptr, *v = nullptr, *part = nullptr, *lpart = nullptr;
    int32_t* idx = nullptr;
    const int bs = std::max(kTB, d->batch / kTB * kTB);
    const int nblk = bs / kTB;
    A(&m, kNP);
    A(&v, kNP);
    A(&part, (size_t)nblk * kNP);
    A(&lpart, (size_t)nblk);
    A(&idx, (size_t)cap);
    auto bail = [&](hh_status s, const char* what) {
        cudaStreamSynchronize(st);
        delete S;
        return fail(s, "%s: %s", what, cudaGetErrorString(e));
    };
    if (e != cudaSuccess)
        return bail(HH_ENOMEM, "surrogate allocation");
    e = cudaMemcpyAsync(dI, hI.data(), ntr * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dV, hV.data(), ntr * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dg, hg.data(), hg.size() * 4, cudaMemcpyHostToDevice, st);
    // data generation: enough windows per neuron for ~2x the cap of candidates
    GenParams gp{};
    gp.n_neurons = ntr;
    gp.windows = (int)std::max<int64_t>(4, (2 * cap + ntr - 1) / ntr);
    gp.W = d->window;
    gp.precision = precision;
    gp.dt = (float)dt;
    gp.v_env = d->v_envelope;
    gp.I = dI;
    gp.V0 = dV;
    gp.gch = dg;
    gp.X = X;
    gp.Y = Y;
    gp.count = cnt;
    gp.cap = cap;
    if (e == cudaSuccess) {
        if (precision == HH_PREC_FAST)
            k_sur_gen<HH_PREC_FAST><<<(ntr + 127) / 128, 128, 0, st>>>(Ms, S->coarse, nm, gp);
        else
            k_sur_gen<HH_PREC_ACCURATE><<<(ntr + 127) / 128, 128, 0, st>>>(Ms, S->coarse, nm, gp);
        e = cudaGetLastError();
    }
    unsigned long long got = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&got, cnt, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return bail(HH_ECUDA, "surrogate training data");
    const int64_t n = std::min<int64_t>((int64_t)got, cap);
    if (n < 4 * kTB) {
        delete S;
        return fail(HH_EINVAL, "only %lld training windows stay inside the envelope", (long long)n);
    }
    // statistics: output scales and the feature envelope
    {
        float *ps, *pq, *pmn, *pmx;
        std::vector<float> hs(kStatChunks * kSO), hq(kStatChunks * kSO), hmn(kStatChunks * kSO),
            hmx(kStatChunks * kSO);
        A(&ps, kStatChunks * kSO);
        A(&pq, kStatChunks * kSO);
        A(&pmn, kStatChunks * kSO);
        A(&pmx, kStatChunks * kSO);
        for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
            const float* src = pass == 0 ? Y : X;
            const int cols = pass == 0 ? kSO : kSF;
            std::vector<float> cs(kStatChunks * cols), cq(kStatChunks * cols), cmn(kStatChunks * cols),
                cmx(kStatChunks * cols);
            float *gs, *gq, *gmn, *gmx;
            A(&gs, kStatChunks * cols);
            A(&gq, kStatChunks * cols);
            A(&gmn, kStatChunks * cols);
            A(&gmx, kStatChunks * cols);
            if (e != cudaSuccess)
                break;
            k_col_stats<<<kStatChunks, 64, 0, st>>>(src, n, cols, gs, gq, gmn, gmx);
            e = cudaMemcpyAsync(cs.data(), gs, cs.size() * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(cq.data(), gq, cq.size() * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(cmn.data(), gmn, cmn.size() * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(cmx.data(), gmx, cmx.size() * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(st);
            for (int col = 0; col < cols; ++col) {
                double s = 0, q = 0;
                float mn = INFINITY, mx = -INFINITY;
                for (int c = 0; c < kStatChunks; ++c) {
                    s += cs[c * cols + col];
                    q += cq[c * cols + col];
                    mn = std::min(mn, cmn[c * cols + col]);
                    mx = std::max(mx, cmx[c * cols + col]);
                }
                if (pass == 0) {
                    const double mean = s / n, var = std::max(0.0, q / n - mean * mean);
                    nm.out_scale[col] = col < n_out ? (float)std::max(std::sqrt(var), 1e-7) : 1.0f;
                } else {
                    // the envelope widened by the margin on both sides
                    const double w = ((double)mx - (double)mn) * S->margin;
                    nm.lo[col] = col < n_feat ? (float)((double)mn - w) : 0.0f;
                    nm.hi[col] = col < n_feat ? (float)((double)mx + w) : 0.0f;
                }
            }
        }
        std::vector<float> inv(kSO);
        for (int k = 0; k < kSO; ++k)
            inv[k] = 1.0f / nm.out_scale[k];
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ps, inv.data(), kSO * 4, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            k_scale_targets<<<(int)((n * kSO + 255) / 256), 256, 0, st>>>(Y, n, ps);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess)
        return bail(HH_ECUDA, "surrogate statistics");
    // initial parameters (uniform, fan-in scaled) and training
    {
        std::vector<float> hp(kNP, 0.0f);
        auto init = [&](int off, int rows, int fan_in) {
            const double a = std::sqrt(6.0 / (fan_in + rows));
            for (int r = 0; r < rows; ++r)
                for (int k = 0; k < fan_in; ++k)
                    hp[off + r * kRow + k] = (float)((2.0 * U(rng) - 1.0) * a);
        };
        init(oW1, kSH, n_feat);
        init(oW2, kSH, kSH);
        init(oW3, kSO, kSH);
        for (int r = n_out; r < kSO; ++r)
            for (int k = 0; k < kRow; ++k)
                hp[oW3 + r * kRow + k] = 0.0f;
        e = cudaMemcpyAsync(S->params, hp.data(), kNP * 4, cudaMemcpyHostToDevice, st);
    }
    const int64_t n_val = std::max<int64_t>(kTB, n / 20);
    const int64_t n_tr = n - n_val;
    std::vector<int32_t> perm(n_tr);
    for (int64_t k = 0; k < n_tr; ++k)
        perm[k] = (int32_t)k;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sur_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
        attr = true;
    }
    int64_t step = 0;
    const int64_t steps_per_epoch = n_tr / bs;
    const int64_t total = steps_per_epoch * d->epochs;
    for (int ep = 0; ep < d->epochs && e == cudaSuccess; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        e = cudaMemcpyAsync(idx, perm.data(), n_tr * 4, cudaMemcpyHostToDevice, st);
        for (int64_t s = 0; s < steps_per_epoch && e == cudaSuccess; ++s, ++step) {
            const float lr = (float)(d->lr * 0.5 * (1.0 + std::cos(M_PI * (double)step / (double)total)));
            k_sur_train<<<nblk, kTB, kTrainSmem, st>>>(S->params, X, Y, idx + s * bs, bs, n_out, part, lpart);
            const float b1t = (float)std::pow(0.9, (double)(step + 1)), b2t = (float)std::pow(0.999, (double)(step + 1));
            k_sur_adam<<<(kNP + 255) / 256, 256, 0, st>>>(S->params, m, v, part, nblk,
                                                          1.0f / ((float)bs * n_out), lr, b1t, b2t);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);  // one host sync per epoch (shuffle buffer reuse)
    }
    if (e != cudaSuccess)
        return bail(HH_ECUDA, "surrogate training");
    // loss on the training tail and on the held-out windows (mean squared scaled error)
    auto eval = [&](int64_t first, int64_t count) -> double {
        std::vector<int32_t> ix(count);
        for (int64_t k = 0; k < count; ++k)
            ix[k] = (int32_t)(first + k);
        double tot = 0.0;
        for (int64_t off = 0; off + kTB <= count && e == cudaSuccess; off += (int64_t)nblk * kTB) {
            const int64_t rows = std::min<int64_t>((int64_t)nblk * kTB, count - off) / kTB * kTB;
            e = cudaMemcpyAsync(idx, ix.data() + off, rows * 4, cudaMemcpyHostToDevice, st);
            k_sur_train<<<(int)(rows / kTB), kTB, kTrainSmem, st>>>(S->params, X, Y, idx, rows, n_out, part, lpart);
            std::vector<float> lp(rows / kTB);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(lp.data(), lpart, lp.size() * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(st);
            for (float x : lp)
                tot += x;
        }
        return tot / ((double)(count / kTB * kTB) * n_out);
    };
    const double train_loss = eval(0, std::min<int64_t>(n_tr, 65536));
    const double val_loss = eval(n_tr, n_val);
    // bf16 weights and fp32 biases for inference
    if (e == cudaSuccess) {
        k_to_bf16<<<(kSH * kRow + 255) / 256, 256, 0, st>>>(S->params + oW1, kSH * kRow, S->wb);
        k_to_bf16<<<(kSH * kRow + 255) / 256, 256, 0, st>>>(S->params + oW2, kSH * kRow, S->wb + kSH * kRow);
        k_to_bf16<<<(kSO * kRow + 255) / 256, 256, 0, st>>>(S->params + oW3, kSO * kRow, S->wb + 2 * kSH * kRow);
        e = cudaMemcpyAsync(S->bias, S->params + ob1, kSH * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->bias + kSH, S->params + ob2, kSH * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(S->bias + 2 * kSH, S->params + ob3, kSO * 4, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess)
        return bail(HH_ECUDA, "surrogate finalisation");
    if (rep) {
        rep->train_windows = n;
        rep->train_loss = (float)train_loss;
        rep->val_loss = (float)val_loss;
        rep->out_scale_V = nm.out_scale[0];
    }
    *out = S;
    return HH_OK;
}

cudaError_t surrogate_window(const DevModels& Ms, Surrogate* S, const NeuronParams& P, int precision,
                             cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_sur_infer<HH_PREC_FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInferSmem);
        cudaFuncSetAttribute(k_sur_infer<HH_PREC_ACCURATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kInferSmem);
        attr = true;
    }
    InferParams q{};
    q.W1 = S->wb;
    q.W2 = S->wb + kSH * kRow;
    q.W3 = S->wb + 2 * kSH * kRow;
    q.b = S->bias;
    q.fb_list = S->fb_list;
    q.fb_count = S->fb_count;
    q.stats = S->stats;
    q.err = S->err;
    q.W = S->W;
    q.err_V = S->err_V;
    q.err_p = S->err_p;
    cudaError_t e = cudaMemsetAsync(S->fb_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess)
        return e;
    const int64_t n_tiles = (P.N + 127) / 128;
    const unsigned grid = (unsigned)std::min<int64_t>(n_tiles, (int64_t)152 * kInferCtasPerSm);
    if (precision == HH_PREC_FAST)
        k_sur_infer<HH_PREC_FAST><<<grid, 128, kInferSmem, st>>>(Ms, S->coarse, S->norm, P, q);
    else
        k_sur_infer<HH_PREC_ACCURATE><<<grid, 128, kInferSmem, st>>>(Ms, S->coarse, S->norm, P, q);
    return cudaGetLastError();
}

int surrogate_window_steps(const Surrogate* S) { return S->W; }
const int32_t* surrogate_fb_list(const Surrogate* S) { return S->fb_list; }
const int32_t* surrogate_fb_count(const Surrogate* S) { return S->fb_count; }
cudaError_t surrogate_stats(const Surrogate* S, unsigned long long* host2, int32_t* err)
{
    cudaError_t e = cudaMemcpy(host2, S->stats, 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(err, S->err, 4, cudaMemcpyDeviceToHost);
    return e;
}
cudaError_t surrogate_reset_stats(Surrogate* S, cudaStream_t st)
{
    return cudaMemsetAsync(S->stats, 0, 16, st);
}

}  // namespace hh
