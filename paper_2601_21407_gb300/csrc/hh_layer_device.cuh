// Device code of the differentiable recurrent HH layer, shared by the
// kernels compiled into libhh.so (the model table read at run time,
// hh_layer.cu) and the per-model kernels compiled at run time with NVRTC
// (hh_jit.cu embeds this file verbatim after hh_device.cuh).  It includes
// nothing.
//
// Forward over T outer steps of K exponential-Euler substeps with I_t held,
// spikes S_t = sum_k H(V_k - theta)(1 - H(V_{k-1} - theta)) (or the smooth
// step), checkpoints of the state every `ckpt` outer steps; the backward
// recomputes each segment from its checkpoint and sweeps every substep in
// reverse with the hand-derived adjoint (Methods, "Gradient learning
// support" and "Engineering optimization": manually derived gradients,
// re-computation), the surrogate 1/(1 + beta|x|)^2 standing in for dH/dx.
#pragma once

namespace hh {

constexpr int kMaxSub = 16;  // substeps per outer step, at most

__device__ __forceinline__ float sur_d(float x, float beta)
{
    const float d = 1.0f + beta * fabsf(x);
    return 1.0f / (d * d);
}
__device__ __forceinline__ float smooth_s(float x, float beta)
{
    return 0.5f + 0.5f * beta * x / (1.0f + beta * fabsf(x));
}
__device__ __forceinline__ float smooth_d(float x, float beta)
{
    const float d = 1.0f + beta * fabsf(x);
    return 0.5f * beta / (d * d);
}

// 1 - e^{-y} for either sign of y on the SFU path: the Taylor polynomial of
// -expm1(-y) up to y^5 for |y| < 0.125 (truncation < 4.3e-8 relative),
// 1 - 2^{-y log2 e} beyond (no cancellation there).
__device__ __forceinline__ float em1_signed(float y)
{
    const float y2 = y * y;
    const float c = fmaf(y2, fmaf(y2, 1.0f / 120.0f, fmaf(y, -1.0f / 24.0f, 1.0f / 6.0f)), fmaf(y, -0.5f, 1.0f));
    const float far = 1.0f - ex2a(-y * kLog2e);
    return fabsf(y) < 0.125f ? y * c : far;
}

// Value (with the offset c) and derivative d/dV of a rate form.  FAST: the
// SFU exponential and reciprocal; otherwise IEEE FP32 (expf, expm1f,
// division).
template <bool FAST>
__device__ __forceinline__ void rate_vd(const DevFn& f, float V, float& r, float& dr)
{
    using M = Mth<FAST>;
    switch (f.form) {
    case HH_FN_CONST:
        r = f.a;
        dr = 0.0f;
        break;
    case HH_FN_EXP: {
        const float e = M::expv(f, V);
        r = f.a * e;
        dr = r * f.ik;
        break;
    }
    case HH_FN_SIGMOID: {
        const float e = M::expv(f, V);
        const float q = M::div(1.0f, 1.0f + e);
        r = f.a * q;
        dr = -f.a * e * q * q * f.ik;
        break;
    }
    case HH_FN_LINOID: {
        // a k g(y), g(y) = y / (1 - e^{-y}), y = (V - vh)/k; dr = a g'(y)
        const float y = (V - f.vh) * f.ik;
        if (fabsf(y) < 1e-3f) {
            r = f.a * f.k * (1.0f + 0.5f * y + y * y * (1.0f / 12.0f));
            dr = f.a * (0.5f + y * (1.0f / 6.0f));
        } else {
            const float em = FAST ? em1_signed(y) : -expm1f(-y);  // 1 - e^{-y}
            const float ie = M::div(1.0f, em);
            r = f.a * f.k * (y * ie);
            dr = f.a * (em - y * (1.0f - em)) * (ie * ie);
        }
        break;
    }
    default: {  // bell
        const float e1 = M::expv(f, V), e2 = M::expv2(f, V);
        const float id = M::div(1.0f, e1 + e2);
        r = f.a * id;
        dr = -f.a * (e1 * f.ik + e2 * f.ik2) * (id * id);
        break;
    }
    }
    r += f.c;
}

// Reverse of one substep (state V, p before it, current I): on entry lamV,
// lamP hold the adjoints of the state after the substep; on exit those of
// the state before it; lamI accumulates dL/dI.  FAST: SFU exponentials,
// reciprocals and 1 - e^{-z}, as in the forward substep of that precision.
template <int MAXG, bool FAST>
__device__ __forceinline__ void substep_adjoint(const DevModel& M, const State<MAXG, 1>& s0, float dt, float I,
                                                float& lamV, float* lamP, float& lamI)
{
    using Mt = Mth<FAST>;
    const float V = s0.V;
    float pn[MAXG], Eq[MAXG], dpdV[MAXG];
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        pn[q] = 0.0f;
        Eq[q] = 0.0f;
        dpdV[q] = 0.0f;
        if (q < M.n_gates) {
            const DevGate& g = M.g[q];
            const float p = s0.p[q];
            float inf, dinf, z, dz;
            if (g.kind == HH_GATE_AB) {
                float al, dal, be, dbe;
                rate_vd<FAST>(g.f1, V, al, dal);
                rate_vd<FAST>(g.f2, V, be, dbe);
                const float sum = al + be;
                const float is = Mt::div(1.0f, sum);
                inf = al * is;
                dinf = (dal * be - al * dbe) * (is * is);
                z = dt * sum;
                dz = dt * (dal + dbe);
            } else {
                float tau, dtau;
                rate_vd<FAST>(g.f1, V, inf, dinf);
                rate_vd<FAST>(g.f2, V, tau, dtau);
                const float it = Mt::div(1.0f, tau);
                z = dt * it;
                dz = -dt * dtau * (it * it);
            }
            const float E = em1<FAST>(z);
            Eq[q] = E;
            pn[q] = p + (inf - p) * E;
            dpdV[q] = E * dinf + (inf - p) * (1.0f - E) * dz;
        }
    }
    float G = s0.gconst, Ip = s0.gconst * V - s0.gconstE;
    {
        float eta = 1.0f;
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            if (q < M.n_gates) {
                eta *= powi(pn[q], M.g[q].power);
                if (M.gate_last[q]) {
                    const float gx = s0.gq[q] * eta;
                    G += gx;
                    Ip += gx * (V - M.gate_E[q]);
                    eta = 1.0f;
                }
            }
    }
    const float EV = em1<FAST>(dt * G * M.inv_C);
    const float iG = Mt::div(1.0f, G);
    const float A = (I - Ip) * iG;
    lamI += lamV * EV * iG;
    float lamVpre = lamV * (1.0f - EV);
    float lamPn[MAXG];
#pragma unroll
    for (int q = 0; q < MAXG; ++q)
        lamPn[q] = lamP[q];
    // conductance paths: dV'/dg_c = -EV ((V - E_c) + A)/G + A (1 - EV) dt/C
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        if (q < M.n_gates && M.gate_last[q]) {
            const int c = M.gate_ch[q];
            const int f = M.ch_first[c], ng = M.ch_ng[c];
            const float dVdg = -EV * ((V - M.gate_E[q]) + A) * iG + A * (1.0f - EV) * dt * M.inv_C;
            const float lg = lamV * dVdg * s0.gq[q];
#pragma unroll
            for (int r = 0; r < MAXG; ++r) {
                if (r >= f && r < f + ng) {
                    float d = (float)M.g[r].power * powi(pn[r], M.g[r].power - 1 > 0 ? M.g[r].power - 1 : 1);
                    if (M.g[r].power == 1)
                        d = 1.0f;
#pragma unroll
                    for (int u = 0; u < MAXG; ++u)
                        if (u >= f && u < f + ng && u != r)
                            d *= powi(pn[u], M.g[u].power);
                    lamPn[r] += lg * d;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        if (q < M.n_gates) {
            lamVpre += lamPn[q] * dpdV[q];
            lamP[q] = lamPn[q] * (1.0f - Eq[q]);
        }
    }
    lamV = lamVpre;
}

struct LayerParams {
    int64_t BN;          // B * N
    int32_t B, N, T, K, ckpt;
    float dt, theta, beta;
    int32_t v_update, smooth;
    const float* bias;   // [N]
    const float* XW;     // [T*B][N]
    const float* recp;   // [splits][B][N] or null
    int32_t rec_splits;
    float* I_all;        // [T][B][N]
    float* V;            // [B*N]
    float* P;            // [kMaxGates][B*N]
    float* ckptV;        // [n_ckpt][B*N]
    float* ckptP;        // [n_ckpt][kMaxGates][B*N]
    uint16_t* S;         // bf16 [(T+1)*B][N]; rows [0,B) zero
    float* Sf;           // fp32 [T][B*N] spikes (for readout / records)
    float* acc;          // [B*N]
    float* segV;         // [ckpt][B*N]
    float* segP;         // [ckpt][kMaxGates][B*N]
    float* lamV;         // [B*N]
    float* lamP;         // [kMaxGates][B*N]
    const float* ds_direct;  // [B*N]
    const float* dS_ext; // [T][B*N] caller's dL/dS_t, or null
    const float* dsp;    // [splits][B*N] partials of dI_{t+1} W_rec^T
    int32_t ds_splits;
    float* dI_all;       // [T][B*N]
    uint16_t* dIb;       // bf16 [B][2N]  (hi | lo) of dI_t
};

__device__ __forceinline__ uint16_t f2bf(float x)
{
    const uint32_t u = __float_as_uint(x);
    const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(r >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

template <int MAXG, int PREC>
__device__ __forceinline__ void layer_load(const DevModel& M, const LayerParams& L, const float* V, const float* P,
                                           int64_t i, State<MAXG, PREC>& s)
{
    s.poly = nullptr;
    s.V = V[i];
    s.Vlo = 0.0f;
    s.Ca = 0.0f;
#pragma unroll
    for (int q = 0; q < MAXG; ++q) {
        s.p[q] = P[(int64_t)q * L.BN + i];
        s.plo[q] = 0.0f;
    }
    load_conductances(M, nullptr, L.BN, i, s);
}

template <int MAXG, int PREC>
__device__ __forceinline__ void layer_fwd_body(const DevModel& M, const LayerParams& L, int t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.BN)
        return;
    const int n = (int)(i % L.N), b = (int)(i / L.N);
    float I = L.bias[n] + L.XW[((int64_t)t * L.B + b) * L.N + n];
    if (L.recp)
        for (int s = 0; s < L.rec_splits; ++s)
            I += L.recp[(int64_t)s * L.BN + i];
    L.I_all[(int64_t)t * L.BN + i] = I;
    State<MAXG, PREC> st;
    layer_load(M, L, L.V, L.P, i, st);
    float spk = 0.0f;
    for (int k = 0; k < L.K; ++k) {
        const float Vp = st.V;
        neuron_step<MAXG, PREC>(M, L.dt, L.v_update, I, 0.0f, 0.0f, 0.0f, 0.0f, st);
        if (L.smooth)
            spk += smooth_s(st.V - L.theta, L.beta) * (1.0f - smooth_s(Vp - L.theta, L.beta));
        else
            spk += (st.V >= L.theta && !(Vp >= L.theta)) ? 1.0f : 0.0f;
    }
    L.V[i] = st.V;
#pragma unroll
    for (int q = 0; q < MAXG; ++q)
        L.P[(int64_t)q * L.BN + i] = st.p[q];
    L.S[(int64_t)(t + 1) * L.BN + i] = f2bf(spk);
    L.Sf[(int64_t)t * L.BN + i] = spk;
    L.acc[i] += spk;
    if ((t + 1) % L.ckpt == 0) {
        const int c = (t + 1) / L.ckpt;
        L.ckptV[(int64_t)c * L.BN + i] = st.V;
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            L.ckptP[((int64_t)c * kMaxGates + q) * L.BN + i] = st.p[q];
    }
}

// Recompute the states at the start of every outer step of segment g.
template <int MAXG, int PREC>
__device__ __forceinline__ void layer_recompute_body(const DevModel& M, const LayerParams& L, int g)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.BN)
        return;
    State<MAXG, PREC> st;
    layer_load(M, L, L.ckptV + (int64_t)g * L.BN, L.ckptP + (int64_t)g * kMaxGates * L.BN, i, st);
    const int t0 = g * L.ckpt, t1 = min(L.T, t0 + L.ckpt);
    for (int t = t0; t < t1; ++t) {
        const int j = t - t0;
        L.segV[(int64_t)j * L.BN + i] = st.V;
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            L.segP[((int64_t)j * kMaxGates + q) * L.BN + i] = st.p[q];
        const float I = L.I_all[(int64_t)t * L.BN + i];
        for (int k = 0; k < L.K; ++k)
            neuron_step<MAXG, PREC>(M, L.dt, L.v_update, I, 0.0f, 0.0f, 0.0f, 0.0f, st);
    }
}

// Reverse of outer step t: recompute its K substeps from the segment state,
// then sweep them backwards.
extern __shared__ float layer_smem[];

// Dynamic shared memory of the adjoint kernel: K + 1 voltages and K x MAXG
// gate values per thread.
__host__ __device__ constexpr int layer_bwd_smem(int K, int maxg, int threads)
{
    return (K + 1 + K * maxg) * threads * 4;
}

template <int MAXG, int PREC>
__device__ __forceinline__ void layer_bwd_body(const DevModel& M, const LayerParams& L, int t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.BN)
        return;
    const int j = t % L.ckpt;
    State<MAXG, PREC> st;
    layer_load(M, L, L.segV + (int64_t)j * L.BN, L.segP + (int64_t)j * kMaxGates * L.BN, i, st);
    const float I = L.I_all[(int64_t)t * L.BN + i];
    // states before each substep (V_0..V_{K-1}) and V_K, in shared memory
    // (layer_bwd_smem bytes per block; thread-minor, so the accesses of a
    // warp fall in distinct banks)
    const int nt = (int)blockDim.x, tid = (int)threadIdx.x;
    float* Vs = layer_smem;                          // [K + 1][nt]
    float* Ps = layer_smem + (L.K + 1) * nt;          // [K][MAXG][nt]
    for (int k = 0; k < L.K; ++k) {
        Vs[k * nt + tid] = st.V;
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            Ps[(k * MAXG + q) * nt + tid] = st.p[q];
        neuron_step<MAXG, PREC>(M, L.dt, L.v_update, I, 0.0f, 0.0f, 0.0f, 0.0f, st);
    }
    Vs[L.K * nt + tid] = st.V;
    float ds = L.ds_direct[i];
    if (L.dS_ext)
        ds += L.dS_ext[(int64_t)t * L.BN + i];
    if (L.dsp)
        for (int s = 0; s < L.ds_splits; ++s)
            ds += L.dsp[(int64_t)s * L.BN + i];
    float lamV = L.lamV[i];
    float lamP[MAXG];
#pragma unroll
    for (int q = 0; q < MAXG; ++q)
        lamP[q] = L.lamP[(int64_t)q * L.BN + i];
    float lamI = 0.0f;
    State<MAXG, 1> s0;
    s0.Ca = 0.0f;
    s0.Vlo = 0.0f;
    load_conductances(M, nullptr, L.BN, i, s0);
    for (int k = L.K; k >= 1; --k) {
        const float Vk = Vs[k * nt + tid], Vp = Vs[(k - 1) * nt + tid];
        // spike c_k depends on V_k (and on V_{k-1})
        if (L.smooth)
            lamV += ds * smooth_d(Vk - L.theta, L.beta) * (1.0f - smooth_s(Vp - L.theta, L.beta));
        else if (!(Vp >= L.theta))
            lamV += ds * sur_d(Vk - L.theta, L.beta);
        s0.V = Vp;
#pragma unroll
        for (int q = 0; q < MAXG; ++q)
            s0.p[q] = Ps[((k - 1) * MAXG + q) * nt + tid];
        substep_adjoint<MAXG, PREC == HH_PREC_FAST>(M, s0, L.dt, I, lamV, lamP, lamI);
        if (L.smooth)
            lamV -= ds * smooth_s(Vk - L.theta, L.beta) * smooth_d(Vp - L.theta, L.beta);
    }
    L.lamV[i] = lamV;
#pragma unroll
    for (int q = 0; q < MAXG; ++q)
        L.lamP[(int64_t)q * L.BN + i] = lamP[q];
    L.dI_all[(int64_t)t * L.BN + i] = lamI;
    const int n = (int)(i % L.N), b = (int)(i / L.N);
    const uint16_t hi = f2bf(lamI);
    L.dIb[(int64_t)b * 2 * L.N + n] = hi;
    L.dIb[(int64_t)b * 2 * L.N + L.N + n] = f2bf(lamI - bf2f(hi));
}

}  // namespace hh
