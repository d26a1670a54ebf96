// Differentiable recurrent HH layer: forward over T outer steps of K
// exponential-Euler substeps, and a hand-derived BPTT adjoint with
// recomputation from checkpoints (Methods, "Gradient learning support" and
// "Engineering optimization": manually derived gradients, re-computation).
//
//   I_t = bias + X_t W_in + S_{t-1} W_rec           (tcgen05 GEMMs, bf16 in, fp32 acc)
//   K substeps of the neuron update with I_t held; S_t = sum_k c_{t,k},
//   c_{t,k} = H(V_k - theta)(1 - H(V_{k-1} - theta))   (or the smooth step)
//   r = (1/T) sum_t S_t,  logits = r W_out^T,  loss = mean_b CE(logits_b, y_b)
// Backward, for L = w CE + <dL/dlogits, logits> + <dL/dS, S> + <dL/dV, V_T>:
// dlogits = w (softmax - onehot)/B + dL/dlogits; dS_t = dr/T + dL/dS_t +
// dI_{t+1} W_rec^T; lambda_V starts at dL/dV_T;
// through each substep in reverse with the surrogate 1/(1 + beta|x|)^2 for
// dH/dx; dW_in = X^T dI, dW_rec = S_prev^T dI, dbias = sum dI (GEMMs over the
// T*B rows, dI split into bf16 hi + lo parts so the products keep ~16 bits).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "hh_internal.h"
#include "hh_layer_device.cuh"

namespace hh {
namespace {

// logits, loss (mean CE) and dlogits; one block per sample.
__global__ void k_layer_readout(const float* __restrict__ acc, const float* __restrict__ W_out,
                                const int32_t* __restrict__ labels, int N, int n_out, float inv_T, int B,
                                float* logits, float* loss_b, float* dlogits)
{
    extern __shared__ float sh[];  // n_out
    const int b = blockIdx.x;
    for (int o = threadIdx.x >> 5; o < n_out; o += blockDim.x >> 5) {
        float s = 0.0f;
        for (int n = threadIdx.x & 31; n < N; n += 32)
            s += acc[(int64_t)b * N + n] * inv_T * W_out[(int64_t)o * N + n];
        for (int off = 16; off; off >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0)
            sh[o] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0 && !labels) {
        // no built-in loss: logits only, no cross-entropy gradient
        for (int o = 0; o < n_out; ++o) {
            if (logits)
                logits[(int64_t)b * n_out + o] = sh[o];
            dlogits[(int64_t)b * n_out + o] = 0.0f;
        }
        return;
    }
    if (threadIdx.x == 0) {
        float mx = -INFINITY;
        for (int o = 0; o < n_out; ++o)
            mx = fmaxf(mx, sh[o]);
        double z = 0.0;
        for (int o = 0; o < n_out; ++o)
            z += exp((double)(sh[o] - mx));
        const int y = labels[b];
        loss_b[b] = (float)(log(z) - (double)(sh[y] - mx));
        for (int o = 0; o < n_out; ++o) {
            if (logits)
                logits[(int64_t)b * n_out + o] = sh[o];
            const float p = (float)(exp((double)(sh[o] - mx)) / z);
            dlogits[(int64_t)b * n_out + o] = (p - (o == y ? 1.0f : 0.0f)) / (float)B;
        }
    }
}

__global__ void k_layer_loss(const float* __restrict__ loss_b, int B, float* loss)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < B; ++b)
            s += loss_b[b];
        *loss = (float)(s / B);
    }
}

// dW_out[o][n] = sum_b dlogits[b][o] r[b][n];  ds_direct[b][n] = (1/T) sum_o dlogits[b][o] W_out[o][n]
__global__ void k_layer_bwd_readout(const float* __restrict__ acc, const float* __restrict__ W_out,
                                    const float* __restrict__ dlogits, int B, int N, int n_out, float inv_T,
                                    float* dW_out, float* ds_direct)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (dW_out && i < (int64_t)n_out * N) {
        const int o = (int)(i / N), n = (int)(i % N);
        float s = 0.0f;
        for (int b = 0; b < B; ++b)
            s += dlogits[(int64_t)b * n_out + o] * acc[(int64_t)b * N + n] * inv_T;
        dW_out[i] = s;
    }
    if (i < (int64_t)B * N) {
        const int b = (int)(i / N), n = (int)(i % N);
        float s = 0.0f;
        for (int o = 0; o < n_out; ++o)
            s += dlogits[(int64_t)b * n_out + o] * W_out[(int64_t)o * N + n];
        ds_direct[i] = s * inv_T;
    }
}

// X (fp32 0/1, [rows][n_in]) -> bf16 [rows][ld] with zero padding
__global__ void k_to_bf16_pad(const float* __restrict__ X, int64_t rows, int cols, int ld, uint16_t* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * ld)
        return;
    const int64_t r = i / ld;
    const int c = (int)(i % ld);
    out[i] = c < cols ? f2bf(X[r * cols + c]) : (uint16_t)0;
}

// out[c][r] = in[r][c] for r < rows, c < cols; out has leading dimension ldo
// (entries r >= rows of out are left untouched).  32x32 tiles via shared memory.
template <class Tin>
__global__ void k_transpose_bf16(const Tin* __restrict__ in, int64_t rows, int cols, int ldi, uint16_t* out,
                                 int64_t ldo, uint16_t* out_lo)
{
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k, c = c0 + threadIdx.x;
        float v = 0.0f;
        if (r < rows && c < cols) {
            if constexpr (sizeof(Tin) == 2)
                v = bf2f(in[r * ldi + c]);
            else
                v = in[r * ldi + c];
        }
        tile[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) {
            const float v = tile[threadIdx.x][k];
            const uint16_t hi = f2bf(v);
            out[c * ldo + r] = hi;
            if (out_lo)
                out_lo[c * ldo + r] = f2bf(v - bf2f(hi));
        }
    }
}

// dst[r][c] = sum_s part[s][c][r]  (transpose back while summing split partials)
__global__ void k_reduce_transpose(const float* __restrict__ part, int splits, int prow, int pcol, int rows,
                                   int cols, float* dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols)
        return;
    const int r = (int)(i / cols), c = (int)(i % cols);
    float s = 0.0f;
    for (int k = 0; k < splits; ++k)
        s += part[((int64_t)k * prow + c) * pcol + r];
    dst[i] = s;
}

// dbias[n] = sum_{t,b} dI[t][b][n], in two deterministic passes: chunk sums
// part[c][n] over rows [c*rows/chunks, (c+1)*rows/chunks), then their sum.
constexpr int kColChunks = 128;
__global__ void k_colsum_part(const float* __restrict__ dI, int64_t rows, int N, float* part)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (n >= N)
        return;
    const int64_t r0 = rows * c / kColChunks, r1 = rows * (c + 1) / kColChunks;
    float s = 0.0f;
    for (int64_t r = r0; r < r1; ++r)
        s += dI[r * N + n];
    part[(int64_t)c * N + n] = s;
}

__global__ void k_colsum_final(const float* __restrict__ part, int N, float* out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N)
        return;
    float s = 0.0f;
    for (int c = 0; c < kColChunks; ++c)
        s += part[(int64_t)c * N + n];
    out[n] = s;
}

// dlog[b][o] = w * ce[b][o] + (ext ? ext[b][o] : 0): the gradient reaching
// the logits from the weighted built-in loss and the caller's cotangent.
__global__ void k_combine_dlogits(const float* __restrict__ ce, float w, const float* __restrict__ ext, int n,
                                  float* dlog)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        dlog[i] = w * ce[i] + (ext ? ext[i] : 0.0f);
}

// dI [rows][N] fp32 -> out [rows][2N] bf16 (hi | lo): the A operand of
// dX = dI W_in^T with ~16 significant bits.
__global__ void k_split_rows_bf16(const float* __restrict__ dI, int64_t rows, int N, uint16_t* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * N)
        return;
    const int64_t r = i / N;
    const int n = (int)(i % N);
    const float v = dI[i];
    const uint16_t hi = f2bf(v);
    out[r * 2 * N + n] = hi;
    out[r * 2 * N + N + n] = f2bf(v - bf2f(hi));
}

// WinT [N][ld] (bf16, W_in transposed) -> W2 [c][2N] = (W_in[c][:] | W_in[c][:])
// for c < rows: the B operand of dX, matching the hi | lo split of dI.
__global__ void k_win2_from_wint(const uint16_t* __restrict__ WinT, int N, int ld, int rows, uint16_t* W2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * N)
        return;
    const int c = (int)(i / N), n = (int)(i % N);
    const uint16_t v = WinT[(int64_t)n * ld + c];
    W2[(int64_t)c * 2 * N + n] = v;
    W2[(int64_t)c * 2 * N + N + n] = v;
}

// dst [rows][cols] = src [rows][ld] (drop the padding columns)
__global__ void k_strip_cols(const float* __restrict__ src, int64_t rows, int cols, int ld, float* dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols)
        return;
    const int64_t r = i / cols;
    const int c = (int)(i % cols);
    dst[i] = src[r * ld + c];
}

__global__ void k_layer_init(const __grid_constant__ DevModels Ms, const __grid_constant__ LayerParams L, float V0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= L.BN)
        return;
    const DevModel& M = Ms.m[0];
    L.V[i] = V0;
    L.ckptV[i] = V0;
    for (int q = 0; q < kMaxGates; ++q) {
        float inf = 0.0f, z;
        if (q < M.n_gates)
            gate_inf_z<false>(M.g[q], V0, 0.0f, 1.0f, inf, z);
        L.P[(int64_t)q * L.BN + i] = inf;
        L.ckptP[(int64_t)q * L.BN + i] = inf;
    }
    L.acc[i] = 0.0f;
    L.lamV[i] = 0.0f;
    for (int q = 0; q < kMaxGates; ++q)
        L.lamP[(int64_t)q * L.BN + i] = 0.0f;
}

int grid1(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------
struct LayerImpl {
    int B, n_in, n_in_pad, N, n_out, T, K, ckpt, n_ckpt, TB, TBp;
    float dt, theta, beta, V0;
    int precision, smooth;
    cudaStream_t st;
    DevModels models{};
    // weights
    float *W_out, *bias;
    uint16_t *WinT, *WrecT, *Wrec2;   // [N][n_in_pad], [N][N], [N][2N]
    // forward
    uint16_t *Xb, *S;                 // [TB][n_in_pad], [(T+1)*B][N]
    float *XW, *recp, *I_all, *Sf, *V, *P, *ckptV, *ckptP, *acc, *dlogits, *loss_b;
    // backward
    float *segV, *segP, *lamV, *lamP, *ds_direct, *dsp, *dI_all, *wpart;
    uint16_t *dIb, *dIT_hi, *dIT_lo, *XT, *SpT;
    int32_t* status;
    int rec_splits, ds_splits, w_splits;
    bool forward_done;
    bool forward_labels;  // the last forward had labels (built-in loss available)
    float* dlog_tot;      // [B][n_out] gradient reaching the logits
    // dX = dI W_in^T operands, allocated at the first request of dX
    uint16_t *dIrow, *Win2;  // [TB][2N], [n_in_pad][2N]
    float* dXpart;           // [TB][n_in_pad]
    bool win2_valid;
    LayerKernels jit;  // fwd / recompute / bwd compiled for the layer's model
    size_t bwd_smem;   // dynamic shared memory of the adjoint kernel
};

LayerParams layer_params(const LayerImpl& L)
{
    LayerParams p{};
    p.BN = (int64_t)L.B * L.N;
    p.B = L.B;
    p.N = L.N;
    p.T = L.T;
    p.K = L.K;
    p.ckpt = L.ckpt;
    p.dt = L.dt;
    p.theta = L.theta;
    p.beta = L.beta;
    p.v_update = HH_V_EXP_EULER;
    p.smooth = L.smooth;
    p.bias = L.bias;
    p.XW = L.XW;
    p.recp = nullptr;
    p.rec_splits = L.rec_splits;
    p.I_all = L.I_all;
    p.V = L.V;
    p.P = L.P;
    p.ckptV = L.ckptV;
    p.ckptP = L.ckptP;
    p.S = L.S;
    p.Sf = L.Sf;
    p.acc = L.acc;
    p.segV = L.segV;
    p.segP = L.segP;
    p.lamV = L.lamV;
    p.lamP = L.lamP;
    p.ds_direct = L.ds_direct;
    p.dS_ext = nullptr;
    p.dsp = nullptr;
    p.ds_splits = L.ds_splits;
    p.dI_all = L.dI_all;
    p.dIb = L.dIb;
    return p;
}

cudaError_t layer_forward(LayerImpl& L, const float* X, const int32_t* labels, float* loss, float* logits)
{
    cudaStream_t st = L.st;
    cudaError_t e;
    LayerParams p = layer_params(L);
    const int64_t BN = p.BN;
    // inputs -> bf16, input projection for all steps at once
    k_to_bf16_pad<<<grid1((int64_t)L.TB * L.n_in_pad, 256), 256, 0, st>>>(X, L.TB, L.n_in, L.n_in_pad, L.Xb);
    GemmArgs gx{L.Xb, L.TB, L.n_in_pad, 0, L.WinT, L.N, L.n_in_pad, 0, L.XW, L.TB, L.N, L.n_in_pad, 1};
    if ((e = launch_gemm_bf16(gx, L.status, st)) != cudaSuccess)
        return e;
    k_layer_init<<<grid1(BN, 256), 256, 0, st>>>(L.models, p, L.V0);
    if ((e = cudaMemsetAsync(L.S, 0, (size_t)L.B * L.N * 2, st)) != cudaSuccess)
        return e;
    for (int t = 0; t < L.T; ++t) {
        LayerParams pt = p;
        if (t > 0) {
            // recurrent projection S_{t-1} W_rec (S rows [t*B, (t+1)*B))
            GemmArgs gr{L.S, (L.T + 1) * L.B, L.N, t * L.B, L.WrecT, L.N, L.N, 0, L.recp, L.B, L.N, L.N,
                        L.rec_splits};
            if ((e = launch_gemm_bf16(gr, L.status, st)) != cudaSuccess)
                return e;
            pt.recp = L.recp;
        }
        if ((e = jit_launch_layer(L.jit.fwd, pt, t, BN, 0, st)) != cudaSuccess)
            return e;
    }
    k_layer_readout<<<L.B, 256, L.n_out * sizeof(float), st>>>(L.acc, L.W_out, labels, L.N, L.n_out,
                                                               1.0f / L.T, L.B, logits, L.loss_b, L.dlogits);
    if (labels)
        k_layer_loss<<<1, 32, 0, st>>>(L.loss_b, L.B, loss);
    L.forward_done = true;
    L.forward_labels = labels != nullptr;
    return cudaGetLastError();
}

// The loss is ce_weight * CE + <dL_dlogits, logits> + <dL_dS, S> + <dL_dV, V_T>
// (any cotangent may be null); every non-null gradient of g is filled.
cudaError_t layer_backward(LayerImpl& L, float ce_weight, const float* dL_dlogits, const float* dL_dS,
                           const float* dL_dV, const hh_grads& g)
{
    cudaStream_t st = L.st;
    cudaError_t e;
    LayerParams p = layer_params(L);
    p.dS_ext = dL_dS;
    const int64_t BN = p.BN;
    const int nlog = L.B * L.n_out;
    k_combine_dlogits<<<grid1(nlog, 256), 256, 0, st>>>(L.dlogits, ce_weight, dL_dlogits, nlog, L.dlog_tot);
    k_layer_bwd_readout<<<grid1(std::max<int64_t>(BN, (int64_t)L.n_out * L.N), 256), 256, 0, st>>>(
        L.acc, L.W_out, L.dlog_tot, L.B, L.N, L.n_out, 1.0f / L.T, g.dW_out, L.ds_direct);
    if (dL_dV)
        e = cudaMemcpyAsync(L.lamV, dL_dV, BN * sizeof(float), cudaMemcpyDeviceToDevice, st);
    else
        e = cudaMemsetAsync(L.lamV, 0, BN * sizeof(float), st);
    if (e != cudaSuccess || (e = cudaMemsetAsync(L.lamP, 0, BN * kMaxGates * sizeof(float), st)) != cudaSuccess)
        return e;
    for (int g = L.n_ckpt - 1; g >= 0; --g) {
        const int t0 = g * L.ckpt;
        if (t0 >= L.T)
            continue;
        if ((e = jit_launch_layer(L.jit.recompute, p, g, BN, 0, st)) != cudaSuccess)
            return e;
        const int t1 = std::min(L.T, t0 + L.ckpt);
        for (int t = t1 - 1; t >= t0; --t) {
            LayerParams pt = p;
            pt.dsp = (t < L.T - 1) ? L.dsp : nullptr;
            if ((e = jit_launch_layer(L.jit.bwd, pt, t, BN, L.bwd_smem, st)) != cudaSuccess)
                return e;
            if (t > 0) {
                // dS_{t-1} = dI_t W_rec^T with dI_t = hi + lo (K = 2N)
                GemmArgs gd{L.dIb, L.B, 2 * L.N, 0, L.Wrec2, L.N, 2 * L.N, 0, L.dsp, L.B, L.N, 2 * L.N,
                            L.ds_splits};
                if ((e = launch_gemm_bf16(gd, L.status, st)) != cudaSuccess)
                    return e;
            }
        }
    }
    // weight gradients over the T*B rows
    dim3 blk(32, 8);
    dim3 g1((L.N + 31) / 32, (L.TB + 31) / 32);
    if (g.dW_in || g.dW_rec)
        k_transpose_bf16<float><<<g1, blk, 0, st>>>(L.dI_all, L.TB, L.N, L.N, L.dIT_hi, L.TBp, L.dIT_lo);
    const int s = L.w_splits;
    if (g.dW_in) {
        dim3 g2((L.n_in_pad + 31) / 32, (L.TB + 31) / 32);
        k_transpose_bf16<uint16_t><<<g2, blk, 0, st>>>(L.Xb, L.TB, L.n_in_pad, L.n_in_pad, L.XT, L.TBp, nullptr);
        const int64_t pin = (int64_t)L.N * L.n_in_pad;
        GemmArgs a1{L.dIT_hi, L.N, L.TBp, 0, L.XT, L.n_in_pad, L.TBp, 0, L.wpart, L.N, L.n_in_pad, L.TBp, s};
        GemmArgs a2 = a1;
        a2.A = L.dIT_lo;
        a2.C = L.wpart + s * pin;
        if ((e = launch_gemm_bf16(a1, L.status, st)) != cudaSuccess ||
            (e = launch_gemm_bf16(a2, L.status, st)) != cudaSuccess)
            return e;
        k_reduce_transpose<<<grid1((int64_t)L.n_in * L.N, 256), 256, 0, st>>>(L.wpart, 2 * s, L.N, L.n_in_pad,
                                                                              L.n_in, L.N, g.dW_in);
    }
    if (g.dW_rec) {
        k_transpose_bf16<uint16_t><<<g1, blk, 0, st>>>(L.S, L.TB, L.N, L.N, L.SpT, L.TBp, nullptr);
        const int64_t prc = (int64_t)L.N * L.N;
        GemmArgs b1{L.dIT_hi, L.N, L.TBp, 0, L.SpT, L.N, L.TBp, 0, L.wpart, L.N, L.N, L.TBp, s};
        GemmArgs b2 = b1;
        b2.A = L.dIT_lo;
        b2.C = L.wpart + s * prc;
        if ((e = launch_gemm_bf16(b1, L.status, st)) != cudaSuccess ||
            (e = launch_gemm_bf16(b2, L.status, st)) != cudaSuccess)
            return e;
        k_reduce_transpose<<<grid1(prc, 256), 256, 0, st>>>(L.wpart, 2 * s, L.N, L.N, L.N, L.N, g.dW_rec);
    }
    if (g.dbias) {
        k_colsum_part<<<dim3(grid1(L.N, 128), kColChunks), 128, 0, st>>>(L.dI_all, L.TB, L.N, L.wpart);
        k_colsum_final<<<grid1(L.N, 128), 128, 0, st>>>(L.wpart, L.N, g.dbias);
    }
    if (g.dI && (e = cudaMemcpyAsync(g.dI, L.dI_all, (size_t)L.TB * L.N * sizeof(float), cudaMemcpyDeviceToDevice,
                                     st)) != cudaSuccess)
        return e;
    if (g.dX) {
        // dX [TB][n_in] = dI [TB][N] W_in^T on the tensor cores, dI as bf16
        // hi | lo (K = 2N) against W_in duplicated (exact: W_in is bf16)
        if (!L.win2_valid) {
            k_win2_from_wint<<<grid1((int64_t)L.n_in_pad * L.N, 256), 256, 0, st>>>(L.WinT, L.N, L.n_in_pad,
                                                                                   L.n_in_pad, L.Win2);
            L.win2_valid = true;
        }
        k_split_rows_bf16<<<grid1((int64_t)L.TB * L.N, 256), 256, 0, st>>>(L.dI_all, L.TB, L.N, L.dIrow);
        GemmArgs gx{L.dIrow, L.TB, 2 * L.N, 0, L.Win2, L.n_in_pad, 2 * L.N, 0, L.dXpart, L.TB, L.n_in_pad,
                    2 * L.N, 1};
        if ((e = launch_gemm_bf16(gx, L.status, st)) != cudaSuccess)
            return e;
        k_strip_cols<<<grid1((int64_t)L.TB * L.n_in, 256), 256, 0, st>>>(L.dXpart, L.TB, L.n_in, L.n_in_pad,
                                                                         g.dX);
    }
    return cudaGetLastError();
}

}  // namespace hh

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

__global__ void k_dup_bf16(const float* __restrict__ W, int64_t rows, int cols, uint16_t* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols)
        return;
    const int64_t r = i / cols;
    const int c = (int)(i % cols);
    const uint16_t v = hh::f2bf(W[i]);
    out[r * 2 * cols + c] = v;
    out[r * 2 * cols + cols + c] = v;
}

#define HH_LCUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return hh::fail(e_ == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA, "%s: %s", \
                            #call, cudaGetErrorString(e_));                                  \
    } while (0)

}  // namespace

struct hh_layer {
    hh::LayerImpl L{};
    std::vector<void*> allocs;
    template <class T>
    cudaError_t alloc(T** p, size_t n)
    {
        *p = nullptr;
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
        if (e == cudaSuccess) {
            allocs.push_back(*p);
            e = cudaMemset(*p, 0, (n ? n : 1) * sizeof(T));
        }
        return e;
    }
    void release()
    {
        cudaStreamSynchronize(L.st);
        for (void* p : allocs)
            cudaFree(p);
        allocs.clear();
    }
};

extern "C" {

hh_status hh_layer_create(const hh_layer_desc* d, const hh_model_desc* model, hh_layer** out)
{
    if (!out)
        return hh::fail(HH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d || !model)
        return hh::fail(HH_EINVAL, "descriptor and model must not be NULL");
    if (d->batch < 1 || d->n_in < 1 || d->n_out < 1 || d->n_steps < 1)
        return hh::fail(HH_EINVAL, "batch, n_in, n_out and n_steps must be >= 1");
    if (d->n_hidden < 32 || d->n_hidden % 32 != 0)
        return hh::fail(HH_EINVAL, "n_hidden must be a positive multiple of 32 (tensor-core tiles)");
    if (d->substeps < 1 || d->substeps > 16)
        return hh::fail(HH_EINVAL, "substeps must be in 1..16");
    if (d->checkpoint_every < 1)
        return hh::fail(HH_EINVAL, "checkpoint_every must be >= 1");
    if (!(d->dt_ms > 0.0) || !(d->surrogate_beta > 0.0f))
        return hh::fail(HH_EINVAL, "dt_ms and surrogate_beta must be > 0");
    if (d->precision != HH_PREC_FAST && d->precision != HH_PREC_ACCURATE)
        return hh::fail(HH_EUNSUPPORTED, "the layer supports HH_PREC_FAST and HH_PREC_ACCURATE");
    if ((int64_t)d->n_steps * d->batch > ((int64_t)1 << 30))
        return hh::fail(HH_EINVAL, "n_steps * batch too large");
    hh::DevModel dm{};
    hh_status s = hh::prep_model(model, d->dt_ms, &dm);
    if (s != HH_OK)
        return s;
    if (dm.ca_ch >= 0)
        return hh::fail(HH_EUNSUPPORTED, "the layer supports models without a calcium pool");
    for (int q = 0; q < dm.n_gates; ++q)
        if (dm.g[q].kind == HH_GATE_CA)
            return hh::fail(HH_EUNSUPPORTED, "the layer supports alpha/beta and inf/tau gates");
    hh_layer* ly = new (std::nothrow) hh_layer();
    if (!ly)
        return hh::fail(HH_ENOMEM, "host allocation failed");
    hh::LayerImpl& L = ly->L;
    L.B = d->batch;
    L.n_in = d->n_in;
    L.n_in_pad = (d->n_in + 31) / 32 * 32;
    L.N = d->n_hidden;
    L.n_out = d->n_out;
    L.T = d->n_steps;
    L.K = d->substeps;
    L.ckpt = d->checkpoint_every;
    L.n_ckpt = (L.T + L.ckpt - 1) / L.ckpt;
    L.TB = L.T * L.B;
    L.TBp = (L.TB + 7) / 8 * 8;
    L.dt = (float)d->dt_ms;
    L.theta = d->v_threshold;
    L.beta = d->surrogate_beta;
    L.V0 = d->v_init;
    L.precision = d->precision;
    L.smooth = d->smooth ? 1 : 0;
    L.st = (cudaStream_t)d->stream;
    L.models.n = 1;
    L.models.max_gates = dm.n_gates;
    L.models.m[0] = dm;
    L.rec_splits = std::max(1, std::min(8, L.N / 128));
    L.ds_splits = std::max(1, std::min(8, 2 * L.N / 256));
    L.w_splits = std::max(1, std::min(8, L.TBp / 4096));
    const size_t BN = (size_t)L.B * L.N, N = L.N, TB = L.TB, TBp = L.TBp;
    cudaError_t e = cudaSuccess;
    auto A = [&](auto** p, size_t n) {
        if (e == cudaSuccess)
            e = ly->alloc(p, n);
    };
    A(&L.W_out, (size_t)L.n_out * N);
    A(&L.bias, N);
    A(&L.WinT, N * L.n_in_pad);
    A(&L.WrecT, N * N);
    A(&L.Wrec2, N * 2 * N);
    A(&L.Xb, TB * L.n_in_pad);
    A(&L.S, (TB + L.B) * N);
    A(&L.XW, TB * N);
    A(&L.recp, (size_t)L.rec_splits * BN);
    A(&L.I_all, TB * N);
    A(&L.Sf, TB * N);
    A(&L.V, BN);
    A(&L.P, BN * hh::kMaxGates);
    A(&L.ckptV, (size_t)(L.n_ckpt + 1) * BN);
    A(&L.ckptP, (size_t)(L.n_ckpt + 1) * hh::kMaxGates * BN);
    A(&L.acc, BN);
    A(&L.dlogits, (size_t)L.B * L.n_out);
    A(&L.loss_b, (size_t)L.B);
    A(&L.dlog_tot, (size_t)L.B * L.n_out);
    A(&L.segV, (size_t)L.ckpt * BN);
    A(&L.segP, (size_t)L.ckpt * hh::kMaxGates * BN);
    A(&L.lamV, BN);
    A(&L.lamP, BN * hh::kMaxGates);
    A(&L.ds_direct, BN);
    A(&L.dsp, (size_t)L.ds_splits * BN);
    A(&L.dI_all, TB * N);
    A(&L.dIb, BN * 2);
    A(&L.dIT_hi, N * TBp);
    A(&L.dIT_lo, N * TBp);
    A(&L.XT, (size_t)L.n_in_pad * TBp);
    A(&L.SpT, N * TBp);
    A(&L.wpart, std::max((size_t)2 * L.w_splits * N * std::max<size_t>(N, L.n_in_pad),
                         (size_t)hh::kColChunks * N));
    A(&L.status, 1);
    if (e != cudaSuccess) {
        ly->release();
        delete ly;
        return hh::fail(e == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA, "layer allocation: %s",
                        cudaGetErrorString(e));
    }
    // the forward, recompute and adjoint kernels with the model compiled in
    // (NVRTC, cached per model for the life of the process)
    std::string err;
    if (!hh::jit_get_layer(L.models, L.precision, &L.jit, &err)) {
        ly->release();
        delete ly;
        return hh::fail(HH_ECUDA, "%s", err.c_str());
    }
    L.bwd_smem = (size_t)hh::layer_bwd_smem(L.K, dm.n_gates > 0 ? dm.n_gates : 1, 128);
    if (L.bwd_smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute((const void*)L.jit.bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)L.bwd_smem)) != cudaSuccess) {
        ly->release();
        delete ly;
        return hh::fail(HH_ECUDA, "adjoint kernel shared memory: %s", cudaGetErrorString(e));
    }
    *out = ly;
    return HH_OK;
}

hh_status hh_layer_set_weights(hh_layer* ly, const float* W_in, const float* W_rec, const float* W_out,
                               const float* bias)
{
    if (!ly || !W_in || !W_rec || !W_out || !bias)
        return hh::fail(HH_EINVAL, "layer and weights must not be NULL");
    hh::LayerImpl& L = ly->L;
    cudaStream_t st = L.st;
    float *win = nullptr, *wrec = nullptr;
    const size_t nin = (size_t)L.n_in * L.N, nrec = (size_t)L.N * L.N;
    HH_LCUDA(cudaMalloc(&win, nin * sizeof(float)));
    cudaError_t e = cudaMalloc(&wrec, nrec * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(win, W_in, nin * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(wrec, W_rec, nrec * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.W_out, W_out, (size_t)L.n_out * L.N * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(L.bias, bias, (size_t)L.N * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) {
        dim3 blk(32, 8);
        hh::k_transpose_bf16<float><<<dim3((L.N + 31) / 32, (L.n_in + 31) / 32), blk, 0, st>>>(
            win, L.n_in, L.N, L.N, L.WinT, L.n_in_pad, nullptr);
        hh::k_transpose_bf16<float><<<dim3((L.N + 31) / 32, (L.N + 31) / 32), blk, 0, st>>>(
            wrec, L.N, L.N, L.N, L.WrecT, L.N, nullptr);
        k_dup_bf16<<<hh::grid1((int64_t)nrec, 256), 256, 0, st>>>(wrec, L.N, L.N, L.Wrec2);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(win);
    cudaFree(wrec);
    if (e == cudaSuccess)
        e = e2;
    if (e != cudaSuccess)
        return hh::fail(HH_ECUDA, "setting weights: %s", cudaGetErrorString(e));
    L.forward_done = false;
    L.win2_valid = false;
    return HH_OK;
}

hh_status hh_layer_forward(hh_layer* ly, const float* X, const int32_t* labels, float* loss, float* logits)
{
    if (!ly || !X)
        return hh::fail(HH_EINVAL, "layer and X must not be NULL");
    if (labels && !loss)
        return hh::fail(HH_EINVAL, "a forward with labels needs the loss output");
    HH_LCUDA(hh::layer_forward(ly->L, X, labels, loss, logits));
    return HH_OK;
}

hh_status hh_backward_from(hh_layer* ly, float ce_weight, const float* dL_dlogits, const float* dL_dS,
                           const float* dL_dV, const hh_grads* g)
{
    if (!ly || !g)
        return hh::fail(HH_EINVAL, "layer and gradient outputs must not be NULL");
    hh::LayerImpl& L = ly->L;
    if (!L.forward_done)
        return hh::fail(HH_ESTATE, "the backward pass needs a preceding hh_layer_forward");
    if (ce_weight != 0.0f && !L.forward_labels)
        return hh::fail(HH_ESTATE, "ce_weight != 0 needs a forward with labels");
    if (!std::isfinite(ce_weight))
        return hh::fail(HH_EINVAL, "ce_weight must be finite");
    if (g->dX && !L.Win2) {
        cudaError_t e = cudaSuccess;
        auto A = [&](auto** p, size_t n) {
            if (e == cudaSuccess)
                e = ly->alloc(p, n);
        };
        A(&L.dIrow, (size_t)L.TB * 2 * L.N);
        A(&L.Win2, (size_t)L.n_in_pad * 2 * L.N);
        A(&L.dXpart, (size_t)L.TB * L.n_in_pad);
        if (e != cudaSuccess) {
            L.Win2 = nullptr;
            return hh::fail(e == cudaErrorMemoryAllocation ? HH_ENOMEM : HH_ECUDA, "dX operands: %s",
                            cudaGetErrorString(e));
        }
        L.win2_valid = false;
    }
    HH_LCUDA(hh::layer_backward(L, ce_weight, dL_dlogits, dL_dS, dL_dV, *g));
    return HH_OK;
}

hh_status hh_backward(hh_layer* ly, const hh_grads* g)
{
    if (!ly || !g || !g->dW_in || !g->dW_rec || !g->dW_out || !g->dbias)
        return hh::fail(HH_EINVAL, "layer and the four weight-gradient buffers must be given");
    if (!ly->L.forward_done)
        return hh::fail(HH_ESTATE, "hh_backward needs a preceding hh_layer_forward");
    if (!ly->L.forward_labels)
        return hh::fail(HH_ESTATE, "hh_backward needs a forward with labels (its built-in loss)");
    return hh_backward_from(ly, 1.0f, nullptr, nullptr, nullptr, g);
}

hh_status hh_layer_readout(hh_layer* ly, int32_t what, void* dst, size_t cap, size_t* n_bytes)
{
    if (!ly || !dst)
        return hh::fail(HH_EINVAL, "layer and dst must not be NULL");
    if (n_bytes)
        *n_bytes = 0;
    hh::LayerImpl& L = ly->L;
    HH_LCUDA(cudaStreamSynchronize(L.st));
    const void* src = nullptr;
    size_t need = 0;
    switch (what) {
    case HH_LAYER_SPIKES: src = L.Sf; need = (size_t)L.TB * L.N * sizeof(float); break;
    case HH_LAYER_V: src = L.V; need = (size_t)L.B * L.N * sizeof(float); break;
    case HH_LAYER_STATUS: src = L.status; need = sizeof(int32_t); break;
    default: return hh::fail(HH_EINVAL, "unknown layer readout %d", what);
    }
    if (cap < need)
        return hh::fail(HH_EOVERFLOW, "layer readout %d needs %zu bytes", what, need);
    HH_LCUDA(cudaMemcpy(dst, src, need, cudaMemcpyDefault));
    if (n_bytes)
        *n_bytes = need;
    return HH_OK;
}

void hh_layer_destroy(hh_layer* ly)
{
    if (!ly)
        return;
    ly->release();
    delete ly;
}

}  // extern "C"
