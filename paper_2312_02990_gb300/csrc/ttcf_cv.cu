// ttcf_cv.cu -- learned control variate for the TTCF estimator.
//
// The paper has no learned part; the estimator it feeds is Eq. 1.  A small
// network f (32 -> 128 -> 128 -> 1, tanh) learns, from the features x of a
// mapped mother state, the per-daughter quantity z = Omega(0) I(t_end) /
// gamma (I = trapezoid integral of B = P_xy), whose group mean is the group's
// TTCF viscosity.  Used as a control variate with its mean taken over an
// independent auxiliary set of mother states, the estimate stays unbiased
// for any network and coefficient c.
//
// Numerics: FP32 master weights and Adam state; the forward and backward
// passes use the BF16 rounding of the weights, staged to FP32 in shared
// memory, with FP32 accumulation.  Every reduction has a fixed order, so
// training and inference are bitwise reproducible.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "ttcf_cv.h"

namespace ttcf {

// --------------------------------------------------- features, targets --
// Mapped features of daughter d (Eq. 3 sign rules) from its group's raw
// features; layout of the 32 outputs as in the oracle's mapped_features.
__global__ void cv_features_kernel(CvFeatArgs a) {
    const long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= a.D) return;
    const int g = (int)(d / a.M), m = a.maps[d % a.M];
    const double *r = a.raw + (size_t)g * FEAT_RAW;
    const double sxy = (m == 2 || m == 3) ? -1.0 : 1.0;
    const double sm = (m == 1 || m == 2) ? -1.0 : 1.0;
    const double sa = (m == 1 || m == 3) ? -1.0 : 1.0;
    const double sig[6] = {1.0, 1.0, 1.0, sxy, sxy, 1.0};
    float *x = a.X + (size_t)d * CV_NF;
    const double iv = 1.0 / a.V;
    for (int k = 0; k < 6; k++) {
        x[k] = (float)(r[k] * sig[k] * iv);
        x[6 + k] = (float)(r[6 + k] * sig[k] * iv);
    }
    x[12] = (float)(r[12] / a.N);
    x[13] = (float)(0.5 * r[13] / a.N);
    x[14] = a.reset_alpha ? 0.f : (float)(sa * (a.alpha ? a.alpha[g] : 0.0));
    const double pxy = (r[3] + r[9]) * sxy * iv;
    x[15] = (float)(pxy * pxy);
    for (int u = 0; u < 8; u++) {
        x[16 + u] = (float)r[14 + u];
        x[24 + u] = (float)(sm * r[22 + u]);
    }
}

// z_d = Omega_d * trapezoid(B_d) / gamma_g.
__global__ void cv_targets_kernel(const double *B, const double *Omega, const double *gamma,
                                  int M, long long D, int S, double ds, double *z) {
    const long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    const double *b = B + (size_t)d * S;
    double I = 0.5 * (b[0] + b[S - 1]);
    for (int s = 1; s < S - 1; s++) I += b[s];
    z[d] = Omega[d] * I * ds / gamma[d / M];
}

// Mean and standard deviation of column c of a [n][ld] float matrix over
// the rows listed in rows[0..n) (one CTA per column, fixed order).
__global__ void cv_colstats_kernel(const float *A, int ld, const int *rows, int n, double *stats) {
    __shared__ double red[32];
    const int c = blockIdx.x, tid = threadIdx.x;
    double s = 0.0;
    for (int r = tid; r < n; r += blockDim.x) s += A[(size_t)rows[r] * ld + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        red[0] = t / n;
    }
    __syncthreads();
    const double mean = red[0];
    __syncthreads();
    double v = 0.0;
    for (int r = tid; r < n; r += blockDim.x) {
        const double e = A[(size_t)rows[r] * ld + c] - mean;
        v += e * e;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        const double sd = n > 1 ? sqrt(t / (n - 1)) : 0.0;
        stats[2 * c] = mean;
        stats[2 * c + 1] = sd > 0.0 ? sd : 1.0;
    }
}

// In place: column c of A (or the vector y) -> (value - mean) / std.
__global__ void cv_standardize_kernel(float *X, long long n, const double *stats, float *y,
                                      const double *zstats, const double *z) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *x = X + (size_t)i * CV_NF;
    for (int c = 0; c < CV_NF; c++) x[c] = (float)((x[c] - stats[2 * c]) / stats[2 * c + 1]);
    if (y) y[i] = (float)((z[i] - zstats[0]) / zstats[1]);
}

// ------------------------------------------------------------- network --
// Parameter offsets in the flat vector (oracle order).
constexpr int OW1 = 0, OB1 = OW1 + CV_H * CV_NF, OW2 = OB1 + CV_H, OB2 = OW2 + CV_H * CV_H,
              OW3 = OB2 + CV_H, OB3 = OW3 + CV_H;
static_assert(OB3 + 1 == CV_NP, "parameter layout");

constexpr int SB = 32;            // samples per CTA
constexpr int LW1 = CV_NF + 1;    // padded shared-memory rows (no bank conflicts)
constexpr int LW2 = CV_H + 1;

struct MlpSmem {
    float W1[CV_H * LW1];
    float W2[CV_H * LW2];
    float b1[CV_H], b2[CV_H], W3[CV_H];
    float X[SB][CV_NF];
    float H1[SB][CV_H];
    float H2[SB][CV_H];
    float dA[SB][CV_H];
    float out[SB];
    float dout[SB];
    float red[4][SB];
};
size_t mlp_smem_bytes() { return sizeof(MlpSmem); }

__device__ void mlp_load_weights(MlpSmem &sm, const __nv_bfloat16 *wb) {
    for (int e = threadIdx.x; e < CV_H * CV_NF; e += blockDim.x)
        sm.W1[(e / CV_NF) * LW1 + e % CV_NF] = __bfloat162float(wb[OW1 + e]);
    for (int e = threadIdx.x; e < CV_H * CV_H; e += blockDim.x)
        sm.W2[(e / CV_H) * LW2 + e % CV_H] = __bfloat162float(wb[OW2 + e]);
    for (int e = threadIdx.x; e < CV_H; e += blockDim.x) {
        sm.b1[e] = __bfloat162float(wb[OB1 + e]);
        sm.b2[e] = __bfloat162float(wb[OB2 + e]);
        sm.W3[e] = __bfloat162float(wb[OW3 + e]);
    }
}

// Forward pass of up to SB samples (rows idx[0..ns) of X); blockDim = CV_H.
__device__ void mlp_forward_tile(MlpSmem &sm, const __nv_bfloat16 *wb, const float *X,
                                 const int *idx, long long base, int ns) {
    const int h = threadIdx.x;
    for (int e = h; e < SB * CV_NF; e += blockDim.x) {
        const int s = e / CV_NF, c = e % CV_NF;
        sm.X[s][c] = s < ns ? X[(size_t)(idx ? idx[base + s] : base + s) * CV_NF + c] : 0.f;
    }
    __syncthreads();
    for (int s = 0; s < SB; s++) {
        float acc = sm.b1[h];
        for (int k = 0; k < CV_NF; k++) acc = fmaf(sm.W1[h * LW1 + k], sm.X[s][k], acc);
        sm.H1[s][h] = tanhf(acc);
    }
    __syncthreads();
    for (int s = 0; s < SB; s++) {
        float acc = sm.b2[h];
        for (int k = 0; k < CV_H; k++) acc = fmaf(sm.W2[h * LW2 + k], sm.H1[s][k], acc);
        sm.H2[s][h] = tanhf(acc);
    }
    __syncthreads();
    // out[s] = b3 + sum_h W3[h] H2[s][h]: warp sums then the four warps in order
    const float b3 = __bfloat162float(wb[OB3]);
    for (int s = 0; s < SB; s++) {
        float v = sm.W3[h] * sm.H2[s][h];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((h & 31) == 0) sm.red[h >> 5][s] = v;
    }
    __syncthreads();
    if (h < SB) sm.out[h] = b3 + ((sm.red[0][h] + sm.red[1][h]) + (sm.red[2][h] + sm.red[3][h]));
    __syncthreads();
}

__global__ void __launch_bounds__(CV_H) mlp_predict_kernel(const __nv_bfloat16 *wb, const float *X,
                                                           long long n, float *out) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smraw);
    mlp_load_weights(sm, wb);
    __syncthreads();
    for (long long base = (long long)blockIdx.x * SB; base < n; base += (long long)gridDim.x * SB) {
        const long long rem = n - base;
        const int ns = rem < SB ? (int)rem : SB;
        mlp_forward_tile(sm, wb, X, nullptr, base, ns);
        if (threadIdx.x < ns) out[base + threadIdx.x] = sm.out[threadIdx.x];
        __syncthreads();
    }
}

// Forward and backward of one tile of the minibatch (CTA b handles samples
// idx[base + SB*b ...]); writes this tile's gradient (loss = mean over the
// whole minibatch of (f - y)^2) and loss share to part[b].
__global__ void __launch_bounds__(CV_H) mlp_grad_kernel(const __nv_bfloat16 *wb, const float *X,
                                                        const float *y, const int *idx, long long base,
                                                        int nbatch, float *part, double *lpart,
                                                        int *step) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smraw);
    if (step && blockIdx.x == 0 && threadIdx.x == 0) step[0] += 1;   // Adam step counter
    mlp_load_weights(sm, wb);
    __syncthreads();
    const long long t0 = base + (long long)blockIdx.x * SB;
    const int ns = max(0, min(SB, (int)(base + nbatch - t0)));
    mlp_forward_tile(sm, wb, X, idx, t0, ns);
    const int h = threadIdx.x;
    if (h < SB) {
        const float r = h < ns ? sm.out[h] - y[idx ? idx[t0 + h] : t0 + h] : 0.f;
        sm.dout[h] = 2.f * r / (float)nbatch;
        sm.red[0][h] = r * r;
    }
    __syncthreads();
    if (h == 0) {
        double l = 0.0;
        for (int s = 0; s < SB; s++) l += sm.red[0][s];
        lpart[blockIdx.x] = l / nbatch;
    }
    float *g = part + (size_t)blockIdx.x * CV_NP;
    // output layer
    {
        float gw = 0.f;
        for (int s = 0; s < SB; s++) gw = fmaf(sm.dout[s], sm.H2[s][h], gw);
        g[OW3 + h] = gw;
        if (h == 0) {
            float gb = 0.f;
            for (int s = 0; s < SB; s++) gb += sm.dout[s];
            g[OB3] = gb;
        }
        for (int s = 0; s < SB; s++) {
            const float a2 = sm.H2[s][h];
            sm.dA[s][h] = sm.dout[s] * sm.W3[h] * (1.f - a2 * a2);
        }
    }
    __syncthreads();
    // layer 2: thread h owns row h of W2
    {
        float dreg[SB];
#pragma unroll
        for (int s = 0; s < SB; s++) dreg[s] = sm.dA[s][h];
        float gb = 0.f;
#pragma unroll
        for (int s = 0; s < SB; s++) gb += dreg[s];
        g[OB2 + h] = gb;
        for (int k = 0; k < CV_H; k++) {
            float gw = 0.f;
#pragma unroll
            for (int s = 0; s < SB; s++) gw = fmaf(dreg[s], sm.H1[s][k], gw);
            g[OW2 + h * CV_H + k] = gw;
        }
    }
    // back through W2: thread k forms dH1[s][k] = sum_h W2[h][k] dA2[s][h]
    __syncthreads();
    {
        const int k = h;
        float dh[SB];
#pragma unroll
        for (int s = 0; s < SB; s++) dh[s] = 0.f;
        for (int hh = 0; hh < CV_H; hh++) {
            const float w = sm.W2[hh * LW2 + k];
#pragma unroll
            for (int s = 0; s < SB; s++) dh[s] = fmaf(w, sm.dA[s][hh], dh[s]);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < SB; s++) {
            const float a1 = sm.H1[s][k];
            sm.dA[s][k] = dh[s] * (1.f - a1 * a1);
        }
    }
    __syncthreads();
    // layer 1: thread h owns row h of W1
    {
        float dreg[SB];
#pragma unroll
        for (int s = 0; s < SB; s++) dreg[s] = sm.dA[s][h];
        float gb = 0.f;
#pragma unroll
        for (int s = 0; s < SB; s++) gb += dreg[s];
        g[OB1 + h] = gb;
        for (int c = 0; c < CV_NF; c++) {
            float gw = 0.f;
#pragma unroll
            for (int s = 0; s < SB; s++) gw = fmaf(dreg[s], sm.X[s][c], gw);
            g[OW1 + h * CV_NF + c] = gw;
        }
    }
}

// Sum of the tiles' gradients in tile order, then (if lr > 0) one Adam
// step on the FP32 master weights and their BF16 copy.  step[0] = t >= 1.
__global__ void mlp_adam_kernel(const float *part, int ntiles, const double *lpart, float *grad,
                                double *loss, float *w, float *mom, float *vel, __nv_bfloat16 *wb,
                                const int *step, float lr, float beta1, float beta2, float eps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss) {
        double l = 0.0;
        for (int b = 0; b < ntiles; b++) l += lpart[b];
        loss[0] += l;
    }
    if (p >= CV_NP) return;
    float gsum = 0.f;
    for (int b = 0; b < ntiles; b++) gsum += part[(size_t)b * CV_NP + p];
    if (grad) grad[p] = gsum;
    if (lr <= 0.f) return;
    const int t = step[0];
    const float m = beta1 * mom[p] + (1.f - beta1) * gsum;
    const float v = beta2 * vel[p] + (1.f - beta2) * gsum * gsum;
    mom[p] = m;
    vel[p] = v;
    const float mh = m / (1.f - powf(beta1, (float)t));
    const float vh = v / (1.f - powf(beta2, (float)t));
    const float nw = w[p] - lr * mh / (sqrtf(vh) + eps);
    w[p] = nw;
    wb[p] = __float2bfloat16_rn(nw);
}

__global__ void f32_to_bf16_kernel(const float *w, __nv_bfloat16 *wb, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) wb[p] = __float2bfloat16_rn(w[p]);
}

// --------------------------------------------------------- estimator --
// Group values of a batch: y_g = -(1/M) sum_m z_{g,m} and
// h_g = -(1/M) sum_m (zmean + zstd * f_{g,m}), over the listed groups.
__global__ void cv_group_kernel(const double *z, const float *f, const double *zstats, int M,
                                const int *groups, int ng, double *yg, double *hg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    const long long g = groups[i];
    double ys = 0.0, hs = 0.0;
    for (int m = 0; m < M; m++) {
        if (z) ys += z[g * M + m];
        hs += zstats[0] + zstats[1] * (double)f[g * M + m];
    }
    if (yg) yg[i] = -ys / M;
    hg[i] = -hs / M;
}

// One CTA: sums in index order and the estimator (eta, se for plain and
// control variate, with c given or fitted when fit_c != 0).
//   out: [0] eta_plain [1] se_plain [2] eta_cv [3] se_cv [4] c [5] gain
//        [6] n_D [7] n_M
__global__ void cv_estimate_kernel(const double *yD, const double *hD, int nD, const double *hM,
                                   int nM, int fit_c, double c_in, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double sy = 0, sh = 0, shm = 0;
    for (int i = 0; i < nD; i++) { sy += yD[i]; sh += hD[i]; }
    for (int i = 0; i < nM; i++) shm += hM[i];
    const double my = sy / nD, mh = sh / nD, mhm = nM > 0 ? shm / nM : 0.0;
    double vyy = 0, vhh = 0, vyh = 0, vm = 0;
    for (int i = 0; i < nD; i++) {
        const double ey = yD[i] - my, eh = hD[i] - mh;
        vyy += ey * ey; vhh += eh * eh; vyh += ey * eh;
    }
    for (int i = 0; i < nM; i++) { const double e = hM[i] - mhm; vm += e * e; }
    const double c = fit_c ? (vhh > 0 ? vyh / vhh : 0.0) : c_in;
    // Var(y - c h) over D
    const double vr = (vyy - 2.0 * c * vyh + c * c * vhh) / (nD - 1);
    const double se_pl = sqrt(vyy / (nD - 1) / nD);
    const double se_cv = sqrt(vr / nD + (nM > 1 ? c * c * vm / (nM - 1) / nM : 0.0));
    out[0] = my; out[1] = se_pl;
    out[2] = my - c * mh + c * mhm; out[3] = se_cv;
    out[4] = c; out[5] = se_pl * se_pl / (se_cv * se_cv);
    out[6] = nD; out[7] = nM;
}

// ------------------------------------------------------------ launchers --
cudaError_t cv_launch_features(const CvFeatArgs &a, cudaStream_t st) {
    cv_features_kernel<<<(unsigned)((a.D + 127) / 128), 128, 0, st>>>(a);
    return cudaGetLastError();
}
cudaError_t cv_launch_targets(const double *B, const double *Omega, const double *gamma, int M,
                              long long D, int S, double ds, double *z, cudaStream_t st) {
    cv_targets_kernel<<<(unsigned)((D + 127) / 128), 128, 0, st>>>(B, Omega, gamma, M, D, S, ds, z);
    return cudaGetLastError();
}
cudaError_t cv_launch_colstats(const float *A, int ld, const int *rows, int n, int ncols,
                               double *stats, cudaStream_t st) {
    cv_colstats_kernel<<<ncols, 256, 0, st>>>(A, ld, rows, n, stats);
    return cudaGetLastError();
}
cudaError_t cv_launch_standardize(float *X, long long n, const double *stats, float *y,
                                  const double *zstats, const double *z, cudaStream_t st) {
    cv_standardize_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(X, n, stats, y, zstats, z);
    return cudaGetLastError();
}
cudaError_t cv_launch_predict(const __nv_bfloat16 *wb, const float *X, long long n, float *out,
                              int nsm, cudaStream_t st) {
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (n + SB - 1) / SB;
    const int grid = (int)std::min<long long>(tiles, (long long)nsm * 2);
    mlp_predict_kernel<<<std::max(grid, 1), CV_H, smem, st>>>(wb, X, n, out);
    return cudaGetLastError();
}
cudaError_t cv_launch_grad(const __nv_bfloat16 *wb, const float *X, const float *y, const int *idx,
                           long long base, int nbatch, float *part, double *lpart, int *step,
                           cudaStream_t st) {
    const size_t smem = sizeof(MlpSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = (nbatch + SB - 1) / SB;
    mlp_grad_kernel<<<tiles, CV_H, smem, st>>>(wb, X, y, idx, base, nbatch, part, lpart, step);
    return cudaGetLastError();
}
cudaError_t cv_launch_adam(const float *part, int ntiles, const double *lpart, float *grad, double *loss,
                           float *w, float *m, float *v, __nv_bfloat16 *wb, const int *step, float lr,
                           float b1, float b2, float eps, cudaStream_t st) {
    mlp_adam_kernel<<<(CV_NP + 255) / 256, 256, 0, st>>>(part, ntiles, lpart, grad, loss, w, m, v, wb,
                                                         step, lr, b1, b2, eps);
    return cudaGetLastError();
}
cudaError_t cv_launch_to_bf16(const float *w, __nv_bfloat16 *wb, cudaStream_t st) {
    f32_to_bf16_kernel<<<(CV_NP + 255) / 256, 256, 0, st>>>(w, wb, CV_NP);
    return cudaGetLastError();
}
cudaError_t cv_launch_group(const double *z, const float *f, const double *zstats, int M,
                            const int *groups, int ng, double *yg, double *hg, cudaStream_t st) {
    cv_group_kernel<<<(ng + 127) / 128, 128, 0, st>>>(z, f, zstats, M, groups, ng, yg, hg);
    return cudaGetLastError();
}
cudaError_t cv_launch_estimate(const double *yD, const double *hD, int nD, const double *hM, int nM,
                               int fit_c, double c_in, double *out, cudaStream_t st) {
    cv_estimate_kernel<<<1, 32, 0, st>>>(yD, hD, nD, hM, nM, fit_c, c_in, out);
    return cudaGetLastError();
}

}  // namespace ttcf
