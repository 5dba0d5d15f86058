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

// Raw features of one mother state per CTA, FP32 arithmetic: positions and
// momenta rounded to float (the hi parts of float-pair slots, or doubles
// rounded to nearest, which is the same number), a cell list of width >= r_c
// sorted by index within each cell (a fixed summation order), WCA pair
// terms in FP32, per-thread FP32 partials and FP64 block sums in a fixed
// order.  Outputs as the spawn kernel's FEAT_RAW layout:
//   [0..5] sum p_a p_b (xx yy zz xy xz yz), [6..11] virial sum over pairs of
//   r_a F_b, [12] U (WCA, shifted), [13] sum p^2, [14..21] (cos, sin) modes
//   q = 1..4 of the density over 40 slabs in y, [22..29] the same of p_x.
constexpr int CV_NSLAB = 40, CV_NACC = 30;

__global__ void __launch_bounds__(256, 4) cv_raw_features_kernel(CvRawArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = blockIdx.x, tid = threadIdx.x, T = blockDim.x, N = a.N;
    float *xf = reinterpret_cast<float *>(smem), *yf = xf + N, *zf = yf + N;
    double *red = reinterpret_cast<double *>(smem + (((size_t)N * 12 + 15) / 16 * 16));
    float *cs = reinterpret_cast<float *>(red + 32 * CV_NACC);   // [40][8]
    int *cnt = reinterpret_cast<int *>(cs + CV_NSLAB * 8);
    int *start = cnt + a.ncell;
    int *warp_tmp = start + a.ncell + 2;
    unsigned short *catom = reinterpret_cast<unsigned short *>(warp_tmp + 32);

    auto ld = [&](int row, int i) -> float {
        const size_t e = ((size_t)g * 6 + row) * N + i;
        if (a.kind == 1) return reinterpret_cast<const float2 *>(a.src)[e].x;
        return __double2float_rn(reinterpret_cast<const double *>(a.src)[e]);
    };
    const float Lx = (float)a.L[0], Ly = (float)a.L[1], Lz = (float)a.L[2];
    const float iLx = (float)(1.0 / a.L[0]), iLy = (float)(1.0 / a.L[1]), iLz = (float)(1.0 / a.L[2]);
    for (int i = tid; i < N; i += T) { xf[i] = ld(0, i); yf[i] = ld(1, i); zf[i] = ld(2, i); }
    for (int c = tid; c < a.ncell; c += T) cnt[c] = 0;
    for (int e = tid; e < CV_NSLAB * 4; e += T) {   // cos, sin of 2 pi q (k + 1/2) / 40
        const int k = e / 4, q = e % 4 + 1;
        float sn, c;
        sincospif(2.0f * q * (k + 0.5f) / CV_NSLAB, &sn, &c);
        cs[k * 8 + 2 * (q - 1)] = c;
        cs[k * 8 + 2 * (q - 1) + 1] = sn;
    }
    __syncthreads();
    auto cell3 = [&](int i, int &cx, int &cy, int &cz) {
        const float x = xf[i] - Lx * rintf(xf[i] * iLx), y = yf[i] - Ly * rintf(yf[i] * iLy),
                    z = zf[i] - Lz * rintf(zf[i] * iLz);
        cx = min(max((int)floorf((x + 0.5f * Lx) * a.nc[0] * iLx), 0), a.nc[0] - 1);
        cy = min(max((int)floorf((y + 0.5f * Ly) * a.nc[1] * iLy), 0), a.nc[1] - 1);
        cz = min(max((int)floorf((z + 0.5f * Lz) * a.nc[2] * iLz), 0), a.nc[2] - 1);
    };
    for (int i = tid; i < N; i += T) {
        int cx, cy, cz;
        cell3(i, cx, cy, cz);
        atomicAdd(&cnt[(cz * a.nc[1] + cy) * a.nc[0] + cx], 1);
    }
    __syncthreads();
    cta_exclusive_scan(cnt, start, a.ncell, warp_tmp);
    __syncthreads();
    for (int c = tid; c < a.ncell; c += T) cnt[c] = start[c];
    __syncthreads();
    for (int i = tid; i < N; i += T) {
        int cx, cy, cz;
        cell3(i, cx, cy, cz);
        catom[atomicAdd(&cnt[(cz * a.nc[1] + cy) * a.nc[0] + cx], 1)] = (unsigned short)i;
    }
    __syncthreads();
    for (int c = tid; c < a.ncell; c += T)   // index order within each cell
        for (int u = start[c] + 1; u < start[c + 1]; u++) {
            const unsigned short v = catom[u];
            int w = u;
            while (w > start[c] && catom[w - 1] > v) { catom[w] = catom[w - 1]; w--; }
            catom[w] = v;
        }
    __syncthreads();

    float acc[CV_NACC];
    for (int k = 0; k < CV_NACC; k++) acc[k] = 0.f;
    const float rc2 = 1.2599210498948732f;
    for (int i = tid; i < N; i += T) {
        const float px = ld(3, i), py = ld(4, i), pz = ld(5, i);
        acc[0] += px * px; acc[1] += py * py; acc[2] += pz * pz;
        acc[3] += px * py; acc[4] += px * pz; acc[5] += py * pz;
        acc[13] += px * px + py * py + pz * pz;
        {
            int k = (int)floorf((yf[i] + 0.5f * Ly) * iLy * CV_NSLAB);
            k = min(max(k, 0), CV_NSLAB - 1);
            for (int u = 0; u < 8; u++) {
                acc[14 + u] += cs[k * 8 + u];
                acc[22 + u] += px * cs[k * 8 + u];
            }
        }
        int cx, cy, cz;
        cell3(i, cx, cy, cz);
        for (int oz = -1; oz <= 1; oz++) {
            const int zz = (cz + oz + a.nc[2]) % a.nc[2];
            for (int oy = -1; oy <= 1; oy++) {
                const int yy = (cy + oy + a.nc[1]) % a.nc[1];
                for (int ox = -1; ox <= 1; ox++) {
                    const int xx = (cx + ox + a.nc[0]) % a.nc[0];
                    const int c = (zz * a.nc[1] + yy) * a.nc[0] + xx;
                    for (int t = start[c]; t < start[c + 1]; t++) {
                        const int j = catom[t];
                        if (j == i) continue;
                        float dx = xf[i] - xf[j], dy = yf[i] - yf[j], dz = zf[i] - zf[j];
                        dx -= Lx * rintf(dx * iLx); dy -= Ly * rintf(dy * iLy); dz -= Lz * rintf(dz * iLz);
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < rc2) {
                            const float sv = 1.0f / r2, s3 = sv * sv * sv;
                            const float hf = 0.5f * s3 * sv * (48.0f * s3 - 24.0f);   // half of |F|/r
                            acc[6] += hf * dx * dx; acc[7] += hf * dy * dy; acc[8] += hf * dz * dz;
                            acc[9] += hf * dx * dy; acc[10] += hf * dx * dz; acc[11] += hf * dy * dz;
                            acc[12] += 0.5f * (4.0f * s3 * (s3 - 1.0f) + 1.0f);
                        }
                    }
                }
            }
        }
    }
    // block sums in 64-bit fixed point of 2^-40 units (integer shuffles:
    // a float partial of magnitude >= 2^-17 is exact there, so the sums
    // are exact and order-free; GB300's FP64 pipe, on which a shuffle tree
    // of 30 doubles per warp took a quarter of this kernel, stays idle)
    // The 64-bit sums hold |total| < 2^23: a state with a thread partial of
    // 2^15 or more (or not finite) takes the FP64 tree instead (normal
    // partials are below 10^3).
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    bool big = false;
    for (int k = 0; k < CV_NACC; k++) big |= !(fabsf(acc[k]) < 32768.f);
    if (!__syncthreads_or(big)) {
        long long *redl = reinterpret_cast<long long *>(red);
        for (int k = 0; k < CV_NACC; k++) {
            long long v = __float2ll_rn(acc[k] * 1099511627776.0f);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) redl[warp * CV_NACC + k] = v;
        }
        __syncthreads();
        if (tid < CV_NACC) {
            long long v = 0;
            for (int w = 0; w < nw; w++) v += redl[w * CV_NACC + tid];
            double x = (double)v * 9.094947017729282e-13;   // x 2^-40
            if (tid >= 14) x /= N;   // modes per atom
            a.raw[(size_t)g * FEAT_RAW + tid] = x;
        }
    } else {
        for (int k = 0; k < CV_NACC; k++) {
            double v = (double)acc[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp * CV_NACC + k] = v;
        }
        __syncthreads();
        if (tid < CV_NACC) {
            double v = 0.0;
            for (int w = 0; w < nw; w++) v += red[w * CV_NACC + tid];
            if (tid >= 14) v /= N;   // modes per atom
            a.raw[(size_t)g * FEAT_RAW + tid] = v;
        }
    }
    if (tid == 0) { a.raw[(size_t)g * FEAT_RAW + 30] = 0.0; a.raw[(size_t)g * FEAT_RAW + 31] = 0.0; }
}

size_t cv_raw_smem_bytes(int N, int ncell) {
    return ((size_t)N * 12 + 15) / 16 * 16 + 32 * CV_NACC * 8 + CV_NSLAB * 8 * 4 +
           (size_t)(2 * ncell + 2 + 32) * 4 + (size_t)N * 2 + 16;
}

cudaError_t cv_launch_raw_features(const CvRawArgs &a, cudaStream_t st) {
    const size_t smem = cv_raw_smem_bytes(a.N, a.ncell);
    cudaError_t e = cudaFuncSetAttribute(cv_raw_features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cv_raw_features_kernel<<<a.G, 256, smem, st>>>(a);
    return cudaGetLastError();
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

// ------------------------------------------- forward on the tensor cores --
// The two hidden layers of the forward pass as tcgen05 matrix products on
// GB300's tensor cores: 128 samples per tile, D = A B^T with A the samples'
// activations [128 x K] and B the BF16 weights [128 x K] (the network's
// weights are used through their BF16 rounding anyway), both K-major in
// shared memory, FP32 accumulators in tensor memory (TMEM, 256 columns:
// layer 1 in columns 0..127, layer 2 in 128..255).  The FP32 activations
// are carried as the sum of two BF16 terms (hi = bf16(x), lo = bf16(x - hi),
// 16 significand bits), each multiplied into the same accumulator, so the
// products keep about 2^-17 relative accuracy (the SIMT path and the FP64
// oracle agree with it to ~1e-5).  One thread issues the MMAs and commits
// them to an mbarrier; every wait is bounded and a timeout sets g_tc_error,
// writes NaN for the tile and ends the CTA after releasing its TMEM.
namespace {

constexpr int TC_M = 128;                          // samples per tile
constexpr int TC_A1 = 2 * TC_M * CV_NF * 2;        // X as two BF16 terms
constexpr int TC_B1 = CV_H * CV_NF * 2;            // W1
constexpr int TC_A2 = 2 * TC_M * CV_H * 2;         // H1 as two BF16 terms
constexpr int TC_B2 = CV_H * CV_H * 2;             // W2
constexpr int TC_OFF_B1 = TC_A1, TC_OFF_A2 = TC_OFF_B1 + TC_B1, TC_OFF_B2 = TC_OFF_A2 + TC_A2;
constexpr int TC_OFF_V = TC_OFF_B2 + TC_B2;        // b1, b2, W3 (FP32)
constexpr int TC_OFF_BAR = TC_OFF_V + 3 * CV_H * 4;
constexpr int TC_SMEM = TC_OFF_BAR + 16 + 128;     // + mbarrier, TMEM address, alignment slack
constexpr long long TC_SPIN = 1ll << 22;           // wait iterations before giving up

__device__ int g_tc_error;

// Byte offset of element (r, k) of a [rows x K] BF16 tile in the K-major
// layout without swizzle: 8 x 8 core matrices of 128 contiguous bytes
// (8 rows of 16 bytes), core matrices adjacent in K 128 bytes apart,
// adjacent in rows K/8 * 128 bytes apart.
__device__ __forceinline__ int tc_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices along K), stride-dimension byte offset
// (between core matrices along rows), the fixed 0b001 at bits 46-48, no
// swizzle (bits 61-63 = 0).
__device__ __forceinline__ unsigned long long tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (unsigned long long)((saddr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// BF16 A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CV_H >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, unsigned long long a, unsigned long long b, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(dtmem), "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

// Bounded wait for the mbarrier phase; false on timeout.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t phase) {
    for (long long it = 0; it < TC_SPIN; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(phase) : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this thread's row (lane).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                 "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int k = 0; k < 32; k++) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tc_split_store(unsigned char *tile, int term_bytes, int r, int k, int K, float x) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    const int o = tc_off(r, k, K);
    *reinterpret_cast<__nv_bfloat16 *>(tile + o) = hi;
    *reinterpret_cast<__nv_bfloat16 *>(tile + term_bytes + o) = lo;
}

}  // namespace

__global__ void __launch_bounds__(TC_M, 1) mlp_predict_tc_kernel(const __nv_bfloat16 *wb, const float *X,
                                                                  long long n, float *out) {
    extern __shared__ __align__(128) unsigned char tcs[];
    unsigned char *base = tcs + ((128 - (smem_addr(tcs) & 127)) & 127);   // 128-byte aligned tiles
    unsigned char *A1 = base, *B1 = base + TC_OFF_B1, *A2 = base + TC_OFF_A2, *B2 = base + TC_OFF_B2;
    float *b1 = reinterpret_cast<float *>(base + TC_OFF_V), *b2 = b1 + CV_H, *W3 = b2 + CV_H;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(base + TC_OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(base + TC_OFF_BAR + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbar = smem_addr(bar);

    // weights: BF16 copies into the K-major layouts, biases and W3 in FP32
    for (int e = tid; e < CV_H * CV_NF; e += TC_M)
        *reinterpret_cast<__nv_bfloat16 *>(B1 + tc_off(e / CV_NF, e % CV_NF, CV_NF)) = wb[OW1 + e];
    for (int e = tid; e < CV_H * CV_H; e += TC_M)
        *reinterpret_cast<__nv_bfloat16 *>(B2 + tc_off(e / CV_H, e % CV_H, CV_H)) = wb[OW2 + e];
    b1[tid] = __bfloat162float(wb[OB1 + tid]);
    b2[tid] = __bfloat162float(wb[OB2 + tid]);
    W3[tid] = __bfloat162float(wb[OW3 + tid]);
    const float b3 = __bfloat162float(wb[OB3]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {   // 256 TMEM columns: two 128 x 128 FP32 accumulators
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(smem_addr(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's 32 lanes
    uint32_t phase = 0;
    bool ok = true;

    for (long long t0 = (long long)blockIdx.x * TC_M; t0 < n && ok; t0 += (long long)gridDim.x * TC_M) {
        // this thread's sample: features into the two BF16 terms of A1
        const long long row = t0 + tid;
        for (int k = 0; k < CV_NF; k++)
            tc_split_store(A1, TC_A1 / 2, tid, k, CV_NF, row < n ? X[(size_t)row * CV_NF + k] : 0.f);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == 0) {   // layer 1: K = 32 in two steps of 16, two activation terms
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t acc = 0;
            for (int term = 0; term < 2; term++)
                for (int j = 0; j < CV_NF / 16; j++) {
                    tc_mma(tmem, tc_desc(smem_addr(A1 + term * (TC_A1 / 2) + j * 256), 128, (CV_NF / 8) * 128),
                           tc_desc(smem_addr(B1 + j * 256), 128, (CV_NF / 8) * 128), acc);
                    acc = 1;
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(sbar)
                         : "memory");
        }
        ok = tc_wait(sbar, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {   // H1 = tanh(acc + b1) into the two BF16 terms of A2
            for (int c0 = 0; c0 < CV_H; c0 += 32) {
                float v[32];
                tc_ld32(trow + (uint32_t)c0, v);
                for (int k = 0; k < 32; k++) tc_split_store(A2, TC_A2 / 2, tid, c0 + k, CV_H, tanhf(v[k] + b1[c0 + k]));
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {   // layer 2: K = 128 in eight steps of 16, two activation terms
            asm volatile("tcgen05.fence::after_thread_sync;");
            uint32_t acc = 0;
            for (int term = 0; term < 2; term++)
                for (int j = 0; j < CV_H / 16; j++) {
                    tc_mma(tmem + CV_H, tc_desc(smem_addr(A2 + term * (TC_A2 / 2) + j * 256), 128, (CV_H / 8) * 128),
                           tc_desc(smem_addr(B2 + j * 256), 128, (CV_H / 8) * 128), acc);
                    acc = 1;
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(sbar)
                         : "memory");
        }
        ok = tc_wait(sbar, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        float o = b3;
        if (ok) {   // output = b3 + sum_h W3[h] tanh(acc + b2), columns in order
            float sacc = 0.f;
            for (int c0 = 0; c0 < CV_H; c0 += 32) {
                float v[32];
                tc_ld32(trow + (uint32_t)(CV_H + c0), v);
                for (int k = 0; k < 32; k++) sacc = fmaf(W3[c0 + k], tanhf(v[k] + b2[c0 + k]), sacc);
            }
            o += sacc;
        } else {
            o = __int_as_float(0x7fc00000);
        }
        if (row < n) out[row] = o;
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
    }
    if (!ok && tid == 0) atomicExch(&g_tc_error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem));
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
    // the forward pass on the tensor cores (one CTA of 128 threads per SM,
    // persistent over the 128-sample tiles)
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_predict_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    const long long tiles = (n + TC_M - 1) / TC_M;
    const int grid = (int)std::min<long long>(tiles, (long long)nsm);
    mlp_predict_tc_kernel<<<std::max(grid, 1), TC_M, TC_SMEM, st>>>(wb, X, n, out);
    return cudaGetLastError();
}

cudaError_t cv_tc_reset(cudaStream_t st) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tc_error);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(p, 0, sizeof(int), st);
}

cudaError_t cv_tc_failed(cudaStream_t st, int *failed) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_tc_error);
    if (e == cudaSuccess) e = cudaMemcpyAsync(failed, p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
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
