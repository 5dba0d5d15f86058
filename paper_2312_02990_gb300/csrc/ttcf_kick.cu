// ttcf_kick.cu -- further mother states from one thermalised state by small
// random momentum kicks.
//
// The paper's thermalisation workflow generates further initial conditions
// from one equilibrated state by adding a small random kick to the
// velocities: the dynamics is chaotic, so the copies decorrelate quickly,
// and a small kick leaves the thermodynamic state in place.  Copy c adds to
// momentum component k of atom i the kick  kick * sqrt(T) * g  with g a
// standard normal number from Philox-4x32-10 (Salmon, Moraes, Dror, Shaw,
// SC'11; keyed by the 64-bit seed, counter (i, c, b, 0), b = 0, 1) and the
// Box-Muller transform of 53-bit uniforms; every group of atoms (types 0, 1,
// 2, or one group) keeps its net momentum, and optionally the kinetic
// energy of its momenta relative to the group mean (rescaled about the
// mean).  IEEE double throughout: a handful of copies is made once per
// thermalisation, so the FP64 rate does not matter here.
#include <stdint.h>

#include "ttcf_internal.h"

namespace ttcf {
namespace {

constexpr uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;   // key increments
constexpr int KICK_THREADS = 256;
constexpr int NV1 = 21;   // pass-1 sums: 3 groups x (3 momentum + 3 kick components + count)
constexpr int NV2 = 6;    // pass-2 sums: 3 groups x (|q|^2, |q'|^2)

// Ten rounds of Philox-4x32 in place.  A round maps (c0, c1, c2, c3) with
// key (k0, k1) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
// lo(M0 c0)); the key advances by (W0, W1) between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint32_t lo0 = PHILOX_M0 * c[0], hi0 = __umulhi(PHILOX_M0, c[0]);
        const uint32_t lo1 = PHILOX_M1 * c[2], hi1 = __umulhi(PHILOX_M1, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += PHILOX_W0; k1 += PHILOX_W1;
    }
}

// Uniform in (0, 1): the high 53 bits of the word pair, plus half a step.
__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
    const unsigned long long v = (((unsigned long long)hi << 32) | lo) >> 11;
    return (double)v * 0x1p-53 + 0x1p-54;
}

// The three normal numbers of atom i in copy c (g0, g1 from block 0, g2 the
// cosine branch of block 1).
__device__ __forceinline__ void kick_normals(uint32_t i, uint32_t c, uint32_t k0, uint32_t k1, double g[3]) {
    const double two_pi = 2.0 * 3.14159265358979323846;
    uint32_t w[4] = {i, c, 0u, 0u};
    philox4x32_10(w, k0, k1);
    double r = sqrt(-2.0 * log(uniform53(w[0], w[1])));
    double th = two_pi * uniform53(w[2], w[3]);
    g[0] = r * cos(th);
    g[1] = r * sin(th);
    uint32_t v[4] = {i, c, 1u, 0u};
    philox4x32_10(v, k0, k1);
    r = sqrt(-2.0 * log(uniform53(v[0], v[1])));
    th = two_pi * uniform53(v[2], v[3]);
    g[2] = r * cos(th);
}

// Sum of NV per-thread values over the block in a fixed order (warp
// butterfly, then the warps in order); the result lands in red[0..NV).
template <int NV>
__device__ void block_sum(double v[NV], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; j++)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    __syncthreads();   // red[] may still be read from the previous sum
    if (lane == 0)
        for (int j = 0; j < NV; j++) red[NV + warp * NV + j] = v[j];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < nw; w++) s += red[NV + w * NV + threadIdx.x];
        red[threadIdx.x] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(KICK_THREADS) kick_kernel(KickArgs a) {
    extern __shared__ double red[];   // [NV1] results + [warps][NV1] partials
    const int N = a.N, c = blockIdx.x, T = blockDim.x;
    const uint32_t k0 = (uint32_t)(a.seed & 0xFFFFFFFFull), k1 = (uint32_t)(a.seed >> 32);
    const double *src = a.src;
    double *out = a.out + (size_t)c * 6 * N;

    // pass 1: positions copied, kicks stored in the momentum rows, group sums
    double v1[NV1];
#pragma unroll
    for (int j = 0; j < NV1; j++) v1[j] = 0.0;
    for (int i = threadIdx.x; i < N; i += T) {
        const int t = a.types ? a.types[i] : 0;
        double g[3];
        kick_normals((uint32_t)i, (uint32_t)c, k0, k1, g);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const double dp = a.ks * g[k];
            out[(size_t)k * N + i] = src[(size_t)k * N + i];
            out[(size_t)(3 + k) * N + i] = dp;
            const double p = src[(size_t)(3 + k) * N + i];
#pragma unroll
            for (int gi = 0; gi < 3; gi++)
                if (gi == t) { v1[7 * gi + k] += p; v1[7 * gi + 3 + k] += dp; }
        }
#pragma unroll
        for (int gi = 0; gi < 3; gi++)
            if (gi == t) v1[7 * gi + 6] += 1.0;
    }
    block_sum<NV1>(v1, red);
    double pbar[3][3], dbar[3][3];
#pragma unroll
    for (int gi = 0; gi < 3; gi++) {
        const double n = red[7 * gi + 6];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            pbar[gi][k] = n > 0.0 ? red[7 * gi + k] / n : 0.0;
            dbar[gi][k] = n > 0.0 ? red[7 * gi + 3 + k] / n : 0.0;
        }
    }

    // pass 2: |q|^2 and |q'|^2 per group, q = p - pbar, q' = q + (dp - dbar)
    double v2[NV2];
#pragma unroll
    for (int j = 0; j < NV2; j++) v2[j] = 0.0;
    for (int i = threadIdx.x; i < N; i += T) {
        const int t = a.types ? a.types[i] : 0;
#pragma unroll
        for (int gi = 0; gi < 3; gi++) {
            if (gi != t) continue;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const double q = src[(size_t)(3 + k) * N + i] - pbar[gi][k];
                const double qk = q + (out[(size_t)(3 + k) * N + i] - dbar[gi][k]);
                v2[2 * gi] += q * q;
                v2[2 * gi + 1] += qk * qk;
            }
        }
    }
    block_sum<NV2>(v2, red);
    double lam[3];
#pragma unroll
    for (int gi = 0; gi < 3; gi++)
        lam[gi] = (a.keep_energy && red[2 * gi + 1] > 0.0) ? sqrt(red[2 * gi] / red[2 * gi + 1]) : 1.0;

    // pass 3: p'' = pbar + lambda q'
    for (int i = threadIdx.x; i < N; i += T) {
        const int t = a.types ? a.types[i] : 0;
#pragma unroll
        for (int gi = 0; gi < 3; gi++) {
            if (gi != t) continue;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const double q = src[(size_t)(3 + k) * N + i] - pbar[gi][k];
                const double qk = q + (out[(size_t)(3 + k) * N + i] - dbar[gi][k]);
                out[(size_t)(3 + k) * N + i] = pbar[gi][k] + lam[gi] * qk;
            }
        }
    }
}

}  // namespace

cudaError_t launch_kick(const KickArgs &a, int n_copies, cudaStream_t st) {
    const size_t smem = sizeof(double) * NV1 * (1 + KICK_THREADS / 32);
    kick_kernel<<<n_copies, KICK_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ttcf
