// ttcf_reduce.cu -- ensemble averages of one batch, IEEE double, fixed
// summation order (bitwise reproducible).
//
// Per mother group g (M mapped daughters m, Eq. 3):
//   Y_g(s) = (1/M) sum_m Omega_m(0) B_m(s)      group integrand (Eq. 2)
//   D_g(s) = (1/M) sum_m B_m(s)                 group direct average
//   J_g(s) = D_g(0) + trapezoid int_0^s Y_g     group TTCF estimate (Eq. 1)
//   O_g    = (1/M) sum_m Omega_m(0)
// Ensemble: means over the groups whose daughters all finished, standard
// errors std_g / sqrt(G) (ddof 1), and the Eq. 4 form
//   corr_c(s) = corr(s) - <Omega(0)> dav(s),  ttcf_c = dav(0) + int corr_c.
#include <math.h>

#include "ttcf_internal.h"

namespace ttcf {

// pass 1: one CTA per group, threads over samples
__global__ void reduce_groups_kernel(ReduceArgs a) {
    __shared__ double wtmp[32];
    const int g = blockIdx.x, o = blockIdx.y, tid = threadIdx.x, T = blockDim.x;
    const int M = a.M, S = a.S, K = a.n_obs;
    const size_t d0 = (size_t)g * M;
    int ok = 1;
    for (int k = 0; k < M; k++) ok &= (a.status[d0 + k] == 0);
    double om[MAX_MAPS];
    for (int k = 0; k < M; k++) om[k] = a.Omega[d0 + k];
    const size_t w0 = ((size_t)o * a.G + g) * S;
    double *Y = a.Y + w0, *D = a.Dg + w0, *J = a.J + w0;
    const double invM = 1.0 / M;
    for (int s = tid; s < S; s += T) {
        double y = 0.0, dsum = 0.0;
        for (int k = 0; k < M; k++) {
            const double bv = a.B[((d0 + k) * K + o) * S + s];
            y += om[k] * bv;
            dsum += bv;
        }
        Y[s] = y * invM;
        D[s] = dsum * invM;
    }
    __syncthreads();
    // J = D(0) + cumulative trapezoid of Y: chunked CTA scan
    const int per = (S + T - 1) / T;
    const int b0 = min(tid * per, S), b1 = min(b0 + per, S);
    double loc = 0.0;
    for (int s = max(b0, 1); s < b1; s++) loc += 0.5 * a.ds * (Y[s - 1] + Y[s]);
    double incl = warp_incl_scan(loc);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 31) wtmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const double v = lane < (T >> 5) ? wtmp[lane] : 0.0;
        const double vi = warp_incl_scan(v);
        if (lane < (T >> 5)) wtmp[lane] = vi - v;
    }
    __syncthreads();
    double run = D[0] + wtmp[warp] + incl - loc;
    for (int s = b0; s < b1; s++) {
        if (s >= 1) run += 0.5 * a.ds * (Y[s - 1] + Y[s]);
        J[s] = run;
    }
    if (tid == 0 && o == 0) {
        double os = 0.0;
        for (int k = 0; k < M; k++) os += om[k];
        a.Og[g] = os * invM;
        a.valid[g] = ok ? 1.0 : 0.0;
    }
}

// pass 2: one thread per sample, groups summed in index order (two passes)
__global__ void reduce_samples_kernel(ReduceArgs a) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.S) return;
    const int G = a.G, S = a.S, o = blockIdx.y;
    const double *Yb = a.Y + (size_t)o * G * S, *Db = a.Dg + (size_t)o * G * S, *Jb = a.J + (size_t)o * G * S;
    double *out = a.out + (size_t)o * 9 * S;
    double n = 0.0, sy = 0.0, sd = 0.0, sj = 0.0;
    for (int g = 0; g < G; g++) {
        const double v = a.valid[g];
        if (v == 0.0) continue;
        n += 1.0;
        sy += Yb[(size_t)g * S + s]; sd += Db[(size_t)g * S + s]; sj += Jb[(size_t)g * S + s];
    }
    const double my = sy / n, md = sd / n, mj = sj / n;
    double vy = 0.0, vd = 0.0, vj = 0.0;
    for (int g = 0; g < G; g++) {
        if (a.valid[g] == 0.0) continue;
        const double ey = Yb[(size_t)g * S + s] - my;
        const double ed = Db[(size_t)g * S + s] - md;
        const double ej = Jb[(size_t)g * S + s] - mj;
        vy += ey * ey; vd += ed * ed; vj += ej * ej;
    }
    const double se = n > 1.0 ? 1.0 / sqrt(n * (n - 1.0)) : NAN;
    out[0 * S + s] = my; out[1 * S + s] = sqrt(vy) * se;
    out[2 * S + s] = md; out[3 * S + s] = sqrt(vd) * se;
    out[4 * S + s] = mj; out[5 * S + s] = sqrt(vj) * se;
    out[8 * S + s] = n;
}

// pass 3: <Omega(0)> and the Eq. 4 form (one thread, sequential)
__global__ void reduce_correct_kernel(ReduceArgs a) {
    if (threadIdx.x != 0) return;
    const int S = a.S, o = blockIdx.x;
    double n = 0.0, so = 0.0;
    for (int g = 0; g < a.G; g++)
        if (a.valid[g] != 0.0) { n += 1.0; so += a.Og[g]; }
    const double om = so / n;
    if (o == 0) { a.Og[a.G] = om; a.Og[a.G + 1] = n; }   // read by ttcf_omega_mean
    double *out = a.out + (size_t)o * 9 * S;
    const double *corr = out, *dav = out + 2 * S;
    double *cc = out + 6 * S, *tc = out + 7 * S;
    double run = dav[0];
    for (int s = 0; s < S; s++) {
        cc[s] = corr[s] - om * dav[s];
        if (s >= 1) run += 0.5 * a.ds * (cc[s - 1] + cc[s]);
        tc[s] = run;
    }
}

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t st) {
    reduce_groups_kernel<<<dim3(a.G, a.n_obs), 256, 0, st>>>(a);
    reduce_samples_kernel<<<dim3((a.S + 127) / 128, a.n_obs), 128, 0, st>>>(a);
    reduce_correct_kernel<<<a.n_obs, 32, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------- equilibrium correlations --
// Time autocorrelation of the series B[g][s0 .. s0+n) of G trajectories,
// averaged over trajectories and time origins (one CTA per lag, fixed-order
// sums):  acf[k]  = <B(t) B(t+k)>,
//         acf2[k] = <(B^2(t) - m2)(B^2(t+k) - m2)>,  m2 = <B^2>.
__device__ double block_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += sh[w];
    __syncthreads();
    return t;   // valid in thread 0
}

__global__ void acf_mean2_kernel(const double *B, int G, int S, int s0, int n, double *m2) {
    __shared__ double sh[32];
    double v = 0.0;
    for (long long q = threadIdx.x; q < (long long)G * n; q += blockDim.x) {
        const double b = B[(q / n) * S + s0 + q % n];
        v += b * b;
    }
    const double t = block_sum(v, sh);
    if (threadIdx.x == 0) *m2 = t / ((double)G * n);
}

__global__ void acf_kernel(const double *B, int G, int S, int s0, int n, const double *m2p,
                           double *acf, double *acf2) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    const int m = n - k;   // time origins at lag k
    const double m2 = *m2p;
    double v1 = 0.0, v2 = 0.0;
    for (long long q = threadIdx.x; q < (long long)G * m; q += blockDim.x) {
        const double *b = B + (q / m) * S + s0 + q % m;
        const double a0 = b[0], ak = b[k];
        v1 += a0 * ak;
        v2 += (a0 * a0 - m2) * (ak * ak - m2);
    }
    const double t1 = block_sum(v1, sh);
    const double t2 = block_sum(v2, sh);
    if (threadIdx.x == 0) {
        acf[k] = t1 / ((double)G * m);
        acf2[k] = t2 / ((double)G * m);
    }
}

cudaError_t launch_acf(const double *B, int G, int S, int s0, int n, int max_lag, double *acf,
                       double *acf2, double *m2, cudaStream_t st) {
    acf_mean2_kernel<<<1, 256, 0, st>>>(B, G, S, s0, n, m2);
    acf_kernel<<<max_lag + 1, 256, 0, st>>>(B, G, S, s0, n, m2, acf, acf2);
    return cudaGetLastError();
}

// ----------------------------------------------- equilibrium friction --
__global__ void slip_force_kernel(SlipArgs a) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)a.D * a.S) return;
    const int d = (int)(q / a.S), s = (int)(q % a.S);
    double dv = 0.0, F = 0.0;
    if (a.status[d] == 0) {
        const double *b = a.B + (size_t)d * a.n_obs * a.S;
        double P = 0.0, n = 0.0;
        for (int j = 0; j < a.n_slabs; j++) {
            P += b[(size_t)(2 + a.slabs[j]) * a.S + s];
            n += b[(size_t)(2 + a.nslab + a.slabs[j]) * a.S + s];
        }
        dv = b[(size_t)(2 + 2 * a.nslab + a.wall) * a.S + s] / a.n_layer - (n > 0.0 ? P / n : 0.0);
        F = -a.area * b[(size_t)a.wall * a.S + s];
    }
    a.dv[q] = dv;
    a.F[q] = F;
}

// One CTA per lag k: sums over valid daughters and origins t = 0 .. S-1-k.
__global__ void slip_xcorr_kernel(SlipArgs a, double *c_dvf, double *c_dvdv) {
    __shared__ double sh[32];
    __shared__ int nvalid_s;
    const int k = blockIdx.x, m = a.S - k;
    if (threadIdx.x == 0) {
        int nv = 0;
        for (int d = 0; d < a.D; d++) nv += a.status[d] == 0;
        nvalid_s = nv;
    }
    double v1 = 0.0, v2 = 0.0;
    for (long long q = threadIdx.x; q < (long long)a.D * m; q += blockDim.x) {
        const size_t d = (size_t)(q / m), t = (size_t)(q % m);
        const double x = a.dv[d * a.S + t];
        v1 += x * a.F[d * a.S + t + k];
        v2 += x * a.dv[d * a.S + t + k];
    }
    const double t1 = block_sum(v1, sh);
    const double t2 = block_sum(v2, sh);
    if (threadIdx.x == 0) {
        const double cnt = (double)nvalid_s * m;
        c_dvf[k] = cnt > 0 ? t1 / cnt : NAN;
        c_dvdv[k] = cnt > 0 ? t2 / cnt : NAN;
    }
}

cudaError_t launch_slip_correlations(const SlipArgs &a, int max_lag, double *c_dvf, double *c_dvdv,
                                     cudaStream_t st) {
    const long long n = (long long)a.D * a.S;
    slip_force_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    slip_xcorr_kernel<<<max_lag + 1, 256, 0, st>>>(a, c_dvf, c_dvdv);
    return cudaGetLastError();
}

}  // namespace ttcf
