// ttcf_spawn.cu -- switch-on of the field for one batch of daughters
// (Figure 1; Algorithm 2 "load system state", "apply mapping", "switch on
// ext. field").  One CTA per mother state.  Kinetic sums, slab modes and
// the results are IEEE double; the pair sums (virial, U) are IEEE double in
// FP64 mode, and in MIXED mode double-float pairs on the FP32 pipe (about
// 48 significand bits; GB300 runs IEEE double at 1/72 of the FP32 rate),
// each candidate first screened in FP32 on the hi parts with a margin:
//   P_ab(0) = (1/V)[sum_i p_a p_b + sum_{i<j} r_ij,a F_ij,b]   (WCA, Eq. 6)
//   B(0)    = P_xy(0) of each mapped daughter: a reflection of x or of y
//             negates it exactly, time reversal and the z-reflection keep
//             it, the x <-> z exchange makes it the mother's P_zy (Eq. 3)
//   Omega   = -gamma V B(0) / (k_B T)                        (Eq. 7)
// so sum over the group of Omega(0) and of B(0) is exactly zero.  Under
// planar elongational flow (grad u = diag(eps, 0, -eps)) B(0) = P_xx(0) -
// P_zz(0) instead: reflections and time reversal keep it, the x <-> z
// exchange negates it, and Omega = -eps V B(0) / (k_B T).
#include "ttcf_internal.h"

namespace ttcf {

constexpr int NACC = 13;   // K_ab (6), W_ab (6), U

size_t spawn_smem_bytes(int N, int ncell) {
    return (size_t)N * 24 + (size_t)(2 * ncell + 2) * 4 + ((size_t)N * 2 + 15) / 16 * 16 +
           32 * NACC * 8 + 256;
}

// Reciprocal of a double-float: the float reciprocal and one Newton step
// in double-float (about 2^-44 relative).
__device__ __forceinline__ df df_rcp(df a) {
    const float y = __frcp_rn(a.hi);
    const df e = df_add_f(df_neg(df_mul_f(a, y)), 1.0f);   // 1 - a y
    return df_add_f(df_mul_f(e, y), y);                      // y + y (1 - a y)
}

__global__ void spawn_kernel(SpawnArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = blockIdx.x, tid = threadIdx.x, T = blockDim.x;
    const int N = a.N;
    const double *src = a.src + (size_t)g * 6 * N;
    // positions, 24 bytes per atom: IEEE doubles (FP64 mode) or double-float
    // pairs as hi and lo rows (MIXED)
    double *xd = (double *)smem, *yd = xd + N, *zd = yd + N;
    float *xh = (float *)smem, *yh = xh + N, *zh = yh + N, *xl = zh + N, *yl = xl + N, *zl = yl + N;
    int *cnt = (int *)(zl + N);
    int *start = cnt + a.ncell;
    unsigned short *catom = (unsigned short *)(start + a.ncell + 2);
    double *red = (double *)((unsigned char *)catom + ((size_t)N * 2 + 15) / 16 * 16);
    int *warp_tmp = (int *)(red + 32 * NACC);

    const double invL[3] = {1.0 / a.L[0], 1.0 / a.L[1], 1.0 / a.L[2]};
    // the mother into the daughter kernel's state format; in MIXED the same
    // float pairs are this pass's positions (one conversion per value)
    unsigned long long *dst = a.mothers + (size_t)g * 6 * N;
    for (int e = tid; e < 6 * N; e += T) {
        const double v = src[e];
        if (a.mixed) {
            const df q = df_from_double(v);
            reinterpret_cast<float2 *>(dst)[e] = make_float2(q.hi, q.lo);
            if (e < 3 * N) { xh[e] = q.hi; xh[3 * N + e] = q.lo; }   // rows x, y, z: hi, then lo
        } else {
            reinterpret_cast<double *>(dst)[e] = v;
            if (e < 3 * N) xd[e] = v;
        }
    }
    for (int c = tid; c < a.ncell; c += T) cnt[c] = 0;
    __syncthreads();
    auto cell3 = [&](int i, int &cx, int &cy, int &cz) {   // binning in IEEE double
        const double xi = src[i], yi = src[N + i], zi = src[2 * N + i];
        double y = yi - a.L[1] * rint(yi * invL[1]);
        double x = xi - rint(yi * invL[1]) * a.delta;
        x -= a.L[0] * rint(x * invL[0]);
        double z = zi - a.L[2] * rint(zi * invL[2]);
        cx = min(max((int)floor((x + 0.5 * a.L[0]) * a.nc[0] * invL[0]), 0), a.nc[0] - 1);
        cy = min(max((int)floor((y + 0.5 * a.L[1]) * a.nc[1] * invL[1]), 0), a.nc[1] - 1);
        cz = min(max((int)floor((z + 0.5 * a.L[2]) * a.nc[2] * invL[2]), 0), a.nc[2] - 1);
    };
    // counting sort of atoms into cells (N <= 4096 -> at most 16 per thread)
    int slot[16], cid[16];
    for (int q = 0, i = tid; i < N; i += T, q++) {
        int cx, cy, cz;
        cell3(i, cx, cy, cz);
        cid[q] = (cz * a.nc[1] + cy) * a.nc[0] + cx;
        slot[q] = atomicAdd(&cnt[cid[q]], 1);
    }
    __syncthreads();
    cta_exclusive_scan(cnt, start, a.ncell, warp_tmp);
    __syncthreads();
    for (int q = 0, i = tid; i < N; i += T, q++) catom[start[cid[q]] + slot[q]] = (unsigned short)i;
    __syncthreads();
    // atomic slots depend on scheduling: sort each cell so that the double
    // sums below run in one fixed order (bitwise reproducible B(0), Omega)
    for (int c = tid; c < a.ncell; c += T) {
        for (int u = start[c] + 1; u < start[c + 1]; u++) {
            const unsigned short v = catom[u];
            int w = u;
            while (w > start[c] && catom[w - 1] > v) { catom[w] = catom[w - 1]; w--; }
            catom[w] = v;
        }
    }
    __syncthreads();

    // partial sums: kinetic K_ab (6), virial W_ab (6), U in IEEE double;
    // in MIXED the pair sums of a thread's atoms run in double-float pairs
    // on the FP32 pipe (pwt) and are converted once (on GB300 the FP64 pipe,
    // conversions included, is the bound of this pass).  The CTA reduction
    // is IEEE double in both modes.
    double acc[NACC];
    for (int k = 0; k < NACC; k++) acc[k] = 0.0;
    df pwt[7];
    for (int k = 0; k < 7; k++) pwt[k] = df_make(0.f);
    const double rc2 = 1.2599210498948732;
    const float rc2_screen = 1.2599210498948732f * (1.0f + 1e-4f);   // hi parts: |error| << 1e-4 r_c^2
    const float Lf[3] = {(float)a.L[0], (float)a.L[1], (float)a.L[2]};
    const float invLf[3] = {(float)invL[0], (float)invL[1], (float)invL[2]};
    const float deltaf = (float)a.delta;
    const df Ld[3] = {df_from_double(a.L[0]), df_from_double(a.L[1]), df_from_double(a.L[2])};
    const df deltad = df_from_double(a.delta);
    const df rc2d = df_from_double(rc2);
    for (int q = 0, i = tid; i < N; i += T, q++) {
        const double px = src[3 * N + i], py = src[4 * N + i], pz = src[5 * N + i];
        acc[0] += px * px; acc[1] += py * py; acc[2] += pz * pz;
        acc[3] += px * py; acc[4] += px * pz; acc[5] += py * pz;
        // the cell from the binning pass (same atoms, same order)
        const int cx = cid[q] % a.nc[0], cy = (cid[q] / a.nc[0]) % a.nc[1], cz = cid[q] / (a.nc[0] * a.nc[1]);
        if (!a.mixed) {   // FP64 mode: the pair sums in IEEE double
            for (int oy = -1; oy <= 1; oy++) {
                int yy = cy + oy;
                const int cross = yy < 0 ? -1 : (yy >= a.nc[1] ? 1 : 0);
                yy = (yy + a.nc[1]) % a.nc[1];
                const int x0 = cross ? 0 : cx - 1, x1 = cross ? a.nc[0] - 1 : cx + 1;
                for (int oz = -1; oz <= 1; oz++) {
                    const int zz = (cz + oz + a.nc[2]) % a.nc[2];
                    for (int xc = x0; xc <= x1; xc++) {
                        const int xx = ((xc % a.nc[0]) + a.nc[0]) % a.nc[0];
                        const int c = (zz * a.nc[1] + yy) * a.nc[0] + xx;
                        for (int t = start[c]; t < start[c + 1]; t++) {
                            const int j = catom[t];
                            if (j == i) continue;
                            double dx = xd[i] - xd[j], dy = yd[i] - yd[j], dz = zd[i] - zd[j];
                            const double ny = rint(dy * invL[1]);
                            dy -= ny * a.L[1]; dx -= ny * a.delta;
                            dx -= rint(dx * invL[0]) * a.L[0];
                            dz -= rint(dz * invL[2]) * a.L[2];
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 < rc2) {
                                const double sv = 1.0 / r2, s3 = sv * sv * sv;
                                const double f = s3 * sv * (48.0 * s3 - 24.0);
                                acc[6] += 0.5 * f * dx * dx; acc[7] += 0.5 * f * dy * dy;
                                acc[8] += 0.5 * f * dz * dz; acc[9] += 0.5 * f * dx * dy;
                                acc[10] += 0.5 * f * dx * dz; acc[11] += 0.5 * f * dy * dz;
                                acc[12] += 0.5 * (4.0 * s3 * (s3 - 1.0) + 1.0);
                            }
                        }
                    }
                }
            }
            continue;
        }
        // pair sums as double-float pairs: 0.5 f d_a d_b, 0.5 U
        const df xi = {xh[i], xl[i]}, yi = {yh[i], yl[i]}, zi = {zh[i], zl[i]};
        for (int oy = -1; oy <= 1; oy++) {
            int yy = cy + oy;
            const int cross = yy < 0 ? -1 : (yy >= a.nc[1] ? 1 : 0);
            yy = (yy + a.nc[1]) % a.nc[1];
            // rows across the y face: scan the whole row (any offset delta)
            const int x0 = cross ? 0 : cx - 1, x1 = cross ? a.nc[0] - 1 : cx + 1;
            for (int oz = -1; oz <= 1; oz++) {
                const int zz = (cz + oz + a.nc[2]) % a.nc[2];
                for (int xc = x0; xc <= x1; xc++) {
                    const int xx = ((xc % a.nc[0]) + a.nc[0]) % a.nc[0];
                    const int c = (zz * a.nc[1] + yy) * a.nc[0] + xx;
                    for (int t = start[c]; t < start[c + 1]; t++) {
                        const int j = catom[t];
                        if (j == i) continue;
                        // FP32 screen on the hi parts: the periodic and
                        // Lees-Edwards images, and r^2 with a margin
                        float dyf = yh[i] - yh[j];
                        const float ny = rintf(dyf * invLf[1]);
                        dyf = __fmaf_rn(-ny, Lf[1], dyf);
                        float dxf = __fmaf_rn(-ny, deltaf, xh[i] - xh[j]);
                        const float nx = rintf(dxf * invLf[0]);
                        dxf = __fmaf_rn(-nx, Lf[0], dxf);
                        float dzf = zh[i] - zh[j];
                        const float nz = rintf(dzf * invLf[2]);
                        dzf = __fmaf_rn(-nz, Lf[2], dzf);
                        if (dxf * dxf + dyf * dyf + dzf * dzf >= rc2_screen) continue;
                        // the pair in double-float with the same images
                        const df dy = df_add(df_add(yi, df_neg({yh[j], yl[j]})), df_mul_f(Ld[1], -ny));
                        const df dx = df_add(df_add(df_add(xi, df_neg({xh[j], xl[j]})), df_mul_f(deltad, -ny)),
                                             df_mul_f(Ld[0], -nx));
                        const df dz = df_add(df_add(zi, df_neg({zh[j], zl[j]})), df_mul_f(Ld[2], -nz));
                        const df r2 = df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz));
                        if (!df_lt(r2, rc2d)) continue;
                        const df sv = df_rcp(r2);
                        const df s3 = df_mul(df_mul(sv, sv), sv);
                        const df hf = df_mul_f(df_mul(df_mul(s3, sv), df_add_f(df_mul_f(s3, 48.0f), -24.0f)), 0.5f);
                        const df hx = df_mul(hf, dx), hy = df_mul(hf, dy);
                        pwt[0] = df_add(pwt[0], df_mul(hx, dx)); pwt[1] = df_add(pwt[1], df_mul(hy, dy));
                        pwt[2] = df_add(pwt[2], df_mul(df_mul(hf, dz), dz)); pwt[3] = df_add(pwt[3], df_mul(hx, dy));
                        pwt[4] = df_add(pwt[4], df_mul(hx, dz)); pwt[5] = df_add(pwt[5], df_mul(hy, dz));
                        // 0.5 (4 s3 (s3 - 1) + 1)
                        pwt[6] = df_add(pwt[6], df_mul_f(df_add_f(df_mul_f(df_mul(s3, df_add_f(s3, -1.0f)), 4.0f), 1.0f),
                                                       0.5f));
                    }
                }
            }
        }
    }
    if (a.mixed)
        for (int k = 0; k < 7; k++) acc[6 + k] = df_to_double(pwt[k]);
    // fixed-order CTA reduction
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    for (int k = 0; k < NACC; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * NACC + k] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double tot[NACC];
        for (int k = 0; k < NACC; k++) {
            double v = 0.0;
            for (int w = 0; w < nw; w++) v += red[w * NACC + k];
            tot[k] = v;
        }
        const double pxy = (tot[3] + tot[9]) / a.V, pyz = (tot[5] + tot[11]) / a.V;
        const double pxz = ((tot[0] + tot[6]) - (tot[2] + tot[8])) / a.V;   // P_xx - P_zz
        const double gm = a.gamma[g];
        for (int k = 0; k < a.M; k++) {
            const int m = a.maps[k];
            const double b0 = a.elong ? (map_swaps_xz(m) ? -pxz : pxz)
                                      : map_pxy_sign(m) * (map_swaps_xz(m) ? pyz : pxy);
            const size_t d = (size_t)g * a.M + k;
            a.B[d * a.S] = b0;
            a.Omega[d] = -gm * a.V * b0 / a.T;
        }
        if (a.feat) {   // raw features of the unmapped mother (FEAT_RAW doubles)
            double *f = a.feat + (size_t)g * FEAT_RAW;
            for (int k = 0; k < 12; k++) f[k] = tot[k];          // K_ab, W_ab
            f[12] = tot[12];                                      // U
            f[13] = tot[0] + tot[1] + tot[2];                     // sum p^2
            for (int u = 14; u < FEAT_RAW; u++) f[u] = 0.0;   // (the slab modes: features kernel)
        }
    }
}

cudaError_t launch_spawn(const SpawnArgs &a, cudaStream_t st) {
    const size_t smem = spawn_smem_bytes(a.N, a.ncell);
    cudaError_t e = cudaFuncSetAttribute(spawn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    spawn_kernel<<<a.G, 256, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ttcf
