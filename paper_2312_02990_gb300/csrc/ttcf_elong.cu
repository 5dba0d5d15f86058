// ttcf_elong.cu -- daughters under planar elongational flow.
//
// The WCA fluid of Example 1 driven by the other homogeneous field that the
// paper's introduction names beside shear: grad u = diag(eps, 0, -eps)
// (stretching along x, compression along z, constant volume) in a periodic
// box that deforms with the flow, Lx(t) = Lx(0) e^{eps t}, Lz(t) = Lz(0)
// e^{-eps t}.  These are the Eq. 5 equations of motion with this grad u:
//   r' = p + (eps x, 0, -eps z),   p' = F - (eps px, 0, -eps pz) - alpha p,
// split as the shear daughters are, E D C' B A' B C' D E, with each part
// solved exactly:
//   E : alpha <- alpha + tau (sum p^2 - g T) / Q
//   D : p <- p e^{-alpha tau}
//   C': px <- px e^{-eps tau}, pz <- pz e^{eps tau}
//   B : p <- p + tau F
//   A': x <- x e^{eps h} + px (e^{eps h} - 1)/eps, y <- y + py h,
//       z <- z e^{-eps h} + pz (1 - e^{-eps h})/eps, then one periodic
//       wrap into the box of the new time.
// The response is B = P_xx - P_zz; the spawn kernel gives B(0) and
// Omega = -eps V B(0) / (k_B T) in IEEE double (Omega = beta dH^ad/dt with
// dH^ad/dt = -V grad u : P).
//
// Layout: one CTA per daughter, the whole daughter in shared memory (the
// phase point as 8-byte slots, forces, a cell-ordered copy of the
// positions).  The box changes every step, so the cell grid (cells at
// least r_c wide) is rebuilt from the new box every step: a counting sort
// of the atoms into cells, each cell put in index order (atomic slots
// depend on scheduling; the order fixes the force sums bit for bit), and a
// force pass over the 27 neighbour cells with one periodic image shift per
// cell.  The force pass takes atoms in cell order, so that neighbouring
// lanes scan nearly the same cells; the integrator passes take them in
// index order.  A grid with fewer than three cells along an axis visits the
// same cell under two or three shifts, each a distinct image: with every box
// edge above 2 r_c at most one of them lies within r_c.
// MIXED: double-float phase point, FP32 pairs, the per-step sums in exact
// 64-bit fixed point; FP64: IEEE double throughout.
#include <algorithm>
#include <type_traits>

#include "ttcf_internal.h"

namespace ttcf {

namespace {

constexpr double RC = 1.1224620483093730;          // 2^(1/6)
constexpr double CELL_MIN = RC * (1.0 + 1e-4);     // smallest cell width

// A cell-ordered position of the FP64 mode (index in w).
struct alignas(16) Pd { double x, y, z, w; };

__device__ __forceinline__ int idx_of(const float4 &p) { return __float_as_int(p.w); }
__device__ __forceinline__ int idx_of(const Pd &p) { return (int)p.w; }
__device__ __forceinline__ float4 make_p4(float x, float y, float z, int i) {
    return make_float4(x, y, z, __int_as_float(i));
}
__device__ __forceinline__ Pd make_p4(double x, double y, double z, int i) { return {x, y, z, (double)i}; }

__device__ __forceinline__ df sexpm1(df x, df sixth) { return df_expm1_small(x, sixth); }
__device__ __forceinline__ double sexpm1(double x, double) { return expm1_small(x); }
__device__ __forceinline__ bool sge(df a, df b) { return df_ge(a, b); }
__device__ __forceinline__ bool sge(double a, double b) { return a >= b; }

// Arithmetic with every rounding explicit (no multiply-add contraction):
// the start-up pass and the step loop compute forces, sums and the
// thermostat chain in separately inlined copies, and a chunked run must
// reproduce an uninterrupted one bit for bit.
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ df xadd(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ double xadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ df xmul(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ df xmulf(df a, float b) { return df_mul_f(a, b); }
__device__ __forceinline__ double xmulf(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ df xone_plus(df x) { return df_add_f(x, 1.0f); }
__device__ __forceinline__ double xone_plus(double x) { return __dadd_rn(1.0, x); }

// One periodic wrap into [-L/2, L/2).
template <class S>
__device__ __forceinline__ S wrap_once(S v, S L, S halfL) {
    if (sge(v, halfL)) return xadd(v, sneg(L));
    if (!sge(v, sneg(halfL))) return xadd(v, L);
    return v;
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) / 16 * 16; }

}  // namespace

// Per-daughter scalars, written by thread 0.
template <class S>
struct ElongScal {
    S alpha;                 // Nose-Hoover multiplier at the end of the last step
    S alpha_mid;             // after the opening E flow of the current step
    S c;                     // e^{-alpha_mid h/2}: the D flows of the current step
    S Lx, Lz;                // box edges of the current positions
    S Lx1, Lz1, hLx1, hLz1;  // box edges one step later and their halves
    S Ly, hLy;
    S ex, ez, phx, phz;      // drift factors e^{+-eps h} and (e^{+-eps h} - 1)/(+-eps)
    S cxh, czh;              // C' factors e^{-eps h/2}, e^{eps h/2}
    S h, hh, hhQ, ngT, nhh, sixth;
    double invV;
    S Lg[3];                 // box edges of the grid (image shifts of the force pass)
    float Lf[3];             // the same in float (binning)
    float sf[3];             // cells per unit length
    int nc[3], ncell;
    int stop;                // TTCF_D_* flags of the daughter
    int flag_lost;           // a per-step sum out of the fixed-point range
    unsigned long long pairs;
    long long slot[MAX_WARPS][2];   // reduction slots (fixed point, or double bits)
};

size_t elong_smem_bytes(bool mixed, int N, int ncellmax) {
    const size_t rsz = mixed ? 4 : 8;
    size_t b = (size_t)6 * N * 8;                 // phase point slots
    b += align16((size_t)3 * N * rsz);            // forces
    b += (size_t)N * (mixed ? 16 : 32);           // cell-ordered positions
    b += 2 * align16((size_t)N * 4);              // cell and slot of each atom
    b += align16((size_t)ncellmax * 4) + align16((size_t)(ncellmax + 2) * 4);
    b += align16(mixed ? sizeof(ElongScal<df>) : sizeof(ElongScal<double>));
    b += 32 * 4 + 16;                             // scan scratch
    return b;
}

int elong_threads(int N) {
    const int t = ((N + 1) / 2 + 31) / 32 * 32;
    return t < 128 ? 128 : (t > 512 ? 512 : t);
}

namespace {

template <bool MIXED>
__device__ void elong_daughter(const ElongArgs &a, int d, unsigned char *smem) {
    using S = typename std::conditional<MIXED, df, double>::type;    // state scalar
    using R = typename std::conditional<MIXED, float, double>::type; // pair arithmetic
    using P4 = typename std::conditional<MIXED, float4, Pd>::type;
    const int tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const BatchDev &b = a.b;
    const int N = b.N;
    const int gl = d / b.M;
    const int map = b.maps[d % b.M];
    const double eps = b.gamma[gl];
    const int ncm = a.ncmax[0] * a.ncmax[1] * a.ncmax[2];

    // shared-memory carve-up (elong_smem_bytes mirrors it)
    unsigned char *sp = smem;
    unsigned long long *st = (unsigned long long *)sp; sp += (size_t)6 * N * 8;
    R *F = (R *)sp; sp += align16((size_t)3 * N * sizeof(R));
    P4 *cpos = (P4 *)sp; sp += (size_t)N * sizeof(P4);
    int *cellof = (int *)sp; sp += align16((size_t)N * 4);
    int *rank = (int *)sp; sp += align16((size_t)N * 4);
    int *cnt = (int *)sp; sp += align16((size_t)ncm * 4);
    int *start = (int *)sp; sp += align16((size_t)(ncm + 2) * 4);
    ElongScal<S> *m = (ElongScal<S> *)sp; sp += align16(sizeof(ElongScal<S>));
    int *warp_tmp = (int *)sp;

    // the cell grid of a box (thread 0): cells at least CELL_MIN wide, at
    // most the planned bound per axis (fewer cells are wider, still valid)
    auto set_grid = [&](S Lx, S Lz) {
        m->Lg[0] = Lx; m->Lg[1] = m->Ly; m->Lg[2] = Lz;
        m->Lf[0] = (float)shi(Lx); m->Lf[1] = (float)b.L[1]; m->Lf[2] = (float)shi(Lz);
        int nct = 1;
        for (int k = 0; k < 3; k++) {
            int n = (int)(m->Lf[k] * (float)(1.0 / CELL_MIN));
            n = n < 1 ? 1 : (n > a.ncmax[k] ? a.ncmax[k] : n);
            m->nc[k] = n;
            m->sf[k] = (float)n / m->Lf[k];
            nct *= n;
        }
        m->ncell = nct;
    };

    if (tid == 0) {
        const double h = a.dt, hh = 0.5 * a.dt;
        m->stop = 0; m->flag_lost = 0; m->pairs = 0ull;
        m->ex = sfrom<S>(exp(eps * h));
        m->ez = sfrom<S>(exp(-eps * h));
        m->phx = sfrom<S>(eps != 0.0 ? expm1(eps * h) / eps : h);
        m->phz = sfrom<S>(eps != 0.0 ? expm1(-eps * h) / (-eps) : h);
        m->cxh = sfrom<S>(exp(-eps * hh));
        m->czh = sfrom<S>(exp(eps * hh));
        m->h = sfrom<S>(h); m->hh = sfrom<S>(hh);
        m->hhQ = sfrom<S>(hh / b.Q); m->ngT = sfrom<S>(-b.gT);
        m->nhh = sfrom<S>(-hh); m->sixth = sfrom<S>(1.0 / 6.0);
        m->Ly = sfrom<S>(b.L[1]); m->hLy = sfrom<S>(0.5 * b.L[1]);
        m->invV = 1.0 / b.V;
        if (a.fresh) {
            const double sa = map_reverses_time(map) ? -1.0 : 1.0;
            m->alpha = sfrom<S>(a.reset_alpha ? 0.0 : sa * b.m_alpha[gl]);
            m->Lx = sfrom<S>(b.L[0]);
            m->Lz = sfrom<S>(b.L[2]);
        } else {   // the loop state of an earlier chunk: the run continues bit for bit
            const unsigned long long *sc = reinterpret_cast<const unsigned long long *>(b.scal) + 4 * (size_t)d;
            m->alpha = load_slot<S>(sc);
            m->Lx = load_slot<S>(sc + 1);
            m->Lz = load_slot<S>(sc + 2);
        }
        set_grid(m->Lx, m->Lz);
    }
    for (int c = tid; c < ncm; c += T) cnt[c] = 0;
    __syncthreads();

    // ---- the phase point: the mapped mother (codes as for shear), or the
    //      saved loop state ----
    {
        const int mp = a.fresh ? map : 0;
        const unsigned long long *src = a.fresh ? b.mothers + (size_t)gl * 6 * N
                                                : b.state + (size_t)d * 6 * N;
        const S L0[3] = {sfrom<S>(b.L[0]), sfrom<S>(b.L[1]), sfrom<S>(b.L[2])};
        const R Lh[3] = {(R)(0.5 * b.L[0]), (R)(0.5 * b.L[1]), (R)(0.5 * b.L[2])};
        auto reflect = [&](S c, int k) {   // -(-L/2) = +L/2 is the periodic point -L/2
            c = sneg(c);
            if (shi(c) >= Lh[k]) c = sadd(c, sneg(L0[k]));
            return c;
        };
        for (int i = tid; i < N; i += T) {
            S x = load_slot<S>(src + i), y = load_slot<S>(src + N + i), z = load_slot<S>(src + 2 * N + i);
            S px = load_slot<S>(src + 3 * N + i), py = load_slot<S>(src + 4 * N + i),
              pz = load_slot<S>(src + 5 * N + i);
            if (map_swaps_xz(mp)) { S t = x; x = z; z = t; t = px; px = pz; pz = t; }
            if (mp & 2) { x = reflect(x, 0); px = sneg(px); }
            if (mp & 4) { y = reflect(y, 1); py = sneg(py); }
            if (mp & 8) { z = reflect(z, 2); pz = sneg(pz); }
            if (map_reverses_time(mp)) { px = sneg(px); py = sneg(py); pz = sneg(pz); }
            store_slot(st + i, x); store_slot(st + N + i, y); store_slot(st + 2 * N + i, z);
            store_slot(st + 3 * N + i, px); store_slot(st + 4 * N + i, py); store_slot(st + 5 * N + i, pz);
        }
    }

    // ---- building blocks ----
    // cell of atom i from its position (hi parts), atomic slot in the cell
    auto bin_atom = [&](int i, R x, R y, R z) {
        const float p[3] = {(float)x, (float)y, (float)z};
        int cc[3];
        for (int k = 0; k < 3; k++) {
            int c = __float2int_rd(__fmul_rn(__fmaf_rn(0.5f, m->Lf[k], p[k]), m->sf[k]));
            cc[k] = c < 0 ? 0 : (c >= m->nc[k] ? m->nc[k] - 1 : c);
        }
        const int c = (cc[2] * m->nc[1] + cc[1]) * m->nc[0] + cc[0];
        cellof[i] = c;
        rank[i] = atomicAdd(&cnt[c], 1);
    };
    // kinetic partials of a thread's atoms (index order): sum p^2 and
    // sum (px^2 - pz^2), from the hi parts in MIXED
    auto kin_partial = [&](R &k2, R &bk) {
        k2 = (R)0; bk = (R)0;
        for (int i = tid; i < N; i += T) {
            const R qx = (R)shi(load_slot<S>(st + 3 * N + i));
            const R qy = (R)shi(load_slot<S>(st + 4 * N + i));
            const R qz = (R)shi(load_slot<S>(st + 5 * N + i));
            k2 = radd(k2, rfma(qz, qz, rfma(qy, qy, rmul(qx, qx))));
            bk = radd(bk, rsub(rmul(qx, qx), rmul(qz, qz)));
        }
    };
    // CTA sums of two per-thread partials, valid in thread 0.  MIXED: 64-bit
    // fixed point of 2^-40 units (exact, order-free; a partial of 2^13 or
    // more, or a non-finite one, marks the daughter non-finite); FP64: a
    // fixed-order double tree.  One __syncthreads.
    auto cta_sum2 = [&](R a0, R a1, S out[2]) {
        if constexpr (MIXED) {
            if (!(fabsf(a0) < 8192.f && fabsf(a1) < 8192.f)) m->flag_lost = 1;
            long long v0 = __float2ll_rn(a0 * 1099511627776.0f), v1 = __float2ll_rn(a1 * 1099511627776.0f);
            for (int o = 16; o > 0; o >>= 1) {
                v0 += __shfl_down_sync(0xffffffffu, v0, o);
                v1 += __shfl_down_sync(0xffffffffu, v1, o);
            }
            if (lane == 0) { m->slot[warp][0] = v0; m->slot[warp][1] = v1; }
            __syncthreads();
            if (warp == 0) {
                long long t0 = lane < nw ? m->slot[lane][0] : 0ll, t1 = lane < nw ? m->slot[lane][1] : 0ll;
                for (int o = 16; o > 0; o >>= 1) {
                    t0 += __shfl_down_sync(0xffffffffu, t0, o);
                    t1 += __shfl_down_sync(0xffffffffu, t1, o);
                }
                if (lane == 0) {
                    auto to_df = [](long long s) -> df {
                        const float hi = __ll2float_rn(s);
                        const float lo = __ll2float_rn(s - __float2ll_rn(hi));
                        return {hi * 9.094947017729282e-13f, lo * 9.094947017729282e-13f};   // x 2^-40
                    };
                    out[0] = to_df(t0);
                    out[1] = to_df(t1);
                }
            }
        } else {
            const double s0 = warp_sum((double)a0), s1 = warp_sum((double)a1);
            if (lane == 0) {
                m->slot[warp][0] = __double_as_longlong(s0);
                m->slot[warp][1] = __double_as_longlong(s1);
            }
            __syncthreads();
            if (warp == 0) {
                double t0 = lane < nw ? __longlong_as_double(m->slot[lane][0]) : 0.0;
                double t1 = lane < nw ? __longlong_as_double(m->slot[lane][1]) : 0.0;
                t0 = warp_sum(t0); t1 = warp_sum(t1);
                if (lane == 0) { out[0] = t0; out[1] = t1; }
            }
        }
    };
    // cell sort, cell-ordered copy, forces into F (the cell counts must be
    // complete); returns the thread's partial of sum over ordered pairs of
    // f (dx^2 - dz^2) and counts the interacting ordered pairs.
    const R rc2 = (R)1.2599210498948732;
    unsigned int npair = 0;
    auto forces = [&]() -> R {
        cta_exclusive_scan(cnt, start, m->ncell, warp_tmp);
        __syncthreads();
        for (int i = tid; i < N; i += T) {
            const R x = (R)shi(load_slot<S>(st + i)), y = (R)shi(load_slot<S>(st + N + i)),
                    z = (R)shi(load_slot<S>(st + 2 * N + i));
            cpos[start[cellof[i]] + rank[i]] = make_p4(x, y, z, i);
        }
        __syncthreads();
        for (int c = tid; c < m->ncell; c += T) {   // each cell in index order
            for (int u = start[c] + 1; u < start[c + 1]; u++) {
                const P4 v = cpos[u];
                int w = u;
                while (w > start[c] && idx_of(cpos[w - 1]) > idx_of(v)) { cpos[w] = cpos[w - 1]; w--; }
                cpos[w] = v;
            }
        }
        __syncthreads();
        const int nc0 = m->nc[0], nc1 = m->nc[1], nc2 = m->nc[2];
        const R Lx = (R)shi(m->Lg[0]), Ly = (R)shi(m->Lg[1]), Lz = (R)shi(m->Lg[2]);
        R wd = (R)0;
        for (int k = tid; k < N; k += T) {
            const P4 pi = cpos[k];
            const int i = idx_of(pi);
            const int c = cellof[i];
            const int cx = c % nc0, cy = (c / nc0) % nc1, cz = c / (nc0 * nc1);
            R fx = (R)0, fy = (R)0, fz = (R)0;
            for (int oz = -1; oz <= 1; oz++) {
                int zc = cz + oz;
                const int kz = zc < 0 ? -1 : (zc >= nc2 ? 1 : 0);
                zc -= kz * nc2;
                const R uz = rfma(-(R)kz, Lz, pi.z);   // i against the image of the cell row
                for (int oy = -1; oy <= 1; oy++) {
                    int yc = cy + oy;
                    const int ky = yc < 0 ? -1 : (yc >= nc1 ? 1 : 0);
                    yc -= ky * nc1;
                    const R uy = rfma(-(R)ky, Ly, pi.y);
                    for (int ox = -1; ox <= 1; ox++) {
                        int xc = cx + ox;
                        const int kx = xc < 0 ? -1 : (xc >= nc0 ? 1 : 0);
                        xc -= kx * nc0;
                        const R ux = rfma(-(R)kx, Lx, pi.x);
                        const int cc = (zc * nc1 + yc) * nc0 + xc;
                        const int t1 = start[cc + 1];
                        for (int t = start[cc]; t < t1; t++) {
                            const P4 pj = cpos[t];
                            const R dx = rsub(ux, pj.x), dy = rsub(uy, pj.y), dz = rsub(uz, pj.z);
                            const R r2 = rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
                            if (r2 < rc2 && idx_of(pj) != i) {
                                const R s = (R)1 / r2;
                                const R s3 = rmul(rmul(s, s), s);
                                const R f = rmul(rmul(s, s3), rfma((R)48, s3, (R)-24));
                                fx = rfma(f, dx, fx); fy = rfma(f, dy, fy); fz = rfma(f, dz, fz);
                                wd = rfma(f, rsub(rmul(dx, dx), rmul(dz, dz)), wd);
                                npair++;
                            }
                        }
                    }
                }
            }
            F[i] = fx; F[N + i] = fy; F[2 * N + i] = fz;
        }
        __syncthreads();
        return wd;
    };
    // thread 0: the box one step on, and its grid (the positions the next
    // drift makes live there)
    auto advance_box = [&]() {
        m->Lx1 = xmul(m->Lx, m->ex);
        m->Lz1 = xmul(m->Lz, m->ez);
        m->hLx1 = xmulf(m->Lx1, (R)0.5);
        m->hLz1 = xmulf(m->Lz1, (R)0.5);
        set_grid(m->Lx1, m->Lz1);
    };
    // thread 0: the opening E flow of a step (alpha at the end of the last
    // step and sum p^2 there) and its D factor
    auto open_step = [&](S inc) {
        m->alpha_mid = xadd(m->alpha, inc);
        m->c = xone_plus(sexpm1(xmul(m->alpha_mid, m->nhh), m->sixth));
    };
    // (sum p^2 - g T) h / (2 Q)
    auto e_increment = [&](S K2) { return xmul(xadd(K2, m->ngT), m->hhQ); };
    // thread 0, after the step's sums: the closing E flow, then the next
    // step's opening one
    auto chain = [&](S K2) {
        const S inc = e_increment(K2);
        m->alpha = xadd(m->alpha_mid, inc);
        open_step(inc);
    };

    // ---- forces and sum p^2 at the starting point ----
    __syncthreads();
    for (int i = tid; i < N; i += T)
        bin_atom(i, (R)shi(load_slot<S>(st + i)), (R)shi(load_slot<S>(st + N + i)),
                 (R)shi(load_slot<S>(st + 2 * N + i)));
    __syncthreads();
    forces();
    npair = 0;   // counted over the steps only
    {
        R k2, bk;
        kin_partial(k2, bk);
        S sums[2];
        cta_sum2(k2, (R)0, sums);
        if (tid == 0) {
            open_step(e_increment(sums[0]));   // the first step's opening E flow
            advance_box();
            if (m->flag_lost || !isfinite(sdbl(sums[0]))) m->stop |= TTCF_D_NONFINITE;
        }
    }
    __syncthreads();

    int steps_run = 0;
    for (int s = a.step0 + 1; s <= a.step1 && !m->stop; s++) {
        // ---- D, C', B half flows, A' drift into the box of step s (Lx1,
        //      Lz1), binning on its grid ----
        for (int c = tid; c < ncm; c += T) cnt[c] = 0;
        __syncthreads();
        {
            const S c = m->c, cxh = m->cxh, czh = m->czh, hh = m->hh;
            const S ex = m->ex, ez = m->ez, phx = m->phx, phz = m->phz, h = m->h;
            const S Lx = m->Lx1, Lz = m->Lz1, hLx = m->hLx1, hLz = m->hLz1, Ly = m->Ly, hLy = m->hLy;
            for (int i = tid; i < N; i += T) {
                S px = load_slot<S>(st + 3 * N + i), py = load_slot<S>(st + 4 * N + i),
                  pz = load_slot<S>(st + 5 * N + i);
                px = xmul(px, c); py = xmul(py, c); pz = xmul(pz, c);
                px = xmul(px, cxh); pz = xmul(pz, czh);
                px = xadd(px, xmulf(hh, F[i]));
                py = xadd(py, xmulf(hh, F[N + i]));
                pz = xadd(pz, xmulf(hh, F[2 * N + i]));
                S x = load_slot<S>(st + i), y = load_slot<S>(st + N + i), z = load_slot<S>(st + 2 * N + i);
                x = wrap_once(xadd(xmul(x, ex), xmul(px, phx)), Lx, hLx);
                y = wrap_once(xadd(y, xmul(py, h)), Ly, hLy);
                z = wrap_once(xadd(xmul(z, ez), xmul(pz, phz)), Lz, hLz);
                store_slot(st + i, x); store_slot(st + N + i, y); store_slot(st + 2 * N + i, z);
                store_slot(st + 3 * N + i, px); store_slot(st + 4 * N + i, py); store_slot(st + 5 * N + i, pz);
                bin_atom(i, (R)shi(x), (R)shi(y), (R)shi(z));
            }
        }
        __syncthreads();
        const R wd = forces();
        // ---- B, C', D half flows with the new forces ----
        {
            const S c = m->c, cxh = m->cxh, czh = m->czh, hh = m->hh;
            for (int i = tid; i < N; i += T) {
                S px = load_slot<S>(st + 3 * N + i), py = load_slot<S>(st + 4 * N + i),
                  pz = load_slot<S>(st + 5 * N + i);
                px = xadd(px, xmulf(hh, F[i]));
                py = xadd(py, xmulf(hh, F[N + i]));
                pz = xadd(pz, xmulf(hh, F[2 * N + i]));
                px = xmul(px, cxh); pz = xmul(pz, czh);
                px = xmul(px, c); py = xmul(py, c); pz = xmul(pz, c);
                store_slot(st + 3 * N + i, px); store_slot(st + 4 * N + i, py); store_slot(st + 5 * N + i, pz);
            }
        }
        R k2, bk;
        kin_partial(k2, bk);
        S sums[2];
        cta_sum2(k2, bk + (R)0.5 * wd, sums);
        steps_run++;
        if (tid == 0) {
            chain(sums[0]);
            const double bv = sdbl(sums[1]) * m->invV;   // P_xx - P_zz
            if (s % a.sample_every == 0) b.B[(size_t)d * b.S + s / a.sample_every] = bv;
            // the positions now live in the box of step s
            m->Lx = m->Lx1;
            m->Lz = m->Lz1;
            advance_box();
            if (m->flag_lost || !isfinite(bv) || !isfinite(sdbl(sums[0]))) m->stop |= TTCF_D_NONFINITE;
            if (a.abort_flag && (s & 63) == 0 && *a.abort_flag) m->stop |= TTCF_D_ABORTED;
        }
        __syncthreads();
    }

    // ---- counters, status, loop state ----
    atomicAdd(&m->pairs, (unsigned long long)npair);
    __syncthreads();
    if (tid == 0) {
        b.pairs[d] += m->pairs;   // ordered pairs, as the other kernels count them
        b.rebuilds[d] += (unsigned int)steps_run;
        if (m->stop) b.status[d] |= m->stop;
        if (a.save_state) {
            unsigned long long *sc = reinterpret_cast<unsigned long long *>(b.scal) + 4 * (size_t)d;
            store_slot(sc, m->alpha);
            store_slot(sc + 1, m->Lx);
            store_slot(sc + 2, m->Lz);
        }
    }
    if (a.save_state) {
        unsigned long long *dst = b.state + (size_t)d * 6 * N;
        for (int e = tid; e < 6 * N; e += T) dst[e] = st[e];
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(512, 2) elong_kernel(const ElongArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long D = (long long)a.b.G * a.b.M;
    for (long long d = blockIdx.x; d < D; d += gridDim.x) {
        elong_daughter<MIXED>(a, (int)d, smem);
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_elong(bool mixed, const ElongArgs &a, int nsm, cudaStream_t st, int *grid_out) {
    const int ncm = a.ncmax[0] * a.ncmax[1] * a.ncmax[2];
    const size_t smem = elong_smem_bytes(mixed, a.b.N, ncm);
    const int T = elong_threads(a.b.N);
    auto fn = mixed ? elong_kernel<true> : elong_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, T, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long D = (long long)a.b.G * a.b.M;
    const long long g = std::min<long long>(D, (long long)nsm * per_sm);
    if (grid_out) *grid_out = (int)g;
    if (g <= 0) return cudaSuccess;
    fn<<<(unsigned)g, T, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ttcf
