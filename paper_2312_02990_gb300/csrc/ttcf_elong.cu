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
// Layout: one CTA per daughter, the whole daughter in shared memory (hi and
// lo parts of the positions, momenta as 8-byte slots, forces, list
// references) except its Verlet lists, which sit in a per-CTA global
// scratch (L2-resident).  The lists hold each atom's neighbours within
// r_l = r_c + skin in index order; the force pass takes every pair at its
// minimum image in the current box, so a list built at any time gives the
// same force sums bit for bit (chunked runs equal uninterrupted ones).
// Because the box deforms, a pair's separation follows the affine flow plus
// the atoms' own displacements u = r - diag(e^{eps dt}, 1, e^{-eps dt}) r0
// since the build; the lists are rebuilt when 2 max|u| reaches
// e^{-|eps| dt} r_l - r_c (the affine flow shrinks distances by at most that
// factor).  Builds bin the atoms into cells at least r_l wide (distinct
// cells only, so an axis with fewer than three cells is scanned once) and
// leave the atoms in cell order, which is the order of the force pass
// (neighbouring lanes then read nearby atoms); the integrator passes take
// atoms in index order, and the per-atom virial terms are summed in index
// order too.
// MIXED: double-float phase point, FP32 pairs, the per-step sums in exact
// 64-bit fixed point; FP64: IEEE double throughout.
#include <algorithm>
#include <type_traits>

#include "ttcf_internal.h"

namespace ttcf {

namespace {

constexpr double RC = 1.1224620483093730;          // 2^(1/6)

// A position (or force and virial term) of the FP64 mode.
struct alignas(16) Pd { double x, y, z, w; };

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
    S Lg[3];                 // box edges of the grid (image shifts of the pair distances)
    double invV;
    float Lf[3], invLf[3];   // the same box in float (binning, image choice)
    float sf[3];             // list cells per unit length
    int nc[3], ncell;
    // Verlet lists: radius r_l = r_c + skin, built from positions r0 at time
    // t0; a pair outside r_l at t0 stays outside r_c while
    // 2 max|u| < e^{-|eps| (t - t0)} r_l - r_c, with u = r - diag(e^{eps(t - t0)},
    // 1, e^{-eps(t - t0)}) r0 (minimum image) the displacement beyond the
    // affine flow
    float rl, rl2;
    float fxa, fza, ea;      // e^{eps (t - t0)}, e^{-eps (t - t0)}, e^{-|eps| (t - t0)} for the next step
    float exf, ezf, eaf;     // their one-step factors
    float thr2;              // rebuild when max |u|^2 >= thr2 (negative: at once)
    unsigned int umax2;      // float bits of this step's max |u|^2
    int rebuild;             // build before the next force pass
    int n_build;
    int stop;                // TTCF_D_* flags of the daughter
    int flag_lost;           // a per-step sum out of the fixed-point range
    unsigned long long pairs;
    long long slot[MAX_WARPS][2];   // reduction slots (fixed point, or double bits)
};

size_t elong_smem_bytes(bool mixed, int N, int ncellmax) {
    size_t b = (size_t)N * 32;                    // positions (hi and lo float4, or double)
    b += align16((size_t)N * 24);                 // momenta (16-byte regions: odd N)
    b += (size_t)N * (mixed ? 16 : 32);           // forces and per-atom virial
    b += (size_t)N * 16;                          // reference positions of the lists
    b += 3 * align16((size_t)N * 2) + align16((size_t)N);   // cell order, cell, slot; list lengths
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
    using R4 = typename std::conditional<MIXED, float4, Pd>::type;
    const int tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const BatchDev &b = a.b;
    const int N = b.N;
    const int gl = d / b.M;
    const int map = b.maps[d % b.M];
    const double eps = b.gamma[gl];
    const int ncm = a.ncmax[0] * a.ncmax[1] * a.ncmax[2];
    // the CTA's lists: [ELONG_CAP / 8][N] groups of 8 uint16 entries
    uint4 *nb4 = reinterpret_cast<uint4 *>(a.nbr + (size_t)blockIdx.x * ELONG_CAP * N);

    // shared-memory carve-up (elong_smem_bytes mirrors it)
    unsigned char *sp = smem;
    float4 *pos4 = nullptr, *plo4 = nullptr;   // MIXED: hi and lo parts of the positions
    Pd *posd = nullptr;                        // FP64
    if constexpr (MIXED) {
        pos4 = (float4 *)sp; plo4 = pos4 + N;
    } else {
        posd = (Pd *)sp;
    }
    sp += (size_t)N * 32;
    unsigned long long *mom = (unsigned long long *)sp; sp += align16((size_t)N * 24);   // [3][N] slots
    R4 *F4 = (R4 *)sp; sp += (size_t)N * sizeof(R4);          // force and per-atom virial
    float4 *ref4 = (float4 *)sp; sp += (size_t)N * 16;
    unsigned short *catom = (unsigned short *)sp; sp += align16((size_t)N * 2);   // atoms in cell order
    unsigned short *cellof = (unsigned short *)sp; sp += align16((size_t)N * 2);
    unsigned short *rank = (unsigned short *)sp; sp += align16((size_t)N * 2);
    unsigned char *cntl = (unsigned char *)sp; sp += align16((size_t)N);       // list lengths (cell order)
    int *cnt = (int *)sp; sp += align16((size_t)ncm * 4);
    int *start = (int *)sp; sp += align16((size_t)(ncm + 2) * 4);
    ElongScal<S> *m = (ElongScal<S> *)sp; sp += align16(sizeof(ElongScal<S>));
    int *warp_tmp = (int *)sp;

    auto ld_pos = [&](int i, S &x, S &y, S &z) {
        if constexpr (MIXED) {
            const float4 h = pos4[i], l = plo4[i];
            x = {h.x, l.x}; y = {h.y, l.y}; z = {h.z, l.z};
        } else {
            const Pd p = posd[i];
            x = p.x; y = p.y; z = p.z;
        }
    };
    auto st_pos = [&](int i, S x, S y, S z) {
        if constexpr (MIXED) {
            pos4[i] = make_float4(x.hi, y.hi, z.hi, 0.f);
            plo4[i] = make_float4(x.lo, y.lo, z.lo, 0.f);
        } else {
            posd[i] = {x, y, z, 0.0};
        }
    };
    auto pos_r = [&](int i) -> R4 {   // the pair-arithmetic positions (hi parts in MIXED)
        if constexpr (MIXED) return pos4[i]; else return posd[i];
    };

    // the list-cell grid of a box (thread 0): cells at least r_l (1 + 1e-4)
    // wide, at most the planned bound per axis (fewer cells are wider)
    auto set_grid = [&](S Lx, S Lz) {
        m->Lg[0] = Lx; m->Lg[1] = m->Ly; m->Lg[2] = Lz;
        m->Lf[0] = (float)shi(Lx); m->Lf[1] = (float)b.L[1]; m->Lf[2] = (float)shi(Lz);
        const float inv_w = 1.0f / (m->rl * 1.0001f);
        int nct = 1;
        for (int k = 0; k < 3; k++) {
            int n = (int)(m->Lf[k] * inv_w);
            n = n < 1 ? 1 : (n > a.ncmax[k] ? a.ncmax[k] : n);
            m->nc[k] = n;
            m->sf[k] = (float)n / m->Lf[k];
            m->invLf[k] = 1.0f / m->Lf[k];
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
        m->rl = (float)(RC + (double)a.skin);
        m->rl2 = m->rl * m->rl;
        m->exf = (float)exp(eps * h); m->ezf = (float)exp(-eps * h); m->eaf = (float)exp(-fabs(eps) * h);
        m->fxa = m->fza = m->ea = 1.f;
        m->thr2 = -1.f; m->umax2 = 0u; m->rebuild = 1; m->n_build = 0;
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
            if (shi(c) >= Lh[k]) c = xadd(c, sneg(L0[k]));
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
            st_pos(i, x, y, z);
            store_slot(mom + i, px); store_slot(mom + N + i, py); store_slot(mom + 2 * N + i, pz);
        }
    }

    // ---- building blocks ----
    // minimum image of a coordinate difference: the image chosen in float
    // (relevant pairs lie far inside half a box edge), applied at R
    auto mimg = [](R dd, float il, R L) -> R {
        const float n = rintf(__fmul_rn((float)dd, il));
        return rfma(-(R)n, L, dd);
    };
    // kinetic partials of a thread's atoms (index order): sum p^2 and
    // sum (px^2 - pz^2) (+ half the atoms' virial terms), hi parts in MIXED
    auto kin_partial = [&](R &k2, R &bk, bool virial) {
        k2 = (R)0; bk = (R)0;
        for (int i = tid; i < N; i += T) {
            const R qx = (R)shi(load_slot<S>(mom + i));
            const R qy = (R)shi(load_slot<S>(mom + N + i));
            const R qz = (R)shi(load_slot<S>(mom + 2 * N + i));
            k2 = radd(k2, rfma(qz, qz, rfma(qy, qy, rmul(qx, qx))));
            bk = radd(bk, rsub(rmul(qx, qx), rmul(qz, qz)));
            if (virial) bk = rfma((R)0.5, F4[i].w, bk);
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
    // Verlet lists: atoms binned into the list cells, then each atom's
    // neighbours within r_l (minimum image) from the distinct cells around
    // it, kept in index order (the force sums then do not depend on when a
    // list was built), written to the CTA's global scratch in cell order.
    auto build_lists = [&]() {
        for (int c = tid; c < ncm; c += T) cnt[c] = 0;
        __syncthreads();
        if (tid == 0) { m->rebuild = 0; m->n_build++; m->fxa = m->fza = m->ea = 1.f; }
        for (int i = tid; i < N; i += T) {
            const R4 p = pos_r(i);
            const float q[3] = {(float)p.x, (float)p.y, (float)p.z};
            int cc[3];
            for (int k = 0; k < 3; k++) {
                const int c = __float2int_rd(__fmul_rn(__fmaf_rn(0.5f, m->Lf[k], q[k]), m->sf[k]));
                cc[k] = c < 0 ? 0 : (c >= m->nc[k] ? m->nc[k] - 1 : c);
            }
            const int c = (cc[2] * m->nc[1] + cc[1]) * m->nc[0] + cc[0];
            cellof[i] = (unsigned short)c;
            rank[i] = (unsigned short)atomicAdd(&cnt[c], 1);
            ref4[i] = make_float4(q[0], q[1], q[2], 0.f);
        }
        __syncthreads();
        cta_exclusive_scan(cnt, start, m->ncell, warp_tmp);
        __syncthreads();
        for (int i = tid; i < N; i += T) catom[start[cellof[i]] + rank[i]] = (unsigned short)i;
        __syncthreads();
        const int nc0 = m->nc[0], nc1 = m->nc[1], nc2 = m->nc[2];
        const R Lx = (R)shi(m->Lg[0]), Ly = (R)shi(m->Lg[1]), Lz = (R)shi(m->Lg[2]);
        const float ilx = m->invLf[0], ily = m->invLf[1], ilz = m->invLf[2];
        const R rl2 = (R)m->rl2;
        for (int k = tid; k < N; k += T) {
            const int i = catom[k];
            const R4 pi = pos_r(i);
            const int c = cellof[i];
            const int cx = c % nc0, cy = (c / nc0) % nc1, cz = c / (nc0 * nc1);
            // each distinct cell within one of the atom's: three per axis, or
            // all of them where the axis has fewer than three
            const int z0 = nc2 >= 3 ? cz + nc2 - 1 : 0, zn = nc2 >= 3 ? 3 : nc2;
            const int y0 = nc1 >= 3 ? cy + nc1 - 1 : 0, yn = nc1 >= 3 ? 3 : nc1;
            const int x0 = nc0 >= 3 ? cx + nc0 - 1 : 0, xn = nc0 >= 3 ? 3 : nc0;
            unsigned short lst[ELONG_CAP];
            int n = 0, over = 0;
            for (int oz = 0; oz < zn; oz++) {
                const int zc = (z0 + oz) % nc2;
                for (int oy = 0; oy < yn; oy++) {
                    const int yc = (y0 + oy) % nc1;
                    for (int ox = 0; ox < xn; ox++) {
                        const int cc = (zc * nc1 + yc) * nc0 + (x0 + ox) % nc0;
                        for (int t = start[cc]; t < start[cc + 1]; t++) {
                            const int j = catom[t];
                            if (j == i) continue;
                            const R4 pj = pos_r(j);
                            const R dx = mimg(rsub(pi.x, pj.x), ilx, Lx);
                            const R dy = mimg(rsub(pi.y, pj.y), ily, Ly);
                            const R dz = mimg(rsub(pi.z, pj.z), ilz, Lz);
                            if (rfma(dz, dz, rfma(dy, dy, rmul(dx, dx))) < rl2) {
                                if (n == ELONG_CAP) { over = 1; continue; }
                                int w = n++;
                                while (w > 0 && lst[w - 1] > j) { lst[w] = lst[w - 1]; w--; }
                                lst[w] = (unsigned short)j;
                            }
                        }
                    }
                }
            }
            for (int w = 0; w * 8 < n; w++) {   // 16-byte groups of 8 entries
                unsigned int q[4];
                for (int hw = 0; hw < 4; hw++) {
                    const int e0 = w * 8 + 2 * hw;
                    const unsigned int lo = e0 < n ? lst[e0] : 0u, hi = e0 + 1 < n ? lst[e0 + 1] : 0u;
                    q[hw] = lo | (hi << 16);
                }
                nb4[(size_t)w * N + k] = make_uint4(q[0], q[1], q[2], q[3]);
            }
            cntl[k] = (unsigned char)n;
            if (over) atomicOr(&m->stop, TTCF_D_NBR_OVERFLOW);
        }
        __syncthreads();
    };
    // forces from the lists (atoms in the lists' cell order), into F4 with
    // each atom's virial term sum_j f (dx^2 - dz^2); counts the interacting
    // ordered pairs
    const R rc2 = (R)1.2599210498948732;
    unsigned int npair = 0;
    auto force_pass = [&]() {
        const R Lx = (R)shi(m->Lg[0]), Ly = (R)shi(m->Lg[1]), Lz = (R)shi(m->Lg[2]);
        const float ilx = m->invLf[0], ily = m->invLf[1], ilz = m->invLf[2];
        for (int k = tid; k < N; k += T) {
            const int i = catom[k];
            const R4 pi = pos_r(i);
            const int n = cntl[k];
            R fx = (R)0, fy = (R)0, fz = (R)0, wv = (R)0;
            auto pair = [&](int j) {
                const R4 pj = pos_r(j);
                const R dx = mimg(rsub(pi.x, pj.x), ilx, Lx);
                const R dy = mimg(rsub(pi.y, pj.y), ily, Ly);
                const R dz = mimg(rsub(pi.z, pj.z), ilz, Lz);
                const R r2 = rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
                if (r2 < rc2) {
                    const R s = (R)1 / r2;
                    const R s3 = rmul(rmul(s, s), s);
                    const R f = rmul(rmul(s, s3), rfma((R)48, s3, (R)-24));
                    fx = rfma(f, dx, fx); fy = rfma(f, dy, fy); fz = rfma(f, dz, fz);
                    wv = rfma(f, rsub(rmul(dx, dx), rmul(dz, dz)), wv);
                    npair++;
                }
            };
            // MIXED: the two entries of a list word side by side on packed
            // FP32 pairs (each lane the same IEEE operations as the scalar
            // pass), accumulated in index order
            auto pair2 = [&](int j0, int j1, bool has1) {
                const float4 p0 = pos4[j0], p1 = pos4[has1 ? j1 : j0];
                float2 dx = sub2(f2((float)pi.x), make_float2(p0.x, p1.x));
                float2 dy = sub2(f2((float)pi.y), make_float2(p0.y, p1.y));
                float2 dz = sub2(f2((float)pi.z), make_float2(p0.z, p1.z));
                dx = __ffma2_rn(neg2(rint2(dx, f2(ilx))), f2((float)Lx), dx);
                dy = __ffma2_rn(neg2(rint2(dy, f2(ily))), f2((float)Ly), dy);
                dz = __ffma2_rn(neg2(rint2(dz, f2(ilz))), f2((float)Lz), dz);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const bool in0 = r2.x < (float)rc2, in1 = has1 && r2.y < (float)rc2;
                if (in0 || in1) {
                    const float2 s = make_float2(in0 ? 1.f / r2.x : 0.f, in1 ? 1.f / r2.y : 0.f);
                    const float2 s3 = __fmul2_rn(__fmul2_rn(s, s), s);
                    const float2 f = __fmul2_rn(__fmul2_rn(s, s3), __ffma2_rn(f2(48.f), s3, f2(-24.f)));
                    const float2 w2 = sub2(__fmul2_rn(dx, dx), __fmul2_rn(dz, dz));
                    fx = rfma((R)f.x, (R)dx.x, fx); fy = rfma((R)f.x, (R)dy.x, fy);
                    fz = rfma((R)f.x, (R)dz.x, fz); wv = rfma((R)f.x, (R)w2.x, wv);
                    fx = rfma((R)f.y, (R)dx.y, fx); fy = rfma((R)f.y, (R)dy.y, fy);
                    fz = rfma((R)f.y, (R)dz.y, fz); wv = rfma((R)f.y, (R)w2.y, wv);
                    npair += (unsigned int)in0 + (unsigned int)in1;
                }
            };
            // one 16-byte group of 8 entries per load, the next one in
            // flight while the current one is worked on
            uint4 q = n > 0 ? nb4[k] : make_uint4(0u, 0u, 0u, 0u);
            for (int w = 0; w * 8 < n; w++) {
                const uint4 cur = q;
                if ((w + 1) * 8 < n) q = nb4[(size_t)(w + 1) * N + k];
                const int m8 = min(8, n - w * 8);
                for (int hw = 0; 2 * hw < m8; hw++) {
                    const unsigned int word = hw == 0 ? cur.x : hw == 1 ? cur.y : hw == 2 ? cur.z : cur.w;
                    if constexpr (MIXED) {
                        pair2((int)(word & 0xFFFFu), (int)(word >> 16), 2 * hw + 1 < m8);
                    } else {
                        pair((int)(word & 0xFFFFu));
                        if (2 * hw + 1 < m8) pair((int)(word >> 16));
                    }
                }
            }
            R4 o;
            o.x = fx; o.y = fy; o.z = fz; o.w = wv;
            F4[i] = o;
        }
        __syncthreads();
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
    // thread 0: the affine factors and the rebuild threshold of the next step
    auto advance_lists = [&]() {
        m->fxa *= m->exf; m->fza *= m->ezf; m->ea *= m->eaf;
        const float thr = 0.5f * (m->ea * m->rl - (float)RC) - 2e-3f;
        m->thr2 = thr > 0.f ? thr * thr : -1.f;
        m->umax2 = 0u;
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

    // ---- the steps.  Pass s = step0 only builds the lists and takes the
    //      forces and sum p^2 at the starting point, so that every force,
    //      list and sum is computed by one copy of the code (the same
    //      roundings in a chunked run as in an uninterrupted one) ----
    __syncthreads();
    int steps_run = 0;
    for (int s = a.step0; s <= a.step1 && !m->stop; s++) {
        const bool first = s == a.step0;
        if (!first) {
            // ---- D, C', B half flows, A' drift into the box of step s (Lx1,
            //      Lz1), displacement beyond the affine flow since the lists ----
            {
                const S c = m->c, cxh = m->cxh, czh = m->czh, hh = m->hh;
                const S ex = m->ex, ez = m->ez, phx = m->phx, phz = m->phz, h = m->h;
                const S Lx = m->Lx1, Lz = m->Lz1, hLx = m->hLx1, hLz = m->hLz1, Ly = m->Ly, hLy = m->hLy;
                const float fxa = m->fxa, fza = m->fza;
                const float Lxf = m->Lf[0], Lyf = m->Lf[1], Lzf = m->Lf[2];
                const float ilx = m->invLf[0], ily = m->invLf[1], ilz = m->invLf[2];
                float umax = 0.f;
                for (int i = tid; i < N; i += T) {
                    S px = load_slot<S>(mom + i), py = load_slot<S>(mom + N + i), pz = load_slot<S>(mom + 2 * N + i);
                    const R4 f = F4[i];
                    px = xmul(px, c); py = xmul(py, c); pz = xmul(pz, c);
                    px = xmul(px, cxh); pz = xmul(pz, czh);
                    px = xadd(px, xmulf(hh, f.x));
                    py = xadd(py, xmulf(hh, f.y));
                    pz = xadd(pz, xmulf(hh, f.z));
                    S x, y, z;
                    ld_pos(i, x, y, z);
                    x = wrap_once(xadd(xmul(x, ex), xmul(px, phx)), Lx, hLx);
                    y = wrap_once(xadd(y, xmul(py, h)), Ly, hLy);
                    z = wrap_once(xadd(xmul(z, ez), xmul(pz, phz)), Lz, hLz);
                    st_pos(i, x, y, z);
                    store_slot(mom + i, px); store_slot(mom + N + i, py); store_slot(mom + 2 * N + i, pz);
                    const float4 r0 = ref4[i];
                    float ux = (float)shi(x) - fxa * r0.x, uy = (float)shi(y) - r0.y, uz = (float)shi(z) - fza * r0.z;
                    ux -= Lxf * rintf(ux * ilx); uy -= Lyf * rintf(uy * ily); uz -= Lzf * rintf(uz * ilz);
                    const float u2 = ux * ux + uy * uy + uz * uz;
                    if (!(u2 <= umax) && umax == umax) umax = u2;   // a NaN stays and forces a rebuild
                }
                if (umax > 0.f || umax != umax) atomicMax(&m->umax2, __float_as_uint(umax));
            }
        }
        __syncthreads();
        if (first || m->rebuild || __uint_as_float(m->umax2) >= m->thr2 || m->umax2 > 0x7f800000u)
            build_lists();
        force_pass();
        if (first) npair = 0;   // counted over the steps only
        else {
            // ---- B, C', D half flows with the new forces ----
            {
                const S c = m->c, cxh = m->cxh, czh = m->czh, hh = m->hh;
                for (int i = tid; i < N; i += T) {
                    S px = load_slot<S>(mom + i), py = load_slot<S>(mom + N + i), pz = load_slot<S>(mom + 2 * N + i);
                    const R4 f = F4[i];
                    px = xadd(px, xmulf(hh, f.x));
                    py = xadd(py, xmulf(hh, f.y));
                    pz = xadd(pz, xmulf(hh, f.z));
                    px = xmul(px, cxh); pz = xmul(pz, czh);
                    px = xmul(px, c); py = xmul(py, c); pz = xmul(pz, c);
                    store_slot(mom + i, px); store_slot(mom + N + i, py); store_slot(mom + 2 * N + i, pz);
                }
            }
        }
        R k2, bk;
        kin_partial(k2, bk, !first);
        S sums[2];
        cta_sum2(k2, bk, sums);
        if (tid == 0) {
            if (first) {
                open_step(e_increment(sums[0]));   // the first step's opening E flow
            } else {
                chain(sums[0]);
                const double bv = sdbl(sums[1]) * m->invV;   // P_xx - P_zz
                if (s % a.sample_every == 0) b.B[(size_t)d * b.S + s / a.sample_every] = bv;
                if (!isfinite(bv)) m->stop |= TTCF_D_NONFINITE;
                // the positions now live in the box of step s
                m->Lx = m->Lx1;
                m->Lz = m->Lz1;
            }
            advance_box();
            advance_lists();
            if (m->flag_lost || !isfinite(sdbl(sums[0]))) m->stop |= TTCF_D_NONFINITE;
            if (a.abort_flag && (s & 63) == 0 && *a.abort_flag) m->stop |= TTCF_D_ABORTED;
        }
        if (!first) steps_run++;
        __syncthreads();
    }

    // ---- counters, status, loop state ----
    atomicAdd(&m->pairs, (unsigned long long)npair);
    __syncthreads();
    if (tid == 0) {
        b.pairs[d] += m->pairs;   // ordered pairs, as the other kernels count them
        b.rebuilds[d] += (unsigned int)m->n_build;
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
        for (int i = tid; i < N; i += T) {
            S x, y, z;
            ld_pos(i, x, y, z);
            store_slot(dst + i, x); store_slot(dst + N + i, y); store_slot(dst + 2 * N + i, z);
            dst[3 * N + i] = mom[i]; dst[4 * N + i] = mom[N + i]; dst[5 * N + i] = mom[2 * N + i];
        }
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

int elong_grid(bool mixed, int N, int ncellmax, int nsm, long long D) {
    const size_t smem = elong_smem_bytes(mixed, N, ncellmax);
    auto fn = mixed ? elong_kernel<true> : elong_kernel<false>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, elong_threads(N), smem) != cudaSuccess) return 0;
    return (int)std::min<long long>(D, (long long)nsm * per_sm);
}

cudaError_t launch_elong(bool mixed, const ElongArgs &a, int grid, cudaStream_t st) {
    const int ncm = a.ncmax[0] * a.ncmax[1] * a.ncmax[2];
    const size_t smem = elong_smem_bytes(mixed, a.b.N, ncm);
    auto fn = mixed ? elong_kernel<true> : elong_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid <= 0) return cudaSuccess;
    fn<<<(unsigned)grid, elong_threads(a.b.N), smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ttcf
