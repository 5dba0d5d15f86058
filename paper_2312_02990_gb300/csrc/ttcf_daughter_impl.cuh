// ttcf_daughter_impl.cuh -- the persistent daughter kernel and its
// launchers as templates, included by two translation units:
// ttcf_daughter.cu instantiates every launch variant but one, and
// ttcf_daughter_u8.cu the MIXED variant of 8 atoms per thread with
// TTCF_UNROLL_ATOMS defined, which unrolls every loop over a thread's atoms
// so that their per-atom state (momenta, forces, list counts) stays in
// registers instead of local memory (a 384-byte stack frame otherwise).
// With the list groups taken one ahead in the force pass (4 and 8 atoms
// per thread) the N = 4000 daughters run 1.12x faster, results unchanged.
// The other variants keep the compiler's own unrolling choices.  The
// kernel itself is described in ttcf_daughter.cu.
#pragma once
#include <type_traits>

#include "ttcf_device.cuh"
#include "ttcf_internal.h"

#ifdef TTCF_UNROLL_ATOMS   // (a count: some of these loops have a second exit condition)
#define TTCF_Q_UNROLL _Pragma("unroll 8")
#else
#define TTCF_Q_UNROLL
#endif

namespace ttcf {

// Per-daughter constants and per-step coefficients, written by thread 0.
template <class S>
struct Coef {
    S e;                   // phase-A momentum factor minus 1
    S h, hh, gh, chalf;    // h, h/2, gamma h, gamma h/2
    S L[3];
    S delta_s;             // Lees-Edwards offset for position wraps
    double delta_d;        // Lees-Edwards offset (FP64 mode forces)
    double invL[3];
    float delta_f;         // Lees-Edwards offset (FP32 forces)
    float Lf[3], invLf[3];
    float thr2;            // rebuild threshold, squared; < 0 forces a rebuild
    float fast2;           // fatal single-step displacement, squared
    float rl2;             // list radius squared
    float ra2;             // active-list radius squared, (r_c + ACTIVE_SKIN)^2
    float thr_a;           // active-list refresh threshold on the path length; < 0 forces one
    int stop;
    int snap;              // snapshot index written after this step, or -1
    double fsnap;          // pending momentum factor for the snapshot
    S f1;                  // (1 + e1)^2, the momentum factor still pending at the step end
};

struct Misc {
    double slot[MAX_WARPS][3];   // per-warp partial sums (df packed or double)
    // per-daughter scalars in IEEE double (the FP64 mode's step-end chain;
    // in MIXED mode the set-up values), touched by thread 0 only
    double a_end, a_cur, K2_end, e1, delta, f1sq;
    double hhQ, invV, ddelta, halfLx;   // per-daughter constants
    // MIXED mode: the same chain in double-float on the FP32 pipe (an IEEE-
    // double instruction on one lane costs about a hundred cycles of latency
    // on GB300, and this chain is on every step's critical path)
    df a_endf, a_curf, K2f, e1f, f1f, deltaf;
    df hhQf, ngTf, nhhf, sixthf, ddeltaf, halfLxf, Lxf;
    float ddelta_abs;
    float dsince;                       // |change of delta| since the list build
    float dsince_a;                     // |change of delta| since the active-list refresh
    unsigned int n_rebuild;
    unsigned int n_filter;              // force passes over the Verlet lists (refreshes)
    unsigned long long np;              // interacting pairs counted on those passes
    int flag_filter[2];
    int warp_tmp[MAX_WARPS];
    int flag_rebuild[2];
    int flag_fast;
    int flag_ovf;
    int flag_lost;
};

// daughter_smem_bytes reserves 2048 bytes for the two structures above
static_assert(((sizeof(Coef<df>) + 15) / 16 * 16) + sizeof(Misc) <= 2048, "Coef + Misc exceed their reserve");
static_assert(((sizeof(Coef<double>) + 15) / 16 * 16) + sizeof(Misc) <= 2048, "Coef + Misc exceed their reserve");

// --------------------------------------------------------- reductions --

// CTA sums of three per-thread partials in a fixed order (float partials
// summed as double-float in MIXED mode).  Contains one __syncthreads; the
// result is valid in lane 0 of warp 0 and of warp `w2` (both reduce the
// per-warp slots in the same fixed order, so their results are identical).
template <bool MIXED, class R>
__device__ __forceinline__ void cta_sum3(R a0, R a1, R a2, Misc *m, double out[3], int w2 = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    if constexpr (MIXED) {
        df s0 = warp_sum(df_make(a0)), s1 = warp_sum(df_make(a1)), s2 = warp_sum(df_make(a2));
        if (lane == 0) {
            float2 *sl = reinterpret_cast<float2 *>(&m->slot[warp][0]);
            sl[0] = make_float2(s0.hi, s0.lo);   // slot[warp] holds three float2
            sl[1] = make_float2(s1.hi, s1.lo);
            sl[2] = make_float2(s2.hi, s2.lo);
        }
        __syncthreads();
        if (warp == 0 || warp == w2) {
            df t0 = {0.f, 0.f}, t1 = {0.f, 0.f}, t2 = {0.f, 0.f};
            if (lane < nw) {
                const float2 *sl = reinterpret_cast<const float2 *>(&m->slot[lane][0]);
                t0 = {sl[0].x, sl[0].y}; t1 = {sl[1].x, sl[1].y}; t2 = {sl[2].x, sl[2].y};
            }
            t0 = warp_sum(t0); t1 = warp_sum(t1); t2 = warp_sum(t2);
            if (lane == 0) { out[0] = df_to_double(t0); out[1] = df_to_double(t1); out[2] = df_to_double(t2); }
        }
    } else {
        double s0 = warp_sum((double)a0), s1 = warp_sum((double)a1), s2 = warp_sum((double)a2);
        if (lane == 0) { m->slot[warp][0] = s0; m->slot[warp][1] = s1; m->slot[warp][2] = s2; }
        __syncthreads();
        if (warp == 0 || warp == w2) {
            double t0 = 0, t1 = 0, t2 = 0;
            if (lane < nw) { t0 = m->slot[lane][0]; t1 = m->slot[lane][1]; t2 = m->slot[lane][2]; }
            t0 = warp_sum(t0); t1 = warp_sum(t1); t2 = warp_sum(t2);
            if (lane == 0) { out[0] = t0; out[1] = t1; out[2] = t2; }
        }
    }
}

// CTA sums of two per-thread float partials (MIXED mode's per-step sums)
// in 64-bit fixed point of 2^-40 units: every float of magnitude >= 2^-17
// is exact there, so the integer sums are exact and independent of order;
// the totals come back as normalised double-float pairs (the same pairs a
// double-float tree gives where its sum is exact, as it is here; about 1 %
// faster).  One __syncthreads; the result is valid in lane 0 of warp 0 and
// of warp w2.
__device__ __forceinline__ long long fix40(float v) { return __float2ll_rn(v * 1099511627776.0f); }
__device__ __forceinline__ df df_from_fix40(long long s) {
    const float hi = __ll2float_rn(s);
    const float lo = __ll2float_rn(s - __float2ll_rn(hi));   // the exact remainder, rounded
    return {hi * 9.094947017729282e-13f, lo * 9.094947017729282e-13f};   // x 2^-40, exact
}
__device__ __forceinline__ void cta_sum2_fix(float a0, float a1, Misc *m, df out[2], int w2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    // the 64-bit sums hold |total| < 2^23; with at most 1024 threads a
    // thread partial of 2^13 or more (or one not finite) stops the daughter
    // as non-finite (normal partials are below 10^2; 2^13 takes a WCA pair
    // nearer than 0.6 sigma, about 1800 kT above contact)
    if (!(fabsf(a0) < 8192.f && fabsf(a1) < 8192.f)) m->flag_lost = 1;
    long long v0 = fix40(a0), v1 = fix40(a1);
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_down_sync(0xffffffffu, v0, o);
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        long long *sl = reinterpret_cast<long long *>(&m->slot[warp][0]);
        sl[0] = v0;
        sl[1] = v1;
    }
    __syncthreads();
    if (warp == 0 || warp == w2) {
        long long t0 = 0, t1 = 0;
        if (lane < nw) {
            const long long *sl = reinterpret_cast<const long long *>(&m->slot[lane][0]);
            t0 = sl[0];
            t1 = sl[1];
        }
        for (int o = 16; o > 0; o >>= 1) {
            t0 += __shfl_down_sync(0xffffffffu, t0, o);
            t1 += __shfl_down_sync(0xffffffffu, t1, o);
        }
        if (lane == 0) {
            out[0] = df_from_fix40(t0);
            out[1] = df_from_fix40(t1);
        }
    }
}


// ------------------------------------------------ sorting a Verlet list --
// Compare-exchange of the uint16 halves of two registers (both halves in
// the same direction), and of the two halves of one register.
__device__ __forceinline__ void ce_reg(unsigned int &a, unsigned int &b, bool asc) {
    const unsigned int lo = __vminu2(a, b), hi = __vmaxu2(a, b);
    a = asc ? lo : hi;
    b = asc ? hi : lo;
}
__device__ __forceinline__ unsigned int ce_half(unsigned int x, bool asc) {
    const unsigned int s = __byte_perm(x, 0u, 0x1032);   // halves swapped
    const unsigned int mn = __vminu2(x, s), mx = __vmaxu2(x, s);
    return asc ? __byte_perm(mn, mx, 0x7610) : __byte_perm(mx, mn, 0x7610);
}
// Bitonic sort of 32 uint16 keys, key e in half (e & 1) of r[e / 2],
// ascending: merges of sizes 2, 4, ..., 32, compare distances j halving;
// distances >= 2 pair two registers, distance 1 the halves of one.
static_assert(CAP == 32, "sort32_u16 sorts the 32 slots of a Verlet list");
__device__ __forceinline__ void sort32_u16(unsigned int r[16]) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j >= 2; j >>= 1) {
#pragma unroll
            for (int m = 0; m < 16; m++) {
                const int mp = m ^ (j >> 1);
                if (mp > m) ce_reg(r[m], r[mp], ((2 * m) & k) == 0);
            }
        }
#pragma unroll
        for (int m = 0; m < 16; m++) r[m] = ce_half(r[m], ((2 * m) & k) == 0);
    }
}

// ------------------------------------------------------- one daughter --
template <bool MIXED, int APT>
__device__ __forceinline__ void run_daughter(const RunArgs &a, int d, unsigned char *smem) {
    using S = typename std::conditional<MIXED, df, double>::type;   // state scalar
    using R = typename std::conditional<MIXED, float, double>::type; // force arithmetic
    const int tid = threadIdx.x, T = blockDim.x;
    const int bi = a.dbatch[d];
    const BatchDev &b = a.batches[bi];
    const int N = b.N;
    const int dl = (int)(d - b.d0);          // daughter index within the batch
    const int gl = dl / b.M;                 // mother group within the batch
    const int map = b.maps[dl % b.M];        // mapping of Eq. 3
    const double gamma = b.gamma[gl];
    const int nmax = a.nmax, ncm = a.ncellmax;
    const int *nc = b.nc;

    // shared-memory carve-up (daughter_smem_bytes mirrors this)
    unsigned char *sp = smem;
    float4 *pos4 = nullptr, *plo4 = nullptr;
    double *xd = nullptr, *yd = nullptr, *zd = nullptr;
    if constexpr (MIXED) {
        pos4 = (float4 *)sp; sp += (size_t)nmax * 16;
        if constexpr (APT >= 8) {   // plo_global: lo parts in the per-CTA global scratch
            plo4 = a.plo_g + (size_t)blockIdx.x * nmax;
        } else {
            plo4 = (float4 *)sp; sp += (size_t)nmax * 16;
        }
    } else {   // each array padded to 16 bytes: ref4 below must stay float4-aligned
        const size_t dn = ((size_t)nmax * 8 + 15) / 16 * 16;
        xd = (double *)sp; sp += dn;
        yd = (double *)sp; sp += dn;
        zd = (double *)sp; sp += dn;
    }
    float4 *ref4 = (float4 *)sp; sp += (size_t)nmax * 16;
    // cell-ordered copy of the wrapped positions (index in w), or the cell
    // members' indices alone where shared memory is short
    float4 *cpos = nullptr;
    unsigned short *catom = nullptr;
    if (a.cpos) { cpos = (float4 *)sp; sp += (size_t)nmax * 16; }
    int *cnt = (int *)sp; sp += (size_t)ncm * 4;
    int *start = (int *)sp; sp += (size_t)(ncm + 2) * 4;
    if (!a.cpos) { catom = (unsigned short *)sp; sp += ((size_t)nmax * 2 + 15) / 16 * 16; }
    Coef<S> *cf = (Coef<S> *)sp; sp += (sizeof(Coef<S>) + 15) / 16 * 16;
    Misc *m = (Misc *)sp;

    // Verlet lists of all CTAs, then the active lists of all CTAs
    uint4 *nbr4 = reinterpret_cast<uint4 *>(a.nbr + (size_t)blockIdx.x * (CAP / 2) * nmax);
    uint4 *nbra4 = reinterpret_cast<uint4 *>(a.nbr + (size_t)gridDim.x * (CAP / 2) * nmax +
                                             (size_t)blockIdx.x * (CAP_A / 2) * nmax);
    unsigned short *nbra16 = reinterpret_cast<unsigned short *>(nbra4);

    // thread 0 keeps the per-daughter scalars in shared memory (IEEE double;
    // MIXED mode steps the double-float copies in Misc)
    double &a_end = m->a_end, &a_cur = m->a_cur, &K2_end = m->K2_end, &e1 = m->e1;
    double &delta = m->delta, &f1sq = m->f1sq;
    float &dsince = m->dsince;
    const double h = a.dt, hh = 0.5 * a.dt;
    if (tid == 0) {
        a_end = a_cur = K2_end = e1 = delta = 0.0;
        f1sq = 1.0;
        dsince = 0.f;
        m->dsince_a = 0.f;
        m->n_rebuild = 0;
        m->n_filter = 0;
        m->np = 0ull;
        m->flag_filter[0] = m->flag_filter[1] = 0;
        // constants of the per-step lane-0 chain (no division in the loop)
        m->hhQ = hh / b.Q;
        m->invV = 1.0 / b.V;
        m->ddelta = gamma * b.L[1] * h;
        m->halfLx = 0.5 * b.L[0];
        cf->h = sfrom<S>(h); cf->hh = sfrom<S>(hh);
        cf->gh = sfrom<S>(gamma * h); cf->chalf = sfrom<S>(gamma * hh);
        for (int k = 0; k < 3; k++) {
            cf->L[k] = sfrom<S>(b.L[k]);
            cf->Lf[k] = (float)b.L[k];
            cf->invLf[k] = (float)(1.0 / b.L[k]);
            cf->invL[k] = 1.0 / b.L[k];
        }
        const float rl = (float)(1.1224620483093730 + (double)b.skin);
        cf->rl2 = rl * rl;
        const float ra = (float)1.1224620483093730 + fminf(ACTIVE_SKIN, b.skin);
        cf->ra2 = ra * ra;
        cf->thr_a = -1.f;
        cf->fast2 = 0.25f * b.skin * b.skin;
        cf->thr2 = -1.f;
        cf->stop = 0; cf->snap = -1; cf->fsnap = 1.0;
        m->flag_rebuild[0] = m->flag_rebuild[1] = 0;
        m->flag_fast = 0; m->flag_ovf = 0; m->flag_lost = 0;
        if (a.fresh) {
            const double sa = map_reverses_time(map) ? -1.0 : 1.0;
            a_end = a.reset_alpha ? 0.0 : sa * b.m_alpha[gl];
            e1 = 0.0;
            delta = a.delta0;
        } else if constexpr (!MIXED) {
            const double *sc = b.scal + 4 * (size_t)dl;
            a_end = sc[0]; K2_end = sc[1]; e1 = sc[2]; delta = sc[3];
            f1sq = (1.0 + e1) * (1.0 + e1);
        }
        if constexpr (MIXED) {
            if (a.fresh) {
                m->a_endf = df_from_double(a_end);
                m->K2f = df_make(0.f);
                m->e1f = df_make(0.f);
                m->deltaf = df_from_double(delta);
            } else {   // saved as float pairs: the run continues bit for bit
                const unsigned long long *sc = reinterpret_cast<const unsigned long long *>(b.scal) + 4 * (size_t)dl;
                m->a_endf = load_slot<df>(sc); m->K2f = load_slot<df>(sc + 1);
                m->e1f = load_slot<df>(sc + 2); m->deltaf = load_slot<df>(sc + 3);
            }
            m->a_curf = m->a_endf;
            const df g = df_add_f(m->e1f, 1.0f);
            m->f1f = df_mul(g, g);
            m->hhQf = df_from_double(m->hhQ);
            m->ngTf = df_from_double(-b.gT);
            m->nhhf = df_from_double(-hh);
            m->sixthf = df_from_double(1.0 / 6.0);
            m->ddeltaf = df_from_double(m->ddelta);
            m->halfLxf = df_from_double(m->halfLx);
            m->Lxf = df_from_double(b.L[0]);
            m->ddelta_abs = fabsf((float)m->ddelta);
            delta = df_to_double(m->deltaf);
            cf->delta_d = delta; cf->delta_s = m->deltaf; cf->delta_f = m->deltaf.hi;
            cf->f1 = m->f1f;
        } else {
            cf->delta_d = delta; cf->delta_s = sfrom<S>(delta); cf->delta_f = (float)delta;
            cf->f1 = sfrom<S>(f1sq);
        }
    }
    __syncthreads();

    // ---- load the phase point (mapped mother, or the saved loop state) ----
    S P[APT][3];
    R F[APT][3];
    int ncnt[APT];
    {
        const int mp = a.fresh ? map : 0;   // mapping code applied at switch-on
        const unsigned long long *src = a.fresh ? b.mothers + (size_t)gl * 6 * N
                                                : b.state + (size_t)dl * 6 * N;
        const R Lh[3] = {(R)(0.5 * b.L[0]), (R)(0.5 * b.L[1]), (R)(0.5 * b.L[2])};
        // c -> -c; -(-L/2) = +L/2 is the same periodic point
        auto reflect = [&](S c, int k) {
            c = sneg(c);
            if (shi(c) >= Lh[k]) c = sadd(c, sneg(cf->L[k]));
            return c;
        };
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            ncnt[q] = 0;
            F[q][0] = F[q][1] = F[q][2] = (R)0;
            P[q][0] = P[q][1] = P[q][2] = sfrom<S>(0.0);
            if (i < N) {
                S x = load_slot<S>(src + i), y = load_slot<S>(src + N + i), z = load_slot<S>(src + 2 * N + i);
                S px = load_slot<S>(src + 3 * N + i), py = load_slot<S>(src + 4 * N + i), pz = load_slot<S>(src + 5 * N + i);
                if (map_swaps_xz(mp)) { S t = x; x = z; z = t; t = px; px = pz; pz = t; }
                if (mp & 2) { x = reflect(x, 0); px = sneg(px); }
                if (mp & 4) { y = reflect(y, 1); py = sneg(py); }
                if (mp & 8) { z = reflect(z, 2); pz = sneg(pz); }
                if (map_reverses_time(mp)) { px = sneg(px); py = sneg(py); pz = sneg(pz); }
                P[q][0] = px; P[q][1] = py; P[q][2] = pz;
                if constexpr (MIXED) {
                    pos4[i] = make_float4(x.hi, y.hi, z.hi, 0.f);
                    plo4[i] = make_float4(x.lo, y.lo, z.lo, 0.f);
                } else {
                    xd[i] = x; yd[i] = y; zd[i] = z;
                }
            }
        }
    }
    __syncthreads();

    // ---- geometry helpers ----
    // minimum-image vector r_i - r_j under Lees-Edwards images (y first)
    auto pair_vec = [&](int i, int j, R &dx, R &dy, R &dz) {
        if constexpr (MIXED) {
            const float4 u = pos4[i], v = pos4[j];
            dx = u.x - v.x; dy = u.y - v.y; dz = u.z - v.z;
            const float ny = rint_fma(dy, cf->invLf[1]);
            dy = __fmaf_rn(-ny, cf->Lf[1], dy);
            dx = __fmaf_rn(-ny, cf->delta_f, dx);
            const float nx = rint_fma(dx, cf->invLf[0]);
            dx = __fmaf_rn(-nx, cf->Lf[0], dx);
            const float nz = rint_fma(dz, cf->invLf[2]);
            dz = __fmaf_rn(-nz, cf->Lf[2], dz);
        } else {
            dx = xd[i] - xd[j]; dy = yd[i] - yd[j]; dz = zd[i] - zd[j];
            const double ny = rint(dy * cf->invL[1]);
            dy -= ny * b.L[1]; dx -= ny * cf->delta_d;
            dx -= rint(dx * cf->invL[0]) * b.L[0];
            dz -= rint(dz * cf->invL[2]) * b.L[2];
        }
    };
    // position of atom i mapped into the primary box (for binning only)
    auto wrapped = [&](int i, float &wx, float &wy, float &wz) {
        R x, y, z;
        if constexpr (MIXED) { const float4 v = pos4[i]; x = v.x; y = v.y; z = v.z; }
        else { x = xd[i]; y = yd[i]; z = zd[i]; }
        if constexpr (MIXED) {
            const float ny = rint_fma(y, cf->invLf[1]);
            y = __fmaf_rn(-ny, cf->Lf[1], y); x = __fmaf_rn(-ny, cf->delta_f, x);
            x = __fmaf_rn(-rint_fma(x, cf->invLf[0]), cf->Lf[0], x);
            z = __fmaf_rn(-rint_fma(z, cf->invLf[2]), cf->Lf[2], z);
        } else {
            const double ny = rint(y * cf->invL[1]);
            y -= ny * b.L[1]; x -= ny * cf->delta_d;
            x -= rint(x * cf->invL[0]) * b.L[0];
            z -= rint(z * cf->invL[2]) * b.L[2];
        }
        wx = (float)x; wy = (float)y; wz = (float)z;
    };
    auto cell_of = [&](float w, int k) {
        int c = ifloor((w + 0.5f * cf->Lf[k]) * ((float)nc[k] * cf->invLf[k]));
        return min(max(c, 0), nc[k] - 1);
    };

    // ---- Verlet list: cell binning (cells cell_frac (r_c + skin) wide; the
    //      window of cells covers r_l = r_c + skin), sorted lists ----
    auto build_list = [&]() {
        const int ncell = b.ncell;
        for (int c = tid; c < ncell; c += T) cnt[c] = 0;
        __syncthreads();
        int mycell[APT], myslot[APT];
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            mycell[q] = 0; myslot[q] = 0;
            if (i < N) {
                float wx, wy, wz;
                wrapped(i, wx, wy, wz);
                const int c = (cell_of(wz, 2) * nc[1] + cell_of(wy, 1)) * nc[0] + cell_of(wx, 0);
                mycell[q] = c;
                myslot[q] = atomicAdd(&cnt[c], 1);
                if constexpr (MIXED) ref4[i] = pos4[i];
                else ref4[i] = make_float4((float)xd[i], (float)yd[i], (float)zd[i], 0.f);
            }
        }
        __syncthreads();
        cta_exclusive_scan(cnt, start, ncell, m->warp_tmp);
        __syncthreads();
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            if (i >= N) continue;
            const int t = start[mycell[q]] + myslot[q];
            if (cpos) {
                float wx, wy, wz;
                wrapped(i, wx, wy, wz);
                cpos[t] = make_float4(wx, wy, wz, __int_as_float(i));
            } else {
                catom[t] = (unsigned short)i;
            }
        }
        __syncthreads();
        const float rl = sqrtf(cf->rl2);
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            if (i >= N) continue;
            float wx, wy, wz;
            wrapped(i, wx, wy, wz);
            // a lost (non-finite or runaway) atom ends the daughter; it must
            // not reach the loops below, whose bounds come from its position.
            // Wrapped coordinates satisfy |w| <= L/2; with |w| <= 3L/4 every
            // window index below lies in (-2 nc, 2 nc).
            if (!(fabsf(wx) <= 0.75f * cf->Lf[0] && fabsf(wy) <= 0.75f * cf->Lf[1] &&
                  fabsf(wz) <= 0.75f * cf->Lf[2])) {
                m->flag_lost = 1;
                ncnt[q] = 0;
                continue;
            }
            // accepted neighbours are appended during the scan and sorted
            // once after it: an insertion inside the divergent scan loops
            // would be paid by every lane of the warp at nearly every
            // candidate
            // entries as uint16, entry e in half e % 2 of word e / 2 (the
            // network's layout) or, one atom per thread, a plain array
            using LstT = typename std::conditional<(APT >= 2), unsigned int, unsigned short>::type;
            LstT lstw[APT >= 2 ? CAP / 2 : CAP];
            int k = 0;
            auto push = [&](int j) {
                if (k < CAP) reinterpret_cast<unsigned short *>(lstw)[k] = (unsigned short)j;
                k++;
            };
            // windows [w - r_l, w + r_l] in cell units; |w| <= L keeps them small
            const float hl0 = 0.5f * cf->Lf[0], hl1 = 0.5f * cf->Lf[1], hl2 = 0.5f * cf->Lf[2];
            const float s0 = (float)nc[0] * cf->invLf[0], s1 = (float)nc[1] * cf->invLf[1],
                        s2 = (float)nc[2] * cf->invLf[2];
            const int z0 = ifloor((wz - rl + hl2) * s2);
            const int z1 = min(ifloor((wz + rl + hl2) * s2), z0 + nc[2] - 1);
            const int y0 = ifloor((wy - rl + hl1) * s1);
            const int y1 = min(ifloor((wy + rl + hl1) * s1), y0 + nc[1] - 1);
            // window indices lie in [-nc, 2nc): wrap by one conditional add
            const float rl2 = cf->rl2;
            for (int zu = z0; zu <= z1; zu++) {
                const int kz = zu < 0 ? -1 : (zu >= nc[2] ? 1 : 0);   // periodic image in z
                const int zz = zu - kz * nc[2];
                const float uz = wz - (float)kz * cf->Lf[2];
                for (int yu = y0; yu <= y1; yu++) {
                    const int cross = yu < 0 ? -1 : (yu >= nc[1] ? 1 : 0);
                    const int yy = yu - cross * nc[1];
                    const float uy = wy - (float)cross * cf->Lf[1];
                    // the row across the y face is seen shifted by cross*delta
                    const float xs = wx - (float)cross * cf->delta_f;
                    int x0 = ifloor((xs - rl + hl0) * s0);
                    int x1 = min(ifloor((xs + rl + hl0) * s0), x0 + nc[0] - 1);
                    const int row = (zz * nc[1] + yy) * nc[0];
                    // the x window as one or two contiguous runs of cell-sorted
                    // atoms; run r holds the periodic image kx + r in x.
                    // x0 lies in [-2nc, 2nc): two conditional wraps
                    int a0 = x0, kx = 0;
                    if (a0 < 0) { a0 += nc[0]; kx = -1; } else if (a0 >= nc[0]) { a0 -= nc[0]; kx = 1; }
                    if (a0 < 0) { a0 += nc[0]; kx -= 1; } else if (a0 >= nc[0]) { a0 -= nc[0]; kx += 1; }
                    int ra[2], rb[2], nr = 0;
                    const int b0 = a0 + (x1 - x0);
                    if (b0 < nc[0]) { ra[0] = a0; rb[0] = b0; nr = 1; }
                    else { ra[0] = a0; rb[0] = nc[0] - 1; ra[1] = 0; rb[1] = b0 - nc[0]; nr = 2; }
                    for (int r = 0; r < nr; r++) {
                        const int t1 = start[row + rb[r] + 1];
                        if (cpos) {
                            // i against the image of each member: one shared load
                            // and the distance to a fixed shift, no rounding
                            const float ux = xs - (float)(kx + r) * cf->Lf[0];
                            // two consecutive members side by side on packed FP32
                            // pairs, accepted in order
                            int t = start[row + ra[r]];
                            for (; t + 1 < t1; t += 2) {
                                const float4 v0 = cpos[t], v1 = cpos[t + 1];
                                const float2 dx = __fadd2_rn(f2(ux), make_float2(-v0.x, -v1.x));
                                const float2 dy = __fadd2_rn(f2(uy), make_float2(-v0.y, -v1.y));
                                const float2 dz = __fadd2_rn(f2(uz), make_float2(-v0.z, -v1.z));
                                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                                if (r2.x < rl2) { const int j = __float_as_int(v0.w); if (j != i) push(j); }
                                if (r2.y < rl2) { const int j = __float_as_int(v1.w); if (j != i) push(j); }
                            }
                            if (t < t1) {
                                const float4 v = cpos[t];
                                const float dx = ux - v.x, dy = uy - v.y, dz = uz - v.z;
                                const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                                if (r2 < rl2) {
                                    const int j = __float_as_int(v.w);
                                    if (j != i) push(j);
                                }
                            }
                        } else {
                            for (int t = start[row + ra[r]]; t < t1; t++) {
                                const int j = catom[t];
                                if (j == i) continue;
                                R dx, dy, dz;
                                pair_vec(i, j, dx, dy, dz);
                                const float r2 = (float)(dx * dx + dy * dy + dz * dz);
                                if (r2 < rl2) push(j);
                            }
                        }
                    }
                }
            }
            if (k > CAP) { m->flag_ovf = 1; k = CAP; }
            // sorted by neighbour index with a bitonic network over the 32
            // slots held as 16 packed uint16 pairs in registers (the same
            // steps on every lane: no divergent insertion loop; free slots
            // hold 0xffff and sort last).  One atom per thread (256-thread
            // CTAs of small daughters) keeps the insertion sort, which is
            // cheaper there.
            if constexpr (APT >= 2) {
                unsigned int r[CAP / 2];
#pragma unroll
                for (int w = 0; w < CAP / 2; w++) {
                    const unsigned int v = 2 * w < k ? lstw[w] : 0xffffffffu;
                    r[w] = v | (2 * w + 1 < k ? 0u : 0xffff0000u);
                }
                sort32_u16(r);
                // eight entries per 16-byte chunk, two per word; slots from
                // k on become i itself (r = 0 is rejected by the force loop)
                const unsigned int ii = (unsigned int)i;
#pragma unroll
                for (int c = 0; c < CAP / 8; c++) {
                    if (8 * c < k) {
                        unsigned int wv[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            unsigned int w = r[4 * c + u];
                            if ((w & 0xffffu) == 0xffffu) w = (w & 0xffff0000u) | ii;
                            if ((w >> 16) == 0xffffu) w = (w & 0xffffu) | (ii << 16);
                            wv[u] = w;
                        }
                        nbr4[(size_t)c * nmax + i] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                    }
                }
            } else {
                unsigned short *lst = lstw;
                for (int e = 1; e < k; e++) {   // insertion sort by neighbour index
                    const unsigned short v = lst[e];
                    int pi = e;
                    while (pi > 0 && lst[pi - 1] > v) { lst[pi] = lst[pi - 1]; pi--; }
                    lst[pi] = v;
                }
                // eight entries per 16-byte chunk, two per word; an odd tail
                // is padded with i itself (r = 0 is rejected by the force loop)
                for (int t = 0; t < k; t += 8) {
                    unsigned int wv[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int e = t + 2 * u;
                        const unsigned int lo = e < k ? lst[e] : (unsigned int)i;
                        const unsigned int hi = e + 1 < k ? lst[e + 1] : (unsigned int)i;
                        wv[u] = lo | (hi << 16);
                    }
                    nbr4[(size_t)(t >> 3) * nmax + i] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
                }
            }
            ncnt[q] = k;
        }
    };

    // ---- WCA forces (Eq. 6) and virial of own atoms ----
    // Two passes share the pair arithmetic.  FILTER: over the Verlet list,
    // counting the interacting pairs; in FP64 mode it also refreshes the
    // atom's active list (the entries within r_c + ACTIVE_SKIN, kept in list
    // order).  Otherwise over the active list (FP64) or again the Verlet list
    // (MIXED).  Both lists are sorted by neighbour index and out-of-range
    // entries add exact zeros, so the two passes give the same sums bit for
    // bit.  ncnt: Verlet count in the low 16 bits, the active count in the
    // high 16 (0xffff: more than CAP_A, use the Verlet list).
    // MIXED mode keeps to the Verlet lists: there the pass is cheap beside
    // its fixed costs, and the active-list bookkeeping (path sums in phase
    // A, appends in the filter pass) raised register spills by more than
    // the shorter lists saved (0.90x on the N = 2048 launch, results equal);
    // the FP64 pass pays for it (1.28x at N = 256).
    constexpr bool ACTIVE = !MIXED;
    unsigned int npairs = 0;
    auto forces = [&](auto filter) -> R {
        constexpr bool FILTER = decltype(filter)::value;
        const R rc2 = (R)1.2599210498948732;   // r_c^2 = 2^(1/3)
        R wsum = 0;
        // Launch variants of 4 or 8 atoms per thread (at most 16 warps per
        // SM, little L1 beside their shared memory) take the list groups
        // one ahead: the load of the next 16-byte group, and of the next
        // atom's first group, is issued before the current group's pairs.
        constexpr bool PREF = MIXED && APT >= 4;
        uint4 nxt = make_uint4(0u, 0u, 0u, 0u);
        if constexpr (PREF) {
            if (tid < N && (ncnt[0] & 0xffff) > 0) nxt = nbr4[tid];
        }
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            R fx = 0, fy = 0, fz = 0, w = 0;
            if (i < N) {
                const int kv = ACTIVE ? ncnt[q] & 0xffff : ncnt[q], kac = (unsigned int)ncnt[q] >> 16;
                const bool verlet = !ACTIVE || FILTER || kac == 0xffff;
                const int kk = verlet ? kv : kac;
                const uint4 *lst = verlet ? nbr4 : nbra4;
                int ka = 0;
                // entry e of atom i's active list
                auto aslot = [&](int e) { return ((size_t)(e >> 3) * nmax + i) * 8 + (e & 7); };
                if constexpr (MIXED) {
                    const float4 u = pos4[i];
                    const float Lx = cf->Lf[0], Ly = cf->Lf[1], Lz = cf->Lf[2];
                    const float ix = cf->invLf[0], iy = cf->invLf[1], iz = cf->invLf[2];
                    const float dl = cf->delta_f;
                    const float2 ux2 = make_float2(u.x, u.x), uy2 = make_float2(u.y, u.y),
                                 uz2 = make_float2(u.z, u.z);
                    const float2 Lx2 = make_float2(Lx, Lx), Ly2 = make_float2(Ly, Ly), Lz2 = make_float2(Lz, Lz);
                    const float2 ix2 = make_float2(ix, ix), iy2 = make_float2(iy, iy), iz2 = make_float2(iz, iz);
                    const float2 dl2 = make_float2(dl, dl);
                    const float2 c48 = make_float2(48.f, 48.f), cm24 = make_float2(-24.f, -24.f);
                    for (int t8 = 0; t8 < kk; t8 += 8) {
                      uint4 ch;
                      if constexpr (PREF) {
                          ch = nxt;
                          if (t8 + 8 < kk) {
                              nxt = lst[(size_t)((t8 >> 3) + 1) * nmax + i];
                          } else if (q + 1 < APT && i + T < N && (ncnt[q + 1] & 0xffff) > 0) {
                              nxt = nbr4[i + T];
                          }
                      } else {
                          ch = lst[(size_t)(t8 >> 3) * nmax + i];
                      }
                      const unsigned int wv[4] = {ch.x, ch.y, ch.z, ch.w};
#pragma unroll
                      for (int wq = 0; wq < 4; wq++) {
                        if (t8 + 2 * wq >= kk) break;
                        const unsigned int word = wv[wq];
                        // the word's two entries as one packed float pair
                        // (FADD2/FFMA2/FMUL2: half the issue slots); the sums
                        // stay in list order, entry 0 then entry 1
                        const float4 v0 = pos4[word & 0xffffu], v1 = pos4[word >> 16];
                        float2 dx = __fadd2_rn(ux2, make_float2(-v0.x, -v1.x));
                        float2 dy = __fadd2_rn(uy2, make_float2(-v0.y, -v1.y));
                        float2 dz = __fadd2_rn(uz2, make_float2(-v0.z, -v1.z));
                        const float2 mny = neg2(rint2(dy, iy2));
                        dy = __ffma2_rn(mny, Ly2, dy);
                        dx = __ffma2_rn(mny, dl2, dx);
                        dx = __ffma2_rn(neg2(rint2(dx, ix2)), Lx2, dx);
                        dz = __ffma2_rn(neg2(rint2(dz, iz2)), Lz2, dz);
                        float2 r2 = __fmul2_rn(dx, dx);
                        r2 = __ffma2_rn(dy, dy, r2);
                        r2 = __ffma2_rn(dz, dz, r2);
                        const float2 sv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
                        const float2 s3 = __fmul2_rn(__fmul2_rn(sv, sv), sv);
                        float2 f = __fmul2_rn(__fmul2_rn(s3, sv), __ffma2_rn(c48, s3, cm24));   // |F|/r
                        const bool in0 = (r2.x < rc2) && (r2.x > 0.f);   // r = 0: padding
                        const bool in1 = (r2.y < rc2) && (r2.y > 0.f);
                        f.x = in0 ? f.x : 0.f;
                        f.y = in1 ? f.y : 0.f;
                        const float2 fdx = __fmul2_rn(f, dx);
                        fx = __fmaf_rn(f.x, dx.x, fx); fy = __fmaf_rn(f.x, dy.x, fy); fz = __fmaf_rn(f.x, dz.x, fz);
                        w = __fmaf_rn(fdx.x, dy.x, w);
                        fx = __fmaf_rn(f.y, dx.y, fx); fy = __fmaf_rn(f.y, dy.y, fy); fz = __fmaf_rn(f.y, dz.y, fz);
                        w = __fmaf_rn(fdx.y, dy.y, w);
                        if constexpr (FILTER) npairs += (in0 ? 1u : 0u) + (in1 ? 1u : 0u);
                      }
                    }
                } else {
                    const R ra2 = (R)cf->ra2;
                    for (int t = 0; t < kk; t++) {
                        const uint4 ch = lst[(size_t)(t >> 3) * nmax + i];
                        const int u = (t >> 1) & 3;
                        const unsigned int word = u == 0 ? ch.x : u == 1 ? ch.y : u == 2 ? ch.z : ch.w;
                        const int j = (t & 1) ? (int)(word >> 16) : (int)(word & 0xffffu);
                        R dx, dy, dz;
                        pair_vec(i, j, dx, dy, dz);
                        const R r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < rc2 && r2 > (R)0) {
                            const R s = 1.0 / r2;
                            const R s3 = s * s * s;
                            const R f = s3 * s * ((R)48 * s3 - (R)24);   // |F|/r
                            fx += f * dx; fy += f * dy; fz += f * dz;
                            w += f * dx * dy;
                            if constexpr (FILTER) npairs++;
                        }
                        if constexpr (FILTER && ACTIVE) {
                            if (r2 < ra2 && r2 > (R)0) {
                                if (ka < CAP_A) nbra16[aslot(ka)] = (unsigned short)j;
                                ka++;
                            }
                        }
                    }
                }
                if constexpr (FILTER && ACTIVE) {
                    // an odd count is padded with i itself (r = 0 adds nothing)
                    if (ka <= CAP_A && (ka & 1)) nbra16[aslot(ka)] = (unsigned short)i;
                    ncnt[q] = kv | ((ka > CAP_A ? 0xffff : ka) << 16);
                    reinterpret_cast<float *>(ref4 + i)[3] = 0.f;   // path length since the refresh
                }
            }
            F[q][0] = fx; F[q][1] = fy; F[q][2] = fz;
            wsum += w;
        }
        return wsum;
    };

    // thread 0: coefficients of the next step from K2_end, a_end, e1, delta.
    // FP64 mode: IEEE double; divisions and rint are avoided on this serial
    // chain.
    auto next_alpha = [&]() {
        const double inc = m->hhQ * (K2_end - b.gT);
        a_cur = a_end + inc;                       // start-of-step alpha half-step
        const double e3 = expm1_small(-a_cur * hh);
        const double ec = fma(e1, e3, e1 + e3);    // (1+e1)(1+e3) - 1
        e1 = e3;
        f1sq = (1.0 + e3) * (1.0 + e3);
        cf->f1 = sfrom<S>(f1sq);
        cf->e = sfrom<S>(ec);
    };
    // Active lists stay complete while every atom's path length since the
    // refresh is at most (s_a - |change of delta|) / 2: a pair then moved
    // together by at most s_a.  1e-4 sigma of margin covers the FP32
    // rounding of the path sums and of r^2.
    auto set_thr_a = [&]() {
        const float tha = 0.5f * (fminf(ACTIVE_SKIN, b.skin) - m->dsince_a) - 1e-4f;
        cf->thr_a = tha > 0.f ? tha : -1.f;
    };
    auto next_delta = [&]() {
        delta += m->ddelta;                        // sliding-brick offset advance
        if (delta >= m->halfLx) delta -= b.L[0];
        else if (delta < -m->halfLx) delta += b.L[0];
        dsince += fabsf((float)m->ddelta);
        m->dsince_a += fabsf((float)m->ddelta);
        cf->delta_d = delta; cf->delta_s = sfrom<S>(delta); cf->delta_f = (float)delta;
        const float thr = 0.5f * (b.skin - dsince);
        cf->thr2 = thr > 0.f ? thr * thr : -1.f;
        set_thr_a();
    };
    // MIXED: the same two updates in double-float; inc = hhQ (K2_end - gT)
    // is the increment of both alpha half-steps
    auto next_alpha_f = [&](df inc) {
        const df acur = df_add(m->a_endf, inc);    // start-of-step alpha half-step
        m->a_curf = acur;
        const df e3 = df_expm1_small(df_mul(m->nhhf, acur), m->sixthf);
        const df ec = df_add(df_add(m->e1f, e3), df_mul(m->e1f, e3));   // (1+e1)(1+e3) - 1
        m->e1f = e3;
        const df g = df_add_f(e3, 1.0f);
        m->f1f = df_mul(g, g);
        cf->f1 = sfrom_df<S>(m->f1f);
        cf->e = sfrom_df<S>(ec);
    };
    auto next_delta_f = [&]() {
        df dl = df_add(m->deltaf, m->ddeltaf);     // sliding-brick offset advance
        if (df_ge(dl, m->halfLxf)) dl = df_add(dl, df_neg(m->Lxf));
        else if (df_lt(dl, df_neg(m->halfLxf))) dl = df_add(dl, m->Lxf);
        m->deltaf = dl;
        dsince += m->ddelta_abs;
        cf->delta_s = sfrom_df<S>(dl); cf->delta_f = dl.hi;
        const float thr = 0.5f * (b.skin - dsince);
        cf->thr2 = thr > 0.f ? thr * thr : -1.f;
    };
    auto next_step = [&]() {
        if constexpr (MIXED) {
            next_alpha_f(df_mul(m->hhQf, df_add(m->K2f, m->ngTf)));
            next_delta_f();
        } else {
            next_alpha(); next_delta();
        }
    };

    // ---- forces and sums of the initial state ----
    build_list();
    if (tid == 0) m->n_rebuild++;
    R w0;
    if constexpr (ACTIVE) {   // the first Verlet pass also builds the active lists
        w0 = forces(std::true_type{});
        if (tid == 0) m->n_filter++;
    } else {
        w0 = forces(std::false_type{});
    }
    if (a.force_out) {
        double *fo = a.force_out + (size_t)d * 3 * N;
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            if (i < N) { fo[i] = (double)F[q][0]; fo[N + i] = (double)F[q][1]; fo[2 * N + i] = (double)F[q][2]; }
        }
    }
    {
        R s2 = 0, sxy = 0;
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            if (i < N) {
                const R px = (R)shi(P[q][0]), py = (R)shi(P[q][1]), pz = (R)shi(P[q][2]);
                s2 += px * px + py * py + pz * pz;
                sxy += px * py;
            }
        }
        double sums[3];
        cta_sum3<MIXED, R>(s2, sxy, w0, m, sums);
        if (tid == 0) {
            if (a.wxy_out) a.wxy_out[d] = 0.5 * sums[2];
            if (a.fresh) {
                K2_end = sums[0];
                if constexpr (MIXED) m->K2f = df_from_double(sums[0]);
            }
            if (m->flag_ovf) cf->stop = TTCF_D_NBR_OVERFLOW;
            if (m->flag_lost) cf->stop |= TTCF_D_NONFINITE;
            if (a.step1 > a.step0) next_step();
        }
    }
    __syncthreads();

    // ---- the steps ----
    const size_t series = (size_t)dl * b.S;
    for (int s = a.step0 + 1; s <= a.step1; s++) {
        if (cf->stop) break;
        const S e = cf->e, chalf = cf->chalf, hS = cf->h, hhS = cf->hh, gh = cf->gh;
        const bool wrap_now = (s % WRAP_EVERY) == 0;
        const int fb = s & 1;
        const float thr2 = cf->thr2, fast2 = cf->fast2, thr_a = cf->thr_a;
        // phase A
        bool packed_a = false;
        if constexpr (MIXED && APT % 2 == 0) {
            // a thread's atoms q and q+1 side by side on packed FP32 pairs:
            // the same operations as the scalar path below, lane by lane
            // (that path runs the steps that re-wrap positions)
            packed_a = !wrap_now;
            if (packed_a) {
                const float2 ef2 = f2(e.hi), ncf2 = f2(-chalf.hi);
                TTCF_Q_UNROLL
                for (int q = 0; q < APT; q += 2) {
                    const int i0 = tid + q * T, i1 = i0 + T;
                    if (i0 >= N) continue;
                    const bool has1 = i1 < N;
                    const int j1 = has1 ? i1 : i0;   // a missing second atom repeats the first
                    df2 pp[3];
#pragma unroll
                    for (int c = 0; c < 3; c++)
                        pp[c] = {make_float2(P[q][c].hi, P[q + 1][c].hi), make_float2(P[q][c].lo, P[q + 1][c].lo)};
#pragma unroll
                    for (int c = 0; c < 3; c++) acc_add2(pp[c], __fmul2_rn(pp[c].hi, ef2));
                    acc_add2(pp[0], __fmul2_rn(ncf2, pp[1].hi));
#pragma unroll
                    for (int c = 0; c < 3; c++) acc_add2(pp[c], mul_cf2(hhS, make_float2(F[q][c], F[q + 1][c])));
#pragma unroll
                    for (int c = 0; c < 3; c++) renorm2(pp[c]);
                    const float4 h0 = pos4[i0], h1 = pos4[j1], l0 = plo4[i0], l1 = plo4[j1];
                    df2 x = {make_float2(h0.x, h1.x), make_float2(l0.x, l1.x)};
                    df2 y = {make_float2(h0.y, h1.y), make_float2(l0.y, l1.y)};
                    df2 z = {make_float2(h0.z, h1.z), make_float2(l0.z, l1.z)};
                    const float2 ddx = mul_cd2(hS, pp[0]), ddy = mul_cd2(hS, pp[1]), ddz = mul_cd2(hS, pp[2]);
                    const float2 ys = __fmul2_rn(f2(gh.hi), __ffma2_rn(f2(hhS.hi), pp[1].hi, y.hi));
                    acc_add2(x, ddx); acc_add2(x, ys); acc_add2(y, ddy); acc_add2(z, ddz);
                    renorm2(x); renorm2(y); renorm2(z);
                    const float2 dxs = __fadd2_rn(ddx, ys);
                    const float2 d2 = __ffma2_rn(ddz, ddz, __ffma2_rn(ddy, ddy, __fmul2_rn(dxs, dxs)));
                    if (d2.x > fast2 || (has1 && d2.y > fast2)) m->flag_fast = 1;
                    const float4 r0 = ref4[i0], r1 = ref4[j1];
                    pos4[i0] = make_float4(x.hi.x, y.hi.x, z.hi.x, 0.f);
                    plo4[i0] = make_float4(x.lo.x, y.lo.x, z.lo.x, 0.f);
                    if (has1) {
                        pos4[i1] = make_float4(x.hi.y, y.hi.y, z.hi.y, 0.f);
                        plo4[i1] = make_float4(x.lo.y, y.lo.y, z.lo.y, 0.f);
                    }
                    const float2 ex = sub2(x.hi, make_float2(r0.x, r1.x));
                    const float2 ey = sub2(y.hi, make_float2(r0.y, r1.y));
                    const float2 ez = sub2(z.hi, make_float2(r0.z, r1.z));
                    const float2 e2 = __ffma2_rn(ez, ez, __ffma2_rn(ey, ey, __fmul2_rn(ex, ex)));
                    if (e2.x > thr2 || (has1 && e2.y > thr2)) m->flag_rebuild[fb] = 1;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        P[q][c] = {pp[c].hi.x, pp[c].lo.x};
                        P[q + 1][c] = {pp[c].hi.y, pp[c].lo.y};
                    }
                }
            }
        }
        TTCF_Q_UNROLL
        for (int q = 0; q < APT && !packed_a; q++) {
            const int i = tid + q * T;
            if (i >= N) continue;
            S px = P[q][0], py = P[q][1], pz = P[q][2];
            S x, y, z;
            float ddx, ddy, ddz;
            if constexpr (MIXED) {
                // p *= 1 + e, p_x -= gamma h/2 p_y, p += h/2 F: the products are
                // small beside p, so they are formed in float from the hi parts
                const float ef = e.hi, cf_ = chalf.hi;
                acc_add(px, px.hi * ef); acc_add(py, py.hi * ef); acc_add(pz, pz.hi * ef);
                acc_add(px, -cf_ * py.hi);
                acc_add(px, mul_cf(hhS, F[q][0]));
                acc_add(py, mul_cf(hhS, F[q][1]));
                acc_add(pz, mul_cf(hhS, F[q][2]));
                renorm(px); renorm(py); renorm(pz);
                const float4 hi = pos4[i], lo = plo4[i];
                x = {hi.x, lo.x}; y = {hi.y, lo.y}; z = {hi.z, lo.z};
                // drift: h p (to float precision of the increment) and the
                // streaming term gamma h (y + h p_y/2) as its own increment
                ddx = mul_cd(hS, px); ddy = mul_cd(hS, py); ddz = mul_cd(hS, pz);
                const float ys = gh.hi * __fmaf_rn(hhS.hi, py.hi, y.hi);
                acc_add(x, ddx); acc_add(x, ys); acc_add(y, ddy); acc_add(z, ddz);
                renorm(x); renorm(y); renorm(z);
                ddx += ys;
            } else {
                px = px + px * e; py = py + py * e; pz = pz + pz * e;
                px = px - chalf * py;
                px += hhS * F[q][0]; py += hhS * F[q][1]; pz += hhS * F[q][2];
                x = xd[i]; y = yd[i]; z = zd[i];
                const double dxs = hS * px + gh * (y + hhS * py);
                const double dys = hS * py, dzs = hS * pz;
                x += dxs; y += dys; z += dzs;
                ddx = (float)dxs; ddy = (float)dys; ddz = (float)dzs;
            }
            const float dd2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (dd2 > fast2) m->flag_fast = 1;
            float4 r = ref4[i];
            if constexpr (ACTIVE) {   // path length since the active-list refresh
                r.w += sqrtf(dd2);
                if (r.w > thr_a) m->flag_filter[fb] = 1;
            }
            if (wrap_now) {   // back into [-L/2, L/2) with the sliding-brick x shift;
                              // the reference moves with it (same periodic image)
                R ny, nx, nz;
                if constexpr (MIXED) ny = rint_fma(y.hi, cf->invLf[1]);
                else ny = rint(y * cf->invL[1]);
                y = sadd(y, sneg(smulf(cf->L[1], ny)));
                x = sadd(x, sneg(smulf(cf->delta_s, ny)));
                if constexpr (MIXED) nx = rint_fma(x.hi, cf->invLf[0]);
                else nx = rint(x * cf->invL[0]);
                x = sadd(x, sneg(smulf(cf->L[0], nx)));
                if constexpr (MIXED) nz = rint_fma(z.hi, cf->invLf[2]);
                else nz = rint(z * cf->invL[2]);
                z = sadd(z, sneg(smulf(cf->L[2], nz)));
                r.x -= (float)ny * cf->delta_f + (float)nx * cf->Lf[0];
                r.y -= (float)ny * cf->Lf[1];
                r.z -= (float)nz * cf->Lf[2];
                ref4[i] = r;
            } else if constexpr (ACTIVE) {
                reinterpret_cast<float *>(ref4 + i)[3] = r.w;
            }
            if constexpr (MIXED) {
                pos4[i] = make_float4(x.hi, y.hi, z.hi, 0.f);
                plo4[i] = make_float4(x.lo, y.lo, z.lo, 0.f);
            } else {
                xd[i] = x; yd[i] = y; zd[i] = z;
            }
            const float ex = (float)shi(x) - r.x, ey = (float)shi(y) - r.y, ez = (float)shi(z) - r.z;
            if (ex * ex + ey * ey + ez * ez > thr2) m->flag_rebuild[fb] = 1;
            P[q][0] = px; P[q][1] = py; P[q][2] = pz;
        }
        __syncthreads();                                        // barrier 1
        if (m->flag_fast) break;
        const bool rebuild = m->flag_rebuild[fb] || thr2 < 0.f;
        if (rebuild) {
            build_list();
            if (tid == 0) { dsince = 0.f; m->n_rebuild++; }
        }
        // FP64: refresh the active lists when due; MIXED: count the pairs on
        // the first of every 16 steps
        const bool refresh = ACTIVE ? (rebuild || m->flag_filter[fb] || thr_a < 0.f)
                                    : ((s - a.step0) & 15) == 1;
        if constexpr (ACTIVE) {   // (MIXED keeps these off thread 0's per-step chain)
            if (refresh && tid == 0) { m->dsince_a = 0.f; m->n_filter++; }
        }
        // phase B: over the Verlet lists (refreshing the active lists) or
        // over the active lists
        const R wsum = refresh ? forces(std::true_type{}) : forces(std::false_type{});
        // phase C
        R s2 = 0, sxy = 0;
        if constexpr (MIXED && APT % 2 == 0) {   // atoms q and q+1 on packed pairs
            const float2 ncf2 = f2(-chalf.hi);
            TTCF_Q_UNROLL
            for (int q = 0; q < APT; q += 2) {
                const int i0 = tid + q * T;
                if (i0 >= N) continue;
                const bool has1 = i0 + T < N;
                df2 pp[3];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    pp[c] = {make_float2(P[q][c].hi, P[q + 1][c].hi), make_float2(P[q][c].lo, P[q + 1][c].lo)};
                    acc_add2(pp[c], mul_cf2(hhS, make_float2(F[q][c], F[q + 1][c])));
                }
                acc_add2(pp[0], __fmul2_rn(ncf2, pp[1].hi));
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    renorm2(pp[c]);
                    P[q][c] = {pp[c].hi.x, pp[c].lo.x};
                    P[q + 1][c] = {pp[c].hi.y, pp[c].lo.y};
                }
                const float2 hx = pp[0].hi, hy = pp[1].hi, hz = pp[2].hi;
                const float2 t2 = __ffma2_rn(hz, hz, __ffma2_rn(hy, hy, __fmul2_rn(hx, hx)));
                s2 = __fadd_rn(s2, t2.x);
                sxy = __fmaf_rn(hx.x, hy.x, sxy);
                if (has1) {
                    s2 = __fadd_rn(s2, t2.y);
                    sxy = __fmaf_rn(hx.y, hy.y, sxy);
                }
            }
        } else {
            TTCF_Q_UNROLL
            for (int q = 0; q < APT; q++) {
                const int i = tid + q * T;
                if (i >= N) continue;
                S px = P[q][0], py = P[q][1], pz = P[q][2];
                if constexpr (MIXED) {
                    acc_add(px, mul_cf(hhS, F[q][0]));
                    acc_add(py, mul_cf(hhS, F[q][1]));
                    acc_add(pz, mul_cf(hhS, F[q][2]));
                    acc_add(px, -chalf.hi * py.hi);
                    renorm(px); renorm(py); renorm(pz);
                } else {
                    px += hhS * F[q][0]; py += hhS * F[q][1]; pz += hhS * F[q][2];
                    px = px - chalf * py;
                }
                P[q][0] = px; P[q][1] = py; P[q][2] = pz;
                const R hx = (R)shi(px), hy = (R)shi(py), hz = (R)shi(pz);
                if constexpr (MIXED) {   // the packed path's operations, in order
                    s2 = __fadd_rn(s2, __fmaf_rn(hz, hz, __fmaf_rn(hy, hy, __fmul_rn(hx, hx))));
                    sxy = __fmaf_rn(hx, hy, sxy);
                } else {
                    s2 += hx * hx + hy * hy + hz * hz;
                    sxy += hx * hy;
                }
            }
        }
        // step end, on three lanes at once (warp 0: the alpha chain; warp
        // wo: B(s), flags, snapshots; warp wd: the Lees-Edwards offset),
        // each reading only what the others do not write before barrier 3
        const int nw = T >> 5;
        const int wo = nw > 1 ? 1 : 0, wd = nw > 2 ? 2 : 0;
        double f1sq_s = 0.0, e1_s = 0.0;
        df e1f_s = df_make(0.f);
        if (tid == 32 * wo) {                                   // this step's values
            if constexpr (MIXED) e1f_s = m->e1f;
            else { f1sq_s = f1sq; e1_s = e1; }
        }
        double sums[3];
        df sumsf[2];
        if constexpr (MIXED) {
            // V P_xy = (1+e1)^2 sum p_x p_y + W_xy/2 formed per thread, so that
            // two sums are reduced instead of three
            const df f1 = cf->f1;
            const float pv = __fmaf_rn(0.5f, wsum, mul_cf(f1, sxy));
            cta_sum2_fix(s2, pv, m, sumsf, wo);                // barrier 2
        } else {
            cta_sum3<MIXED, R>(s2, sxy, wsum, m, sums, wo);     // barrier 2
        }
        const bool last_save = s == a.step1 && a.save_state;
        int snap_k = -1;
        if (a.snap && s >= a.snap_first && (s - a.snap_first) % a.snap_every == 0 &&
            (s - a.snap_first) / a.snap_every < a.n_snap)
            snap_k = (s - a.snap_first) / a.snap_every;
        double *sc = last_save ? b.scal + 4 * (size_t)dl : nullptr;
        if (tid == 32 * wo) {
            // end of step s: pending factor (1+e1)^2 = f1sq from the scale half-step
            double pxy;
            int st = 0;
            if constexpr (MIXED) {
                pxy = df_to_double(sumsf[1]) * m->invV;
                if (!isfinite(sumsf[0].hi + sumsf[1].hi)) st |= TTCF_D_NONFINITE;
            } else {
                pxy = fma(f1sq_s, sums[1], 0.5 * sums[2]) * m->invV;
                if (!isfinite(sums[0] + sums[1] + sums[2])) st |= TTCF_D_NONFINITE;
            }
            if (m->flag_ovf) st |= TTCF_D_NBR_OVERFLOW;
            if (m->flag_lost) st |= TTCF_D_NONFINITE;
            if (a.abort_flag && (s & 63) == 0 && *a.abort_flag) st |= TTCF_D_ABORTED;
            if (st) atomicOr(&cf->stop, st);
            if (s % a.sample_every == 0) b.B[series + s / a.sample_every] = pxy;
            cf->snap = snap_k;
            if (snap_k >= 0) cf->fsnap = MIXED ? df_to_double(df_add_f(e1f_s, 1.0f)) : 1.0 + e1_s;
        }
        unsigned long long *scu = reinterpret_cast<unsigned long long *>(sc);
        if (tid == 32 * wd) {
            if constexpr (MIXED) {
                if (last_save) store_slot(scu + 3, m->deltaf);
                next_delta_f();
            } else {
                if (last_save) sc[3] = delta;
                next_delta();
            }
        }
        if (tid == 0) {
            if constexpr (MIXED) {
                const df K2 = df_mul(m->f1f, sumsf[0]);
                m->K2f = K2;
                const df inc = df_mul(m->hhQf, df_add(K2, m->ngTf));
                const df aend = df_add(m->a_curf, inc);          // end-of-step alpha half-step
                m->a_endf = aend;
                if (snap_k >= 0) a.snap_alpha[(size_t)d * a.n_snap + snap_k] = df_to_double(aend);
                if (last_save) { store_slot(scu, aend); store_slot(scu + 1, K2); store_slot(scu + 2, m->e1f); }
                next_alpha_f(inc);
            } else {
                K2_end = f1sq * sums[0];
                a_end = a_cur + m->hhQ * (K2_end - b.gT);       // end-of-step alpha half-step
                if (snap_k >= 0) a.snap_alpha[(size_t)d * a.n_snap + snap_k] = a_end;
                if (last_save) { sc[0] = a_end; sc[1] = K2_end; sc[2] = e1; }
                next_alpha();
            }
            m->flag_rebuild[fb ^ 1] = 0;
            if constexpr (ACTIVE) m->flag_filter[fb ^ 1] = 0;
        }
        __syncthreads();                                        // barrier 3
        if (cf->snap >= 0) {   // mother mode: store the clean phase point
            double *o = a.snap + ((size_t)d * a.n_snap + cf->snap) * 6 * N;
            const double fs = cf->fsnap;
            TTCF_Q_UNROLL
            for (int q = 0; q < APT; q++) {
                const int i = tid + q * T;
                if (i >= N) continue;
                double x, y, z;
                if constexpr (MIXED) {
                    const float4 hi = pos4[i], lo = plo4[i];
                    x = df_to_double({hi.x, lo.x}); y = df_to_double({hi.y, lo.y}); z = df_to_double({hi.z, lo.z});
                } else { x = xd[i]; y = yd[i]; z = zd[i]; }
                y -= b.L[1] * rint(y * cf->invL[1]);   // mothers have gamma = 0, delta = 0
                x -= b.L[0] * rint(x * cf->invL[0]);
                z -= b.L[2] * rint(z * cf->invL[2]);
                if (x >= 0.5 * b.L[0]) x -= b.L[0];
                if (y >= 0.5 * b.L[1]) y -= b.L[1];
                if (z >= 0.5 * b.L[2]) z -= b.L[2];
                o[i] = x; o[N + i] = y; o[2 * N + i] = z;
                o[3 * N + i] = fs * sdbl(P[q][0]);
                o[4 * N + i] = fs * sdbl(P[q][1]);
                o[5 * N + i] = fs * sdbl(P[q][2]);
            }
        }
    }

    // ---- end of the chunk ----
    if (a.save_state && b.state) {
        unsigned long long *dst = b.state + (size_t)dl * 6 * N;
        TTCF_Q_UNROLL
        for (int q = 0; q < APT; q++) {
            const int i = tid + q * T;
            if (i >= N) continue;
            S x, y, z;
            if constexpr (MIXED) {
                const float4 hi = pos4[i], lo = plo4[i];
                x = {hi.x, lo.x}; y = {hi.y, lo.y}; z = {hi.z, lo.z};
            } else { x = xd[i]; y = yd[i]; z = zd[i]; }
            store_slot(dst + i, x); store_slot(dst + N + i, y); store_slot(dst + 2 * N + i, z);
            store_slot(dst + 3 * N + i, P[q][0]); store_slot(dst + 4 * N + i, P[q][1]);
            store_slot(dst + 5 * N + i, P[q][2]);
        }
        if (tid == 0 && a.step1 == a.step0) {   // no step ran: state unchanged
            double *sc = b.scal + 4 * (size_t)dl;
            if constexpr (MIXED) {
                unsigned long long *scu = reinterpret_cast<unsigned long long *>(sc);
                store_slot(scu, m->a_endf); store_slot(scu + 1, m->K2f);
                store_slot(scu + 2, m->e1f); store_slot(scu + 3, m->deltaf);
            } else {
                sc[0] = a_end; sc[1] = K2_end; sc[2] = e1; sc[3] = delta;
            }
        }
    }
    {
        unsigned long long np = npairs;
        for (int o = 16; o > 0; o >>= 1) np += __shfl_down_sync(0xffffffffu, np, o);
        if ((tid & 31) == 0 && np) atomicAdd(&m->np, np);
    }
    __syncthreads();
    if (tid == 0) {
        // pairs were counted on the Verlet-list passes (FP64: the initial
        // pass and the refreshes; MIXED: the first of every 16 steps): their
        // mean per pass times the steps of this run
        const int nrun = a.step1 - a.step0;
        const unsigned int passes = ACTIVE ? m->n_filter : (unsigned int)((nrun + 15) / 16);
        if (passes && nrun > 0)
            atomicAdd(&b.pairs[dl], (unsigned long long)llrint((double)m->np * (double)nrun / (double)passes));
        int st = cf->stop;
        if (m->flag_fast) st |= TTCF_D_FAST_ATOM;
        if (m->flag_ovf) st |= TTCF_D_NBR_OVERFLOW;
        if (m->flag_lost) st |= TTCF_D_NONFINITE;
        b.status[dl] |= st;
        b.rebuilds[dl] += m->n_rebuild;
    }
    __syncthreads();
}

template <bool MIXED, int APT, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) daughter_kernel(RunArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int w = s_item;
        __syncthreads();
        if (w >= a.n_work) break;
        run_daughter<MIXED, APT>(a, a.work[w], smem);
    }
}

// ------------------------------------------------------------ launchers --
template <bool MIXED, int APT, int MAXT, int MINB>
cudaError_t launch_one(const RunArgs &a, int threads, int grid, size_t smem,
                              cudaStream_t st) {
    auto k = daughter_kernel<MIXED, APT, MAXT, MINB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <bool MIXED, int APT, int MAXT, int MINB>
int occupancy_one(int threads, size_t smem) {
    auto k = daughter_kernel<MIXED, APT, MAXT, MINB>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace ttcf
