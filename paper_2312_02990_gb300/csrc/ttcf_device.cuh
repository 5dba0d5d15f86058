// ttcf_device.cuh -- device-side building blocks of the TTCF engine.
//
// Precision scheme of the MIXED mode (GB300 runs IEEE double at 1/72 of the
// FP32 rate, and float<->double conversions on the same slow pipe):
//  * positions and momenta are unevaluated sums hi + lo of two floats
//    ("double-float", about 48 significand bits), updated with the
//    error-free transformations TwoSum (Knuth) and FMA-based TwoProduct
//    (Dekker 1971), all on the FP32 pipe;
//  * pair forces and the virial are plain FP32, from the hi parts;
//  * the per-step chain of per-daughter scalars (Nose-Hoover alpha, the
//    momentum factor, the Lees-Edwards offset, the CTA sums behind B(s))
//    is double-float too, computed by one lane each: an IEEE-double
//    instruction costs about a hundred cycles of latency there;
//  * Omega(0), B(s) as stored and every accumulation over daughters are
//    IEEE double.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ttcf {

constexpr int CAP = 32;          // Verlet neighbours kept per atom
// Active list: the Verlet entries within r_c + ACTIVE_SKIN, refreshed from
// the (index-sorted) Verlet list whenever an atom's path length since the
// last refresh could close the gap; the force loop walks it on the other
// steps.  Up to CAP_A entries; an atom with more uses its Verlet list.
constexpr int CAP_A = 24;
constexpr float ACTIVE_SKIN = 0.1f;
constexpr int NBR_WORDS = (CAP + CAP_A) / 2;   // uint32 words per atom, both lists
constexpr int WRAP_EVERY = 64;   // positions re-wrapped into the box every 64 steps
constexpr int MAX_WARPS = 32;

// Phase-space mappings of a mother state (Eq. 3 and the further choices the
// paper lists after it).  Mapping code m: bit 0 time reversal (p -> -p,
// alpha -> -alpha), bit 1 x-reflection (x -> -x, p_x -> -p_x), bit 2
// y-reflection, bit 3 z-reflection, bit 4 exchange of the x and z
// components of positions and momenta (needs L_x = L_z), applied in the
// order exchange, reflections, time reversal.  Codes 0..3 are the four
// mappings of Eq. 3 (identity, p -> -p, the x-reflection, and the two
// combined).  Each is an isometry of the periodic box combined, for odd
// codes, with the time reversal of the Nose-Hoover flow, so it preserves the
// equilibrium measure.
constexpr int MAX_MAPS = 32;
__host__ __device__ inline bool map_reverses_time(int m) { return (m & 1) != 0; }
// sign of P_xy of the mapped state relative to the source component
// (P_xy, or P_zy = P_yz after the exchange): -1 for one reflection of x or y
__host__ __device__ inline double map_pxy_sign(int m) { return (((m >> 1) ^ (m >> 2)) & 1) ? -1.0 : 1.0; }
__host__ __device__ inline bool map_swaps_xz(int m) { return (m & 16) != 0; }

// ----------------------------------------------------------------- df ---
struct df { float hi, lo; };

__device__ __forceinline__ df df_make(float h) { return {h, 0.0f}; }

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
// Dekker's Fast2Sum, valid for |a| >= |b| (or a == 0).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
// TwoProduct with FMA; the lo*lo term is below the format's precision.
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mul_f(df a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return fast_two_sum(p, e);
}
// Lazy accumulation: add a float increment into an unnormalised pair with
// TwoSum (the rounding error goes to lo), 7 FP32 operations; renorm() makes
// |lo| <= ulp(hi)/2 again with Fast2Sum.
__device__ __forceinline__ void acc_add(df &a, float t) {
    const float s = __fadd_rn(a.hi, t);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, e);
}
__device__ __forceinline__ void renorm(df &a) { a = fast_two_sum(a.hi, a.lo); }
// Float product of a double-float constant c and a float v (one rounding).
__device__ __forceinline__ float mul_cf(df c, float v) { return __fmaf_rn(c.hi, v, __fmul_rn(c.lo, v)); }
// Float product c * a of two pairs, to float precision.
__device__ __forceinline__ float mul_cd(df c, df a) {
    return __fmaf_rn(c.hi, a.hi, __fmaf_rn(c.hi, a.lo, __fmul_rn(c.lo, a.hi)));
}
__device__ __forceinline__ df df_from_double(double x) {
    float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }
// Order of two normalised pairs (|lo| <= ulp(hi)/2): by hi, then by lo.
__device__ __forceinline__ bool df_ge(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
__device__ __forceinline__ bool df_lt(df a, df b) { return !df_ge(a, b); }

// exp(x) - 1 in double-float for the small arguments -alpha h/2, on the
// FP32 pipe.  With e = x + x^2 q, q = 1/2 + x/6 + x^2 r and
// r = 1/24 + x/120 + x^2/720 + x^3/5040: for |x| < 5e-3 the truncation is
// below 1e-16 relative, x^2 and x/6 are formed as pairs, and x^2 r (at most
// 1e-6 beside 1/2) in float, which keeps e within about 2^-48 relative.
// `sixth` is 1/6 as a pair.  Larger |x| goes through the IEEE-double routine.
__device__ __forceinline__ df df_expm1_small(df x, df sixth) {
    const float xf = x.hi;
    if (!(fabsf(xf) < 5e-3f)) return df_from_double(expm1(df_to_double(x)));
    const float r = __fmaf_rn(xf, __fmaf_rn(xf, __fmaf_rn(xf, 1.f / 5040.f, 1.f / 720.f), 1.f / 120.f),
                              1.f / 24.f);
    const df x2 = df_mul(x, x);
    df q = df_add_f(df_mul(x, sixth), __fmul_rn(x2.hi, r));
    q = df_add_f(q, 0.5f);
    return df_add(x, df_mul(x2, q));
}

// Round to nearest integer (ties to even) on the FP32 add pipe: valid for
// |v| < 2^22.  1.5*2^23 has unit spacing, so v + M rounds v once.
__device__ __forceinline__ float rint_fma(float v, float s) {
    const float M = 12582912.0f;
    return __fsub_rn(__fmaf_rn(v, s, M), M);
}

// floor(x) as an int for |x| < 2^22 on the FP32 add pipe: x + 1.5*2^23
// rounded down has floor(x) in its low mantissa bits (float->int
// conversions run at 1/8 of the FP32 rate).  NaN gives some int, which the
// callers clamp or have excluded before.
__device__ __forceinline__ int ifloor(float x) {
    return __float_as_int(__fadd_rd(x, 12582912.0f)) - 0x4B400000;
}

// Packed float pairs (sm_100+ FADD2/FFMA2/FMUL2, each lane IEEE round to
// nearest): rint_fma on both halves, and negation.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 rint2(float2 v, float2 s) {
    const float2 M = make_float2(12582912.0f, 12582912.0f);
    return __fadd2_rn(__ffma2_rn(v, s, M), neg2(M));
}

// Two float pairs side by side (lane x: one atom, lane y: another), with the
// float-pair operations above on packed FP32 instructions.  Each lane is
// IEEE round-to-nearest, so every lane gives bit for bit what the scalar
// helper gives.  a - b is formed as fma(b, -1, a), which is exact.
struct df2 { float2 hi, lo; };
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ df2 df2_add(df2 a, df2 b) {
    const float2 s = __fadd2_rn(a.hi, b.hi);          // TwoSum of the hi parts
    const float2 bb = sub2(s, a.hi);
    const float2 e = __fadd2_rn(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
    const float2 lo = __fadd2_rn(e, __fadd2_rn(a.lo, b.lo));
    const float2 h = __fadd2_rn(s, lo);               // Fast2Sum
    return {h, sub2(lo, sub2(h, s))};
}
__device__ __forceinline__ void acc_add2(df2 &a, float2 t) {   // acc_add on both lanes
    const float2 s = __fadd2_rn(a.hi, t);
    const float2 bb = sub2(s, a.hi);
    const float2 e = __fadd2_rn(sub2(a.hi, sub2(s, bb)), sub2(t, bb));
    a.hi = s;
    a.lo = __fadd2_rn(a.lo, e);
}
__device__ __forceinline__ void renorm2(df2 &a) {
    const float2 s = __fadd2_rn(a.hi, a.lo);
    a = {s, sub2(a.lo, sub2(s, a.hi))};
}
__device__ __forceinline__ float2 mul_cf2(df c, float2 v) {
    return __ffma2_rn(f2(c.hi), v, __fmul2_rn(f2(c.lo), v));
}
__device__ __forceinline__ float2 mul_cd2(df c, df2 a) {
    return __ffma2_rn(f2(c.hi), a.hi, __ffma2_rn(f2(c.hi), a.lo, __fmul2_rn(f2(c.lo), a.hi)));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// exp(x) - 1 for the small arguments -alpha h/2 (Taylor to x^7 when
// |x| < 1e-2: truncation below 1e-18 relative), else the library routine.
__device__ __forceinline__ double expm1_small(double x) {
    if (fabs(x) < 1e-2) {
        // x (1 + x/2! + ... + x^6/7!) with Estrin's grouping: four dependent
        // IEEE-double operations instead of seven (latency on one lane)
        const double x2 = x * x;
        const double q0 = fma(x, 0.5, 1.0);
        const double q1 = fma(x, 1.0 / 24.0, 1.0 / 6.0);
        const double q2 = fma(x, 1.0 / 720.0, 1.0 / 120.0);
        const double q3 = fma(x2, 1.0 / 5040.0, q2);
        const double x4 = x2 * x2;
        const double r = fma(x4, q3, fma(x2, q1, q0));
        return x * r;
    }
    return expm1(x);
}

// ------------------------------------------------ generic state algebra --
__device__ __forceinline__ df sadd(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ double sadd(double a, double b) { return a + b; }
__device__ __forceinline__ df smul(df a, df b) { return df_mul(a, b); }
__device__ __forceinline__ double smul(double a, double b) { return a * b; }
__device__ __forceinline__ df smulf(df a, float b) { return df_mul_f(a, b); }
__device__ __forceinline__ double smulf(double a, double b) { return a * b; }
__device__ __forceinline__ df sneg(df a) { return df_neg(a); }
__device__ __forceinline__ double sneg(double a) { return -a; }
__device__ __forceinline__ float shi(df a) { return a.hi; }
__device__ __forceinline__ double shi(double a) { return a; }
__device__ __forceinline__ double sdbl(df a) { return df_to_double(a); }
__device__ __forceinline__ double sdbl(double a) { return a; }
template <class S> __device__ __forceinline__ S sfrom(double x);
template <> __device__ __forceinline__ df sfrom<df>(double x) { return df_from_double(x); }
template <> __device__ __forceinline__ double sfrom<double>(double x) { return x; }
template <class S> __device__ __forceinline__ S sfrom_df(df x);
template <> __device__ __forceinline__ df sfrom_df<df>(df x) { return x; }
template <> __device__ __forceinline__ double sfrom_df<double>(df x) { return df_to_double(x); }

template <class S> __device__ __forceinline__ S load_slot(const unsigned long long *p);
template <> __device__ __forceinline__ df load_slot<df>(const unsigned long long *p) {
    float2 v = *reinterpret_cast<const float2 *>(p);
    return {v.x, v.y};
}
template <> __device__ __forceinline__ double load_slot<double>(const unsigned long long *p) {
    return *reinterpret_cast<const double *>(p);
}
__device__ __forceinline__ void store_slot(unsigned long long *p, df v) {
    *reinterpret_cast<float2 *>(p) = make_float2(v.hi, v.lo);
}
__device__ __forceinline__ void store_slot(unsigned long long *p, double v) {
    *reinterpret_cast<double *>(p) = v;
}

// Warp sums (lane 0 holds the total).
__device__ __forceinline__ df shfl_df(df v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ df warp_sum(df v) {
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, shfl_df(v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------- warp/CTA helpers --
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}
__device__ __forceinline__ double warp_incl_scan(double v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of cnt[0..n) into start[0..n], start[n] = total, over the
// whole CTA (blockDim a multiple of 32, <= 1024).  warp_tmp: 32 ints of
// shared memory.  Contains two __syncthreads.
__device__ inline void cta_exclusive_scan(const int *cnt, int *start, int n, int *warp_tmp) {
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (n + T - 1) / T;
    const int b0 = min(tid * per, n), b1 = min(b0 + per, n);
    int s = 0;
    for (int c = b0; c < b1; c++) s += cnt[c];
    int incl = warp_incl_scan(s);
    if (lane == 31) warp_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < (T >> 5) ? warp_tmp[lane] : 0;
        int vi = warp_incl_scan(v);
        if (lane < (T >> 5)) warp_tmp[lane] = vi - v;
    }
    __syncthreads();
    int off = warp_tmp[warp] + incl - s;
    for (int c = b0; c < b1; c++) { start[c] = off; off += cnt[c]; }
    if (tid == T - 1) start[n] = off;
}

// --------------------------------------------------------- descriptors ---
// One batch: the daughters spawned from mother states of one size N.
struct BatchDev {
    int N, M, G, S;          // atoms, mappings per group, groups, samples
    int maps[MAX_MAPS];      // selected mapping codes (Eq. 3 and its generalisations)
    int nc[3];               // cells per side for the neighbour build
    int ncell;
    double L[3];
    double V, Q, gT;         // volume, Nose-Hoover mass, g*T
    double T;                // k_B T
    float skin;              // Verlet skin of this batch
    int pad_;
    long long d0;            // global index of daughter 0
    const unsigned long long *mothers;   // [G][6][N] 8-byte slots
    const double *m_alpha;   // [G]
    const double *gamma;     // [G]
    double *B;               // [D][S]
    double *Omega;           // [D]
    int *status;             // [D]
    unsigned long long *pairs;   // [D]
    unsigned int *rebuilds;  // [D]
    double *scal;            // [D][4]: alpha_end, K2_end, e1, delta
    unsigned long long *state;   // [D][6][N] slots, or null
};

struct RunArgs {
    const BatchDev *batches;
    const int *work;               // global daughter indices, launch order
    const int *dbatch;             // batch of each global daughter
    int n_work;
    int *queue;                    // persistent work counter
    unsigned int *nbr;             // [grid][CAP/2][nmax] Verlet lists, then
                                   // [grid][CAP_A/2][nmax] active lists; two uint16
                                   // entries per word (NBR_WORDS words per atom)
    int nmax, ncellmax;
    int step0, step1;              // run absolute steps step0+1 .. step1
    int sample_every;
    int fresh;                     // start from the mapped mother state
    int save_state;                // write the loop state at step1
    int reset_alpha;
    double dt;
    double delta0;                 // Lees-Edwards offset of fresh daughters
    const volatile int *abort_flag;  // host-mapped, may be null
    double *snap;                  // mother mode: [D][n_snap][6][N] or null
    double *snap_alpha;            // [D][n_snap]
    int snap_first, snap_every, n_snap;
    double *force_out;             // [D][3][N] forces at step0, or null
    double *wxy_out;               // [D] virial W_xy at step0, or null
    float4 *plo_g;                 // [grid][nmax] position lo parts (plo_global variants)
    int cpos;                      // shared-memory layout: 1 = cell-ordered wrapped
                                   // positions for the list build, 0 = cell members'
                                   // indices only (see daughter_smem_bytes)
};

// Launch variants of the daughter kernel: atoms per thread, maximum block
// size and minimum resident blocks per SM (register budget).
struct Variant { int apt, maxt, minb; };
constexpr int N_VARIANTS = 6;
__host__ __device__ inline Variant variant_of(int v) {
    switch (v) {
    case 0: return {1, 256, 4};
    case 1: return {2, 512, 2};
    case 2: return {2, 1024, 1};
    case 3: return {4, 512, 2};
    case 4: return {4, 512, 1};
    default: return {8, 512, 1};
    }
}

// Default launch variant for a daughter of N atoms and the default skin
// (measured on GB300; ttcf_autotune refines both per N).
constexpr double DEFAULT_SKIN = 0.4;
__host__ __device__ inline int default_variant(int N) {
    return N <= 1024 ? 1 : N <= 2048 ? 2 : 5;
}

// Shared-memory bytes of a daughter CTA (must match the carve-up in
// ttcf_daughter.cu).  cpos: the list build reads a cell-ordered copy of the
// wrapped positions (16 bytes per atom) instead of the cell members' indices
// (2 bytes per atom).
// The MIXED variant of 8 atoms per thread keeps the lo parts of its
// positions in a per-CTA global scratch ([grid][nmax] float4, read and
// written by the owner thread in phase A only) rather than in shared
// memory; the 16 bytes per atom it frees let its N ~ 4000 daughters use the
// cell-ordered list build.
__host__ __device__ inline bool plo_global(bool mixed, int variant) { return mixed && variant >= 5; }

__host__ __device__ inline size_t daughter_smem_bytes(bool mixed, int nmax, int ncellmax,
                                                      bool cpos = false, bool plo_smem = true) {
    size_t b = mixed ? (size_t)nmax * (plo_smem ? 48 : 32)
                     : 3 * (((size_t)nmax * 8 + 15) / 16 * 16) + (size_t)nmax * 16;
    b += (size_t)ncellmax * 4 + (size_t)(ncellmax + 2) * 4;
    b += cpos ? (size_t)nmax * 16 : ((size_t)nmax * 2 + 15) / 16 * 16;
    b += 2048;   // coefficients, reduction slots and flags
    return b;
}

}  // namespace ttcf
