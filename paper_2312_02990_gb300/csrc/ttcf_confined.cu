// ttcf_confined.cu -- daughters of the confined system (Example 2).
//
// A Lennard-Jones fluid between two walls of atoms tethered by springs of
// stiffness k to lattice sites; during a daughter the bottom lattice slides
// at -v and the top one at +v in x, v = gamma h / 2 (Eq. 10).  Pair
// potential 4[r^-12 - c_ij r^-6] cut at r_c (Eq. 9), c_ij = c_ff, c_wf or,
// for wall-wall pairs, c_ww (switchable: with it off only the tethers hold
// the walls).  Fluid: velocity Verlet.  Walls: the same plus a
// Nose-Hoover multiplier on their momenta, alpha' = (sum_w p^2 - g T)/Q,
// split symmetrically E B A B E around the velocity-Verlet step.  x and z
// are periodic, y is bounded by the walls.
//
// Omega(0) = -(1/T) sum_w k (x_w - x_l) s_w v (Eq. 11 times beta with the
// sign of beta dH/dt) and the t = 0 responses come from the spawn kernel in
// IEEE double.  Each sample of a daughter records
//   B[0], B[1]   x force of the fluid on the bottom / top wall per area
//   B[2 + k]     sum of fluid p_x in slab k of 40 spanning y
//   B[42 + k]    number of fluid atoms in slab k
//   B[82], B[83] sum of p_x over the innermost layer of the bottom / top
//                wall (the wall's atoms whose tether site lies within 0.1
//                sigma in y of its site plane nearest the channel): the wall
//                velocity of the paper's slip velocity.
//
// One CTA of 1024 threads runs one daughter: the hi parts of the positions
// and the atom type sit in shared memory (float4); lo parts, momenta, forces,
// list references and tether sites of the current daughter live in a per-CTA
// global scratch.  Positions and momenta are float pairs (as in the bulk
// MIXED mode), pair forces FP32, alpha and all sums IEEE double.
#include "ttcf.h"
#include "ttcf_confined.h"

namespace ttcf {

namespace {

constexpr float FIX_SCALE = 1099511627776.0f;   // 2^40: fixed point of slab sums
constexpr double FIX_INV = 1.0 / 1099511627776.0;

__device__ __forceinline__ float pbc_f(float d, float L, float iL) {
    return __fmaf_rn(-rint_fma(d, iL), L, d);
}

// Minimum image of a float-pair difference along a periodic edge L.
__device__ __forceinline__ float pbc_df(df d, df L, float iL) {
    const float n = rint_fma(d.hi, iL);
    const df r = df_add(d, df_mul_f(L, -n));
    return r.hi + r.lo;
}

struct ConfCoef {
    df e;                      // combined wall momentum factor minus 1 (phase A)
    df h, hh;
    df disp;                   // lattice displacement v t at the current step
    df Ldf[3];
    float Lf[3], invLf[3];
    float skin_eff, fast2, rl2;   // rebuild threshold on |d1| + |d2|
    int stop;
};

struct ConfMisc {
    double slot[MAX_WARPS][3];
    double a_end, a_cur, K2_end, e1, f1sq, disp, hhQ, vh, snap_f;
    unsigned int n_rebuild;
    int warp_tmp[MAX_WARPS];
    float2 dtop[MAX_WARPS];       // per-warp two largest squared displacements
    int flag_fast, flag_ovf, flag_lost;
    unsigned long long slab_px[CONF_NSLAB];   // fixed point, units of 2^-40
    int slab_n[CONF_NSLAB];
    unsigned long long wall_px[2];            // inner wall layers, fixed point
};

// Shared-memory carve-up of a daughter CTA; every region starts on a
// 16-byte boundary (ConfMisc holds 8-byte fields, whatever the cell count).
__host__ __device__ inline size_t r16(size_t b) { return (b + 15) & ~(size_t)15; }
struct ConfSmem { size_t cnt, start, catom, coef, misc, total; };
__host__ __device__ inline ConfSmem conf_layout(int nmax, int ncm) {
    ConfSmem l;
    size_t o = r16((size_t)(nmax + 1) * 16);   // positions + ghost
    l.cnt = o;   o += r16((size_t)ncm * 4);
    l.start = o; o += r16((size_t)(ncm + 2) * 4);
    l.catom = o; o += r16((size_t)nmax * 2);
    l.coef = o;  o += r16(sizeof(ConfCoef));
    l.misc = o;  o += r16(sizeof(ConfMisc));
    l.total = o;
    return l;
}

__device__ __forceinline__ df shfl_down_df(df v, int o) {
    return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ df warp_sum_df(df v) {
    for (int o = 16; o > 0; o >>= 1) v = df_add(v, shfl_down_df(v, o));
    return v;
}

// Fixed-order CTA sums of three float partials in float-pair arithmetic;
// the doubles land in out[] of thread 0.  One __syncthreads.
__device__ void conf_sum3(float a0, float a1, float a2, ConfMisc *m, double out[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const df s0 = warp_sum_df(df_make(a0)), s1 = warp_sum_df(df_make(a1)), s2 = warp_sum_df(df_make(a2));
    float2 *sl = reinterpret_cast<float2 *>(&m->slot[warp][0]);
    if (lane == 0) {
        sl[0] = make_float2(s0.hi, s0.lo);
        sl[1] = make_float2(s1.hi, s1.lo);
        sl[2] = make_float2(s2.hi, s2.lo);
    }
    __syncthreads();
    if (warp == 0) {
        df t0 = {0.f, 0.f}, t1 = {0.f, 0.f}, t2 = {0.f, 0.f};
        if (lane < nw) {
            const float2 *q = reinterpret_cast<const float2 *>(&m->slot[lane][0]);
            t0 = {q[0].x, q[0].y}; t1 = {q[1].x, q[1].y}; t2 = {q[2].x, q[2].y};
        }
        t0 = warp_sum_df(t0); t1 = warp_sum_df(t1); t2 = warp_sum_df(t2);
        if (lane == 0) { out[0] = df_to_double(t0); out[1] = df_to_double(t1); out[2] = df_to_double(t2); }
    }
}

// Slab of a fluid atom, decided in double like the definition of the profile.
__device__ __forceinline__ int slab_of(double y, double Ly) {
    const int k = (int)floor((y + 0.5 * Ly) / Ly * CONF_NSLAB);
    return min(max(k, 0), CONF_NSLAB - 1);
}

__device__ void conf_daughter(const ConfRunArgs &a, int d, unsigned char *smem) {
    const int tid = threadIdx.x, T = blockDim.x;
    const ConfBatchDev &b = a.batches[a.dbatch[d]];
    const int N = b.N;
    const int dl = (int)(d - b.d0), gl = dl / b.M, map = b.maps[dl % b.M];
    const int nmax = a.nmax, ncm = a.ncellmax;
    const int nc0 = b.nc[0], nc1 = b.nc[1], nc2 = b.nc[2];

    const ConfSmem lay = conf_layout(nmax, ncm);
    float4 *pos4 = reinterpret_cast<float4 *>(smem);   // [nmax] + ghost
    int *cnt = reinterpret_cast<int *>(smem + lay.cnt);
    int *start = reinterpret_cast<int *>(smem + lay.start);
    unsigned short *catom = reinterpret_cast<unsigned short *>(smem + lay.catom);
    ConfCoef *cf = reinterpret_cast<ConfCoef *>(smem + lay.coef);
    ConfMisc *m = reinterpret_cast<ConfMisc *>(smem + lay.misc);

    // per-slot state in the CTA's global scratch: two copies of the five
    // permuted rows (the list build sorts atoms into cell order), forces and
    // list references; plo.w carries the atom's original index
    float4 *scr = a.scratch + (size_t)blockIdx.x * CONF_SCRATCH_F4 * nmax;
    float4 *plo = scr, *phi = scr + nmax, *pml = scr + 2 * (size_t)nmax;
    float4 *lath = scr + 3 * (size_t)nmax, *latl = scr + 4 * (size_t)nmax;
    float4 *alt = scr + 5 * (size_t)nmax;   // second copy of the five rows
    float4 *F4 = scr + 10 * (size_t)nmax, *ref = scr + 11 * (size_t)nmax;
    uint4 *nbr = a.nbr + (size_t)blockIdx.x * CONF_GROUPS * nmax;
    int *ncnt = a.ncnt + (size_t)blockIdx.x * nmax;

    const double h = a.dt, hh = 0.5 * a.dt;
    const float rc2 = (float)(b.rc * b.rc);
    if (tid == 0) {
        cf->h = df_from_double(h);
        cf->hh = df_from_double(hh);
        for (int k = 0; k < 3; k++) {
            cf->Ldf[k] = df_from_double(b.L[k]);
            cf->Lf[k] = (float)b.L[k];
            cf->invLf[k] = (float)(1.0 / b.L[k]);
        }
        const float rl = (float)(b.rc + b.skin);
        cf->rl2 = rl * rl;
        cf->fast2 = 0.25f * b.skin * b.skin;
        cf->skin_eff = b.skin * 0.9999f;
        cf->stop = 0;
        cf->disp = df_from_double(0.0);
        m->flag_fast = m->flag_ovf = m->flag_lost = 0;
        m->n_rebuild = 0;
        const double sa = (map == 1 || map == 3) ? -1.0 : 1.0;
        m->a_end = a.reset_alpha ? 0.0 : sa * b.m_alpha[gl];
        m->e1 = 0.0;
        m->f1sq = 1.0;
        m->disp = 0.0;
        m->hhQ = hh / b.Q;
        m->vh = b.gamma[gl] * b.half_h * h;   // lattice advance per step
        m->snap_f = 1.0;
        // the ghost that pads neighbour groups: far outside the channel in y
        // (y is not periodic), so every pair with it is out of range
        pos4[nmax] = make_float4(0.f, 1.0e4f, 0.f, 0.f);
    }
    for (int k = tid; k < CONF_NSLAB; k += T) { m->slab_px[k] = 0ull; m->slab_n[k] = 0; }
    if (tid < 2) m->wall_px[tid] = 0ull;
    __syncthreads();

    // ---- the mapped mother (Eq. 3 sign rules) and the tether sites ----
    // (lath.w marks the atoms of the innermost wall layers)
    {
        const bool flipx = map == 2 || map == 3;
        const bool flippx = map == 1 || map == 2;
        const bool flippyz = map == 1 || map == 3;
        const float2 *src = reinterpret_cast<const float2 *>(b.mothers + (size_t)gl * 6 * N);
        const float Lhx = 0.5f * cf->Lf[0];
        const df mL = df_neg(cf->Ldf[0]);
        for (int i = tid; i < N; i += T) {
            auto ld = [&](int r) { const float2 v = src[(size_t)r * N + i]; return df{v.x, v.y}; };
            df x = ld(0), y = ld(1), z = ld(2), px = ld(3), py = ld(4), pz = ld(5);
            df xl = df_from_double(b.lattice[i]);
            const df yl = df_from_double(b.lattice[(size_t)N + i]);
            const df zl = df_from_double(b.lattice[2 * (size_t)N + i]);
            if (flipx) {
                x = df_neg(x); xl = df_neg(xl);
                if (x.hi >= Lhx) x = df_add(x, mL);
                if (xl.hi >= Lhx) xl = df_add(xl, mL);
            }
            if (flippx) px = df_neg(px);
            if (flippyz) { py = df_neg(py); pz = df_neg(pz); }
            pos4[i] = make_float4(x.hi, y.hi, z.hi, (float)b.types[i]);
            plo[i] = make_float4(x.lo, y.lo, z.lo, __int_as_float(i));
            phi[i] = make_float4(px.hi, py.hi, pz.hi, 0.f);
            pml[i] = make_float4(px.lo, py.lo, pz.lo, 0.f);
            const int ty = b.types[i];
            const double ys = b.lattice[(size_t)N + i];
            const bool inner = (ty == 1 && ys >= b.inner_y[0]) || (ty == 2 && ys <= b.inner_y[1]);
            lath[i] = make_float4(xl.hi, yl.hi, zl.hi, inner ? 1.f : 0.f);
            latl[i] = make_float4(xl.lo, yl.lo, zl.lo, 0.f);
        }
    }
    __syncthreads();

    const float s0 = (float)nc0 * cf->invLf[0], s1 = (float)nc1 * cf->invLf[1], s2 = (float)nc2 * cf->invLf[2];
    const float hl0 = 0.5f * cf->Lf[0], hl1 = 0.5f * cf->Lf[1], hl2 = 0.5f * cf->Lf[2];
    auto clampc = [](int c, int n) { return min(max(c, 0), n - 1); };

    // ---- cell sort and Verlet lists (no wall-wall pairs) ----
    // Atoms are binned (x and z wrapped, y clamped to the edge cells), each
    // cell's atoms ordered by their current slot, and the per-atom state is
    // permuted into that cell order: a warp's atoms are then neighbours in
    // space, so they scan the same cells and read nearby positions.  A
    // cell's candidates are a contiguous slot range; every step is in a fixed
    // order, so lists and force sums do not depend on atomic ordering.
    auto build_list = [&]() {
        const int ncell = b.ncell;
        const float Lx = cf->Lf[0], iLx = cf->invLf[0], Ly = cf->Lf[1], Lz = cf->Lf[2], iLz = cf->invLf[2];
        const float rl2 = cf->rl2;
        const bool ww_on = b.ww_on != 0;
        for (int c = tid; c < ncell; c += T) cnt[c] = 0;
        __syncthreads();
        for (int i = tid; i < N; i += T) {
            const float4 u = pos4[i];
            const float wx = pbc_f(u.x, Lx, iLx);
            const float wz = pbc_f(u.z, Lz, iLz);
            int c = 0;
            if (fabsf(wx) <= Lx && fabsf(u.y) <= Ly && fabsf(wz) <= Lz)
                c = (clampc(ifloor((wz + hl2) * s2), nc2) * nc1 + clampc(ifloor((u.y + hl1) * s1), nc1)) * nc0 +
                    clampc(ifloor((wx + hl0) * s0), nc0);
            ref[i] = u;
            ncnt[i] = c;   // cell of the slot until the lists are written
            atomicAdd(&cnt[c], 1);
        }
        __syncthreads();
        cta_exclusive_scan(cnt, start, ncell, m->warp_tmp);
        __syncthreads();
        for (int c = tid; c < ncell; c += T) cnt[c] = start[c];
        __syncthreads();
        for (int i = tid; i < N; i += T) catom[atomicAdd(&cnt[ncnt[i]], 1)] = (unsigned short)i;
        __syncthreads();
        for (int c = tid; c < ncell; c += T)
            for (int u = start[c] + 1; u < start[c + 1]; u++) {
                const unsigned short v = catom[u];
                int w = u;
                while (w > start[c] && catom[w - 1] > v) { catom[w] = catom[w - 1]; w--; }
                catom[w] = v;
            }
        __syncthreads();
        // permutation: new slot k takes old slot catom[k]
        for (int k = tid; k < N; k += T) {
            const int o = catom[k];
            pos4[k] = ref[o];
            alt[k] = plo[o];
            alt[(size_t)nmax + k] = phi[o];
            alt[2 * (size_t)nmax + k] = pml[o];
            alt[3 * (size_t)nmax + k] = lath[o];
            alt[4 * (size_t)nmax + k] = latl[o];
        }
        {
            float4 *t = plo;
            plo = alt; phi = alt + nmax; pml = alt + 2 * (size_t)nmax;
            lath = alt + 3 * (size_t)nmax; latl = alt + 4 * (size_t)nmax;
            alt = t;
        }
        __syncthreads();
        const float rl = sqrtf(rl2);
        for (int i = tid; i < N; i += T) {
            const float4 u = pos4[i];
            ref[i] = u;
            const bool wall_i = u.w != 0.f;
            const float2 ux2 = f2(u.x), uy2 = f2(u.y), uz2 = f2(u.z);
            const float wx = pbc_f(u.x, Lx, iLx);
            const float wy = u.y;
            const float wz = pbc_f(u.z, Lz, iLz);
            // a non-finite atom, or one that left the slab extent by more
            // than Ly/2 (an atom that crossed a wall into the vacuum behind
            // it), stops the daughter and bounds the loops below.  Fluid
            // atoms inside a wall are allowed: with non-interacting tethered
            // wall atoms the model lets them through the first layers.
            if (!(fabsf(wx) <= Lx && fabsf(wy) <= Ly && fabsf(wz) <= Lz)) {
                m->flag_lost = 1;
                ncnt[i] = 0;
                continue;
            }
            const int z0 = ifloor((wz - rl + hl2) * s2);
            const int z1 = min(ifloor((wz + rl + hl2) * s2), z0 + nc2 - 1);
            const int y0 = max(ifloor((wy - rl + hl1) * s1), 0);
            const int y1 = min(ifloor((wy + rl + hl1) * s1), nc1 - 1);
            // Entries enter a 128-bit shift register (w0 holds the oldest)
            // and leave as one 16-byte store per group of 8, from group 0 up.
            // A wall atom's wall neighbours go to the last groups instead
            // (one 2-byte store each, from the last group down), so that the
            // force loop meets its fluid and wall neighbours separately.
            int k = 0, kw = 0;
            unsigned short *nbr16 = reinterpret_cast<unsigned short *>(nbr);
            unsigned int w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
            auto push = [&](unsigned int j) {
                w0 = __byte_perm(w0, w1, 0x5432);
                w1 = __byte_perm(w1, w2, 0x5432);
                w2 = __byte_perm(w2, w3, 0x5432);
                w3 = __byte_perm(w3, j, 0x5432);
            };
            // cell widths, and r_l^2 with a margin for the rounding below
            const float cw1 = Ly / (float)nc1, cw2 = Lz / (float)nc2, rl2m = rl2 * (1.f + 1e-5f);
            for (int zu = z0; zu <= z1; zu++) {
                const int zz = zu < 0 ? zu + nc2 : (zu >= nc2 ? zu - nc2 : zu);
                const float zlo = __fmaf_rn((float)zu, cw2, -hl2);
                const float dz = fmaxf(0.f, fmaxf(zlo - wz, wz - (zlo + cw2)));
                for (int yy = y0; yy <= y1; yy++) {
                    // the row's cells lie at least (dy, dz) away: rows beyond
                    // r_l are skipped and the x window is trimmed to
                    // |dx| <= sqrt(r_l^2 - dy^2 - dz^2) (lists are unchanged).
                    // The edge rows in y also hold the atoms clamped into
                    // them, so they are open towards the outside.
                    const float ylo = __fmaf_rn((float)yy, cw1, -hl1);
                    const float below = yy > 0 ? ylo - wy : 0.f;
                    const float above = yy < nc1 - 1 ? wy - (ylo + cw1) : 0.f;
                    const float dy = fmaxf(0.f, fmaxf(below, above));
                    const float h2 = rl2m - __fmaf_rn(dz, dz, dy * dy);
                    if (h2 < 0.f) continue;
                    const float hw = sqrtf(h2);
                    const int xa = ifloor((wx - hw + hl0) * s0);
                    const int xb = min(ifloor((wx + hw + hl0) * s0), xa + nc0 - 1);
                    int ra[2], rb[2], nr;
                    {
                        const int a0 = xa < 0 ? xa + nc0 : (xa >= nc0 ? xa - nc0 : xa);
                        const int b0 = a0 + (xb - xa);
                        if (b0 < nc0) { ra[0] = a0; rb[0] = b0; ra[1] = rb[1] = 0; nr = 1; }
                        else { ra[0] = a0; rb[0] = nc0 - 1; ra[1] = 0; rb[1] = b0 - nc0; nr = 2; }
                    }
                    const int row = (zz * nc1 + yy) * nc0;
                    for (int r = 0; r < nr; r++) {
                        const int t1 = start[row + rb[r] + 1];
                        auto accept = [&](int j, float r2, bool ww) {
                            if (j == i || (ww && !ww_on) || !(r2 < rl2)) return;
                            if (ww) {
                                if (kw < CONF_CAP)
                                    nbr16[((size_t)(CONF_GROUPS - 1 - (kw >> 3)) * nmax + i) * 8 + (kw & 7)] =
                                        (unsigned short)j;
                                kw++;
                            } else {
                                if (k < CONF_CAP) {
                                    push((unsigned int)j);
                                    if ((k & 7) == 7) nbr[(size_t)(k >> 3) * nmax + i] = make_uint4(w0, w1, w2, w3);
                                }
                                k++;
                            }
                        };
                        // two consecutive candidates side by side on packed
                        // FP32 pairs, accepted in order
                        int j = start[row + ra[r]];
                        for (; j + 1 < t1; j += 2) {
                            const float4 v0 = pos4[j], v1 = pos4[j + 1];
                            const float2 ddx = __fadd2_rn(ux2, make_float2(-v0.x, -v1.x));
                            const float2 dx = __ffma2_rn(neg2(rint2(ddx, f2(iLx))), f2(Lx), ddx);
                            const float2 dy = __fadd2_rn(uy2, make_float2(-v0.y, -v1.y));
                            const float2 ddz = __fadd2_rn(uz2, make_float2(-v0.z, -v1.z));
                            const float2 dz = __ffma2_rn(neg2(rint2(ddz, f2(iLz))), f2(Lz), ddz);
                            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                            accept(j, r2.x, wall_i && v0.w != 0.f);
                            accept(j + 1, r2.y, wall_i && v1.w != 0.f);
                        }
                        if (j < t1) {
                            const float4 v = pos4[j];
                            const float dx = pbc_f(u.x - v.x, Lx, iLx);
                            const float dy = u.y - v.y;
                            const float dz = pbc_f(u.z - v.z, Lz, iLz);
                            accept(j, __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))), wall_i && v.w != 0.f);
                        }
                    }
                }
            }
            const int gf = (k + 7) >> 3, gw = (kw + 7) >> 3;   // groups used
            if (gf + gw > CONF_GROUPS) {   // the two ends met: overflow
                m->flag_ovf = 1;
                ncnt[i] = 0;
                continue;
            }
            if (k & 7) {   // pad the last groups with the ghost
                for (int q = k & 7; q < 8; q++) push((unsigned int)nmax);
                nbr[(size_t)(k >> 3) * nmax + i] = make_uint4(w0, w1, w2, w3);
            }
            for (int q = kw; q < gw * 8; q++)
                nbr16[((size_t)(CONF_GROUPS - 1 - (q >> 3)) * nmax + i) * 8 + (q & 7)] = (unsigned short)nmax;
            ncnt[i] = gf | (gw << 16);
        }
    };

    // ---- pair and tether forces; x force of the fluid on each wall ----
    unsigned int npairs = 0;
    auto forces = [&](float &swb, float &swt) {
        swb = swt = 0.f;
        const float Lx = cf->Lf[0], iLx = cf->invLf[0], Lz = cf->Lf[2], iLz = cf->invLf[2];
        const float m24cwf = -24.f * (float)b.c_wf, m24cww = -24.f * (float)b.c_ww, kt = (float)b.k;
        const df disp = cf->disp;
        for (int i = tid; i < N; i += T) {
            const float4 u = pos4[i];
            const int ti = (int)u.w;
            const int kgf = ncnt[i] & 0xffff, kgw = ncnt[i] >> 16;
            // -24 c_ij for a fluid neighbour (c_fj) and a wall neighbour
            // (c_wj); a wall atom meets walls only in its last groups
            const float m24c_fj = ti == 0 ? -24.f * (float)b.c_ff : m24cwf;
            float m24c_wj = m24cwf;
            float fx = 0.f, fy = 0.f, fz = 0.f;
            // the two entries of a word side by side on packed FP32 pairs
            // (the scalar pair's operations lane by lane; the sums in list
            // order, entry 0 then entry 1)
            const float2 ux2 = f2(u.x), uy2 = f2(u.y), uz2 = f2(u.z);
            auto pair2 = [&](unsigned int w) {
                const float4 v0 = pos4[w & 0xffffu], v1 = pos4[w >> 16];
                const float2 ddx = __fadd2_rn(ux2, make_float2(-v0.x, -v1.x));
                const float2 dx = __ffma2_rn(neg2(rint2(ddx, f2(iLx))), f2(Lx), ddx);
                const float2 dy = __fadd2_rn(uy2, make_float2(-v0.y, -v1.y));
                const float2 ddz = __fadd2_rn(uz2, make_float2(-v0.z, -v1.z));
                const float2 dz = __ffma2_rn(neg2(rint2(ddz, f2(iLz))), f2(Lz), ddz);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const bool in0 = r2.x < rc2, in1 = r2.y < rc2;
                const float2 m24c = make_float2(v0.w == 0.f ? m24c_fj : m24c_wj, v1.w == 0.f ? m24c_fj : m24c_wj);
                const float2 sv = make_float2(rcp_approx(r2.x), rcp_approx(r2.y));
                const float2 s3 = __fmul2_rn(__fmul2_rn(sv, sv), sv);
                float2 f = __fmul2_rn(__fmul2_rn(s3, sv), __ffma2_rn(f2(48.f), s3, m24c));
                f.x = in0 ? f.x : 0.f;
                f.y = in1 ? f.y : 0.f;
                fx = __fmaf_rn(f.x, dx.x, fx); fy = __fmaf_rn(f.x, dy.x, fy); fz = __fmaf_rn(f.x, dz.x, fz);
                fx = __fmaf_rn(f.y, dx.y, fx); fy = __fmaf_rn(f.y, dy.y, fy); fz = __fmaf_rn(f.y, dz.y, fz);
                npairs += (in0 ? 1u : 0u) + (in1 ? 1u : 0u);
            };
            auto group = [&](int t) {
                const uint4 q = nbr[(size_t)t * nmax + i];
                pair2(q.x); pair2(q.y); pair2(q.z); pair2(q.w);
            };
            for (int t = 0; t < kgf; t++) group(t);
            if (ti != 0) {
                // so far the fluid's force on this wall atom
                if (ti == 2) swt += fx; else swb += fx;
                m24c_wj = m24cww;
                for (int t = CONF_GROUPS - kgw; t < CONF_GROUPS; t++) group(t);
                // tether to the site x_l(t) = x_l(0) + s_w v t
                const float4 lh = lath[i], ll = latl[i], xo = plo[i];
                const df xl = df_add({lh.x, ll.x}, ti == 2 ? disp : df_neg(disp));
                const float tx = pbc_df(df_add({u.x, xo.x}, df_neg(xl)), cf->Ldf[0], iLx);
                const float ty = (u.y - lh.y) + (xo.y - ll.y);
                const float tz = pbc_df(df_add({u.z, xo.z}, df{-lh.z, -ll.z}), cf->Ldf[2], iLz);
                fx = __fmaf_rn(-kt, tx, fx);
                fy = __fmaf_rn(-kt, ty, fy);
                fz = __fmaf_rn(-kt, tz, fz);
            }
            F4[i] = make_float4(fx, fy, fz, 0.f);
        }
    };

    // lane 0: alpha half step of the next step, its momentum factor and the
    // lattice displacement at the end of the next step
    auto next_step = [&]() {
        m->a_cur = m->a_end + m->hhQ * (m->K2_end - b.gT);
        const double e3 = expm1_small(-m->a_cur * hh);
        const double ec = fma(m->e1, e3, m->e1 + e3);   // (1+e1)(1+e3) - 1
        m->e1 = e3;
        m->f1sq = (1.0 + e3) * (1.0 + e3);
        cf->e = df_from_double(ec);
        m->disp += m->vh;
        cf->disp = df_from_double(m->disp);
    };

    // ---- t = 0: lists, forces, wall kinetic sum ----
    build_list();
    if (tid == 0) m->n_rebuild++;
    __syncthreads();
    {
        float swb, swt;
        forces(swb, swt);
        float k2 = 0.f;
        for (int i = tid; i < N; i += T)
            if ((int)pos4[i].w != 0) { const float4 p = phi[i]; k2 += p.x * p.x + p.y * p.y + p.z * p.z; }
        double sums[3];
        conf_sum3(k2, swb, swt, m, sums);
        if (tid == 0) {
            m->K2_end = sums[0];
            if (m->flag_ovf) cf->stop |= TTCF_D_NBR_OVERFLOW;
            if (m->flag_lost) cf->stop |= TTCF_D_ESCAPED;
            if (!isfinite(sums[0] + sums[1] + sums[2])) cf->stop |= TTCF_D_NONFINITE;
            next_step();
        }
    }
    __syncthreads();

    const double iA = 1.0 / b.A;
    const double Ly = b.L[1];
    double *Bo = b.B + (size_t)dl * b.n_obs * b.S;
    for (int s = 1; s <= a.n_steps; s++) {
        if (cf->stop) break;
        const df e = cf->e, hS = cf->h, hhS = cf->hh;
        const float fast2 = cf->fast2;
        float t1 = 0.f, t2 = 0.f;   // two largest squared displacements since the build
        // phase A: wall factor (end of the previous step and start of this
        // one), half kick, drift
        for (int i = tid; i < N; i += T) {
            const float4 u = pos4[i];
            const float4 ph = phi[i], pl = pml[i], fo = F4[i], xo = plo[i];
            df px = {ph.x, pl.x}, py = {ph.y, pl.y}, pz = {ph.z, pl.z};
            if ((int)u.w != 0) { acc_add(px, px.hi * e.hi); acc_add(py, py.hi * e.hi); acc_add(pz, pz.hi * e.hi); }
            acc_add(px, mul_cf(hhS, fo.x)); acc_add(py, mul_cf(hhS, fo.y)); acc_add(pz, mul_cf(hhS, fo.z));
            renorm(px); renorm(py); renorm(pz);
            df x = {u.x, xo.x}, y = {u.y, xo.y}, z = {u.z, xo.z};
            const float ddx = mul_cd(hS, px), ddy = mul_cd(hS, py), ddz = mul_cd(hS, pz);
            acc_add(x, ddx); acc_add(y, ddy); acc_add(z, ddz);
            renorm(x); renorm(y); renorm(z);
            if (!(ddx * ddx + ddy * ddy + ddz * ddz <= fast2)) m->flag_fast = 1;
            pos4[i] = make_float4(x.hi, y.hi, z.hi, u.w);
            plo[i] = make_float4(x.lo, y.lo, z.lo, xo.w);   // w: original index
            phi[i] = make_float4(px.hi, py.hi, pz.hi, 0.f);
            pml[i] = make_float4(px.lo, py.lo, pz.lo, 0.f);
            const float4 r = ref[i];
            const float ex = pbc_f(x.hi - r.x, cf->Lf[0], cf->invLf[0]), ey = y.hi - r.y,
                        ez = pbc_f(z.hi - r.z, cf->Lf[2], cf->invLf[2]);
            const float e2 = ex * ex + ey * ey + ez * ez;
            t2 = fmaxf(t2, fminf(t1, e2));   // (a NaN position stops the daughter
            t1 = fmaxf(t1, e2);              //  through the step's sums)
        }
        {
            for (int o = 16; o > 0; o >>= 1) {
                const float a1 = __shfl_down_sync(0xffffffffu, t1, o), a2 = __shfl_down_sync(0xffffffffu, t2, o);
                const float n2 = fmaxf(fminf(t1, a1), fmaxf(t2, a2));
                t1 = fmaxf(t1, a1);
                t2 = n2;
            }
            if ((tid & 31) == 0) m->dtop[tid >> 5] = make_float2(t1, t2);
        }
        __syncthreads();                                        // barrier 1
        if (m->flag_fast) break;
        // Rebuild when two atoms may together have closed the skin: the
        // largest plus the second largest displacement since the build.
        bool rebuild;
        {
            float m1 = 0.f, m2 = 0.f;
            for (int w = 0; w < (T >> 5); w++) {
                const float2 q = m->dtop[w];
                m2 = fmaxf(fmaxf(m2, q.y), fminf(m1, q.x));
                m1 = fmaxf(m1, q.x);
            }
            rebuild = !(sqrtf(m1) + sqrtf(m2) <= cf->skin_eff);
        }
        if (rebuild) {
            build_list();
            if (tid == 0) m->n_rebuild++;
            __syncthreads();
        }
        float swb, swt;
        forces(swb, swt);
        // phase C: half kick, wall kinetic sum, slab profile at samples
        const bool sample = (s % a.sample_every) == 0;
        float k2 = 0.f;
        for (int i = tid; i < N; i += T) {
            const float4 u = pos4[i];
            const float4 ph = phi[i], pl = pml[i], fo = F4[i];
            df px = {ph.x, pl.x}, py = {ph.y, pl.y}, pz = {ph.z, pl.z};
            acc_add(px, mul_cf(hhS, fo.x)); acc_add(py, mul_cf(hhS, fo.y)); acc_add(pz, mul_cf(hhS, fo.z));
            renorm(px); renorm(py); renorm(pz);
            phi[i] = make_float4(px.hi, py.hi, pz.hi, 0.f);
            pml[i] = make_float4(px.lo, py.lo, pz.lo, 0.f);
            if ((int)u.w != 0) {
                k2 += px.hi * px.hi + py.hi * py.hi + pz.hi * pz.hi;
                if (sample && lath[i].w != 0.f) {
                    const long long q = __float2ll_rn(px.hi * FIX_SCALE) + __float2ll_rn(px.lo * FIX_SCALE);
                    atomicAdd(&m->wall_px[(int)u.w - 1], (unsigned long long)q);
                }
            } else if (sample) {
                const int k = slab_of((double)u.y + (double)plo[i].y, Ly);
                const long long q = __float2ll_rn(px.hi * FIX_SCALE) + __float2ll_rn(px.lo * FIX_SCALE);
                atomicAdd(&m->slab_px[k], (unsigned long long)q);
                atomicAdd(&m->slab_n[k], 1);
            }
        }
        double sums[3];
        conf_sum3(k2, swb, swt, m, sums);                       // barrier 2
        const bool snap_now = a.snap && s >= a.snap_first && (s - a.snap_first) % a.snap_every == 0 &&
                              (s - a.snap_first) / a.snap_every < a.n_snap;
        if (tid == 0) {
            m->K2_end = m->f1sq * sums[0];
            m->a_end = m->a_cur + m->hhQ * (m->K2_end - b.gT);
            if (!isfinite(sums[0] + sums[1] + sums[2])) cf->stop |= TTCF_D_NONFINITE;
            if (m->flag_ovf) cf->stop |= TTCF_D_NBR_OVERFLOW;
            if (m->flag_lost) cf->stop |= TTCF_D_ESCAPED;
            if (sample) {
                const int si = s / a.sample_every;
                Bo[si] = sums[1] * iA;
                Bo[(size_t)b.S + si] = sums[2] * iA;
                for (int k = 0; k < CONF_NSLAB; k++) {
                    Bo[(size_t)(2 + k) * b.S + si] = (double)(long long)m->slab_px[k] * FIX_INV;
                    Bo[(size_t)(2 + CONF_NSLAB + k) * b.S + si] = (double)m->slab_n[k];
                    m->slab_px[k] = 0ull;
                    m->slab_n[k] = 0;
                }
                // wall momenta still owe this step's closing thermostat
                // factor 1 + e1 (applied in the next step's phase A)
                for (int w = 0; w < 2; w++) {
                    Bo[(size_t)(2 + 2 * CONF_NSLAB + w) * b.S + si] =
                        (double)(long long)m->wall_px[w] * FIX_INV * (1.0 + m->e1);
                    m->wall_px[w] = 0ull;
                }
            }
            if (a.abort_flag && (s & 63) == 0 && *a.abort_flag) cf->stop |= TTCF_D_ABORTED;
            m->snap_f = 1.0 + m->e1;   // wall factor still owed to this step's momenta
            if (snap_now) a.snap_alpha[(size_t)dl * a.n_snap + (s - a.snap_first) / a.snap_every] = m->a_end;
            next_step();
        }
        __syncthreads();                                        // barrier 3
        if (snap_now) {
            // mother mode: the phase point in double, x and z wrapped
            double *o = a.snap + ((size_t)dl * a.n_snap + (s - a.snap_first) / a.snap_every) * 6 * N;
            const double f = m->snap_f;
            for (int i = tid; i < N; i += T) {
                const float4 u = pos4[i], xo = plo[i], ph = phi[i], pl = pml[i];
                double x = (double)u.x + (double)xo.x;
                const double y = (double)u.y + (double)xo.y;
                double z = (double)u.z + (double)xo.z;
                x -= b.L[0] * floor((x + 0.5 * b.L[0]) / b.L[0]);
                z -= b.L[2] * floor((z + 0.5 * b.L[2]) / b.L[2]);
                const double w = (int)u.w != 0 ? f : 1.0;
                const int id = __float_as_int(xo.w);   // original index of the slot
                o[id] = x; o[(size_t)N + id] = y; o[2 * (size_t)N + id] = z;
                o[3 * (size_t)N + id] = w * ((double)ph.x + (double)pl.x);
                o[4 * (size_t)N + id] = w * ((double)ph.y + (double)pl.y);
                o[5 * (size_t)N + id] = w * ((double)ph.z + (double)pl.z);
            }
        }
    }
    {
        unsigned long long np = npairs;
        for (int o = 16; o > 0; o >>= 1) np += __shfl_down_sync(0xffffffffu, np, o);
        if ((tid & 31) == 0 && np) atomicAdd(&b.pairs[dl], np);
    }
    if (tid == 0) {
        int st = cf->stop;
        if (m->flag_fast) st |= TTCF_D_FAST_ATOM;
        if (m->flag_ovf) st |= TTCF_D_NBR_OVERFLOW;
        if (m->flag_lost) st |= TTCF_D_ESCAPED;
        b.status[dl] |= st;
        b.rebuilds[dl] += m->n_rebuild;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(CONF_THREADS, 1) conf_kernel(ConfRunArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int w = s_item;
        __syncthreads();
        if (w >= a.n_work) break;
        conf_daughter(a, a.work[w], smem);
    }
}

// ------------------------------------------------------------- spawn --
// One CTA per mother.  In IEEE double: Omega of the unmapped state at the
// group's rate, the x force of the fluid on each wall, the slab sums of
// fluid p_x and counts (exact fixed point); then B(0) and Omega(0) of each
// mapped daughter by the sign rules of the mappings, and the mother as
// float-pair slots.
__global__ void __launch_bounds__(512) conf_spawn_kernel(ConfSpawnArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = blockIdx.x, tid = threadIdx.x, T = blockDim.x, N = a.N;
    const double *src = a.src + (size_t)g * 6 * N;
    unsigned char *sp = smem;
    double *red = reinterpret_cast<double *>(sp); sp += 32 * 4 * sizeof(double);
    unsigned long long *spx = reinterpret_cast<unsigned long long *>(sp); sp += (CONF_NSLAB + 2) * 8;
    int *sn = reinterpret_cast<int *>(sp); sp += CONF_NSLAB * 4;
    int *warp_tmp = reinterpret_cast<int *>(sp); sp += 32 * 4;
    int *cnt = reinterpret_cast<int *>(sp); sp += (size_t)a.ncell * 4;
    int *start = reinterpret_cast<int *>(sp); sp += (size_t)(a.ncell + 2) * 4;
    unsigned short *catom = reinterpret_cast<unsigned short *>(sp);

    // float-pair slots of the mother
    {
        float2 *dst = reinterpret_cast<float2 *>(a.mothers + (size_t)g * 6 * N);
        for (int q = tid; q < 6 * N; q += T) {
            const double v = src[q];
            const float hi = __double2float_rn(v);
            dst[q] = make_float2(hi, __double2float_rn(v - (double)hi));
        }
    }
    const double iLx = 1.0 / a.L[0], iLz = 1.0 / a.L[2];
    auto cell3 = [&](int i, int &cx, int &cy, int &cz) {
        const double x = src[i] - a.L[0] * floor(src[i] * iLx + 0.5);
        const double y = src[(size_t)N + i];
        const double z = src[2 * (size_t)N + i] - a.L[2] * floor(src[2 * (size_t)N + i] * iLz + 0.5);
        cx = min(max((int)floor((x + 0.5 * a.L[0]) * a.nc[0] * iLx), 0), a.nc[0] - 1);
        cy = min(max((int)floor((y + 0.5 * a.L[1]) * a.nc[1] / a.L[1]), 0), a.nc[1] - 1);
        cz = min(max((int)floor((z + 0.5 * a.L[2]) * a.nc[2] * iLz), 0), a.nc[2] - 1);
    };
    auto cellid = [&](int i) {
        int cx, cy, cz;
        cell3(i, cx, cy, cz);
        return (cz * a.nc[1] + cy) * a.nc[0] + cx;
    };
    for (int c = tid; c < a.ncell; c += T) cnt[c] = 0;
    for (int k = tid; k < CONF_NSLAB; k += T) { spx[k] = 0ull; sn[k] = 0; }
    if (tid < 2) spx[CONF_NSLAB + tid] = 0ull;   // inner wall layers
    __syncthreads();
    for (int i = tid; i < N; i += T) atomicAdd(&cnt[cellid(i)], 1);
    __syncthreads();
    cta_exclusive_scan(cnt, start, a.ncell, warp_tmp);
    __syncthreads();
    for (int c = tid; c < a.ncell; c += T) cnt[c] = start[c];
    __syncthreads();
    for (int i = tid; i < N; i += T) catom[atomicAdd(&cnt[cellid(i)], 1)] = (unsigned short)i;
    __syncthreads();
    for (int c = tid; c < a.ncell; c += T)   // fixed order inside each cell
        for (int u = start[c] + 1; u < start[c + 1]; u++) {
            const unsigned short v = catom[u];
            int w = u;
            while (w > start[c] && catom[w - 1] > v) { catom[w] = catom[w - 1]; w--; }
            catom[w] = v;
        }
    __syncthreads();

    // partial sums: [0] -sum_w k (x_w - x_l) s_w, [1] / [2] fluid x force on
    // the bottom / top wall
    double acc[3] = {0.0, 0.0, 0.0};
    const double rc2 = a.rc * a.rc;
    for (int i = tid; i < N; i += T) {
        const int ti = a.types[i];
        if (ti == 0) {
            const int k = slab_of(src[(size_t)N + i], a.L[1]);
            atomicAdd(&spx[k], (unsigned long long)llrint(src[3 * (size_t)N + i] * 1099511627776.0));
            atomicAdd(&sn[k], 1);
            continue;
        }
        const double xi = src[i], yi = src[(size_t)N + i], zi = src[2 * (size_t)N + i];
        {
            const double ys = a.lattice[(size_t)N + i];
            if ((ti == 1 && ys >= a.inner_y[0]) || (ti == 2 && ys <= a.inner_y[1]))
                atomicAdd(&spx[CONF_NSLAB + ti - 1],
                          (unsigned long long)llrint(src[3 * (size_t)N + i] * 1099511627776.0));
        }
        double tx = xi - a.lattice[i];
        tx -= a.L[0] * rint(tx * iLx);
        acc[0] -= a.k * tx * (ti == 2 ? 1.0 : -1.0);
        int cx, cy, cz;
        cell3(i, cx, cy, cz);
        double fsum = 0.0;
        for (int oz = -1; oz <= 1; oz++) {
            const int zz = (cz + oz + a.nc[2]) % a.nc[2];
            for (int oy = -1; oy <= 1; oy++) {
                const int yy = cy + oy;
                if (yy < 0 || yy >= a.nc[1]) continue;
                for (int ox = -1; ox <= 1; ox++) {
                    const int xx = (cx + ox + a.nc[0]) % a.nc[0];
                    const int c = (zz * a.nc[1] + yy) * a.nc[0] + xx;
                    for (int t = start[c]; t < start[c + 1]; t++) {
                        const int j = catom[t];
                        if (a.types[j] != 0) continue;
                        double dx = xi - src[j];
                        const double dy = yi - src[(size_t)N + j];
                        double dz = zi - src[2 * (size_t)N + j];
                        dx -= a.L[0] * rint(dx * iLx);
                        dz -= a.L[2] * rint(dz * iLz);
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < rc2) {
                            const double s = 1.0 / r2, s3 = s * s * s;
                            fsum += s3 * s * (48.0 * s3 - 24.0 * a.c_wf) * dx;
                        }
                    }
                }
            }
        }
        acc[ti == 2 ? 2 : 1] += fsum;
    }
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    for (int k = 0; k < 3; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * 4 + k] = v;
    }
    __syncthreads();
    if (tid == 0) {
        double tot[3] = {0.0, 0.0, 0.0};
        for (int w = 0; w < nw; w++)
            for (int k = 0; k < 3; k++) tot[k] += red[w * 4 + k];
        const double om = tot[0] * a.gamma[g] * a.half_h / a.Tw;
        for (int q = 0; q < a.M; q++) {
            const int mm = a.maps[q];
            const double sx = (mm == 2 || mm == 3) ? -1.0 : 1.0;    // x -> -x
            const double sp_ = (mm == 1 || mm == 2) ? -1.0 : 1.0;   // p_x -> -p_x
            const size_t d = (size_t)g * a.M + q;
            a.Omega[d] = sx * om;
            double *Bo = a.B + d * a.n_obs * a.S;
            Bo[0] = sx * tot[1] / a.A;
            Bo[(size_t)a.S] = sx * tot[2] / a.A;
            for (int k = 0; k < CONF_NSLAB; k++) {
                Bo[(size_t)(2 + k) * a.S] = sp_ * ((double)(long long)spx[k] * FIX_INV);
                Bo[(size_t)(2 + CONF_NSLAB + k) * a.S] = (double)sn[k];
            }
        }
    }
    // the inner wall layers' p_x sums, one thread per mapped daughter
    // (p_x odd under mappings 1 and 2)
    if (tid < a.M) {
        const int mm = a.maps[tid];
        const double sp_ = (mm == 1 || mm == 2) ? -1.0 : 1.0;
        double *Bo = a.B + ((size_t)g * a.M + tid) * a.n_obs * a.S;
        for (int w = 0; w < 2; w++)
            Bo[(size_t)(2 + 2 * CONF_NSLAB + w) * a.S] = sp_ * ((double)(long long)spx[CONF_NSLAB + w] * FIX_INV);
    }
}

}  // namespace

size_t conf_smem_bytes(int nmax, int ncellmax) { return conf_layout(nmax, ncellmax).total; }

size_t conf_spawn_smem_bytes(int N, int ncell) {
    return 32 * 4 * sizeof(double) + CONF_NSLAB * 12 + 16 + 32 * 4 + (size_t)ncell * 4 + (size_t)(ncell + 2) * 4 +
           (size_t)N * 2 + 16;
}

cudaError_t launch_confined(const ConfRunArgs &a, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(conf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conf_kernel<<<grid, CONF_THREADS, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_conf_spawn(const ConfSpawnArgs &a, cudaStream_t st) {
    const size_t smem = conf_spawn_smem_bytes(a.N, a.ncell);
    cudaError_t e = cudaFuncSetAttribute(conf_spawn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    conf_spawn_kernel<<<a.G, 512, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ttcf
