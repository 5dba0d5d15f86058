/*
 * ttcf_oracle.c -- plain FP64 CPU oracle of the TTCF daughter ensemble.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only users of this library.  It
 * shares no code, header or constant table with the CUDA path, and the CUDA
 * path never calls it.
 *
 * Everything is IEEE double precision, written for readability, not speed.
 * What each part follows (arXiv:2312.02990):
 *   - WCA pair potential, shifted so that phi(r_c) = 0 ............ Eq. 6
 *   - thermostatted SLLOD equations of motion, one Nose-Hoover
 *     multiplier alpha, g = 3N degrees of freedom ................. Eq. 5
 *   - Lees-Edwards sliding-brick images, equivalent to the deforming
 *     box of Example 1 ("fix deform")
 *   - shear pressure P_xy and dissipation function
 *     Omega = -gamma V P_xy / (k_B T) ................... Eq. 7 with Eq. 5
 *     (the sign follows from Omega = beta dH^ad/dt, Mathematical
 *      Framework, with the standard pressure tensor; Eq. 7 as printed
 *      reads P_xy as a stress)
 *   - the four phase-space mappings .................................. Eq. 3
 *   - mother sampling and daughter runs .......... Algorithm 2, Figure 1
 *   - responses B(s) and dissipation Omega(0) per daughter ..... Eq. 1-2
 *   - the same dynamics under planar elongational flow, the other
 *     homogeneous field the introduction lists beside shear (end of file)
 *
 * The time discretisation is not stated in the paper beyond "velocity
 * Verlet".  The oracle uses the symmetric splitting (Strang) of the Eq. 5
 * vector field into five exactly solvable flows, each with its own closed
 * form:
 *     E: alpha' = (sum p^2/m - g T)/Q          (p frozen)
 *     D: p' = -alpha p                          (alpha frozen)
 *     C: px' = -gamma py                        (SLLOD coupling alone)
 *     B: p' = F(r)                              (kick)
 *     A: r' = p/m + x_hat gamma y               (drift with streaming)
 * one step = E D C B A B C D E with half steps everywhere except A.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

/* ------------------------------------------------------------------ */
/* Parameters of one bulk system (reduced units, m = sigma = eps = 1). */
/* ------------------------------------------------------------------ */
typedef struct {
    int    n;        /* number of atoms                              */
    int    use_cells;/* 1: linked-cell search, 0: explicit images    */
    double L[3];     /* box edges Lx, Ly, Lz                         */
    double dt;       /* time step h                                  */
    double T;        /* thermostat temperature k_B T                 */
    double Q;        /* Nose-Hoover mass                             */
    double g;        /* thermostat degrees of freedom (3N, Eq. 5)    */
    double rc;       /* pair cutoff; WCA: 2^(1/6)                    */
} orc_bulk;

/* ------------------------------------------------------------------ */
/* Eq. 6: WCA potential phi(r) = 4[r^-12 - r^-6] + 1 for r <= 2^(1/6). */
/* Returns phi and writes f/r = -(1/r) dphi/dr = 48 r^-14 - 24 r^-8.   */
/* ------------------------------------------------------------------ */
double orc_wca(double r2, double *f_over_r)
{
    const double rc2 = pow(2.0, 1.0 / 3.0);
    if (r2 >= rc2) { *f_over_r = 0.0; return 0.0; }
    double ir2 = 1.0 / r2;
    double ir6 = ir2 * ir2 * ir2;
    double ir12 = ir6 * ir6;
    *f_over_r = (48.0 * ir12 - 24.0 * ir6) * ir2;
    return 4.0 * (ir12 - ir6) + 1.0;
}

/* Lees-Edwards minimum image: choose the y image first (it carries the  */
/* x offset delta of the sliding brick), then x, then z.  rint() rounds  */
/* half to even.                                                          */
static void min_image(const double L[3], double delta,
                      double *dx, double *dy, double *dz)
{
    double ny = rint(*dy / L[1]);
    *dy -= ny * L[1];
    *dx -= ny * delta;
    *dx -= rint(*dx / L[0]) * L[0];
    *dz -= rint(*dz / L[2]) * L[2];
}

/* Accumulate one pair (i gets force f/r * d).  W is sum over ordered    */
/* pairs of 0.5 d_a d_b f/r, i.e. the virial sum over unordered pairs.   */
static void add_pair(double dx, double dy, double dz, double for_,
                     double phi, double *fx, double *fy, double *fz,
                     double W[6], double *U)
{
    *fx += for_ * dx; *fy += for_ * dy; *fz += for_ * dz;
    W[0] += 0.5 * for_ * dx * dx;
    W[1] += 0.5 * for_ * dy * dy;
    W[2] += 0.5 * for_ * dz * dz;
    W[3] += 0.5 * for_ * dx * dy;
    W[4] += 0.5 * for_ * dx * dz;
    W[5] += 0.5 * for_ * dy * dz;
    *U += 0.5 * phi;
}

/* Brute force: every ordered pair, every one of the 27 images           */
/* (nx, ny, nz) in {-1,0,1}^3, image of j at                             */
/*   (x_j + nx Lx + ny delta, y_j + ny Ly, z_j + nz Lz).                 */
/* Valid when L > 2 r_c and |delta| <= Lx/2 (at most one image of j lies */
/* within r_c of i).                                                      */
int orc_forces_brute(const orc_bulk *b, double delta, const double *x,
                     const double *y, const double *z, double *fx,
                     double *fy, double *fz, double W[6], double *U)
{
    int n = b->n;
    double rc2 = b->rc * b->rc;
    memset(W, 0, 6 * sizeof(double));
    *U = 0.0;
    for (int i = 0; i < n; i++) {
        double ax = 0, ay = 0, az = 0;
        for (int j = 0; j < n; j++) {
            if (j == i) continue;
            for (int ny = -1; ny <= 1; ny++)
            for (int nx = -1; nx <= 1; nx++)
            for (int nz = -1; nz <= 1; nz++) {
                double dx = x[i] - (x[j] + nx * b->L[0] + ny * delta);
                double dy = y[i] - (y[j] + ny * b->L[1]);
                double dz = z[i] - (z[j] + nz * b->L[2]);
                double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < rc2) {
                    double for_;
                    double phi = orc_wca(r2, &for_);
                    add_pair(dx, dy, dz, for_, phi, &ax, &ay, &az, W, U);
                }
            }
        }
        fx[i] = ax; fy[i] = ay; fz[i] = az;
    }
    return 0;
}

static int wrapi(int c, int n) { return (c % n + n) % n; }

/* Linked-cell search with the Lees-Edwards minimum image.  Cells have    */
/* width >= r_c.  A neighbour row that crosses the y boundary is scanned  */
/* along its whole x extent, because its images are shifted by delta.     */
int orc_forces_cells(const orc_bulk *b, double delta, const double *x,
                     const double *y, const double *z, double *fx,
                     double *fy, double *fz, double W[6], double *U)
{
    int n = b->n, nc[3];
    double w[3], rc2 = b->rc * b->rc;
    for (int d = 0; d < 3; d++) {
        nc[d] = (int)floor(b->L[d] / b->rc);
        if (nc[d] < 3) return orc_forces_brute(b, delta, x, y, z, fx, fy, fz, W, U);
        w[d] = b->L[d] / nc[d];
    }
    int ncell = nc[0] * nc[1] * nc[2];
    int *head = (int *)malloc(sizeof(int) * ncell);
    int *next = (int *)malloc(sizeof(int) * n);
    int *cell = (int *)malloc(sizeof(int) * 3 * n);
    if (!head || !next || !cell) { free(head); free(next); free(cell); return -1; }
    for (int c = 0; c < ncell; c++) head[c] = -1;
    const double *r[3] = {x, y, z};
    for (int i = n - 1; i >= 0; i--) {
        int c3[3];
        for (int d = 0; d < 3; d++) {
            int c = (int)floor((r[d][i] + 0.5 * b->L[d]) / w[d]);
            if (c < 0) c = 0;
            if (c >= nc[d]) c = nc[d] - 1;
            c3[d] = c; cell[3 * i + d] = c;
        }
        int ci = (c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        next[i] = head[ci];
        head[ci] = i;
    }
    memset(W, 0, 6 * sizeof(double));
    *U = 0.0;
    for (int i = 0; i < n; i++) {
        double ax = 0, ay = 0, az = 0;
        int cx = cell[3 * i], cy = cell[3 * i + 1], cz = cell[3 * i + 2];
        for (int oy = -1; oy <= 1; oy++) {
            int yy = cy + oy;
            int crosses = (yy < 0 || yy >= nc[1]);
            yy = wrapi(yy, nc[1]);
            for (int oz = -1; oz <= 1; oz++) {
                int zz = wrapi(cz + oz, nc[2]);
                int x0 = crosses ? 0 : cx - 1;
                int x1 = crosses ? nc[0] - 1 : cx + 1;
                for (int xc = x0; xc <= x1; xc++) {
                    int xx = wrapi(xc, nc[0]);
                    for (int j = head[(zz * nc[1] + yy) * nc[0] + xx]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
                        min_image(b->L, delta, &dx, &dy, &dz);
                        double r2 = dx * dx + dy * dy + dz * dz;
                        if (r2 < rc2) {
                            double for_;
                            double phi = orc_wca(r2, &for_);
                            add_pair(dx, dy, dz, for_, phi, &ax, &ay, &az, W, U);
                        }
                    }
                }
            }
        }
        fx[i] = ax; fy[i] = ay; fz[i] = az;
    }
    free(head); free(next); free(cell);
    return 0;
}

int orc_forces(const orc_bulk *b, double delta, const double *x,
               const double *y, const double *z, double *fx, double *fy,
               double *fz, double W[6], double *U)
{
    if (b->use_cells)
        return orc_forces_cells(b, delta, x, y, z, fx, fy, fz, W, U);
    return orc_forces_brute(b, delta, x, y, z, fx, fy, fz, W, U);
}

/* ------------------------------------------------------------------ */
/* Phase point of one trajectory.                                      */
/* ------------------------------------------------------------------ */
typedef struct {
    double *x, *y, *z, *px, *py, *pz, *fx, *fy, *fz;
    double alpha;   /* Nose-Hoover multiplier                         */
    double xi;      /* integral of alpha dt (extended energy only)    */
    double delta;   /* Lees-Edwards x offset of the image above       */
    double W[6];    /* configurational virial at the current r        */
    double U;       /* potential energy at the current r              */
    double *buf;
} orc_state;

static int state_alloc(orc_state *s, int n)
{
    s->buf = (double *)calloc((size_t)9 * n, sizeof(double));
    if (!s->buf) return -1;
    double *p = s->buf;
    s->x = p; s->y = p + n; s->z = p + 2 * n;
    s->px = p + 3 * n; s->py = p + 4 * n; s->pz = p + 5 * n;
    s->fx = p + 6 * n; s->fy = p + 7 * n; s->fz = p + 8 * n;
    s->alpha = s->xi = s->delta = s->U = 0.0;
    memset(s->W, 0, sizeof(s->W));
    return 0;
}

static void state_free(orc_state *s) { free(s->buf); s->buf = NULL; }

static double kin2(const orc_bulk *b, const orc_state *s)
{
    double k = 0.0;
    for (int i = 0; i < b->n; i++)
        k += s->px[i] * s->px[i] + s->py[i] * s->py[i] + s->pz[i] * s->pz[i];
    return k;   /* sum p^2 / m */
}

static int compute_forces(const orc_bulk *b, orc_state *s)
{
    return orc_forces(b, s->delta, s->x, s->y, s->z, s->fx, s->fy, s->fz, s->W, &s->U);
}

/* Shear pressure P_xy = (1/V)[sum px py / m + sum_{i<j} x_ij F_ij,y].    */
static double pxy(const orc_bulk *b, const orc_state *s)
{
    double k = 0.0;
    for (int i = 0; i < b->n; i++) k += s->px[i] * s->py[i];
    return (k + s->W[3]) / (b->L[0] * b->L[1] * b->L[2]);
}

static void wrap_into_box(double *v, double L)
{
    /* into [-L/2, L/2) */
    *v -= L * floor((*v + 0.5 * L) / L);
    if (*v >= 0.5 * L) *v -= L;   /* guards floor() rounding at the edge */
}

/* Flow E for a time tau (p frozen).                                      */
static void flow_alpha(const orc_bulk *b, orc_state *s, double tau)
{
    s->alpha += tau * (kin2(b, s) - b->g * b->T) / b->Q;
}

/* Flow D for a time tau (alpha frozen): p <- p exp(-alpha tau).          */
static void flow_scale(const orc_bulk *b, orc_state *s, double tau)
{
    double c = exp(-s->alpha * tau);
    s->xi += s->alpha * tau;
    for (int i = 0; i < b->n; i++) { s->px[i] *= c; s->py[i] *= c; s->pz[i] *= c; }
}

/* Flow C for a time tau: px <- px - gamma tau py.                        */
static void flow_shear(const orc_bulk *b, orc_state *s, double gamma, double tau)
{
    for (int i = 0; i < b->n; i++) s->px[i] -= gamma * tau * s->py[i];
}

/* Flow B for a time tau: p <- p + tau F.                                  */
static void flow_kick(const orc_bulk *b, orc_state *s, double tau)
{
    for (int i = 0; i < b->n; i++) {
        s->px[i] += tau * s->fx[i]; s->py[i] += tau * s->fy[i]; s->pz[i] += tau * s->fz[i];
    }
}

/* Flow A for a time h: r' = p + x_hat gamma y with p frozen, then the     */
/* sliding-brick offset advances by gamma Ly h and atoms that left the    */
/* box through y = +-Ly/2 re-enter shifted by -+delta in x.               */
static void flow_drift(const orc_bulk *b, orc_state *s, double gamma, double h)
{
    const double *L = b->L;
    s->delta += gamma * L[1] * h;
    s->delta -= L[0] * rint(s->delta / L[0]);
    for (int i = 0; i < b->n; i++) {
        double y0 = s->y[i];
        s->x[i] += h * s->px[i] + gamma * h * (y0 + 0.5 * h * s->py[i]);
        s->y[i] += h * s->py[i];
        s->z[i] += h * s->pz[i];
        if (s->y[i] >= 0.5 * L[1]) { s->y[i] -= L[1]; s->x[i] -= s->delta; }
        else if (s->y[i] < -0.5 * L[1]) { s->y[i] += L[1]; s->x[i] += s->delta; }
        wrap_into_box(&s->x[i], L[0]);
        wrap_into_box(&s->z[i], L[2]);
    }
}

/* One step E D C B A B C D E of length h.  Forces must be current on     */
/* entry; they are current again on exit.                                  */
static int orc_step(const orc_bulk *b, orc_state *s, double gamma)
{
    double hh = 0.5 * b->dt;
    flow_alpha(b, s, hh);
    flow_scale(b, s, hh);
    flow_shear(b, s, gamma, hh);
    flow_kick(b, s, hh);
    flow_drift(b, s, gamma, b->dt);
    if (compute_forces(b, s)) return -1;
    flow_kick(b, s, hh);
    flow_shear(b, s, gamma, hh);
    flow_scale(b, s, hh);
    flow_alpha(b, s, hh);
    return 0;
}

static void load_state(const orc_bulk *b, orc_state *s, const double *soa)
{
    int n = b->n;
    memcpy(s->x, soa, sizeof(double) * 6 * n);   /* x y z px py pz rows */
}

static void store_state(const orc_bulk *b, const orc_state *s, double *soa)
{
    memcpy(soa, s->x, sizeof(double) * 6 * b->n);
}

/* ------------------------------------------------------------------ */
/* Exported drivers.                                                   */
/* ------------------------------------------------------------------ */

/* Pressure tensor P_ab (xx yy zz xy xz yz), potential energy U and        */
/* sum p^2 of a state [6][n] at Lees-Edwards offset delta.                 */
int orc_pressure(const orc_bulk *b, const double *soa, double delta,
                 double P[6], double *U, double *K2)
{
    orc_state s;
    if (state_alloc(&s, b->n)) return -1;
    load_state(b, &s, soa);
    s.delta = delta;
    if (compute_forces(b, &s)) { state_free(&s); return -1; }
    double V = b->L[0] * b->L[1] * b->L[2];
    double k[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < b->n; i++) {
        k[0] += s.px[i] * s.px[i]; k[1] += s.py[i] * s.py[i]; k[2] += s.pz[i] * s.pz[i];
        k[3] += s.px[i] * s.py[i]; k[4] += s.px[i] * s.pz[i]; k[5] += s.py[i] * s.pz[i];
    }
    for (int a = 0; a < 6; a++) P[a] = (k[a] + s.W[a]) / V;
    *U = s.U;
    *K2 = k[0] + k[1] + k[2];
    state_free(&s);
    return 0;
}

/* Forces of a state [6][n] (rows 0-2 used) into F [3][n], virial W[6], U. */
int orc_state_forces(const orc_bulk *b, const double *soa, double delta,
                     double *F, double W[6], double *U)
{
    int n = b->n;
    return orc_forces(b, delta, soa, soa + n, soa + 2 * n, F, F + n, F + 2 * n, W, U);
}

/* Mappings of a phase point: Eq. 3 and the further choices listed after   */
/* it (each position and momentum component mirrored, x and z exchanged in */
/* a box with Lx = Lz).  Mapping code m, applied in this order:            */
/*   bit 4  exchange of x and z, positions and momenta                     */
/*   bit 1  x-reflection   x -> -x, px -> -px                              */
/*   bit 2  y-reflection   y -> -y, py -> -py                              */
/*   bit 3  z-reflection   z -> -z, pz -> -pz                              */
/*   bit 0  time reversal  p -> -p, and the Nose-Hoover multiplier         */
/*          alpha -> -alpha (set to zero instead when reset_alpha != 0)    */
/* Codes 0..3 are the four mappings of Eq. 3:                              */
/*   m = 0: identity                                                       */
/*   m = 1: (x, y, z, -px, -py, -pz)                                       */
/*   m = 2: (-x, y, z, -px, py, pz)                                        */
/*   m = 3: (-x, y, z, px, -py, -pz)                                       */
/* A reflected coordinate that lands on +L/2 is the periodic point -L/2.   */
void orc_apply_mapping(const orc_bulk *b, int m, const double *in, double alpha_in,
                       int reset_alpha, double *out, double *alpha_out)
{
    int n = b->n;
    for (int e = 0; e < 6 * n; e++) out[e] = in[e];
    if (m & 16) {                                   /* x <-> z */
        for (int i = 0; i < n; i++) {
            double t = out[i]; out[i] = out[2 * n + i]; out[2 * n + i] = t;
            t = out[3 * n + i]; out[3 * n + i] = out[5 * n + i]; out[5 * n + i] = t;
        }
    }
    for (int a = 0; a < 3; a++) {                   /* reflections */
        if (!(m & (2 << a))) continue;
        for (int i = 0; i < n; i++) {
            double c = -out[a * n + i];
            if (c >= 0.5 * b->L[a]) c -= b->L[a];
            out[a * n + i] = c;
            out[(3 + a) * n + i] = -out[(3 + a) * n + i];
        }
    }
    if (m & 1)                                      /* time reversal */
        for (int e = 3 * n; e < 6 * n; e++) out[e] = -out[e];
    double sa = (m & 1) ? -1.0 : 1.0;
    *alpha_out = reset_alpha ? 0.0 : sa * alpha_in;
}

/* Run n_steps steps from state [6][n] (in/out) with alpha, delta (in/out) */
/* and record per step s = 0..n_steps the row                              */
/*   obs[s] = {K2, U, alpha, xi, Pxy, Wxy, delta, H_ext}                   */
/* where H_ext = K2/2 + U + Q alpha^2/2 + g T xi.                           */
int orc_trajectory(const orc_bulk *b, double gamma, double *soa,
                   double *alpha_io, double *delta_io, int n_steps, double *obs)
{
    orc_state s;
    if (state_alloc(&s, b->n)) return -1;
    load_state(b, &s, soa);
    s.alpha = *alpha_io;
    s.delta = *delta_io;
    if (compute_forces(b, &s)) { state_free(&s); return -1; }
    for (int t = 0; t <= n_steps; t++) {
        if (t > 0 && orc_step(b, &s, gamma)) { state_free(&s); return -1; }
        if (obs) {
            double K2 = kin2(b, &s);
            double *o = obs + 8 * t;
            o[0] = K2; o[1] = s.U; o[2] = s.alpha; o[3] = s.xi;
            o[4] = pxy(b, &s); o[5] = s.W[3]; o[6] = s.delta;
            o[7] = 0.5 * K2 + s.U + 0.5 * b->Q * s.alpha * s.alpha + b->g * b->T * s.xi;
        }
    }
    store_state(b, &s, soa);
    *alpha_io = s.alpha;
    *delta_io = s.delta;
    state_free(&s);
    return 0;
}

/* Algorithm 2 (mother part): thermalise n_eq steps at zero field, then    */
/* store a phase point and alpha every `spacing` steps, n_states times.    */
int orc_mother(const orc_bulk *b, const double *init, double alpha0, int n_eq,
               int n_states, int spacing, double *out_states, double *out_alpha)
{
    orc_state s;
    if (state_alloc(&s, b->n)) return -1;
    load_state(b, &s, init);
    s.alpha = alpha0;
    if (compute_forces(b, &s)) { state_free(&s); return -1; }
    for (int t = 0; t < n_eq; t++)
        if (orc_step(b, &s, 0.0)) { state_free(&s); return -1; }
    for (int k = 0; k < n_states; k++) {
        for (int t = 0; t < spacing; t++)
            if (orc_step(b, &s, 0.0)) { state_free(&s); return -1; }
        store_state(b, &s, out_states + (size_t)k * 6 * b->n);
        out_alpha[k] = s.alpha;
    }
    state_free(&s);
    return 0;
}

/* One daughter (Figure 1, Algorithm 2 inner loop): map the mother state,  */
/* switch the field on (delta = 0, peculiar momenta keep the streaming     */
/* profile superimposed), record B(0) = P_xy(0) and                        */
/* Omega(0) = -gamma V P_xy(0) / T, then B(s) = P_xy every sample_every    */
/* steps.  B has n_steps/sample_every + 1 entries.  Optionally returns the */
/* final state [6][n] and alpha.                                           */
int orc_daughter(const orc_bulk *b, const double *mother, double mother_alpha,
                 int m, int reset_alpha, double gamma, int n_steps, int sample_every,
                 double *B, double *Omega, double *final_state, double *final_alpha)
{
    orc_state s;
    if (state_alloc(&s, b->n)) return -1;
    double a0;
    orc_apply_mapping(b, m, mother, mother_alpha, reset_alpha, s.x, &a0);
    s.alpha = a0;
    s.delta = 0.0;
    if (compute_forces(b, &s)) { state_free(&s); return -1; }
    double V = b->L[0] * b->L[1] * b->L[2];
    double p0 = pxy(b, &s);
    *Omega = -gamma * V * p0 / b->T;
    B[0] = p0;
    for (int t = 1; t <= n_steps; t++) {
        if (orc_step(b, &s, gamma)) { state_free(&s); return -1; }
        if (t % sample_every == 0) B[t / sample_every] = pxy(b, &s);
    }
    if (final_state) store_state(b, &s, final_state);
    if (final_alpha) *final_alpha = s.alpha;
    state_free(&s);
    return 0;
}

/* The ensemble: daughters d = g*M + k for mother group g and the k-th set */
/* bit m of mapping_mask (M = number of set bits).  Independent daughters  */
/* run on n_threads OpenMP threads (one daughter per thread at a time).    */
int orc_daughters(const orc_bulk *b, int n_groups, const double *mothers,
                  const double *mother_alpha, const double *gammas,
                  unsigned mapping_mask, int reset_alpha, int n_steps,
                  int sample_every, double *B, double *Omega, int n_threads)
{
    int maps[32], M = 0;
    for (int m = 0; m < 32; m++) if (mapping_mask & (1u << m)) maps[M++] = m;
    if (M == 0 || sample_every <= 0 || n_steps % sample_every) return -2;
    for (int k = 0; k < M; k++)
        if ((maps[k] & 16) && b->L[0] != b->L[2]) return -3;   /* x <-> z needs Lx = Lz */
    int S = n_steps / sample_every + 1;
    int D = n_groups * M;
    int err = 0;
    (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(|:err)
    for (int d = 0; d < D; d++) {
        int g = d / M, m = maps[d % M];
        err |= orc_daughter(b, mothers + (size_t)g * 6 * b->n, mother_alpha[g], m,
                            reset_alpha, gammas[g], n_steps, sample_every,
                            B + (size_t)d * S, Omega + d, NULL, NULL) ? 1 : 0;
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Planar elongational flow (the other homogeneous field the paper's    */
/* introduction lists beside shear).  The streaming velocity is          */
/* u(r) = r . grad u with grad u = diag(eps, 0, -eps): stretching along  */
/* x, compression along z, y neutral, so the volume is constant.  The    */
/* Eq. 5 vector field with this grad u:                                  */
/*     r' = p/m + (eps x, 0, -eps z)                                     */
/*     p' = F - (eps px, 0, -eps pz) - alpha p                           */
/* The periodic box deforms with the flow, Lx(t) = Lx(0) exp(eps t),     */
/* Lz(t) = Lz(0) exp(-eps t) (no Kraynik-Reinelt remapping: a daughter   */
/* is short enough that the compressed edge stays above 2 r_c, which the */
/* callers check).  The dissipation function (Omega = beta dH^ad/dt with  */
/* dH^ad/dt = -V grad u : P) is                                          */
/*     Omega = -eps V (P_xx - P_zz) / (k_B T)                            */
/* and the response B = P_xx - P_zz; the planar elongational viscosity  */
/* is eta_1 = -<P_xx - P_zz> / (4 eps), the shear viscosity in the       */
/* Newtonian limit.  The x <-> z exchange (mapping bit 4) negates Omega  */
/* and time reversal keeps it, so the set {0, 1, 16, 17} cancels          */
/* <Omega(0)> per group, as Eq. 3's set does for shear.                  */
/* Splitting as for shear, with the shear flows replaced by:             */
/*     C': px <- px exp(-eps tau), pz <- pz exp(eps tau)                 */
/*     A': the exact drift with p frozen,                                */
/*         x <- x exp(eps h) + px (exp(eps h) - 1)/eps                   */
/*         z <- z exp(-eps h) + pz (1 - exp(-eps h))/eps                 */
/*         y <- y + py h,                                                 */
/*         then the box edges at the new time and one periodic wrap.    */
/* ------------------------------------------------------------------ */

/* Flow C' for a time tau. */
static void flow_elong(const orc_bulk *b, orc_state *s, double eps, double tau)
{
    double cx = exp(-eps * tau), cz = exp(eps * tau);
    for (int i = 0; i < b->n; i++) { s->px[i] *= cx; s->pz[i] *= cz; }
}

/* One periodic wrap into [-L/2, L/2) (a step moves an atom far less     */
/* than L/2).                                                             */
static double wrap_once(double v, double L)
{
    if (v >= 0.5 * L) return v - L;
    if (v < -0.5 * L) return v + L;
    return v;
}

/* Flow A' for a time h; bt->L holds the box at the start and is set to  */
/* the box at time t_new = (step number) h from the switch-on box L0.     */
static void flow_drift_elong(orc_bulk *bt, orc_state *s, double eps, double h,
                             const double L0[3], double t_new)
{
    double ex = exp(eps * h), ez = exp(-eps * h);
    double phx = eps != 0.0 ? expm1(eps * h) / eps : h;
    double phz = eps != 0.0 ? expm1(-eps * h) / (-eps) : h;
    bt->L[0] = L0[0] * exp(eps * t_new);
    bt->L[1] = L0[1];
    bt->L[2] = L0[2] * exp(-eps * t_new);
    for (int i = 0; i < bt->n; i++) {
        s->x[i] = wrap_once(s->x[i] * ex + s->px[i] * phx, bt->L[0]);
        s->y[i] = wrap_once(s->y[i] + s->py[i] * h, bt->L[1]);
        s->z[i] = wrap_once(s->z[i] * ez + s->pz[i] * phz, bt->L[2]);
    }
}

/* B = P_xx - P_zz of the current state in the current box. */
static double pxx_pzz(const orc_bulk *bt, const orc_state *s)
{
    double k = 0.0;
    for (int i = 0; i < bt->n; i++) k += s->px[i] * s->px[i] - s->pz[i] * s->pz[i];
    return (k + s->W[0] - s->W[2]) / (bt->L[0] * bt->L[1] * bt->L[2]);
}

/* One step E D C' B A' B C' D E taking the box from step n-1 to step n.  */
static int orc_step_elong(orc_bulk *bt, orc_state *s, double eps, const double L0[3], int n)
{
    double hh = 0.5 * bt->dt;
    flow_alpha(bt, s, hh);
    flow_scale(bt, s, hh);
    flow_elong(bt, s, eps, hh);
    flow_kick(bt, s, hh);
    flow_drift_elong(bt, s, eps, bt->dt, L0, n * bt->dt);
    if (compute_forces(bt, s)) return -1;   /* minimum image in the new box */
    flow_kick(bt, s, hh);
    flow_elong(bt, s, eps, hh);
    flow_scale(bt, s, hh);
    flow_alpha(bt, s, hh);
    return 0;
}

/* Run n_steps under elongation rate eps from a state [6][n] (in/out) at  */
/* the switch-on box b->L, recording per step s = 0..n_steps              */
/*   obs[s] = {K2, U, alpha, xi, Pxx - Pzz, Wxx - Wzz, Lx, Lz, H_ext}      */
/* with H_ext = K2/2 + U + Q alpha^2/2 + g T xi, whose rate of change is  */
/* -V eps (P_xx - P_zz).  The final state is in the final box.            */
int orc_trajectory_elong(const orc_bulk *b, double eps, double *soa, double *alpha_io,
                         int n_steps, double *obs)
{
    orc_bulk bt = *b;
    orc_state s;
    if (state_alloc(&s, b->n)) return -1;
    load_state(b, &s, soa);
    s.alpha = *alpha_io;
    if (compute_forces(&bt, &s)) { state_free(&s); return -1; }
    for (int t = 0; t <= n_steps; t++) {
        if (t > 0 && orc_step_elong(&bt, &s, eps, b->L, t)) { state_free(&s); return -1; }
        if (obs) {
            double K2 = kin2(&bt, &s);
            double *o = obs + 9 * t;
            o[0] = K2; o[1] = s.U; o[2] = s.alpha; o[3] = s.xi;
            o[4] = pxx_pzz(&bt, &s); o[5] = s.W[0] - s.W[2];
            o[6] = bt.L[0]; o[7] = bt.L[2];
            o[8] = 0.5 * K2 + s.U + 0.5 * b->Q * s.alpha * s.alpha + b->g * b->T * s.xi;
        }
    }
    store_state(b, &s, soa);
    *alpha_io = s.alpha;
    state_free(&s);
    return 0;
}

/* One daughter under elongation: map the mother (codes as for shear, in  */
/* the switch-on box), B(0) = P_xx - P_zz, Omega(0) = -eps V B(0) / T,    */
/* then B(s) every sample_every steps.                                     */
int orc_daughter_elong(const orc_bulk *b, const double *mother, double mother_alpha,
                       int m, int reset_alpha, double eps, int n_steps, int sample_every,
                       double *B, double *Omega, double *final_state, double *final_alpha)
{
    orc_bulk bt = *b;
    orc_state s;
    if (state_alloc(&s, b->n)) return -1;
    double a0;
    orc_apply_mapping(b, m, mother, mother_alpha, reset_alpha, s.x, &a0);
    s.alpha = a0;
    if (compute_forces(&bt, &s)) { state_free(&s); return -1; }
    double V = b->L[0] * b->L[1] * b->L[2];
    double b0 = pxx_pzz(&bt, &s);
    *Omega = -eps * V * b0 / b->T;
    B[0] = b0;
    for (int t = 1; t <= n_steps; t++) {
        if (orc_step_elong(&bt, &s, eps, b->L, t)) { state_free(&s); return -1; }
        if (t % sample_every == 0) B[t / sample_every] = pxx_pzz(&bt, &s);
    }
    if (final_state) store_state(b, &s, final_state);
    if (final_alpha) *final_alpha = s.alpha;
    state_free(&s);
    return 0;
}

/* The elongational ensemble, laid out as orc_daughters (gammas are the    */
/* elongation rates of the groups).                                        */
int orc_daughters_elong(const orc_bulk *b, int n_groups, const double *mothers,
                        const double *mother_alpha, const double *rates,
                        unsigned mapping_mask, int reset_alpha, int n_steps,
                        int sample_every, double *B, double *Omega, int n_threads)
{
    int maps[32], M = 0;
    for (int m = 0; m < 32; m++) if (mapping_mask & (1u << m)) maps[M++] = m;
    if (M == 0 || sample_every <= 0 || n_steps % sample_every) return -2;
    for (int k = 0; k < M; k++)
        if ((maps[k] & 16) && b->L[0] != b->L[2]) return -3;
    int S = n_steps / sample_every + 1;
    int D = n_groups * M;
    int err = 0;
    (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(|:err)
    for (int d = 0; d < D; d++) {
        int g = d / M, m = maps[d % M];
        err |= orc_daughter_elong(b, mothers + (size_t)g * 6 * b->n, mother_alpha[g], m,
                                  reset_alpha, rates[g], n_steps, sample_every,
                                  B + (size_t)d * S, Omega + d, NULL, NULL) ? 1 : 0;
    }
    return err ? -1 : 0;
}
