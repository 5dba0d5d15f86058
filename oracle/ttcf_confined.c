/*
 * ttcf_confined.c -- FP64 CPU oracle of the confined (Example 2) daughters.
 *
 * TEST INFRASTRUCTURE ONLY (see ttcf_oracle.c).
 *
 * System (arXiv:2312.02990, Example 2):
 *   - pair potential 4[r^-12 - c_ij r^-6] truncated at r_c (Eq. 9) between
 *     every pair of atoms: fluid-fluid c_ff, wall-fluid c_wf (the two values
 *     the paper gives), wall-wall c_ww (not given: plain Lennard-Jones,
 *     c_ww = 1, by default; ww_on = 0 switches wall-wall pairs off so that
 *     only the tethers hold the walls);
 *   - equations of motion as printed in Eq. 10: fluid ṙ = p, ṗ = F; wall
 *     ṙ = p, ṗ = F - k (r - r_l) - alpha p, alpha' = (sum_w p^2 - g T_w)/Q,
 *     lattice sites ṙ_l = (+-v_wall, 0, 0) (bottom -, top +);
 *   - x and z periodic, y bounded by the walls.
 * Dissipation function (Eq. 11 with beta and the sign from Omega = beta
 * dH^ad/dt): Omega = -(1/T_w) sum_w k (x_w - x_l) s_w v_wall.
 * Responses B per sample: the x force exerted by the fluid on the bottom and
 * on the top wall per unit area, then the fluid's sum of p_x and its atom
 * count in each of nslab slabs spanning y in [-Ly/2, Ly/2), then the sum of
 * p_x over the innermost layer of the bottom and of the top wall (the wall
 * layer whose velocity enters the slip velocity of the friction study): the
 * wall's atoms whose tether site lies within 0.1 sigma in y of the wall's
 * site plane nearest the channel (sites slide in x only, so layers stay
 * planar).
 *
 * Discretisation (the paper says "velocity Verlet"): the symmetric splitting
 * E D B A B D E, E = alpha flow, D = wall friction flow, B = kick with all
 * forces (pair + tether), A = drift of atoms and lattice sites.  The fluid
 * alone sees B A B, plain velocity Verlet.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n;            /* atoms                                              */
    int nslab;        /* slabs of the velocity profile                       */
    int use_cells;    /* 1: linked cells, 0: all pairs                       */
    int pad_;
    double L[3];      /* Lx, Ly (slab extent; y is not periodic), Lz          */
    double dt, Tw, Q, g, k, rc;
    double c_ff, c_wf, c_ww;
    double vwall;     /* lattice speed: bottom wall -vwall, top wall +vwall  */
    int ww_on;        /* 1: wall-wall pairs interact with c_ww               */
    int pad2_;
} orc_conf;

static int is_wall(int t) { return t != 0; }
static double wall_sign(int t) { return t == 2 ? 1.0 : (t == 1 ? -1.0 : 0.0); }

static double pbc(double d, double L) { return d - L * rint(d / L); }

/* One pair: force on i from j (i gets f/r * d), LJ energy shared 1/2 each. */
static void cf_pair(const orc_conf *c, int ti, int tj, double dx, double dy, double dz,
                    double *fx, double *fy, double *fz, double *U, double *swx)
{
    if (is_wall(ti) && is_wall(tj) && !c->ww_on) return;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= c->rc * c->rc) return;
    double cij = (ti == 0 && tj == 0) ? c->c_ff : ((ti == 0 || tj == 0) ? c->c_wf : c->c_ww);
    double s = 1.0 / r2, s3 = s * s * s;
    double f = s3 * s * (48.0 * s3 - 24.0 * cij);   /* -(1/r) dphi/dr */
    *fx += f * dx; *fy += f * dy; *fz += f * dz;
    /* energy shifted to zero at r_c (Eq. 9 is truncated; the shift leaves the
       forces unchanged and makes the energy continuous) */
    double rc6 = 1.0 / (c->rc * c->rc * c->rc * c->rc * c->rc * c->rc);
    *U += 0.5 * (4.0 * s3 * (s3 - cij) - 4.0 * rc6 * (rc6 - cij));
    if (is_wall(ti) && tj == 0) *swx += f * dx;
}

/* Pair forces + tether forces.  sw[0], sw[1]: x force of the fluid on the */
/* bottom and top wall.  U[0] = pair energy, U[1] = tether energy.          */
int orc_conf_forces(const orc_conf *c, const int *type, const double *x, const double *y,
                    const double *z, const double *xl, const double *yl, const double *zl,
                    double *fx, double *fy, double *fz, double U[2], double sw[2])
{
    int n = c->n;
    U[0] = U[1] = 0.0;
    sw[0] = sw[1] = 0.0;
    int *head = NULL, *next = NULL, *cell = NULL, nc[3] = {1, 1, 1};
    double w[3] = {c->L[0], c->L[1], c->L[2]};
    double ylo = 0.0, yspan = 0.0;
    if (c->use_cells) {
        ylo = y[0]; double yhi = y[0];
        for (int i = 1; i < n; i++) { if (y[i] < ylo) ylo = y[i]; if (y[i] > yhi) yhi = y[i]; }
        yspan = yhi - ylo + 1e-9;
        nc[0] = (int)floor(c->L[0] / c->rc);
        nc[2] = (int)floor(c->L[2] / c->rc);
        nc[1] = (int)floor(yspan / c->rc);
        if (nc[1] < 1) nc[1] = 1;
        if (nc[0] < 3 || nc[2] < 3) return -2;
        w[0] = c->L[0] / nc[0]; w[1] = yspan / nc[1]; w[2] = c->L[2] / nc[2];
        head = (int *)malloc(sizeof(int) * nc[0] * nc[1] * nc[2]);
        next = (int *)malloc(sizeof(int) * n);
        cell = (int *)malloc(sizeof(int) * 3 * n);
        if (!head || !next || !cell) { free(head); free(next); free(cell); return -1; }
        for (int q = 0; q < nc[0] * nc[1] * nc[2]; q++) head[q] = -1;
        for (int i = n - 1; i >= 0; i--) {
            int cx = (int)floor((x[i] + 0.5 * c->L[0]) / w[0]);
            int cy = (int)floor((y[i] - ylo) / w[1]);
            int cz = (int)floor((z[i] + 0.5 * c->L[2]) / w[2]);
            cx = cx < 0 ? 0 : (cx >= nc[0] ? nc[0] - 1 : cx);
            cy = cy < 0 ? 0 : (cy >= nc[1] ? nc[1] - 1 : cy);
            cz = cz < 0 ? 0 : (cz >= nc[2] ? nc[2] - 1 : cz);
            cell[3 * i] = cx; cell[3 * i + 1] = cy; cell[3 * i + 2] = cz;
            int q = (cz * nc[1] + cy) * nc[0] + cx;
            next[i] = head[q]; head[q] = i;
        }
    }
    for (int i = 0; i < n; i++) {
        double ax = 0, ay = 0, az = 0, swx = 0;
        if (!c->use_cells) {
            for (int j = 0; j < n; j++) {
                if (j == i) continue;
                cf_pair(c, type[i], type[j], pbc(x[i] - x[j], c->L[0]), y[i] - y[j],
                        pbc(z[i] - z[j], c->L[2]), &ax, &ay, &az, &U[0], &swx);
            }
        } else {
            int cx = cell[3 * i], cy = cell[3 * i + 1], cz = cell[3 * i + 2];
            for (int oy = -1; oy <= 1; oy++) {
                int yy = cy + oy;
                if (yy < 0 || yy >= nc[1]) continue;
                for (int oz = -1; oz <= 1; oz++) {
                    int zz = ((cz + oz) % nc[2] + nc[2]) % nc[2];
                    for (int ox = -1; ox <= 1; ox++) {
                        int xx = ((cx + ox) % nc[0] + nc[0]) % nc[0];
                        for (int j = head[(zz * nc[1] + yy) * nc[0] + xx]; j >= 0; j = next[j]) {
                            if (j == i) continue;
                            cf_pair(c, type[i], type[j], pbc(x[i] - x[j], c->L[0]), y[i] - y[j],
                                    pbc(z[i] - z[j], c->L[2]), &ax, &ay, &az, &U[0], &swx);
                        }
                    }
                }
            }
        }
        if (is_wall(type[i])) {   /* tether -k (r_w - r_l) */
            double tx = pbc(x[i] - xl[i], c->L[0]), ty = y[i] - yl[i], tz = pbc(z[i] - zl[i], c->L[2]);
            ax -= c->k * tx; ay -= c->k * ty; az -= c->k * tz;
            U[1] += 0.5 * c->k * (tx * tx + ty * ty + tz * tz);
            sw[type[i] == 2 ? 1 : 0] += swx;
        }
        fx[i] = ax; fy[i] = ay; fz[i] = az;
    }
    free(head); free(next); free(cell);
    return 0;
}

typedef struct {
    double *x, *y, *z, *px, *py, *pz, *fx, *fy, *fz, *xl, *yl, *zl;
    double alpha, xi, U[2], sw[2];
    double *buf;
} conf_state;

static int cs_alloc(conf_state *s, int n)
{
    s->buf = (double *)calloc((size_t)12 * n, sizeof(double));
    if (!s->buf) return -1;
    double *p = s->buf;
    s->x = p; s->y = p + n; s->z = p + 2 * n; s->px = p + 3 * n; s->py = p + 4 * n;
    s->pz = p + 5 * n; s->fx = p + 6 * n; s->fy = p + 7 * n; s->fz = p + 8 * n;
    s->xl = p + 9 * n; s->yl = p + 10 * n; s->zl = p + 11 * n;
    s->alpha = s->xi = 0.0;
    return 0;
}

static int cs_forces(const orc_conf *c, const int *type, conf_state *s)
{
    return orc_conf_forces(c, type, s->x, s->y, s->z, s->xl, s->yl, s->zl, s->fx, s->fy, s->fz,
                           s->U, s->sw);
}

static double wall_k2(const orc_conf *c, const int *type, const conf_state *s)
{
    double k = 0.0;
    for (int i = 0; i < c->n; i++)
        if (is_wall(type[i])) k += s->px[i] * s->px[i] + s->py[i] * s->py[i] + s->pz[i] * s->pz[i];
    return k;
}

/* Rate at which the moving lattice does work on the system:             */
/* dH0/dt = -sum_w k (x_w - x_l) s_w v_wall.                               */
static double lattice_power(const orc_conf *c, const int *type, const conf_state *s)
{
    double P = 0.0;
    for (int i = 0; i < c->n; i++)
        if (is_wall(type[i])) P -= c->k * pbc(s->x[i] - s->xl[i], c->L[0]) * wall_sign(type[i]) * c->vwall;
    return P;
}

static int cs_step(const orc_conf *c, const int *type, conf_state *s)
{
    int n = c->n;
    double h = c->dt, hh = 0.5 * c->dt;
    s->alpha += hh * (wall_k2(c, type, s) - c->g * c->Tw) / c->Q;
    double e = exp(-s->alpha * hh);
    s->xi += s->alpha * hh;
    for (int i = 0; i < n; i++)
        if (is_wall(type[i])) { s->px[i] *= e; s->py[i] *= e; s->pz[i] *= e; }
    for (int i = 0; i < n; i++) { s->px[i] += hh * s->fx[i]; s->py[i] += hh * s->fy[i]; s->pz[i] += hh * s->fz[i]; }
    for (int i = 0; i < n; i++) {
        s->x[i] += h * s->px[i]; s->y[i] += h * s->py[i]; s->z[i] += h * s->pz[i];
        s->x[i] -= c->L[0] * floor((s->x[i] + 0.5 * c->L[0]) / c->L[0]);
        s->z[i] -= c->L[2] * floor((s->z[i] + 0.5 * c->L[2]) / c->L[2]);
        if (is_wall(type[i])) {
            s->xl[i] += wall_sign(type[i]) * c->vwall * h;
            s->xl[i] -= c->L[0] * floor((s->xl[i] + 0.5 * c->L[0]) / c->L[0]);
        }
    }
    if (cs_forces(c, type, s)) return -1;
    for (int i = 0; i < n; i++) { s->px[i] += hh * s->fx[i]; s->py[i] += hh * s->fy[i]; s->pz[i] += hh * s->fz[i]; }
    e = exp(-s->alpha * hh);
    s->xi += s->alpha * hh;
    for (int i = 0; i < n; i++)
        if (is_wall(type[i])) { s->px[i] *= e; s->py[i] *= e; s->pz[i] *= e; }
    s->alpha += hh * (wall_k2(c, type, s) - c->g * c->Tw) / c->Q;
    return 0;
}

static void cs_load(const orc_conf *c, conf_state *s, const double *soa, const double *lat)
{
    memcpy(s->x, soa, sizeof(double) * 6 * c->n);
    memcpy(s->xl, lat, sizeof(double) * 3 * c->n);
}

/* Responses at the current state: sw_bottom/A, sw_top/A, slab sums of     */
/* fluid p_x, slab counts of fluid atoms, inner-layer p_x sums of the       */
/* bottom and top wall (2 + 2 nslab + 2 values).                            */
static void cs_observe(const orc_conf *c, const int *type, const conf_state *s, double *B)
{
    int ns = c->nslab;
    double A = c->L[0] * c->L[2];
    B[0] = s->sw[0] / A;
    B[1] = s->sw[1] / A;
    for (int k = 0; k < 2 * ns + 2; k++) B[2 + k] = 0.0;
    /* the site planes nearest the channel: highest bottom, lowest top     */
    double ybot = -INFINITY, ytop = INFINITY;
    for (int i = 0; i < c->n; i++) {
        if (type[i] == 1 && s->yl[i] > ybot) ybot = s->yl[i];
        if (type[i] == 2 && s->yl[i] < ytop) ytop = s->yl[i];
    }
    for (int i = 0; i < c->n; i++) {
        if (type[i] == 1) {
            if (s->yl[i] >= ybot - 0.1) B[2 + 2 * ns] += s->px[i];
            continue;
        }
        if (type[i] == 2) {
            if (s->yl[i] <= ytop + 0.1) B[3 + 2 * ns] += s->px[i];
            continue;
        }
        int k = (int)floor((s->y[i] + 0.5 * c->L[1]) / c->L[1] * ns);
        k = k < 0 ? 0 : (k >= ns ? ns - 1 : k);
        B[2 + k] += s->px[i];
        B[2 + ns + k] += 1.0;
    }
}

/* Trajectory with per-step observables for the conservation pins:        */
/* obs[t] = {K (sum p^2/2), U_pair, U_tether, alpha, xi, H_ext, P_lattice}  */
int orc_conf_trajectory(const orc_conf *c, const int *type, double *soa, double *lat,
                        double *alpha_io, int n_steps, double *obs)
{
    conf_state s;
    if (cs_alloc(&s, c->n)) return -1;
    cs_load(c, &s, soa, lat);
    s.alpha = *alpha_io;
    if (cs_forces(c, type, &s)) { free(s.buf); return -1; }
    for (int t = 0; t <= n_steps; t++) {
        if (t > 0 && cs_step(c, type, &s)) { free(s.buf); return -1; }
        if (obs) {
            double K = 0.0;
            for (int i = 0; i < c->n; i++) K += s.px[i] * s.px[i] + s.py[i] * s.py[i] + s.pz[i] * s.pz[i];
            K *= 0.5;
            double *o = obs + 7 * t;
            o[0] = K; o[1] = s.U[0]; o[2] = s.U[1]; o[3] = s.alpha; o[4] = s.xi;
            o[5] = K + s.U[0] + s.U[1] + 0.5 * c->Q * s.alpha * s.alpha + c->g * c->Tw * s.xi;
            o[6] = lattice_power(c, type, &s);
        }
    }
    memcpy(soa, s.x, sizeof(double) * 6 * c->n);
    memcpy(lat, s.xl, sizeof(double) * 3 * c->n);
    *alpha_io = s.alpha;
    free(s.buf);
    return 0;
}

/* Mother (lattice at rest): n_eq steps, then n_states states `spacing`   */
/* steps apart (phase point and alpha; the lattice does not move).         */
int orc_conf_mother(const orc_conf *c0, const int *type, const double *init, const double *lat,
                    int n_eq, int n_states, int spacing, double *out, double *out_alpha)
{
    orc_conf c = *c0;
    c.vwall = 0.0;
    conf_state s;
    if (cs_alloc(&s, c.n)) return -1;
    cs_load(&c, &s, init, lat);
    if (cs_forces(&c, type, &s)) { free(s.buf); return -1; }
    for (int t = 0; t < n_eq; t++) if (cs_step(&c, type, &s)) { free(s.buf); return -1; }
    for (int k = 0; k < n_states; k++) {
        for (int t = 0; t < spacing; t++) if (cs_step(&c, type, &s)) { free(s.buf); return -1; }
        memcpy(out + (size_t)k * 6 * c.n, s.x, sizeof(double) * 6 * c.n);
        out_alpha[k] = s.alpha;
    }
    free(s.buf);
    return 0;
}

/* Eq. 3 for the confined system: the mapping of a phase point also maps   */
/* the tether sites (x_l -> -x_l for the x-reflections); alpha is carried  */
/* and negated by the time-reversing mappings 1 and 3 (or reset).          */
void orc_conf_map(const orc_conf *c, int m, const double *in, const double *lat, double alpha_in,
                  int reset_alpha, double *out, double *lat_out, double *alpha_out)
{
    int n = c->n;
    double sx = (m == 2 || m == 3) ? -1.0 : 1.0;
    double spx = (m == 1 || m == 2) ? -1.0 : 1.0;
    double spyz = (m == 1 || m == 3) ? -1.0 : 1.0;
    for (int i = 0; i < n; i++) {
        double x = sx * in[i], xl = sx * lat[i];
        if (x >= 0.5 * c->L[0]) x -= c->L[0];
        if (xl >= 0.5 * c->L[0]) xl -= c->L[0];
        out[i] = x; out[n + i] = in[n + i]; out[2 * n + i] = in[2 * n + i];
        out[3 * n + i] = spx * in[3 * n + i];
        out[4 * n + i] = spyz * in[4 * n + i];
        out[5 * n + i] = spyz * in[5 * n + i];
        lat_out[i] = xl; lat_out[n + i] = lat[n + i]; lat_out[2 * n + i] = lat[2 * n + i];
    }
    double sa = (m == 1 || m == 3) ? -1.0 : 1.0;
    *alpha_out = reset_alpha ? 0.0 : sa * alpha_in;
}

/* One confined daughter: B has (n_steps/sample_every + 1) rows of         */
/* 2 + 2 nslab + 2 responses; Omega as in the header.                      */
int orc_conf_daughter(const orc_conf *c, const int *type, const double *mother, const double *lat,
                      double mother_alpha, int m, int reset_alpha, int n_steps, int sample_every,
                      double *B, double *Omega, double *final_state)
{
    conf_state s;
    if (cs_alloc(&s, c->n)) return -1;
    double a0;
    orc_conf_map(c, m, mother, lat, mother_alpha, reset_alpha, s.x, s.xl, &a0);
    s.alpha = a0;
    if (cs_forces(c, type, &s)) { free(s.buf); return -1; }
    *Omega = lattice_power(c, type, &s) / c->Tw;
    int nb = 2 + 2 * c->nslab + 2;
    cs_observe(c, type, &s, B);
    for (int t = 1; t <= n_steps; t++) {
        if (cs_step(c, type, &s)) { free(s.buf); return -1; }
        if (t % sample_every == 0) cs_observe(c, type, &s, B + (size_t)(t / sample_every) * nb);
    }
    if (final_state) memcpy(final_state, s.x, sizeof(double) * 6 * c->n);
    free(s.buf);
    return 0;
}

int orc_conf_daughters(const orc_conf *c, const int *type, int n_groups, const double *mothers,
                       const double *lat, const double *alpha, int n_steps, int sample_every,
                       double *B, double *Omega, int n_threads)
{
    int S = n_steps / sample_every + 1, nb = 2 + 2 * c->nslab + 2, D = 4 * n_groups, err = 0;
    (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads) reduction(|:err)
    for (int d = 0; d < D; d++) {
        int g = d / 4, m = d % 4;
        err |= orc_conf_daughter(c, type, mothers + (size_t)g * 6 * c->n, lat, alpha[g], m, 0,
                                 n_steps, sample_every, B + (size_t)d * S * nb, Omega + d, NULL) ? 1 : 0;
    }
    return err ? -1 : 0;
}
