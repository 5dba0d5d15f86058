// ttcf_internal.h -- host-side declarations shared by the library's
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include "ttcf.h"
#include "ttcf_device.cuh"

namespace ttcf {

// persistent daughter kernel (ttcf_daughter.cu)
cudaError_t launch_daughters(bool mixed, int variant, const RunArgs &a, int threads, int grid,
                             size_t smem, cudaStream_t st);
int daughter_occupancy(bool mixed, int variant, int threads, size_t smem);

// daughters under planar elongational flow (ttcf_elong.cu): one CTA per
// daughter of one batch (gamma holds the elongation rates), persistent over
// the batch; Verlet lists of radius r_c + skin, built on cell grids of at
// most ncmax[k] cells along axis k (the bound of the largest box the run
// reaches), ELONG_CAP entries per atom in a [grid][ELONG_CAP][N] scratch.
constexpr int ELONG_CAP = 32;
constexpr double ELONG_SKIN = 0.35;
struct ElongArgs {
    BatchDev b;
    int step0, step1;              // run absolute steps step0+1 .. step1
    int sample_every;
    int fresh;                     // start from the mapped mother state
    int save_state;                // write the loop state at step1
    int reset_alpha;
    int ncmax[3];
    float skin;
    double dt;
    unsigned short *nbr;           // Verlet list scratch [grid][ELONG_CAP][N]
    const volatile int *abort_flag;  // host-mapped, may be null
};
size_t elong_smem_bytes(bool mixed, int N, int ncellmax);
int elong_threads(int N);
// CTAs of a launch over D daughters (0 if one does not fit)
int elong_grid(bool mixed, int N, int ncellmax, int nsm, long long D);
cudaError_t launch_elong(bool mixed, const ElongArgs &a, int grid, cudaStream_t st);

// momentum kicks of copies of one phase point (ttcf_kick.cu)
struct KickArgs {
    int N;
    int keep_energy;
    double ks;                    // kick * sqrt(T): standard deviation of a kick
    unsigned long long seed;      // Philox key (low word k0)
    const double *src;            // [6][N]
    const int *types;             // [N] groups 0..2, or null (one group)
    double *out;                  // [n_copies][6][N]
};
cudaError_t launch_kick(const KickArgs &a, int n_copies, cudaStream_t st);

// spawn (ttcf_spawn.cu): per mother group, IEEE-double pressure tensor of
// the mother, B(0) and Omega(0) of its mapped daughters, conversion of the
// mother into the state format of the daughter kernel.
struct SpawnArgs {
    int N, M, G;
    int maps[MAX_MAPS];        // mapping codes (see MAX_MAPS)
    int nc[3];                 // cells per side, width >= r_c
    int ncell;
    double L[3], V, T;
    int mixed;                 // 1: write float pairs, 0: doubles
    const double *src;         // [G][6][N] mother phase points
    const double *gamma;       // [G]
    unsigned long long *mothers;  // [G][6][N] slots (out)
    double *B;                 // [D][S]: writes B[d][0]
    int S;
    double *Omega;             // [D]
    double *feat;              // [G][FEAT_RAW] raw features, or null
    double delta;              // Lees-Edwards offset of the phase points
    int elong;                 // 1: B(0) = P_xx - P_zz (planar elongational
                               // flow; the x <-> z exchange negates it)
};
cudaError_t launch_spawn(const SpawnArgs &a, cudaStream_t st);

// Raw per-state features: K_ab = sum p_a p_b (6: xx yy zz xy xz yz), W_ab
// virial sums (6), U, sum p^2, then for q = 1..4 (cos, sin) modes over 40
// slabs in y of the density (8) and of the x momentum (8), each divided by
// N; two unused slots.  The spawn kernel writes the first 14 (its pressure
// tensor pass) and zeros; the FP32 features kernel of the control variate
// writes all of them.
constexpr int FEAT_RAW = 32;
size_t spawn_smem_bytes(int N, int ncell);

// reduction (ttcf_reduce.cu): fixed-order ensemble averages of one batch.
struct ReduceArgs {
    int M, G, S;
    int n_obs;                 // observables per sample (1 for the bulk P_xy)
    const double *B;           // [G*M][n_obs][S]
    const double *Omega;       // [G*M]
    const int *status;         // [G*M]
    double ds;                 // sample spacing in time
    double *Y, *Dg, *J;        // [n_obs][G][S] work arrays
    double *Og;                // [G + 2]: group means of Omega(0), then <Omega(0)> and the valid count
    double *valid;             // [G] 1 if every daughter of the group is OK
    double *out;               // [n_obs][9][S]: corr, corr_se, dav, dav_se,
                               //   ttcf, ttcf_se, corr_c, ttcf_c, n_valid
};
cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t st);

// Time autocorrelations of B[g][s0 .. s0+n) (row stride S) over G
// trajectories for lags 0 .. max_lag (< n): acf = <B(t)B(t+k)>, acf2 of
// B^2 - <B^2>; m2 (device scalar) receives <B^2>.
cudaError_t launch_acf(const double *B, int G, int S, int s0, int n, int max_lag, double *acf,
                       double *acf2, double *m2, cudaStream_t st);

// Equilibrium friction (Eq. 12 by the equilibrium method): per confined
// daughter d and sample s, the slip velocity dv = (inner wall layer p_x
// sum) / n_layer - (adjacent slabs' p_x sum) / (their fluid count) and the
// wall's force on the fluid F = -A sigma_w; then, for lags k = 0 .. max_lag,
// the correlations <dv(t) F(t+k)> and <dv(t) dv(t+k)> over the valid
// daughters (status 0) and all time origins, in a fixed summation order.
constexpr int SLIP_MAX_SLABS = 8;
struct SlipArgs {
    const double *B;           // [D][n_obs][S]
    const int *status;         // [D]
    int D, n_obs, S, nslab, wall, n_slabs;
    int slabs[SLIP_MAX_SLABS]; // slabs adjacent to the wall
    double n_layer, area;
    double *dv, *F;            // [D][S] out (zeros for invalid daughters)
};
cudaError_t launch_slip_correlations(const SlipArgs &a, int max_lag, double *c_dvf, double *c_dvdv,
                                     cudaStream_t st);

// Sets the text returned by ttcf_last_error(NULL) (calls without a context).
void set_global_error(const char *msg);

}  // namespace ttcf
