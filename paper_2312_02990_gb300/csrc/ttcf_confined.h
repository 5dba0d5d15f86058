// ttcf_confined.h -- device descriptors of the confined system (Example 2):
// Lennard-Jones fluid between two walls of tethered atoms whose lattice
// sites slide at +-v in x (Eq. 10), dissipation function of Eq. 11.
// Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include "ttcf_device.cuh"

namespace ttcf {

constexpr int CONF_NSLAB = 40;                     // slabs of the velocity profile
constexpr int CONF_NOBS = 2 + 2 * CONF_NSLAB + 2;  // responses per sample (see ttcf_confined.cu)
constexpr double CONF_LAYER_TOL = 0.1;             // inner wall layer: sites within this of the plane
constexpr int CONF_CAP = 128;                      // Verlet neighbours per atom
constexpr int CONF_GROUPS = CONF_CAP / 8;          // 16-byte groups of 8 uint16 entries
constexpr int CONF_THREADS = 1024;                 // one CTA per daughter
constexpr int CONF_NMAX = 12288;                   // atoms per daughter
constexpr int CONF_SCRATCH_F4 = 12;                // float4 rows of per-CTA scratch
constexpr double CONF_DEFAULT_SKIN = 0.5;          // fastest measured for the Example 2 channel

// One batch of confined daughters (same geometry and types).
struct ConfBatchDev {
    int N, M, G, S, n_obs;
    int maps[4];
    int nc[3], ncell;          // list cells (x, y, z); y clamps at the edges
    double L[3];               // Lx, Ly (slab extent, y not periodic), Lz
    double A;                  // wall area Lx * Lz
    double Q, gT;              // wall thermostat: Q = g T tau^2, g = 3 N_w
    double rc, k, c_ff, c_wf, c_ww;   // Eq. 9 cut-off and wetting, tether stiffness
    int ww_on;                 // wall-wall pairs interact (c_ww)
    int pad2_;
    double half_h;             // v_wall = gamma * half_h
    double inner_y[2];         // inner wall layers: bottom sites y >= inner_y[0],
                               // top sites y <= inner_y[1]
    float skin;
    int pad_;
    long long d0;
    const unsigned long long *mothers;   // [G][6][N] float-pair slots
    const double *m_alpha;               // [G]
    const double *gamma;                 // [G]
    const int *types;                    // [N] 0 fluid, 1 bottom wall, 2 top wall
    const double *lattice;               // [3][N] tether sites at t = 0
    double *B;                           // [D][n_obs][S]
    double *Omega;                       // [D]
    int *status;                         // [D]
    unsigned long long *pairs;           // [D]
    unsigned int *rebuilds;              // [D]
};

struct ConfRunArgs {
    const ConfBatchDev *batches;
    const int *work;           // global daughter indices
    const int *dbatch;         // batch of each global daughter
    int n_work;
    int *queue;
    float4 *scratch;           // [grid][CONF_SCRATCH_F4][nmax]
    uint4 *nbr;                // [grid][CONF_GROUPS][nmax]: 8 uint16 per entry,
                               // padded with the ghost index nmax
    int *ncnt;                 // [grid][nmax]
    int nmax, ncellmax;
    int n_steps, sample_every, reset_alpha;
    double dt;
    const volatile int *abort_flag;
    double *snap;              // mother mode: [D][n_snap][6][N] or null
    double *snap_alpha;        // [D][n_snap]
    int snap_first, snap_every, n_snap;
};

// Spawn: per mother g, in IEEE double, Omega(0) (Eq. 11), the x force of the
// fluid on each wall, slab sums of fluid p_x and counts; the values of each
// mapped daughter follow from the sign rules of the mappings.
struct ConfSpawnArgs {
    int N, M, G, S, n_obs;
    int maps[4];
    int nc[3], ncell;          // cells of width >= r_c
    double L[3], A, Tw, rc, k, c_wf, half_h;
    double inner_y[2];         // as in ConfBatchDev
    const double *src;         // [G][6][N]
    const double *gamma;       // [G]
    const int *types;          // [N]
    const double *lattice;     // [3][N]
    unsigned long long *mothers;   // [G][6][N] float-pair slots (out)
    double *B;                 // [D][n_obs][S]: writes sample 0
    double *Omega;             // [D]
};

size_t conf_smem_bytes(int nmax, int ncellmax);
size_t conf_spawn_smem_bytes(int N, int ncell);
cudaError_t launch_confined(const ConfRunArgs &a, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_conf_spawn(const ConfSpawnArgs &a, cudaStream_t st);

}  // namespace ttcf
