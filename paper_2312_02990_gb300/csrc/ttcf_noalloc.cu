// ttcf_noalloc.cu -- ttcf_run_noalloc: spawn and run a small batch of
// daughters without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they want
// the daughters run: a host application whose device memory is entirely
// owned by its own pool allocator (a cudaMalloc there fails or fragments
// that pool), a latency-critical loop that cannot pay for cudaMalloc and
// cudaFree (both can synchronise the device), or a plugin whose host forbids
// allocation after start-up.  ttcf_spawn_daughters/ttcf_run allocate their
// working buffers per context, so this entry point instead carves them out
// of one fixed array that lives in the library's own device image.
//
// The array is a file-scope static __device__ array of NOALLOC_BYTES; every
// GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// stand-in), so the first call on each device, with that device current,
// looks the address up with cudaGetSymbolAddress and caches it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "ttcf_internal.h"

namespace ttcf {

constexpr size_t NOALLOC_BYTES = 32u << 20;   // 32 MiB
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[MAX_DEVICES] = {nullptr};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Writes the batch table (passed by value, so no host buffer has to outlive
// the call) and the launch order 0..n-1 of the daughters.
__global__ void noalloc_init_kernel(BatchDev bd, BatchDev *d_b, int *w, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *d_b = bd;
    if (i < n) w[i] = i;
}

// True if p is memory the current device can address as device memory
// (device or managed allocations); a plain host pointer is rejected.
bool is_device_pointer(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

ttcf_status noalloc_fail(ttcf_status s, const std::string &m) {
    set_global_error(m.c_str());   // read back with ttcf_last_error(NULL)
    return s;
}

}  // namespace

}  // namespace ttcf

using namespace ttcf;

extern "C" ttcf_status ttcf_run_noalloc(const ttcf_config *cfg, int n_atoms, const double box[3],
                                        int n_mothers, const double *mother_soa,
                                        const double *mother_alpha, const double *shear_rates,
                                        double *B, double *Omega, int *status) {
    if (!cfg || !box || !mother_soa || !shear_rates || !B || !Omega || !status)
        return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: NULL argument");
    if (!is_device_pointer(mother_soa) || !is_device_pointer(shear_rates) || !is_device_pointer(B) ||
        !is_device_pointer(Omega) || !is_device_pointer(status) ||
        (mother_alpha && !is_device_pointer(mother_alpha)))
        return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: every array must be device memory");
    const ttcf_config &c = *cfg;
    if (c.system != TTCF_BULK_WCA || (c.precision != TTCF_FP64 && c.precision != TTCF_MIXED) ||
        !(c.dt > 0) || !(c.T > 0) || !(c.tau_T > 0) || c.n_steps < 1 || c.sample_every < 1 ||
        c.n_steps % c.sample_every || c.mapping_mask == 0 ||
        c.kernel_variant < 0 || c.kernel_variant > N_VARIANTS || c.block_threads < 0 ||
        c.block_threads % 32 || c.skin > 1.0 ||
        (c.cell_frac != 0.0 && !(c.cell_frac >= 0.4 && c.cell_frac <= 1.0)))
        return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: invalid configuration");
    if (n_atoms < 4 || n_atoms > 4096 || n_mothers < 1)
        return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: n_atoms must be in [4, 4096], n_mothers >= 1");
    const double rc = 1.1224620483093730;
    const double skin = c.skin > 0 ? c.skin : DEFAULT_SKIN;
    const int N = n_atoms, G = n_mothers;
    int maps[MAX_MAPS], M = 0;
    for (int m = 0; m < MAX_MAPS; m++) if (c.mapping_mask & (1u << m)) maps[M++] = m;
    for (int k = 0; k < M; k++)
        if (map_swaps_xz(maps[k]) && !(fabs(box[0] - box[2]) <= 1e-12 * box[0]))
            return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: the x <-> z exchange mappings need L_x = L_z");
    const long long D = (long long)G * M;
    const int S = c.n_steps / c.sample_every + 1;

    // launch shape: the default table of the context path
    int variant = c.kernel_variant > 0 ? c.kernel_variant - 1 : default_variant(N);
    const Variant v = variant_of(variant);
    int threads = c.block_threads > 0 ? c.block_threads : (N + v.apt - 1) / v.apt;
    threads = (threads + 31) / 32 * 32;
    if (threads > v.maxt || threads * v.apt < N)
        return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: launch variant cannot hold n_atoms");

    SpawnArgs sa;
    memset(&sa, 0, sizeof(sa));
    BatchDev bd;
    memset(&bd, 0, sizeof(bd));
    sa.N = bd.N = N; sa.M = bd.M = M; sa.G = bd.G = G; bd.S = sa.S = S;
    for (int k = 0; k < MAX_MAPS; k++) sa.maps[k] = bd.maps[k] = k < M ? maps[k] : 0;
    for (int k = 0; k < 3; k++) {
        if (!isfinite(box[k]) || !(box[k] >= 3.0 * (rc + skin)))
            return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: box edge not finite or shorter than 3*(r_c+skin)");
        sa.L[k] = bd.L[k] = box[k];
        sa.nc[k] = (int)(box[k] / rc);
    }
    sa.ncell = sa.nc[0] * sa.nc[1] * sa.nc[2];
    sa.V = bd.V = box[0] * box[1] * box[2];
    sa.T = bd.T = c.T;
    const double g = c.dof_mode == 1 ? 3.0 * N - 3.0 : 3.0 * N;
    bd.Q = g * c.T * c.tau_T * c.tau_T;
    bd.gT = g * c.T;
    bd.skin = (float)skin;
    const bool mixed = c.precision == TTCF_MIXED;

    // carve-up of the static array; reject sizes beyond it before any work
    size_t off = 0;
    const size_t o_batch = off; off += align256(sizeof(BatchDev));
    const size_t o_dbatch = off; off += align256(sizeof(int) * D);
    const size_t o_work = off; off += align256(sizeof(int) * D);
    const size_t o_queue = off; off += align256(sizeof(int));
    const size_t o_alpha = off; off += align256(sizeof(double) * G);
    const size_t o_moth = off; off += align256(sizeof(unsigned long long) * G * 6 * N);
    const size_t o_feat = off; off += align256(sizeof(double) * G * FEAT_RAW);
    const size_t o_pairs = off; off += align256(sizeof(unsigned long long) * D);
    const size_t o_reb = off; off += align256(sizeof(unsigned int) * D);
    const size_t o_scal = off; off += align256(sizeof(double) * D * 4);
    const size_t nbr_per_cta = sizeof(unsigned int) * NBR_WORDS * (size_t)N;
    // per CTA: its neighbour lists and, for the plo_global variant, the lo
    // parts of its daughter's positions
    const size_t plo_per_cta = plo_global(mixed, variant) ? sizeof(float4) * (size_t)N : 0;
    if (off + nbr_per_cta + plo_per_cta > NOALLOC_BYTES)
        return noalloc_fail(TTCF_E_INVALID,
                            "ttcf_run_noalloc: batch needs more than the 32 MiB static scratch "
                            "(reduce n_mothers or n_atoms, or use ttcf_spawn_daughters)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return noalloc_fail(TTCF_E_CUDA, "ttcf_run_noalloc: no current CUDA device");
    }
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {   // once per device, with that device current
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(TTCF_E_CUDA, std::string("ttcf_run_noalloc: cudaGetSymbolAddress: ") +
                                                     cudaGetErrorString(e));
            }
            g_noalloc_ptr[dev] = (unsigned char *)p;
        }
        base = g_noalloc_ptr[dev];
    }
    int nsm = 0, optin = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(TTCF_E_CUDA, "ttcf_run_noalloc: device query failed");
    }
    // list cells and list-build layout by the rule of ttcf_spawn_daughters +
    // ttcf_run for a batch alone (cells cell_frac r_l wide, coarser where the
    // variant's resident CTAs need the shared memory; the cell-ordered build
    // where its larger shared memory keeps them), so both give the same bits
    {
        const double rl = rc + skin;
        const double frac = c.cell_frac > 0 ? c.cell_frac : 2.0 / 3.0;
        const double fracs[3] = {frac, std::max(frac, 2.0 / 3.0), 1.0};
        for (int f = 0; f < 3; f++) {
            int ncf[3];
            for (int k = 0; k < 3; k++) ncf[k] = std::max(3, (int)floor(box[k] / (rl * fracs[f])));
            const int ncell = ncf[0] * ncf[1] * ncf[2];
            const size_t sm = daughter_smem_bytes(mixed, N, ncell, false, !plo_global(mixed, variant));
            if (f == 2 || (size_t)v.minb * (sm + 1024) <= (size_t)per_sm) {
                for (int k = 0; k < 3; k++) bd.nc[k] = ncf[k];
                bd.ncell = ncell;
                break;
            }
        }
    }
    const bool plo_smem = !plo_global(mixed, variant);
    size_t smem = daughter_smem_bytes(mixed, N, bd.ncell, false, plo_smem);
    if (smem > (size_t)optin)
        return noalloc_fail(TTCF_E_INVALID, "ttcf_run_noalloc: daughter needs more shared memory than a CTA has");
    int nb = daughter_occupancy(mixed, variant, threads, smem);
    int cpos = 0;
    {
        const size_t s2 = daughter_smem_bytes(mixed, N, bd.ncell, true, plo_smem);
        if (s2 <= (size_t)optin) {
            const int nb2 = daughter_occupancy(mixed, variant, threads, s2);
            if (nb2 >= 1 && nb2 >= std::min(nb, v.minb)) { cpos = 1; smem = s2; nb = nb2; }
        }
    }
    if (nb < 1) nb = 1;
    long long grid = std::min<long long>(D, (long long)nb * nsm);
    grid = std::min<long long>(grid, (long long)((NOALLOC_BYTES - off) / (nbr_per_cta + plo_per_cta)));
    if (grid < 1) grid = 1;

    cudaStream_t st = (cudaStream_t)c.stream;
    BatchDev *d_b = (BatchDev *)(base + o_batch);
    int *d_dbatch = (int *)(base + o_dbatch), *d_work = (int *)(base + o_work);
    int *d_queue = (int *)(base + o_queue);
    double *d_alpha = (double *)(base + o_alpha);
    unsigned long long *d_moth = (unsigned long long *)(base + o_moth);
    bd.mothers = d_moth;
    bd.m_alpha = mother_alpha ? mother_alpha : d_alpha;
    bd.gamma = shear_rates;
    bd.B = B; bd.Omega = Omega; bd.status = status;
    bd.pairs = (unsigned long long *)(base + o_pairs);
    bd.rebuilds = (unsigned int *)(base + o_reb);
    bd.scal = (double *)(base + o_scal);
    bd.state = nullptr;
    bd.d0 = 0;

    // the array keeps the previous call's contents: clear what starts at
    // zero.  Only kernels and memsets are queued: no host buffer is read
    // after this function returns.
    cudaError_t e = cudaMemsetAsync(d_dbatch, 0, sizeof(int) * D, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_queue, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_alpha, 0, sizeof(double) * G, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bd.pairs, 0, sizeof(unsigned long long) * D, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bd.rebuilds, 0, sizeof(unsigned int) * D, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int) * D, st);
    if (e == cudaSuccess) {
        noalloc_init_kernel<<<(unsigned)((D + 255) / 256), 256, 0, st>>>(bd, d_b, d_work, (int)D);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        sa.mixed = mixed ? 1 : 0;
        sa.src = mother_soa; sa.gamma = shear_rates; sa.mothers = d_moth;
        sa.B = B; sa.Omega = Omega; sa.feat = (double *)(base + o_feat); sa.delta = 0.0;
        e = launch_spawn(sa, st);
    }
    if (e == cudaSuccess) {
        RunArgs a;
        memset(&a, 0, sizeof(a));
        a.batches = d_b; a.work = d_work; a.dbatch = d_dbatch; a.n_work = (int)D;
        a.queue = d_queue;
        a.nbr = (unsigned int *)(base + off);
        a.plo_g = plo_per_cta ? (float4 *)(base + off + (size_t)grid * nbr_per_cta) : nullptr;
        a.nmax = N; a.ncellmax = bd.ncell; a.cpos = cpos;
        a.step0 = 0; a.step1 = c.n_steps; a.sample_every = c.sample_every;
        a.fresh = 1; a.save_state = 0; a.reset_alpha = c.reset_alpha;
        a.dt = c.dt; a.delta0 = 0.0;
        e = launch_daughters(mixed, variant, a, threads, (int)grid, smem, st);
    }
    if (e != cudaSuccess)
        return noalloc_fail(TTCF_E_CUDA, std::string("ttcf_run_noalloc: ") + cudaGetErrorString(e));
    return TTCF_OK;
}
