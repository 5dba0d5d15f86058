// ttcf_daughter.cu -- the persistent daughter kernel (hot path).
//
// One CTA runs one daughter trajectory at a time and pops the next one from
// an atomic work counter.  A daughter's positions live in shared memory;
// thread t owns atoms i = t + q*blockDim (q < APT) and keeps their momenta
// and forces in registers.  One step of the thermostatted SLLOD equations
// (Eq. 5), split into exactly solvable flows as E D C B A B C D E:
//   phase A  p *= exp(-alpha h/2) (the end-of-step and start-of-step
//            halves folded into one factor), p_x -= gamma (h/2) p_y,
//            p += (h/2) F, drift r += h p + x_hat gamma h (y + h p_y/2)
//                                                              -> barrier 1
//   list     Verlet list rebuilt from a Lees-Edwards-aware cell binning
//            when an atom moved more than (skin - |change of delta|)/2
//   phase B  WCA pair forces (Eq. 6) and virial W_xy over sorted lists
//   phase C  p += (h/2) F, p_x -= gamma (h/2) p_y, per-warp partial sums
//                                                              -> barrier 2
//   lane 0   the two Nose-Hoover half-steps of alpha, the factor
//            exp(-alpha h/2) - 1, the sample B(s) = P_xy(s) of Eq. 7, the
//            Lees-Edwards offset (double-float in MIXED mode, IEEE double
//            in FP64 mode; B(s) is stored as IEEE double)     -> barrier 3
// Lists are sorted by neighbour index and only pairs with r < r_c
// contribute, so forces are a function of the positions alone; positions
// are wrapped into the box every WRAP_EVERY steps of absolute time; hence
// a run split into chunks reproduces one long run bit for bit.
#include "ttcf_daughter_impl.cuh"

namespace ttcf {

// instantiated in ttcf_daughter_u8.cu (per-atom loops unrolled)
extern template cudaError_t launch_one<true, 8, 512, 1>(const RunArgs &, int, int, size_t, cudaStream_t);
extern template int occupancy_one<true, 8, 512, 1>(int, size_t);

#define TTCF_DISPATCH(MIX, FN, ...)                                              \
    switch (variant) {                                                           \
    case 0: return FN<MIX, 1, 256, 4>(__VA_ARGS__);                              \
    case 1: return FN<MIX, 2, 512, 2>(__VA_ARGS__);                              \
    case 2: return FN<MIX, 2, 1024, 1>(__VA_ARGS__);                             \
    case 3: return FN<MIX, 4, 512, 2>(__VA_ARGS__);                              \
    case 4: return FN<MIX, 4, 512, 1>(__VA_ARGS__);                              \
    default: return FN<MIX, 8, 512, 1>(__VA_ARGS__);                             \
    }

cudaError_t launch_daughters(bool mixed, int variant, const RunArgs &a, int threads, int grid,
                             size_t smem, cudaStream_t st) {
    if (mixed) { TTCF_DISPATCH(true, launch_one, a, threads, grid, smem, st) }
    TTCF_DISPATCH(false, launch_one, a, threads, grid, smem, st)
}

int daughter_occupancy(bool mixed, int variant, int threads, size_t smem) {
    if (mixed) { TTCF_DISPATCH(true, occupancy_one, threads, smem) }
    TTCF_DISPATCH(false, occupancy_one, threads, smem)
}



}  // namespace ttcf
