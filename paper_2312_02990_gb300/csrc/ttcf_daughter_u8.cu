// ttcf_daughter_u8.cu -- the MIXED launch variant of 8 atoms per thread
// (512 threads, 128 registers), compiled with its per-atom loops unrolled
// (see ttcf_daughter_impl.cuh).
#define TTCF_UNROLL_ATOMS 1
#include "ttcf_daughter_impl.cuh"

namespace ttcf {

template cudaError_t launch_one<true, 8, 512, 1>(const RunArgs &, int, int, size_t, cudaStream_t);
template int occupancy_one<true, 8, 512, 1>(int, size_t);

}  // namespace ttcf
