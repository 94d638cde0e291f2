// Phase-1 kernels for T = 1 taps (one translation unit per tap count so the
// instantiations compile in parallel).
#include "k_phase1.cuh"

namespace fe {
template cudaError_t launch_phase1_n1<1>(int, const Phase1Params &, int, cudaStream_t);
template cudaError_t launch_phase1_group_n1<1>(int, const Phase1Group &, cudaStream_t);
}  // namespace fe
