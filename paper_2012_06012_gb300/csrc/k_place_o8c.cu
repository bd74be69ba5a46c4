// Level-2 kernels instantiated for int64_t offsets and RecC records (one
// translation unit per combination so that they compile in parallel).
#include "k_place_impl.cuh"

namespace mgt {
template cudaError_t launch_level2_t<int64_t, RecC>(const Params &, const Inputs &, const Outputs &,
                                                  const Ws &, cudaStream_t, int);
}  // namespace mgt
