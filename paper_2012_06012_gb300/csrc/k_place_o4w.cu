// Level-2 kernels instantiated for int32_t offsets and RecW records (one
// translation unit per combination so that they compile in parallel).
#include "k_place_impl.cuh"

namespace mgt {
template cudaError_t launch_level2_t<int32_t, RecW>(const Mat &, const BatchArgs &, long long, size_t,
                                                  cudaStream_t, int);
template long long resident_clusters_t<int32_t, RecW>(int, size_t);
}  // namespace mgt
