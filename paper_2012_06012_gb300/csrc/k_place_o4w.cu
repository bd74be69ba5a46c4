// Instantiations of the sort/place kernel for int32_t offsets and RecW records
// (one translation unit per combination so they compile in parallel).
#include "k_place_impl.cuh"

namespace mgt {

template <>
cudaError_t launch_place_cs<int32_t, RecW>(const Params &p, const Inputs &in, const Outputs &out,
                                          const Ws &ws, cudaStream_t st) {
#define MGT_PLACE_U(CS)                                                                   \
    switch (p.unroll) {                                                                   \
    case 1: return launch_place_t<int32_t, RecW, CS, 1>(p, in, out, ws, st);               \
    case 2: return launch_place_t<int32_t, RecW, CS, 2>(p, in, out, ws, st);               \
    default: return launch_place_t<int32_t, RecW, CS, 4>(p, in, out, ws, st);              \
    }
    switch (p.cs) {
    case 1: MGT_PLACE_U(1)
    case 2: MGT_PLACE_U(2)
    case 4: MGT_PLACE_U(4)
    default: MGT_PLACE_U(8)
    }
#undef MGT_PLACE_U
}

}  // namespace mgt
