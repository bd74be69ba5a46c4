// Dispatch of the level-2 kernels (sort/place and the large-bucket chunk
// passes) over offset width and record format.
#include "k_place_impl.cuh"

namespace mgt {

cudaError_t launch_place(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                         cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    if (p.o == 4)
        return p.wide ? launch_place_cs<int32_t, RecW>(p, in, out, ws, st)
                      : launch_place_cs<int32_t, RecC>(p, in, out, ws, st);
    return p.wide ? launch_place_cs<int64_t, RecW>(p, in, out, ws, st)
                  : launch_place_cs<int64_t, RecC>(p, in, out, ws, st);
}

size_t place_smem_bytes(const Params &p) {
    const int w = 1 << p.bshift;
    return p.wide ? place_layout<RecW>(p.cap, w).total : place_layout<RecC>(p.cap, w).total;
}

template <typename OffT, typename Rec>
static cudaError_t launch_chunk_t(const Params &p, const Inputs &in, const Outputs &out,
                                  const Ws &ws, cudaStream_t st, bool scan) {
    const int w = 1 << p.bshift;
    const int grid = 2 * sm_count();
    if (!scan) {
        size_t smem = (size_t)w * 4 + 8 + (size_t)w * 8;
        auto kern = k_chunk_hist<OffT, Rec>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, P_THREADS, smem, st>>>(reinterpret_cast<const Rec *>(ws.recs), ws.items,
                                            ws.multi_items, ws.mc, p.bshift, in.cell_ptr, p.C, p.V, ws.hdr);
    } else {
        size_t smem = (size_t)w * 16 + 48 * 8;
        auto kern = k_chunk_scan<OffT>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, P_THREADS, smem, st>>>(ws.multi_buckets, ws.mc, p.bshift, p.N, ws.bucket_base,
                                            ws.bucket_vbase, out.row_ptr, ws.hdr);
    }
    return cudaGetLastError();
}

cudaError_t launch_chunk_hist(const Params &p, const Inputs &in, const Ws &ws, cudaStream_t st) {
    if (p.B == 0 || p.max_multi_rows == 0) return cudaSuccess;
    Outputs none = {};
    if (p.o == 4)
        return p.wide ? launch_chunk_t<int32_t, RecW>(p, in, none, ws, st, false)
                      : launch_chunk_t<int32_t, RecC>(p, in, none, ws, st, false);
    return p.wide ? launch_chunk_t<int64_t, RecW>(p, in, none, ws, st, false)
                  : launch_chunk_t<int64_t, RecC>(p, in, none, ws, st, false);
}

cudaError_t launch_chunk_scan(const Params &p, const Outputs &out, const Ws &ws, cudaStream_t st) {
    if (p.B == 0 || p.max_multi_rows == 0) return cudaSuccess;
    Inputs none = {};
    if (p.o == 4) return launch_chunk_t<int32_t, RecC>(p, none, out, ws, st, true);
    return launch_chunk_t<int64_t, RecC>(p, none, out, ws, st, true);
}


}  // namespace mgt
