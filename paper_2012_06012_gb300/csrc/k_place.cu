// Dispatch of the level-2 kernels (sort/place and the large-bucket chunk
// passes) over offset width and record format.
#include "k_place_impl.cuh"

namespace mgt {

static cudaError_t level2(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                          cudaStream_t st, int which) {
    if (p.o == 4)
        return p.wide ? launch_level2_t<int32_t, RecW>(p, in, out, ws, st, which)
                      : launch_level2_t<int32_t, RecC>(p, in, out, ws, st, which);
    return p.wide ? launch_level2_t<int64_t, RecW>(p, in, out, ws, st, which)
                  : launch_level2_t<int64_t, RecC>(p, in, out, ws, st, which);
}

cudaError_t launch_place(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                         cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    return level2(p, in, out, ws, st, 0);
}
cudaError_t launch_place_chunks(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                                cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    return level2(p, in, out, ws, st, 1);
}
cudaError_t launch_place_fallback(const Params &p, const Inputs &in, const Outputs &out,
                                  const Ws &ws, cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    return level2(p, in, out, ws, st, 2);
}
cudaError_t launch_copy(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                        cudaStream_t st) {
    return level2(p, in, out, ws, st, 3);
}

size_t place_smem_bytes(const Params &p) {
    const int logcs = p.cs == 1 ? 0 : p.cs == 2 ? 1 : p.cs == 4 ? 2 : 3;
    const int wsub = 1 << (p.bshift - logcs);
    switch (p.cs) {
    case 1: return p.wide ? cl_layout<RecW, 1>(p.cap, wsub).total : cl_layout<RecC, 1>(p.cap, wsub).total;
    case 2: return p.wide ? cl_layout<RecW, 2>(p.cap, wsub).total : cl_layout<RecC, 2>(p.cap, wsub).total;
    case 4: return p.wide ? cl_layout<RecW, 4>(p.cap, wsub).total : cl_layout<RecC, 4>(p.cap, wsub).total;
    default: return p.wide ? cl_layout<RecW, 8>(p.cap, wsub).total : cl_layout<RecC, 8>(p.cap, wsub).total;
    }
}
size_t chunk_smem_bytes(const Params &p) {
    return p.wide ? ch_layout<RecW>(p.chm, 1 << p.bshift).total : ch_layout<RecC>(p.chm, 1 << p.bshift).total;
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
