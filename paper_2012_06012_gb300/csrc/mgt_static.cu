// mgt_transpose_static: the transpose with its scratch memory in a fixed
// device array owned by the library instead of a caller-provided workspace.
//
// For callers that cannot allocate device memory themselves -- for example a
// plug-in whose host framework owns every device allocation, or a loop where
// the implicit device-wide synchronisation of cudaMalloc/cudaFree is not
// acceptable.  The call allocates nothing: no cudaMalloc, cudaFree, pinned
// host memory or allocating library routine.  Its limits: the scratch is
// MGT_STATIC_SCRATCH_BYTES (64 MiB) per device, so only matrices whose
// default-plan workspace fits are accepted (others: MGT_ENOMEM), and
// P <= MGT_STATIC_MAX_PARTS row blocks.
#include "mgt_internal.cuh"

#include <mutex>

namespace mgt {

constexpr size_t kStaticScratch = (size_t)64 << 20;
static_assert(kStaticScratch == MGT_STATIC_SCRATCH_BYTES, "header and library disagree");

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratch];

// Device address of g_static_scratch (the host-side name is only a stand-in
// for the symbol, not a device address).  It is looked up with
// cudaGetSymbolAddress on the first call on a device, and again whenever the
// current context is not the one the cached address belongs to (after a
// cudaDeviceReset the module is loaded anew, possibly at another address).
// Contexts are told apart by the driver's unique context id; without it the
// address is looked up on every call (the lookup allocates nothing).
using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;
static std::once_flag g_ctx_once;

static unsigned long long current_context_id() {
    std::call_once(g_ctx_once, [] {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
                cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(g);
        }
        cudaGetLastError();
    });
    if (!g_ctx_current || !g_ctx_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

struct ScratchEntry {
    unsigned long long ctx;  // context id the address belongs to (0: unknown)
    void *addr;
};
static ScratchEntry g_scratch[64];
static std::mutex g_scratch_mu;

static int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MGT_ECUDA;
    if (dev < 0 || dev >= 64) return MGT_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long ctx = current_context_id();
    ScratchEntry &e = g_scratch[dev];
    if (ctx == 0 || e.ctx != ctx || !e.addr) {
        void *ptr = nullptr;
        const cudaError_t rc = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (rc != cudaSuccess || !ptr) return note_cuda(rc, "static scratch address");
        e.addr = ptr;
        e.ctx = current_context_id();  // the lookup made the device's context current
    }
    *out = e.addr;
    return MGT_OK;
}

// Row-block offsets travel as kernel parameters (no host staging buffer).
constexpr int kOffChunk = 480;
struct OffChunk {
    long long v[kOffChunk];
};
__global__ void k_static_offsets(OffChunk c, int first, int count, long long R, int P, int equal,
                                 long long *poff) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const int d = first + i;
        poff[d] = equal ? (long long)(((__int128)d * R) / P) : c.v[i];
    }
}

}  // namespace mgt

using namespace mgt;

extern "C" int mgt_transpose_static(const mgt_desc *desc, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                                    mgt_stream_t stream) {
    if (!desc || !in || !out) return MGT_EINVAL;
    if (desc->n_parts > MGT_STATIC_MAX_PARTS || desc->flags != 0) return MGT_EINVAL;
    Params p;
    int rc = default_params(desc, &p);
    if (rc != MGT_OK) return rc;
    const WsLayout L = layout_for(p);
    if (L.total > kStaticScratch) return MGT_ENOMEM;
    if (!in->row_ptr || !in->cell_ptr || !out->row_ptr || !out->cell_ptr) return MGT_EINVAL;
    if (p.C > 0 && (!in->col_idx || !out->col_idx)) return MGT_EINVAL;
    if (p.V > 0 && (!in->values || !out->values)) return MGT_EINVAL;
    if ((out->part_cells == nullptr) != (out->part_values == nullptr)) return MGT_EINVAL;
    void *base = nullptr;
    rc = scratch_address(&base);
    if (rc != MGT_OK) return rc;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Ws ws = ws_from(base, L);
    Inputs I{in->row_ptr, in->col_idx, in->cell_ptr, static_cast<const uint8_t *>(in->values)};
    Outputs O{out->row_ptr, out->col_idx, out->cell_ptr, static_cast<uint8_t *>(out->values),
              reinterpret_cast<long long *>(out->part_cells),
              reinterpret_cast<long long *>(out->part_values)};
    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(ws.hdr, 0, 256, st) != cudaSuccess) return MGT_ECUDA;
    if (p.B > 0 && cudaMemsetAsync(ws.bucket_vtot, 0, (size_t)p.B * 8, st) != cudaSuccess)
        return MGT_ECUDA;
    if (O.part_cells && cudaMemsetAsync(O.part_cells, 0, (size_t)p.P * p.P * 8, st) != cudaSuccess)
        return MGT_ECUDA;
    if (O.part_values && cudaMemsetAsync(O.part_values, 0, (size_t)p.P * p.P * 8, st) != cudaSuccess)
        return MGT_ECUDA;
    for (int first = 0; first <= p.P; first += kOffChunk) {
        OffChunk c{};
        const int count = (p.P + 1 - first) < kOffChunk ? (p.P + 1 - first) : kOffChunk;
        if (desc->part_off)
            for (int i = 0; i < count; ++i) c.v[i] = desc->part_off[first + i];
        k_static_offsets<<<1, 256, 0, st>>>(c, first, count, p.R, p.P, desc->part_off ? 0 : 1,
                                            ws.poff);
        if (cudaGetLastError() != cudaSuccess) return MGT_ECUDA;
    }
    return enqueue_kernels(p, I, O, ws, st, nullptr);
}

extern "C" int mgt_static_status(mgt_stream_t stream) {
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != MGT_OK) return rc;
    return mgt_read_status(base, stream);
}
