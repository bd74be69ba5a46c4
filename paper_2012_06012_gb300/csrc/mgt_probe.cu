// Memory-system probe behind the choice of the value copy's order.
//
// The value exchange of the paper's view swap (Sec. 3, second step) moves
// every cell's run of values from its place in the input to its place in the
// output.  On one GPU that permutation of runs can be walked in output order
// (a gather: random reads, sequential writes -- what the value-copy kernel
// does) or in input order (a scatter: sequential reads, random writes; it
// needs each input cell's output offset first, one more random write per
// cell).  This kernel measures the raw rates of the two orders on runs of a
// fixed size, and of the scatter's extra offset writes, so that the choice
// rests on measurements of this memory system.
#include "mgt_internal.cuh"

namespace mgt {

constexpr int PR_THREADS = 512;
constexpr int PR_UNROLL = 4;

// mode 0: dst[r] <- src[perm[r]]   (gather; runs of `rb` bytes)
// mode 1: dst[perm[r]] <- src[r]   (scatter)
// mode 2: ((uint32_t *)dst)[perm[r]] = r   (one 4-byte random write per run)
// mode 3: dst[r] <- src[r]         (sequential copy, the reference rate)
// A warp takes 32 * PR_UNROLL consecutive 16-byte units per round; unit u
// belongs to run u / (rb / 16).  Every index stays below n (perm is a
// permutation of [0, n)), so every access is inside the n * rb bytes.
__global__ void __launch_bounds__(PR_THREADS) k_probe_runs(int mode, const uint8_t *__restrict__ src,
                                                           uint8_t *__restrict__ dst,
                                                           const uint32_t *__restrict__ perm,
                                                           long long n, int rb) {
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (mode == 2) {
        uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
        for (long long r = tid; r < n; r += nthreads) d32[__ldcs(perm + r)] = (uint32_t)r;
        return;
    }
    const int upr = rb / 16;  // 16-byte units per run
    const long long units = n * upr;
    for (long long u0 = tid; u0 < units; u0 += nthreads * PR_UNROLL) {
        int4 v[PR_UNROLL];
        long long dofs[PR_UNROLL];
#pragma unroll
        for (int j = 0; j < PR_UNROLL; ++j) {
            const long long u = u0 + j * nthreads;
            if (u < units) {
                const long long r = u / upr, w = u - r * upr;
                long long sr = r, dr = r;
                if (mode == 0) sr = __ldg(perm + r);
                else if (mode == 1) dr = __ldg(perm + r);
                v[j] = __ldcs(reinterpret_cast<const int4 *>(src + sr * rb) + w);
                dofs[j] = dr * rb + w * 16;
            }
        }
#pragma unroll
        for (int j = 0; j < PR_UNROLL; ++j) {
            const long long u = u0 + j * nthreads;
            if (u < units) __stcs(reinterpret_cast<int4 *>(dst + dofs[j]), v[j]);
        }
    }
}

}  // namespace mgt

using namespace mgt;

extern "C" int mgt_probe_runs(int mode, const void *src, void *dst, const uint32_t *perm,
                              int64_t n_runs, int32_t run_bytes, mgt_stream_t stream) {
    if (mode < 0 || mode > 3 || n_runs < 0 || n_runs > 0xFFFFFFFFLL) return MGT_EINVAL;
    if (mode != 2 && (run_bytes < 16 || run_bytes % 16 != 0)) return MGT_EINVAL;
    if (mode == 2 && run_bytes < 4) return MGT_EINVAL;
    if (!dst || (mode != 2 && !src) || (mode <= 2 && !perm)) return MGT_EINVAL;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) != 0)
        return MGT_EINVAL;
    if (n_runs == 0) return MGT_OK;
    const long long grid = 4LL * sm_count();
    k_probe_runs<<<(unsigned)grid, PR_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
        mode, static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst), perm, n_runs, run_bytes);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MGT_OK : note_cuda(e, "probe");
}
