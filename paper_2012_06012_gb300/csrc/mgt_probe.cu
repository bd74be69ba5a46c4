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

// mode 4: the gather of mode 0, its loads staged in shared memory with
// cp.async (PR_STAGES stages of PR_UNROLL 16-byte units per thread in
// flight, no registers held by data in flight); each thread stores the units
// it loaded itself, so no barrier is involved.
constexpr int PR_STAGES = 2;
__global__ void __launch_bounds__(PR_THREADS) k_probe_staged(const uint8_t *__restrict__ src,
                                                             uint8_t *__restrict__ dst,
                                                             const uint32_t *__restrict__ perm,
                                                             long long n, int rb) {
    extern __shared__ __align__(16) int4 stage[];  // [PR_STAGES][PR_UNROLL][PR_THREADS]
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int upr = rb / 16;
    const long long units = n * upr;
    const long long step = nthreads * PR_UNROLL;
    long long dofs[PR_STAGES][PR_UNROLL];
    int it = 0;
    for (long long u0 = tid; u0 < units + step * (PR_STAGES - 1); u0 += step, ++it) {
        const int sl = it % PR_STAGES;
        if (u0 < units) {  // issue this iteration's loads
#pragma unroll
            for (int j = 0; j < PR_UNROLL; ++j) {
                const long long u = u0 + j * nthreads;
                dofs[sl][j] = -1;
                if (u < units) {
                    const long long r = u / upr, w = u - r * upr;
                    const long long sr = __ldg(perm + r);
                    const int4 *g = reinterpret_cast<const int4 *>(src + sr * rb) + w;
                    const unsigned sa = (unsigned)__cvta_generic_to_shared(
                        &stage[(sl * PR_UNROLL + j) * PR_THREADS + threadIdx.x]);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
                    dofs[sl][j] = r * rb + w * 16;
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        // the iteration PR_STAGES - 1 back is complete: store its units
        asm volatile("cp.async.wait_group %0;\n" ::"n"(PR_STAGES - 1) : "memory");
        const long long back = u0 - step * (PR_STAGES - 1);
        if (back >= 0 && it >= PR_STAGES - 1) {
            const int sb = (it - (PR_STAGES - 1)) % PR_STAGES;
#pragma unroll
            for (int j = 0; j < PR_UNROLL; ++j)
                if (dofs[sb][j] >= 0)
                    __stcs(reinterpret_cast<int4 *>(dst + dofs[sb][j]),
                           stage[(sb * PR_UNROLL + j) * PR_THREADS + threadIdx.x]);
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// mode 5: the gather of mode 0 through the TMA engine: one thread per CTA
// issues a bulk copy (cp.async.bulk) of each run of a chunk of TMA_RUNS
// output runs into a shared-memory stage, completing on the stage's
// mbarrier, then one bulk store of the whole stage (the chunk's output runs
// are contiguous).  TMA_STAGES stages in flight.  Every wait on an mbarrier
// is bounded: past the limit the kernel counts an error in *err, waits once
// more (bounded) for its copies in flight, and returns.
static __device__ unsigned g_probe_err;  // mode 5: waits that ran out of polls
constexpr int TMA_RUNS = 32;
constexpr int TMA_STAGES = 4;
constexpr long long TMA_POLLS = 1LL << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (long long i = 0; i < TMA_POLLS; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(32) k_probe_tma(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                                  const uint32_t *__restrict__ perm, long long n, int rb,
                                                  unsigned *err) {
    extern __shared__ __align__(128) uint8_t tstage[];  // [TMA_STAGES][TMA_RUNS * rb]
    __shared__ __align__(8) unsigned long long bar[TMA_STAGES];
    if (threadIdx.x == 0) {
        for (int s = 0; s < TMA_STAGES; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar[s])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const long long chunks = (n + TMA_RUNS - 1) / TMA_RUNS;
    const long long sbytes = (long long)TMA_RUNS * rb;
    auto chunk_of = [&](long long k) { return (long long)blockIdx.x + k * gridDim.x; };
    auto runs_in = [&](long long c) { return (int)min((long long)TMA_RUNS, n - c * TMA_RUNS); };
    auto issue_loads = [&](long long k) {
        const long long c = chunk_of(k);
        const int s = (int)(k % TMA_STAGES), nr = runs_in(c);
        const unsigned b = smem_u32(&bar[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n"
                     ::"r"(b), "r"((unsigned)(nr * rb)) : "memory");
        for (int r = 0; r < nr; ++r) {
            const uint8_t *g = src + (long long)__ldg(perm + c * TMA_RUNS + r) * rb;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                ::"r"(smem_u32(tstage + s * sbytes + (long long)r * rb)), "l"(g), "r"((unsigned)rb), "r"(b)
                : "memory");
        }
    };
    long long issued = 0;
    for (; issued < TMA_STAGES - 1 && chunk_of(issued) < chunks; ++issued) issue_loads(issued);
    bool ok = true;
    for (long long k = 0; chunk_of(k) < chunks; ++k) {
        if (issued == k + TMA_STAGES - 1 && chunk_of(issued) < chunks) {
            // the stage of chunk k - 1 gets the next chunk: its store must have read it
            asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
            issue_loads(issued);
            ++issued;
        }
        const int s = (int)(k % TMA_STAGES);
        if (!mbar_wait(smem_u32(&bar[s]), (unsigned)((k / TMA_STAGES) & 1))) {
            atomicAdd(err, 1u);
            ok = false;
            break;
        }
        const long long c = chunk_of(k);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
                     ::"l"(dst + c * sbytes), "r"(smem_u32(tstage + s * sbytes)), "r"((unsigned)(runs_in(c) * rb))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    }
    if (!ok) {  // copies may still be in flight into shared memory: one more bounded wait on each
        for (long long k = issued - (TMA_STAGES - 1); k < issued; ++k)
            if (k >= 0) mbar_wait(smem_u32(&bar[k % TMA_STAGES]), (unsigned)((k / TMA_STAGES) & 1));
    }
    asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

}  // namespace mgt

using namespace mgt;

extern "C" int mgt_probe_runs(int mode, const void *src, void *dst, const uint32_t *perm,
                              int64_t n_runs, int32_t run_bytes, mgt_stream_t stream) {
    if (mode < 0 || mode > 5 || n_runs < 0 || n_runs > 0xFFFFFFFFLL) return MGT_EINVAL;
    if (mode != 2 && (run_bytes < 16 || run_bytes % 16 != 0)) return MGT_EINVAL;
    if (mode == 2 && run_bytes < 4) return MGT_EINVAL;
    if (!dst || (mode != 2 && !src) || ((mode <= 2 || mode >= 4) && !perm)) return MGT_EINVAL;
    if (mode == 5 && run_bytes > 1024) return MGT_EINVAL;  // four stages of 32 runs fit in 128 KB
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) != 0)
        return MGT_EINVAL;
    if (n_runs == 0) return MGT_OK;
    const long long grid = 4LL * sm_count();
    if (mode == 5) {
        unsigned *err = nullptr;  // the device's count of waits that ran out (g_probe_err)
        cudaError_t e = cudaGetSymbolAddress((void **)&err, g_probe_err);
        if (e != cudaSuccess) return note_cuda(e, "probe");
        const size_t smem = (size_t)TMA_STAGES * TMA_RUNS * run_bytes;
        e = cudaFuncSetAttribute(k_probe_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return note_cuda(e, "probe");
        const long long chunks = (n_runs + TMA_RUNS - 1) / TMA_RUNS;
        long long g = 16LL * sm_count();
        if (g > chunks) g = chunks;
        k_probe_tma<<<(unsigned)g, 32, smem, static_cast<cudaStream_t>(stream)>>>(
            static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst), perm, n_runs, run_bytes, err);
    } else if (mode == 4) {
        const size_t smem = (size_t)PR_STAGES * PR_UNROLL * PR_THREADS * 16;
        cudaError_t e = cudaFuncSetAttribute(k_probe_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return note_cuda(e, "probe");
        k_probe_staged<<<(unsigned)grid, PR_THREADS, smem, static_cast<cudaStream_t>(stream)>>>(
            static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst), perm, n_runs, run_bytes);
    } else {
        k_probe_runs<<<(unsigned)grid, PR_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(
            mode, static_cast<const uint8_t *>(src), static_cast<uint8_t *>(dst), perm, n_runs, run_bytes);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MGT_OK : note_cuda(e, "probe");
}

// Waits of the TMA probe (mode 5) that ran out of polls since the library was
// loaded on the current device (0 when every bulk copy completed).
extern "C" int mgt_probe_errors(unsigned *count) {
    if (!count) return MGT_EINVAL;
    const cudaError_t e = cudaMemcpyFromSymbol(count, g_probe_err, sizeof(unsigned));
    return e == cudaSuccess ? MGT_OK : note_cuda(e, "probe errors");
}

// The context's L2 fetch granularity hint (cudaLimitMaxL2FetchGranularity,
// 0-128 bytes): *prev_bytes receives the current value; set_bytes >= 0 sets
// a new one for later launches of this context on the current device.
extern "C" int mgt_l2_fetch_granularity(int32_t set_bytes, int32_t *prev_bytes) {
    if (set_bytes > 128) return MGT_EINVAL;
    size_t v = 0;
    cudaError_t e = cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity);
    if (e != cudaSuccess) return note_cuda(e, "l2 fetch granularity");
    if (prev_bytes) *prev_bytes = (int32_t)v;
    if (set_bytes >= 0) {
        e = cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)set_bytes);
        if (e != cudaSuccess) return note_cuda(e, "l2 fetch granularity");
    }
    return MGT_OK;
}
