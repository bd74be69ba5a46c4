// Value copy for values of individual byte widths: the paper's second
// variation of the exchange (Sec. 2, heterogeneous datatypes across edges,
// one MPI datatype per edge through MPI_Alltoallw).
//
// The cells are placed by the same kernels as for fixed-width values; their
// runs are then moved as byte ranges.  Every output cell q knows the first
// input value of its run (src) and its value count (from cell_ptr'); the
// run's bytes are [val_off[src], val_off[src + len]).  Three kernels:
//   KV1 sizes: the byte size and input byte start of every output cell's
//              run, and per-tile sums
//   KV2 scan:  exclusive prefix of the tile sums (tile byte bases)
//   KV3 copy:  per tile, the cells' byte bases (block scan), the warp-
//              cooperative byte copy of the runs in output order, and the
//              output value offsets, value by value in output order.
#include "k_place_impl.cuh"

namespace mgt {

constexpr int VT_THREADS = 256;
constexpr int VT_WARPS = VT_THREADS / 32;
constexpr int VT_MIN_BLOCKS = 4;  // blocks per SM the copy kernel's registers allow

// Warp-cooperative copy of up to 32 runs (one per lane) whose offsets and
// lengths are multiples of 4 but not necessarily of 16: the work units are
// the 16-byte destination chunks the runs overlap, spread over the lanes,
// A4_U of them in flight per lane.  A chunk inside its run is written with
// one 16-byte store from a 16-, 8- or 4-byte aligned read of the source; the
// partial chunks at a run's ends are written word by word.  No byte outside
// a run is read or written.
constexpr int A4_U = 2;
__device__ __forceinline__ void warp_copy_runs_a4(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                                                  unsigned long long s_off, unsigned long long d_off,
                                                  unsigned long long nbytes) {
    const int lane = lane_id();
    const unsigned long long cfirst = d_off >> 4;
    const unsigned long long units = nbytes ? ((d_off + nbytes + 15) >> 4) - cfirst : 0ull;
    const unsigned long long incl = warp_inclusive_scan(units);
    const unsigned long long excl = incl - units;
    const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
    for (unsigned long long u0 = 0; u0 < total; u0 += 32ull * A4_U) {  // total is warp-uniform
        int4 v[A4_U];
        unsigned long long dst_at[A4_U], src_at[A4_U], part[A4_U];  // part: b1 - b0 of a partial chunk
#pragma unroll
        for (int j = 0; j < A4_U; ++j) {
            const unsigned long long u = u0 + (unsigned long long)(j * 32 + lane);
            int lo = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const unsigned long long x = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                if (x <= u) lo += step;
            }
            const unsigned long long ex = __shfl_sync(0xffffffffu, excl, lo);
            const unsigned long long so = __shfl_sync(0xffffffffu, s_off, lo);
            const unsigned long long dd = __shfl_sync(0xffffffffu, d_off, lo);
            const unsigned long long nb = __shfl_sync(0xffffffffu, nbytes, lo);
            const unsigned long long cf = __shfl_sync(0xffffffffu, cfirst, lo);
            dst_at[j] = 0;
            src_at[j] = 0;
            part[j] = 0;
            if (u < total) {
                const unsigned long long D = (cf + (u - ex)) << 4;
                const unsigned long long b0 = D > dd ? D : dd;
                const unsigned long long b1 = (D + 16 < dd + nb) ? D + 16 : dd + nb;
                dst_at[j] = b0;
                src_at[j] = so + (b0 - dd);
                if (b0 == D && b1 == D + 16) {
                    const uint8_t *sp = src + src_at[j];
                    const uintptr_t sa = reinterpret_cast<uintptr_t>(sp);
                    if ((sa & 15) == 0) {
                        v[j] = __ldcs(reinterpret_cast<const int4 *>(sp));
                    } else if ((sa & 7) == 0) {
                        const int2 a = __ldcs(reinterpret_cast<const int2 *>(sp));
                        const int2 b = __ldcs(reinterpret_cast<const int2 *>(sp) + 1);
                        v[j] = make_int4(a.x, a.y, b.x, b.y);
                    } else {
                        const int *w = reinterpret_cast<const int *>(sp);
                        v[j] = make_int4(__ldcs(w), __ldcs(w + 1), __ldcs(w + 2), __ldcs(w + 3));
                    }
                    part[j] = 16;
                } else {
                    part[j] = b1 - b0;  // 4, 8 or 12 bytes: written below, word by word
                }
            }
        }
#pragma unroll
        for (int j = 0; j < A4_U; ++j) {
            if (part[j] == 16) {
                __stcs(reinterpret_cast<int4 *>(dst + dst_at[j]), v[j]);
            } else {
                for (unsigned long long x = 0; x < part[j]; x += 4)
                    __stcs(reinterpret_cast<int *>(dst + dst_at[j] + x),
                           __ldcs(reinterpret_cast<const int *>(src + src_at[j] + x)));
            }
        }
    }
}

// Copy of up to 32 runs (one per lane) with the widest unit that every
// lane's source offset, destination offset and length allow.
__device__ __forceinline__ void copy_bytes(const uint8_t *src, uint8_t *dst, unsigned long long s_off,
                                           unsigned long long d_off, unsigned long long nbytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src) + s_off;
    const uintptr_t b = reinterpret_cast<uintptr_t>(dst) + d_off;
    const unsigned long long m = (unsigned long long)(a | b) | nbytes;
    if (__all_sync(0xffffffffu, (m & 15) == 0 || nbytes == 0))
        warp_copy_runs<16, 2>(src, dst, s_off, d_off, nbytes);
    else if (__all_sync(0xffffffffu, (m & 3) == 0 || nbytes == 0))
        warp_copy_runs_a4(src, dst, s_off, d_off, nbytes);
    else
        warp_copy_runs<1, 4>(src, dst, s_off, d_off, nbytes);
}

__device__ __forceinline__ bool structure_ok(const DevHeader *hdr) {
    return (*(volatile const unsigned *)&hdr->status & (ST_BADINPUT | ST_OVERFLOW)) == 0;
}

// KV1: vsz[q] = bytes of output cell q's run, vso[q] = its first byte in the
// input values; vblk[t] = sum over tile t.
// Block 0 also checks the end points of val_off and writes the output's.
template <typename OffT, typename SrcT>
__global__ void __launch_bounds__(VT_THREADS) k_var_sizes(const __grid_constant__ Mat m) {
    __shared__ unsigned long long red[VT_WARPS];
    const long long C = m.p.C, V = m.p.V, nb = m.p.nbytes;
    const SrcT *__restrict__ src = reinterpret_cast<const SrcT *>(m.ws.src);
    const void *cp = m.out.cell_ptr;
    const long long *__restrict__ vo = m.in.val_off;
    DevHeader *hdr = m.ws.hdr;
    const bool ok = structure_ok(hdr);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (__ldg(vo) != 0 || __ldg(vo + V) != nb) flag(hdr, ST_BADINPUT);
        m.out.val_off[0] = 0;
        m.out.val_off[V] = nb;
    }
    const long long ntiles = (C + VAR_TILE - 1) / VAR_TILE;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long q0 = t * VAR_TILE, q1 = min(C, q0 + VAR_TILE);
        unsigned long long sum = 0;
        bool bad = false;
        // a thread's VAR_TILE / VT_THREADS cells: their run starts and lengths,
        // then every value-offset load in flight before any is used
        constexpr int PER = VAR_TILE / VT_THREADS;
        long long s0[PER], len[PER], a[PER], b[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const long long q = q0 + threadIdx.x + (long long)k * VT_THREADS;
            s0[k] = 0;
            len[k] = -1;
            if (ok && q < q1) {
                s0[k] = (long long)src[q];
                len[k] = ldo<OffT>(cp, q + 1) - ldo<OffT>(cp, q);
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            a[k] = b[k] = 0;
            const long long q = q0 + threadIdx.x + (long long)k * VT_THREADS;
            if (ok && q < q1) {
                if (s0[k] < 0 || len[k] < 0 || s0[k] + len[k] > V) {
                    bad = true;
                } else {
                    a[k] = __ldg(vo + s0[k]);
                    b[k] = __ldg(vo + s0[k] + len[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const long long q = q0 + threadIdx.x + (long long)k * VT_THREADS;
            if (q >= q1) continue;
            long long sz = 0;
            if (ok && len[k] >= 0) {
                if (a[k] < 0 || b[k] < a[k] || b[k] > nb) bad = true;
                else sz = b[k] - a[k];
            }
            m.ws.vsz[q] = sz;
            m.ws.vso[q] = a[k];  // also for a run of zero-width values: it anchors their offsets
            sum += (unsigned long long)sz;
        }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
        if (__syncthreads_or(bad) && threadIdx.x == 0) flag(hdr, ST_BADINPUT);
        if (threadIdx.x == 0) {
            unsigned long long tot = 0;
            for (int w = 0; w < VT_WARPS; ++w) tot += red[w];
            m.ws.vblk[t] = tot;
        }
        __syncthreads();
    }
}

// KV2: one block, exclusive prefix of the tile sums in place; vblk[ntiles] =
// the total, which must equal n_bytes (every value lies in exactly one run).
__global__ void __launch_bounds__(1024) k_var_scan(const __grid_constant__ Mat m) {
    __shared__ unsigned long long scratch[33];
    const long long n = (m.p.C + VAR_TILE - 1) / VAR_TILE;
    unsigned long long *a = m.ws.vblk;
    const int nt = blockDim.x, tid = threadIdx.x;
    const long long per = (n + nt - 1) / nt, lo = min(n, tid * per), hi = min(n, lo + per);
    unsigned long long sum = 0;
    for (long long i = lo; i < hi; ++i) sum += a[i];
    const unsigned long long incl = warp_inclusive_scan(sum);
    if ((tid & 31) == 31) scratch[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        const unsigned long long v = tid < (nt >> 5) ? scratch[tid] : 0ull;
        const unsigned long long vi = warp_inclusive_scan(v);
        scratch[tid] = vi - v;
        if (tid == 31) scratch[32] = vi;
    }
    __syncthreads();
    unsigned long long run = scratch[tid >> 5] + incl - sum;
    for (long long i = lo; i < hi; ++i) {
        const unsigned long long x = a[i];
        a[i] = run;
        run += x;
    }
    if (tid == 0) {
        a[n] = scratch[32];
        if (structure_ok(m.ws.hdr) && scratch[32] != (unsigned long long)m.p.nbytes)
            flag(m.ws.hdr, ST_BADINPUT);
    }
}

// KV3: per tile of VAR_TILE output cells: byte base of every cell (block
// scan of vsz on the tile's base), then per warp 32 cells at a time: their
// runs' bytes, and the output offset of each of their values.
template <typename OffT, typename SrcT>
__global__ void __launch_bounds__(VT_THREADS, VT_MIN_BLOCKS) k_var_copy(const __grid_constant__ Mat m) {
    __shared__ unsigned long long base[VAR_TILE];
    __shared__ unsigned long long scratch[33];
    DevHeader *hdr = m.ws.hdr;
    if (!structure_ok(hdr)) return;  // malformed input or inconsistent value offsets
    const long long C = m.p.C, V = m.p.V, nb = m.p.nbytes;
    const SrcT *__restrict__ src = reinterpret_cast<const SrcT *>(m.ws.src);
    const void *cp = m.out.cell_ptr;
    const long long *__restrict__ vo = m.in.val_off;
    long long *__restrict__ ovo = m.out.val_off;
    const uint8_t *__restrict__ in_b = m.in.values;
    uint8_t *__restrict__ out_b = m.out.values;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long ntiles = (C + VAR_TILE - 1) / VAR_TILE;
    bool bad = false;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long q0 = t * VAR_TILE;
        const int n = (int)min((long long)VAR_TILE, C - q0);
        for (int i = threadIdx.x; i < n; i += VT_THREADS) base[i] = (unsigned long long)m.ws.vsz[q0 + i];
        __syncthreads();
        block_exclusive_scan<unsigned long long>(base, n, scratch);
        const unsigned long long tb = m.ws.vblk[t];
        // rounds of 32 cells per warp (one per lane): the cell's run, its
        // start in the input bytes and its place in the output bytes
        for (int r0 = warp * 32; r0 < n; r0 += VT_WARPS * 32) {
            const int r = r0 + lane;
            long long s0 = 0, c0 = 0, len = 0, so = 0;
            unsigned long long dd = 0, nbytes = 0;
            if (r < n) {
                const long long q = q0 + r;
                s0 = (long long)src[q];
                c0 = ldo<OffT>(cp, q);
                len = ldo<OffT>(cp, q + 1) - c0;
                dd = tb + base[r];
                nbytes = (unsigned long long)m.ws.vsz[q];
                if (s0 < 0 || len < 0 || s0 + len > V || c0 < 0 || c0 + len > V ||
                    dd + nbytes > (unsigned long long)nb) {
                    bad = true;
                    len = 0;
                    nbytes = 0;
                } else {
                    so = m.ws.vso[q];  // (KV1 read it from val_off)
                    if (so < 0 || (unsigned long long)so + nbytes > (unsigned long long)nb) {
                        bad = true;
                        len = 0;
                        nbytes = 0;
                        so = 0;
                    }
                }
            }
            copy_bytes(in_b, out_b, (unsigned long long)so, dd, nbytes);
            // output value offsets: the lanes' runs' values spread over the warp
            const unsigned long long incl = warp_inclusive_scan((unsigned long long)len);
            const unsigned long long excl = incl - (unsigned long long)len;
            const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
            // (every lane runs every iteration: total is warp-uniform); two
            // value offsets in flight per lane
            constexpr int VO_U = 2;
            for (unsigned long long u0 = 0; u0 < total; u0 += 32ull * VO_U) {
                long long a[VO_U], b[VO_U], at[VO_U], rso[VO_U], rdd[VO_U];
                unsigned long long rnb[VO_U];
                bool in[VO_U];
#pragma unroll
                for (int j = 0; j < VO_U; ++j) {
                    const unsigned long long u = u0 + (unsigned long long)(j * 32 + lane);
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const unsigned long long x = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                        if (x <= u) lo += step;
                    }
                    const unsigned long long ex = __shfl_sync(0xffffffffu, excl, lo);
                    const long long rs0 = __shfl_sync(0xffffffffu, s0, lo);
                    const long long rc0 = __shfl_sync(0xffffffffu, c0, lo);
                    rso[j] = __shfl_sync(0xffffffffu, so, lo);
                    rdd[j] = (long long)__shfl_sync(0xffffffffu, dd, lo);
                    rnb[j] = __shfl_sync(0xffffffffu, nbytes, lo);
                    in[j] = u < total;
                    a[j] = b[j] = at[j] = 0;
                    if (in[j]) {
                        const long long k = (long long)(u - ex);
                        a[j] = __ldg(vo + rs0 + k);
                        b[j] = __ldg(vo + rs0 + k + 1);
                        at[j] = rc0 + k;
                    }
                }
#pragma unroll
                for (int j = 0; j < VO_U; ++j) {
                    if (!in[j]) continue;
                    if (a[j] < rso[j] || b[j] < a[j] || (unsigned long long)(b[j] - rso[j]) > rnb[j]) bad = true;
                    ovo[at[j]] = rdd[j] + (a[j] - rso[j]);
                }
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) flag(hdr, ST_BADINPUT);
}

template <typename OffT, typename SrcT>
static cudaError_t launch_var_t(const Mat &m, cudaStream_t st) {
    const long long ntiles = (m.p.C + VAR_TILE - 1) / VAR_TILE;
    long long g = 8LL * sm_count();
    if (g > ntiles) g = ntiles;
    k_var_sizes<OffT, SrcT><<<(unsigned)(g < 1 ? 1 : g), VT_THREADS, 0, st>>>(m);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_var_scan<<<1, 1024, 0, st>>>(m);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ntiles == 0) return cudaSuccess;
    k_var_copy<OffT, SrcT><<<(unsigned)g, VT_THREADS, 0, st>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_var_copy(const Mat &m, cudaStream_t st) {
    if (m.p.o == 4)
        return m.p.wide ? launch_var_t<int32_t, unsigned long long>(m, st)
                        : launch_var_t<int32_t, uint32_t>(m, st);
    return m.p.wide ? launch_var_t<int64_t, unsigned long long>(m, st)
                    : launch_var_t<int64_t, uint32_t>(m, st);
}

}  // namespace mgt
