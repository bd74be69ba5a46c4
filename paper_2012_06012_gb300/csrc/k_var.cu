// Value copy for values of individual byte widths: the paper's second
// variation of the exchange (Sec. 2, heterogeneous datatypes across edges,
// one MPI datatype per edge through MPI_Alltoallw).
//
// The cells are placed by the same kernels as for fixed-width values; their
// runs are then moved as byte ranges.  Every output cell q knows the first
// input value of its run (src) and its value count (from cell_ptr'); the
// run's bytes are [val_off[src], val_off[src + len]).  One kernel, over tiles
// of VAR_TILE output cells taken in order from a counter:
//   1. each cell's run start and byte size (its val_off end points), the
//      tile's byte offsets (block scan) and byte total;
//   2. the tile's byte base from the tiles before it: a chained scan (each
//      tile publishes its total, then its inclusive prefix, and adds up its
//      predecessors' words until one holds an inclusive prefix -- Merrill and
//      Garland's decoupled look-back); the wait for a predecessor is bounded;
//   3. the warp-cooperative byte copy of the runs in output order, and the
//      output value offsets, value by value in output order.
// A tile only ever waits for tiles taken before it, by CTAs that are
// running and publish their totals without waiting, so the chain always
// completes; a wait that runs out of iterations flags MGT_ETIMEOUT and the
// tile publishes anyway so that no later tile waits on it.
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

// Tile words of the chained scan: flag in the top two bits, bytes below.
constexpr unsigned long long TW_AGG = 1ull << 62;  // the tile's own byte total
constexpr unsigned long long TW_PRE = 2ull << 62;  // its inclusive prefix
constexpr unsigned long long TW_VAL = (1ull << 62) - 1;
constexpr long long LOOKBACK_POLLS = 1LL << 22;    // polls of one predecessor before giving up

template <typename OffT, typename SrcT>
__global__ void __launch_bounds__(VT_THREADS, VT_MIN_BLOCKS) k_var_copy(const __grid_constant__ Mat m) {
    __shared__ unsigned long long base[VAR_TILE];  // run sizes, then tile-relative byte offsets
    __shared__ long long sstart[VAR_TILE];         // each run's first byte in the input values
    __shared__ unsigned long long scratch[33];
    __shared__ long long tile_sh;
    __shared__ unsigned long long tbase_sh;
    __shared__ int stop_sh;
    DevHeader *hdr = m.ws.hdr;
    const long long C = m.p.C, V = m.p.V, nb = m.p.nbytes;
    const SrcT *__restrict__ src = reinterpret_cast<const SrcT *>(m.ws.src);
    const void *cp = m.out.cell_ptr;
    const long long *__restrict__ vo = m.in.val_off;
    long long *__restrict__ ovo = m.out.val_off;
    const uint8_t *__restrict__ in_b = m.in.values;
    uint8_t *__restrict__ out_b = m.out.values;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long ntiles = (C + VAR_TILE - 1) / VAR_TILE;
    unsigned long long *words = m.ws.vblk;          // [ntiles], zeroed before the launch
    unsigned long long *counter = words + ntiles;    // next tile to take, zeroed too
    if (blockIdx.x == 0 && tid == 0) {
        if (__ldg(vo) != 0 || __ldg(vo + V) != nb) flag(hdr, ST_BADINPUT);
        ovo[0] = 0;
        ovo[V] = nb;
    }
    if (!structure_ok(hdr)) return;  // malformed input: the cells were not placed
    bool bad = false;
    for (;;) {
        if (tid == 0) {
            tile_sh = (long long)atomicAdd(counter, 1ull);
            stop_sh = 0;
        }
        __syncthreads();
        const long long t = tile_sh;
        if (t >= ntiles) break;
        const long long q0 = t * VAR_TILE;
        const int n = (int)min((long long)VAR_TILE, C - q0);
        // 1. run starts and sizes: a thread's cells' metadata first, then all
        // its val_off loads in flight
        constexpr int PER = VAR_TILE / VT_THREADS;
        long long s0[PER], len[PER], a[PER], b[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * VT_THREADS;
            s0[k] = 0;
            len[k] = -1;
            if (i < n) {
                s0[k] = (long long)src[q0 + i];
                len[k] = ldo<OffT>(cp, q0 + i + 1) - ldo<OffT>(cp, q0 + i);
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            a[k] = b[k] = 0;
            if (tid + k * VT_THREADS < n) {
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
            const int i = tid + k * VT_THREADS;
            if (i >= n) continue;
            long long sz = 0;
            if (a[k] < 0 || b[k] < a[k] || b[k] > nb) bad = true;
            else sz = b[k] - a[k];
            base[i] = (unsigned long long)sz;
            sstart[i] = a[k];
        }
        __syncthreads();
        const unsigned long long agg = block_exclusive_scan<unsigned long long>(base, n, scratch);
        // 2. the tile's byte base: publish the total, add up the predecessors'
        if (tid == 0) {
            unsigned long long prefix = 0;
            if (t == 0) {
                atomicExch(words, TW_PRE | (agg & TW_VAL));
            } else {
                atomicExch(words + t, TW_AGG | (agg & TW_VAL));
                long long p = t - 1, polls = 0;
                while (p >= 0) {
                    const unsigned long long w = *reinterpret_cast<volatile unsigned long long *>(words + p);
                    if ((w & ~TW_VAL) == 0) {  // not published yet
                        if (++polls > LOOKBACK_POLLS) {
                            flag(hdr, ST_TIMEOUT);
                            stop_sh = 1;
                            break;
                        }
                        __nanosleep(64);
                        continue;
                    }
                    prefix += w & TW_VAL;
                    if (w & TW_PRE) break;
                    --p;
                    polls = 0;
                }
                // published even after a timeout, so that no later tile waits on this one
                atomicExch(words + t, TW_PRE | ((prefix + agg) & TW_VAL));
            }
            if (t == ntiles - 1 && prefix + agg != (unsigned long long)nb && structure_ok(hdr))
                flag(hdr, ST_BADINPUT);  // the runs do not cover the value bytes exactly
            tbase_sh = prefix;
        }
        __syncthreads();
        if (stop_sh) break;
        const unsigned long long tb = tbase_sh;
        // 3. rounds of 32 cells per warp (one per lane): the bytes, then the
        // output value offsets
        for (int r0 = warp * 32; r0 < n; r0 += VT_WARPS * 32) {
            const int r = r0 + lane;
            long long rs0 = 0, c0 = 0, rlen = 0, so = 0;
            unsigned long long dd = 0, nbytes = 0;
            if (r < n) {
                const long long q = q0 + r;
                rs0 = (long long)src[q];
                c0 = ldo<OffT>(cp, q);
                rlen = ldo<OffT>(cp, q + 1) - c0;
                so = sstart[r];
                dd = tb + base[r];
                nbytes = (r + 1 < n ? base[r + 1] : agg) - base[r];
                if (rs0 < 0 || rlen < 0 || rs0 + rlen > V || c0 < 0 || c0 + rlen > V || so < 0 ||
                    (unsigned long long)so + nbytes > (unsigned long long)nb ||
                    dd + nbytes > (unsigned long long)nb) {
                    bad = true;
                    rlen = 0;
                    nbytes = 0;
                    so = 0;
                }
            }
            copy_bytes(in_b, out_b, (unsigned long long)so, dd, nbytes);
            // the lanes' runs' values spread over the warp; total is warp-uniform
            const unsigned long long incl = warp_inclusive_scan((unsigned long long)rlen);
            const unsigned long long excl = incl - (unsigned long long)rlen;
            const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
            constexpr int VO_U = 2;  // value offsets in flight per lane
            for (unsigned long long u0 = 0; u0 < total; u0 += 32ull * VO_U) {
                long long va[VO_U], vb[VO_U], at[VO_U], wso[VO_U], wdd[VO_U];
                unsigned long long wnb[VO_U];
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
                    const long long ws0 = __shfl_sync(0xffffffffu, rs0, lo);
                    const long long wc0 = __shfl_sync(0xffffffffu, c0, lo);
                    wso[j] = __shfl_sync(0xffffffffu, so, lo);
                    wdd[j] = (long long)__shfl_sync(0xffffffffu, dd, lo);
                    wnb[j] = __shfl_sync(0xffffffffu, nbytes, lo);
                    in[j] = u < total;
                    va[j] = vb[j] = at[j] = 0;
                    if (in[j]) {
                        const long long k = (long long)(u - ex);
                        va[j] = __ldg(vo + ws0 + k);
                        vb[j] = __ldg(vo + ws0 + k + 1);
                        at[j] = wc0 + k;
                    }
                }
#pragma unroll
                for (int j = 0; j < VO_U; ++j) {
                    if (!in[j]) continue;
                    if (va[j] < wso[j] || vb[j] < va[j] || (unsigned long long)(vb[j] - wso[j]) > wnb[j]) bad = true;
                    ovo[at[j]] = wdd[j] + (va[j] - wso[j]);
                }
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bad) && tid == 0) flag(hdr, ST_BADINPUT);
}

template <typename OffT, typename SrcT>
static cudaError_t launch_var_t(const Mat &m, cudaStream_t st) {
    const long long ntiles = (m.p.C + VAR_TILE - 1) / VAR_TILE;
    // the chained scan's tile words and tile counter start at zero
    cudaError_t e = cudaMemsetAsync(m.ws.vblk, 0, (size_t)(ntiles + 1) * 8, st);
    if (e != cudaSuccess) return e;
    // every CTA resident at once (VT_MIN_BLOCKS per SM): none waits for a
    // tile held by a CTA that has not started
    long long g = (long long)VT_MIN_BLOCKS * sm_count();
    if (g > ntiles) g = ntiles;
    k_var_copy<OffT, SrcT><<<(unsigned)(g < 1 ? 1 : g), VT_THREADS, 0, st>>>(m);
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
