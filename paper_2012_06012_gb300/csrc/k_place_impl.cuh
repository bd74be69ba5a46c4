// Level 2 of the transpose: per-bucket stable sort by column and output.
//
// A bucket holds the records of w consecutive columns in input order (K3).
// One thread-block cluster takes one bucket chunk: each CTA loads a slice of
// the records into shared memory, sorts it by column (stable radix sort),
// publishes per-column counts and value sums in its shared memory, reads the
// other CTAs' tables through distributed shared memory to place its slice
// after the slices of lower-ranked CTAs, and writes col_idx', cell_ptr' and
// the value runs.  This is the paper's final "row-column ordering" of the
// received cells (Sec. 3, view swap step 2), with source order kept inside
// each output row.
#pragma once
#include "mgt_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace mgt {

constexpr int P_THREADS = 512;

// ------------------------------------------------------------ value copy
template <int VEC>
struct VecT;
template <>
struct VecT<16> {
    using T = int4;
};
template <>
struct VecT<8> {
    using T = int2;
};
template <>
struct VecT<4> {
    using T = int;
};

// Warp-cooperative copy of up to 32 runs (one per lane: source byte offset,
// destination byte offset, byte count), VEC bytes per access, spreading the
// concatenated units of all runs over the lanes so long and short runs
// load-balance.  U independent loads are in flight per lane.
template <int VEC, int U>
__device__ __forceinline__ void warp_copy_runs(const uint8_t *__restrict__ src,
                                               uint8_t *__restrict__ dst,
                                               unsigned long long s_off,
                                               unsigned long long d_off,
                                               unsigned long long nbytes) {
    using V = typename VecT<VEC>::T;
    const int lane = lane_id();
    const unsigned long long units = nbytes / VEC;
    const unsigned long long incl = warp_inclusive_scan(units);
    const unsigned long long excl = incl - units;
    const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
    for (unsigned long long u0 = 0; u0 < total; u0 += 32ull * U) {
        V v[U];
        unsigned long long dpos[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const unsigned long long u = u0 + (unsigned long long)(j * 32 + lane);
            int lo = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                unsigned long long x = __shfl_sync(0xffffffffu, incl, lo + step - 1);
                if (x <= u) lo += step;
            }
            const unsigned long long ex = __shfl_sync(0xffffffffu, excl, lo);
            const unsigned long long so = __shfl_sync(0xffffffffu, s_off, lo);
            const unsigned long long dd = __shfl_sync(0xffffffffu, d_off, lo);
            const unsigned long long off = (u - ex) * VEC;
            dpos[j] = dd + off;
            if (u < total) v[j] = __ldcs(reinterpret_cast<const V *>(src + so + off));
        }
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const unsigned long long u = u0 + (unsigned long long)(j * 32 + lane);
            if (u < total) __stcs(reinterpret_cast<V *>(dst + dpos[j]), v[j]);
        }
    }
}

template <int U>
__device__ __forceinline__ void copy_runs(const uint8_t *src, uint8_t *dst, unsigned long long s_off,
                                          unsigned long long d_off, unsigned long long nbytes) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src) + s_off;
    const uintptr_t b = reinterpret_cast<uintptr_t>(dst) + d_off;
    const unsigned long long m = (unsigned long long)(a | b) | nbytes;
    if (__all_sync(0xffffffffu, (m & 15) == 0 || nbytes == 0))
        warp_copy_runs<16, U>(src, dst, s_off, d_off, nbytes);
    else if (__all_sync(0xffffffffu, (m & 7) == 0 || nbytes == 0))
        warp_copy_runs<8, U>(src, dst, s_off, d_off, nbytes);
    else
        warp_copy_runs<4, U>(src, dst, s_off, d_off, nbytes);
}

// ------------------------------------------------------- K5 chunk hist
// For chunks of buckets too large for one cluster: per-column cell counts
// and value sums of each chunk, into its row of the cursor matrix.
template <typename OffT, typename Rec>
__global__ void __launch_bounds__(P_THREADS)
    k_chunk_hist(const Rec *__restrict__ recs, const WorkItem *__restrict__ items,
                 const uint32_t *__restrict__ multi_items, Cursor *__restrict__ mc, int bshift,
                 const void *cell_ptr, long long C, long long V, const DevHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = 1 << bshift;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);
    unsigned long long *vs = reinterpret_cast<unsigned long long *>(cnt + w + (w & 1));
    const unsigned long long nmi = hdr->n_multi_items;
    for (unsigned long long j = blockIdx.x; j < nmi; j += gridDim.x) {
        const WorkItem it = items[multi_items[j]];
        for (int c = threadIdx.x; c < w; c += blockDim.x) { cnt[c] = 0; vs[c] = 0; }
        __syncthreads();
        for (unsigned long long r = it.r0 + threadIdx.x; r < it.r1; r += blockDim.x) {
            const Rec rc = recs[r];
            const uint32_t cl = rc.meta >> 16;
            atomicAdd(&cnt[cl], 1u);
            atomicAdd(&vs[cl], rec_len<OffT>(rc.meta, rc.start, cell_ptr, C, V));
        }
        __syncthreads();
        Cursor *row = mc + it.mc * (unsigned long long)w;
        for (int c = threadIdx.x; c < w; c += blockDim.x) {
            Cursor x;
            x.a = cnt[c];
            x.b = vs[c];
            row[c] = x;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- K6 chunk scan
// Per large bucket: for each column, exclusive prefix over the bucket's
// chunks (in order), then column starts from the column totals; turns the
// cursor rows into absolute (slot, value offset) bases and writes row_ptr'
// for the bucket's columns.
template <typename OffT>
__global__ void __launch_bounds__(P_THREADS)
    k_chunk_scan(const MultiBucket *__restrict__ mbs, Cursor *__restrict__ mc, int bshift,
                 long long N, const unsigned long long *__restrict__ bucket_base,
                 const unsigned long long *__restrict__ bucket_vbase, void *out_row_ptr,
                 const DevHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = 1 << bshift;
    unsigned long long *tc = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *tv = tc + w;
    unsigned long long *scratch = tv + w;  // 33
    const unsigned long long nmb = hdr->n_multi_buckets;
    for (unsigned long long j = blockIdx.x; j < nmb; j += gridDim.x) {
        const MultiBucket mb = mbs[j];
        Cursor *rows = mc + mb.mc0 * (unsigned long long)w;
        for (int c = threadIdx.x; c < w; c += blockDim.x) {
            unsigned long long rc = 0, rv = 0;
            for (uint32_t h = 0; h < mb.nch; ++h) {
                Cursor x = rows[(unsigned long long)h * w + c];
                Cursor y;
                y.a = rc;
                y.b = rv;
                rows[(unsigned long long)h * w + c] = y;
                rc += x.a;
                rv += x.b;
            }
            tc[c] = rc;
            tv[c] = rv;
        }
        __syncthreads();
        block_exclusive_scan<unsigned long long>(tc, w, scratch);
        block_exclusive_scan<unsigned long long>(tv, w, scratch);
        const unsigned long long bb = bucket_base[mb.bucket], vb = bucket_vbase[mb.bucket];
        const long long c0 = (long long)mb.bucket << bshift;
        for (int c = threadIdx.x; c < w; c += blockDim.x) {
            if (c0 + c < N) sto<OffT>(out_row_ptr, c0 + c, (long long)(bb + tc[c]));
            for (uint32_t h = 0; h < mb.nch; ++h) {
                Cursor x = rows[(unsigned long long)h * w + c];
                x.a += bb + tc[c];
                x.b += vb + tv[c];
                rows[(unsigned long long)h * w + c] = x;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- K7 place
struct PlaceSmem {
    size_t recs, k0, k1, A, Bv, lstart, befc, befv, sbase, vbase, whist, scratch, misc, total;
};
template <typename Rec>
__host__ __device__ inline PlaceSmem place_layout(int cap, int w) {
    PlaceSmem L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = (o + bytes + 15) & ~size_t(15);
        return r;
    };
    L.recs = take((size_t)cap * sizeof(Rec));
    L.k0 = take((size_t)(cap + 1) * 4);
    L.k1 = take((size_t)(cap + 1) * 4);
    L.A = take((size_t)w * 4);
    L.Bv = take((size_t)w * 8);
    L.lstart = take((size_t)w * 4);
    L.befc = take((size_t)w * 4);
    L.befv = take((size_t)w * 8);
    L.sbase = take((size_t)w * 8);
    L.vbase = take((size_t)w * 8);
    L.whist = take((size_t)64 * (P_THREADS / 32) * 4);
    L.scratch = take(48 * 8);
    L.misc = take(64);
    L.total = o;
    return L;
}

template <typename OffT, typename Rec, int CS, int U>
__global__ void __launch_bounds__(P_THREADS, 1)
    k_place(const Rec *__restrict__ recs, const WorkItem *__restrict__ items,
            const Cursor *__restrict__ mc, int bshift, int cap, long long N, long long C,
            long long V, int stride, const unsigned long long *__restrict__ bucket_base,
            const unsigned long long *__restrict__ bucket_vbase, const void *__restrict__ cell_ptr,
            const uint8_t *__restrict__ in_values, void *out_row_ptr, int32_t *__restrict__ out_col,
            void *out_cell_ptr, uint8_t *__restrict__ out_values, DevHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = 1 << bshift;
    const PlaceSmem L = place_layout<Rec>(cap, w);
    Rec *srec = reinterpret_cast<Rec *>(smem + L.recs);
    uint32_t *k0 = reinterpret_cast<uint32_t *>(smem + L.k0);
    uint32_t *k1 = reinterpret_cast<uint32_t *>(smem + L.k1);
    uint32_t *A = reinterpret_cast<uint32_t *>(smem + L.A);
    unsigned long long *Bv = reinterpret_cast<unsigned long long *>(smem + L.Bv);
    uint32_t *lstart = reinterpret_cast<uint32_t *>(smem + L.lstart);
    uint32_t *befc = reinterpret_cast<uint32_t *>(smem + L.befc);
    unsigned long long *befv = reinterpret_cast<unsigned long long *>(smem + L.befv);
    long long *sbase = reinterpret_cast<long long *>(smem + L.sbase);
    long long *vbase = reinterpret_cast<long long *>(smem + L.vbase);
    uint32_t *whist = reinterpret_cast<uint32_t *>(smem + L.whist);
    unsigned long long *scratch = reinterpret_cast<unsigned long long *>(smem + L.scratch);
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(smem + L.misc);

    const int tid = threadIdx.x, nt = blockDim.x;
    const int ib = 32 - __clz(cap - 1);  // bits of a slot index
    unsigned rank = 0;
    if constexpr (CS > 1) rank = cg::this_cluster().block_rank();
    const unsigned long long n_items = hdr->n_items;

    for (;;) {
        if (rank == 0 && tid == 0) misc[0] = atomicAdd(&hdr->item_counter, 1ull);
        unsigned long long j;
        if constexpr (CS > 1) {
            cg::this_cluster().sync();
            j = *cg::this_cluster().map_shared_rank(&misc[0], 0);
            cg::this_cluster().sync();
        } else {
            __syncthreads();
            j = misc[0];
            __syncthreads();
        }
        if (j >= n_items) break;
        const WorkItem it = items[j];
        const unsigned long long n = it.r1 - it.r0;
        const unsigned long long lo = it.r0 + n * rank / CS, hi = it.r0 + n * (rank + 1) / CS;
        const int m = (int)(hi - lo);
        const bool multi = it.mc != ~0ull;

        // load the slice (word-granular, coalesced) and build sort keys
        {
            constexpr int W = sizeof(Rec) / 4;
            const uint32_t *g = reinterpret_cast<const uint32_t *>(recs + lo);
            uint32_t *s = reinterpret_cast<uint32_t *>(srec);
            for (int x = tid; x < m * W; x += nt) s[x] = __ldcs(g + x);
        }
        for (int c = tid; c < w; c += nt) { A[c] = 0; Bv[c] = 0; }
        __syncthreads();
        for (int x = tid; x < m; x += nt) k0[x] = ((srec[x].meta >> 16) << ib) | (uint32_t)x;
        __syncthreads();
        uint32_t *sorted = bshift > 0 ? block_radix_sort<6>(k0, k1, m, ib, bshift, whist,
                                                              reinterpret_cast<uint32_t *>(scratch))
                                      : k0;
        uint32_t *lpre = sorted == k0 ? k1 : k0;
        const uint32_t imask = (1u << ib) - 1;
        // run lengths in sorted order -> exclusive prefix (per slice, < 2^32)
        bool ovf = false;
        for (int p = tid; p < m; p += nt) {
            const Rec r = srec[sorted[p] & imask];
            unsigned long long len = rec_len<OffT>(r.meta, r.start, cell_ptr, C, V);
            if (len > 0xFFFFFFFFull) ovf = true;
            lpre[p] = (uint32_t)len;
        }
        if (tid == 0) lpre[m] = 0;
        __syncthreads();
        {
            uint32_t tot = block_exclusive_scan<uint32_t>(lpre, m, reinterpret_cast<uint32_t *>(scratch));
            if (tid == 0) lpre[m] = tot;
        }
        // per-column local runs
        for (int p = tid; p < m; p += nt) {
            const uint32_t c = sorted[p] >> ib;
            if (p == 0 || (sorted[p - 1] >> ib) != c) lstart[c] = (uint32_t)p;
        }
        __syncthreads();
        for (int p = tid; p < m; p += nt) {
            const uint32_t c = sorted[p] >> ib;
            if (p == m - 1 || (sorted[p + 1] >> ib) != c) {
                A[c] = (uint32_t)(p + 1) - lstart[c];
                Bv[c] = (unsigned long long)lpre[p + 1] - lpre[lstart[c]];
            }
        }
        if constexpr (CS > 1) cg::this_cluster().sync();
        else __syncthreads();
        // cross-CTA placement: counts and value sums of lower-ranked slices
        for (int c = tid; c < w; c += nt) {
            unsigned long long bc = 0, bv = 0, tcn = A[c], tvv = Bv[c];
            if constexpr (CS > 1) {
                tcn = 0;
                tvv = 0;
                auto cl = cg::this_cluster();
#pragma unroll
                for (int r = 0; r < CS; ++r) {
                    const uint32_t a = *cl.map_shared_rank(&A[c], r);
                    const unsigned long long v = *cl.map_shared_rank(&Bv[c], r);
                    if ((unsigned)r < rank) { bc += a; bv += v; }
                    tcn += a;
                    tvv += v;
                }
            }
            befc[c] = (uint32_t)bc;
            befv[c] = bv;
            sbase[c] = (long long)tcn;
            vbase[c] = (long long)tvv;
        }
        __syncthreads();
        const unsigned long long bb = bucket_base[it.bucket], vb = bucket_vbase[it.bucket];
        const long long c0 = (long long)it.bucket << bshift;
        if (!multi) {
            block_exclusive_scan<unsigned long long>(reinterpret_cast<unsigned long long *>(sbase), w,
                                                     scratch);
            block_exclusive_scan<unsigned long long>(reinterpret_cast<unsigned long long *>(vbase), w,
                                                     scratch);
            if (rank == 0)
                for (int c = tid; c < w; c += nt)
                    if (c0 + c < N) sto<OffT>(out_row_ptr, c0 + c, (long long)bb + sbase[c]);
        }
        __syncthreads();
        const Cursor *crow = multi ? mc + it.mc * (unsigned long long)w : nullptr;
        for (int c = tid; c < w; c += nt) {
            long long sb, vv;
            if (multi) {
                const Cursor x = crow[c];
                sb = (long long)x.a;
                vv = (long long)x.b;
            } else {
                sb = (long long)bb + sbase[c];
                vv = (long long)vb + vbase[c];
            }
            const uint32_t ls = A[c] ? lstart[c] : 0u;
            sbase[c] = sb + (long long)befc[c] - (long long)ls;
            vbase[c] = vv + (long long)befv[c] - (long long)(A[c] ? lpre[ls] : 0u);
        }
        if constexpr (CS > 1) cg::this_cluster().sync();  // remote reads of A, Bv done
        else __syncthreads();
        if (__syncthreads_or(ovf)) {
            if (tid == 0) flag(hdr, ST_OVERFLOW);
            continue;
        }
        // outputs: col_idx', cell_ptr' and the value runs
        for (int p = tid; p < m; p += nt) {
            const uint32_t key = sorted[p];
            const Rec r = srec[key & imask];
            const uint32_t c = key >> ib;
            const long long slot = sbase[c] + p;
            out_col[slot] = (int32_t)r.i;
            sto<OffT>(out_cell_ptr, slot, vbase[c] + (long long)lpre[p]);
        }
        const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
        for (int p0 = warp * 32; p0 < m; p0 += nw * 32) {
            const int p = p0 + lane;
            unsigned long long so = 0, dd = 0, nb = 0;
            if (p < m) {
                const uint32_t key = sorted[p];
                const Rec r = srec[key & imask];
                const uint32_t c = key >> ib;
                const unsigned long long len = (unsigned long long)lpre[p + 1] - lpre[p];
                so = (unsigned long long)r.start * (unsigned long long)stride;
                dd = (unsigned long long)(vbase[c] + (long long)lpre[p]) * (unsigned long long)stride;
                nb = len * (unsigned long long)stride;
            }
            copy_runs<U>(in_values, out_values, so, dd, nb);
        }
        __syncthreads();
    }
    if constexpr (CS > 1) cg::this_cluster().sync();
}

template <typename OffT, typename Rec, int CS, int U>
cudaError_t launch_place_t(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                                  cudaStream_t st) {
    const int w = 1 << p.bshift;
    const size_t smem = place_layout<Rec>(p.cap, w).total;
    auto kern = k_place<OffT, Rec, CS, U>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    int nclusters = 0;
    if (CS > 1) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(CS);
        e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
        if (e != cudaSuccess) return e;
    } else {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P_THREADS, smem);
        if (e != cudaSuccess) return e;
        nclusters = per_sm * sm_count();
    }
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    long long want = p.max_items;
    if (want < nclusters) nclusters = (int)(want < 1 ? 1 : want);
    cfg.gridDim = dim3((unsigned)(nclusters * CS));
    e = cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<const Rec *>(ws.recs),
                           (const WorkItem *)ws.items, (const Cursor *)ws.mc, p.bshift, p.cap, p.N,
                           p.C, p.V, p.s, (const unsigned long long *)ws.bucket_base,
                           (const unsigned long long *)ws.bucket_vbase, in.cell_ptr, in.values,
                           out.row_ptr, out.col, out.cell_ptr, out.values, ws.hdr);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}


template <typename OffT, typename Rec>
cudaError_t launch_place_cs(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                            cudaStream_t st);

}  // namespace mgt
