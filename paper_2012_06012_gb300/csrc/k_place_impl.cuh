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
template <>
struct VecT<1> {
    using T = unsigned char;
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

// Copies records [0, n) from global to shared memory, four loads in flight
// per thread.
template <typename Rec>
__device__ __forceinline__ void load_records(Rec *dst, const Rec *__restrict__ src, int n) {
    for (int x0 = threadIdx.x; x0 < n; x0 += 4 * P_THREADS) {
        Rec r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (x0 + u * P_THREADS < n) r[u] = src[x0 + u * P_THREADS];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (x0 + u * P_THREADS < n) dst[x0 + u * P_THREADS] = r[u];
    }
}

// Adds 1 and the run length of every valid lane to cnt[c] and vs[c] (c < w):
// one atomic pair per lane when a narrow bucket's columns are spread over
// the warp, one per distinct column otherwise (the hot columns of skewed
// inputs would serialize their lanes on one address).  Lengths of
// 2^16 and more (rare) are added one by one there.
template <typename CT>
__device__ __forceinline__ void warp_count_add(CT *cnt, unsigned long long *vs, uint32_t c,
                                               unsigned long long len, bool valid, int w) {
    // every valid lane on one column (the rounds of a hot column): no match
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (vm == 0) return;
    const int first = __ffs(vm) - 1;
    const uint32_t c0 = __shfl_sync(0xffffffffu, c, first);
    if (__all_sync(0xffffffffu, !valid || c == c0)) {
        const unsigned sum = __reduce_add_sync(0xffffffffu, (valid && len < 65536ull) ? (unsigned)len : 0u);
        if (lane_id() == first) {
            atomicAdd(&cnt[c0], (CT)__popc(vm));
            if (sum) atomicAdd(&vs[c0], (unsigned long long)sum);
        }
        if (valid && len >= 65536ull) atomicAdd(&vs[c0], len);
        return;
    }
    // narrow buckets (w <= 128 columns) whose columns are spread over the
    // warp (at most 4 lanes share the first lane's column, or the first
    // other one): one atomic pair per lane, cheaper than grouping the lanes
    // (measured: 64-column buckets 2.5x faster, 512-column ones slower);
    // otherwise one pair per group of equal columns
    const unsigned same0 = __ballot_sync(0xffffffffu, valid && c == c0);
    if (w <= 128 && __popc(same0) <= 4) {
        const unsigned rest = vm & ~same0;
        const uint32_t c1 = __shfl_sync(0xffffffffu, c, rest ? __ffs(rest) - 1 : first);
        if (__popc(__ballot_sync(0xffffffffu, valid && c == c1)) <= 4) {
            if (valid) {
                atomicAdd(&cnt[c], (CT)1);
                if (len) atomicAdd(&vs[c], len);
            }
            return;
        }
    }
    const unsigned peers = __match_any_sync(0xffffffffu, valid ? c : 0xFFFFFFFFu);
    const unsigned small = (valid && len < 65536ull) ? (unsigned)len : 0u;
    const unsigned sum = __reduce_add_sync(peers, small);  // each group reduces over itself
    if (valid && (peers & lanemask_lt()) == 0) {
        atomicAdd(&cnt[c], (CT)__popc(peers));
        if (sum) atomicAdd(&vs[c], (unsigned long long)sum);
    }
    if (valid && len >= 65536ull) atomicAdd(&vs[c], len);
}

// Ranks of a warp's records [a, e) among equal bins (bin = bin_of(idx)),
// in rounds of 32 records: per-(bin, warp) counters in wc (padded layout,
// see wc_at), each record's rank written to rank_out[idx].  The peer
// matches of four rounds are issued together so that their latencies
// overlap; the counter updates stay in round order (stability).
template <typename BinFn>
__device__ __forceinline__ void warp_rank_pass(int a, int e, int nbins, uint32_t *wc,
                                               uint32_t *rank_out, BinFn bin_of) {
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int base = a; base < e; base += 4 * 32) {
        uint32_t bk[4];
        unsigned pk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * 32 + lane;
            bk[u] = idx < e ? bin_of(idx) : 0xFFFFFFFFu;
            // up to 64 bins: a vote per bin bit beats the hardware match on
            // spread keys (measured; wider buckets keep the match)
            pk[u] = nbins <= 64 ? vote_peers(bk[u], nbins) : __match_any_sync(0xffffffffu, bk[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int idx = base + u * 32 + lane;
            const bool v = idx < e;
            const unsigned lower = pk[u] & lanemask_lt();
            uint32_t before = 0;
            if (v) before = wc[wc_at(bk[u], warp, nbins)];
            __syncwarp();
            if (v && lower == 0) wc[wc_at(bk[u], warp, nbins)] = before + __popc(pk[u]);
            if (v) rank_out[idx] = before + __popc(lower);
            __syncwarp();
        }
    }
}

// In-place exclusive scan of a[0..n) in shared memory with each warp owning
// a contiguous segment read 32 consecutive words at a time (no bank
// conflicts); returns nothing, ends with a barrier.  scratch: >= 33 words.
__device__ __forceinline__ void block_scan_segmented(uint32_t *a, int n, uint32_t *scratch) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int seg = (((n + nw - 1) / nw) + 31) & ~31;
    const int lo = min(n, warp * seg), hi = min(n, lo + seg);
    uint32_t sum = 0;
    for (int x = lo + lane; x < hi; x += 32) sum += a[x];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) scratch[warp] = sum;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < nw ? scratch[lane] : 0u;
        const uint32_t inc = warp_inclusive_scan(v);
        if (lane < nw) scratch[lane] = inc - v;
    }
    __syncthreads();
    uint32_t carry = scratch[warp];
    for (int x0 = lo; x0 < hi; x0 += 32) {
        const int x = x0 + lane;
        const uint32_t v = x < hi ? a[x] : 0u;
        const uint32_t inc = warp_inclusive_scan(v);
        if (x < hi) a[x] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncthreads();
}

// ------------------------------------------------------- K5 chunk hist
// For chunks of buckets too large for one cluster: per-column cell counts
// and value sums of each chunk, into its row of the cursor matrix.
template <typename OffT, typename Rec, bool BATCH>
__global__ void __launch_bounds__(P_THREADS, 2)
    k_chunk_hist(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    Units<BATCH> U(m0, ba, blockIdx.x, gridDim.x);
    while (U.next([](const Mat &X) { return X.ws.hdr->n_multi_items; })) {
    const Mat &M = *U.M;
    const unsigned long long j = U.j;
    const Rec *__restrict__ recs = reinterpret_cast<const Rec *>(M.ws.recs);
    const WorkItem *__restrict__ items = M.ws.items;
    const uint32_t *__restrict__ multi_items = M.ws.multi_items;
    Cursor *__restrict__ mc = M.ws.mc;
    const int bshift = M.p.bshift;
    const void *cell_ptr = M.in.cell_ptr;
    const long long C = M.p.C, V = M.p.V;
    const DevHeader *hdr = M.ws.hdr;
    const int w = 1 << bshift;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem);
    unsigned long long *vs = reinterpret_cast<unsigned long long *>(cnt + w + (w & 1));
    {
        const WorkItem it = items[multi_items[j]];
        if (!MGT_IN(const_cast<DevHeader *>(hdr), it.mc, hdr->max_rows)) continue;
        for (int c = threadIdx.x; c < w; c += blockDim.x) { cnt[c] = 0; vs[c] = 0; }
        __syncthreads();
        // four record loads in flight per thread, then their counts
        constexpr int HU = 4;
        for (unsigned long long r0 = it.r0; r0 < it.r1; r0 += (unsigned long long)HU * blockDim.x) {
            Rec rc[HU];
            bool v[HU];
#pragma unroll
            for (int u = 0; u < HU; ++u) {
                const unsigned long long r = r0 + (unsigned long long)u * blockDim.x + threadIdx.x;
                v[u] = r < it.r1 && MGT_IN(const_cast<DevHeader *>(hdr), r, C);
                if (v[u]) rc[u] = recs[r];
            }
#pragma unroll
            for (int u = 0; u < HU; ++u) {
                uint32_t cl = 0;
                unsigned long long len = 0;
                if (v[u]) {
                    cl = rc[u].meta >> 16;
                    len = rec_len<OffT>(rc[u].meta, rc[u].start, cell_ptr, C, V);
                }
                warp_count_add(cnt, vs, cl, len, v[u], w);
            }
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
}

// ------------------------------------------------------- K6 chunk scan
// Per large bucket: for each column, exclusive prefix over the bucket's
// chunks (in order), then column starts from the column totals; turns the
// cursor rows into absolute (slot, value offset) bases and writes row_ptr'
// for the bucket's columns.  The hottest bucket has thousands of chunks, and
// the kernel lasts as long as its chain of cursor loads: each column's
// chunks are cut into K6_THREADS / w segments, one thread each, with CU
// loads in flight per thread.  Pass 1 sums each segment (reads only); the
// segment sums give every segment its start; pass 2 writes the absolute
// cursors.
constexpr int K6_THREADS = 1024;
__host__ __device__ inline size_t chunk_scan_smem(int bshift) {
    const size_t w = (size_t)1 << bshift;
    const size_t segcols = w < (size_t)K6_THREADS ? (size_t)K6_THREADS : w;  // nseg * w
    return w * 16 + segcols * 16 + 48 * 8;
}
template <typename OffT, bool BATCH>
__global__ void __launch_bounds__(K6_THREADS)
    k_chunk_scan(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    Units<BATCH> U(m0, ba, blockIdx.x, gridDim.x);
    while (U.next([](const Mat &X) { return X.ws.hdr->n_multi_buckets; })) {
    const Mat &M = *U.M;
    const unsigned long long j = U.j;
    const MultiBucket *__restrict__ mbs = M.ws.multi_buckets;
    Cursor *__restrict__ mc = M.ws.mc;
    const int bshift = M.p.bshift;
    const long long N = M.p.N;
    const unsigned long long *__restrict__ bucket_base = M.ws.bucket_base;
    const unsigned long long *__restrict__ bucket_vbase = M.ws.bucket_vbase;
    void *out_row_ptr = M.out.row_ptr;
    const DevHeader *hdr = M.ws.hdr;
    const int w = 1 << bshift;
    const int nseg = w < K6_THREADS ? K6_THREADS / w : 1;
    unsigned long long *tc = reinterpret_cast<unsigned long long *>(smem);
    unsigned long long *tv = tc + w;
    unsigned long long *sc = tv + w;                       // [nseg][w] segment cell sums
    unsigned long long *sv = sc + (size_t)nseg * w;        // [nseg][w] segment value sums
    unsigned long long *scratch = sv + (size_t)nseg * w;   // 33
    {
        const MultiBucket mb = mbs[j];
        if (!MGT_IN(const_cast<DevHeader *>(hdr), mb.mc0 + mb.nch, hdr->max_rows + 1)) continue;
        Cursor *rows = mc + mb.mc0 * (unsigned long long)w;
        constexpr uint32_t CU = 8;
        const int seg = threadIdx.x / (K6_THREADS / nseg);     // segment of this thread
        const int c0t = threadIdx.x % (K6_THREADS / nseg);     // first column of this thread
        const int cstep = K6_THREADS / nseg;
        const uint32_t per = (mb.nch + nseg - 1) / nseg;
        const uint32_t h0 = min(mb.nch, (uint32_t)seg * per), h1 = min(mb.nch, h0 + per);
        // pass 1: sums of this segment's chunks, per column
        for (int c = c0t; c < w; c += cstep) {
            unsigned long long rc = 0, rv = 0;
            for (uint32_t hb = h0; hb < h1; hb += CU) {
                Cursor x[CU];
#pragma unroll
                for (uint32_t u = 0; u < CU; ++u)
                    if (hb + u < h1) x[u] = rows[(unsigned long long)(hb + u) * w + c];
#pragma unroll
                for (uint32_t u = 0; u < CU; ++u)
                    if (hb + u < h1) {
                        rc += x[u].a;
                        rv += x[u].b;
                    }
            }
            sc[(size_t)seg * w + c] = rc;
            sv[(size_t)seg * w + c] = rv;
        }
        __syncthreads();
        // column totals; then column starts
        for (int c = threadIdx.x; c < w; c += K6_THREADS) {
            unsigned long long a = 0, b = 0;
            for (int s2 = 0; s2 < nseg; ++s2) {
                a += sc[(size_t)s2 * w + c];
                b += sv[(size_t)s2 * w + c];
            }
            tc[c] = a;
            tv[c] = b;
        }
        __syncthreads();
        block_exclusive_scan<unsigned long long>(tc, w, scratch);
        block_exclusive_scan<unsigned long long>(tv, w, scratch);
        const unsigned long long bb = bucket_base[mb.bucket], vb = bucket_vbase[mb.bucket];
        const long long cb = (long long)mb.bucket << bshift;
        // pass 2: absolute cursors of this segment's chunks
        for (int c = c0t; c < w; c += cstep) {
            unsigned long long ac = bb + tc[c], av = vb + tv[c];
            for (int s2 = 0; s2 < seg; ++s2) {
                ac += sc[(size_t)s2 * w + c];
                av += sv[(size_t)s2 * w + c];
            }
            if (seg == 0 && cb + c < N) sto<OffT>(out_row_ptr, cb + c, (long long)(bb + tc[c]));
            for (uint32_t hb = h0; hb < h1; hb += CU) {
                Cursor x[CU];
#pragma unroll
                for (uint32_t u = 0; u < CU; ++u)
                    if (hb + u < h1) x[u] = rows[(unsigned long long)(hb + u) * w + c];
#pragma unroll
                for (uint32_t u = 0; u < CU; ++u)
                    if (hb + u < h1) {
                        Cursor y;
                        y.a = ac;
                        y.b = av;
                        rows[(unsigned long long)(hb + u) * w + c] = y;
                        ac += x[u].a;
                        av += x[u].b;
                    }
            }
        }
        __syncthreads();
    }
    }
}

// ------------------------------------------------ shared-memory layouts
constexpr int P_WARPS = P_THREADS / 32;

struct ClLayout {
    size_t in, inv, lpre, wc, cst, ocnt, olen, pub_cnt, pub_len, allc, alll, scratch, misc, total;
};
// per-owner stride of the (owner, round, warp) counters, odd so that one
// warp's leaders for different owners fall on different banks
__host__ __device__ inline int ocnt_stride(int cap) {
    return ((cap + P_THREADS - 1) / P_THREADS) * (P_THREADS / 32) + 1;
}
template <typename Rec, int CS>
__host__ __device__ inline ClLayout cl_layout(int cap, int wsub) {
    ClLayout L;
    size_t o = 0;
    const int rmax = (cap + P_THREADS - 1) / P_THREADS;
#define MGT_TAKE(field, bytes) L.field = o; o = (o + (size_t)(bytes) + 15) & ~size_t(15);
    MGT_TAKE(in, (size_t)cap * sizeof(Rec))
    MGT_TAKE(inv, (size_t)cap * 2)
    MGT_TAKE(lpre, (size_t)(cap + 1) * 4)
    MGT_TAKE(wc, (size_t)(wsub + 1) * P_WARPS * 4)
    MGT_TAKE(cst, (size_t)(wsub + 1) * 4)
    MGT_TAKE(ocnt, (size_t)CS * ocnt_stride(cap) * 4)
    MGT_TAKE(olen, (size_t)CS * 8)
    MGT_TAKE(pub_cnt, (size_t)CS * 4)
    MGT_TAKE(pub_len, (size_t)CS * 8)
    MGT_TAKE(allc, (size_t)CS * CS * 4)
    MGT_TAKE(alll, (size_t)CS * CS * 8)
    MGT_TAKE(scratch, 48 * 8)
    MGT_TAKE(misc, 64)
#undef MGT_TAKE
    L.total = o;
    return L;
}

// ------------------------------------------------------ K7a cluster place
// One thread-block cluster of CS CTAs per bucket (buckets of at most CS x cap
// records).  CTA r owns the bucket's columns [r w/CS, (r+1) w/CS):
//   1. each CTA counts, per owner, the records of its slice of the bucket
//      (slices in input order) and their value totals; cluster barrier;
//   2. from the CS x CS counts every CTA knows where its records go in each
//      owner's buffer; it stores them there through distributed shared
//      memory (stable: slices in order, records in order); cluster barrier;
//   3. each owner sorts its records by column with a one-pass stable
//      multisplit (per-warp counters), writes row_ptr' for its columns and,
//      in output order, col_idx', cell_ptr' and each run's source offset.
// An owner receiving more than cap records is left to K7c (fallback list).
template <typename OffT, typename Rec, int CS, bool BATCH>
__global__ void __launch_bounds__(P_THREADS, 2)
    k_place_cluster(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned rank = 0;
    if constexpr (CS > 1) rank = cg::this_cluster().block_rank();
    // one work item per cluster at a time (same sequence on all its CTAs)
    Units<BATCH> U(m0, ba, blockIdx.x / CS, gridDim.x / CS);
    while (U.next([](const Mat &X) { return X.ws.hdr->n_items; })) {
    const Mat &M = *U.M;
    const unsigned long long j = U.j;
    const Rec *__restrict__ recs = reinterpret_cast<const Rec *>(M.ws.recs);
    const WorkItem *__restrict__ items = M.ws.items;
    const int bshift = M.p.bshift, cap = M.p.cap;
    const long long N = M.p.N, C = M.p.C, V = M.p.V;
    const unsigned long long *__restrict__ bucket_base = M.ws.bucket_base;
    const unsigned long long *__restrict__ bucket_vbase = M.ws.bucket_vbase;
    const void *cell_ptr = M.in.cell_ptr;
    void *out_row_ptr = M.out.row_ptr;
    int32_t *__restrict__ out_col = M.out.col;
    void *out_cell_ptr = M.out.cell_ptr;
    decltype(Rec::start) *__restrict__ src_start = reinterpret_cast<decltype(Rec::start) *>(M.ws.src);
    uint32_t *fallback = M.ws.fallback;
    DevHeader *hdr = M.ws.hdr;
    constexpr int LOGCS = CS == 1 ? 0 : CS == 2 ? 1 : CS == 4 ? 2 : 3;
    const int w = 1 << bshift;
    const int osh = bshift - LOGCS;
    const int wsub = 1 << osh;
    const ClLayout L = cl_layout<Rec, CS>(cap, wsub);
    const int rmax = (cap + P_THREADS - 1) / P_THREADS;
    Rec *IN = reinterpret_cast<Rec *>(smem + L.in);
    uint16_t *inv = reinterpret_cast<uint16_t *>(smem + L.inv);
    uint32_t *lpre = reinterpret_cast<uint32_t *>(smem + L.lpre);
    uint32_t *wc = reinterpret_cast<uint32_t *>(smem + L.wc);
    uint32_t *cst = reinterpret_cast<uint32_t *>(smem + L.cst);
    uint32_t *ocnt = reinterpret_cast<uint32_t *>(smem + L.ocnt);
    unsigned long long *olen = reinterpret_cast<unsigned long long *>(smem + L.olen);
    uint32_t *pub_cnt = reinterpret_cast<uint32_t *>(smem + L.pub_cnt);
    unsigned long long *pub_len = reinterpret_cast<unsigned long long *>(smem + L.pub_len);
    uint32_t *allc = reinterpret_cast<uint32_t *>(smem + L.allc);
    unsigned long long *alll = reinterpret_cast<unsigned long long *>(smem + L.alll);
    unsigned long long *scratch = reinterpret_cast<unsigned long long *>(smem + L.scratch);
    (void)w;
    const int ostr = ocnt_stride(cap);
    const int nocnt = CS * ostr;
    (void)rmax;
    {
        const WorkItem it = items[j];
        if (it.mc != ~0ull) continue;  // chunk of an oversized bucket: K7b
        const unsigned long long n = it.r1 - it.r0;
        uint32_t nin = 0;
        unsigned long long slot0 = bucket_base[it.bucket], vb0 = bucket_vbase[it.bucket];
        if constexpr (CS == 1) {
            // one CTA holds the whole bucket: load it, no ownership exchange
            if (n > (unsigned long long)cap) {
                if (tid == 0) {
                    const unsigned long long fi = atomicAdd(&hdr->n_fallback, 1ull);
                    if (MGT_IN(hdr, fi, hdr->max_items)) fallback[fi] = (uint32_t)j;
                }
                continue;
            }
            nin = (uint32_t)n;
            load_records(IN, recs + it.r0, (int)nin);
        } else {
        const unsigned long long lo = it.r0 + n * rank / CS, hi = it.r0 + n * (rank + 1) / CS;
        const int m = n > (unsigned long long)CS * (unsigned long long)cap ? 0 : (int)(hi - lo);
        for (int x = tid; x < nocnt; x += P_THREADS) ocnt[x] = 0;
        if (tid < CS) olen[tid] = 0;
        __syncthreads();
        // ---- 1. per-owner counts and value totals of my slice (four
        // rounds of loads in flight at a time)
        unsigned long long lsum[CS];
#pragma unroll
        for (int q = 0; q < CS; ++q) lsum[q] = 0;
        for (int k0 = 0; k0 * P_THREADS < m; k0 += 4) {
            Rec r4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = (k0 + u) * P_THREADS + warp * 32 + lane;
                if (idx < m && MGT_IN(hdr, lo + idx, C)) r4[u] = recs[lo + idx];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + u;
                const int idx = k * P_THREADS + warp * 32 + lane;
                const bool v = idx < m;
                uint32_t o = 0;
                if (v) {
                    o = (r4[u].meta >> 16) >> osh;
                    const unsigned long long len = rec_len<OffT>(r4[u].meta, r4[u].start, cell_ptr, C, V);
#pragma unroll
                    for (int q = 0; q < CS; ++q)
                        if ((int)o == q) lsum[q] += len;
                }
                const unsigned peers = digit_peers(o, LOGCS, v);
                if (v && (peers & lanemask_lt()) == 0) ocnt[(int)o * ostr + k * P_WARPS + warp] = __popc(peers);
            }
        }
#pragma unroll
        for (int q = 0; q < CS; ++q) {
            unsigned long long x = lsum[q];
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
            if (lane == 0 && x) atomicAdd(&olen[q], x);
        }
        __syncthreads();
        // owner segment totals, then offsets in (owner, round, warp) order
        if (tid < CS) {
            uint32_t s = 0;
            for (int x = 0; x < ostr; ++x) s += ocnt[tid * ostr + x];
            pub_cnt[tid] = s;
            pub_len[tid] = olen[tid];
        }
        __syncthreads();
        block_exclusive_scan<uint32_t>(ocnt, nocnt, reinterpret_cast<uint32_t *>(scratch));
        if constexpr (CS > 1) cg::this_cluster().sync();  // #1: counts published
        else __syncthreads();
        // ---- 2. all CTAs' counts; shuffle to owners
        if (tid < CS * CS) {
            const int rr = tid / CS, q = tid % CS;
            if constexpr (CS > 1) {
                auto cl = cg::this_cluster();
                allc[tid] = *cl.map_shared_rank(&pub_cnt[q], rr);
                alll[tid] = *cl.map_shared_rank(&pub_len[q], rr);
            } else {
                allc[tid] = pub_cnt[q];
                alll[tid] = pub_len[q];
            }
        }
        __syncthreads();
        bool overflow = n > (unsigned long long)CS * (unsigned long long)cap;  // defensive
#pragma unroll
        for (int q = 0; q < CS; ++q) {
            uint32_t s = 0;
            for (int rr = 0; rr < CS; ++rr) s += allc[rr * CS + q];
            overflow |= s > (uint32_t)cap;
        }
        if (!overflow) {
            for (int k0 = 0; k0 * P_THREADS < m; k0 += 4) {
                Rec r4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int idx = (k0 + u) * P_THREADS + warp * 32 + lane;
                    if (idx < m) r4[u] = recs[lo + idx];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + u;
                    const int idx = k * P_THREADS + warp * 32 + lane;
                    const bool v = idx < m;
                    const uint32_t o = v ? (r4[u].meta >> 16) >> osh : 0u;
                    const unsigned peers = digit_peers(o, LOGCS, v);
                    if (v) {
                        uint32_t before = 0;
                        for (unsigned rr = 0; rr < rank; ++rr) before += allc[rr * CS + o];
                        const uint32_t segstart = ocnt[(int)o * ostr];
                        const uint32_t pos = before + ocnt[(int)o * ostr + k * P_WARPS + warp] - segstart +
                                             __popc(peers & lanemask_lt());
                        if (MGT_IN(hdr, pos, cap) && MGT_IN(hdr, o, CS)) {
                            Rec *dst = cg::this_cluster().map_shared_rank(IN, o);
                            dst[pos] = r4[u];
                        }
                    }
                }
            }
        }
        cg::this_cluster().sync();  // #2: shuffle complete
        if (overflow) {
            if (rank == 0 && tid == 0) {
                const unsigned long long fi = atomicAdd(&hdr->n_fallback, 1ull);
                if (MGT_IN(hdr, fi, hdr->max_items)) fallback[fi] = (uint32_t)j;
            }
            continue;
        }
        for (int q = 0; q < CS; ++q) {
            uint32_t s = 0;
            unsigned long long vs = 0;
            for (int rr = 0; rr < CS; ++rr) { s += allc[rr * CS + q]; vs += alll[rr * CS + q]; }
            if ((unsigned)q < rank) { slot0 += s; vb0 += vs; }
            if ((unsigned)q == rank) nin = s;
        }
        }  // CS > 1
        // ---- 3. my columns: stable multisplit by column, then outputs
        const int seg = ((((int)nin + P_WARPS - 1) / P_WARPS) + 31) & ~31;
        const int a = warp * seg, e = min((int)nin, a + seg);
        for (int x = tid; x < (wsub + 1) * P_WARPS; x += P_THREADS) wc[x] = 0;
        __syncthreads();
        const uint32_t binbase = (uint32_t)rank << osh;
        // ranks among equal columns: one peer match per record, the rank
        // kept in lpre until the lengths need it
        warp_rank_pass(a, e, wsub, wc, lpre,
                       [&](int idx) { return (uint32_t)((IN[idx].meta >> 16) - binbase); });
        __syncthreads();
        wc_scan(wc, wsub, P_WARPS, cst, reinterpret_cast<uint32_t *>(scratch));
        {
            const long long c0 = ((long long)it.bucket << bshift) + binbase;
            for (int bin = tid; bin < wsub; bin += P_THREADS)
                if (c0 + bin < N && MGT_IN(hdr, c0 + bin, N + 1))
                    sto<OffT>(out_row_ptr, c0 + bin, (long long)(slot0 + cst[bin]));
        }
        for (int base = a; base < e; base += 32) {
            const int idx = base + lane;
            if (idx < e) {
                const uint32_t bin = (IN[idx].meta >> 16) - binbase;
                inv[wc[wc_at(bin, warp, wsub)] + lpre[idx]] = (uint16_t)idx;
            }
        }
        __syncthreads();
        // one gather per record in output order: its row and run start go out
        // now, its length to the scan for cell_ptr'
        for (int p = tid; p < (int)nin; p += P_THREADS) {
            const Rec r = IN[inv[p]];
            const unsigned long long q = slot0 + p;
            lpre[p] = (uint32_t)rec_len<OffT>(r.meta, r.start, cell_ptr, C, V);
            if (MGT_IN(hdr, q, C)) {
                out_col[q] = (int32_t)r.i;
                src_start[q] = r.start;
            }
        }
        __syncthreads();
        block_scan_segmented(lpre, (int)nin, reinterpret_cast<uint32_t *>(scratch));
        for (int p = tid; p < (int)nin; p += P_THREADS) {
            const unsigned long long q = slot0 + p;
            if (MGT_IN(hdr, q, C)) sto<OffT>(out_cell_ptr, (long long)q, (long long)(vb0 + lpre[p]));
        }
        __syncthreads();
    }
    }
}

// ------------------------------------------------------ K7b chunk place
// One CTA per chunk of an oversized bucket: stable multisplit of the chunk's
// records by column, then each record goes to its column's cursor (from K6)
// plus its rank among the chunk's records of that column.
struct ChLayout {
    size_t in, inv, lpre, wc, cstart, scratch, total;
};
template <typename Rec>
__host__ __device__ inline ChLayout ch_layout(int chm, int w) {
    ChLayout L;
    size_t o = 0;
#define MGT_TAKE(field, bytes) L.field = o; o = (o + (size_t)(bytes) + 15) & ~size_t(15);
    MGT_TAKE(in, (size_t)chm * sizeof(Rec))
    MGT_TAKE(inv, (size_t)chm * 2)
    MGT_TAKE(lpre, (size_t)(chm + 1) * 4)
    MGT_TAKE(wc, (size_t)(w + 1) * P_WARPS * 4)
    MGT_TAKE(cstart, (size_t)(w + 1) * 4)
    MGT_TAKE(scratch, 48 * 8)
#undef MGT_TAKE
    L.total = o;
    return L;
}

template <typename OffT, typename Rec, bool BATCH>
__global__ void __launch_bounds__(P_THREADS, 1)
    k_place_chunk(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    Units<BATCH> U(m0, ba, blockIdx.x, gridDim.x);
    while (U.next([](const Mat &X) { return X.ws.hdr->n_multi_items; })) {
    const Mat &M = *U.M;
    const unsigned long long jj = U.j;
    const Rec *__restrict__ recs = reinterpret_cast<const Rec *>(M.ws.recs);
    const WorkItem *__restrict__ items = M.ws.items;
    const uint32_t *__restrict__ multi_items = M.ws.multi_items;
    const Cursor *__restrict__ mc = M.ws.mc;
    const int bshift = M.p.bshift, chm = M.p.chm;
    const long long C = M.p.C, V = M.p.V;
    const void *cell_ptr = M.in.cell_ptr;
    int32_t *__restrict__ out_col = M.out.col;
    void *out_cell_ptr = M.out.cell_ptr;
    decltype(Rec::start) *__restrict__ src_start = reinterpret_cast<decltype(Rec::start) *>(M.ws.src);
    const DevHeader *hdr = M.ws.hdr;
    const int w = 1 << bshift;
    const ChLayout L = ch_layout<Rec>(chm, w);
    Rec *IN = reinterpret_cast<Rec *>(smem + L.in);
    uint16_t *inv = reinterpret_cast<uint16_t *>(smem + L.inv);
    uint32_t *lpre = reinterpret_cast<uint32_t *>(smem + L.lpre);
    uint32_t *wc = reinterpret_cast<uint32_t *>(smem + L.wc);
    uint32_t *cstart = reinterpret_cast<uint32_t *>(smem + L.cstart);
    uint32_t *scratch = reinterpret_cast<uint32_t *>(smem + L.scratch);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const WorkItem it = items[multi_items[jj]];
        const int m = (int)(it.r1 - it.r0);
        if (!MGT_IN(const_cast<DevHeader *>(hdr), m, chm + 1) ||
            !MGT_IN(const_cast<DevHeader *>(hdr), it.mc, hdr->max_rows) ||
            !MGT_IN(const_cast<DevHeader *>(hdr), it.r1, C + 1))
            continue;
        load_records(IN, recs + it.r0, m);
        for (int x = tid; x < (w + 1) * P_WARPS; x += P_THREADS) wc[x] = 0;
        __syncthreads();
        const int seg = (((m + P_WARPS - 1) / P_WARPS) + 31) & ~31;
        const int a = warp * seg, e = min(m, a + seg);
        // ranks among equal columns (one peer match per record), kept in lpre
        warp_rank_pass(a, e, w, wc, lpre, [&](int idx) { return (uint32_t)(IN[idx].meta >> 16); });
        __syncthreads();
        wc_scan(wc, w, P_WARPS, cstart, scratch);
        for (int base = a; base < e; base += 32) {
            const int idx = base + lane;
            if (idx < e) inv[wc[wc_at(IN[idx].meta >> 16, warp, w)] + lpre[idx]] = (uint16_t)idx;
        }
        __syncthreads();
        for (int p = tid; p < m; p += P_THREADS) {
            const Rec r = IN[inv[p]];
            lpre[p] = (uint32_t)rec_len<OffT>(r.meta, r.start, cell_ptr, C, V);
        }
        __syncthreads();
        block_scan_segmented(lpre, m, scratch);
        const Cursor *crow = mc + it.mc * (unsigned long long)w;
        for (int p = tid; p < m; p += P_THREADS) {
            const Rec r = IN[inv[p]];
            const uint32_t c = r.meta >> 16;
            const uint32_t cs = cstart[c];
            const Cursor cur = crow[c];
            const unsigned long long q = cur.a + (p - cs);
            if (!MGT_IN(const_cast<DevHeader *>(hdr), q, C)) continue;
            out_col[q] = (int32_t)r.i;
            sto<OffT>(out_cell_ptr, (long long)q, (long long)(cur.b + (lpre[p] - lpre[cs])));
            src_start[q] = r.start;
        }
        __syncthreads();
    }
    }
}

// --------------------------------------------------- K7c fallback place
// One CTA per bucket that overflowed a K7a owner (a few very frequent
// columns): per-column counts and value sums, column starts, then one warp
// deals the records in input order to their columns' cursors.
template <typename OffT, typename Rec, bool BATCH>
__global__ void __launch_bounds__(P_THREADS, 1)
    k_place_fallback(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    Units<BATCH> U(m0, ba, blockIdx.x, gridDim.x);
    while (U.next([](const Mat &X) { return X.ws.hdr->n_fallback; })) {
    const Mat &M = *U.M;
    const unsigned long long jj = U.j;
    const Rec *__restrict__ recs = reinterpret_cast<const Rec *>(M.ws.recs);
    const WorkItem *__restrict__ items = M.ws.items;
    const uint32_t *__restrict__ fallback = M.ws.fallback;
    const int bshift = M.p.bshift;
    const long long N = M.p.N, C = M.p.C, V = M.p.V;
    const unsigned long long *__restrict__ bucket_base = M.ws.bucket_base;
    const unsigned long long *__restrict__ bucket_vbase = M.ws.bucket_vbase;
    const void *cell_ptr = M.in.cell_ptr;
    void *out_row_ptr = M.out.row_ptr;
    int32_t *__restrict__ out_col = M.out.col;
    void *out_cell_ptr = M.out.cell_ptr;
    decltype(Rec::start) *__restrict__ src_start = reinterpret_cast<decltype(Rec::start) *>(M.ws.src);
    const DevHeader *hdr = M.ws.hdr;
    const int w = 1 << bshift;
    unsigned long long *cur = reinterpret_cast<unsigned long long *>(smem);  // [w] slots
    unsigned long long *vcur = cur + w;                                       // [w] values
    unsigned long long *scratch = vcur + w;                                   // [48]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const WorkItem it = items[fallback[jj]];
        if (!MGT_IN(const_cast<DevHeader *>(hdr), it.r1, C + 1)) continue;
        for (int c = tid; c < w; c += P_THREADS) { cur[c] = 0; vcur[c] = 0; }
        __syncthreads();
        for (unsigned long long r0 = it.r0; r0 < it.r1; r0 += P_THREADS) {
            const unsigned long long r = r0 + tid;
            const bool v = r < it.r1;
            uint32_t c = 0;
            unsigned long long len = 0;
            if (v) {
                const Rec rc = recs[r];
                c = rc.meta >> 16;
                len = rec_len<OffT>(rc.meta, rc.start, cell_ptr, C, V);
            }
            warp_count_add(cur, vcur, c, len, v, 1 << bshift);
        }
        __syncthreads();
        block_exclusive_scan<unsigned long long>(cur, w, scratch);
        block_exclusive_scan<unsigned long long>(vcur, w, scratch);
        const unsigned long long bb = bucket_base[it.bucket], vb = bucket_vbase[it.bucket];
        const long long c0 = (long long)it.bucket << bshift;
        for (int c = tid; c < w; c += P_THREADS) {
            cur[c] += bb;
            vcur[c] += vb;
            if (c0 + c < N) sto<OffT>(out_row_ptr, c0 + c, (long long)cur[c]);
        }
        __syncthreads();
        if (warp == 0) {
            for (unsigned long long r0 = it.r0; r0 < it.r1; r0 += 32) {
                const unsigned long long r = r0 + lane;
                const bool v = r < it.r1;
                Rec rc{};
                uint32_t c = 0xFFFFFFFFu;
                unsigned long long len = 0;
                if (v) {
                    rc = recs[r];
                    c = rc.meta >> 16;
                    len = rec_len<OffT>(rc.meta, rc.start, cell_ptr, C, V);
                }
                const unsigned peers = digit_peers(v ? c : 0u, bshift, v);
                const unsigned lower = peers & lanemask_lt();
                unsigned long long pre = 0, tot = 0;
                for (int l = 0; l < 32; ++l) {
                    const unsigned long long x = __shfl_sync(0xffffffffu, len, l);
                    if ((peers >> l) & 1u) {
                        tot += x;
                        if ((lower >> l) & 1u) pre += x;
                    }
                }
                unsigned long long s = 0, vv = 0;
                if (v && lower == 0) {
                    s = cur[c];
                    vv = vcur[c];
                    cur[c] = s + __popc(peers);
                    vcur[c] = vv + tot;
                }
                const int leader = __ffs(peers) - 1;
                s = __shfl_sync(0xffffffffu, s, leader);
                vv = __shfl_sync(0xffffffffu, vv, leader);
                if (v) {
                    const unsigned long long q = s + __popc(lower);
                    if (MGT_IN(const_cast<DevHeader *>(hdr), q, C)) {
                    out_col[q] = (int32_t)rc.i;
                    sto<OffT>(out_cell_ptr, (long long)q, (long long)(vv + pre));
                    src_start[q] = rc.start;
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
    }
}

// ------------------------------------------------------------- K8 copy
constexpr int COPY_UNIT = 256;  // output cells per work unit (8 warp rounds)

// What the value copy reads of one matrix's launch context.
template <typename SrcT>
struct CopyCtx {
    const SrcT *src_start;
    const void *out_cell_ptr;
    long long C, V;
    int stride;
    const uint8_t *in_values;
    uint8_t *out_values;
    DevHeader *hdr;
};
template <typename SrcT>
__device__ __forceinline__ CopyCtx<SrcT> copy_ctx(const Mat &M) {
    return CopyCtx<SrcT>{reinterpret_cast<const SrcT *>(M.ws.src), M.out.cell_ptr, M.p.C, M.p.V, M.p.s,
                         M.in.values, M.out.values, M.ws.hdr};
}

// Every value run, in output order: source offset from src_start, target
// and length from cell_ptr'.  Grid-stride over warps of 32 output cells.
template <typename OffT, typename SrcT, int U, bool BATCH>
__global__ void __launch_bounds__(P_THREADS)
    k_copy_values(const __grid_constant__ Mat m0, const BatchArgs ba) {
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    // units: groups of COPY_UNIT output cells, one warp each, 32 cells per
    // round; none for a matrix whose sort kernels placed nothing (malformed
    // input or an internal limit).  One matrix: warp w takes units w,
    // w + warps, ... (the warps write neighbouring output at any time).  A
    // batch: each warp a contiguous range of the members' units, so that it
    // stays on one member for many units and keeps that member's fields in
    // registers instead of reloading them from the member table per unit.
    Units<BATCH> units(m0, ba, gw, nw);
    if constexpr (BATCH) {
        const unsigned long long per = (ba.uprefix[ba.n] + nw - 1) / nw;
        units.g = (unsigned long long)gw * per;
        units.stride = 1;
        units.end = units.g + per;
    }
    const Mat *cur = nullptr;
    CopyCtx<SrcT> cached{};
    while (units.next([](const Mat &X) {
        return (X.ws.hdr->status & (ST_BADINPUT | ST_OVERFLOW))
                   ? 0ull
                   : (unsigned long long)((X.p.C + COPY_UNIT - 1) / COPY_UNIT);
    })) {
        CopyCtx<SrcT> K;
        if constexpr (BATCH) {
            if (units.M != cur) {
                cur = units.M;
                cached = copy_ctx<SrcT>(*cur);
            }
            K = cached;
        } else {
            K = copy_ctx<SrcT>(*units.M);  // the kernel parameter itself
        }
        const SrcT *__restrict__ src_start = K.src_start;
        const void *__restrict__ out_cell_ptr = K.out_cell_ptr;
        const long long C = K.C, V = K.V;
        const int stride = K.stride;
        const uint8_t *__restrict__ in_values = K.in_values;
        uint8_t *__restrict__ out_values = K.out_values;
        DevHeader *hdr = K.hdr;
        const unsigned long long vbytes = (unsigned long long)V * (unsigned long long)stride;
        const long long qb = (long long)units.j * COPY_UNIT;
        const long long qe = min(C, qb + COPY_UNIT);
        // a round's metadata: cell_ptr'[q] (q <= C; the lane above supplies
        // the run's end, lane 31 loads it) and the run's source offset; the
        // next round's loads are issued before this round's copy
        long long nd0 = 0, ndl = 0;
        unsigned long long nsv = 0;
        auto load_round = [&](long long q0) {
            const long long q = q0 + lane;
            nd0 = q <= C ? ldo<OffT>(out_cell_ptr, q) : 0;
            ndl = (lane == 31 && q < C) ? ldo<OffT>(out_cell_ptr, q + 1) : 0;
            nsv = q < C ? (unsigned long long)__ldcs(src_start + q) : 0ull;
        };
        load_round(qb);
        for (long long q0 = qb; q0 < qe; q0 += 32) {
            const long long d0 = nd0, dl = ndl;
            const unsigned long long sv = nsv;
            if (q0 + 32 < qe) load_round(q0 + 32);
            const long long up = __shfl_down_sync(0xffffffffu, d0, 1);
            const long long d1 = lane == 31 ? dl : up;
            const long long q = q0 + lane;
            unsigned long long so = 0, dd = 0, nb = 0;
            if (q < C) {
                so = sv * (unsigned long long)stride;
                dd = (unsigned long long)d0 * (unsigned long long)stride;
                nb = d1 > d0 ? (unsigned long long)(d1 - d0) * (unsigned long long)stride : 0ull;
                if (d0 < 0 || so > vbytes || nb > vbytes - so || dd > vbytes || nb > vbytes - dd) {
                    atomicOr(&hdr->status, ST_OVERFLOW);  // never happens for consistent outputs
                    nb = 0;
                }
            }
            copy_runs<U>(in_values, out_values, so, dd, nb);
        }
    }
}

// Launch of one level-2 phase for one (offset, record) format; `which`:
// 0 = chunk hist (K5), 1 = chunk scan (K6), 2 = cluster place (K7a),
// 3 = chunk place (K7b), 4 = fallback place (K7c), 5 = value copy (K8).
template <typename OffT, typename Rec>
cudaError_t launch_level2_t(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                            cudaStream_t st, int which);

template <typename OffT, typename Rec, int CS>
static cudaError_t launch_cluster_cs(const Mat &m0, const BatchArgs &ba, long long grid,
                                     size_t smem, cudaStream_t st) {
    auto kern = ba.n ? k_place_cluster<OffT, Rec, CS, true> : k_place_cluster<OffT, Rec, CS, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.gridDim = dim3((unsigned)grid);
    if (CS > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, m0, ba);
}

// Sort clusters of the cluster-place kernel that fit on the GPU at once.
template <typename OffT, typename Rec, int CS>
static long long resident_clusters_cs(size_t smem) {
    auto kern = k_place_cluster<OffT, Rec, CS, false>;  // same limits as the batch variant
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (CS == 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P_THREADS, smem) != cudaSuccess)
            return 0;
        return (long long)per_sm * sm_count();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(P_THREADS);
    cfg.gridDim = dim3(CS);
    cfg.dynamicSmemBytes = smem;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) return 0;
    return n;
}

template <typename OffT, typename Rec>
long long resident_clusters_t(int cs, size_t smem) {
    switch (cs) {
    case 1: return resident_clusters_cs<OffT, Rec, 1>(smem);
    case 2: return resident_clusters_cs<OffT, Rec, 2>(smem);
    case 4: return resident_clusters_cs<OffT, Rec, 4>(smem);
    default: return resident_clusters_cs<OffT, Rec, 8>(smem);
    }
}

template <typename OffT, typename Rec>
cudaError_t launch_level2_t(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                            cudaStream_t st, int which) {
    using SrcT = decltype(Rec::start);
    cudaError_t e = cudaSuccess;
    switch (which) {
    case 0: {
        auto kern = ba.n ? k_chunk_hist<OffT, Rec, true> : k_chunk_hist<OffT, Rec, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)grid, P_THREADS, smem, st>>>(m0, ba);
        break;
    }
    case 1: {
        auto kern = ba.n ? k_chunk_scan<OffT, true> : k_chunk_scan<OffT, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)grid, K6_THREADS, smem, st>>>(m0, ba);
        break;
    }
    case 2:
        switch (m0.p.cs) {
        case 1: e = launch_cluster_cs<OffT, Rec, 1>(m0, ba, grid, smem, st); break;
        case 2: e = launch_cluster_cs<OffT, Rec, 2>(m0, ba, grid, smem, st); break;
        case 4: e = launch_cluster_cs<OffT, Rec, 4>(m0, ba, grid, smem, st); break;
        default: e = launch_cluster_cs<OffT, Rec, 8>(m0, ba, grid, smem, st); break;
        }
        break;
    case 3: {
        auto kern = ba.n ? k_place_chunk<OffT, Rec, true> : k_place_chunk<OffT, Rec, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)grid, P_THREADS, smem, st>>>(m0, ba);
        break;
    }
    case 4: {
        auto kern = ba.n ? k_place_fallback<OffT, Rec, true> : k_place_fallback<OffT, Rec, false>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)grid, P_THREADS, smem, st>>>(m0, ba);
        break;
    }
    default:
        auto kern = m0.p.unroll >= 4 ? (ba.n ? k_copy_values<OffT, SrcT, 4, true> : k_copy_values<OffT, SrcT, 4, false>)
                    : m0.p.unroll == 2 ? (ba.n ? k_copy_values<OffT, SrcT, 2, true> : k_copy_values<OffT, SrcT, 2, false>)
                                       : (ba.n ? k_copy_values<OffT, SrcT, 1, true> : k_copy_values<OffT, SrcT, 1, false>);
        kern<<<(unsigned)grid, P_THREADS, 0, st>>>(m0, ba);
        break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mgt
