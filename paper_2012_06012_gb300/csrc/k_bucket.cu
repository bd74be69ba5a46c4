// Level 1 of the transpose: stable scatter of cell records into column buckets.
//
// The paper exchanges cells between ranks by destination (Sec. 3, view swap:
// metadata, then values).  On one GPU the destination of a cell is a bucket of
// consecutive output rows (= input columns); K1-K3 deal every cell's record
// into its bucket, keeping row-major input order inside each bucket, so that
// the per-bucket sort of K7 only has to order by column.
#include "mgt_internal.cuh"

#include <cooperative_groups.h>

namespace mgt {

constexpr int K_THREADS = 512;

// ------------------------------------------------------------------ K0 prep
// Checks the pointer arrays' end points and that row_ptr never decreases;
// writes the source blocks' cell offsets pcoff[s] = row_ptr[off[s]], the
// output sentinels row_ptr'[N] = C and cell_ptr'[C] = V, and the P = 1 counts.
template <typename OffT>
__global__ void k_prep(const void *row_ptr, const void *cell_ptr, long long R, long long N,
                       long long C, long long V, int P, const long long *poff, long long *pcoff,
                       void *out_row_ptr, void *out_cell_ptr, long long *part_cells,
                       long long *part_values, DevHeader *hdr) {
    long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    if (gid == 0) {
        if (ldo<OffT>(row_ptr, 0) != 0 || ldo<OffT>(row_ptr, R) != C) flag(hdr, ST_BADINPUT);
        if (ldo<OffT>(cell_ptr, 0) != 0 || ldo<OffT>(cell_ptr, C) != V) flag(hdr, ST_BADINPUT);
        sto<OffT>(out_row_ptr, N, C);
        sto<OffT>(out_cell_ptr, C, V);
        if (P == 1 && part_cells) part_cells[0] = C;
        if (P == 1 && part_values) part_values[0] = V;
    }
    for (long long s = gid; s <= P; s += stride) {
        long long r = poff[s];
        pcoff[s] = (r >= 0 && r <= R) ? ldo<OffT>(row_ptr, r) : 0;
    }
    bool bad = false;
    for (long long i = gid; i < R; i += stride)
        bad |= ldo<OffT>(row_ptr, i + 1) < ldo<OffT>(row_ptr, i);
    if (__syncthreads_or(bad) && threadIdx.x == 0) flag(hdr, ST_BADINPUT);
}

cudaError_t launch_prep(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                        cudaStream_t st) {
    int sms = sm_count();
    long long want = (p.R + K_THREADS - 1) / K_THREADS;
    int grid = (int)(want < 1 ? 1 : (want > 2LL * sms ? 2LL * sms : want));
    if (p.o == 4)
        k_prep<int32_t><<<grid, K_THREADS, 0, st>>>(in.row_ptr, in.cell_ptr, p.R, p.N, p.C, p.V,
                                                     p.P, ws.poff, ws.pcoff, out.row_ptr,
                                                     out.cell_ptr, out.part_cells,
                                                     out.part_values, ws.hdr);
    else
        k_prep<int64_t><<<grid, K_THREADS, 0, st>>>(in.row_ptr, in.cell_ptr, p.R, p.N, p.C, p.V,
                                                     p.P, ws.poff, ws.pcoff, out.row_ptr,
                                                     out.cell_ptr, out.part_cells,
                                                     out.part_values, ws.hdr);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K1 hist
// Cells per bucket for one tile of `tile` consecutive cells, in a shared
// memory histogram; written as row t of the T x B count matrix.
__global__ void k_hist(const int32_t *__restrict__ col, long long C, long long N, int bshift,
                       int B, int tile, uint32_t *__restrict__ cnt, DevHeader *hdr) {
    extern __shared__ uint32_t hist[];
    const long long t = blockIdx.x;
    for (int b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const long long k0 = t * (long long)tile;
    const long long k1 = min(C, k0 + tile);
    bool bad = false;
    const bool vec = ((reinterpret_cast<uintptr_t>(col) & 15) == 0);
    if (vec) {
        long long q0 = k0 >> 2, q1 = k1 >> 2;  // tile is a multiple of 4
        const int4 *c4 = reinterpret_cast<const int4 *>(col);
        for (long long q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            int4 v = __ldcs(c4 + q);
            int cs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                long long c = cs[u];
                if (c < 0 || c >= N) { bad = true; c = c < 0 ? 0 : N - 1; }
                atomicAdd(&hist[c >> bshift], 1u);
            }
        }
        for (long long k = (q1 << 2) + threadIdx.x; k < k1; k += blockDim.x) {
            long long c = __ldcs(col + k);
            if (c < 0 || c >= N) { bad = true; c = c < 0 ? 0 : N - 1; }
            atomicAdd(&hist[c >> bshift], 1u);
        }
    } else {
        for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            long long c = __ldcs(col + k);
            if (c < 0 || c >= N) { bad = true; c = c < 0 ? 0 : N - 1; }
            atomicAdd(&hist[c >> bshift], 1u);
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) flag(hdr, ST_BADINPUT);
    uint32_t *row = cnt + t * (long long)B;
    for (int b = threadIdx.x; b < B; b += blockDim.x) row[b] = hist[b];
}

cudaError_t launch_hist(const Params &p, const Inputs &in, const Ws &ws, cudaStream_t st) {
    if (p.T == 0) return cudaSuccess;
    size_t smem = (size_t)p.B * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_hist<<<(unsigned)p.T, K_THREADS, smem, st>>>(in.col, p.C, p.N, p.bshift, (int)p.B, p.tile,
                                                   ws.cnt, ws.hdr);
    return cudaGetLastError();
}

// ------------------------------------------------------------ K2 scan tiles
// For 32 buckets per block: replace cnt[t][b] by the exclusive prefix over
// tiles t' < t (keeps tiles, hence input order, inside each bucket) and
// write the bucket totals.
__global__ void k_scan_tiles(uint32_t *cnt, long long T, long long B,
                             unsigned long long *bucket_tot) {
    __shared__ unsigned long long part[32][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long b = blockIdx.x * 32LL + lane;
    const long long t0 = T * warp / nw, t1 = T * (warp + 1) / nw;
    unsigned long long sum = 0;
    if (b < B)
        for (long long t = t0; t < t1; ++t) sum += cnt[t * B + b];
    part[warp][lane] = sum;
    __syncthreads();
    if (warp == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < nw; ++w) {
            unsigned long long v = part[w][lane];
            part[w][lane] = run;
            run += v;
        }
        if (b < B) bucket_tot[b] = run;
    }
    __syncthreads();
    if (b < B) {
        unsigned long long run = part[warp][lane];
        for (long long t = t0; t < t1; ++t) {
            uint32_t v = cnt[t * B + b];
            cnt[t * B + b] = (uint32_t)run;  // within-bucket offset (< 2^32 by plan)
            run += v;
        }
    }
}

cudaError_t launch_scan_tiles(const Params &p, const Ws &ws, cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    if (p.T == 0) {
        return cudaMemsetAsync(ws.bucket_tot, 0, (size_t)p.B * 8, st);
    }
    k_scan_tiles<<<(unsigned)((p.B + 31) / 32), 256, 0, st>>>(ws.cnt, p.T, p.B, ws.bucket_tot);
    return cudaGetLastError();
}

// ---------------------------------------------------------- K2b scan buckets
// One block: exclusive prefix of 64-bit per-bucket totals (in == out allowed).
__global__ void k_scan_u64(const unsigned long long *in, unsigned long long *out, long long n) {
    __shared__ unsigned long long scratch[33];
    const int nt = blockDim.x, tid = threadIdx.x;
    long long per = (n + nt - 1) / nt, lo = min(n, tid * per), hi = min(n, lo + per);
    unsigned long long sum = 0;
    for (long long i = lo; i < hi; ++i) sum += in[i];
    unsigned long long incl = warp_inclusive_scan(sum);
    if ((tid & 31) == 31) scratch[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        unsigned long long v = tid < (nt >> 5) ? scratch[tid] : 0ull;
        unsigned long long vi = warp_inclusive_scan(v);
        scratch[tid] = vi - v;
    }
    __syncthreads();
    unsigned long long run = scratch[tid >> 5] + incl - sum;
    for (long long i = lo; i < hi; ++i) {
        unsigned long long x = in[i];
        out[i] = run;
        run += x;
    }
}

cudaError_t launch_scan_buckets(const Params &p, const Ws &ws, cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    k_scan_u64<<<1, 1024, 0, st>>>(ws.bucket_tot, ws.bucket_base, p.B);
    return cudaGetLastError();
}

// --------------------------------------------------------------- K3 scatter
// One block per tile of `tile` consecutive cells, in sub-chunks of `sub`:
//   A. every thread takes SC_IPT consecutive cells: one binary search for the
//      row of its first cell, then a walk; builds the 12/16-byte records in
//      shared memory, with the bucket of each cell;
//   B. one warp deals the sub-chunk's records to their buckets in input
//      order (32 at a time; peers in a bucket are ranked by lane, and the
//      per-bucket cursor is a shared-memory fetch-and-add issued by the
//      group's first lane, so the order is deterministic and stable);
//   C. every thread stores its records at the assigned positions.
// Cursors start at bucket base + within-bucket tile offset (K2), so tiles keep
// input order inside a bucket.  Also: per-bucket value totals and the P x P
// counts (source block from the cell index, destination block from the
// column via a per-bucket first-block table and a short walk).
constexpr int SC_THREADS = 256;
constexpr int SC_IPT = 8;          // cells per thread per sub-chunk
constexpr int SC_SUB = SC_THREADS * SC_IPT;
constexpr int SC_PSMEM = 256;      // P up to which block tables live in shared memory

struct ScLayout {
    size_t cursor, vacc, d0, rec, bkt, dst, rows, pcs, pos, ppc, ppv, misc, total;
};
template <typename OffT, typename Rec>
__host__ __device__ inline ScLayout sc_layout(int B, int rowc, int P) {
    ScLayout L;
    size_t o = 0;
    const int Ps = P <= SC_PSMEM ? P : 0;
    L.cursor = o; o += (size_t)B * 4;
    L.vacc = o; o += (size_t)B * 4;
    L.d0 = o; o += (((size_t)B * 2) + 15) & ~size_t(15);
    L.rec = o; o += (((size_t)SC_SUB * sizeof(Rec)) + 15) & ~size_t(15);
    L.bkt = o; o += (size_t)SC_SUB * 2;
    L.dst = o; o += (size_t)SC_SUB * 4;
    L.rows = o; o += (((size_t)rowc * sizeof(OffT)) + 15) & ~size_t(15);
    L.pcs = o; o += (size_t)(Ps + 1) * 8;
    L.pos = o; o += (size_t)(Ps + 1) * 8;
    L.ppc = o; o += (((size_t)2 * Ps * 4) + 15) & ~size_t(15);
    L.ppv = o; o += (size_t)2 * Ps * 8;
    L.misc = o; o += 64;
    L.total = o;
    return L;
}

template <typename OffT, typename Rec>
__global__ void __launch_bounds__(SC_THREADS, 2)
    k_scatter(const void *__restrict__ row_ptr, const int32_t *__restrict__ col,
              const void *__restrict__ cell_ptr, long long R, long long N, long long C, long long V,
              int bshift, int B, int tile, int rowc, const uint32_t *__restrict__ cnt,
              const unsigned long long *__restrict__ bucket_base,
              unsigned long long *bucket_vtot, Rec *__restrict__ recs, int P,
              const long long *__restrict__ pcoff, const long long *__restrict__ poff,
              long long *part_cells, long long *part_values, DevHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ScLayout L = sc_layout<OffT, Rec>(B, rowc, P);
    uint32_t *cursor = reinterpret_cast<uint32_t *>(smem + L.cursor);
    uint32_t *vacc = reinterpret_cast<uint32_t *>(smem + L.vacc);
    uint16_t *d0 = reinterpret_cast<uint16_t *>(smem + L.d0);
    Rec *rec = reinterpret_cast<Rec *>(smem + L.rec);
    uint16_t *bkt = reinterpret_cast<uint16_t *>(smem + L.bkt);
    uint32_t *dstv = reinterpret_cast<uint32_t *>(smem + L.dst);
    OffT *rows = reinterpret_cast<OffT *>(smem + L.rows);
    long long *pcs = reinterpret_cast<long long *>(smem + L.pcs);
    long long *pos_ = reinterpret_cast<long long *>(smem + L.pos);
    uint32_t *ppc = reinterpret_cast<uint32_t *>(smem + L.ppc);
    unsigned long long *ppv = reinterpret_cast<unsigned long long *>(smem + L.ppv);
    long long *sh = reinterpret_cast<long long *>(smem + L.misc);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long t = blockIdx.x;
    const long long kt0 = t * (long long)tile, kt1 = min(C, kt0 + tile);
    const bool want_pp = (part_cells != nullptr) && P > 1;
    const bool pp_smem = want_pp && P <= SC_PSMEM;
    const long long *pc_tab = pp_smem ? pcs : pcoff;
    const long long *po_tab = pp_smem ? pos_ : poff;
    for (int b = tid; b < B; b += SC_THREADS) {
        cursor[b] = (uint32_t)(bucket_base[b] + cnt[t * B + b]);
        vacc[b] = 0;
    }
    if (pp_smem)
        for (int i = tid; i <= P; i += SC_THREADS) { pcs[i] = pcoff[i]; pos_[i] = poff[i]; }
    if (tid == 0) {
        long long s_first = upper_bound_ll(pcoff, 0, P + 1, kt0) - 1;
        long long s_last = upper_bound_ll(pcoff, 0, P + 1, kt1 - 1) - 1;
        sh[0] = s_first < 0 ? 0 : s_first;
        sh[1] = s_last < 0 ? 0 : s_last;
    }
    __syncthreads();
    const long long s_first = sh[0];
    const bool pp_local = pp_smem && (sh[1] - s_first) < 2;
    if (want_pp) {
        // destination block of each bucket's first column
        for (int b = tid; b < B; b += SC_THREADS) {
            long long c0 = (long long)b << bshift;
            long long d = (pp_smem ? upper_bound_sm(po_tab, 0, P + 1, c0)
                                   : upper_bound_ll(po_tab, 0, P + 1, c0)) - 1;
            d0[b] = (uint16_t)(d < 0 ? 0 : (d >= P ? P - 1 : d));
        }
        if (pp_local)
            for (int i = tid; i < 2 * P; i += SC_THREADS) { ppc[i] = 0; ppv[i] = 0; }
    }
    const long long wmask = (1LL << bshift) - 1;
    bool bad = false;

    for (long long s0 = kt0; s0 < kt1; s0 += SC_SUB) {
        const long long s1 = min(kt1, s0 + (long long)SC_SUB);
        const int n = (int)(s1 - s0);
        __syncthreads();
        if (tid == 0) {
            long long i0 = upper_bound_g<OffT>(row_ptr, 0, R + 1, s0) - 1;
            long long i1 = upper_bound_g<OffT>(row_ptr, i0 < 0 ? 0 : i0, R + 1, s1 - 1) - 1;
            if (i0 < 0) i0 = 0;
            if (i0 > R - 1) i0 = R - 1;
            if (i1 < i0) i1 = i0;
            if (i1 > R - 1) i1 = R - 1;
            sh[2] = i0;
            sh[3] = i1;
        }
        __syncthreads();
        const long long i0 = sh[2], i1 = sh[3];
        const long long nr = i1 - i0 + 2;  // row pointers i0 .. i1 + 1
        const bool cached = nr <= rowc;
        if (cached)
            for (long long r = tid; r < nr; r += SC_THREADS) rows[r] = (OffT)ldo<OffT>(row_ptr, i0 + r);
        __syncthreads();
        // ---- A: build records (thread owns cells [x0, x0 + SC_IPT))
        {
            const int x0 = tid * SC_IPT;
            if (x0 < n) {
                const long long k0 = s0 + x0;
                // row of the first cell, then walk
                long long i, nxt;
                if (cached) {
                    int lo = 0, hi = (int)nr;
                    while (lo < hi) {
                        int mid = (lo + hi) >> 1;
                        if ((long long)rows[mid] <= k0) lo = mid + 1;
                        else hi = mid;
                    }
                    i = lo - 1;  // relative to i0
                    nxt = (i + 1 < nr) ? (long long)rows[i + 1] : C;
                } else {
                    i = upper_bound_g<OffT>(row_ptr, i0, i1 + 2, k0) - 1 - i0;
                    nxt = ldo<OffT>(row_ptr, i0 + i + 1);
                }
                long long sp = s_first;
                if (want_pp) while (sp + 1 <= P && pc_tab[sp + 1] <= k0 && sp < P - 1) ++sp;
                long long stp = ldo<OffT>(cell_ptr, k0);
#pragma unroll
                for (int u = 0; u < SC_IPT; ++u) {
                    const int x = x0 + u;
                    if (x >= n) break;
                    const long long k = k0 + u;
                    while (nxt <= k && i0 + i + 1 < R) {
                        ++i;
                        nxt = cached ? ((i + 1 < nr) ? (long long)rows[i + 1] : C)
                                     : ldo<OffT>(row_ptr, i0 + i + 1);
                    }
                    long long c = __ldg(col + k);
                    if (c < 0 || c >= N) { bad = true; c = c < 0 ? 0 : N - 1; }
                    long long st = stp, en = ldo<OffT>(cell_ptr, k + 1);
                    stp = en;
                    if (st < 0 || st > V) { bad = true; st = st < 0 ? 0 : V; }
                    if (en < st || en > V) { bad = true; en = en > V ? V : st; }
                    long long irow = i0 + i;
                    if (irow >= R) irow = R - 1;
                    const uint32_t b = (uint32_t)(c >> bshift);
                    const unsigned long long len = (unsigned long long)(en - st);
                    Rec r;
                    r.i = (uint32_t)irow;
                    r.meta = pack_meta((uint32_t)(c & wmask), len);
                    r.start = (decltype(r.start))st;
                    rec[x] = r;
                    bkt[x] = (uint16_t)b;
                    if (len < LEN_ESC) atomicAdd(&vacc[b], (uint32_t)len);
                    else atomicAdd(&bucket_vtot[b], len);
                    if (want_pp) {
                        while (sp < P - 1 && pc_tab[sp + 1] <= k) ++sp;
                        long long d = d0[b];
                        while (d < P - 1 && po_tab[d + 1] <= c) ++d;
                        if (pp_local && sp - s_first < 2) {
                            const int rowp = (int)(sp - s_first);
                            atomicAdd(&ppc[rowp * P + d], 1u);
                            atomicAdd(&ppv[rowp * P + d], len);
                        } else {
                            atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[sp * P + d]), 1ull);
                            atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[sp * P + d]), len);
                        }
                    }
                }
            }
        }
        __syncthreads();
        // ---- B: one warp deals the records to their buckets, in order
        if (warp == 0) {
            for (int base = 0; base < n; base += 32) {
                const int x = base + lane;
                const bool v = x < n;
                const uint32_t b = v ? (uint32_t)bkt[x] : 0xFFFFFFFFu;
                const unsigned peers = __match_any_sync(0xffffffffu, b);
                const unsigned lower = peers & lanemask_lt();
                uint32_t pos = 0;
                if (v && lower == 0) pos = atomicAdd(&cursor[b], (uint32_t)__popc(peers));
                pos = __shfl_sync(0xffffffffu, pos, __ffs(peers) - 1);
                if (v) dstv[x] = pos + (uint32_t)__popc(lower);
            }
        }
        __syncthreads();
        // ---- C: store the records
        for (int x = tid; x < n; x += SC_THREADS)
            if (MGT_IN(hdr, dstv[x], C)) recs[dstv[x]] = rec[x];
    }
    __syncthreads();
    for (int b = tid; b < B; b += SC_THREADS)
        if (vacc[b]) atomicAdd(&bucket_vtot[b], (unsigned long long)vacc[b]);
    if (pp_local) {
        for (int x = tid; x < 2 * P; x += SC_THREADS) {
            long long sp = s_first + x / P, dp = x % P;
            if (sp < P && ppc[x]) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[sp * P + dp]),
                          (unsigned long long)ppc[x]);
                atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[sp * P + dp]), ppv[x]);
            }
        }
    }
    if (__syncthreads_or(bad) && tid == 0) flag(hdr, ST_BADINPUT);
}

size_t scatter_smem_bytes(const Params &p) {
    if (p.o == 4)
        return p.wide ? sc_layout<int32_t, RecW>((int)p.B, p.rowc, p.P).total
                      : sc_layout<int32_t, RecC>((int)p.B, p.rowc, p.P).total;
    return p.wide ? sc_layout<int64_t, RecW>((int)p.B, p.rowc, p.P).total
                  : sc_layout<int64_t, RecC>((int)p.B, p.rowc, p.P).total;
}

template <typename OffT, typename Rec>
static cudaError_t launch_scatter_t(const Params &p, const Inputs &in, const Outputs &out,
                                    const Ws &ws, cudaStream_t st) {
    const size_t smem = sc_layout<OffT, Rec>((int)p.B, p.rowc, p.P).total;
    auto kern = k_scatter<OffT, Rec>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)p.T, SC_THREADS, smem, st>>>(
        in.row_ptr, in.col, in.cell_ptr, p.R, p.N, p.C, p.V, p.bshift, (int)p.B, p.tile, p.rowc,
        ws.cnt, ws.bucket_base, ws.bucket_vtot, reinterpret_cast<Rec *>(ws.recs), p.P, ws.pcoff,
        ws.poff, out.part_cells, out.part_values, ws.hdr);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const Params &p, const Inputs &in, const Outputs &out, const Ws &ws,
                           cudaStream_t st) {
    if (p.T == 0) return cudaSuccess;
    if (p.o == 4)
        return p.wide ? launch_scatter_t<int32_t, RecW>(p, in, out, ws, st)
                      : launch_scatter_t<int32_t, RecC>(p, in, out, ws, st);
    return p.wide ? launch_scatter_t<int64_t, RecW>(p, in, out, ws, st)
                  : launch_scatter_t<int64_t, RecC>(p, in, out, ws, st);
}


// ------------------------------------------------------------ K4 build work
// One block: value bases per bucket (exclusive prefix of bucket_vtot) and the
// sort work list.  A bucket with at most `ch` records (one sort cluster) is
// one item; a larger one is cut into ceil(n / chm) chunks that get
// cursor-matrix rows.
__global__ void k_build_work(long long B, long long ch, long long chm, long long V, const unsigned long long *bucket_tot,
                             const unsigned long long *bucket_base,
                             const unsigned long long *bucket_vtot,
                             unsigned long long *bucket_vbase, WorkItem *items,
                             uint32_t *multi_items, MultiBucket *multi_buckets, DevHeader *hdr,
                             long long max_items, long long max_rows, long long max_mb) {
    __shared__ unsigned long long sc[3][33];
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long per = (B + nt - 1) / nt, lo = min(B, tid * per), hi = min(B, lo + per);
    // three running sums: values, items, multi-chunk rows (and multi buckets)
    unsigned long long sv = 0, si = 0, sr = 0, smb = 0;
    for (long long b = lo; b < hi; ++b) {
        unsigned long long n = bucket_tot[b];
        const bool big = n > (unsigned long long)ch;  // more than one sort cluster holds
        unsigned long long nch = big ? (n + chm - 1) / chm : 1;
        sv += bucket_vtot[b];
        si += nch;
        if (big) { sr += nch; smb += 1; }
    }
    unsigned long long iv = warp_inclusive_scan(sv), ii = warp_inclusive_scan(si),
                       ir = warp_inclusive_scan(sr), imb = warp_inclusive_scan(smb);
    __shared__ unsigned long long smb_s[33];
    if (lane == 31) { sc[0][warp] = iv; sc[1][warp] = ii; sc[2][warp] = ir; smb_s[warp] = imb; }
    __syncthreads();
    if (tid < 32) {
        int nw = nt >> 5;
        for (int q = 0; q < 3; ++q) {
            unsigned long long v = tid < nw ? sc[q][tid] : 0ull;
            unsigned long long vi = warp_inclusive_scan(v);
            sc[q][tid] = vi - v;
            if (tid == 31) sc[q][32] = vi;
        }
        unsigned long long v = tid < nw ? smb_s[tid] : 0ull;
        unsigned long long vi = warp_inclusive_scan(v);
        smb_s[tid] = vi - v;
        if (tid == 31) smb_s[32] = vi;
    }
    __syncthreads();
    unsigned long long rv = sc[0][warp] + iv - sv, ri = sc[1][warp] + ii - si,
                       rr = sc[2][warp] + ir - sr, rmb = smb_s[warp] + imb - smb;
    const bool consistent = (hdr->status & ST_BADINPUT) == 0 && sc[0][32] == (unsigned long long)V;
    const bool fits = consistent && sc[1][32] <= (unsigned long long)max_items &&
                      sc[2][32] <= (unsigned long long)max_rows &&
                      smb_s[32] <= (unsigned long long)max_mb;
    for (long long b = lo; b < hi && fits; ++b) {
        unsigned long long n = bucket_tot[b], bb = bucket_base[b];
        const bool big = n > (unsigned long long)ch;
        unsigned long long nch = big ? (n + chm - 1) / chm : 1;
        bucket_vbase[b] = rv;
        rv += bucket_vtot[b];
        if (big) {
            MultiBucket mb;
            mb.mc0 = rr;
            mb.bucket = (uint32_t)b;
            mb.nch = (uint32_t)nch;
            multi_buckets[rmb++] = mb;
        }
        for (unsigned long long h = 0; h < nch; ++h) {
            WorkItem it;
            it.r0 = bb + (n * h) / nch;
            it.r1 = bb + (n * (h + 1)) / nch;
            it.bucket = (uint32_t)b;
            it.chunk = (uint32_t)h;
            it.mc = big ? rr + h : ~0ull;
            items[ri] = it;
            if (big) multi_items[rr + h] = (uint32_t)ri;
            ++ri;
        }
        if (big) rr += nch;
    }
    if (tid == 0) {
        if (!consistent) flag(hdr, ST_BADINPUT);
        else if (!fits) flag(hdr, ST_OVERFLOW);
        hdr->n_items = fits ? sc[1][32] : 0;
        hdr->n_multi_items = fits ? sc[2][32] : 0;
        hdr->n_multi_buckets = fits ? smb_s[32] : 0;
        hdr->reserved[3] = (unsigned long long)max_items;  // bounds for debug-build checks
        hdr->reserved[4] = (unsigned long long)max_rows;
    }
}

cudaError_t launch_build_work(const Params &p, const Ws &ws, cudaStream_t st) {
    if (p.B == 0) return cudaSuccess;
    k_build_work<<<1, 1024, 0, st>>>(p.B, p.ch, p.chm, p.V, ws.bucket_tot, ws.bucket_base, ws.bucket_vtot,
                                     ws.bucket_vbase, ws.items, ws.multi_items, ws.multi_buckets,
                                     ws.hdr, p.max_items, p.max_multi_rows, p.max_multi_buckets);
    return cudaGetLastError();
}

}  // namespace mgt
