// Level 1 of the transpose: stable scatter of cell records into column buckets.
//
// The paper exchanges cells between ranks by destination (Sec. 3, view swap:
// metadata, then values).  On one GPU the destination of a cell is a bucket of
// consecutive output rows (= input columns); K1-K3 deal every cell's record
// into its bucket, keeping row-major input order inside each bucket, so that
// the per-bucket sort of K7 only has to order by column.
#include "mgt_internal.cuh"

#include <algorithm>
#include <climits>

#include <cooperative_groups.h>

namespace mgt {

constexpr int K_THREADS = 512;

// ------------------------------------------------------------------ K0 prep
// Checks the pointer arrays' end points and that row_ptr never decreases;
// writes the source blocks' cell offsets pcoff[s] = row_ptr[off[s]], the
// output sentinels row_ptr'[N] = C and cell_ptr'[C] = V, and the P = 1 counts.
template <typename OffT, bool BATCH>
__global__ void __launch_bounds__(K_THREADS) k_prep(const __grid_constant__ Mat m0, const BatchArgs ba) {
    const VBlock vb = vblock<BATCH>(m0, ba);
    const Mat &M = *vb.m;
    const void *row_ptr = M.in.row_ptr, *cell_ptr = M.in.cell_ptr;
    const long long R = M.p.R, N = M.p.N, C = M.p.C, V = M.p.V, B = M.p.B;
    const int P = M.p.P, bshift = M.p.bshift;
    const long long *poff = M.ws.poff;
    long long *pcoff = M.ws.pcoff;
    uint16_t *dblock = M.ws.dblock;
    void *out_row_ptr = M.out.row_ptr, *out_cell_ptr = M.out.cell_ptr;
    long long *part_cells = M.out.part_cells, *part_values = M.out.part_values;
    DevHeader *hdr = M.ws.hdr;
    long long gid = vb.b * (long long)blockDim.x + threadIdx.x;
    long long stride = vb.g * (long long)blockDim.x;
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
    // destination block of each bucket's columns, or 0xFFFF when they span two
    for (long long b = gid; b < B && P > 1; b += stride) {
        const long long c0 = b << bshift, c1 = min(N, c0 + (1LL << bshift)) - 1;
        long long da = upper_bound_ll(poff, 0, P + 1, c0) - 1, db = upper_bound_ll(poff, 0, P + 1, c1) - 1;
        da = da < 0 ? 0 : (da >= P ? P - 1 : da);
        dblock[b] = (da == db) ? (uint16_t)da : (uint16_t)0xFFFFu;
    }
    bool bad = false;
    for (long long i = gid; i < R; i += stride)
        bad |= ldo<OffT>(row_ptr, i + 1) < ldo<OffT>(row_ptr, i);
    if (__syncthreads_or(bad) && threadIdx.x == 0) flag(hdr, ST_BADINPUT);
}

static long long grid_prep(const Params &p, double share) {
    const long long full = 2LL * sm_count();
    long long want = (p.R + K_THREADS - 1) / K_THREADS;
    long long cap = (long long)(full * share + 0.999);
    if (cap < 1) cap = 1;
    if (want > cap) want = cap;
    return want < 1 ? 1 : want;
}
static size_t smem_none(const Params &) { return 0; }
static cudaError_t launch_prep(const Mat &m0, const BatchArgs &ba, long long grid, size_t,
                               cudaStream_t st) {
    auto kern = m0.p.o == 4 ? (ba.n ? k_prep<int32_t, true> : k_prep<int32_t, false>)
                            : (ba.n ? k_prep<int64_t, true> : k_prep<int64_t, false>);
    kern<<<(unsigned)grid, K_THREADS, 0, st>>>(m0, ba);
    return cudaGetLastError();
}

// Zeroes the header, the per-bucket value totals and the P x P outputs of
// every matrix of a batch (one transpose alone uses memsets instead).
template <bool BATCH>
__global__ void __launch_bounds__(K_THREADS) k_zero(const __grid_constant__ Mat m0, const BatchArgs ba) {
    const VBlock vb = vblock<BATCH>(m0, ba);
    const Mat &M = *vb.m;
    const long long gid = vb.b * (long long)blockDim.x + threadIdx.x;
    const long long stride = vb.g * (long long)blockDim.x;
    unsigned long long *h = reinterpret_cast<unsigned long long *>(M.ws.hdr);
    for (long long i = gid; i < 32; i += stride) h[i] = 0;
    for (long long i = gid; i < M.p.B; i += stride) M.ws.bucket_vtot[i] = 0;
    const long long pp = (long long)M.p.P * M.p.P;
    if (M.out.part_cells)
        for (long long i = gid; i < pp; i += stride) { M.out.part_cells[i] = 0; M.out.part_values[i] = 0; }
}

long long grid_zero(const Params &p, double) {
    const long long n = std::max<long long>(std::max<long long>(32, p.B), (long long)p.P * p.P);
    const long long g = (n + K_THREADS - 1) / K_THREADS;
    return g < 64 ? g : 64;
}
cudaError_t launch_zero(const Mat &m0, const BatchArgs &ba, long long grid, size_t, cudaStream_t st) {
    k_zero<true><<<(unsigned)grid, K_THREADS, 0, st>>>(m0, ba);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ K1 hist
// Cells per bucket for one tile of `tile` consecutive cells, in a shared
// memory histogram; written as row t of the T x B count matrix.
template <bool BATCH>
__global__ void __launch_bounds__(K_THREADS) k_hist(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ uint32_t hist[];
    const VBlock vb = vblock<BATCH>(m0, ba);
    const Mat &M = *vb.m;
    const int32_t *__restrict__ col = M.in.col;
    const long long C = M.p.C, N = M.p.N;
    const int bshift = M.p.bshift, B = (int)M.p.B, tile = M.p.tile;
    uint32_t *__restrict__ cnt = M.ws.cnt;
    DevHeader *hdr = M.ws.hdr;
    const long long t = vb.b;
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

static long long grid_hist(const Params &p, double) { return p.T; }
static size_t smem_hist(const Params &p) { return (size_t)p.B * sizeof(uint32_t); }
static cudaError_t launch_hist(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                               cudaStream_t st) {
    auto kern = ba.n ? k_hist<true> : k_hist<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, K_THREADS, smem, st>>>(m0, ba);
    return cudaGetLastError();
}

// ------------------------------------------------------------ K2 scan tiles
// For 32 K buckets per block: replace cnt[t][b] by the exclusive prefix over
// tiles t' < t (keeps tiles, hence input order, inside each bucket) and
// write the bucket totals; warp w takes tiles [T w / 32, T (w + 1) / 32).
// K = 1: a lane per bucket.  K = 4, for count matrices of many tiles: a lane
// per 4 neighbouring buckets (16-byte loads when B is a multiple of 4), so
// that a warp reads 512 contiguous bytes of a tile's row instead of 128 (the
// rows lie tens of kilobytes apart); with few tiles the 4x larger blocks
// would leave SMs idle.
__host__ __device__ inline int scan_tiles_k(const Params &p) { return p.T >= 4096 ? 4 : 1; }

template <int K>
__device__ __forceinline__ void scan_tiles_body(const Mat &M, long long blk,
                                                unsigned long long (*part)[32][33]) {
    uint32_t *cnt = M.ws.cnt;
    const long long T = M.p.T, B = M.p.B;
    unsigned long long *bucket_tot = M.ws.bucket_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long b = blk * (32LL * K) + (long long)K * lane;  // buckets b .. b + K - 1
    const bool vec = K == 4 && (B & 3) == 0;
    const long long t0 = T * warp / nw, t1 = T * (warp + 1) / nw;
    auto load = [&](long long t, uint32_t *x) {
        const uint32_t *r = cnt + t * B;
        if (vec) {
            const uint4 v = *reinterpret_cast<const uint4 *>(r + b);
            x[0] = v.x;
            if (K == 4) { x[1] = v.y; x[2] = v.z; x[3] = v.w; }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) x[k] = b + k < B ? r[b + k] : 0u;
        }
    };
    unsigned long long sum[K];
#pragma unroll
    for (int k = 0; k < K; ++k) sum[k] = 0;
    if (b < B) {
        long long t = t0;
        for (; t + 4 / K <= t1 && K == 1; t += 4) {  // K = 1: four loads in flight
            uint32_t x0[K], x1[K], x2[K], x3[K];
            load(t, x0); load(t + 1, x1); load(t + 2, x2); load(t + 3, x3);
            sum[0] += (unsigned long long)x0[0] + x1[0] + x2[0] + x3[0];
        }
        for (; t + 2 <= t1 && K == 4; t += 2) {
            uint32_t x[K], y[K];
            load(t, x);
            load(t + 1, y);
#pragma unroll
            for (int k = 0; k < K; ++k) sum[k] += (unsigned long long)x[k] + y[k];
        }
        for (; t < t1; ++t) {
            uint32_t x[K];
            load(t, x);
#pragma unroll
            for (int k = 0; k < K; ++k) sum[k] += x[k];
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) part[k][warp][lane] = sum[k];
    __syncthreads();
    if (warp < K) {  // warp q: the prefix over warps of each lane's bucket b + q
        unsigned long long run = 0;
        for (int w = 0; w < nw; ++w) {
            const unsigned long long v = part[warp][w][lane];
            part[warp][w][lane] = run;
            run += v;
        }
        if (b + warp < B) bucket_tot[b + warp] = run;
    }
    __syncthreads();
    if (b < B) {
        unsigned long long run[K];
#pragma unroll
        for (int k = 0; k < K; ++k) run[k] = part[k][warp][lane];
        long long t = t0;
        for (; t + 4 <= t1 && K == 1; t += 4) {  // K = 1: four loads in flight
            uint32_t x0[K], x1[K], x2[K], x3[K];
            load(t, x0); load(t + 1, x1); load(t + 2, x2); load(t + 3, x3);
            uint32_t *r = cnt + t * B + b;
            r[0] = (uint32_t)run[0];
            r[B] = (uint32_t)(run[0] + x0[0]);
            r[2 * B] = (uint32_t)(run[0] + x0[0] + x1[0]);
            r[3 * B] = (uint32_t)(run[0] + x0[0] + x1[0] + x2[0]);
            run[0] += (unsigned long long)x0[0] + x1[0] + x2[0] + x3[0];
        }
        for (; t < t1; ++t) {
            uint32_t x[K];
            load(t, x);
            uint32_t *r = cnt + t * B;  // within-bucket offsets (< 2^32 by plan)
            if (vec) {
                *reinterpret_cast<uint4 *>(r + b) =
                    make_uint4((uint32_t)run[0], (uint32_t)run[K > 1 ? 1 : 0], (uint32_t)run[K > 2 ? 2 : 0],
                               (uint32_t)run[K > 3 ? 3 : 0]);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k)
                    if (b + k < B) r[b + k] = (uint32_t)run[k];
            }
#pragma unroll
            for (int k = 0; k < K; ++k) run[k] += x[k];
        }
    }
}

template <bool BATCH>
__global__ void __launch_bounds__(1024) k_scan_tiles(const __grid_constant__ Mat m0, const BatchArgs ba) {
    __shared__ unsigned long long part[4][32][33];
    const VBlock vb = vblock<BATCH>(m0, ba);
    if (scan_tiles_k(vb.m->p) == 4) scan_tiles_body<4>(*vb.m, vb.b, part);
    else scan_tiles_body<1>(*vb.m, vb.b, part);
}

static long long grid_scan_tiles(const Params &p, double) {
    const long long per = 32LL * scan_tiles_k(p);
    return (p.B + per - 1) / per;
}
static cudaError_t launch_scan_tiles(const Mat &m0, const BatchArgs &ba, long long grid, size_t,
                                     cudaStream_t st) {
    (ba.n ? k_scan_tiles<true> : k_scan_tiles<false>)<<<(unsigned)grid, 1024, 0, st>>>(m0, ba);
    return cudaGetLastError();
}

// ---------------------------------------------------------- K2b scan buckets
// One block: exclusive prefix of the 64-bit per-bucket totals.
template <bool BATCH>
__global__ void __launch_bounds__(1024) k_scan_u64(const __grid_constant__ Mat m0, const BatchArgs ba) {
    __shared__ unsigned long long scratch[33];
    const VBlock vb = vblock<BATCH>(m0, ba);
    const Mat &M = *vb.m;
    const unsigned long long *in = M.ws.bucket_tot;
    unsigned long long *out = M.ws.bucket_base;
    const long long n = M.p.B;
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

static long long grid_one_if_buckets(const Params &p, double) { return p.B > 0 ? 1 : 0; }
static cudaError_t launch_scan_buckets(const Mat &m0, const BatchArgs &ba, long long grid, size_t,
                                       cudaStream_t st) {
    (ba.n ? k_scan_u64<true> : k_scan_u64<false>)<<<(unsigned)grid, 1024, 0, st>>>(m0, ba);
    return cudaGetLastError();
}

// --------------------------------------------------------------- K3 scatter
// Two stable passes, like the digit passes of a radix sort, so that every
// pass writes runs of records instead of isolated ones:
//   K3a (cells -> super-buckets): one block per tile of `tile` cells, in
//       sub-chunks of SA_SUB.  A: every thread builds the records of
//       SA_IPT consecutive cells (row by a search in a shared copy of the
//       sub-chunk's row pointers, then a walk); B: stable multisplit of the
//       sub-chunk by super-bucket (bucket >> p2) with per-warp counters, all
//       warps in parallel, staged in shared memory; C: runs written out at
//       the super-bucket cursors.
//   K3b (super-bucket -> buckets): one block per (super-bucket, tile group)
//       item, same multisplit by the low p2 bits of the bucket, written at
//       the final bucket cursors.
// Cursors come from the tile-by-bucket offsets of K2, so input order is kept
// inside every bucket.  K3a also produces the P x P counts (source block
// from the cell index, destination block per super-bucket, or per cell
// where a super-bucket spans two destination blocks); K3b the per-bucket
// value totals (K3a when there is a single pass).
constexpr int SA_THREADS = 256;
constexpr int SA_WARPS = SA_THREADS / 32;
constexpr int SA_IPT = 8;
constexpr int SA_SUB = SA_THREADS * SA_IPT;  // 2048
constexpr int SA_PSMEM = 256;                 // P up to which block tables live in shared memory
constexpr uint16_t SC_STRADDLE = 0xFFFFu;     // spans a destination block boundary

// The second-pass digit (low p2 bits of the bucket) rides in a record
// between the passes: above the column bits of meta for compact records
// (the planner keeps bshift + p2 <= 16 there, else it uses wide records
// between the passes), in bits 48.. of start for wide ones (V < 2^48).
__device__ __forceinline__ void put_d2(RecC &r, uint32_t d2, int bshift) { r.meta |= d2 << (16 + bshift); }
__device__ __forceinline__ void put_d2(RecW &r, uint32_t d2, int) {
    r.start |= (unsigned long long)d2 << 48;
}
__device__ __forceinline__ uint32_t take_d2(RecC &r, int bshift, int p2) {
    const uint32_t m = ((1u << p2) - 1u) << (16 + bshift);
    const uint32_t d = (r.meta & m) >> (16 + bshift);
    r.meta &= ~m;
    return d;
}
__device__ __forceinline__ uint32_t take_d2(RecW &r, int, int) {
    const uint32_t d = (uint32_t)(r.start >> 48);
    r.start &= (1ull << 48) - 1ull;
    return d;
}
__device__ __forceinline__ void rec_convert(const RecC &a, RecC &b) { b = a; }
__device__ __forceinline__ void rec_convert(const RecW &a, RecW &b) { b = a; }
__device__ __forceinline__ void rec_convert(const RecW &a, RecC &b) {
    b.i = a.i;
    b.meta = a.meta;
    b.start = (uint32_t)a.start;
}

// Stable multisplit of n (<= SA_SUB) keys by digit (< nbins <= SA_THREADS)
// for one block: warp w owns keys [w SEG, (w+1) SEG), lane l key
// w SEG + 32 u + l in round u.
//   1. Per round, a peer mask from votes groups the lanes of equal digit;
//      every lane reads its digit's count in the warp, the group's lowest
//      lane adds the group's size; rank = that count + the group's lanes
//      below.
//   2. Digit-major scan of the (digit, warp) counts: one thread per digit
//      (its warps' counts in registers), a block scan of the digit totals;
//      position = digit start + earlier warps' count + rank keeps equal
//      digits in key order.
//   3. Positions out; each warp then clears its own counters (no other warp
//      reads them after the scan), which the next call expects.
// Fills stg_pos[x] (position of key x), stg_dig[position] and
// bstart[0..nbins].  wcnt: SA_WARPS * (nbins + 1) u32 (see wc_at), zero on
// entry and on return; scratch: >= SA_WARPS words.  Ends with a barrier.
__device__ __forceinline__ void block_multisplit(const uint8_t *digit, int n, int nbins,
                                                 uint32_t *wcnt, uint32_t *bstart,
                                                 uint16_t *stg_pos, uint8_t *stg_dig,
                                                 uint32_t *scratch) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int SEG = SA_SUB / SA_WARPS;
    constexpr int ROUNDS = SEG / 32;
    uint32_t dk[ROUNDS], rk[ROUNDS];
    unsigned pk[ROUNDS];
#pragma unroll
    for (int u = 0; u < ROUNDS; ++u) {
        const int x = warp * SEG + u * 32 + lane;
        dk[u] = x < n ? (uint32_t)digit[x] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int u = 0; u < ROUNDS; ++u) pk[u] = vote_peers(dk[u], nbins);
#pragma unroll
    for (int u = 0; u < ROUNDS; ++u) {
        const bool v = dk[u] != 0xFFFFFFFFu;
        const unsigned lower = pk[u] & lanemask_lt();
        uint32_t before = 0;
        if (v) before = wcnt[wc_at(dk[u], warp, nbins)];
        __syncwarp();
        if (v && lower == 0) wcnt[wc_at(dk[u], warp, nbins)] = before + __popc(pk[u]);
        __syncwarp();
        rk[u] = before + __popc(lower);
    }
    __syncthreads();
    uint32_t c[SA_WARPS], tot = 0;
#pragma unroll
    for (int w = 0; w < SA_WARPS; ++w) {
        c[w] = tid < nbins ? wcnt[wc_at(tid, w, nbins)] : 0u;
        tot += c[w];
    }
    const uint32_t inc = warp_inclusive_scan(tot);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < SA_WARPS; ++w) {
        const uint32_t v = scratch[w];
        before += w < warp ? v : 0u;
        total += v;
    }
    if (tid < nbins) {
        uint32_t run = before + inc - tot;
        bstart[tid] = run;
#pragma unroll
        for (int w = 0; w < SA_WARPS; ++w) {
            wcnt[wc_at(tid, w, nbins)] = run;
            run += c[w];
        }
    }
    if (tid == 0) bstart[nbins] = total;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < ROUNDS; ++u) {
        const int x = warp * SEG + u * 32 + lane;
        if (x < n) {
            const uint32_t pos = wcnt[wc_at(dk[u], warp, nbins)] + rk[u];
            stg_pos[x] = (uint16_t)pos;
            stg_dig[pos] = (uint8_t)dk[u];
        }
    }
    __syncwarp();
    for (int d = lane; d <= nbins; d += 32) wcnt[wc_at(d, warp, nbins)] = 0;
    __syncthreads();
}

struct SaLayout {
    size_t cur, tcnt, tvs, tvs32, sblk, slo, shi, sspl, wcnt, bstart, stg, dig, spos, sdig, rows, pcs, pos,
        ppt, ppc, ppc32, scratch, misc, total;
};
template <typename OffT, typename Rec>
__host__ __device__ inline SaLayout sa_layout(int nbins, int rowc, int P) {
    SaLayout L;
    size_t o = 0;
    const int Ps = P <= SA_PSMEM ? P : 0;
#define MGT_TAKE(field, bytes) L.field = o; o = (o + (size_t)(bytes) + 15) & ~size_t(15);
    MGT_TAKE(cur, (size_t)nbins * 4)
    MGT_TAKE(tcnt, (size_t)nbins * 4)
    MGT_TAKE(tvs, (size_t)nbins * 8)
    MGT_TAKE(tvs32, (size_t)nbins * 4)
    MGT_TAKE(sblk, (size_t)nbins * 2)
    MGT_TAKE(slo, (size_t)nbins * 2)
    MGT_TAKE(shi, (size_t)nbins * 2)
    MGT_TAKE(sspl, (size_t)nbins * 4)
    MGT_TAKE(wcnt, (size_t)(nbins + 1) * SA_WARPS * 4)
    MGT_TAKE(bstart, (size_t)(nbins + 1) * 4)
    MGT_TAKE(stg, (size_t)SA_SUB * sizeof(Rec))
    MGT_TAKE(dig, (size_t)SA_SUB)
    MGT_TAKE(spos, (size_t)SA_SUB * 2)
    MGT_TAKE(sdig, (size_t)SA_SUB)
    MGT_TAKE(rows, (size_t)rowc * sizeof(OffT))
    MGT_TAKE(pcs, (size_t)(Ps + 1) * 8)
    MGT_TAKE(pos, (size_t)(Ps + 1) * 8)
    MGT_TAKE(ppt, (size_t)2 * Ps * 8)
    MGT_TAKE(ppc, (size_t)4 * Ps * 8)
    MGT_TAKE(ppc32, (size_t)4 * Ps * 4)
    MGT_TAKE(scratch, 48 * 4)
    MGT_TAKE(misc, 64)
#undef MGT_TAKE
    L.total = o;
    return L;
}

// PP = false: an instantiation without the P x P counting (the counts come
// from the output pass, or none are asked for): fewer registers and no
// counter tables in shared memory.
template <typename OffT, typename Rec, bool BATCH, bool PP>
__global__ void __launch_bounds__(SA_THREADS, PP ? 2 : 3)
    k_scatter(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    const VBlock vb = vblock<BATCH>(m0, ba);
    const Mat &M = *vb.m;
    const void *__restrict__ row_ptr = M.in.row_ptr;
    const int32_t *__restrict__ col = M.in.col;
    const void *__restrict__ cell_ptr = M.in.cell_ptr;
    const long long R = M.p.R, N = M.p.N, C = M.p.C, V = M.p.V;
    const int bshift = M.p.bshift, B = (int)M.p.B, p2 = M.p.p2, tile = M.p.tile, rowc = M.p.rowc;
    const int P = M.p.P;
    const uint32_t *__restrict__ cnt = M.ws.cnt;
    const unsigned long long *__restrict__ bucket_base = M.ws.bucket_base;
    unsigned long long *bucket_vtot = M.ws.bucket_vtot;
    Rec *__restrict__ out = reinterpret_cast<Rec *>(p2 > 0 ? M.ws.recs1 : M.ws.recs);
    const long long *__restrict__ pcoff = M.ws.pcoff;
    const long long *__restrict__ poff = M.ws.poff;
    const uint16_t *__restrict__ dblock = M.ws.dblock;
    long long *part_cells = M.out.part_cells, *part_values = M.out.part_values;
    DevHeader *hdr = M.ws.hdr;
    const int nbins = (B + (1 << p2) - 1) >> p2;
    const SaLayout L = sa_layout<OffT, Rec>(nbins, rowc, PP ? P : 0);
    uint32_t *cur = reinterpret_cast<uint32_t *>(smem + L.cur);
    uint32_t *tcnt = reinterpret_cast<uint32_t *>(smem + L.tcnt);
    unsigned long long *tvs = reinterpret_cast<unsigned long long *>(smem + L.tvs);
    uint32_t *tvs32 = reinterpret_cast<uint32_t *>(smem + L.tvs32);  // per sub-chunk
    uint16_t *sblk = reinterpret_cast<uint16_t *>(smem + L.sblk);  // destination block of a super-bucket (or STRADDLE)
    uint16_t *slo = reinterpret_cast<uint16_t *>(smem + L.slo);    // block of its first column
    uint16_t *shi = reinterpret_cast<uint16_t *>(smem + L.shi);    // block of its last column
    int32_t *sspl = reinterpret_cast<int32_t *>(smem + L.sspl);    // first column of block shi when it spans two
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(smem + L.wcnt);
    uint32_t *bstart = reinterpret_cast<uint32_t *>(smem + L.bstart);
    Rec *stg = reinterpret_cast<Rec *>(smem + L.stg);
    uint8_t *dig = smem + L.dig;
    uint16_t *spos = reinterpret_cast<uint16_t *>(smem + L.spos);
    uint8_t *sdig = smem + L.sdig;
    OffT *rows = reinterpret_cast<OffT *>(smem + L.rows);
    long long *pcs = reinterpret_cast<long long *>(smem + L.pcs);
    long long *pos_ = reinterpret_cast<long long *>(smem + L.pos);
    unsigned long long *ppt = reinterpret_cast<unsigned long long *>(smem + L.ppt);  // [2][P]
    unsigned long long *ppc = reinterpret_cast<unsigned long long *>(smem + L.ppc);  // [2 blocks][2][P]
    uint32_t *ppc32 = reinterpret_cast<uint32_t *>(smem + L.ppc32);  // the same, per sub-chunk
    uint32_t *scratch = reinterpret_cast<uint32_t *>(smem + L.scratch);
    long long *sh = reinterpret_cast<long long *>(smem + L.misc);

    const int tid = threadIdx.x;
    const long long t = vb.b;
    const long long kt0 = t * (long long)tile, kt1 = min(C, kt0 + tile);
    const bool want_pp = PP && (part_cells != nullptr) && P > 1 && !M.p.pp_out;
    const bool pp_smem = want_pp && P <= SA_PSMEM;
    const long long *pc_tab = pp_smem ? pcs : pcoff;
    const long long *po_tab = pp_smem ? pos_ : poff;
    const uint32_t mask2 = (1u << p2) - 1u;
    // cursors: super-bucket base + this tile's offsets inside its buckets
    for (int d = tid; d < nbins; d += SA_THREADS) {
        cur[d] = 0;
        tcnt[d] = 0;
        tvs[d] = 0;
        tvs32[d] = 0;
    }
    for (int i = tid; i < (nbins + 1) * SA_WARPS; i += SA_THREADS) wcnt[i] = 0;  // the multisplit's invariant
    if (pp_smem) {
        for (int i = tid; i <= P; i += SA_THREADS) { pcs[i] = pcoff[i]; pos_[i] = poff[i]; }
        for (int i = tid; i < 2 * P; i += SA_THREADS) ppt[i] = 0;
        for (int i = tid; i < 4 * P; i += SA_THREADS) { ppc[i] = 0; ppc32[i] = 0; }
    }
    __syncthreads();
    // this tile's offset inside each super-bucket: sum of its buckets'
    // offsets (the 2^p2 buckets of a super-bucket are consecutive), reduced
    // over the lanes that share a super-bucket, eight loads in flight
    for (int b0 = 0; b0 < B; b0 += 8 * SA_THREADS) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + u * SA_THREADS + tid;
            v[u] = b < B ? cnt[t * B + b] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + u * SA_THREADS + tid;
            const uint32_t S = b < B ? (uint32_t)(b >> p2) : 0xFFFFFFFFu;
            const unsigned peers = __match_any_sync(0xffffffffu, S);
            const uint32_t sum = __reduce_add_sync(peers, v[u]);
            if (b < B && (peers & lanemask_lt()) == 0) atomicAdd(&cur[S], sum);
        }
    }
    if (tid == 0) {
        long long s_first = upper_bound_ll(pcoff, 0, P + 1, kt0) - 1;
        long long s_last = upper_bound_ll(pcoff, 0, P + 1, kt1 - 1) - 1;
        sh[0] = s_first < 0 ? 0 : s_first;
        sh[1] = s_last < 0 ? 0 : s_last;
        long long i0 = upper_bound_g<OffT>(row_ptr, 0, R + 1, kt0) - 1;
        sh[4] = i0 < 0 ? 0 : (i0 > R - 1 ? R - 1 : i0);
    }
    __syncthreads();
    for (int d = tid; d < nbins; d += SA_THREADS) {
        cur[d] += (uint32_t)bucket_base[d << p2];
        if (want_pp) {
            // destination blocks of the super-bucket's first and last columns
            const long long c0 = (long long)d << (p2 + bshift);
            const long long c1 = min(N, ((long long)(d + 1)) << (p2 + bshift)) - 1;
            long long lo = (pp_smem ? upper_bound_sm(pos_, 0, P + 1, c0) : upper_bound_ll(poff, 0, P + 1, c0)) - 1;
            long long hi = (pp_smem ? upper_bound_sm(pos_, 0, P + 1, c1) : upper_bound_ll(poff, 0, P + 1, c1)) - 1;
            lo = lo < 0 ? 0 : (lo >= P ? P - 1 : lo);
            hi = hi < lo ? lo : (hi >= P ? P - 1 : hi);
            sblk[d] = lo == hi ? (uint16_t)lo : SC_STRADDLE;
            // spanning exactly two blocks: the split column decides per cell
            slo[d] = (uint16_t)lo;
            shi[d] = (uint16_t)hi;
            sspl[d] = hi == lo + 1 ? (int32_t)min(pp_smem ? pos_[hi] : poff[hi], (long long)INT_MAX) : -1;
        }
    }
    const long long s_first = sh[0];
    const bool one_src = sh[1] == s_first;
    const long long wmask = (1LL << bshift) - 1;
    bool bad = false;

    for (long long s0 = kt0; s0 < kt1; s0 += SA_SUB) {
        const long long s1 = min(kt1, s0 + (long long)SA_SUB);
        const int n = (int)(s1 - s0);
        __syncthreads();
        const long long i0 = sh[4];
        // cache row_ptr[i0 ..]; count entries <= s1 - 1 (rows of this sub-chunk)
        // and <= s1 (the next sub-chunk's first row)
        const long long nload = min((long long)rowc, R + 1 - i0);
        for (long long r = tid; r < nload; r += SA_THREADS) rows[r] = (OffT)ldo<OffT>(row_ptr, i0 + r);
        __syncthreads();
        int le_last = 0, le_next = 0;
        for (int r0 = 0; r0 < nload; r0 += SA_THREADS) {
            const int r = r0 + tid;
            const long long v = r < nload ? (long long)rows[r] : LLONG_MAX;
            le_last += __syncthreads_count(v <= s1 - 1);
            le_next += __syncthreads_count(v <= s1);
        }
        const bool cached = le_last < nload;
        long long i1;
        if (cached) {
            i1 = i0 + le_last - 1;
        } else {
            if (tid == 0) sh[3] = upper_bound_g<OffT>(row_ptr, i0, R + 1, s1 - 1) - 1;
            __syncthreads();
            i1 = sh[3];
        }
        if (i1 < i0) i1 = i0;
        if (i1 > R - 1) i1 = R - 1;
        const long long nr = i1 - i0 + 2;
        __syncthreads();
        if (tid == 0) {
            long long nx = cached ? i0 + le_next - 1 : i1;
            if (!cached && s1 < kt1) nx = upper_bound_g<OffT>(row_ptr, i1, R + 1, s1) - 1;
            sh[4] = nx < 0 ? 0 : (nx > R - 1 ? R - 1 : nx);
        }
        // ---- A: build records (thread owns cells [x0, x0 + SA_IPT)); all loads
        // first; the records stay in registers until their staged positions are known
        const int x0 = tid * SA_IPT;
        const int cntc = min(SA_IPT, n - x0);
        Rec rk[SA_IPT];
        {
            uint32_t dg[SA_IPT];
            if (cntc > 0) {
                const long long k0 = s0 + x0;
                int cv[SA_IPT];
                long long cp[SA_IPT + 1];
                if (cntc == SA_IPT && ((reinterpret_cast<uintptr_t>(col + k0) & 15) == 0)) {
                    const int4 a = __ldcs(reinterpret_cast<const int4 *>(col + k0));
                    const int4 b = __ldcs(reinterpret_cast<const int4 *>(col + k0) + 1);
                    cv[0] = a.x; cv[1] = a.y; cv[2] = a.z; cv[3] = a.w;
                    cv[4] = b.x; cv[5] = b.y; cv[6] = b.z; cv[7] = b.w;
                } else {
#pragma unroll
                    for (int u = 0; u < SA_IPT; ++u) cv[u] = u < cntc ? __ldcs(col + k0 + u) : 0;
                }
#pragma unroll
                for (int u = 0; u <= SA_IPT; ++u) cp[u] = u <= cntc ? ldo<OffT>(cell_ptr, k0 + u) : 0;
                // row of the first cell, then a walk; positions relative to the
                // sub-chunk (32-bit: a sub-chunk has SA_SUB cells)
                int i;                      // row relative to i0
                long long nxt;              // start of row i + 1 (absolute)
                if (cached) {
                    int lo = 0, hi = (int)nr;
                    while (lo < hi) {
                        int mid = (lo + hi) >> 1;
                        if ((long long)rows[mid] <= k0) lo = mid + 1;
                        else hi = mid;
                    }
                    i = lo - 1;
                    nxt = (i + 1 < nr) ? (long long)rows[i + 1] : C;
                } else {
                    i = (int)(upper_bound_g<OffT>(row_ptr, i0, i1 + 2, k0) - 1 - i0);
                    nxt = ldo<OffT>(row_ptr, i0 + i + 1);
                }
                const int imax = (int)min(R - 1 - i0, (long long)INT_MAX);  // last row index, relative
                int nrel = (int)min(max(nxt - k0, -1LL), (long long)INT_MAX);  // next row start, relative to k0
                long long sp = s_first;
                if (want_pp && !one_src) while (sp < P - 1 && pc_tab[sp + 1] <= k0) ++sp;
#pragma unroll
                for (int u = 0; u < SA_IPT; ++u) {
                    if (u < cntc) {
                        const long long k = k0 + u;
                        while (nrel <= u && i < imax) {
                            ++i;
                            const long long nx = cached ? ((i + 1 < nr) ? (long long)rows[i + 1] : C)
                                                        : ldo<OffT>(row_ptr, i0 + i + 1);
                            nrel = (int)min(max(nx - k0, -1LL), (long long)INT_MAX);
                        }
                        int c = cv[u];
                        if ((unsigned)c >= (unsigned)N) { bad = true; c = c < 0 ? 0 : (int)(N - 1); }
                        long long st = cp[u], en = cp[u + 1];
                        if ((unsigned long long)st > (unsigned long long)V) { bad = true; st = st < 0 ? 0 : V; }
                        if (en < st || en > V) { bad = true; en = en > V ? V : st; }
                        const int irow = min(max(i, -(int)i0), imax) + (int)i0;  // in [0, R)
                        const uint32_t b = (uint32_t)c >> bshift;
                        const uint32_t d = b >> p2;
                        const unsigned long long len = (unsigned long long)(en - st);
                        const bool esc = len >= LEN_ESC;
                        Rec r;
                        r.i = (uint32_t)irow;
                        r.meta = pack_meta((uint32_t)c & (uint32_t)wmask, len);
                        r.start = (decltype(r.start))st;
                        if (p2 > 0) put_d2(r, b & mask2, bshift);
                        rk[u] = r;
                        dg[u] = d;
                        // value totals per super-bucket: the tile's P x P values, or
                        // the bucket totals of a single pass
                        if (!esc && (want_pp || p2 == 0)) atomicAdd(&tvs32[d], (uint32_t)len);
                        if (p2 == 0 && esc) atomicAdd(&bucket_vtot[b], len);
                        if (want_pp && (!one_src || esc || sblk[d] == SC_STRADDLE)) {
                            if (!one_src) while (sp < P - 1 && pc_tab[sp + 1] <= k) ++sp;
                            // destination block of the column: the super-bucket's, the
                            // side of its split column, else the bucket's or a search
                            long long dd;
                            const uint16_t lo = slo[d], hi = shi[d];
                            if (lo == hi) {
                                dd = lo;
                            } else if (hi == lo + 1) {
                                dd = c < sspl[d] ? lo : hi;
                            } else {
                                const uint16_t db = __ldg(dblock + b);
                                dd = db != SC_STRADDLE ? (long long)db
                                                       : (pp_smem ? upper_bound_sm(po_tab, 0, P + 1, c)
                                                                  : upper_bound_ll(po_tab, 0, P + 1, c)) - 1;
                            }
                            if (dd < 0) dd = 0;
                            if (dd >= P) dd = P - 1;
                            const bool by_tile = one_src && sblk[d] != SC_STRADDLE;
                            if (pp_smem && sp - s_first < 2 && !esc) {
                                // 32-bit counters per sub-chunk (< 2^16 cells x < 2^16 values),
                                // added to the tile's 64-bit ones after each sub-chunk
                                const int rowp = (int)(sp - s_first);
                                atomicAdd(&ppc32[(rowp * 2 + 0) * P + dd], 1u);
                                atomicAdd(&ppc32[(rowp * 2 + 1) * P + dd], (uint32_t)len);
                            } else {
                                if (!by_tile)
                                    atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[sp * P + dd]), 1ull);
                                if (!by_tile || esc)
                                    atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[sp * P + dd]), len);
                            }
                        }
                    }
                }
                // this thread's digits: 8 consecutive bytes, one 8-byte store
                unsigned long long packed = 0;
#pragma unroll
                for (int u = 0; u < SA_IPT; ++u)
                    if (u < cntc) packed |= (unsigned long long)(dg[u] & 0xFFu) << (8 * u);
                *reinterpret_cast<unsigned long long *>(dig + x0) = packed;
            }
        }
        __syncthreads();
        // ---- B: stable multisplit by super-bucket, staged in shared memory
        block_multisplit(dig, n, nbins, wcnt, bstart, spos, sdig, scratch);
        if (cntc > 0) {
            const uint4 ps = *reinterpret_cast<const uint4 *>(spos + x0);  // 8 positions
            const uint16_t pos8[SA_IPT] = {(uint16_t)(ps.x & 0xFFFF), (uint16_t)(ps.x >> 16),
                                           (uint16_t)(ps.y & 0xFFFF), (uint16_t)(ps.y >> 16),
                                           (uint16_t)(ps.z & 0xFFFF), (uint16_t)(ps.z >> 16),
                                           (uint16_t)(ps.w & 0xFFFF), (uint16_t)(ps.w >> 16)};
#pragma unroll
            for (int u = 0; u < SA_IPT; ++u)
                if (u < cntc) stg[pos8[u]] = rk[u];
        }
        __syncthreads();
        // ---- C: write the runs
        for (int pidx = tid; pidx < n; pidx += SA_THREADS) {
            const int d = sdig[pidx];
            const uint32_t g = cur[d] + ((uint32_t)pidx - bstart[d]);
            if (MGT_IN(hdr, g, C)) out[g] = stg[pidx];
        }
        __syncthreads();
        for (int d = tid; d < nbins; d += SA_THREADS) {
            const uint32_t c = bstart[d + 1] - bstart[d];
            cur[d] += c;
            tcnt[d] += c;
            tvs[d] += tvs32[d];
            tvs32[d] = 0;
        }
        if (pp_smem)
            for (int i = tid; i < 4 * P; i += SA_THREADS) {
                if (ppc32[i]) {
                    ppc[i] += ppc32[i];
                    ppc32[i] = 0;
                }
            }
    }
    __syncthreads();
    // tile totals: bucket value totals (single pass) and P x P by super-bucket
    for (int d = tid; d < nbins; d += SA_THREADS) {
        if (p2 == 0 && tvs[d]) atomicAdd(&bucket_vtot[d], tvs[d]);
        if (want_pp && one_src && sblk[d] != SC_STRADDLE && tcnt[d]) {
            if (pp_smem) {
                atomicAdd(&ppt[sblk[d]], (unsigned long long)tcnt[d]);
                atomicAdd(&ppt[P + sblk[d]], tvs[d]);
            } else {
                atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[s_first * P + sblk[d]]),
                          (unsigned long long)tcnt[d]);
                atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[s_first * P + sblk[d]]), tvs[d]);
            }
        }
    }
    __syncthreads();
    if (pp_smem) {
        for (int dd = tid; dd < P; dd += SA_THREADS) {
            if (ppt[dd]) {
                atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[s_first * P + dd]), ppt[dd]);
                atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[s_first * P + dd]), ppt[P + dd]);
            }
            for (int rowp = 0; rowp < 2; ++rowp) {
                const long long sp = s_first + rowp;
                const unsigned long long cc = ppc[(rowp * 2 + 0) * P + dd], vv = ppc[(rowp * 2 + 1) * P + dd];
                if (sp < P && (cc || vv)) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[sp * P + dd]), cc);
                    atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[sp * P + dd]), vv);
                }
            }
        }
    }
    if (__syncthreads_or(bad) && tid == 0) flag(hdr, ST_BADINPUT);
}

// K3b: one item = (super-bucket S, tile group g).  Its records are the
// contiguous K3a output for tiles [t0, t1) of S; they go to S's buckets at
// cursors bucket base + tile t0's offset inside the bucket.
struct Sb2Layout {
    size_t cur, bst, wcnt, vs, vs32, stg, dig, spos, sdig, scratch, misc, total;
};
template <typename Rec>
__host__ __device__ inline Sb2Layout sb2_layout(int nbins) {
    Sb2Layout L;
    size_t o = 0;
#define MGT_TAKE(field, bytes) L.field = o; o = (o + (size_t)(bytes) + 15) & ~size_t(15);
    MGT_TAKE(cur, (size_t)nbins * 4)
    MGT_TAKE(bst, (size_t)(nbins + 1) * 4)
    MGT_TAKE(wcnt, (size_t)(nbins + 1) * SA_WARPS * 4)
    MGT_TAKE(vs, (size_t)nbins * 8)
    MGT_TAKE(vs32, (size_t)nbins * 4)
    MGT_TAKE(stg, (size_t)SA_SUB * sizeof(Rec))
    MGT_TAKE(dig, (size_t)SA_SUB)
    MGT_TAKE(spos, (size_t)SA_SUB * 2)
    MGT_TAKE(sdig, (size_t)SA_SUB)
    MGT_TAKE(scratch, 48 * 4)
    MGT_TAKE(misc, 32)
#undef MGT_TAKE
    L.total = o;
    return L;
}

// Second-pass items of one matrix: (super-bucket, group of G tiles).
__host__ __device__ inline long long scatter2_items(const Params &p) {
    if (p.T == 0 || p.p2 == 0) return 0;
    return ((p.B + (1LL << p.p2) - 1) >> p.p2) * ((p.T + p.G - 1) / p.G);
}

template <typename OffT, typename Rec1, typename Rec, bool BATCH>
__global__ void __launch_bounds__(SA_THREADS, 2)
    k_scatter2(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    // items (super-bucket, tile group), dealt round-robin to the blocks
    Units<BATCH> U(m0, ba, blockIdx.x, gridDim.x);
    while (U.next([](const Mat &X) { return scatter2_items(X.p); })) {
    const Mat &M = *U.M;
    const Rec1 *__restrict__ in = reinterpret_cast<const Rec1 *>(M.ws.recs1);
    Rec *__restrict__ out = reinterpret_cast<Rec *>(M.ws.recs);
    const long long C = M.p.C, V = M.p.V, T = M.p.T;
    const int bshift = M.p.bshift, B = (int)M.p.B, p2 = M.p.p2, G = M.p.G;
    const uint32_t *__restrict__ cnt = M.ws.cnt;
    const unsigned long long *__restrict__ bucket_base = M.ws.bucket_base;
    const unsigned long long *__restrict__ bucket_tot = M.ws.bucket_tot;
    unsigned long long *bucket_vtot = M.ws.bucket_vtot;
    const void *cell_ptr = M.in.cell_ptr;
    DevHeader *hdr = M.ws.hdr;
    const Sb2Layout SL = sb2_layout<Rec>(1 << p2);
    uint32_t *cur = reinterpret_cast<uint32_t *>(smem + SL.cur);
    uint32_t *bst = reinterpret_cast<uint32_t *>(smem + SL.bst);
    uint32_t *wcnt = reinterpret_cast<uint32_t *>(smem + SL.wcnt);
    unsigned long long *vs = reinterpret_cast<unsigned long long *>(smem + SL.vs);
    uint32_t *vs32 = reinterpret_cast<uint32_t *>(smem + SL.vs32);  // per sub-chunk
    Rec *stg = reinterpret_cast<Rec *>(smem + SL.stg);
    uint8_t *dig = smem + SL.dig;
    uint16_t *spos = reinterpret_cast<uint16_t *>(smem + SL.spos);
    uint8_t *sdig = smem + SL.sdig;
    uint32_t *scratch = reinterpret_cast<uint32_t *>(smem + SL.scratch);
    unsigned long long *misc = reinterpret_cast<unsigned long long *>(smem + SL.misc);
    unsigned long long *lohi = misc + 1;
    const int tid = threadIdx.x;
    const int nbins = 1 << p2;
    const long long ngroups = (T + G - 1) / G;
    (void)hdr;
    {
        const unsigned long long it = U.j;
        const int S = (int)(it / ngroups);
        const long long g = (long long)(it % ngroups);
        const long long t0 = g * G, t1 = min(T, t0 + G);
        // record range of this item inside K3a's output for S
        if (tid < 64) {
            // warp 0: offset of tile t0 inside S; warp 1: of tile t1 (S's total at T)
            const long long tt = tid < 32 ? t0 : t1;
            uint32_t off = 0;
            for (int d = tid & 31; d < nbins; d += 32) {
                const int b = (S << p2) + d;
                if (b < B) off += tt < T ? cnt[tt * B + b] : (uint32_t)bucket_tot[b];
            }
            off = __reduce_add_sync(0xffffffffu, off);
            if ((tid & 31) == 0) lohi[tid >> 5] = bucket_base[S << p2] + off;
        }
        for (int d = tid; d < nbins; d += SA_THREADS) {
            const int b = (S << p2) + d;
            cur[d] = b < B ? (uint32_t)(bucket_base[b] + cnt[t0 * B + b]) : 0u;
            vs[d] = 0;
            vs32[d] = 0;
        }
        // the multisplit's counters start at zero (the layout depends on p2,
        // which may change between the matrices of a batch)
        for (int i = tid; i < (nbins + 1) * SA_WARPS; i += SA_THREADS) wcnt[i] = 0;
        __syncthreads();
        const unsigned long long lo = lohi[0], hi = lohi[1];
        for (unsigned long long s0 = lo; s0 < hi; s0 += SA_SUB) {
            const int n = (int)min((unsigned long long)SA_SUB, hi - s0);
            // all of this thread's loads in flight before any use
            // records in registers (striped: x = u * SA_THREADS + tid) until
            // their staged positions are known
            Rec1 rin[SA_IPT];
            Rec rk[SA_IPT];
#pragma unroll
            for (int u = 0; u < SA_IPT; ++u)
                if (u * SA_THREADS + tid < n) rin[u] = in[s0 + u * SA_THREADS + tid];
#pragma unroll
            for (int u = 0; u < SA_IPT; ++u) {
                const int x = u * SA_THREADS + tid;
                if (x < n) {
                    Rec1 r1 = rin[u];
                    const uint32_t d = take_d2(r1, bshift, p2);
                    rec_convert(r1, rk[u]);
                    const Rec &r = rk[u];
                    if ((r.meta & 0xFFFFu) != LEN_ESC) {
                        atomicAdd(&vs32[d], r.meta & 0xFFFFu);
                    } else if ((S << p2) + (int)d < B) {
                        atomicAdd(&bucket_vtot[(S << p2) + d], rec_len<OffT>(r.meta, r.start, cell_ptr, C, V));
                    }
                    dig[x] = (uint8_t)d;
                }
            }
            __syncthreads();
            block_multisplit(dig, n, nbins, wcnt, bst, spos, sdig, scratch);
#pragma unroll
            for (int u = 0; u < SA_IPT; ++u) {
                const int x = u * SA_THREADS + tid;
                if (x < n) stg[spos[x]] = rk[u];
            }
            __syncthreads();
            for (int p = tid; p < n; p += SA_THREADS) {
                const int l = sdig[p];
                const uint32_t q = cur[l] + ((uint32_t)p - bst[l]);
                if (MGT_IN(hdr, q, C)) out[q] = stg[p];
            }
            __syncthreads();
            for (int d = tid; d < nbins; d += SA_THREADS) {
                cur[d] += bst[d + 1] - bst[d];
                vs[d] += vs32[d];
                vs32[d] = 0;
            }
            __syncthreads();
        }
        for (int d = tid; d < nbins; d += SA_THREADS) {
            const int b = (S << p2) + d;
            if (b < B && vs[d]) atomicAdd(&bucket_vtot[b], vs[d]);
        }
        __syncthreads();
    }
    }
}

// Shared memory of the scatter pass; pp: with the P x P counter tables.
static size_t smem_scatter_pp(const Params &p, bool pp) {
    const int nbins = (int)((p.B + (1LL << p.p2) - 1) >> p.p2);
    const bool w1 = p.wide || p.wide_mid;
    const int P = pp ? p.P : 0;
    return p.o == 4 ? (w1 ? sa_layout<int32_t, RecW>(nbins, p.rowc, P).total
                          : sa_layout<int32_t, RecC>(nbins, p.rowc, P).total)
                    : (w1 ? sa_layout<int64_t, RecW>(nbins, p.rowc, P).total
                          : sa_layout<int64_t, RecC>(nbins, p.rowc, P).total);
}
static size_t smem_scatter(const Params &p) { return smem_scatter_pp(p, true); }
static size_t smem_scatter2(const Params &p) {
    return p.wide ? sb2_layout<RecW>(1 << p.p2).total : sb2_layout<RecC>(1 << p.p2).total;
}
size_t scatter_smem_bytes(const Params &p) {
    const size_t a = smem_scatter(p), b = smem_scatter2(p);
    return a > b ? a : b;
}

static long long grid_scatter(const Params &p, double) { return p.T; }
static long long grid_scatter2(const Params &p, double share) {
    const long long items = scatter2_items(p);
    if (items == 0) return 0;
    long long grid = (long long)(2.0 * sm_count() * share + 0.999);
    if (grid < 1) grid = 1;
    return items < grid ? items : grid;
}
static long long units_scatter2(const Params &p) { return scatter2_items(p); }
static long long full_scatter2(const Params &, long long total) {
    const long long g = 2LL * sm_count();
    return total < g ? total : g;
}

template <typename OffT, typename Rec1>
static cudaError_t launch_scatter_t(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                                    cudaStream_t st) {
    // one transpose that counts P x P elsewhere (or not at all): the lean
    // instantiation with its own, smaller shared memory
    // (a batch: every member of the launch shares scatter_counts_pp, its group key)
    const bool pp = scatter_counts_pp(m0.p) && (ba.n || m0.out.part_cells != nullptr);
    auto kern = ba.n ? (pp ? k_scatter<OffT, Rec1, true, true> : k_scatter<OffT, Rec1, true, false>)
                     : (pp ? k_scatter<OffT, Rec1, false, true> : k_scatter<OffT, Rec1, false, false>);
    // one transpose without P x P tables: its own, smaller shared memory (a
    // batch keeps the maximum over its members, which bounds the lean layout)
    if (!pp && !ba.n) smem = smem_scatter_pp(m0.p, false);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, SA_THREADS, smem, st>>>(m0, ba);
    return cudaGetLastError();
}

template <typename OffT, typename Rec1, typename Rec>
static cudaError_t launch_scatter2_t(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                                     cudaStream_t st) {
    auto kern2 = ba.n ? k_scatter2<OffT, Rec1, Rec, true> : k_scatter2<OffT, Rec1, Rec, false>;
    cudaError_t e = cudaFuncSetAttribute(kern2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern2<<<(unsigned)grid, SA_THREADS, smem, st>>>(m0, ba);
    return cudaGetLastError();
}

static cudaError_t launch_scatter(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                                  cudaStream_t st) {
    const Params &p = m0.p;
    const bool w1 = p.wide || p.wide_mid;
    if (p.o == 4)
        return w1 ? launch_scatter_t<int32_t, RecW>(m0, ba, grid, smem, st)
                  : launch_scatter_t<int32_t, RecC>(m0, ba, grid, smem, st);
    return w1 ? launch_scatter_t<int64_t, RecW>(m0, ba, grid, smem, st)
              : launch_scatter_t<int64_t, RecC>(m0, ba, grid, smem, st);
}

static cudaError_t launch_scatter2(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                                   cudaStream_t st) {
    const Params &p = m0.p;
    if (p.o == 4) {
        if (p.wide) return launch_scatter2_t<int32_t, RecW, RecW>(m0, ba, grid, smem, st);
        return p.wide_mid ? launch_scatter2_t<int32_t, RecW, RecC>(m0, ba, grid, smem, st)
                          : launch_scatter2_t<int32_t, RecC, RecC>(m0, ba, grid, smem, st);
    }
    if (p.wide) return launch_scatter2_t<int64_t, RecW, RecW>(m0, ba, grid, smem, st);
    return p.wide_mid ? launch_scatter2_t<int64_t, RecW, RecC>(m0, ba, grid, smem, st)
                      : launch_scatter2_t<int64_t, RecC, RecC>(m0, ba, grid, smem, st);
}

// ------------------------------------------------------------ K4 build work
// One block: value bases per bucket (exclusive prefix of bucket_vtot) and the
// sort work list.  A bucket with at most `ch` records (one sort cluster) is
// one item; a larger one is cut into ceil(n / chm) chunks that get
// cursor-matrix rows.
template <bool BATCH>
__global__ void __launch_bounds__(1024) k_build_work(const __grid_constant__ Mat m0, const BatchArgs ba) {
    __shared__ unsigned long long sc[4][33];
    __shared__ uint32_t huge[64];
    __shared__ int nhuge;
    const VBlock vb = vblock<BATCH>(m0, ba);
    const Mat &M = *vb.m;
    const long long B = M.p.B, ch = M.p.ch, chm = M.p.chm, V = M.p.V;
    const unsigned long long *bucket_tot = M.ws.bucket_tot, *bucket_base = M.ws.bucket_base,
                             *bucket_vtot = M.ws.bucket_vtot;
    unsigned long long *bucket_vbase = M.ws.bucket_vbase;
    WorkItem *items = M.ws.items;
    uint32_t *multi_items = M.ws.multi_items;
    MultiBucket *multi_buckets = M.ws.multi_buckets;
    DevHeader *hdr = M.ws.hdr;
    const unsigned long long max_items = M.p.max_items, max_rows = M.p.max_multi_rows,
                             max_mb = M.p.max_multi_buckets;
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    if (tid == 0) nhuge = 0;
    // Rounds of nt consecutive buckets (coalesced loads, one bucket per
    // thread): a block scan of four running sums -- values, items,
    // multi-chunk rows, multi-chunk buckets -- gives each bucket its value
    // base and the place of its items.  A bucket of one sort cluster is one
    // item, written here; a larger one gets its MultiBucket entry, and the
    // index of its first item is parked in multi_items[mc0] for the last
    // pass, which writes its chunks' items.  Writes past the plan's
    // capacities are skipped and reported at the end.
    unsigned long long cv = 0, ci = 0, cr = 0, cm = 0;  // carries (block-uniform)
    for (long long c0 = 0; c0 < B; c0 += nt) {
        const long long b = c0 + tid;
        const bool valid = b < B;
        unsigned long long n = 0, vt = 0, bb = 0, nch = 0;
        if (valid) {
            n = bucket_tot[b];
            vt = bucket_vtot[b];
            bb = bucket_base[b];
        }
        const bool big = valid && n > (unsigned long long)ch;
        if (big) nch = (n + chm - 1) / chm;
        unsigned long long x[4] = {vt, valid ? (big ? nch : 1ull) : 0ull, nch, big ? 1ull : 0ull};
        unsigned long long inc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            inc[q] = warp_inclusive_scan(x[q]);
            if (lane == 31) sc[q][warp] = inc[q];
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned long long v = lane < nw ? sc[q][lane] : 0ull;
                const unsigned long long vi = warp_inclusive_scan(v);
                sc[q][lane] = vi - v;
                if (lane == 31) sc[q][32] = vi;
            }
        }
        __syncthreads();
        const unsigned long long ev = cv + sc[0][warp] + inc[0] - x[0];
        const unsigned long long ei = ci + sc[1][warp] + inc[1] - x[1];
        const unsigned long long er = cr + sc[2][warp] + inc[2] - x[2];
        const unsigned long long em = cm + sc[3][warp] + inc[3] - x[3];
        if (valid) {
            bucket_vbase[b] = ev;
            if (!big) {
                if (ei < max_items) {
                    WorkItem it;
                    it.r0 = bb;
                    it.r1 = bb + n;
                    it.bucket = (uint32_t)b;
                    it.chunk = 0;
                    it.mc = ~0ull;
                    items[ei] = it;
                }
            } else if (em < max_mb && er + nch <= max_rows) {
                MultiBucket mb;
                mb.mc0 = er;
                mb.bucket = (uint32_t)b;
                mb.nch = (uint32_t)nch;
                multi_buckets[em] = mb;
                multi_items[er] = (uint32_t)ei;  // first item; the last pass completes the row
            }
        }
        cv += sc[0][32];
        ci += sc[1][32];
        cr += sc[2][32];
        cm += sc[3][32];
        __syncthreads();
    }
    const bool consistent = (hdr->status & ST_BADINPUT) == 0 && cv == (unsigned long long)V;
    const bool fits = consistent && ci <= max_items && cr <= max_rows && cm <= max_mb;
    // the chunks of multi-chunk buckets: one thread per bucket, the whole
    // block for the buckets of many chunks (the hot columns' buckets)
    auto chunk_items = [&](const MultiBucket &mb, unsigned long long h0, unsigned long long hs) {
        const unsigned long long n = bucket_tot[mb.bucket], bb = bucket_base[mb.bucket];
        const unsigned long long ri0 = multi_items[mb.mc0], nch = mb.nch;
        for (unsigned long long h = h0; h < nch; h += hs) {
            WorkItem it;
            it.r0 = bb + (n * h) / nch;
            it.r1 = bb + (n * (h + 1)) / nch;
            it.bucket = mb.bucket;
            it.chunk = (uint32_t)h;
            it.mc = mb.mc0 + h;
            items[ri0 + h] = it;
            multi_items[mb.mc0 + h] = (uint32_t)(ri0 + h);  // h = 0 rewrites the parked value
        }
    };
    if (fits) {
        for (unsigned long long m = tid; m < cm; m += nt) {
            const MultiBucket mb = multi_buckets[m];
            if (mb.nch > 64) {
                const int k = atomicAdd(&nhuge, 1);
                if (k < 64) {
                    huge[k] = (uint32_t)m;
                    continue;
                }
            }
            chunk_items(mb, 0, 1);
        }
        __syncthreads();
        const int nh = min(nhuge, 64);
        for (int k = 0; k < nh; ++k) chunk_items(multi_buckets[huge[k]], tid, nt);
    }
    if (tid == 0) {
        if (!consistent) flag(hdr, ST_BADINPUT);
        else if (!fits) flag(hdr, ST_OVERFLOW);
        hdr->n_items = fits ? ci : 0;
        hdr->n_multi_items = fits ? cr : 0;
        hdr->n_multi_buckets = fits ? cm : 0;
        hdr->max_items = max_items;  // bounds for debug-build checks
        hdr->max_rows = max_rows;
    }
}

static cudaError_t launch_build_work(const Mat &m0, const BatchArgs &ba, long long grid, size_t,
                                     cudaStream_t st) {
    (ba.n ? k_build_work<true> : k_build_work<false>)<<<(unsigned)grid, 1024, 0, st>>>(m0, ba);
    return cudaGetLastError();
}

const PhaseOps kBucketPhases[7] = {
    {"setup", grid_prep, smem_none, launch_prep, nullptr, nullptr},
    {"hist", grid_hist, smem_hist, launch_hist, nullptr, nullptr},
    {"scan_tiles", grid_scan_tiles, smem_none, launch_scan_tiles, nullptr, nullptr},
    {"scan_buckets", grid_one_if_buckets, smem_none, launch_scan_buckets, nullptr, nullptr},
    {"scatter", grid_scatter, smem_scatter, launch_scatter, nullptr, nullptr},
    {"scatter2", grid_scatter2, smem_scatter2, launch_scatter2, units_scatter2, full_scatter2},
    {"build_work", grid_one_if_buckets, smem_none, launch_build_work, nullptr, nullptr},
};

}  // namespace mgt
