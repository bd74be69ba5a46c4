// Internal declarations shared by the mgt kernels and the host library.
//
// Pipeline of one transpose (the paper's LocalTranspose o ViewSwap, Sec. 3,
// realised as a two-level stable counting sort by column):
//   K0 prep       validate pointers, source-block cell offsets, final sentinels
//   K1 hist       per scatter tile, cell counts per column bucket (shared-memory histogram)
//   K2 scan_tiles per bucket, exclusive prefix over tiles (stable tile order)
//   K2b scan_buckets bucket bases (exclusive prefix over buckets)
//   K3a scatter   stable scatter of 12/16-byte cell records into <= 256
//                 super-buckets (high bits of the bucket id); P x P counts (the
//                 view swap's count matrices, Sec. 3)
//   K3b scatter2  stable split of each super-bucket into its buckets
//   K4 build_work value bases per bucket and the sort work list
//   K5/K6         per-column counts and cursors for buckets larger than one cluster
//   K7a place     one thread-block cluster per bucket: records shuffled through
//                 distributed shared memory to the CTA owning their column range,
//                 stable in-shared-memory multisplit by column, coalesced output of
//                 row_ptr', col_idx', cell_ptr' and each run's source offset
//   K7b/K7c       oversized buckets (chunk cursors) and skewed buckets (fallback)
//   K8 copy       every value run, in output order, internal order kept
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mgt.h"

namespace mgt {

// ------------------------------------------------------------ status word
// First bytes of every workspace: error bits written by the kernels.
enum : unsigned {
    ST_BADINPUT = 1u,  // column out of range, decreasing pointers, wrong totals
    ST_OVERFLOW = 2u,  // an internal per-tile limit was exceeded
    ST_TIMEOUT = 4u,   // a bounded wait expired
    ST_DEBUG_BOUNDS = 8u,  // debug builds: an access outside its array was caught and skipped
};
struct DevHeader {
    unsigned status;
    unsigned pad0;
    unsigned long long item_counter;   // K7 work queue head
    unsigned long long item_counter2;  // second scatter pass work queue head
    unsigned long long n_items;        // written by K4
    unsigned long long n_multi_items;  // written by K4
    unsigned long long n_multi_buckets;// written by K4
    unsigned long long n_fallback;     // buckets K7a left to K7c
    unsigned long long dbg_line;       // debug builds: source line of the first bad access,
    unsigned long long dbg_index;      //   its index
    unsigned long long dbg_bound;      //   and the bound it broke
    unsigned long long max_items;      // written by K4: fallback list capacity (debug checks)
    unsigned long long max_rows;       // written by K4: cursor rows of the chunk path
    unsigned long long unused[4];
};
static_assert(sizeof(DevHeader) <= 256, "header");

// ------------------------------------------------------------ records
// A cell record carries what the sort and the copy need: source row i (the
// output column index), the start of the value run, the column inside its
// bucket and the run length (clamped at 0xFFFF; longer runs are recovered
// from cell_ptr by binary search).
constexpr uint32_t LEN_ESC = 0xFFFFu;
struct RecC { uint32_t i, start, meta; };            // 12 bytes, V < 2^32
struct RecW { uint32_t i, meta; unsigned long long start; };  // 16 bytes
__host__ __device__ inline uint32_t pack_meta(uint32_t cl, uint64_t len) {
    return (cl << 16) | (uint32_t)(len < LEN_ESC ? len : LEN_ESC);
}

// ------------------------------------------------------------ work items
struct WorkItem {
    unsigned long long r0, r1;  // record range (global record indices)
    unsigned long long mc;      // row of the chunk-cursor matrix, or ~0 for single-chunk buckets
    uint32_t bucket;
    uint32_t chunk;             // chunk index inside its bucket
};
struct MultiBucket {
    unsigned long long mc0;     // first cursor-matrix row
    uint32_t bucket, nch;
};
struct Cursor { unsigned long long a, b; };  // hist: (count, value sum); scan: (slot base, value base)

// ------------------------------------------------------------ launch params
struct Params {
    // problem
    int64_t R, N, C, V;
    int o;           // offset bytes
    int s;           // payload stride (1 for variable-width values)
    int P;
    int var;         // 1: variable-width values (byte offsets per value)
    int pp_out;      // 1: P x P counts by the pass over the output (else by the scatter pass)
    int64_t nbytes;  // variable-width values: total bytes (set per call)
    // tiles
    int bshift;      // log2 columns per bucket
    int64_t B;       // buckets
    int tile;        // cells per K1/K3 tile
    int sub;         // cells per K3 sub-chunk
    int64_t T;       // tiles
    int cs;          // cluster size
    int cap;         // records per K7 CTA
    int64_t ch;      // records a sort cluster takes = cs * cap
    int chm;         // records per chunk of an oversized bucket (one CTA)
    int p2;          // bits of the bucket id handled by the second scatter pass (0: one pass)
    int G;           // tiles per second-pass item
    bool wide_mid;   // wide records between the scatter passes (bshift + p2 > 16)
    int wide;        // 1: 16-byte records
    int unroll;      // copy unroll
    int rowc;        // K3 row-pointer cache entries
    // derived bounds
    int64_t max_items, max_multi_rows, max_multi_buckets;
};

struct WsLayout {
    size_t header, cnt, bucket_tot, bucket_base, bucket_vtot, bucket_vbase, items, multi_items,
        multi_buckets, mc, recs, recs1, src, fallback, pcoff, poff, dblock, vblk, total;
};

struct Inputs {
    const void *row_ptr;
    const int32_t *col;
    const void *cell_ptr;
    const uint8_t *values;
    const long long *val_off;  // variable-width values: byte offset of each value (V + 1)
};
struct Outputs {
    void *row_ptr;
    int32_t *col;
    void *cell_ptr;
    uint8_t *values;
    long long *part_cells, *part_values;
    long long *val_off;        // variable-width values: output byte offsets (V + 1)
};

// pointers into one workspace
struct Ws {
    DevHeader *hdr;
    uint32_t *cnt;          // [T][B]
    unsigned long long *bucket_tot, *bucket_base, *bucket_vtot, *bucket_vbase;
    WorkItem *items;
    uint32_t *multi_items;  // indices of multi-chunk items
    MultiBucket *multi_buckets;
    Cursor *mc;             // [rows][w]
    void *recs;
    void *recs1;            // records after the first scatter pass (super-bucket order)
    void *src;              // per output cell: start of its value run in the input
    uint32_t *fallback;     // items K7a could not place
    long long *pcoff;       // P+1 cell offsets of the source blocks
    long long *poff;        // P+1 row offsets
    uint16_t *dblock;       // [B] destination block of each bucket (0xFFFF: spans two)
    unsigned long long *vblk;  // variable-width values: per-tile words of the chained byte scan, then a tile counter
};

// One matrix's launch context: problem and tile choice, its buffers and its
// workspace.  A kernel takes it by value for one transpose, or finds it in a
// device table when one launch serves a batch of matrices (BatchArgs).
struct Mat {
    Params p;
    Inputs in;
    Outputs out;
    Ws ws;
};

// Batch launch.  Phases with per-matrix grids: blocks [bstart[i],
// bstart[i + 1]) work on tab[i] as if they were a grid of their own.
// Persistent phases: the work units (items, groups of cells) of all members
// back to back, member i owning units [uprefix[i], uprefix[i + 1]), dealt
// to the whole grid.  n = 0: one matrix, passed by value.
struct BatchArgs {
    const Mat *tab;
    const uint32_t *bstart;
    const unsigned long long *uprefix;
    int n;
};

// One pipeline phase: the blocks it needs for one matrix (0: nothing to do;
// `share` = the matrix's share of the GPU for persistent grids, 1 when
// alone), its dynamic shared memory per block, and its launch (template
// dispatch on m0's formats; grid and smem cover the whole batch).
// Persistent phases also give, per matrix, a host bound on their work units
// (units != nullptr) and the grid that fills the GPU for `total` units of a
// batch; their batch launches deal units instead of blocks.
struct PhaseOps {
    const char *name;
    long long (*grid)(const Params &p, double share);
    size_t (*smem)(const Params &p);
    cudaError_t (*launch)(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                          cudaStream_t st);
    long long (*units)(const Params &p);
    long long (*full_grid)(const Params &p, long long total);
};

WsLayout layout_for(const Params &p);
int default_params(const mgt_desc *d, Params *p);
Ws ws_from(void *base, const WsLayout &L);

// the pipeline, in order (phase 0 = setup); defined with the kernels
constexpr int kPhases = 14;
const PhaseOps &phase_op(int i);
extern const char *const kPhaseNames[kPhases];
int kernel_launches(const Params &p);
// phases 0-6 (k_bucket.cu), 7-11 (k_place.cu), 12 (k_parts.cu), 13: the
// value copy (k_place.cu, last entry of kPlacePhases)
extern const PhaseOps kBucketPhases[7];
extern const PhaseOps kPlacePhases[6];
extern const PhaseOps kPartsPhase;
// P x P counts from the output (k_parts.cu): up to this many row blocks, and
// whether a plan with these row-block offsets uses that pass.
constexpr int PC_MAX_PARTS = 2048;
bool parts_from_output(const Params &p, const long long *off);
// Zeroes what every transpose must start from (header, value totals, P x P
// counts) for a batch; one launch.
long long grid_zero(const Params &p, double share);
cudaError_t launch_zero(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                        cudaStream_t st);
size_t place_smem_bytes(const Params &p);
size_t chunk_scan_smem_bytes(const Params &p);
// The value copy of a variable-width plan (k_var.cu): per tile of VAR_TILE
// output cells, the runs' byte sizes, the tile's byte base by a chained scan
// over the tiles, then the byte copy and the output value offsets.
constexpr int VAR_TILE = 2048;
cudaError_t launch_var_copy(const Mat &m, cudaStream_t st);
size_t chunk_smem_bytes(const Params &p);
// The kernel sequence of one transpose (everything after the workspace
// header is cleared and the row-block offsets are in place).  ev: optional
// events, ev[i] recorded after phase i (phase 0 = prep).
// Phases [first, last) of one transpose on st (ev: optional per-phase events).
int enqueue_kernels(const Params &p, const Inputs &I, const Outputs &O, const Ws &ws,
                    cudaStream_t st, cudaEvent_t *ev, int first = 0, int last = kPhases);
size_t scatter_smem_bytes(const Params &p);
// Whether the scatter pass counts P x P for a plan (row blocks, and the
// output pass not chosen): batch members differing in it launch apart.
inline bool scatter_counts_pp(const Params &p) { return p.P > 1 && !p.pp_out; }

int sm_count();

}  // namespace mgt

struct mgt_plan_s {
    mgt_desc desc;
    mgt::Params p;
    mgt::WsLayout L;
    mgt_tile_cfg cfg;
    long long *part_off_pinned;  // P + 1 row offsets (pinned host memory when available)
    bool pinned;
};

namespace mgt {
// Remembers (per host thread) the last failed CUDA call for mgt_last_error;
// returns MGT_ECUDA.
int note_cuda(cudaError_t e, const char *where);
// Batched launches (mgt_batch.cu): the launch-group key of a plan, the size
// of a batch's table region, and an enqueue that stages the tables through
// caller-provided pinned host memory (never blocks the host).
unsigned long long batch_group_key(const Params &p);
size_t batched_table_bytes(int n, mgt_plan_t *const *plans);
size_t batched_table_bound(int n, int max_parts);  // any n members of <= max_parts blocks
int batched_enqueue(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                    void *workspace, size_t workspace_bytes, cudaStream_t st, void *staging,
                    size_t staging_bytes);
// Argument checks shared by the single and batched calls.
int check_call(const mgt_plan_t *plan, const mgt_xcsr_in *in, const mgt_xcsr_out *out,
               const void *workspace, size_t workspace_bytes);
}  // namespace mgt

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
namespace mgt {

template <typename OffT>
__device__ __forceinline__ long long ldo(const void *p, long long i) {
    return (long long)__ldg(reinterpret_cast<const OffT *>(p) + i);
}
template <typename OffT>
__device__ __forceinline__ void sto(void *p, long long i, long long v) {
    reinterpret_cast<OffT *>(p)[i] = (OffT)v;
}

__device__ __forceinline__ void flag(DevHeader *h, unsigned bit) { atomicOr(&h->status, bit); }

// Debug builds (-DMGT_DEBUG) check every index against its array before the
// access, record the first violation in the header (dbg_line, dbg_index,
// dbg_bound) and skip the access; release builds compile the checks away.
#ifdef MGT_DEBUG
__device__ __forceinline__ bool dbg_in(DevHeader *h, unsigned long long i, unsigned long long n,
                                       int line) {
    if (i < n) return true;
    if (atomicCAS(&h->dbg_line, 0ull, (unsigned long long)line) == 0ull) {
        h->dbg_index = i;
        h->dbg_bound = n;
    }
    atomicOr(&h->status, ST_DEBUG_BOUNDS);
    return false;
}
#define MGT_IN(h, i, n) dbg_in((h), (unsigned long long)(i), (unsigned long long)(n), __LINE__)
#else
#define MGT_IN(h, i, n) true
#endif

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// The matrix this block works on, and the block's index and the grid size
// within that matrix's share of the launch.
struct VBlock {
    const Mat *m;
    long long b, g;
};
// BATCH = false: the context is the kernel's own (grid-constant) parameter,
// read straight from the parameter bank.
template <bool BATCH>
__device__ __forceinline__ VBlock vblock(const Mat &m0, const BatchArgs &ba) {
    if constexpr (!BATCH) return VBlock{&m0, (long long)blockIdx.x, (long long)gridDim.x};
    int lo = 0, hi = ba.n;  // bstart[lo] <= blockIdx.x < bstart[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ba.bstart[mid] <= blockIdx.x) lo = mid;
        else hi = mid;
    }
    return VBlock{ba.tab + lo, (long long)(blockIdx.x - ba.bstart[lo]),
                  (long long)(ba.bstart[lo + 1] - ba.bstart[lo])};
}

// Work units of a persistent phase: j = first, first + stride, ... while
// j < count(matrix) for one matrix (count read from the device each time);
// in a batch, the units of all members back to back, each member's units
// at or beyond its own count skipped.  A caller's units only grow, so the
// member of the last unit (its unit range and count) is kept and the next
// unit usually falls in it or the member after it: no search per unit.
template <bool BATCH>
struct Units {
    const Mat &m0;
    const BatchArgs &ba;
    unsigned long long g, stride;
    const Mat *M = nullptr;
    unsigned long long j = 0;
    int lo = -1;                              // member of the last lookup (batch)
    unsigned long long lo_base = 0, lo_end = 0, lo_count = 0;
    unsigned long long end = ~0ull;           // batch: first unit not to take
    __device__ Units(const Mat &m0_, const BatchArgs &ba_, unsigned long long first,
                     unsigned long long stride_)
        : m0(m0_), ba(ba_), g(first), stride(stride_) {}
    template <typename CountFn>
    __device__ __forceinline__ bool next(CountFn count) {
        if constexpr (!BATCH) {
            if (g >= (unsigned long long)count(m0)) return false;
            M = &m0;
            j = g;
            g += stride;
            return true;
        } else {
            const unsigned long long all = ba.uprefix[ba.n], total = all < end ? all : end;
            for (; g < total; g += stride) {
                if (lo < 0 || g >= lo_end) {
                    if (lo >= 0 && lo + 2 <= ba.n && ba.uprefix[lo + 2] > g) {
                        ++lo;  // the member after the last one
                    } else {
                        int a = lo < 0 ? 0 : lo, b = ba.n;  // uprefix[a] <= g < uprefix[b]
                        while (b - a > 1) {
                            const int mid = (a + b) >> 1;
                            if (ba.uprefix[mid] <= g) a = mid;
                            else b = mid;
                        }
                        lo = a;
                    }
                    lo_base = ba.uprefix[lo];
                    lo_end = ba.uprefix[lo + 1];
                    lo_count = (unsigned long long)count(ba.tab[lo]);
                }
                const unsigned long long jj = g - lo_base;
                if (jj < lo_count) {
                    M = ba.tab + lo;
                    j = jj;
                    g += stride;
                    return true;
                }
            }
            return false;
        }
    }
};

// Lanes holding the same key as mine, a key being a value below nbins
// (nbins <= 256) or 0xFFFFFFFF for a lane without one, from one vote per key
// bit.  Its cost is the same whatever the keys, where the hardware peer
// match (__match_any_sync) takes longer the more distinct keys a warp holds:
// on the scatter passes' digits the votes are quicker.
__device__ __forceinline__ unsigned vote_peers(uint32_t key, int nbins) {
    const bool none = key == 0xFFFFFFFFu;
    unsigned m = __ballot_sync(0xffffffffu, none);
    if (!none) m = ~m;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if ((1 << b) < nbins) {
            const bool bit = (key >> b) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, bit);
            m &= bit ? bb : ~bb;
        }
    }
    return m;
}

// lanes whose `bits`-bit digit (bits <= 31) equals mine, among lanes with
// `valid` set (an invalid lane's own mask is meaningless)
__device__ __forceinline__ unsigned digit_peers(unsigned d, int bits, bool valid) {
    const unsigned key = valid ? (d & ((1u << bits) - 1u)) : 0xFFFFFFFFu;
    return __match_any_sync(0xffffffffu, key);
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T n = __shfl_up_sync(0xffffffffu, v, d);
        if (lane_id() >= d) v += n;
    }
    return v;
}

// In-place exclusive scan of a[0..n) in shared memory by the whole block;
// returns the total.  scratch: >= 33 elements of T in shared memory.
template <typename T>
__device__ T block_exclusive_scan(T *a, long long n, T *scratch) {
    const int nt = blockDim.x, tid = threadIdx.x;
    long long per = (n + nt - 1) / nt;
    long long lo = (long long)tid * per, hi = lo + per;
    if (lo > n) lo = n;
    if (hi > n) hi = n;
    T sum = 0;
    for (long long i = lo; i < hi; ++i) sum += a[i];
    T incl = warp_inclusive_scan(sum);
    if (lane_id() == 31) scratch[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        int nw = (nt + 31) >> 5;
        T v = tid < nw ? scratch[tid] : T(0);
        T vi = warp_inclusive_scan(v);
        scratch[tid] = vi - v;
        if (tid == 31) scratch[32] = vi;
    }
    __syncthreads();
    T run = scratch[tid >> 5] + incl - sum;
    for (long long i = lo; i < hi; ++i) {
        T x = a[i];
        a[i] = run;
        run += x;
    }
    T total = scratch[32];
    __syncthreads();
    return total;
}

// Per-(digit, warp) counters of a stable multisplit live warp-major with one
// word of padding per warp: index warp * (nbins + 1) + digit.  The leaders
// of one warp (distinct digits) and the threads of the scan below (one
// digit each) then fall on distinct banks.
__device__ __forceinline__ int wc_at(int digit, int warp, int nbins) {
    return warp * (nbins + 1) + digit;
}

// Turns the counters into exclusive offsets in (digit, warp) order -- the
// order that keeps equal digits in key order -- and writes each digit's
// first position to dstart[0..nbins] (dstart[nbins] = total).  scratch: >= 33
// words of shared memory.  Ends with a barrier.
__device__ __forceinline__ void wc_scan(uint32_t *wc, int nbins, int nwarps, uint32_t *dstart,
                                        uint32_t *scratch) {
    const int nt = blockDim.x, tid = threadIdx.x;
    for (int d = tid; d < nbins; d += nt) {
        uint32_t s = 0;
        for (int w = 0; w < nwarps; ++w) s += wc[w * (nbins + 1) + d];
        dstart[d] = s;
    }
    __syncthreads();
    const uint32_t total = block_exclusive_scan<uint32_t>(dstart, nbins, scratch);
    for (int d = tid; d < nbins; d += nt) {
        uint32_t run = dstart[d];
        for (int w = 0; w < nwarps; ++w) {
            const uint32_t x = wc[w * (nbins + 1) + d];
            wc[w * (nbins + 1) + d] = run;
            run += x;
        }
    }
    if (tid == 0) dstart[nbins] = total;
    __syncthreads();
}

// Stable LSD radix sort, in shared memory, of keys[0..n) by the key bits
// [lo_bit, lo_bit + nbits), DIGIT bits per pass.  Each warp ranks a
// contiguous segment with ballot-built peer masks; per-warp digit counts
// are scanned in (digit, warp) order, which keeps equal digits in input
// order.  whist: (1 << DIGIT) * warps uint32.  Returns the sorted buffer
// (k0 or k1).
template <int DIGIT>
__device__ uint32_t *block_radix_sort(uint32_t *k0, uint32_t *k1, int n, int lo_bit, int nbits,
                                      uint32_t *whist, uint32_t *scratch) {
    const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = lane_id();
    const int seg = (((n + nwarps - 1) / nwarps) + 31) & ~31;
    const int a = warp * seg, e = min(n, a + seg);
    for (int shift = lo_bit; shift < lo_bit + nbits; shift += DIGIT) {
        const int bits = min(DIGIT, lo_bit + nbits - shift);
        const int nb = 1 << bits;
        for (int i = threadIdx.x; i < nb * nwarps; i += blockDim.x) whist[i] = 0;
        __syncthreads();
        for (int base = a; base < e; base += 32) {
            int idx = base + lane;
            bool v = idx < e;
            unsigned d = v ? (k0[idx] >> shift) & (nb - 1) : 0u;
            unsigned peers = digit_peers(d, bits, v);
            if (v && (peers & lanemask_lt()) == 0) whist[d * nwarps + warp] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        block_exclusive_scan<uint32_t>(whist, (long long)nb * nwarps, scratch);
        for (int base = a; base < e; base += 32) {
            int idx = base + lane;
            bool v = idx < e;
            uint32_t key = v ? k0[idx] : 0u;
            unsigned d = (key >> shift) & (nb - 1);
            unsigned peers = digit_peers(d, bits, v);
            if (v) {
                uint32_t pos = whist[d * nwarps + warp] + __popc(peers & lanemask_lt());
                k1[pos] = key;
            }
            __syncwarp();
            if (v && (peers & lanemask_lt()) == 0) whist[d * nwarps + warp] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        uint32_t *t = k0;
        k0 = k1;
        k1 = t;
    }
    return k0;
}

// first index in [lo, hi) whose element is > key (OffT array in global memory)
template <typename OffT>
__device__ __forceinline__ long long upper_bound_g(const void *a, long long lo, long long hi,
                                                   long long key) {
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (ldo<OffT>(a, mid) <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ long long upper_bound_ll(const long long *a, long long lo, long long hi,
                                                    long long key) {
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (__ldg(a + mid) <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// same, for a table in shared memory (plain loads)
__device__ __forceinline__ long long upper_bound_sm(const long long *a, long long lo, long long hi,
                                                    long long key) {
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// true run length of a record (escape: search cell_ptr for the run's cell)
template <typename OffT>
__device__ __forceinline__ unsigned long long rec_len(uint32_t meta, unsigned long long start,
                                                      const void *cell_ptr, long long C, long long V) {
    uint32_t l = meta & 0xFFFFu;
    if (l != LEN_ESC) return l;
    if (C <= 0 || (long long)start >= V) return 0;
    long long k = upper_bound_g<OffT>(cell_ptr, 0, C + 1, (long long)start) - 1;
    if (k < 0) k = 0;
    if (k >= C) k = C - 1;
    long long end = ldo<OffT>(cell_ptr, k + 1);
    if (end > V) end = V;
    return end > (long long)start ? (unsigned long long)(end - (long long)start) : 0ull;
}

}  // namespace mgt
#endif
