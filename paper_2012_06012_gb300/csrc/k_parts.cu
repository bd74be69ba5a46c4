// P x P cell and value counts from the transposed matrix (the metadata-count
// and value-count matrices of the paper's view swap, Sec. 3: how many cells
// and values source block s sends to destination block d).
//
// An output cell q belongs to destination block d when it lies in that
// block's output cell range [row_ptr'[off[d]], row_ptr'[off[d + 1]]); its
// source block is the block of its source row col_idx'[q].  So the counts
// need one sequential pass over col_idx' and cell_ptr' and P + 1 entries of
// row_ptr', with the counters of each tile of output cells in shared memory
// (a tile spans few destination blocks).  The planner picks this pass when
// the row blocks cut through many of the first scatter pass's super-buckets
// (there the scatter pass would have to find every cell's destination block
// on its own); otherwise the scatter pass counts per tile.
#include "mgt_internal.cuh"

namespace mgt {

constexpr int PC_THREADS = 512;
constexpr int PC_TILE = 65536;  // output cells per work unit
constexpr int PC_WIN = 4;       // destination blocks counted in shared memory per tile
constexpr int PC_TAB = 4096;    // entries of the row -> block table

__host__ __device__ inline long long parts_units(const Params &p) {
    return (p.pp_out && p.P > 1 && p.C > 0) ? (p.C + PC_TILE - 1) / PC_TILE : 0;
}

// Shared memory: off[P+1] and the output cell offsets co[P+1] of the blocks
// (int64); cell and value counters (u32) of the tile's first PC_WIN
// destination blocks, [PC_WIN][P]; a row -> block table (u16): entry k is the
// block of row k << tsh, so a lookup walks at most a few blocks.
__host__ __device__ inline size_t parts_smem(int P) {
    return (size_t)(P + 1) * 16 + (size_t)2 * PC_WIN * P * 4 + (size_t)PC_TAB * 2 + 64;
}

// A tile's cells are counted in 32-bit shared counters: at most PC_TILE
// cells, and runs shorter than 2^16 values (longer ones go straight to the
// global counters), so no counter overflows.
template <typename OffT, bool BATCH>
__global__ void __launch_bounds__(PC_THREADS) k_part_counts(const __grid_constant__ Mat m0, const BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    Units<BATCH> U(m0, ba, blockIdx.x, gridDim.x);
    const Mat *cur = nullptr;  // the matrix whose tables are in shared memory
    const int tid = threadIdx.x;
    while (U.next([](const Mat &X) {
        return (X.out.part_cells == nullptr || (X.ws.hdr->status & (ST_BADINPUT | ST_OVERFLOW)))
                   ? 0ull
                   : (unsigned long long)parts_units(X.p);
    })) {
        const Mat &M = *U.M;
        const int P = M.p.P;
        const long long C = M.p.C, R = M.p.R, N = M.p.N;
        long long *po = reinterpret_cast<long long *>(smem);
        long long *co = po + (P + 1);
        uint32_t *cnt = reinterpret_cast<uint32_t *>(co + (P + 1));
        uint32_t *val = cnt + PC_WIN * P;
        uint16_t *tab = reinterpret_cast<uint16_t *>(val + PC_WIN * P);
        long long *dfirst = reinterpret_cast<long long *>(
            reinterpret_cast<unsigned char *>(tab) + (((size_t)PC_TAB * 2 + 15) & ~size_t(15)));
        int tsh = 0;
        while ((R >> tsh) >= PC_TAB) ++tsh;
        if (cur != &M) {  // tables of this matrix (block-uniform: every thread has the same U.M)
            __syncthreads();
            for (int d = tid; d <= P; d += PC_THREADS) {
                const long long r0 = M.ws.poff[d];
                const long long r = r0 < 0 ? 0 : (r0 > N ? N : r0);
                po[d] = r0;
                co[d] = ldo<OffT>(M.out.row_ptr, r);
            }
            __syncthreads();
            for (int k = tid; k < PC_TAB; k += PC_THREADS) {
                const long long b = upper_bound_sm(po, 0, P + 1, (long long)k << tsh) - 1;
                tab[k] = (uint16_t)(b < 0 ? 0 : (b > P - 1 ? P - 1 : b));
            }
            cur = &M;
        }
        for (int x = tid; x < PC_WIN * P; x += PC_THREADS) { cnt[x] = 0; val[x] = 0; }
        const long long q0 = (long long)U.j * PC_TILE, q1 = min(C, q0 + PC_TILE);
        if (tid == 0) {
            const long long d = upper_bound_sm(co, 0, P + 1, q0) - 1;
            dfirst[0] = d < 0 ? 0 : (d > P - 1 ? P - 1 : d);
        }
        __syncthreads();
        const int32_t *__restrict__ ocol = M.out.col;
        const void *ocp = M.out.cell_ptr;
        long long *part_cells = M.out.part_cells, *part_values = M.out.part_values;
        const long long dA = dfirst[0];
        long long d = dA;
        // rounds of PC_U x PC_THREADS consecutive cells, all their loads in
        // flight first (the same trip count for every thread, so the
        // warp-wide votes below see all lanes)
        constexpr int PC_U = 4;
        for (long long base = q0; base < q1; base += (long long)PC_U * PC_THREADS) {
            long long iu[PC_U], lu[PC_U];
#pragma unroll
            for (int u = 0; u < PC_U; ++u) {
                const long long q = base + (long long)u * PC_THREADS + tid;
                iu[u] = 0;
                lu[u] = 0;
                if (q < q1) {
                    iu[u] = ocol[q];
                    lu[u] = ldo<OffT>(ocp, q + 1) - ldo<OffT>(ocp, q);
                }
            }
#pragma unroll
            for (int u = 0; u < PC_U; ++u) {
                const long long q = base + (long long)u * PC_THREADS + tid;
                uint32_t key = 0xFFFFFFFFu, len32 = 0;
                if (q < q1) {
                    while (d < P - 1 && co[d + 1] <= q) ++d;  // cells of empty blocks: none
                    const long long i = iu[u] < 0 ? 0 : (iu[u] > R - 1 ? R - 1 : iu[u]);
                    long long s = tab[i >> tsh];  // block of the table row at or below i
                    while (s < P - 1 && po[s + 1] <= i) ++s;
                    const unsigned long long len = lu[u] > 0 ? (unsigned long long)lu[u] : 0ull;
                    const long long dl = d - dA;
                    if (dl < PC_WIN && len < 65536ull) {
                        key = (uint32_t)(dl * P + s);
                        len32 = (uint32_t)len;
                    } else {  // past the tile's window of blocks, or a very long run
                        atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[s * P + d]), 1ull);
                        atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[s * P + d]), len);
                    }
                }
                // consecutive output cells of a long (hot) output row come from
                // nearby source rows, so a warp there usually holds one key: one
                // counter update for the whole warp; otherwise one per lane
                const uint32_t k0 = __shfl_sync(0xffffffffu, key, 0);
                if (__all_sync(0xffffffffu, key == k0)) {
                    const unsigned sum = __reduce_add_sync(0xffffffffu, len32);
                    if (lane_id() == 0 && k0 != 0xFFFFFFFFu) {
                        atomicAdd(&cnt[k0], 32u);
                        atomicAdd(&val[k0], sum);
                    }
                } else if (key != 0xFFFFFFFFu) {
                    atomicAdd(&cnt[key], 1u);
                    atomicAdd(&val[key], len32);
                }
            }
        }
        __syncthreads();
        for (int x = tid; x < PC_WIN * P; x += PC_THREADS) {
            if (cnt[x] == 0) continue;
            const long long dd = dA + x / P, s = x % P;
            if (dd >= P) continue;
            atomicAdd(reinterpret_cast<unsigned long long *>(&part_cells[s * P + dd]),
                      (unsigned long long)cnt[x]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&part_values[s * P + dd]),
                      (unsigned long long)val[x]);
        }
        __syncthreads();
    }
}

static long long grid_parts(const Params &p, double share) {
    const long long u = parts_units(p);
    if (u == 0) return 0;
    long long g = (long long)((p.P <= 512 ? 4.0 : 2.0) * sm_count() * share + 0.999);
    if (g < 1) g = 1;
    return u < g ? u : g;
}
static size_t smem_parts(const Params &p) { return p.pp_out ? parts_smem(p.P) : 0; }
static long long units_parts(const Params &p) { return parts_units(p); }
static long long full_parts(const Params &p, long long total) {
    const long long g = (p.P <= 512 ? 4LL : 2LL) * sm_count();
    return total < g ? (total < 1 ? 1 : total) : g;
}
static cudaError_t launch_parts(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                                cudaStream_t st) {
    if (ba.n == 0 && m0.out.part_cells == nullptr) return cudaSuccess;  // counts not asked for
    auto kern = m0.p.o == 4 ? (ba.n ? k_part_counts<int32_t, true> : k_part_counts<int32_t, false>)
                            : (ba.n ? k_part_counts<int64_t, true> : k_part_counts<int64_t, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, PC_THREADS, smem, st>>>(m0, ba);
    return cudaGetLastError();
}

const PhaseOps kPartsPhase = {"part_counts", grid_parts, smem_parts, launch_parts, units_parts, full_parts};

// Whether the planner hands the P x P counts to this pass: P within the
// shared-memory table, and at least one super-bucket of the first scatter
// pass in eight cut by a row-block boundary (each of their cells would need
// a search in the scatter pass).
bool parts_from_output(const Params &p, const long long *off) {
    if (p.P <= 1 || p.P > PC_MAX_PARTS || p.B == 0 || !off) return false;
    const int sh = p.p2 + p.bshift;  // log2 of the columns of a super-bucket
    const long long nbins = (p.B + (1LL << p.p2) - 1) >> p.p2;
    long long cut = 0, last = -1;
    for (int d = 1; d < p.P; ++d) {
        const long long c = off[d];
        if (c <= 0 || c >= p.N || (c & ((1LL << sh) - 1)) == 0) continue;  // on a super-bucket edge
        const long long S = c >> sh;
        if (S != last) { ++cut; last = S; }
    }
    return cut * 8 >= nbins;
}

}  // namespace mgt
