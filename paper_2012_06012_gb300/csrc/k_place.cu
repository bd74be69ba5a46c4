// Dispatch of the level-2 phases (sort/place, the large-bucket chunk passes
// and the value copy) over offset width and record format, and their grid
// and shared-memory sizes.
#include "k_place_impl.cuh"

namespace mgt {

static cudaError_t level2(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                          cudaStream_t st, int which) {
    const Params &p = m0.p;
    if (p.o == 4)
        return p.wide ? launch_level2_t<int32_t, RecW>(m0, ba, grid, smem, st, which)
                      : launch_level2_t<int32_t, RecC>(m0, ba, grid, smem, st, which);
    return p.wide ? launch_level2_t<int64_t, RecW>(m0, ba, grid, smem, st, which)
                  : launch_level2_t<int64_t, RecC>(m0, ba, grid, smem, st, which);
}

size_t place_smem_bytes(const Params &p) {
    const int logcs = p.cs == 1 ? 0 : p.cs == 2 ? 1 : p.cs == 4 ? 2 : 3;
    const int wsub = 1 << (p.bshift - logcs);
    switch (p.cs) {
    case 1: return p.wide ? cl_layout<RecW, 1>(p.cap, wsub).total : cl_layout<RecC, 1>(p.cap, wsub).total;
    case 2: return p.wide ? cl_layout<RecW, 2>(p.cap, wsub).total : cl_layout<RecC, 2>(p.cap, wsub).total;
    case 4: return p.wide ? cl_layout<RecW, 4>(p.cap, wsub).total : cl_layout<RecC, 4>(p.cap, wsub).total;
    default: return p.wide ? cl_layout<RecW, 8>(p.cap, wsub).total : cl_layout<RecC, 8>(p.cap, wsub).total;
    }
}
size_t chunk_smem_bytes(const Params &p) {
    return p.wide ? ch_layout<RecW>(p.chm, 1 << p.bshift).total : ch_layout<RecC>(p.chm, 1 << p.bshift).total;
}

// persistent grids: the matrix's share of `per_sm` blocks per SM, at most `work`
static long long share_grid(double per_sm, double share, long long work) {
    long long g = (long long)(per_sm * sm_count() * share + 0.999);
    if (g < 1) g = 1;
    return work < g ? work : g;
}

// Sort clusters the cluster-place kernel can keep resident, for this plan
// (0 without a device: the grid then takes one cluster per SM pair).
static long long resident_clusters(const Params &p) {
    const size_t smem = place_smem_bytes(p);
    long long n = p.o == 4 ? (p.wide ? resident_clusters_t<int32_t, RecW>(p.cs, smem)
                                     : resident_clusters_t<int32_t, RecC>(p.cs, smem))
                           : (p.wide ? resident_clusters_t<int64_t, RecW>(p.cs, smem)
                                     : resident_clusters_t<int64_t, RecC>(p.cs, smem));
    if (n < 1) n = sm_count() / (p.cs > 1 ? p.cs : 1);
    return n < 1 ? 1 : n;
}

static long long grid_chunk(const Params &p, double share) {
    if (p.B == 0 || p.max_multi_rows == 0) return 0;
    return share_grid(2.0, share, p.max_multi_rows);
}
static long long grid_place(const Params &p, double share) {
    if (p.B == 0) return 0;
    long long ncl = (long long)(resident_clusters(p) * share + 0.999);
    if (ncl < 1) ncl = 1;
    if (ncl > p.max_items) ncl = p.max_items < 1 ? 1 : p.max_items;
    return ncl * p.cs;
}
static long long grid_place_chunks(const Params &p, double share) {
    if (p.B == 0 || p.max_multi_rows == 0) return 0;
    return share_grid(1.0, share, p.max_multi_rows);
}
static long long grid_fallback(const Params &p, double share) {
    if (p.B == 0) return 0;
    return share_grid(1.0, share, p.max_items);
}
static long long units_copy(const Params &p) {
    return (p.C == 0 || p.V == 0) ? 0 : (p.C + COPY_UNIT - 1) / COPY_UNIT;
}
static long long grid_copy(const Params &p, double share) {
    if (p.var) return 1;  // variable-width values: launch_var_copy sizes its own grids
    if (p.C == 0 || p.V == 0) return 0;
    // one warp per unit of COPY_UNIT cells
    return share_grid(4.0, share, (units_copy(p) + P_THREADS / 32 - 1) / (P_THREADS / 32));
}

static size_t smem_chunk_hist(const Params &p) {
    const size_t w = (size_t)1 << p.bshift;
    return w * 4 + 8 + w * 8;
}
static size_t smem_wide_scan(const Params &p) { return ((size_t)1 << p.bshift) * 16 + 48 * 8; }
static size_t smem_chunk_scan(const Params &p) { return chunk_scan_smem(p.bshift); }
size_t chunk_scan_smem_bytes(const Params &p) { return smem_chunk_scan(p); }
static size_t smem_place(const Params &p) { return place_smem_bytes(p); }
static size_t smem_chunk(const Params &p) { return chunk_smem_bytes(p); }
static size_t smem_zero(const Params &) { return 0; }

#define MGT_L2(fn, which)                                                                    \
    static cudaError_t fn(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem, \
                          cudaStream_t st) {                                                  \
        return level2(m0, ba, grid, smem, st, which);                                         \
    }
MGT_L2(launch_chunk_hist, 0)
MGT_L2(launch_chunk_scan, 1)
MGT_L2(launch_place, 2)
MGT_L2(launch_place_chunks, 3)
MGT_L2(launch_place_fallback, 4)
#undef MGT_L2
static cudaError_t launch_copy(const Mat &m0, const BatchArgs &ba, long long grid, size_t smem,
                               cudaStream_t st) {
    if (m0.p.var) return launch_var_copy(m0, st);  // single transposes only
    return level2(m0, ba, grid, smem, st, 5);
}

// Host bounds on the work units of the persistent phases (a batch deals
// them to one GPU-filling grid), and that grid for `total` units.
static long long units_multi_rows(const Params &p) { return p.B == 0 ? 0 : p.max_multi_rows; }
static long long units_multi_buckets(const Params &p) { return p.B == 0 ? 0 : p.max_multi_buckets; }
static long long units_items(const Params &p) { return p.B == 0 ? 0 : p.max_items; }
static long long cap_total(long long g, long long total) { return total < g ? (total < 1 ? 1 : total) : g; }
static long long full_two_per_sm(const Params &, long long total) { return cap_total(2LL * sm_count(), total); }
static long long full_one_per_sm(const Params &, long long total) { return cap_total(sm_count(), total); }
static long long full_place(const Params &p, long long total) {
    return cap_total(resident_clusters(p), total) * p.cs;
}
static long long full_copy(const Params &, long long total) {
    // units are warps: P_THREADS / 32 per block
    return cap_total(4LL * sm_count(), (total + P_THREADS / 32 - 1) / (P_THREADS / 32));
}

const PhaseOps kPlacePhases[6] = {
    {"chunk_hist", grid_chunk, smem_chunk_hist, launch_chunk_hist, units_multi_rows, full_two_per_sm},
    {"chunk_scan", grid_chunk, smem_chunk_scan, launch_chunk_scan, units_multi_buckets, full_two_per_sm},
    {"place", grid_place, smem_place, launch_place, units_items, full_place},
    {"place_chunks", grid_place_chunks, smem_chunk, launch_place_chunks, units_multi_rows, full_one_per_sm},
    {"place_fallback", grid_fallback, smem_wide_scan, launch_place_fallback, units_items, full_one_per_sm},
    {"copy", grid_copy, smem_zero, launch_copy, units_copy, full_copy},
};

}  // namespace mgt
