// C ABI of the mgt library: plans, workspace layout and the launch sequence.
#include "mgt_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

namespace mgt {

static constexpr size_t SMEM_BUDGET = 227 * 1024;
static constexpr int BMAX = 32768;

int sm_count() {
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    std::call_once(once[dev], [dev] {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
        cached[dev] = n;
    });
    return cached[dev];
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

WsLayout layout_for(const Params &p) {
    WsLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align256(o + bytes);
        return r;
    };
    const int w = 1 << p.bshift;
    L.header = take(256);
    L.cnt = take((size_t)p.T * (size_t)p.B * 4);
    L.bucket_tot = take((size_t)p.B * 8);
    L.bucket_base = take((size_t)p.B * 8);
    L.bucket_vtot = take((size_t)p.B * 8);
    L.bucket_vbase = take((size_t)p.B * 8);
    L.items = take((size_t)p.max_items * sizeof(WorkItem));
    L.multi_items = take((size_t)p.max_multi_rows * 4);
    L.multi_buckets = take((size_t)p.max_multi_buckets * sizeof(MultiBucket));
    L.mc = take((size_t)p.max_multi_rows * (size_t)w * sizeof(Cursor));
    L.recs = take((size_t)p.C * (p.wide ? sizeof(RecW) : sizeof(RecC)));
    L.recs1 = take(p.p2 > 0 ? (size_t)p.C * (p.wide || p.wide_mid ? sizeof(RecW) : sizeof(RecC)) : 0);
    L.src = take((size_t)p.C * (p.wide ? 8 : 4));
    L.fallback = take((size_t)p.max_items * 4);
    L.pcoff = take((size_t)(p.P + 1) * 8);
    L.poff = take((size_t)(p.P + 1) * 8);
    L.dblock = take((size_t)p.B * 2);
    L.vblk = take(p.var ? (size_t)((p.C + VAR_TILE - 1) / VAR_TILE + 1) * 8 : 0);
    L.total = o;
    return L;
}

Ws ws_from(void *base, const WsLayout &L) {
    char *b = static_cast<char *>(base);
    Ws w;
    w.hdr = reinterpret_cast<DevHeader *>(b + L.header);
    w.cnt = reinterpret_cast<uint32_t *>(b + L.cnt);
    w.bucket_tot = reinterpret_cast<unsigned long long *>(b + L.bucket_tot);
    w.bucket_base = reinterpret_cast<unsigned long long *>(b + L.bucket_base);
    w.bucket_vtot = reinterpret_cast<unsigned long long *>(b + L.bucket_vtot);
    w.bucket_vbase = reinterpret_cast<unsigned long long *>(b + L.bucket_vbase);
    w.items = reinterpret_cast<WorkItem *>(b + L.items);
    w.multi_items = reinterpret_cast<uint32_t *>(b + L.multi_items);
    w.multi_buckets = reinterpret_cast<MultiBucket *>(b + L.multi_buckets);
    w.mc = reinterpret_cast<Cursor *>(b + L.mc);
    w.recs = b + L.recs;
    w.recs1 = b + L.recs1;
    w.src = b + L.src;
    w.fallback = reinterpret_cast<uint32_t *>(b + L.fallback);
    w.pcoff = reinterpret_cast<long long *>(b + L.pcoff);
    w.poff = reinterpret_cast<long long *>(b + L.poff);
    w.dblock = reinterpret_cast<uint16_t *>(b + L.dblock);
    w.vblk = reinterpret_cast<unsigned long long *>(b + L.vblk);
    return w;
}

static constexpr size_t SMEM_HALF = 113 * 1024;  // two CTAs per SM

// Largest cluster-sort capacity per CTA (multiple of 512, <= 8192) whose
// shared memory fits `budget`.
static int cap_for(Params p, int cs, int bshift, size_t budget) {
    p.cs = cs;
    p.bshift = bshift;
    for (int cap = 8192; cap >= 512; cap -= 512) {
        p.cap = cap;
        if (place_smem_bytes(p) <= budget) return cap;
    }
    return 0;
}
static int chm_for(Params p, int bshift) {
    p.bshift = bshift;
    for (int c = 8192; c >= 512; c -= 512) {
        p.chm = c;
        if (chunk_smem_bytes(p) <= SMEM_BUDGET) return c;
    }
    return 0;
}

static int ilog2_ceil(long long x) {
    int b = 0;
    while ((1LL << b) < x) ++b;
    return b;
}

// Fills the derived fields of p from the problem and the tile choice.
static int finish_params(Params &p) {
    const int w = 1 << p.bshift;
    p.B = p.N == 0 ? 0 : (p.N + w - 1) / w;
    if (p.B > BMAX) return MGT_EINVAL;
    if ((1 << (p.cs == 1 ? 0 : p.cs == 2 ? 1 : p.cs == 4 ? 2 : 3)) > w) return MGT_EINVAL;
    p.ch = (long long)p.cs * p.cap;
    p.chm = chm_for(p, p.bshift);
    if (p.chm < 512) return MGT_EINVAL;
    if (place_smem_bytes(p) > SMEM_BUDGET || chunk_scan_smem_bytes(p) > SMEM_BUDGET) return MGT_EINVAL;
    if (p.tile <= 0) {
        // T x B count matrix of at most 16M entries, and >= 2 tiles per SM when small
        long long need = (p.C * (long long)p.B + (1LL << 24) - 1) >> 24;
        long long t = 2048;
        while (t < need) t <<= 1;
        long long small = (p.C + 2LL * sm_count() - 1) / (2LL * sm_count());
        while (t < small && t < 32768) t <<= 1;
        if (t > 65536) t = 65536;
        p.tile = (int)t;
    }
    p.sub = 2048;
    {
        // bucket id bits: up to 8 in the first scatter pass, the rest (<= 6) in the second
        int bbits = 0;
        while ((1LL << bbits) < p.B) ++bbits;
        p.p2 = bbits > 8 ? bbits - 8 : 0;
        if (p.p2 > 8) return MGT_EINVAL;
        p.wide_mid = !p.wide && p.p2 > 0 && p.bshift + p.p2 > 16;
    }
    if (scatter_smem_bytes(p) > SMEM_BUDGET) return MGT_EINVAL;
    p.T = p.C == 0 ? 0 : (p.C + p.tile - 1) / p.tile;
    {
        // second-pass items of ~4K records: tiles per item
        const long long nS = (p.B + (1LL << p.p2) - 1) >> p.p2;
        const double per = p.T > 0 && nS > 0 ? (double)p.C / ((double)nS * (double)p.T) : 1.0;
        long long G = (long long)(4096.0 / (per > 1.0 ? per : 1.0));
        if (G < 1) G = 1;
        if (G > p.T && p.T > 0) G = p.T;
        p.G = (int)(G < 1 ? 1 : G);
    }
    p.max_multi_rows = p.C > p.ch ? p.C / p.chm + p.C / p.ch + 2 : 0;
    p.max_multi_buckets = p.C > p.ch ? p.C / p.ch + 1 : 0;
    p.max_items = p.B + p.max_multi_rows + 1;
    return MGT_OK;
}

static int check_desc(const mgt_desc *d) {
    if (!d) return MGT_EINVAL;
    if (d->n_rows < 0 || d->n_cols < 0 || d->n_cells < 0 || d->n_values < 0) return MGT_EINVAL;
    if (d->n_rows > 2147483647LL || d->n_cols > 2147483647LL) return MGT_EINVAL;
    if (d->offset_bytes != 4 && d->offset_bytes != 8) return MGT_EINVAL;
    if (d->offset_bytes == 4 && (d->n_cells > 2147483647LL || d->n_values > 2147483647LL))
        return MGT_EINVAL;
    if (d->n_cells >= (1LL << 32)) return MGT_EINVAL;  // per-bucket offsets are 32-bit
    if (d->n_values >= (1LL << 48)) return MGT_EINVAL; // record start offsets carry 48 bits
    if ((d->flags & ~MGT_FLAG_VAR_WIDTH) != 0) return MGT_EINVAL;
    if (d->flags & MGT_FLAG_VAR_WIDTH) {
        if (d->payload_stride != 1) return MGT_EINVAL;  // values are measured in bytes
    } else if (d->payload_stride <= 0 || (d->payload_stride % 4) != 0) {
        return MGT_EINVAL;
    }
    if (d->n_parts < 1 || d->n_parts > 65535) return MGT_EINVAL;
    if (d->n_parts > 1 && d->n_rows != d->n_cols) return MGT_EINVAL;
    if (d->n_cells > 0 && (d->n_rows == 0 || d->n_cols == 0)) return MGT_EINVAL;
    if (d->n_values > 0 && d->n_cells == 0) return MGT_EINVAL;
    if (d->part_off) {
        if (d->part_off[0] != 0 || d->part_off[d->n_parts] != d->n_rows) return MGT_EINVAL;
        for (int i = 0; i < d->n_parts; ++i)
            if (d->part_off[i + 1] < d->part_off[i]) return MGT_EINVAL;
    }
    return MGT_OK;
}

static void base_params(const mgt_desc *d, Params &p) {
    memset(&p, 0, sizeof(p));
    p.R = d->n_rows;
    p.N = d->n_cols;
    p.C = d->n_cells;
    p.V = d->n_values;
    p.o = d->offset_bytes;
    p.s = d->payload_stride;
    p.P = d->n_parts;
    p.wide = d->n_values >= (1LL << 32) ? 1 : 0;
    p.var = (d->flags & MGT_FLAG_VAR_WIDTH) ? 1 : 0;
    p.nbytes = 0;
    p.rowc = 256;
    p.unroll = 2;
}

// Default tile choice: the smallest sort cluster (one CTA first: no
// ownership exchange between CTAs, and skewed buckets go to the chunked
// path instead of an overflowing owner), two sort CTAs per SM when the
// buckets fit, and the widest buckets whose expected size stays below 80% of
// the cluster's capacity.
static int choose_tiles(const mgt_desc *d, Params &p) {
    const double avg = d->n_cols > 0 ? (double)d->n_cells / (double)d->n_cols : 0.0;
    for (int cs = 1; cs <= 8; cs <<= 1) {
        for (size_t budget : {SMEM_HALF, SMEM_BUDGET}) {
            for (int bs = 12; bs >= 0; --bs) {
                const int w = 1 << bs;
                if (cs > w) break;
                if (d->n_cols > 0 && (d->n_cols + w - 1) / w > BMAX) break;
                const double wn = d->n_cols < w ? (double)d->n_cols : (double)w;
                const int cap = cap_for(p, cs, bs, budget);
                if (cap < 512) continue;
                if (avg * wn <= 0.8 * (double)cs * cap || bs == 0) {
                    Params q = p;
                    q.bshift = bs;
                    q.cs = cs;
                    q.cap = cap;
                    if (finish_params(q) != MGT_OK) continue;
                    p.bshift = bs;
                    p.cs = cs;
                    p.cap = cap;
                    return MGT_OK;
                }
            }
        }
    }
    // dense inputs: smallest bucket the scatter allows, largest cluster
    const int bs = std::max(3, ilog2_ceil((d->n_cols + BMAX - 1) / BMAX));
    p.bshift = bs;
    p.cs = 8;
    p.cap = cap_for(p, 8, bs, SMEM_BUDGET);
    return p.cap >= 512 ? MGT_OK : MGT_EINVAL;
}

// Parameters of the default plan for a descriptor, without creating a plan.
int default_params(const mgt_desc *d, Params *p) {
    int rc = check_desc(d);
    if (rc != MGT_OK) return rc;
    base_params(d, *p);
    rc = choose_tiles(d, *p);
    if (rc != MGT_OK) return rc;
    return finish_params(*p);
}

static thread_local char g_last_error[256];

int note_cuda(cudaError_t e, const char *where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e),
             cudaGetErrorString(e));
    return MGT_ECUDA;
}

const PhaseOps &phase_op(int i) {
    if (i < 7) return kBucketPhases[i];
    if (i < 12) return kPlacePhases[i - 7];
    return i == 12 ? kPartsPhase : kPlacePhases[5];
}

const char *const kPhaseNames[kPhases] = {
    "setup", "hist", "scan_tiles", "scan_buckets", "scatter", "scatter2", "build_work", "chunk_hist",
    "chunk_scan", "place", "place_chunks", "place_fallback", "part_counts", "copy"};

int enqueue_kernels(const Params &p, const Inputs &I, const Outputs &O, const Ws &ws,
                    cudaStream_t st, cudaEvent_t *ev, int first, int last) {
    const Mat m{p, I, O, ws};
    const BatchArgs alone{nullptr, nullptr, nullptr, 0};
    for (int i = first; i < last; ++i) {
        const PhaseOps &op = phase_op(i);
        const long long g = op.grid(p, 1.0);
        if (g > 0) {
            const cudaError_t e = op.launch(m, alone, g, op.smem(p), st);
            if (e != cudaSuccess) return note_cuda(e, op.name);
        }
        if (ev && cudaEventRecord(ev[i + 1], st) != cudaSuccess) return MGT_ECUDA;
    }
    return MGT_OK;
}

// Kernel launches one transpose makes (memsets and the offsets copy excluded).
int kernel_launches(const Params &p) {
    int n = 0;
    for (int i = 0; i < kPhases; ++i) n += phase_op(i).grid(p, 1.0) > 0 ? 1 : 0;
    return n;
}

}  // namespace mgt

using namespace mgt;

int mgt::check_call(const mgt_plan_t *plan, const mgt_xcsr_in *in, const mgt_xcsr_out *out,
                      const void *workspace, size_t workspace_bytes) {
    if (!plan || !in || !out || !workspace) return MGT_EINVAL;
    if (workspace_bytes < plan->L.total) return MGT_ENOMEM;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return MGT_EINVAL;
    const Params &p = plan->p;
    if (!in->row_ptr || !in->cell_ptr || !out->row_ptr || !out->cell_ptr) return MGT_EINVAL;
    if (p.C > 0 && (!in->col_idx || !out->col_idx)) return MGT_EINVAL;
    if (!p.var && p.V > 0 && (!in->values || !out->values)) return MGT_EINVAL;
    if ((out->part_cells == nullptr) != (out->part_values == nullptr)) return MGT_EINVAL;
    return MGT_OK;
}

extern "C" {

const char *mgt_version(void) { return "mgt 0.1 (sm_103a)"; }

const char *mgt_last_error(void) { return mgt::g_last_error; }

const char *mgt_strerror(int code) {
    switch (code) {
    case MGT_OK: return "ok";
    case MGT_EINVAL: return "invalid argument or descriptor";
    case MGT_ENOMEM: return "out of memory or workspace too small";
    case MGT_EBADINPUT: return "malformed XCSR input detected on the device";
    case MGT_ETIMEOUT: return "a bounded device wait expired";
    case MGT_EAGAIN: return "admission refused, retry later";
    case MGT_ECUDA: return "CUDA runtime error";
    case MGT_EOVERFLOW: return "an internal per-tile limit was exceeded";
    case MGT_ENOTFOUND: return "unknown ticket";
    default: return "unknown error";
    }
}

int64_t mgt_minimal_bytes(const mgt_desc *d) {
    if (check_desc(d) != MGT_OK) return -1;
    const int64_t o = d->offset_bytes, C = d->n_cells, V = d->n_values, s = d->payload_stride;
    const int64_t side = 4 * C + (C + 1) * o +
                         ((d->flags & MGT_FLAG_VAR_WIDTH) ? 8 * (V + 1) : V * s);
    return (d->n_rows + 1) * o + side + (d->n_cols + 1) * o + side;
}

static int make_plan(const mgt_desc *desc, const mgt_tile_cfg *cfg, mgt_plan_t **out,
                     size_t *ws_bytes) {
    if (!out) return MGT_EINVAL;
    *out = nullptr;
    int rc = check_desc(desc);
    if (rc != MGT_OK) return rc;
    Params p;
    base_params(desc, p);
    if (cfg && cfg->bucket_shift > 0) {
        if (cfg->bucket_shift > 16) return MGT_EINVAL;
        p.bshift = cfg->bucket_shift;
    }
    if (cfg && cfg->cluster) {
        if (cfg->cluster != 1 && cfg->cluster != 2 && cfg->cluster != 4 && cfg->cluster != 8)
            return MGT_EINVAL;
    }
    if (cfg && cfg->copy_unroll) {
        if (cfg->copy_unroll != 1 && cfg->copy_unroll != 2 && cfg->copy_unroll != 4) return MGT_EINVAL;
        p.unroll = cfg->copy_unroll;
    }
    if (!cfg || (cfg->bucket_shift == 0 && cfg->cluster == 0 && cfg->chunk_cap == 0)) {
        rc = choose_tiles(desc, p);
        if (rc != MGT_OK) return rc;
    } else {
        if (cfg->bucket_shift == 0) {
            Params q = p;
            rc = choose_tiles(desc, q);
            if (rc != MGT_OK) return rc;
            p.bshift = q.bshift;
        }
        p.cs = cfg->cluster ? cfg->cluster : 8;
        if ((1 << p.bshift) < p.cs) return MGT_EINVAL;
        const int capmax = cap_for(p, p.cs, p.bshift, SMEM_BUDGET);
        p.cap = cfg->chunk_cap ? cfg->chunk_cap : capmax;
        if (p.cap < 512 || p.cap > capmax || (p.cap % 512) != 0) return MGT_EINVAL;
    }
    if (cfg && cfg->scatter_tile) {
        if (cfg->scatter_tile < 512 || (cfg->scatter_tile % 512) != 0 || cfg->scatter_tile > 262144)
            return MGT_EINVAL;
        p.tile = cfg->scatter_tile;
    }
    rc = finish_params(p);
    if (rc != MGT_OK) return rc;
    mgt_plan_t *plan = new (std::nothrow) mgt_plan_t;
    if (!plan) return MGT_ENOMEM;
    plan->desc = *desc;
    plan->desc.part_off = nullptr;
    plan->p = p;
    plan->L = layout_for(p);
    memset(&plan->cfg, 0, sizeof(plan->cfg));
    plan->cfg.bucket_shift = p.bshift;
    plan->cfg.scatter_tile = p.tile;
    plan->cfg.cluster = p.cs;
    plan->cfg.chunk_cap = p.cap;
    plan->cfg.copy_unroll = p.unroll;
    plan->part_off_pinned = nullptr;
    plan->pinned = cudaMallocHost((void **)&plan->part_off_pinned, (size_t)(p.P + 1) * 8) == cudaSuccess;
    if (!plan->pinned) {
        cudaGetLastError();  // no device here: keep the offsets in pageable memory
        plan->part_off_pinned = static_cast<long long *>(malloc((size_t)(p.P + 1) * 8));
        if (!plan->part_off_pinned) {
            delete plan;
            return MGT_ENOMEM;
        }
    }
    for (int dd = 0; dd <= p.P; ++dd)
        plan->part_off_pinned[dd] = desc->part_off ? desc->part_off[dd]
                                                   : (long long)(((__int128)dd * p.R) / p.P);
    plan->p.pp_out = parts_from_output(plan->p, plan->part_off_pinned) ? 1 : 0;
    *out = plan;
    if (ws_bytes) *ws_bytes = plan->L.total;
    return MGT_OK;
}

int mgt_plan(const mgt_desc *desc, mgt_plan_t **plan, size_t *workspace_bytes) {
    return make_plan(desc, nullptr, plan, workspace_bytes);
}

int mgt_plan_tuned(const mgt_desc *desc, const mgt_tile_cfg *cfg, mgt_plan_t **plan,
                   size_t *workspace_bytes) {
    return make_plan(desc, cfg, plan, workspace_bytes);
}

int mgt_plan_config(const mgt_plan_t *plan, mgt_tile_cfg *cfg) {
    if (!plan || !cfg) return MGT_EINVAL;
    *cfg = plan->cfg;
    return MGT_OK;
}

void mgt_plan_destroy(mgt_plan_t *plan) {
    if (!plan) return;
    if (plan->part_off_pinned) {
        if (plan->pinned) cudaFreeHost(plan->part_off_pinned);
        else free(plan->part_off_pinned);
    }
    delete plan;
}



// Enqueues the whole pipeline for one matrix.  With ev != nullptr, ev[0] is
// recorded first and ev[i + 1] after phase i.
static int enqueue_pipeline(const mgt_plan_t *plan, const Params &p, const Inputs &I,
                            const Outputs &O, void *ws_base, cudaStream_t st,
                            cudaEvent_t *ev = nullptr, int last = kPhases) {
    Ws ws = ws_from(ws_base, plan->L);
    cudaError_t e = cudaSuccess;
#define MGT_MARK(i)                                                        \
    if (ev && (e = cudaEventRecord(ev[i], st)) != cudaSuccess) return MGT_ECUDA;
    MGT_MARK(0)
    if ((e = cudaMemsetAsync(ws.hdr, 0, 256, st)) != cudaSuccess) return MGT_ECUDA;
    if (p.B > 0 && (e = cudaMemsetAsync(ws.bucket_vtot, 0, (size_t)p.B * 8, st)) != cudaSuccess)
        return MGT_ECUDA;
    if (O.part_cells && (e = cudaMemsetAsync(O.part_cells, 0, (size_t)p.P * p.P * 8, st)) != cudaSuccess)
        return MGT_ECUDA;
    if (O.part_values && (e = cudaMemsetAsync(O.part_values, 0, (size_t)p.P * p.P * 8, st)) != cudaSuccess)
        return MGT_ECUDA;
    if ((e = cudaMemcpyAsync(ws.poff, plan->part_off_pinned, (size_t)(p.P + 1) * 8,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return MGT_ECUDA;
    return enqueue_kernels(p, I, O, ws, st, ev, 0, last);
#undef MGT_MARK
}

static int enqueue_one(const mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out, void *ws_base,
                       cudaStream_t st, cudaEvent_t *ev = nullptr, int last = kPhases) {
    Inputs I{in->row_ptr, in->col_idx, in->cell_ptr, static_cast<const uint8_t *>(in->values), nullptr};
    Outputs O{out->row_ptr, out->col_idx, out->cell_ptr, static_cast<uint8_t *>(out->values),
              reinterpret_cast<long long *>(out->part_cells),
              reinterpret_cast<long long *>(out->part_values), nullptr};
    return enqueue_pipeline(plan, plan->p, I, O, ws_base, st, ev, last);
}

// One host-to-device or device-to-host copy of `bytes` (none when 0).
static int copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
    if (bytes == 0) return MGT_OK;
    const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, st);
    return e == cudaSuccess ? MGT_OK : note_cuda(e, kind == cudaMemcpyHostToDevice ? "upload" : "download");
}

// Events of one mgt_transpose_host call; released once their work completes.
struct CallEvents {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    int create() {
        for (auto &x : e) {
            const cudaError_t r = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
            if (r != cudaSuccess) return note_cuda(r, "event");
        }
        return MGT_OK;
    }
    ~CallEvents() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
};

// Records ev on `from` and makes `to` wait for it.
static int join(cudaEvent_t ev, cudaStream_t from, cudaStream_t to) {
    cudaError_t e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    return e == cudaSuccess ? MGT_OK : note_cuda(e, "stream join");
}


int mgt_plan_phases(const mgt_plan_t *plan, const char **names, int max_names) {
    if (!plan) return MGT_EINVAL;
    for (int i = 0; names && i < max_names && i < kPhases; ++i) names[i] = kPhaseNames[i];
    return kPhases;
}

int mgt_plan_kernel_launches(const mgt_plan_t *plan) {
    if (!plan) return MGT_EINVAL;
    return kernel_launches(plan->p);
}

int mgt_transpose_profiled(mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                           void *workspace, size_t workspace_bytes, mgt_stream_t stream,
                           void *const *events, int n_events) {
    int rc = check_call(plan, in, out, workspace, workspace_bytes);
    if (rc != MGT_OK) return rc;
    if (plan->p.var) return MGT_EINVAL;  // variable-width values: mgt_transpose_var
    if (!events || n_events < kPhases + 1) return MGT_EINVAL;
    cudaEvent_t ev[kPhases + 1];
    for (int i = 0; i <= kPhases; ++i) ev[i] = static_cast<cudaEvent_t>(events[i]);
    return enqueue_one(plan, in, out, workspace, static_cast<cudaStream_t>(stream), ev);
}

int mgt_transpose(mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out, void *workspace,
                  size_t workspace_bytes, mgt_stream_t stream) {
    int rc = check_call(plan, in, out, workspace, workspace_bytes);
    if (rc != MGT_OK) return rc;
    if (plan->p.var) return MGT_EINVAL;  // variable-width values: mgt_transpose_var
    return enqueue_one(plan, in, out, workspace, static_cast<cudaStream_t>(stream));
}

int mgt_transpose_host(mgt_plan_t *plan, const mgt_xcsr_in *host_in, mgt_xcsr_out *host_out,
                       const mgt_xcsr_buf *dev_in, mgt_xcsr_out *dev_out, void *workspace,
                       size_t workspace_bytes, mgt_stream_t stream, mgt_stream_t copy_stream) {
    if (!host_in || !host_out || !dev_in) return MGT_EINVAL;
    const mgt_xcsr_in din{dev_in->row_ptr, dev_in->col_idx, dev_in->cell_ptr, dev_in->values};
    int rc = check_call(plan, &din, dev_out, workspace, workspace_bytes);
    if (rc != MGT_OK) return rc;
    if (plan->p.var) return MGT_EINVAL;
    const Params &p = plan->p;
    if (!host_in->row_ptr || !host_in->cell_ptr || !host_out->row_ptr || !host_out->cell_ptr)
        return MGT_EINVAL;
    if (p.C > 0 && (!host_in->col_idx || !host_out->col_idx)) return MGT_EINVAL;
    if (p.V > 0 && (!host_in->values || !host_out->values)) return MGT_EINVAL;
    if ((host_out->part_cells == nullptr) != (host_out->part_values == nullptr)) return MGT_EINVAL;
    if (host_out->part_cells && !dev_out->part_cells) return MGT_EINVAL;
    const size_t o = (size_t)p.o;
    const size_t b_rp_in = (size_t)(p.R + 1) * o, b_rp_out = (size_t)(p.N + 1) * o;
    const size_t b_col = (size_t)p.C * 4, b_cp = (size_t)(p.C + 1) * o;
    const size_t b_val = (size_t)p.V * (size_t)p.s, b_pp = (size_t)p.P * (size_t)p.P * 8;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
    const bool overlap = cs != nullptr && cs != st;
    CallEvents ev;
    if (overlap && (rc = ev.create()) != MGT_OK) return rc;
    const cudaMemcpyKind up = cudaMemcpyHostToDevice, down = cudaMemcpyDeviceToHost;
#define MGT_DO(x)                       \
    if ((rc = (x)) != MGT_OK) return rc;
    // structure first: the first kernels need it
    MGT_DO(copy_async(dev_in->row_ptr, host_in->row_ptr, b_rp_in, up, st))
    MGT_DO(copy_async(dev_in->col_idx, host_in->col_idx, b_col, up, st))
    MGT_DO(copy_async(dev_in->cell_ptr, host_in->cell_ptr, b_cp, up, st))
    if (overlap) {
        // values behind the structure uploads, and after stream's earlier work
        // (a previous call's value copy may still read dev_in->values)
        MGT_DO(join(ev.e[0], st, cs))
        MGT_DO(copy_async(dev_in->values, host_in->values, b_val, up, cs))
        const cudaError_t e = cudaEventRecord(ev.e[1], cs);
        if (e != cudaSuccess) return note_cuda(e, "event");
    } else {
        MGT_DO(copy_async(dev_in->values, host_in->values, b_val, up, st))
    }
    // every phase but the value copy
    MGT_DO(enqueue_one(plan, &din, dev_out, workspace, st, nullptr, kPhases - 1))
    cudaStream_t ds = overlap ? cs : st;  // stream of the structure downloads
    if (overlap) {
        MGT_DO(join(ev.e[2], st, cs))
        const cudaError_t e = cudaStreamWaitEvent(st, ev.e[1], 0);
        if (e != cudaSuccess) return note_cuda(e, "stream join");
    }
    MGT_DO(enqueue_kernels(p, Inputs{din.row_ptr, din.col_idx, din.cell_ptr,
                                      static_cast<const uint8_t *>(din.values)},
                           Outputs{dev_out->row_ptr, dev_out->col_idx, dev_out->cell_ptr,
                                   static_cast<uint8_t *>(dev_out->values),
                                   reinterpret_cast<long long *>(dev_out->part_cells),
                                   reinterpret_cast<long long *>(dev_out->part_values)},
                           ws_from(workspace, plan->L), st, nullptr, kPhases - 1, kPhases))
    // the structure downloads need only the phases before the value copy
    MGT_DO(copy_async(host_out->row_ptr, dev_out->row_ptr, b_rp_out, down, ds))
    MGT_DO(copy_async(host_out->col_idx, dev_out->col_idx, b_col, down, ds))
    MGT_DO(copy_async(host_out->cell_ptr, dev_out->cell_ptr, b_cp, down, ds))
    if (host_out->part_cells) {
        MGT_DO(copy_async(host_out->part_cells, dev_out->part_cells, b_pp, down, ds))
        MGT_DO(copy_async(host_out->part_values, dev_out->part_values, b_pp, down, ds))
    }
    MGT_DO(copy_async(host_out->values, dev_out->values, b_val, down, st))
    if (overlap) MGT_DO(join(ev.e[3], cs, st))
#undef MGT_DO
    return MGT_OK;
}

int mgt_transpose_values(mgt_plan_t *plan, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                         void *workspace, size_t workspace_bytes, mgt_stream_t stream) {
    if (!plan || !in || !out || !workspace) return MGT_EINVAL;
    if (workspace_bytes < plan->L.total) return MGT_ENOMEM;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return MGT_EINVAL;
    const Params &p = plan->p;
    if (p.var) return MGT_EINVAL;
    if (!out->cell_ptr) return MGT_EINVAL;
    if (p.V > 0 && (!in->values || !out->values)) return MGT_EINVAL;
    // the structure (cell_ptr' and each run's source offset in the
    // workspace) is the previous full transpose's; only the copy runs
    const Ws ws = ws_from(workspace, plan->L);
    const Inputs I{in->row_ptr, in->col_idx, in->cell_ptr, static_cast<const uint8_t *>(in->values)};
    const Outputs O{out->row_ptr, out->col_idx, out->cell_ptr, static_cast<uint8_t *>(out->values),
                    reinterpret_cast<long long *>(out->part_cells),
                    reinterpret_cast<long long *>(out->part_values)};
    const Mat m{p, I, O, ws};
    const PhaseOps &op = phase_op(kPhases - 1);  // the value copy
    const long long g = op.grid(p, 1.0);
    if (g == 0) return MGT_OK;
    const cudaError_t e = op.launch(m, BatchArgs{nullptr, nullptr, nullptr, 0}, g, op.smem(p),
                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MGT_OK : note_cuda(e, op.name);
}

int mgt_transpose_var(mgt_plan_t *plan, const mgt_xcsr_in *in, const int64_t *in_val_off,
                      mgt_xcsr_out *out, int64_t *out_val_off, int64_t n_bytes, void *workspace,
                      size_t workspace_bytes, mgt_stream_t stream, void *const *events,
                      int n_events) {
    int rc = check_call(plan, in, out, workspace, workspace_bytes);
    if (rc != MGT_OK) return rc;
    if (!plan->p.var || !in_val_off || !out_val_off || n_bytes < 0) return MGT_EINVAL;
    if (n_bytes > 0 && (!in->values || !out->values)) return MGT_EINVAL;
    if (events && n_events < kPhases + 1) return MGT_EINVAL;
    cudaEvent_t ev[kPhases + 1];
    if (events)
        for (int i = 0; i <= kPhases; ++i) ev[i] = static_cast<cudaEvent_t>(events[i]);
    Params p = plan->p;
    p.nbytes = n_bytes;
    const Inputs I{in->row_ptr, in->col_idx, in->cell_ptr, static_cast<const uint8_t *>(in->values),
                   reinterpret_cast<const long long *>(in_val_off)};
    const Outputs O{out->row_ptr, out->col_idx, out->cell_ptr, static_cast<uint8_t *>(out->values),
                    reinterpret_cast<long long *>(out->part_cells),
                    reinterpret_cast<long long *>(out->part_values),
                    reinterpret_cast<long long *>(out_val_off)};
    return enqueue_pipeline(plan, p, I, O, workspace, static_cast<cudaStream_t>(stream),
                            events ? ev : nullptr);
}

int mgt_read_status(const void *workspace, mgt_stream_t stream) {
    if (!workspace) return MGT_EINVAL;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MGT_ECUDA;
    unsigned bits = 0;
    if (cudaMemcpy(&bits, workspace, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MGT_ECUDA;
    if (bits & ST_BADINPUT) return MGT_EBADINPUT;
    if (bits & (ST_OVERFLOW | ST_DEBUG_BOUNDS)) return MGT_EOVERFLOW;  // (the latter: debug builds only)
    if (bits & ST_TIMEOUT) return MGT_ETIMEOUT;
    return MGT_OK;
}

}  // extern "C"
