// Batched transposes: every pipeline phase is one launch over all matrices of
// a batch.  Grid blocks are dealt to the members through a device table
// (BatchArgs); each member still gets its own workspace, so the members are
// exactly the independent transposes the single call computes.  A batch can
// be captured once into a CUDA graph and replayed.
#include "mgt_internal.cuh"

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

using namespace mgt;

namespace {

constexpr int kSteps = kPhases + 1;  // step 0: zeroing, step i + 1: phase i

size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

}  // namespace

// Members whose kernels instantiate the same templates share launches.
unsigned long long mgt::batch_group_key(const Params &p) {
    return (unsigned long long)p.o | ((unsigned long long)p.wide << 4) |
           ((unsigned long long)p.wide_mid << 5) | ((unsigned long long)p.cs << 8) |
           ((unsigned long long)p.unroll << 16) |
           ((unsigned long long)scatter_counts_pp(p) << 24);
}

namespace {

unsigned long long group_key(const Params &p) { return batch_group_key(p); }

struct Group {
    int first, count;             // members [first, first + count) of the sorted table
    long long grid[kSteps];       // blocks of the whole group for each step
    size_t smem[kSteps];          // dynamic shared memory per block (max over members)
    size_t bstart_off[kSteps];    // table-region offsets of the step's block starts
    size_t uprefix_off[kSteps];   // ... and of its unit prefix (persistent phases)
};

// Table region: Mat table, per (group, step) block starts (u32) and unit
// prefixes (u64), each with count + 1 entries (sum over groups <= 2n), then
// every member's row-block offsets.
size_t off_bstart(int n) { return align_up((size_t)n * sizeof(Mat), 256); }
size_t off_uprefix(int n) { return off_bstart(n) + align_up((size_t)kSteps * 2 * (size_t)(n + 1) * 4, 256); }
size_t off_poff(int n) { return off_uprefix(n) + align_up((size_t)kSteps * 2 * (size_t)(n + 1) * 8, 256); }

size_t table_bytes(int n, mgt_plan_t *const *plans) {
    size_t b = off_poff(n);
    for (int m = 0; m < n; ++m) b += align_up((size_t)(plans[m]->p.P + 1) * 8, 16);
    return align_up(b, 256);
}

long long work_of(const Params &p) {  // bytes one transpose moves, roughly
    return 2 * (p.R + p.N + 8 * p.C + p.V * (long long)p.s) + 1;
}

}  // namespace

struct mgt_batch_s {
    int n = 0;
    std::vector<Mat> mats;   // sorted by group key; mats[k] is member order[k]
    std::vector<int> order;
    std::vector<Group> groups;
    std::vector<unsigned char> blob;  // host image of the table region
    char *ws = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

namespace {

int build_batch(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                void *workspace, size_t workspace_bytes, mgt_batch_t *b) {
    size_t need = 0;
    int rc = mgt_batched_workspace(n, plans, &need);
    if (rc != MGT_OK) return rc;
    if (n < 1 || !in || !out || !workspace) return MGT_EINVAL;
    if (workspace_bytes < need) return MGT_ENOMEM;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return MGT_EINVAL;
    char *ws = static_cast<char *>(workspace);
    const size_t tb = table_bytes(n, plans);
    // members in group order (stable inside a group)
    std::vector<int> order(n);
    for (int m = 0; m < n; ++m) order[m] = m;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return group_key(plans[a]->p) < group_key(plans[c]->p);
    });
    const size_t off_tab = 0;
    size_t off_poffs = off_poff(n);
    std::vector<unsigned char> blob(tb, 0);
    b->mats.resize(n);
    b->order = order;
    // member workspaces after the table region, in call order
    std::vector<size_t> ws_off(n);
    size_t o = tb;
    for (int m = 0; m < n; ++m) {
        ws_off[m] = o;
        o += align_up(plans[m]->L.total, 256);
    }
    for (int k = 0; k < n; ++k) {
        const int m = order[k];
        const mgt_plan_t *pl = plans[m];
        rc = check_call(pl, &in[m], &out[m], ws + ws_off[m], pl->L.total);
        if (rc != MGT_OK) return rc;
        Mat &M = b->mats[k];
        M.p = pl->p;
        M.in = Inputs{in[m].row_ptr, in[m].col_idx, in[m].cell_ptr,
                      static_cast<const uint8_t *>(in[m].values)};
        M.out = Outputs{out[m].row_ptr, out[m].col_idx, out[m].cell_ptr,
                        static_cast<uint8_t *>(out[m].values),
                        reinterpret_cast<long long *>(out[m].part_cells),
                        reinterpret_cast<long long *>(out[m].part_values)};
        M.ws = ws_from(ws + ws_off[m], pl->L);
        // the member's row-block offsets live in the table region
        const size_t pbytes = (size_t)(pl->p.P + 1) * 8;
        memcpy(blob.data() + off_poffs, pl->part_off_pinned, pbytes);
        M.ws.poff = reinterpret_cast<long long *>(ws + off_poffs);
        off_poffs += align_up(pbytes, 16);
    }
    // groups, their per-step grids and block starts
    b->groups.clear();
    size_t bst = off_bstart(n), upo = off_uprefix(n);
    b->launches = 0;
    for (int k = 0; k < n;) {
        int e = k + 1;
        while (e < n && group_key(b->mats[e].p) == group_key(b->mats[k].p)) ++e;
        Group g{};
        g.first = k;
        g.count = e - k;
        long long work = 0;
        for (int q = k; q < e; ++q) work += work_of(b->mats[q].p);
        for (int s = 0; s < kSteps; ++s) {
            uint32_t *starts = reinterpret_cast<uint32_t *>(blob.data() + bst);
            unsigned long long *upre = reinterpret_cast<unsigned long long *>(blob.data() + upo);
            const PhaseOps *op = s == 0 ? nullptr : &phase_op(s - 1);
            long long run = 0;
            unsigned long long units = 0;
            size_t smem = 0;
            for (int q = k; q < e; ++q) {
                const Params &p = b->mats[q].p;
                const double share = (double)work_of(p) / (double)work;
                const long long gq = s == 0 ? grid_zero(p, share) : op->grid(p, share);
                const long long uq = (op && op->units) ? op->units(p) : 0;
                starts[q - k] = (uint32_t)run;
                upre[q - k] = units;
                run += gq;
                units += (unsigned long long)uq;
                if (gq > 0 && op) smem = std::max(smem, op->smem(p));
                if (run >= (1LL << 31)) return MGT_EINVAL;
            }
            starts[e - k] = (uint32_t)run;
            upre[e - k] = units;
            // persistent phases: one GPU-filling grid over all members' units
            if (op && op->units) run = units > 0 ? op->full_grid(b->mats[k].p, (long long)units) : 0;
            g.grid[s] = run;
            g.smem[s] = smem;
            g.bstart_off[s] = bst;
            g.uprefix_off[s] = upo;
            bst += (size_t)(e - k + 1) * 4;
            upo += (size_t)(e - k + 1) * 8;
            if (run > 0) ++b->launches;
        }
        b->groups.push_back(g);
        k = e;
    }
    if (bst > off_uprefix(n) || upo > off_poff(n)) return MGT_EINVAL;  // cannot happen: <= n groups
    memcpy(blob.data() + off_tab, b->mats.data(), (size_t)n * sizeof(Mat));
    b->blob.swap(blob);
    b->ws = ws;
    b->n = n;
    return MGT_OK;
}

// ev (optional, kSteps + 1 events): ev[0] before the first step, ev[s + 1]
// after step s (step 0 = zeroing, step i + 1 = phase i).
int enqueue_batch(const mgt_batch_t *b, cudaStream_t st, cudaEvent_t *ev = nullptr) {
    const Mat *tab = reinterpret_cast<const Mat *>(b->ws);
    if (ev && cudaEventRecord(ev[0], st) != cudaSuccess) return MGT_ECUDA;
    for (int s = 0; s < kSteps; ++s) {
        for (const Group &g : b->groups) {
            if (g.grid[s] == 0) continue;
            const BatchArgs ba{tab + g.first, reinterpret_cast<const uint32_t *>(b->ws + g.bstart_off[s]),
                               reinterpret_cast<const unsigned long long *>(b->ws + g.uprefix_off[s]),
                               g.count};
            const Mat &m0 = b->mats[g.first];
            const cudaError_t e = s == 0 ? launch_zero(m0, ba, g.grid[s], 0, st)
                                         : phase_op(s - 1).launch(m0, ba, g.grid[s], g.smem[s], st);
            if (e != cudaSuccess) return note_cuda(e, s == 0 ? "zero" : phase_op(s - 1).name);
        }
        if (ev && cudaEventRecord(ev[s + 1], st) != cudaSuccess) return MGT_ECUDA;
    }
    return MGT_OK;
}

void release(mgt_batch_t *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->exec = nullptr;
    b->graph = nullptr;
    b->cap_stream = nullptr;
}

}  // namespace

int mgt::batched_enqueue(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in,
                         mgt_xcsr_out *out, void *workspace, size_t workspace_bytes,
                         cudaStream_t st, void *staging, size_t staging_bytes) {
    if (n == 0) return MGT_OK;
    mgt_batch_t b;
    int rc = build_batch(n, plans, in, out, workspace, workspace_bytes, &b);
    if (rc != MGT_OK) return rc;
    if (!staging || staging_bytes < b.blob.size()) return MGT_EINVAL;
    memcpy(staging, b.blob.data(), b.blob.size());
    const cudaError_t e = cudaMemcpyAsync(b.ws, staging, b.blob.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return note_cuda(e, "batch tables");
    return enqueue_batch(&b, st);
}

size_t mgt::batched_table_bytes(int n, mgt_plan_t *const *plans) { return table_bytes(n, plans); }

size_t mgt::batched_table_bound(int n, int max_parts) {
    return align_up(off_poff(n) + (size_t)n * align_up((size_t)(max_parts + 1) * 8, 16), 256);
}

extern "C" {

int mgt_batched_workspace(int n, mgt_plan_t *const *plans, size_t *workspace_bytes) {
    if (n < 0 || (n > 0 && !plans) || !workspace_bytes) return MGT_EINVAL;
    for (int m = 0; m < n; ++m)
        if (!plans[m] || plans[m]->p.var) return MGT_EINVAL;  // variable-width plans: not batched
    size_t total = n > 0 ? table_bytes(n, plans) : 0;
    for (int m = 0; m < n; ++m) total += align_up(plans[m]->L.total, 256);
    *workspace_bytes = total;
    return MGT_OK;
}

int mgt_transpose_batched(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in,
                          mgt_xcsr_out *out, void *workspace, size_t workspace_bytes,
                          mgt_stream_t stream) {
    if (n == 0) return MGT_OK;
    mgt_batch_t b;
    int rc = build_batch(n, plans, in, out, workspace, workspace_bytes, &b);
    if (rc != MGT_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // pageable source: the call returns once the bytes are staged, so the
    // host image may go away with b
    if (cudaMemcpyAsync(b.ws, b.blob.data(), b.blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MGT_ECUDA;
    return enqueue_batch(&b, st);
}

int mgt_transpose_batched_profiled(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in,
                                   mgt_xcsr_out *out, void *workspace, size_t workspace_bytes,
                                   mgt_stream_t stream, void *const *events, int n_events) {
    if (!events || n_events < kSteps + 1) return MGT_EINVAL;
    if (n == 0) return MGT_OK;
    mgt_batch_t b;
    int rc = build_batch(n, plans, in, out, workspace, workspace_bytes, &b);
    if (rc != MGT_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(b.ws, b.blob.data(), b.blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return MGT_ECUDA;
    cudaEvent_t ev[kSteps + 1];
    for (int i = 0; i <= kSteps; ++i) ev[i] = static_cast<cudaEvent_t>(events[i]);
    return enqueue_batch(&b, st, ev);
}

int mgt_batch_create(int n, mgt_plan_t *const *plans, const mgt_xcsr_in *in, mgt_xcsr_out *out,
                     void *workspace, size_t workspace_bytes, mgt_batch_t **batch) {
    if (!batch) return MGT_EINVAL;
    *batch = nullptr;
    mgt_batch_t *b = new (std::nothrow) mgt_batch_t;
    if (!b) return MGT_ENOMEM;
    int rc = build_batch(n, plans, in, out, workspace, workspace_bytes, b);
    if (rc == MGT_OK &&
        cudaMemcpy(b->ws, b->blob.data(), b->blob.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = MGT_ECUDA;
    if (rc == MGT_OK &&
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = MGT_ECUDA;
    if (rc == MGT_OK) {
        // capture the whole launch sequence once
        if (cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rc = MGT_ECUDA;
        } else {
            const int erc = enqueue_batch(b, b->cap_stream);
            const cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &b->graph);
            if (erc != MGT_OK || ce != cudaSuccess) rc = MGT_ECUDA;
            else if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) rc = MGT_ECUDA;
        }
    }
    if (rc != MGT_OK) {
        cudaGetLastError();
        release(b);
        delete b;
        return rc;
    }
    *batch = b;
    return MGT_OK;
}

int mgt_batch_launch(mgt_batch_t *batch, mgt_stream_t stream) {
    if (!batch || !batch->exec) return MGT_EINVAL;
    return cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? MGT_OK
                                                                                       : MGT_ECUDA;
}

int mgt_batch_kernel_launches(const mgt_batch_t *batch) {
    if (!batch) return MGT_EINVAL;
    return batch->launches;
}

int mgt_batch_status(const mgt_batch_t *batch, mgt_stream_t stream, int *status) {
    if (!batch || !status) return MGT_EINVAL;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return MGT_ECUDA;
    int worst = MGT_OK;
    for (int k = 0; k < batch->n; ++k) {
        unsigned bits = 0;
        if (cudaMemcpy(&bits, batch->mats[k].ws.hdr, sizeof(bits), cudaMemcpyDeviceToHost) != cudaSuccess)
            return MGT_ECUDA;
        int rc = MGT_OK;
        if (bits & ST_BADINPUT) rc = MGT_EBADINPUT;
        else if (bits & (ST_OVERFLOW | ST_DEBUG_BOUNDS)) rc = MGT_EOVERFLOW;
        else if (bits & ST_TIMEOUT) rc = MGT_ETIMEOUT;
        status[batch->order[k]] = rc;
        if (rc != MGT_OK && worst == MGT_OK) worst = rc;
    }
    return worst;
}

void mgt_batch_destroy(mgt_batch_t *batch) {
    if (!batch) return;
    release(batch);
    delete batch;
}

}  // extern "C"
