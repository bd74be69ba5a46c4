// Autotuner: times candidate tile shapes on the caller's own buffers and
// keeps the fastest.  The shapes change only how the work is cut (bucket
// width, sort cluster size, value-copy width); every candidate computes the
// same transpose, so tuning never changes a result.
#include "mgt_internal.cuh"

#include <vector>

using namespace mgt;

namespace {

bool valid(const mgt_desc *d, const mgt_tile_cfg &c, size_t *ws) {
    mgt_plan_t *p = nullptr;
    size_t w = 0;
    if (mgt_plan_tuned(d, &c, &p, &w) != MGT_OK) return false;
    mgt_plan_destroy(p);
    if (ws) *ws = w;
    return true;
}

// Coordinate search around the default plan: the default shape itself (its
// sort capacity may be the two-CTAs-per-SM one, which the shapes below,
// sized to the whole shared-memory budget, never take), then bucket width x
// cluster size (copy width fixed), then the copy width for the best of those.
std::vector<mgt_tile_cfg> stage1(const mgt_desc *d, const mgt_tile_cfg &base) {
    std::vector<mgt_tile_cfg> out;
    out.push_back(base);
    for (int db = -1; db <= 1; ++db) {
        for (int cs : {1, 2, 4, 8}) {
            mgt_tile_cfg c = {};
            c.bucket_shift = base.bucket_shift + db;
            c.cluster = cs;
            c.copy_unroll = base.copy_unroll;
            if (c.bucket_shift < 1 || c.bucket_shift > 16) continue;
            if (valid(d, c, nullptr)) out.push_back(c);
        }
    }
    return out;
}

}  // namespace

extern "C" {

int mgt_autotune_candidates(const mgt_desc *desc, mgt_tile_cfg *cands, int max) {
    if (desc && desc->flags) return MGT_EINVAL;  // fixed-width descriptors only
    mgt_plan_t *p = nullptr;
    int rc = mgt_plan(desc, &p, nullptr);
    if (rc != MGT_OK) return rc;
    mgt_tile_cfg base;
    mgt_plan_config(p, &base);
    mgt_plan_destroy(p);
    std::vector<mgt_tile_cfg> c = stage1(desc, base);
    for (int u : {1, 2, 4}) {
        if (u == base.copy_unroll) continue;
        mgt_tile_cfg x = base;
        x.copy_unroll = u;
        c.push_back(x);
    }
    const int n = (int)c.size();
    for (int i = 0; cands && i < n && i < max; ++i) cands[i] = c[i];
    return n;
}

int mgt_autotune_workspace(const mgt_desc *desc, size_t *bytes) {
    if (!bytes) return MGT_EINVAL;
    std::vector<mgt_tile_cfg> c(64);
    const int n = mgt_autotune_candidates(desc, c.data(), 64);
    if (n < 0) return n;
    size_t most = 0;
    for (int i = 0; i < n && i < 64; ++i) {
        size_t w = 0;
        if (valid(desc, c[i], &w) && w > most) most = w;
    }
    *bytes = most;
    return MGT_OK;
}

int mgt_autotune(const mgt_desc *desc, const mgt_xcsr_in *in, mgt_xcsr_out *out, void *workspace,
                 size_t workspace_bytes, mgt_stream_t stream, int reps, mgt_tile_cfg *best,
                 float *best_ms) {
    if (!desc || !in || !out || !workspace || !best || reps < 1 || desc->flags) return MGT_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mgt_plan_t *p0 = nullptr;
    int rc = mgt_plan(desc, &p0, nullptr);
    if (rc != MGT_OK) return rc;
    mgt_tile_cfg base;
    mgt_plan_config(p0, &base);
    mgt_plan_destroy(p0);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return note_cuda(cudaGetLastError(), "autotune");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return note_cuda(cudaGetLastError(), "autotune");
    }
    float best_t = -1.0f;
    mgt_tile_cfg best_c = base;
    // times one candidate: one warm-up, then `reps` runs between two events
    auto time_one = [&](const mgt_tile_cfg &c, float *ms) -> int {
        mgt_plan_t *p = nullptr;
        size_t w = 0;
        int r = mgt_plan_tuned(desc, &c, &p, &w);
        if (r != MGT_OK) return r;
        if (w > workspace_bytes) {
            mgt_plan_destroy(p);
            return MGT_ENOMEM;
        }
        r = mgt_transpose(p, in, out, workspace, workspace_bytes, stream);
        if (r == MGT_OK && cudaEventRecord(e0, st) != cudaSuccess) r = MGT_ECUDA;
        for (int k = 0; r == MGT_OK && k < reps; ++k)
            r = mgt_transpose(p, in, out, workspace, workspace_bytes, stream);
        if (r == MGT_OK && cudaEventRecord(e1, st) != cudaSuccess) r = MGT_ECUDA;
        if (r == MGT_OK && cudaEventSynchronize(e1) != cudaSuccess) r = MGT_ECUDA;
        if (r == MGT_OK) {
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            *ms = t / reps;
            r = mgt_read_status(workspace, stream);
        }
        mgt_plan_destroy(p);
        return r;
    };
    auto consider = [&](const mgt_tile_cfg &c) -> int {
        float t = 0;
        const int r = time_one(c, &t);
        if (r == MGT_ENOMEM) return MGT_OK;  // does not fit the caller's workspace: skip
        if (r != MGT_OK) return r;
        if (best_t < 0 || t < best_t) {
            best_t = t;
            best_c = c;
        }
        return MGT_OK;
    };
    for (const mgt_tile_cfg &c : stage1(desc, base)) {
        rc = consider(c);
        if (rc != MGT_OK) break;
    }
    if (rc == MGT_OK) {
        const mgt_tile_cfg shape = best_c;
        for (int u : {1, 2, 4}) {
            if (u == shape.copy_unroll) continue;
            mgt_tile_cfg c = shape;
            c.copy_unroll = u;
            rc = consider(c);
            if (rc != MGT_OK) break;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MGT_OK) return rc;
    if (best_t < 0) return MGT_ENOMEM;
    // report the complete shape of the winner
    mgt_plan_t *p = nullptr;
    if (mgt_plan_tuned(desc, &best_c, &p, nullptr) == MGT_OK) {
        mgt_plan_config(p, best);
        mgt_plan_destroy(p);
    } else {
        *best = best_c;
    }
    if (best_ms) *best_ms = best_t;
    return MGT_OK;
}

}  // extern "C"
