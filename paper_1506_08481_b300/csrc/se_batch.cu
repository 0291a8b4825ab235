// Batches of independent configurations of uneven size: one CUDA graph holds the
// products of every box, the boxes' kernel chains running concurrently on a pool of
// streams (fork from the caller's stream, join back), so a step of the whole batch
// is one graph launch.  Each box keeps its own context (own M, P, xi, rc chosen per
// box by the autotuner in params.py).
#include <vector>

#include "se_internal.cuh"

struct se_batch {
    int device = 0;
    cudaStream_t main = nullptr;                 // borrowed
    std::vector<se_ctx *> box;                   // borrowed contexts
    std::vector<cudaStream_t> streams;           // owned
    std::vector<cudaEvent_t> join;               // owned, one per stream
    cudaEvent_t fork = nullptr;                  // owned
    cudaEvent_t done = nullptr;                  // owned
    cudaStream_t cap = nullptr;                  // owned: the graph is captured on it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the persistent launch (mode 2): its plan, and whether the graph holds it
    se::PersistPlan pp;
    bool pp_ok = false;
    // what the graph was captured for (mode 1 or 2)
    int g_mode = 0, g_ncomp = 0, g_dtype = -1;
    long long wait_ns = 2000000000ll;            // limit of the persistent launch's waits
    int stall_box = -1;                          // failure-injection hook (se_batch_inject_stall)
    std::vector<const void *> g_x;
    std::vector<void *> g_y;
    std::string err;
};

static void batch_drop_graph(se_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

extern "C" int se_batch_create(se_batch **out, se_ctx *const *ctx, int nbox, int nstreams, void *stream)
{
    if (!out || !ctx || nbox < 1 || nstreams < 1 || nstreams > 64) return SE_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < nbox; ++i)
        if (!ctx[i] || !ctx[i]->have_config || ctx[i]->device != ctx[0]->device) return SE_ERR_STATE;
    se_batch *b = new se_batch();
    b->device = ctx[0]->device;
    cudaSetDevice(b->device);
    b->main = (cudaStream_t)stream;
    b->box.assign(ctx, ctx + nbox);
    b->streams.resize(nstreams);
    b->join.resize(nstreams);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (int q = 0; q < nstreams && ok; ++q)
        ok = cudaStreamCreateWithFlags(&b->streams[q], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[q], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        delete b;
        return SE_ERR_CUDA;
    }
    *out = b;
    return SE_OK;
}

extern "C" int se_batch_destroy(se_batch *b)
{
    if (!b) return SE_OK;
    cudaSetDevice(b->device);
    for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
    if (b->main) cudaStreamSynchronize(b->main);
    batch_drop_graph(b);
    se::persist_free(b->pp);
    for (size_t q = 0; q < b->streams.size(); ++q) {
        if (b->join[q]) cudaEventDestroy(b->join[q]);
        if (b->streams[q]) cudaStreamDestroy(b->streams[q]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return SE_OK;
}

// enqueue every box's product between a fork from and a join into stream `root`;
// box i runs on stream i mod nstreams (its context's stream is swapped only meanwhile)
static int batch_enqueue(se_batch *b, cudaStream_t root, int ncomp, const void *const *x, void *const *y, int dtype)
{
    SE_CUDA_CHECK(b, cudaEventRecord(b->fork, root));
    for (cudaStream_t s : b->streams) SE_CUDA_CHECK(b, cudaStreamWaitEvent(s, b->fork, 0));
    for (size_t i = 0; i < b->box.size(); ++i) {
        se_ctx *c = b->box[i];
        cudaStream_t own = c->stream;
        // the boxes run concurrently, so no box splits its spreading tiles over CTAs
        c->stream = b->streams[i % b->streams.size()];
        c->split_cap = 1;
        const int rc = se::se_apply_internal(c, ncomp, x[i], y[i], dtype, c->precision);
        c->stream = own;
        c->split_cap = 16;
        if (rc != SE_OK) {
            b->err = "box " + std::to_string(i) + ": " + c->err;
            return rc;
        }
    }
    for (size_t q = 0; q < b->streams.size(); ++q) {
        SE_CUDA_CHECK(b, cudaEventRecord(b->join[q], b->streams[q]));
        SE_CUDA_CHECK(b, cudaStreamWaitEvent(root, b->join[q], 0));
    }
    return SE_OK;
}

// mode 2: one persistent launch for all boxes, captured into the batch's graph when the
// runtime accepts the capture of a cooperative launch, else launched directly
static int batch_persistent(se_batch *b, int ncomp, const void *const *x, void *const *y, int dtype)
{
    const size_t n = b->box.size();
    bool same = b->pp_ok && b->pp.ncomp == ncomp && b->pp.dtype == dtype;
    for (size_t i = 0; same && i < n; ++i) same = b->g_x[i] == x[i] && b->g_y[i] == y[i];
    if (!same) {
        batch_drop_graph(b);
        b->pp_ok = false;
        // one eager pass sets up every box's tables and grids (and computes this step)
        int rc = batch_enqueue(b, b->main, ncomp, x, y, dtype);
        if (rc != SE_OK) return rc;
        SE_CUDA_CHECK(b, cudaStreamSynchronize(b->main));
        rc = se::persist_prepare(b->box.data(), (int)n, ncomp, x, y, dtype, b->pp, b->err);
        if (rc != SE_OK) return rc;
        b->pp.wait_ns = b->wait_ns;
        b->pp.stall_box = b->stall_box;
        b->pp_ok = true;
        b->g_mode = 2;
        b->g_ncomp = ncomp;
        b->g_dtype = dtype;
        b->g_x.assign(x, x + n);
        b->g_y.assign(y, y + n);
        if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
            std::string e;
            const int lr = se::persist_launch(b->pp, b->cap, e);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
            if (lr == SE_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
                b->graph = g;
            } else {
                if (g) cudaGraphDestroy(g);
                b->exec = nullptr;
            }
        }
        cudaGetLastError();
        return SE_OK;                 // this step was computed by the eager pass
    }
    b->box[0]->launches++;
    if (b->exec) {
        SE_CUDA_CHECK(b, cudaGraphLaunch(b->exec, b->main));
        return SE_OK;
    }
    return se::persist_launch(b->pp, b->main, b->err);
}

extern "C" int se_batch_apply(se_batch *b, int ncomp, const void *const *x, void *const *y, int dtype,
                              int use_graph)
{
    if (!b || !x || !y) return SE_ERR_ARG;
    if (ncomp != 3 && ncomp != 6 && ncomp != 11 && ncomp != 12) return SE_ERR_ARG;
    if (dtype != SE_F32 && dtype != SE_F64) return SE_ERR_ARG;
    if (use_graph < 0 || use_graph > 2) return SE_ERR_ARG;
    const size_t n = b->box.size();
    for (size_t i = 0; i < n; ++i)
        if (!x[i] || !y[i]) return SE_ERR_ARG;
    cudaSetDevice(b->device);
    if (!use_graph) return batch_enqueue(b, b->main, ncomp, x, y, dtype);
    if (use_graph == 2) return batch_persistent(b, ncomp, x, y, dtype);
    bool same = b->exec && b->g_mode == 1 && b->g_ncomp == ncomp && b->g_dtype == dtype;
    for (size_t i = 0; same && i < n; ++i) same = b->g_x[i] == x[i] && b->g_y[i] == y[i];
    if (!same) {
        b->pp_ok = false;
        batch_drop_graph(b);
        // one eager pass sets up every box's tables and grids outside the capture; the
        // capture runs on the batch's own stream (the caller's may be the legacy stream)
        int rc = batch_enqueue(b, b->main, ncomp, x, y, dtype);
        if (rc != SE_OK) return rc;
        SE_CUDA_CHECK(b, cudaStreamSynchronize(b->main));
        SE_CUDA_CHECK(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
        rc = batch_enqueue(b, b->cap, ncomp, x, y, dtype);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
        if (rc != SE_OK || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            if (rc == SE_OK) b->err = std::string("graph capture: ") + cudaGetErrorString(ec);
            return rc != SE_OK ? rc : SE_ERR_CUDA;
        }
        b->graph = g;
        SE_CUDA_CHECK(b, cudaGraphInstantiate(&b->exec, b->graph, 0));
        b->g_mode = 1;
        b->g_ncomp = ncomp;
        b->g_dtype = dtype;
        b->g_x.assign(x, x + n);
        b->g_y.assign(y, y + n);
    }
    SE_CUDA_CHECK(b, cudaGraphLaunch(b->exec, b->main));
    return SE_OK;
}

extern "C" int se_batch_status(se_batch *b)
{
    if (!b) return SE_ERR_ARG;
    cudaSetDevice(b->device);
    SE_CUDA_CHECK(b, cudaStreamSynchronize(b->main));
    if (b->pp.ctl && se::persist_failed(b->pp, b->main)) {
        b->err = "a persistent batch launch gave up waiting for work of an earlier phase";
        return SE_ERR_CUDA;
    }
    return SE_OK;
}

extern "C" const char *se_batch_last_error(const se_batch *b) { return b ? b->err.c_str() : ""; }

extern "C" int se_batch_set_wait_limit(se_batch *b, double seconds)
{
    if (!b || !(seconds > 0) || !(seconds <= 600)) return SE_ERR_ARG;
    b->wait_ns = (long long)(seconds * 1e9);
    batch_drop_graph(b);          // the launch's arguments change: prepare and capture again
    b->pp_ok = false;
    return SE_OK;
}

extern "C" int se_batch_inject_stall(se_batch *b, int box)
{
    if (!b || box < -1 || box >= (int)b->box.size()) return SE_ERR_ARG;
    b->stall_box = box;
    batch_drop_graph(b);
    b->pp_ok = false;
    return SE_OK;
}
