// Batched depth stage (C ABI in include/simsense.h): many rectified pairs of
// uneven sizes, disparity ranges and parameters in one call.
//
// Pairs with identical parameters form a class.  A compute call records, for
// every class on a stream of its own, the same four stages as the plain path
// (census, cost, paths, selection), each stage one launch over all the class's
// pairs (pair index from the grid, pointers passed by value).  The classes'
// branches are forked from and joined back into the caller's stream, and the
// whole call is captured once into a CUDA graph that later calls replay
// (re-captured when the caller's buffers change), so a batch costs one graph
// launch on the host.  Concurrent branches fill the SMs that a single pair
// leaves idle, e.g. behind the long horizontal scanlines of the path stage.
//
// Each class has its own launch choices (Tuning); simsense_batch_tune times
// the candidates on the device and keeps the fastest per class.
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

using namespace simsense;

namespace {

struct BatchClass {
    Params p{};
    simsense_pair_params_t key{};
    std::vector<int> members;
    Tuning tune{};
    cudaStream_t stream = nullptr;
    cudaEvent_t join = nullptr;
};

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

bool same_params(const simsense_pair_params_t& a, const simsense_pair_params_t& b)
{
    return a.W == b.W && a.H == b.H && a.D == b.D && a.census_win == b.census_win && a.P1 == b.P1 &&
           a.P2 == b.P2 && a.paths == b.paths && a.uniq_ratio == b.uniq_ratio &&
           a.lr_max_diff == b.lr_max_diff && a.subpixel == b.subpixel && a.f == b.f && a.baseline == b.baseline;
}

}  // namespace

struct simsense_batch {
    int n = 0;
    int device = 0;
    std::vector<PairPtrs> pairs;
    std::vector<BatchClass> classes;
    void* scratch = nullptr;
    size_t bytes = 0;
    int* status = nullptr;
    cudaStream_t cap = nullptr;        // internal stream the graph is captured on
    cudaEvent_t fork = nullptr;
    cudaEvent_t done = nullptr;
    bool use_graph = true;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> graph_ptrs;
    int last_cuda_error = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(simsense_batch* b, cudaError_t e)
{
    b->last_cuda_error = (int)e;
    return SIMSENSE_ERR_CUDA;
}

void release(simsense_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& c : b->classes) {
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.join) cudaEventDestroy(c.join);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    cudaFree(b->scratch);
    cudaFree(b->status);
}

// The four stages of class c on stream s.
cudaError_t enqueue_class(simsense_batch* b, const BatchClass& c, cudaStream_t s)
{
    std::vector<PairPtrs> pp;
    pp.reserve(c.members.size());
    for (int i : c.members) pp.push_back(b->pairs[i]);
    const int n = (int)pp.size();
    const SelectDebug none{};
    cudaError_t e = launch_census(c.p, pp.data(), n, s);
    if (e == cudaSuccess) e = launch_cost(c.p, pp.data(), n, b->status, s);
    if (e == cudaSuccess) e = launch_paths(c.p, pp.data(), n, c.tune, nullptr, s);
    if (e == cudaSuccess) e = launch_select(c.p, pp.data(), n, c.tune, none, b->status, s);
    return e;
}

// Fork every class onto its stream from `s`, run them, join back into `s`.
cudaError_t enqueue_all(simsense_batch* b, cudaStream_t s)
{
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (auto& c : b->classes) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c.stream, b->fork, 0);
        if (e == cudaSuccess) e = enqueue_class(b, c, c.stream);
        if (e == cudaSuccess) e = cudaEventRecord(c.join, c.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c.join, 0);
    }
    return e;
}

void set_io(simsense_batch* b, const uint8_t* const* left, const uint8_t* const* right, float* const* depth)
{
    for (int i = 0; i < b->n; i++) {
        b->pairs[i].left = left[i];
        b->pairs[i].right = right[i];
        b->pairs[i].depth = depth[i];
    }
}

bool io_valid(int n, const uint8_t* const* left, const uint8_t* const* right, float* const* depth)
{
    if (!left || !right || !depth) return false;
    for (int i = 0; i < n; i++)
        if (!left[i] || !right[i] || !depth[i]) return false;
    return true;
}

}  // namespace

extern "C" {

int simsense_batch_create(simsense_batch_t* out, const simsense_pair_params_t* prm, int n)
{
    if (!out || !prm || n < 1) return SIMSENSE_ERR_INVALID_ARG;
    *out = nullptr;
    simsense_batch* b = new (std::nothrow) simsense_batch();
    if (!b) return SIMSENSE_ERR_OOM;
    b->n = n;
    b->pairs.resize(n);
    std::vector<int> cls(n, -1);
    for (int i = 0; i < n; i++) {
        int found = -1;
        for (size_t c = 0; c < b->classes.size(); c++)
            if (same_params(b->classes[c].key, prm[i])) { found = (int)c; break; }
        if (found < 0) {
            BatchClass c;
            c.key = prm[i];
            const int rc = make_params(c.p, prm[i].W, prm[i].H, prm[i].D, prm[i].census_win, prm[i].P1, prm[i].P2,
                                       prm[i].paths, prm[i].uniq_ratio, prm[i].lr_max_diff, prm[i].f,
                                       prm[i].baseline, prm[i].subpixel);
            if (rc != SIMSENSE_OK) { delete b; return rc; }
            b->classes.push_back(c);
            found = (int)b->classes.size() - 1;
        }
        b->classes[found].members.push_back(i);
        cls[i] = found;
    }
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return SIMSENSE_ERR_CUDA; }

    // one allocation: per pair left codes | right codes | cost | path volume
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; i++) {
        const Params& p = b->classes[cls[i]].p;
        const size_t npx = (size_t)p.W * p.H;
        off[i] = total;
        total += 2 * round256(npx * (p.wide_codes ? 8 : 4)) + round256(npx * p.Dp) +
                 round256(path_volume_bytes(p));
    }
    bool ok = dev_alloc(&b->scratch, total) == cudaSuccess && dev_alloc((void**)&b->status, sizeof(int)) == cudaSuccess &&
              cudaMemset(b->status, 0, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(b);
        delete b;
        return SIMSENSE_ERR_OOM;
    }
    b->bytes = total + sizeof(int);
    for (int i = 0; i < n; i++) {
        const Params& p = b->classes[cls[i]].p;
        const size_t npx = (size_t)p.W * p.H;
        const size_t cb = round256(npx * (p.wide_codes ? 8 : 4));
        uint8_t* base = static_cast<uint8_t*>(b->scratch) + off[i];
        PairPtrs& pp = b->pairs[i];
        pp.codes_left = base;
        pp.codes_right = base + cb;
        pp.cost = base + 2 * cb;
        pp.vol = pp.cost + round256(npx * p.Dp);
        pp.left = pp.right = nullptr;
        pp.depth = nullptr;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    for (auto& c : b->classes) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.join, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return SIMSENSE_ERR_CUDA;
    }
    *out = b;
    return SIMSENSE_OK;
}

int simsense_batch_compute(simsense_batch_t b, const uint8_t* const* left, const uint8_t* const* right,
                           float* const* depth, struct CUstream_st* stream)
{
    if (!b || !io_valid(b->n, left, right, depth)) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    if (!g.ok) return fail(b, cudaGetLastError());
    cudaStream_t s = (cudaStream_t)stream;
    set_io(b, left, right, depth);
    if (!b->use_graph) {
        cudaError_t e = enqueue_all(b, s);
        return e == cudaSuccess ? SIMSENSE_OK : fail(b, e);
    }
    std::vector<const void*> ptrs;
    ptrs.reserve(3 * b->n);
    for (int i = 0; i < b->n; i++) {
        ptrs.push_back(left[i]);
        ptrs.push_back(right[i]);
        ptrs.push_back(depth[i]);
    }
    if (!b->exec || ptrs != b->graph_ptrs) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(b, e);
        cudaError_t ee = enqueue_all(b, b->cap);
        e = cudaStreamEndCapture(b->cap, &graph);
        if (ee != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(b, ee != cudaSuccess ? ee : e);
        }
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return fail(b, e);
        }
        b->graph_ptrs = ptrs;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    return e == cudaSuccess ? SIMSENSE_OK : fail(b, e);
}

int simsense_batch_set_option(simsense_batch_t b, int opt, int value)
{
    if (!b) return SIMSENSE_ERR_INVALID_ARG;
    if (opt == SIMSENSE_BATCH_OPT_GRAPH) {
        if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
        b->use_graph = value != 0;
        return SIMSENSE_OK;
    }
    return SIMSENSE_ERR_INVALID_ARG;
}

int simsense_batch_num_classes(simsense_batch_t b)
{
    return b ? (int)b->classes.size() : SIMSENSE_ERR_INVALID_ARG;
}

int simsense_batch_class_info(simsense_batch_t b, int c, simsense_pair_params_t* params, int* npairs)
{
    if (!b || c < 0 || c >= (int)b->classes.size()) return SIMSENSE_ERR_INVALID_ARG;
    if (params) *params = b->classes[c].key;
    if (npairs) *npairs = (int)b->classes[c].members.size();
    return SIMSENSE_OK;
}

int simsense_batch_get_tuning(simsense_batch_t b, int c, int* prefetch, int* select_blocks)
{
    if (!b || c < 0 || c >= (int)b->classes.size()) return SIMSENSE_ERR_INVALID_ARG;
    if (prefetch) *prefetch = b->classes[c].tune.prefetch;
    if (select_blocks) *select_blocks = b->classes[c].tune.select_blocks;
    return SIMSENSE_OK;
}

int simsense_batch_set_tuning(simsense_batch_t b, int c, int prefetch, int select_blocks)
{
    if (!b || c < 0 || c >= (int)b->classes.size()) return SIMSENSE_ERR_INVALID_ARG;
    if (prefetch != 8 && prefetch != 12 && prefetch != 16) return SIMSENSE_ERR_INVALID_ARG;
    if (select_blocks != 1 && select_blocks != 2) return SIMSENSE_ERR_INVALID_ARG;
    b->classes[c].tune.prefetch = prefetch;
    b->classes[c].tune.select_blocks = select_blocks;
    if (b->exec) {                       // the captured graph holds the old choices
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return SIMSENSE_OK;
}

int simsense_batch_tune(simsense_batch_t b, const uint8_t* const* left, const uint8_t* const* right,
                        float* const* depth, int reps, struct CUstream_st* stream)
{
    if (!b || !io_valid(b->n, left, right, depth) || reps < 1 || reps > 100) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    if (!g.ok) return fail(b, cudaGetLastError());
    cudaStream_t s = (cudaStream_t)stream;
    set_io(b, left, right, depth);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    static const int kPrefetch[3] = {8, 12, 16};
    for (auto& c : b->classes) {
        Tuning best = c.tune;
        float best_ms = -1.0f;
        for (int pf = 0; pf < 3 && e == cudaSuccess; pf++) {
            for (int sb = 1; sb <= 2 && e == cudaSuccess; sb++) {
                c.tune.prefetch = kPrefetch[pf];
                c.tune.select_blocks = sb;
                e = enqueue_class(b, c, s);                       // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(t0, s);
                for (int r = 0; r < reps && e == cudaSuccess; r++) e = enqueue_class(b, c, s);
                if (e == cudaSuccess) e = cudaEventRecord(t1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e == cudaSuccess && (best_ms < 0.0f || ms < best_ms)) {
                    best_ms = ms;
                    best = c.tune;
                }
            }
        }
        c.tune = best;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return e == cudaSuccess ? SIMSENSE_OK : fail(b, e);
}

size_t simsense_batch_scratch_bytes(simsense_batch_t b)
{
    return b ? b->bytes : 0;
}

int simsense_batch_device_status(simsense_batch_t b, struct CUstream_st* stream)
{
    if (!b) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    int v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&v, b->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(b->status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(b, e);
    return v == 0 ? SIMSENSE_OK : v;
}

int simsense_batch_last_cuda_error(simsense_batch_t b)
{
    return b ? b->last_cuda_error : 0;
}

int simsense_batch_destroy(simsense_batch_t b)
{
    if (!b) return SIMSENSE_OK;
    DeviceGuard g(b->device);
    release(b);
    delete b;
    return SIMSENSE_OK;
}

}  // extern "C"
