// Batched depth stage (C ABI in include/simsense.h): many rectified pairs of
// uneven sizes, disparity ranges and parameters in one call.
//
// Pairs with identical parameters form a class.  A compute call records, for
// every class on a stream of its own, the census and the cost of the class's
// pairs (one launch per stage over all the class's pairs, pair index from the
// grid, pointers passed by value); the classes' branches are forked from and
// joined back into the caller's stream.  Then, in the fused form (the
// default), ONE persistent launch runs the path aggregation and the selection
// of every pair of the batch from a task list in device memory
// (csrc/sgm_fused.cu); in the per-class form each class runs its own path and
// selection launches on its branch instead.  The whole call is captured once
// into a CUDA graph that later calls replay (re-captured when the caller's
// buffers change), so a batch costs one graph launch on the host.
//
// The schedule of the fused launch (pair order, the lag between a pair's
// paths and its selection, the store policy of the path volume) and the
// per-class launch choices are chosen by simsense_batch_tune, which times
// the candidates on the device and keeps the fastest form.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
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
    std::vector<int> cls_of;           // class of each pair
    void* scratch = nullptr;
    size_t bytes = 0;
    int* status = nullptr;
    // fused form: pair descriptors, task list and counters (inside scratch)
    simsense_batch_schedule_t sched{1, 16, 1, 1, 1};
    FusedPair* fpairs = nullptr;       // n
    int4* ftasks = nullptr;            // ntasks
    int* fctl = nullptr;               // 1 + n
    int ntasks = 0;
    std::vector<Params> cls_params;    // the classes' parameters, for the fused launch
    std::vector<FusedPair> host_fpairs;
    bool fpairs_dirty = true;          // descriptors to upload before the next launch
    bool test_drop = false;            // SIMSENSE_BATCH_OPT_TEST_STALL: pair 0's path tasks left out
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

// Census and cost of class c on stream s (the fused form's per-class part).
cudaError_t enqueue_class_front(simsense_batch* b, const BatchClass& c, cudaStream_t s)
{
    std::vector<PairPtrs> pp;
    pp.reserve(c.members.size());
    for (int i : c.members) pp.push_back(b->pairs[i]);
    const int n = (int)pp.size();
    cudaError_t e = launch_census(c.p, pp.data(), n, s);
    if (e == cudaSuccess) e = launch_cost(c.p, pp.data(), n, b->status, s);
    return e;
}

// Fork every class onto its stream from `s`, run them, join back into `s`;
// in the fused form the classes run census and cost, then one launch on `s`
// does the paths and selection of every pair.
cudaError_t enqueue_all(simsense_batch* b, cudaStream_t s)
{
    const bool fused = b->sched.fused != 0;
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (auto& c : b->classes) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c.stream, b->fork, 0);
        if (e == cudaSuccess) e = fused ? enqueue_class_front(b, c, c.stream) : enqueue_class(b, c, c.stream);
        if (e == cudaSuccess) e = cudaEventRecord(c.join, c.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c.join, 0);
    }
    if (fused) {
        if (e == cudaSuccess) e = cudaMemsetAsync(b->fctl, 0, sizeof(int) * (1 + (size_t)b->n), s);
        if (e == cudaSuccess)
            e = launch_fused(b->fpairs, b->ftasks, b->ntasks, b->fctl, b->status, b->cls_params.data(),
                             (int)b->cls_params.size(), b->sched.keep_paths, s);
    }
    return e;
}

// The fused launch's task list for schedule sc: pairs in the chosen order,
// each pair's path tasks (its work items, longest first, 8 per task), and the
// rows of the k-th pair of the order after the path tasks of the (k + lag)-th.
std::vector<int4> build_tasks(const simsense_batch* b, const simsense_batch_schedule_t& sc)
{
    std::vector<int> order(b->n);
    std::iota(order.begin(), order.end(), 0);
    auto cells = [&](int i) {
        const Params& p = b->classes[b->cls_of[i]].p;
        return (long long)p.W * p.H * p.D;
    };
    if (sc.order == 1) std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cells(a) > cells(c); });
    if (sc.order == 2) std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cells(a) < cells(c); });
    std::vector<int4> t;
    auto rows = [&](int i) {
        const int H = b->classes[b->cls_of[i]].p.H;
        for (int y = 0; y < H; y++) t.push_back(make_int4(1, i, y, 0));
    };
    for (int k = 0; k < b->n; k++) {
        const int i = order[k];
        const int np = b->host_fpairs[i].path_tasks;
        for (int j = 0; j < np; j++)
            t.push_back(b->test_drop && i == 0 ? make_int4(2, i, j, 0) : make_int4(0, i, j, 0));
        if (k >= sc.lag) rows(order[k - sc.lag]);
    }
    for (int k = std::max(0, b->n - sc.lag); k < b->n; k++) rows(order[k]);
    return t;
}

// Uploads the task list of schedule sc (waits for the device first: a graph
// replay in flight may still read the old list).
cudaError_t upload_tasks(simsense_batch* b, const simsense_batch_schedule_t& sc)
{
    const std::vector<int4> t = build_tasks(b, sc);
    if ((int)t.size() != b->ntasks) return cudaErrorInvalidValue;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(b->ftasks, t.data(), t.size() * sizeof(int4), cudaMemcpyHostToDevice);
    return e;
}

// Uploads the pair descriptors (their depth pointers come from the caller)
// on stream s if they changed.
cudaError_t upload_fpairs(simsense_batch* b, cudaStream_t s)
{
    if (!b->fpairs_dirty) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(b->fpairs, b->host_fpairs.data(), b->host_fpairs.size() * sizeof(FusedPair),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host copy may change with the next call
    if (e == cudaSuccess) b->fpairs_dirty = false;
    return e;
}

void set_io(simsense_batch* b, const uint8_t* const* left, const uint8_t* const* right, float* const* depth)
{
    for (int i = 0; i < b->n; i++) {
        b->pairs[i].left = left[i];
        b->pairs[i].right = right[i];
        b->pairs[i].depth = depth[i];
        if (b->host_fpairs[i].depth != depth[i]) {
            b->host_fpairs[i].depth = depth[i];
            b->fpairs_dirty = true;
        }
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
    b->cls_of = cls;

    // the fused form's pair descriptors (depth pointers come with each call)
    b->host_fpairs.resize(n);
    b->ntasks = 0;
    for (int i = 0; i < n; i++) {
        const Params& p = b->classes[cls[i]].p;
        FusedPair& q = b->host_fpairs[i];
        q = FusedPair{};
        q.W = p.W; q.H = p.H; q.D = p.D; q.Dp = p.Dp; q.paths = p.paths; q.P1 = p.P1; q.P2 = p.P2;
        q.uniq = p.uniq; q.lr_max_diff = p.lr_max_diff; q.subpixel = p.subpixel; q.fb = p.fb;
        q.umagic = uniq_magic(p.uniq);
        q.path_tasks = fused_path_tasks(p);
        b->ntasks += q.path_tasks + p.H;
    }
    for (const auto& c : b->classes) b->cls_params.push_back(c.p);

    // one allocation: per pair left codes | right codes | cost | path volume,
    // then the fused form's descriptors, task list and counters
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; i++) {
        const Params& p = b->classes[cls[i]].p;
        const size_t npx = (size_t)p.W * p.H;
        off[i] = total;
        total += 2 * round256(npx * (p.wide_codes ? 8 : 4)) + round256(npx * p.Dp) +
                 round256(path_volume_bytes(p));
    }
    const size_t off_fpairs = total;
    total += round256(sizeof(FusedPair) * (size_t)n);
    const size_t off_tasks = total;
    total += round256(sizeof(int4) * (size_t)b->ntasks);
    const size_t off_ctl = total;
    total += round256(sizeof(int) * (1 + (size_t)n));
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
        b->host_fpairs[i].cost = pp.cost;
        b->host_fpairs[i].vol = pp.vol;
    }
    uint8_t* base = static_cast<uint8_t*>(b->scratch);
    b->fpairs = reinterpret_cast<FusedPair*>(base + off_fpairs);
    b->ftasks = reinterpret_cast<int4*>(base + off_tasks);
    b->fctl = reinterpret_cast<int*>(base + off_ctl);
    cudaError_t e = upload_tasks(b, b->sched);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
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
    if (b->sched.fused) {
        const cudaError_t e = upload_fpairs(b, s);
        if (e != cudaSuccess) return fail(b, e);
    }
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

namespace {
int apply_schedule(simsense_batch* b, const simsense_batch_schedule_t& sc);
}  // namespace

int simsense_batch_set_option(simsense_batch_t b, int opt, int value)
{
    if (!b) return SIMSENSE_ERR_INVALID_ARG;
    if (opt == SIMSENSE_BATCH_OPT_GRAPH) {
        if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
        b->use_graph = value != 0;
        return SIMSENSE_OK;
    }
    if (opt == SIMSENSE_BATCH_OPT_TEST_STALL) {
        if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
        DeviceGuard g(b->device);
        if (!g.ok) return fail(b, cudaGetLastError());
        b->test_drop = value != 0;
        return apply_schedule(b, b->sched);     // rebuilds the task list
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

int simsense_batch_get_schedule(simsense_batch_t b, simsense_batch_schedule_t* out)
{
    if (!b || !out) return SIMSENSE_ERR_INVALID_ARG;
    *out = b->sched;
    return SIMSENSE_OK;
}

namespace {

bool schedule_valid(const simsense_batch_schedule_t& sc)
{
    return (sc.fused == 0 || sc.fused == 1) && sc.prefetch == 16 && (sc.keep_paths == 0 || sc.keep_paths == 1) &&
           (sc.lag == 1 || sc.lag == 2) && sc.order >= 0 && sc.order <= 2;
}

int apply_schedule(simsense_batch* b, const simsense_batch_schedule_t& sc)
{
    if (sc.fused) {
        const cudaError_t e = upload_tasks(b, sc);
        if (e != cudaSuccess) return fail(b, e);
    }
    b->sched = sc;
    if (b->exec) {                       // the captured graph holds the old form
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return SIMSENSE_OK;
}

// Device time of `reps` whole-batch runs after one warm-up, on stream s.
cudaError_t time_batch(simsense_batch* b, int reps, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1, float* ms)
{
    cudaError_t e = b->sched.fused ? upload_fpairs(b, s) : cudaSuccess;
    if (e == cudaSuccess) e = enqueue_all(b, s);
    if (e == cudaSuccess) e = cudaEventRecord(t0, s);
    for (int r = 0; r < reps && e == cudaSuccess; r++) e = enqueue_all(b, s);
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    return e;
}

}  // namespace

int simsense_batch_set_schedule(simsense_batch_t b, const simsense_batch_schedule_t* sc)
{
    if (!b || !sc || !schedule_valid(*sc)) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(b->device);
    if (!g.ok) return fail(b, cudaGetLastError());
    return apply_schedule(b, *sc);
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
    // 1. the per-class form: each class's launch choices, class by class
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
    // 2. whole batches: the per-class form with those choices against every
    //    schedule of the fused form (pair order x lag x path-volume store
    //    policy); the fastest is kept
    simsense_batch_schedule_t best = b->sched;
    float best_ms = -1.0f;
    std::vector<simsense_batch_schedule_t> cand;
    cand.push_back(simsense_batch_schedule_t{0, 16, 1, 1, 1});
    for (int order = 0; order <= 2; order++)
        for (int lag = 1; lag <= 2; lag++)
            for (int keep = 0; keep <= 1; keep++) cand.push_back(simsense_batch_schedule_t{1, 16, keep, lag, order});
    for (const auto& sc : cand) {
        if (e != cudaSuccess) break;
        if (apply_schedule(b, sc) != SIMSENSE_OK) {
            e = (cudaError_t)b->last_cuda_error;
            break;
        }
        float ms = 0.0f;
        e = time_batch(b, reps, s, t0, t1, &ms);
        if (e == cudaSuccess && (best_ms < 0.0f || ms < best_ms)) {
            best_ms = ms;
            best = sc;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) return fail(b, e);
    return apply_schedule(b, best);
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
