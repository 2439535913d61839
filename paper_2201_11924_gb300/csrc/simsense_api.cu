// C ABI of libsimsense (declared in include/simsense.h): argument checks,
// scratch ownership and the launch sequence census -> cost -> paths -> select.
#include <errno.h>
#include <math.h>
#include <unistd.h>
#include <atomic>
#include <new>

#include "internal.h"

#include <nvtx3/nvToolsExt.h>

using namespace simsense;

namespace {

// allocations left before the one that fails (0: none fails)
std::atomic<int> g_fail_alloc{0};

}  // namespace

cudaError_t simsense::dev_alloc(void** ptr, size_t bytes)
{
    int k = g_fail_alloc.load();
    while (k > 0 && !g_fail_alloc.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *ptr = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(ptr, bytes);
}

namespace {

// Makes the handle's device current for the duration of a call.
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

int cuda_fail(simsense_ctx* h, cudaError_t e)
{
    if (h) h->last_cuda_error = (int)e;
    return SIMSENSE_ERR_CUDA;
}

void free_scratch(Scratch& s)
{
    cudaFree(s.codes_left);
    cudaFree(s.codes_right);
    cudaFree(s.cost);
    cudaFree(s.paths);
    cudaFree(s.status);
    cudaFree(s.stage_left);
    cudaFree(s.stage_right);
    cudaFree(s.stage_depth);
    s = Scratch{};
}

void free_profile(ProfileRing& r)
{
    if (r.ev) {
        for (int i = 0; i < ProfileRing::kSlots * 2 * SIMSENSE_NUM_STAGES; i++)
            if (r.ev[i]) cudaEventDestroy(r.ev[i]);
        delete[] r.ev;
    }
    r = ProfileRing{};
}

// Records the start (end = false) or end of `stage` for the current call:
// a named NVTX range on the host (seen by nsys / ncu, free without a tool)
// and, with SIMSENSE_OPT_PROFILE, CUDA events on the stream.
cudaError_t mark(simsense_ctx* h, int stage, bool end, cudaStream_t st)
{
    if (end) nvtxRangePop();
    else nvtxRangePushA(simsense_stage_name(stage));
    ProfileRing& r = h->prof;
    if (!r.on || r.count >= ProfileRing::kSlots) return cudaSuccess;
    return cudaEventRecord(r.ev[r.count * 2 * SIMSENSE_NUM_STAGES + 2 * stage + (end ? 1 : 0)], st);
}

int run(simsense_ctx* h, const uint8_t* left, const uint8_t* right, float* depth,
        const simsense_debug_t* dbg, cudaStream_t st)
{
    const Params& p = h->p;
    Scratch& s = h->s;
    cudaError_t e = cudaSuccess;
    if (h->noise_on) {
        // sensor noise (Sec. VI-C) of both views into the staging buffers
        // (in place when the host-buffer call staged the inputs there)
        e = launch_noise(h->noise, left, s.stage_left, right, s.stage_right, p.W * p.H, h->noise_frame++, 0, st);
        if (e != cudaSuccess) return cuda_fail(h, e);
        left = s.stage_left;
        right = s.stage_right;
    }
    if (h->rect_map[0]) {
        // rectification (Sec. VI-D) of both views through their maps
        e = launch_remap(left, h->rect_map[0], h->rect_img[0], right, h->rect_map[1], h->rect_img[1], p.W, p.H, st);
        if (e != cudaSuccess) return cuda_fail(h, e);
        left = h->rect_img[0];
        right = h->rect_img[1];
    }
    const PairPtrs pair{left, right, s.codes_left, s.codes_right, s.cost, s.paths, depth};
    const Tuning tune{};
    e = mark(h, SIMSENSE_STAGE_CENSUS, false, st);
    if (e == cudaSuccess) e = launch_census(p, &pair, 1, st);
    {
        const cudaError_t e_end = mark(h, SIMSENSE_STAGE_CENSUS, true, st);   // pops the range in any case
        if (e == cudaSuccess) e = e_end;
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    e = mark(h, SIMSENSE_STAGE_COST, false, st);
    if (block_active(p)) {
        // SGBM: the per-pixel costs go to the path volume (free until the
        // path stage), their block mean to the cost volume
        PairPtrs raw = pair;
        raw.cost = s.paths;
        if (e == cudaSuccess) e = launch_cost(p, &raw, 1, s.status, st);
        if (e == cudaSuccess) e = launch_block_cost(p, &pair, 1, st);
    } else if (e == cudaSuccess) {
        e = launch_cost(p, &pair, 1, s.status, st);
    }
    {
        const cudaError_t e_end = mark(h, SIMSENSE_STAGE_COST, true, st);   // pops the range in any case
        if (e == cudaSuccess) e = e_end;
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    // debug dumps of the census codes and of the cost volume, read before the
    // path stage (the median variant reuses the left codes' memory later)
    if (dbg && dbg->census_left) {
        e = launch_widen_codes(p, s.codes_left, dbg->census_left, st);
        if (e != cudaSuccess) return cuda_fail(h, e);
    }
    if (dbg && dbg->census_right) {
        e = launch_widen_codes(p, s.codes_right, dbg->census_right, st);
        if (e != cudaSuccess) return cuda_fail(h, e);
    }
    if (dbg && dbg->cost) {
        e = cudaMemcpy2DAsync(dbg->cost, p.D, s.cost, p.Dp, p.D, (size_t)p.W * p.H, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e);
    }
    e = mark(h, SIMSENSE_STAGE_PATHS, false, st);
    if (e == cudaSuccess) e = launch_paths(p, &pair, 1, tune, dbg ? dbg->paths : nullptr, st);
    {
        const cudaError_t e_end = mark(h, SIMSENSE_STAGE_PATHS, true, st);   // pops the range in any case
        if (e == cudaSuccess) e = e_end;
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    SelectDebug sd{};
    if (dbg) {
        sd.aggregated = dbg->aggregated;
        sd.disparity_int = dbg->disparity_int;
        sd.disparity = dbg->disparity;
        sd.mask = dbg->mask;
    }
    e = mark(h, SIMSENSE_STAGE_SELECT, false, st);
    if (p.median > 1) {
        // the selection writes the disparity into the left census codes' memory
        // (at least 4 bytes per pixel, free after the cost stage), the median
        // filter turns it into depth
        PairPtrs sel = pair;
        sel.depth = reinterpret_cast<float*>(s.codes_left);
        if (e == cudaSuccess) e = launch_select(p, &sel, 1, tune, sd, s.status, st);
        if (e == cudaSuccess) e = launch_median(p, sel.depth, depth, sd.disparity, st);
    } else if (e == cudaSuccess) {
        e = launch_select(p, &pair, 1, tune, sd, s.status, st);
    }
    {
        const cudaError_t e_end = mark(h, SIMSENSE_STAGE_SELECT, true, st);   // pops the range in any case
        if (e == cudaSuccess) e = e_end;
    }
    if (e != cudaSuccess) return cuda_fail(h, e);
    if (h->prof.on && h->prof.count < ProfileRing::kSlots) h->prof.count++;
    return SIMSENSE_OK;
}

}  // namespace

namespace simsense {

int make_params(Params& p, int W, int H, int D, int census_win, int P1, int P2, int paths, int uniq_ratio,
                int lr_max_diff, float f, float baseline, int subpixel)
{
    const int ww = census_win & 0xff;
    int wh = (census_win >> 8) & 0xff;
    if (wh == 0) wh = ww;
    if ((census_win >> 16) != 0) return SIMSENSE_ERR_INVALID_ARG;
    if (ww < 1 || wh < 1 || ww > kMaxWin || wh > kMaxWin || !(ww & 1) || !(wh & 1))
        return SIMSENSE_ERR_INVALID_ARG;
    const int nbits = ww * wh - 1;
    if (nbits < 1 || nbits > 64) return SIMSENSE_ERR_INVALID_ARG;
    if (W < ww || H < wh || W > kMaxW || H > (1 << 14)) return SIMSENSE_ERR_INVALID_ARG;
    if (D < 1 || D > kMaxD || D > W) return SIMSENSE_ERR_INVALID_ARG;
    if (P1 < 0 || P2 < P1 || nbits + P2 > 255) return SIMSENSE_ERR_INVALID_ARG;
    if (paths != 4 && paths != 8) return SIMSENSE_ERR_INVALID_ARG;
    if (uniq_ratio < 0 || uniq_ratio > 99) return SIMSENSE_ERR_INVALID_ARG;
    if (subpixel != 0 && subpixel != 1) return SIMSENSE_ERR_INVALID_ARG;
    if (!(f > 0.0f) || !(baseline > 0.0f) || !isfinite(f) || !isfinite(baseline))
        return SIMSENSE_ERR_INVALID_ARG;
    p = Params{};
    p.W = W; p.H = H; p.D = D;
    p.win_w = ww; p.win_h = wh; p.nbits = nbits;
    p.P1 = P1; p.P2 = P2; p.paths = paths;
    p.uniq = uniq_ratio; p.lr_max_diff = lr_max_diff;
    p.subpixel = subpixel;
    p.f = f; p.baseline = baseline;
    p.fb = (float)((double)f * (double)baseline);
    p.dpt = 2 * ((D + 63) / 64);
    p.Dp = 32 * p.dpt;
    p.wide_codes = nbits > 32;
    return SIMSENSE_OK;
}

int set_variant(Params& p, int opt, int value)
{
    switch (opt) {
        case SIMSENSE_OPT_CENSUS_CS: {
            if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
            const int full = p.win_w * p.win_h - 1;
            const int nbits = value ? full / 2 : full;
            if (nbits < 1 || nbits + p.P2 > 255) return SIMSENSE_ERR_INVALID_ARG;
            p.census_cs = value;
            p.nbits = nbits;
            p.wide_codes = nbits > 32;
            return SIMSENSE_OK;
        }
        case SIMSENSE_OPT_BLOCK: {
            const int bw = value & 0xff, bh = (value >> 8) & 0xff;
            if ((value >> 16) != 0 || bw < 1 || bh < 1 || bw > 7 || bh > 7 || !(bw & 1) || !(bh & 1))
                return SIMSENSE_ERR_INVALID_ARG;
            p.block_w = bw;
            p.block_h = bh;
            return SIMSENSE_OK;
        }
        case SIMSENSE_OPT_MEDIAN:
            if (value != 0 && value != 3 && value != 5) return SIMSENSE_ERR_INVALID_ARG;
            p.median = value;
            return SIMSENSE_OK;
        default:
            return SIMSENSE_ERR_INVALID_ARG;
    }
}

}  // namespace simsense

extern "C" {

int simsense_create(simsense_t* out, int W, int H, int D, int census_win, int P1, int P2,
                    int paths, int uniq_ratio, int lr_max_diff, float f, float baseline)
{
    if (!out) return SIMSENSE_ERR_INVALID_ARG;
    *out = nullptr;
    Params pv;
    const int rc = make_params(pv, W, H, D, census_win, P1, P2, paths, uniq_ratio, lr_max_diff, f, baseline, 1);
    if (rc != SIMSENSE_OK) return rc;
    simsense_ctx* h = new (std::nothrow) simsense_ctx();
    if (!h) return SIMSENSE_ERR_OOM;
    Params& p = h->p;
    p = pv;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return SIMSENSE_ERR_CUDA; }

    const size_t npx = (size_t)W * H;
    const size_t code_bytes = npx * (p.wide_codes ? 8 : 4);
    const size_t cost_bytes = npx * p.Dp;
    const size_t vol_bytes = path_volume_bytes(p);
    Scratch& s = h->s;
    bool ok = dev_alloc(&s.codes_left, code_bytes) == cudaSuccess &&
              dev_alloc(&s.codes_right, code_bytes) == cudaSuccess &&
              dev_alloc((void**)&s.cost, cost_bytes) == cudaSuccess &&
              dev_alloc((void**)&s.paths, vol_bytes) == cudaSuccess &&
              dev_alloc((void**)&s.status, sizeof(int)) == cudaSuccess &&
              cudaMemset(s.status, 0, sizeof(int)) == cudaSuccess &&
              dev_alloc((void**)&s.stage_left, npx) == cudaSuccess &&
              dev_alloc((void**)&s.stage_right, npx) == cudaSuccess &&
              dev_alloc((void**)&s.stage_depth, npx * sizeof(float)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();   // clear the sticky-free allocation error
        free_scratch(s);
        delete h;
        return SIMSENSE_ERR_OOM;
    }
    s.bytes = 2 * code_bytes + cost_bytes + vol_bytes + 2 * npx + npx * sizeof(float);
    *out = h;
    return SIMSENSE_OK;
}

int simsense_compute(simsense_t h, const uint8_t* left_u8, const uint8_t* right_u8, float* depth_f32,
                     struct CUstream_st* stream)
{
    return simsense_compute_debug(h, left_u8, right_u8, depth_f32, nullptr, stream);
}

int simsense_compute_debug(simsense_t h, const uint8_t* left_u8, const uint8_t* right_u8,
                           float* depth_f32, const simsense_debug_t* dbg, struct CUstream_st* stream)
{
    if (!h || !left_u8 || !right_u8 || !depth_f32) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return cuda_fail(h, cudaGetLastError());
    return run(h, left_u8, right_u8, depth_f32, dbg, (cudaStream_t)stream);
}

int simsense_compute_host(simsense_t h, const uint8_t* left_host, const uint8_t* right_host,
                          float* depth_host, struct CUstream_st* stream)
{
    if (!h || !left_host || !right_host || !depth_host) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return cuda_fail(h, cudaGetLastError());
    cudaStream_t st = (cudaStream_t)stream;
    const size_t npx = (size_t)h->p.W * h->p.H;
    cudaError_t e = cudaMemcpyAsync(h->s.stage_left, left_host, npx, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->s.stage_right, right_host, npx, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e);
    int rc = run(h, h->s.stage_left, h->s.stage_right, h->s.stage_depth, nullptr, st);
    if (rc != SIMSENSE_OK) return rc;
    e = cudaMemcpyAsync(depth_host, h->s.stage_depth, npx * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return SIMSENSE_OK;
}

int simsense_set_option(simsense_t h, int opt, int value)
{
    if (!h) return SIMSENSE_ERR_INVALID_ARG;
    switch (opt) {
        case SIMSENSE_OPT_SUBPIXEL:
            if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
            h->p.subpixel = value;
            return SIMSENSE_OK;
        case SIMSENSE_OPT_PROFILE: {
            if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
            ProfileRing& r = h->prof;
            if (value && !r.ev) {
                DeviceGuard g(h->device);
                const int n = ProfileRing::kSlots * 2 * SIMSENSE_NUM_STAGES;
                r.ev = new (std::nothrow) cudaEvent_t[n]();
                if (!r.ev) return SIMSENSE_ERR_OOM;
                for (int i = 0; i < n; i++) {
                    cudaError_t e = cudaEventCreate(&r.ev[i]);
                    if (e != cudaSuccess) { free_profile(r); return cuda_fail(h, e); }
                }
            }
            r.on = value != 0;
            r.count = 0;
            return SIMSENSE_OK;
        }
        case SIMSENSE_OPT_CENSUS_CS:
        case SIMSENSE_OPT_BLOCK:
        case SIMSENSE_OPT_MEDIAN:
            return set_variant(h->p, opt, value);
        case SIMSENSE_OPT_TEST_STALL:
            if (value != 0 && value != 1) return SIMSENSE_ERR_INVALID_ARG;
            h->p.test_stall = value;
            return SIMSENSE_OK;
        default:
            return SIMSENSE_ERR_INVALID_ARG;
    }
}

namespace {

void free_rectify(simsense_ctx* h)
{
    for (int v = 0; v < 2; v++) {
        cudaFree(h->rect_map[v]);
        cudaFree(h->rect_img[v]);
        h->rect_map[v] = nullptr;
        h->rect_img[v] = nullptr;
    }
}

}  // namespace

int simsense_set_rectify(simsense_t h, const simsense_camera_t* left, const simsense_camera_t* right)
{
    if (!h || (!left) != (!right)) return SIMSENSE_ERR_INVALID_ARG;
    if (left && (check_camera(*left) != SIMSENSE_OK || check_camera(*right) != SIMSENSE_OK))
        return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    if (!g.ok) return cuda_fail(h, cudaGetLastError());
    cudaError_t e = cudaDeviceSynchronize();       // no earlier call still reads the old maps
    if (e != cudaSuccess) return cuda_fail(h, e);
    free_rectify(h);
    if (!left) return SIMSENSE_OK;
    const size_t npx = (size_t)h->p.W * h->p.H;
    for (int v = 0; v < 2; v++) {
        if (dev_alloc((void**)&h->rect_map[v], npx * sizeof(short4)) != cudaSuccess ||
            dev_alloc((void**)&h->rect_img[v], npx) != cudaSuccess) {
            cudaGetLastError();
            free_rectify(h);
            return SIMSENSE_ERR_OOM;
        }
    }
    e = launch_rect_map(*left, h->p.W, h->p.H, h->rect_map[0], nullptr);
    if (e == cudaSuccess) e = launch_rect_map(*right, h->p.W, h->p.H, h->rect_map[1], nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_rectify(h);
        return cuda_fail(h, e);
    }
    return SIMSENSE_OK;
}

int simsense_set_noise(simsense_t h, int enable, float mu, float sigma, float k, float theta,
                       unsigned long long seed)
{
    if (!h || (enable != 0 && enable != 1)) return SIMSENSE_ERR_INVALID_ARG;
    NoiseParams n;
    n.mu = mu;
    n.sigma = sigma;
    n.k = k;
    n.theta = theta;
    n.seed = seed;
    if (enable && check_noise(n) != SIMSENSE_OK) return SIMSENSE_ERR_INVALID_ARG;
    h->noise_on = enable != 0;
    h->noise = n;
    h->noise_frame = 0;
    return SIMSENSE_OK;
}

int simsense_add_noise(const uint8_t* clean, uint8_t* noisy, int W, int H, float mu, float sigma, float k,
                       float theta, unsigned long long seed, unsigned int frame, unsigned int view,
                       struct CUstream_st* stream)
{
    if (!clean || !noisy || W < 1 || H < 1 || (long long)W * H > (1ll << 30)) return SIMSENSE_ERR_INVALID_ARG;
    NoiseParams n;
    n.mu = mu;
    n.sigma = sigma;
    n.k = k;
    n.theta = theta;
    n.seed = seed;
    if (check_noise(n) != SIMSENSE_OK) return SIMSENSE_ERR_INVALID_ARG;
    cudaError_t e = launch_noise(n, clean, noisy, nullptr, nullptr, W * H, frame, view, (cudaStream_t)stream);
    return e == cudaSuccess ? SIMSENSE_OK : SIMSENSE_ERR_CUDA;
}

int simsense_profile_read(simsense_t h, double* stage_ms, int* n_calls)
{
    if (!h) return SIMSENSE_ERR_INVALID_ARG;
    ProfileRing& r = h->prof;
    double tot[SIMSENSE_NUM_STAGES] = {0};
    DeviceGuard g(h->device);
    for (int c = 0; c < r.count; c++) {
        for (int st = 0; st < SIMSENSE_NUM_STAGES; st++) {
            cudaEvent_t a = r.ev[c * 2 * SIMSENSE_NUM_STAGES + 2 * st];
            cudaEvent_t b = r.ev[c * 2 * SIMSENSE_NUM_STAGES + 2 * st + 1];
            cudaError_t e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e != cudaSuccess) return cuda_fail(h, e);
            tot[st] += ms;
        }
    }
    if (stage_ms)
        for (int st = 0; st < SIMSENSE_NUM_STAGES; st++) stage_ms[st] = tot[st];
    if (n_calls) *n_calls = r.count;
    r.count = 0;
    return SIMSENSE_OK;
}

const char* simsense_stage_name(int i)
{
    switch (i) {
        case SIMSENSE_STAGE_CENSUS: return "census";
        case SIMSENSE_STAGE_COST: return "cost";
        case SIMSENSE_STAGE_PATHS: return "paths";
        case SIMSENSE_STAGE_SELECT: return "select";
        default: return nullptr;
    }
}

int simsense_device_status(simsense_t h, struct CUstream_st* stream)
{
    if (!h) return SIMSENSE_ERR_INVALID_ARG;
    DeviceGuard g(h->device);
    int v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&v, h->s.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(h->s.status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e);
    return v == 0 ? SIMSENSE_OK : v;
}

size_t simsense_scratch_bytes(simsense_t h)
{
    return h ? h->s.bytes : 0;
}

int simsense_destroy(simsense_t h)
{
    if (!h) return SIMSENSE_OK;
    DeviceGuard g(h->device);
    free_scratch(h->s);
    free_profile(h->prof);
    free_rectify(h);
    delete h;
    return SIMSENSE_OK;
}

namespace {

struct Notify {
    int fd;
    unsigned long long tag;
};

// Runs on the CUDA driver's callback thread once the stream reaches it: writes
// the tag (8 bytes, one atomic pipe write) and makes no CUDA call.
void CUDART_CB notify_host(void* arg)
{
    Notify* n = static_cast<Notify*>(arg);
    const char* b = reinterpret_cast<const char*>(&n->tag);
    size_t left = sizeof(n->tag);
    while (left > 0) {
        const ssize_t w = write(n->fd, b, left);
        if (w < 0) {
            if (errno == EINTR) continue;
            break;
        }
        b += w;
        left -= (size_t)w;
    }
    delete n;
}

}  // namespace

int simsense_notify_on_completion(struct CUstream_st* stream, int fd, unsigned long long tag)
{
    if (fd < 0) return SIMSENSE_ERR_INVALID_ARG;
    Notify* n = new (std::nothrow) Notify{fd, tag};
    if (!n) return SIMSENSE_ERR_OOM;
    const cudaError_t e = cudaLaunchHostFunc((cudaStream_t)stream, notify_host, n);
    if (e != cudaSuccess) {
        delete n;
        cudaGetLastError();
        return SIMSENSE_ERR_CUDA;
    }
    return SIMSENSE_OK;
}

void simsense_test_fail_allocation(int nth)
{
    g_fail_alloc.store(nth > 0 ? nth : 0);
}

const char* simsense_strerror(int code)
{
    switch (code) {
        case SIMSENSE_OK: return "ok";
        case SIMSENSE_ERR_INVALID_ARG: return "invalid argument";
        case SIMSENSE_ERR_OOM: return "out of device memory";
        case SIMSENSE_ERR_CUDA: return "CUDA error";
        case SIMSENSE_ERR_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

int simsense_last_cuda_error(simsense_t h)
{
    return h ? h->last_cuda_error : 0;
}

}  // extern "C"
