// simsense_compute_noalloc: the whole depth stage without a handle and without
// allocating anything.
//
// Who needs this: some callers are not allowed to call cudaMalloc at all.
// A plugin inside a host application that owns every byte of device memory
// through its own pool, a real-time loop that forbids allocation after start-up
// (cudaMalloc can block the host and synchronise the device, stalling other
// streams), or a process whose device memory is already reserved by another
// framework's caching allocator.  simsense_create allocates the handle's
// scratch with cudaMalloc, so such callers cannot use it.  This entry point
// instead takes every parameter per call and runs the same census, cost, path
// and selection kernels on a scratch buffer that is a file-scope __device__ array
// of fixed size, part of the library image itself.
//
// Costs and rules of that choice:
//  - every GPU that loads this library's code holds the array
//    (SIMSENSE_NOALLOC_SCRATCH_BYTES) until the process exits;
//  - all calls share the one array, so calls whose kernels overlap on the GPU
//    (two streams, two host threads) race and corrupt each other's results;
//    callers must order them, e.g. by issuing them all on one stream;
//  - nothing in the array has to start at zero: every byte a call reads was
//    written earlier in that same call, so leftovers of a previous call are
//    harmless;
//  - problems whose scratch does not fit are rejected.
#include <mutex>

#include "internal.h"

using namespace simsense;

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol, never a device address: it must be translated with
// cudaGetSymbolAddress before a kernel may be given it.
static __device__ __align__(256) uint8_t g_noalloc_scratch[SIMSENSE_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices];   // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SIMSENSE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SIMSENSE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return SIMSENSE_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SIMSENSE_OK;
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" int simsense_compute_noalloc(const uint8_t* left_u8, const uint8_t* right_u8,
                                        float* depth_f32, int W, int H, int D, int census_win,
                                        int P1, int P2, int paths, int uniq_ratio, int lr_max_diff,
                                        float f, float baseline, int subpixel,
                                        struct CUstream_st* stream)
{
    if (!left_u8 || !right_u8 || !depth_f32) return SIMSENSE_ERR_INVALID_ARG;
    Params p{};
    int rc = make_params(p, W, H, D, census_win, P1, P2, paths, uniq_ratio, lr_max_diff, f, baseline, subpixel);
    if (rc != SIMSENSE_OK) return rc;

    // carve the fixed array: left codes | right codes | cost volume | path volume
    const size_t npx = (size_t)W * H;
    const size_t code_bytes = round256(npx * (p.wide_codes ? 8 : 4));
    const size_t cost_bytes = round256(npx * p.Dp);
    const size_t vol_bytes = (size_t)paths * npx * p.Dp;
    if (2 * code_bytes + cost_bytes + vol_bytes > (size_t)SIMSENSE_NOALLOC_SCRATCH_BYTES)
        return SIMSENSE_ERR_INVALID_ARG;
    void* base = nullptr;
    rc = scratch_address(&base);
    if (rc != SIMSENSE_OK) return rc;
    uint8_t* b = static_cast<uint8_t*>(base);
    void* codes_left = b;
    void* codes_right = b + code_bytes;
    uint8_t* cost = b + 2 * code_bytes;
    uint8_t* vol = cost + cost_bytes;

    cudaStream_t st = (cudaStream_t)stream;
    const PairPtrs pair{left_u8, right_u8, codes_left, codes_right, cost, vol, depth_f32};
    const Tuning tune{};
    const SelectDebug none{};
    cudaError_t e = launch_census(p, &pair, 1, st);
    if (e == cudaSuccess) e = launch_cost(p, &pair, 1, nullptr, st);
    if (e == cudaSuccess) e = launch_paths(p, &pair, 1, tune, st);
    if (e == cudaSuccess) e = launch_select(p, &pair, 1, tune, none, nullptr, st);
    return e == cudaSuccess ? SIMSENSE_OK : SIMSENSE_ERR_CUDA;
}
