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
//  - the status word is sticky: a call whose bounded wait gave up leaves
//    SIMSENSE_ERR_TIMEOUT there until simsense_noalloc_status reads and clears
//    it (it starts at zero when the module loads);
//  - the first call on a device looks up the array's address (and, with lazy
//    module loading, loads the library's device code there, which is when the
//    array is reserved), so it belongs in the caller's start-up, before any
//    stream capture;
//  - problems whose scratch does not fit are rejected.
#include <mutex>

#include "internal.h"

using namespace simsense;

// The scratch itself, and the status word of the calls' bounded device-side
// waits (SIMSENSE_ERR_TIMEOUT once one gave up; zero when the module loads).
// In host code these names are only stand-ins for the device symbols, never
// device addresses: they must be translated with cudaGetSymbolAddress before a
// kernel may be given them.
static __device__ __align__(256) uint8_t g_noalloc_scratch[SIMSENSE_NOALLOC_SCRATCH_BYTES];
static __device__ int g_noalloc_status;

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_mu;
struct Addrs {
    void* scratch = nullptr;   // device address of g_noalloc_scratch
    int* status = nullptr;     // device address of g_noalloc_status
};
Addrs g_addr[kMaxDevices];     // per device

// Device addresses of the scratch array and the status word on the current
// device, looked up once per device (with that device current) and cached.
// Under lazy module loading the first lookup also loads the library's device
// code on that device and reserves the array there.  The cache is not
// refreshed after cudaDeviceReset.
int device_addrs(Addrs* out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SIMSENSE_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return SIMSENSE_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    Addrs& a = g_addr[dev];
    if (!a.scratch || !a.status) {
        void* p = nullptr;
        void* q = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_status);
        if (e != cudaSuccess || !p || !q) {
            cudaGetLastError();   // leave no error pending for the caller's next CUDA call
            return SIMSENSE_ERR_CUDA;
        }
        a.scratch = p;
        a.status = static_cast<int*>(q);
    }
    *out = a;
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
    const size_t vol_bytes = path_volume_bytes(p);
    if (2 * code_bytes + cost_bytes + vol_bytes > (size_t)SIMSENSE_NOALLOC_SCRATCH_BYTES)
        return SIMSENSE_ERR_INVALID_ARG;
    Addrs a;
    rc = device_addrs(&a);
    if (rc != SIMSENSE_OK) return rc;
    uint8_t* b = static_cast<uint8_t*>(a.scratch);
    void* codes_left = b;
    void* codes_right = b + code_bytes;
    uint8_t* cost = b + 2 * code_bytes;
    uint8_t* vol = cost + cost_bytes;

    cudaStream_t st = (cudaStream_t)stream;
    const PairPtrs pair{left_u8, right_u8, codes_left, codes_right, cost, vol, depth_f32};
    const Tuning tune{};
    const SelectDebug none{};
    cudaError_t e = launch_census(p, &pair, 1, st);
    if (e == cudaSuccess) e = launch_cost(p, &pair, 1, a.status, st);
    if (e == cudaSuccess) e = launch_paths(p, &pair, 1, tune, nullptr, st);
    if (e == cudaSuccess) e = launch_select(p, &pair, 1, tune, none, a.status, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SIMSENSE_ERR_CUDA;
    }
    return SIMSENSE_OK;
}

extern "C" int simsense_noalloc_status(struct CUstream_st* stream)
{
    Addrs a;
    const int rc = device_addrs(&a);
    if (rc != SIMSENSE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, a.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(a.status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SIMSENSE_ERR_CUDA;
    }
    return v == 0 ? SIMSENSE_OK : v;
}
