// Internal declarations shared by the CUDA translation units of libsimsense.
// Nothing here is part of the public ABI (include/simsense.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "simsense.h"

namespace simsense {

// Largest census window side the kernels stage in shared memory.
constexpr int kMaxWin = 15;
// Largest disparity range.
constexpr int kMaxD = 256;
// Largest image width (the selection kernel keeps per-pixel arrays of a row
// next to its copy ring in shared memory).
constexpr int kMaxW = 8192;

struct Params {
    int W, H, D;
    int win_w, win_h, nbits;
    int P1, P2, paths;
    int uniq, lr_max_diff;
    int subpixel;
    float f, baseline, fb;   // fb = (float)((double)f * (double)baseline)
    int dpt;                 // disparities per lane of a 32-lane scanline group (2, 4, 6, 8)
    int Dp;                  // padded disparity pitch = 32 * dpt
    bool wide_codes;         // census codes need 64 bits (nbits > 32)
    // variants (Sec. VI-D): centre-symmetric census, SGBM block cost over
    // block_w x block_h (1 x 1 = per-pixel cost), median filter (0 = off, 3, 5)
    int census_cs = 0;
    int block_w = 1, block_h = 1;
    int median = 0;
    // test of the bounded waits (SIMSENSE_OPT_TEST_STALL): the cost stage
    // issues no MMAs and gives up after a short wait
    int test_stall = 0;
};

// Whether the SGBM block cost changes anything: a block that covers a single
// in-image pixel everywhere (1 pixel across in each direction where the
// image is 1 pixel across or the block is) averages each cost with itself,
// so the per-pixel cost is the block cost.  Otherwise every pixel's block
// holds at least 2 in-image pixels.
inline bool block_active(const Params& p)
{
    return (p.block_w > 1 && p.W > 1) || (p.block_h > 1 && p.H > 1);
}

// Applies a variant option to p (re-deriving nbits and the code width) after
// checking the ranges; returns a SIMSENSE status.
int set_variant(Params& p, int opt, int value);

// Rectification (Sec. VI-D): checks a camera, computes a view's per-pixel
// map (x0, y0, ax, ay) and resamples both views through their maps.
int check_camera(const simsense_camera_t& c);
cudaError_t launch_rect_map(const simsense_camera_t& c, int W, int H, short4* map, cudaStream_t s);
cudaError_t launch_remap(const uint8_t* raw0, const short4* map0, uint8_t* out0, const uint8_t* raw1,
                         const short4* map1, uint8_t* out1, int W, int H, cudaStream_t s);

// Sensor-noise model (Sec. VI-C) and generator seed.
struct NoiseParams {
    float mu = 0.0f, sigma = 0.0f, k = 1.0f, theta = 1.0f;
    uint64_t seed = 0;
};
int check_noise(const NoiseParams& n);
// Noise of one view (clean1 == nullptr) or of two views (views view0 and
// view0 + 1) of npx pixels each; clean and noisy may be the same buffer.
cudaError_t launch_noise(const NoiseParams& n, const uint8_t* clean0, uint8_t* noisy0, const uint8_t* clean1,
                         uint8_t* noisy1, int npx, uint32_t frame, uint32_t view0, cudaStream_t s);

// Device scratch of one handle (all owned by the handle).
struct Scratch {
    void* codes_left = nullptr;    // H x W uint32 or uint64
    void* codes_right = nullptr;
    uint8_t* cost = nullptr;       // H x W x Dp uint8, Hamming cost C
    uint8_t* paths = nullptr;      // H x W x paths x Dp uint8, L_r per path
    int* status = nullptr;         // device status word (SIMSENSE_ERR_TIMEOUT after a bounded wait gave up)
    uint8_t* stage_left = nullptr; // host-call staging: H x W uint8
    uint8_t* stage_right = nullptr;
    float* stage_depth = nullptr;  // H x W float32
    size_t bytes = 0;
};

// Device buffers of one pair (one stereo pair of a batch, or the single pair
// of a plain call).
struct PairPtrs {
    const uint8_t* left;
    const uint8_t* right;
    void* codes_left;        // H x W uint32 or uint64
    void* codes_right;
    uint8_t* cost;           // H x W x Dp
    uint8_t* vol;            // H x W x paths x Dp
    float* depth;            // H x W
};

// Pairs of one launch, passed by value as a kernel parameter (nothing to
// upload per call; a captured graph keeps it).  Kernels take the pair index
// from the grid.
constexpr int kMaxBatch = 32;
template <int N>
struct PairTable {
    PairPtrs p[N];
};

// Launch choices the autotuner may change (defaults are the measured best
// for 1280x720, D = 128 on GB300).
struct Tuning {
    int prefetch = 16;       // path kernel: pixels of cost in flight per scanline (8, 12 or 16)
    int select_blocks = 1;   // selection kernel: 1 = one 1024-thread block per SM, 2 = two 512-thread blocks
};

// Programmatic dependent launch.  The census, cost and selection kernels are
// launched with programmatic stream serialisation (the path kernel with a
// plain launch, which measured faster after the cost kernel): the next kernel on the stream may
// be scheduled once every block of the running one has started, and it waits
// at its first instruction (pdl_wait: griddepcontrol.wait, which returns once
// the previous kernel has completed and its memory is visible; at once when
// the kernel was launched without the attribute) before it reads or writes
// anything.  What overlaps is the launch and the block scheduling of the next
// kernel with the tail of the running one.
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
// Lets the next kernel be scheduled (called by every block once it runs).
__device__ __forceinline__ void pdl_trigger()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The same launch without programmatic stream serialisation: the kernel
// starts once its predecessor in the stream has completed (griddepcontrol.wait
// then returns at once).
template <typename... KArgs, typename... Args>
cudaError_t launch_plain(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Limits of the current device (read once per device).
struct DevLimits {
    int nsm = 0, optin = 0, per_sm = 0;
};
cudaError_t device_limits(DevLimits& out);

// Raises a kernel's dynamic shared-memory limit to `bytes` when a launch needs
// more than any earlier launch of that kernel on the current device, and on
// its first call asks for the largest shared-memory carve-out.
cudaError_t ensure_smem(const void* kernel, size_t bytes);

// Every device allocation of the library's scratch (cudaMalloc, except that
// the test hook simsense_test_fail_allocation can make one of them fail as
// if the device were out of memory).
cudaError_t dev_alloc(void** ptr, size_t bytes);

// Optional outputs of the selection kernel (device pointers, may be null).
struct SelectDebug {
    uint16_t* aggregated;
    int16_t* disparity_int;
    float* disparity;
    uint8_t* mask;
};

// Each launcher runs one stage for pairs[0 .. n-1], all with parameters p
// (n > kMaxBatch is split into several launches).
cudaError_t launch_census(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s);
cudaError_t launch_widen_codes(const Params& p, const void* codes, uint64_t* out, cudaStream_t s);
cudaError_t launch_cost(const Params& p, const PairPtrs* pairs, int n, int* status, cudaStream_t s);
// SGBM block cost: pairs[i].vol holds the per-pixel cost volume on entry,
// pairs[i].cost receives its block mean.
cudaError_t launch_block_cost(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s);
// k x k median filter of the disparity map disp (invalid = 0) into depth,
// and the filtered disparity (invalid = -1) into disp_out when it is not null.
cudaError_t launch_median(const Params& p, const float* disp, float* depth, float* disp_out, cudaStream_t s);
// Path aggregation: the path volume holds, per pixel, P planes of L_r bytes.
// dbg_paths (n == 1 only; may be null): paths x H x W x D bytes of every L_r,
// direction r in the oracle's order (->, <-, down, up, down-right, down-left,
// up-right, up-left), copied from the path kernel's output.
cudaError_t launch_paths(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, uint8_t* dbg_paths,
                         cudaStream_t s);
// The L_r planes of vol into the dense debug layout.
cudaError_t launch_unpack_paths(const Params& p, const uint8_t* vol, uint8_t* dbg_paths, cudaStream_t s);
cudaError_t launch_select(const Params& p, const PairPtrs* pairs, int n, const Tuning& t,
                          const SelectDebug& dbg, int* status, cudaStream_t s);

// Bytes of the path volume of one pair (what the path kernel writes and the
// selection kernel reads).
inline size_t path_volume_bytes(const Params& p)
{
    return (size_t)p.paths * p.W * p.H * p.Dp;
}

// One pair of a batch as the fused batch kernel reads it (device memory).
struct FusedPair {
    const uint8_t* cost;     // H x W x Dp
    uint8_t* vol;            // H x W x paths x Dp
    float* depth;            // H x W
    int W, H, D, Dp, paths, P1, P2;
    int uniq, lr_max_diff, subpixel;
    float fb;
    uint32_t umagic;         // the uniqueness test's multiply-high divisor for 100 - uniq
    int path_tasks;          // path tasks of the pair (8 work items each)
};

// Path tasks of a pair in the fused batch kernel.
int fused_path_tasks(const Params& p);
// One persistent launch over `ntasks` tasks (int4: kind 0 = path task / 1 =
// selection row, pair, index) of the pairs in `pairs`; ctl (1 + pairs ints)
// must be zero at launch.  cls: the parameters of the batch's ncls classes
// (the shared memory of the selection rows is sized for the largest).
cudaError_t launch_fused(const FusedPair* pairs, const int4* tasks, int ntasks, int* ctl, int* status,
                         const Params* cls, int ncls, int keep, cudaStream_t s);

// Multiply-high divisor of the uniqueness test (0 when u is 0 or 99).
inline uint32_t uniq_magic(int uniq)
{
    return (uniq > 0 && uniq < 99) ? (uint32_t)(0x100000000ull / (uint64_t)(100 - uniq)) + 1u : 0u;
}

// Validation and derived fields shared by every entry point that takes a
// parameter set (the ranges of simsense_create).
int make_params(Params& p, int W, int H, int D, int census_win, int P1, int P2, int paths,
                int uniq_ratio, int lr_max_diff, float f, float baseline, int subpixel);

}  // namespace simsense

// Stage timing record kept while SIMSENSE_OPT_PROFILE is on.
struct ProfileRing {
    static constexpr int kSlots = 4096;
    cudaEvent_t* ev = nullptr;    // kSlots x (2 * SIMSENSE_NUM_STAGES) events
    int count = 0;                // calls recorded since the last read
    bool on = false;
};

struct simsense_ctx {
    simsense::Params p;
    simsense::Scratch s;
    ProfileRing prof;
    int device = 0;
    int last_cuda_error = 0;
    bool noise_on = false;             // sensor noise before the census
    simsense::NoiseParams noise;
    uint32_t noise_frame = 0;          // frame index of the next compute call
    short4* rect_map[2] = {nullptr, nullptr};    // rectification maps (both or none)
    uint8_t* rect_img[2] = {nullptr, nullptr};   // rectified views
};
