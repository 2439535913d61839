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
};

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

// Optional outputs of the selection kernel (device pointers, may be null).
struct SelectDebug {
    uint16_t* aggregated;
    int16_t* disparity_int;
    float* disparity;
    uint8_t* mask;
};

cudaError_t launch_census(const Params& p, const uint8_t* left, const uint8_t* right,
                          void* codes_left, void* codes_right, cudaStream_t s);
cudaError_t launch_widen_codes(const Params& p, const void* codes, uint64_t* out, cudaStream_t s);
cudaError_t launch_cost(const Params& p, const void* codes_left, const void* codes_right,
                        uint8_t* cost, cudaStream_t s);
cudaError_t launch_paths(const Params& p, const uint8_t* cost, uint8_t* paths, cudaStream_t s);
cudaError_t launch_select(const Params& p, const uint8_t* paths, float* depth,
                          const SelectDebug& dbg, int* status, cudaStream_t s);

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
};
