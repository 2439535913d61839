// SGM cost aggregation along scanline paths (arxiv 2201.11924 Sec. VI-D:
// "semi-global matching ... with hamming distance as the cost function";
// cost aggregation "accelerated with warp-based optimization").
//
// Every path direction r splits the image into independent scanlines (rows,
// columns or diagonals).  One warp walks one scanline; its 32 lanes split the
// disparity range, lane l holding d = l*DPT .. l*DPT+DPT-1.  At each pixel p a
// lane
//   1. recomputes the matching cost C(p, d) = popcount(cL(p) ^ cR(p - d)) of
//      its disparities (nbits where x - d < 0), never storing a cost volume;
//   2. applies the recurrence
//        L(p,d) = C(p,d) + min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m'+P2) - m'
//      taking L'(d-1) / L'(d+1) at its range ends from the neighbouring lanes
//      by shuffle and m' = min_d L' from a warp min-reduction (redux.sync);
//   3. stores L(p, .) as bytes (L <= nbits + P2 <= 255) into the direction's
//      slice of the path volume, layout [r][y][x][Dp], d fastest.
// Disparities d >= D that pad the range to 32*DPT carry a large constant cost,
// so they never become the minimum and never undercut the m'+P2 term.
#include "internal.h"

namespace simsense {
namespace {

constexpr int kPathThreads = 256;
constexpr uint32_t kPadCost = 1u << 12;   // > any real L' + P2 (L' <= 255, P2 <= 255)
constexpr uint32_t kInf = 1u << 20;

// Path directions: the value at p comes from p - r.  The first four are the
// 4-path set (horizontal and vertical), the last four the diagonals.
__device__ __forceinline__ void path_dir(int r, int& rx, int& ry)
{
    switch (r) {
        case 0: rx = 1; ry = 0; break;
        case 1: rx = -1; ry = 0; break;
        case 2: rx = 0; ry = 1; break;
        case 3: rx = 0; ry = -1; break;
        case 4: rx = 1; ry = 1; break;
        case 5: rx = -1; ry = 1; break;
        case 6: rx = 1; ry = -1; break;
        default: rx = -1; ry = -1; break;
    }
}

// Entry pixel of scanline `scan` of direction (rx, ry); false if there is none.
// Entry pixels are those whose predecessor p - r lies outside the image.
__device__ __forceinline__ bool scan_start(int scan, int rx, int ry, int W, int H, int& x, int& y)
{
    if (ry == 0) {
        if (scan >= H) return false;
        y = scan;
        x = rx > 0 ? 0 : W - 1;
    } else if (rx == 0) {
        if (scan >= W) return false;
        x = scan;
        y = ry > 0 ? 0 : H - 1;
    } else {
        if (scan >= W + H - 1) return false;
        if (scan < W) {               // entries on the first row the path meets
            x = scan;
            y = ry > 0 ? 0 : H - 1;
        } else {                      // entries on the first column, other rows
            int k = scan - W + 1;
            x = rx > 0 ? 0 : W - 1;
            y = ry > 0 ? k : H - 1 - k;
        }
    }
    return true;
}

__device__ __forceinline__ uint32_t popc(uint32_t v) { return __popc(v); }
__device__ __forceinline__ uint32_t popc(uint64_t v) { return __popcll(v); }

template <int DPT>
__device__ __forceinline__ void store_bytes(uint8_t* dst, const uint32_t (&v)[DPT])
{
    if constexpr (DPT == 2) {
        *reinterpret_cast<uint16_t*>(dst) = (uint16_t)(v[0] | (v[1] << 8));
    } else if constexpr (DPT == 4) {
        *reinterpret_cast<uint32_t*>(dst) = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
    } else if constexpr (DPT == 6) {
        uint16_t* d16 = reinterpret_cast<uint16_t*>(dst);
        d16[0] = (uint16_t)(v[0] | (v[1] << 8));
        d16[1] = (uint16_t)(v[2] | (v[3] << 8));
        d16[2] = (uint16_t)(v[4] | (v[5] << 8));
    } else {
        uint2 w;
        w.x = v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24);
        w.y = v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24);
        *reinterpret_cast<uint2*>(dst) = w;
    }
}

template <typename CodeT, int DPT>
__global__ void __launch_bounds__(kPathThreads)
sgm_paths_kernel(const CodeT* __restrict__ cL, const CodeT* __restrict__ cR, int W, int H, int D,
                 int Dp, int nbits, int P1, int P2, uint8_t* __restrict__ vol)
{
    const int r = blockIdx.y;
    int rx, ry;
    path_dir(r, rx, ry);
    const int lane = threadIdx.x & 31;
    const int scan = blockIdx.x * (kPathThreads / 32) + (threadIdx.x >> 5);
    int x, y;
    if (!scan_start(scan, rx, ry, W, H, x, y)) return;   // uniform across the warp

    const int d0 = lane * DPT;
    uint8_t* out = vol + (size_t)r * H * W * Dp + d0;
    uint32_t Lp[DPT];
    uint32_t mp = 0;
    bool first = true;
    for (; x >= 0 && x < W && y >= 0 && y < H; x += rx, y += ry) {
        const size_t pix = (size_t)y * W + x;
        const CodeT cl = cL[pix];
        uint32_t L[DPT];
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int d = d0 + j;
            uint32_t c;
            if (d >= D) c = kPadCost;
            else if (x - d < 0) c = (uint32_t)nbits;
            else c = popc(cl ^ cR[pix - d]);
            L[j] = c;
        }
        if (!first) {
            uint32_t lo = __shfl_up_sync(0xffffffffu, Lp[DPT - 1], 1);
            uint32_t hi = __shfl_down_sync(0xffffffffu, Lp[0], 1);
            if (lane == 0) lo = kInf;
            if (lane == 31) hi = kInf;
            const uint32_t cap = mp + (uint32_t)P2;
#pragma unroll
            for (int j = 0; j < DPT; j++) {
                const uint32_t a = j == 0 ? lo : Lp[j - 1];
                const uint32_t b = j == DPT - 1 ? hi : Lp[j + 1];
                uint32_t t = min(min(a, b) + (uint32_t)P1, Lp[j]);
                t = min(t, cap);
                L[j] += t - mp;
            }
        }
        first = false;
        store_bytes<DPT>(out + pix * Dp, L);
        uint32_t m = L[0];
#pragma unroll
        for (int j = 1; j < DPT; j++) m = min(m, L[j]);
        mp = __reduce_min_sync(0xffffffffu, m);
#pragma unroll
        for (int j = 0; j < DPT; j++) Lp[j] = L[j];
    }
}

template <typename CodeT, int DPT>
cudaError_t launch_t(const Params& p, const void* cl, const void* cr, uint8_t* vol, cudaStream_t s)
{
    const int nscan = p.W + p.H - 1;   // the most scanlines any direction has
    const int warps = kPathThreads / 32;
    dim3 grid((nscan + warps - 1) / warps, p.paths);
    sgm_paths_kernel<CodeT, DPT><<<grid, kPathThreads, 0, s>>>(
        (const CodeT*)cl, (const CodeT*)cr, p.W, p.H, p.D, p.Dp, p.nbits, p.P1, p.P2, vol);
    return cudaGetLastError();
}

template <typename CodeT>
cudaError_t launch_code(const Params& p, const void* cl, const void* cr, uint8_t* vol, cudaStream_t s)
{
    switch (p.dpt) {
        case 2: return launch_t<CodeT, 2>(p, cl, cr, vol, s);
        case 4: return launch_t<CodeT, 4>(p, cl, cr, vol, s);
        case 6: return launch_t<CodeT, 6>(p, cl, cr, vol, s);
        case 8: return launch_t<CodeT, 8>(p, cl, cr, vol, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_paths(const Params& p, const void* codes_left, const void* codes_right,
                         uint8_t* paths, cudaStream_t s)
{
    if (p.wide_codes) return launch_code<uint64_t>(p, codes_left, codes_right, paths, s);
    return launch_code<uint32_t>(p, codes_left, codes_right, paths, s);
}

}  // namespace simsense
