// SGM cost aggregation along scanline paths (arxiv 2201.11924 Sec. VI-D:
// semi-global matching with Hamming cost; cost aggregation "accelerated with
// warp-based optimization").
//
// Every path direction r splits the image into independent scanlines (rows,
// columns or diagonals); one warp walks one scanline, its 32 lanes splitting
// the padded disparity range Dp = 32 * DPT, lane l holding the DPT consecutive
// disparities l*DPT .. l*DPT + DPT - 1 as DPT/2 packed 16-bit pairs.  At each
// pixel p the warp
//   1. takes C(p, .) from the byte cost volume (loaded one step ahead, so the
//      load latency overlaps the previous step);
//   2. evaluates  L(p,d) = C(p,d) + min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m'+P2) - m'
//      on the pairs: min(L'(d-1), L'(d+1)) of both cells of a pair is one
//      min.u16x2 of the pair shifted down and up by one cell (byte permutes
//      of neighbouring pairs, plus one shuffle from each neighbouring lane for
//      the cells beyond the lane's range), then +P1, min with L'(d), min with
//      m'+P2, and one 3-input add of C - m';
//   3. stores L(p, .) as bytes (L <= nbits + P2 <= 255) into the path volume,
//      layout [y][x][r][Dp] so that the selection kernel reads one pixel's
//      paths contiguously;
//   4. forms m = min_d L(p, d): a min.u16x2 over the lane's pairs, then the
//      warp minimum with redux.sync.
// Padded disparities carry cost 255 in the cost volume (see cost.cu).  The
// cells d = -1 and d = Dp beyond the first and last lane read 0x3FFF, larger
// than any m' + P2, which is the recurrence's +infinity.
#include "internal.h"
#include "simd.cuh"

namespace simsense {
namespace {

constexpr int kPathThreads = 256;
constexpr uint32_t kInfPair = 0x3fff3fffu;

// Path directions: the value at p comes from p - r.  The first four are the
// 4-path set (horizontal and vertical), the last four the diagonals.  The
// horizontal ones come first so that their long scanlines start first.
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
            const int k = scan - W + 1;
            x = rx > 0 ? 0 : W - 1;
            y = ry > 0 ? k : H - 1 - k;
        }
    }
    return true;
}

// Raw bytes of NP pairs (2*NP consecutive bytes, aligned to 2*NP when NP is
// 1, 2 or 4; to 2 when NP is 3).
template <int NP>
struct Raw { uint32_t w[(NP + 1) / 2]; };

template <int NP>
__device__ __forceinline__ Raw<NP> load_raw(const uint8_t* p)
{
    Raw<NP> r;
    if constexpr (NP == 1) {
        r.w[0] = __ldg(reinterpret_cast<const unsigned short*>(p));
    } else if constexpr (NP == 2) {
        r.w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
    } else if constexpr (NP == 3) {
        const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
        r.w[0] = (uint32_t)__ldg(q) | ((uint32_t)__ldg(q + 1) << 16);
        r.w[1] = __ldg(q + 2);
    } else {
        uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
        r.w[0] = v.x;
        r.w[1] = v.y;
    }
    return r;
}

template <int NP>
__device__ __forceinline__ void unpack(const Raw<NP>& r, uint32_t (&c)[NP])
{
#pragma unroll
    for (int k = 0; k < NP; k++) c[k] = (k & 1) ? hi_bytes(r.w[k >> 1]) : lo_bytes(r.w[k >> 1]);
}

template <int NP>
__device__ __forceinline__ void store_pairs(uint8_t* p, const uint32_t (&L)[NP])
{
    if constexpr (NP == 1) {
        *reinterpret_cast<unsigned short*>(p) = (unsigned short)__byte_perm(L[0], 0, 0x0020);
    } else if constexpr (NP == 2) {
        __stcs(reinterpret_cast<unsigned int*>(p), pack_bytes(L[0], L[1]));
    } else if constexpr (NP == 3) {
        unsigned short* q = reinterpret_cast<unsigned short*>(p);
        q[0] = (unsigned short)__byte_perm(L[0], 0, 0x0020);
        q[1] = (unsigned short)__byte_perm(L[1], 0, 0x0020);
        q[2] = (unsigned short)__byte_perm(L[2], 0, 0x0020);
    } else {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2(pack_bytes(L[0], L[1]), pack_bytes(L[2], L[3])));
    }
}

template <int NP>
__global__ void __launch_bounds__(kPathThreads)
sgm_paths_kernel(const uint8_t* __restrict__ C, int W, int H, int P1, int P2, int paths,
                 uint8_t* __restrict__ vol)
{
    constexpr int DPT = 2 * NP;
    constexpr int Dp = 32 * DPT;
    const int r = blockIdx.y;
    int rx, ry;
    path_dir(r, rx, ry);
    const int lane = threadIdx.x & 31;
    const int scan = blockIdx.x * (kPathThreads / 32) + (threadIdx.x >> 5);
    int x, y;
    if (!scan_start(scan, rx, ry, W, H, x, y)) return;   // uniform across the warp

    const uint32_t p1 = (uint32_t)P1 * 0x10001u;
    const uint32_t p2 = (uint32_t)P2 * 0x10001u;
    const uint8_t* cbase = C + lane * DPT;
    uint8_t* obase = vol + (size_t)r * Dp + lane * DPT;
    const size_t ostride = (size_t)paths * Dp;
    const int step = ry * W + rx;            // pixel index increment along the path

    size_t pix = (size_t)y * W + x;
    Raw<NP> raw = load_raw<NP>(cbase + pix * Dp);
    uint32_t Lp[NP];
    uint32_t mm = 0, cap = 0;
    bool first = true;
    for (;;) {
        uint32_t Cp[NP];
        unpack<NP>(raw, Cp);
        const int xn = x + rx, yn = y + ry;
        const bool more = xn >= 0 && xn < W && yn >= 0 && yn < H;   // uniform
        if (more) raw = load_raw<NP>(cbase + (pix + step) * Dp);

        uint32_t L[NP];
        if (first) {
#pragma unroll
            for (int k = 0; k < NP; k++) L[k] = Cp[k];
            first = false;
        } else {
            uint32_t lo = __shfl_up_sync(0xffffffffu, Lp[NP - 1], 1);
            uint32_t hi = __shfl_down_sync(0xffffffffu, Lp[0], 1);
            if (lane == 0) lo = kInfPair;
            if (lane == 31) hi = kInfPair;
            uint32_t S[NP + 1];
            S[0] = shift_pair(lo, Lp[0]);
#pragma unroll
            for (int k = 1; k < NP; k++) S[k] = shift_pair(Lp[k - 1], Lp[k]);
            S[NP] = shift_pair(Lp[NP - 1], hi);
#pragma unroll
            for (int k = 0; k < NP; k++) {
                uint32_t t = vmin2(S[k], S[k + 1]) + p1;
                t = vmin2(vmin2(t, Lp[k]), cap);
                L[k] = t + Cp[k] - mm;      // no borrow: every half of t is >= m'
            }
        }
        store_pairs<NP>(obase + pix * ostride, L);
        uint32_t mn = L[0];
#pragma unroll
        for (int k = 1; k < NP; k++) mn = vmin2(mn, L[k]);
        const uint32_t m = __reduce_min_sync(0xffffffffu, hmin(mn));
        mm = m * 0x10001u;
        cap = mm + p2;
#pragma unroll
        for (int k = 0; k < NP; k++) Lp[k] = L[k];
        if (!more) break;
        x = xn;
        y = yn;
        pix += step;
    }
}

template <int NP>
cudaError_t launch_t(const Params& p, const uint8_t* C, uint8_t* vol, cudaStream_t s)
{
    const int nscan = p.W + p.H - 1;   // the most scanlines any direction has
    const int warps = kPathThreads / 32;
    dim3 grid((nscan + warps - 1) / warps, p.paths);
    sgm_paths_kernel<NP><<<grid, kPathThreads, 0, s>>>(C, p.W, p.H, p.P1, p.P2, p.paths, vol);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_paths(const Params& p, const uint8_t* C, uint8_t* paths, cudaStream_t s)
{
    switch (p.dpt) {
        case 2: return launch_t<1>(p, C, paths, s);
        case 4: return launch_t<2>(p, C, paths, s);
        case 6: return launch_t<3>(p, C, paths, s);
        case 8: return launch_t<4>(p, C, paths, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace simsense
