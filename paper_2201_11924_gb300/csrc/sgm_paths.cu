// SGM cost aggregation along scanline paths (arxiv 2201.11924 Sec. VI-D:
// semi-global matching with Hamming cost; cost aggregation "accelerated with
// warp-based optimization").
//
// Every path direction r splits the image into independent scanlines (rows,
// columns or diagonals).  A group of G lanes walks one scanline (G = 8, 16 or
// 32 so that a lane holds 8 disparities, or 6 when Dp = 192; a warp walks
// 32 / G scanlines side by side); lane l of a group holds the disparities
// l*DPT .. l*DPT + DPT - 1 of the padded range Dp as DPT/2 packed 16-bit
// pairs.  At each pixel p the group
//   1. takes C(p, .) from the byte cost volume (loaded 8 steps ahead, so the
//      load latency overlaps the recurrence);
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
//      group minimum with redux.sync.
// The scanlines of a warp may differ in length (diagonals); the warp runs to
// the longest and the lanes of a finished scanline stop loading and storing.
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

// Entry pixel of scanline `scan` of direction (rx, ry) and the number of
// pixels on it (0 if there is no such scanline).  Entry pixels are those whose
// predecessor p - r lies outside the image.
__device__ __forceinline__ int scan_start(int scan, int rx, int ry, int W, int H, int& x, int& y)
{
    if (ry == 0) {
        if (scan >= H) return 0;
        y = scan;
        x = rx > 0 ? 0 : W - 1;
        return W;
    }
    if (rx == 0) {
        if (scan >= W) return 0;
        x = scan;
        y = ry > 0 ? 0 : H - 1;
        return H;
    }
    if (scan >= W + H - 1) return 0;
    if (scan < W) {                   // entries on the first row the path meets
        x = scan;
        y = ry > 0 ? 0 : H - 1;
    } else {                          // entries on the first column, other rows
        const int k = scan - W + 1;
        x = rx > 0 ? 0 : W - 1;
        y = ry > 0 ? k : H - 1 - k;
    }
    const int nx = rx > 0 ? W - x : x + 1;
    const int ny = ry > 0 ? H - y : y + 1;
    return nx < ny ? nx : ny;
}

// Raw bytes of NP pairs (2*NP consecutive bytes; 8-byte aligned for NP = 4,
// 4-byte for NP = 2, 2-byte otherwise).
template <int NP>
struct Raw { uint32_t w[(NP + 1) / 2]; };

__device__ __forceinline__ uint64_t keep_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

template <int NP>
__device__ __forceinline__ Raw<NP> load_raw(const uint8_t* p, uint64_t pol)
{
    Raw<NP> r;
    if constexpr (NP == 1) {
        unsigned short v;
        asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
        r.w[0] = v;
    } else if constexpr (NP == 2) {
        asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r.w[0]) : "l"(p), "l"(pol));
    } else if constexpr (NP == 3) {
        const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
        r.w[0] = (uint32_t)__ldg(q) | ((uint32_t)__ldg(q + 1) << 16);
        r.w[1] = __ldg(q + 2);
    } else {
        asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;"
                     : "=r"(r.w[0]), "=r"(r.w[1]) : "l"(p), "l"(pol));
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
        __stcs(reinterpret_cast<unsigned short*>(p), (unsigned short)__byte_perm(L[0], 0, 0x0020));
    } else if constexpr (NP == 2) {
        __stcs(reinterpret_cast<unsigned int*>(p), pack_bytes(L[0], L[1]));
    } else if constexpr (NP == 3) {
        unsigned short* q = reinterpret_cast<unsigned short*>(p);
        __stcs(q, (unsigned short)__byte_perm(L[0], 0, 0x0020));
        __stcs(q + 1, (unsigned short)__byte_perm(L[1], 0, 0x0020));
        __stcs(q + 2, (unsigned short)__byte_perm(L[2], 0, 0x0020));
    } else {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2(pack_bytes(L[0], L[1]), pack_bytes(L[2], L[3])));
    }
}

// (m, m) with m the minimum over the group's cells: the lane minimum is
// duplicated into both halves, so the 32-bit group minimum of redux.sync is
// the pair minimum as well.
template <int NP>
__device__ __forceinline__ uint32_t group_min(const uint32_t (&L)[NP], unsigned gmask)
{
    uint32_t mn = L[0];
#pragma unroll
    for (int k = 1; k < NP; k++) mn = vmin2(mn, L[k]);
    mn = vmin2(mn, __byte_perm(mn, 0, 0x1032));
    return __reduce_min_sync(gmask, mn);
}

// G lanes walk one scanline (32 / G scanlines per warp), each holding NP pairs.
// The cost of the next PF pixels is kept in flight in a register ring (slot
// i % PF, a static index inside the PF-times unrolled loop), which hides the
// DRAM latency behind PF steps of the recurrence.
template <int NP, int G, int PF>
__global__ void __launch_bounds__(kPathThreads)
sgm_paths_kernel(const uint8_t* __restrict__ C, int W, int H, int P1, int P2, int paths,
                 uint8_t* __restrict__ vol)
{
    constexpr int DPT = 2 * NP;
    constexpr int Dp = G * DPT;
    constexpr int SPW = 32 / G;
    const int r = blockIdx.y;
    int rx, ry;
    path_dir(r, rx, ry);
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int scan = (blockIdx.x * (kPathThreads / 32) + (threadIdx.x >> 5)) * SPW + lane / G;
    int x = 0, y = 0;
    const int len = scan_start(scan, rx, ry, W, H, x, y);
    const int n = SPW > 1 ? (int)__reduce_max_sync(0xffffffffu, (unsigned)len) : len;
    if (n == 0) return;                       // uniform across the warp
    const unsigned gmask = SPW > 1 ? (((1u << G) - 1u) << ((lane / G) * G)) : 0xffffffffu;

    const uint32_t p1 = (uint32_t)P1 * 0x10001u;
    const uint32_t p2 = (uint32_t)P2 * 0x10001u;
    const long long pix0 = (long long)y * W + x;
    const long long step = (long long)ry * W + rx;      // pixel index increment along the path
    const long long cstep = step * Dp;
    const long long ostep = step * paths * Dp;
    const uint8_t* cf = C + pix0 * Dp + gl * DPT;        // cost of the next pixel to fetch
    uint8_t* op = vol + (pix0 * paths + r) * Dp + gl * DPT;
    const uint64_t pol = keep_policy();

    Raw<NP> ring[PF] = {};
#pragma unroll
    for (int k = 0; k < PF; k++) {
        if (k < len) ring[k] = load_raw<NP>(cf, pol);
        cf += cstep;
    }
    // L' = 0 and m' = 0 before the entry pixel make the recurrence return
    // exactly C there, which is the path's start condition.
    uint32_t Lp[NP];
#pragma unroll
    for (int k = 0; k < NP; k++) Lp[k] = 0;
    uint32_t mm = 0, cap = p2;

    for (int base = 0; base < n; base += PF) {
#pragma unroll
        for (int k = 0; k < PF; k++) {
            const int i = base + k;
            if (i >= n) break;                 // uniform
            uint32_t Cp[NP];
            unpack<NP>(ring[k], Cp);
            if (i + PF < len) ring[k] = load_raw<NP>(cf, pol);
            cf += cstep;
            uint32_t lo = __shfl_up_sync(0xffffffffu, Lp[NP - 1], 1, G);
            uint32_t hi = __shfl_down_sync(0xffffffffu, Lp[0], 1, G);
            if (gl == 0) lo = kInfPair;
            if (gl == G - 1) hi = kInfPair;
            uint32_t S[NP + 1];
            S[0] = shift_pair(lo, Lp[0]);
#pragma unroll
            for (int q = 1; q < NP; q++) S[q] = shift_pair(Lp[q - 1], Lp[q]);
            S[NP] = shift_pair(Lp[NP - 1], hi);
#pragma unroll
            for (int q = 0; q < NP; q++) {
                uint32_t t = vmin2(S[q], S[q + 1]) + p1;
                t = vmin2(vmin2(t, Lp[q]), cap);
                Lp[q] = t + Cp[q] - mm;      // no borrow: every half of t is >= m'
            }
            if (i < len) store_pairs<NP>(op, Lp);
            op += ostep;
            mm = group_min<NP>(Lp, gmask);
            cap = mm + p2;
        }
    }
}

template <int NP, int G>
cudaError_t launch_t(const Params& p, const uint8_t* C, uint8_t* vol, cudaStream_t s)
{
    constexpr int PF = 8;
    const int nscan = p.W + p.H - 1;          // the most scanlines any direction has
    const int per_block = (kPathThreads / 32) * (32 / G);
    dim3 grid((nscan + per_block - 1) / per_block, p.paths);
    sgm_paths_kernel<NP, G, PF><<<grid, kPathThreads, 0, s>>>(C, p.W, p.H, p.P1, p.P2, p.paths, vol);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_paths(const Params& p, const uint8_t* C, uint8_t* paths, cudaStream_t s)
{
    switch (p.Dp) {                            // lanes per scanline x 8 (or 6) disparities per lane
        case 64: return launch_t<4, 8>(p, C, paths, s);
        case 128: return launch_t<4, 16>(p, C, paths, s);
        case 192: return launch_t<3, 32>(p, C, paths, s);
        case 256: return launch_t<4, 32>(p, C, paths, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace simsense
