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
//   4. forms m = min_d L(p, d): a min.u16x2 over the lane's pairs, then a
//      shuffle butterfly over the group.
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

// Loads the 2*NP cost bytes at p into r when pred holds, else leaves r as it
// is.  The predicate sits inside the asm and r is a read-write operand, so
// the load writes the ring registers directly and nothing waits for it until
// the ring slot is unpacked PF steps later (a load into a temporary followed
// by a conditional move would wait for the data at once).
template <int NP>
__device__ __forceinline__ void load_raw(Raw<NP>& r, const uint8_t* p, uint64_t pol, bool pred)
{
    if constexpr (NP == 1) {
        asm volatile("{\n\t.reg .pred q;\n\t.reg .b16 h;\n\tsetp.ne.b32 q, %2, 0;\n\t"
                     "@q ld.global.nc.L2::cache_hint.b16 h, [%1], %3;\n\t"
                     "@q cvt.u32.u16 %0, h;\n\t}"
                     : "+r"(r.w[0]) : "l"(p), "r"((int)pred), "l"(pol));
    } else if constexpr (NP == 2) {
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t"
                     "@q ld.global.nc.L2::cache_hint.b32 %0, [%1], %3;\n\t}"
                     : "+r"(r.w[0]) : "l"(p), "r"((int)pred), "l"(pol));
    } else if constexpr (NP == 3) {
        asm volatile("{\n\t.reg .pred q;\n\t.reg .b16 a, b, c;\n\tsetp.ne.b32 q, %3, 0;\n\t"
                     "@q ld.global.nc.L2::cache_hint.b16 a, [%2], %4;\n\t"
                     "@q ld.global.nc.L2::cache_hint.b16 b, [%2+2], %4;\n\t"
                     "@q ld.global.nc.L2::cache_hint.b16 c, [%2+4], %4;\n\t"
                     "@q mov.b32 %0, {a, b};\n\t"
                     "@q cvt.u32.u16 %1, c;\n\t}"
                     : "+r"(r.w[0]), "+r"(r.w[1]) : "l"(p), "r"((int)pred), "l"(pol));
    } else {
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t"
                     "@q ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %4;\n\t}"
                     : "+r"(r.w[0]), "+r"(r.w[1]) : "l"(p), "r"((int)pred), "l"(pol));
    }
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
// duplicated into both halves, then reduced over the group: one redux.sync
// for a whole warp, a shuffle butterfly for a partial-warp group (measured
// faster here than redux.sync with a partial mask).
template <int NP, int G>
__device__ __forceinline__ uint32_t group_min(const uint32_t (&L)[NP])
{
    uint32_t mn = L[0];
#pragma unroll
    for (int k = 1; k < NP; k++) mn = vmin2(mn, L[k]);
    mn = vmin2(mn, __byte_perm(mn, 0, 0x1032));
    if constexpr (G == 32) {
        return __reduce_min_sync(0xffffffffu, mn);
    } else {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) mn = vmin2(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        return mn;
    }
}

// G lanes walk one scanline (32 / G scanlines per warp), each holding NP pairs.
// The cost of the next PF pixels is kept in flight in a register ring (slot
// i % PF, a static index inside the PF-times unrolled loop), which hides the
// DRAM latency behind PF steps of the recurrence.
template <int NP, int G, int PF>
__device__ __forceinline__ void walk(const uint8_t* __restrict__ C, int W, int H, int P1, int P2, int paths,
                                     uint8_t* __restrict__ vol, int r, int rx, int ry)
{
    constexpr int DPT = 2 * NP;
    constexpr int Dp = G * DPT;
    constexpr int SPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int scan = (blockIdx.x * (kPathThreads / 32) + (threadIdx.x >> 5)) * SPW + lane / G;
    int x = 0, y = 0;
    const int len = scan_start(scan, rx, ry, W, H, x, y);
    const int n = SPW > 1 ? (int)__reduce_max_sync(0xffffffffu, (unsigned)len) : len;
    if (n == 0) return;                       // uniform across the warp

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
        load_raw<NP>(ring[k], cf, pol, k < len);
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
            load_raw<NP>(ring[k], cf, pol, i + PF < len);
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
            mm = group_min<NP, G>(Lp);
            cap = mm + p2;
        }
    }
}

// The horizontal directions have the longest scanlines (W steps of a
// recurrence that is inherently sequential), so they decide the kernel's
// critical path: they are walked by whole warps (NPH pairs per lane, group
// minimum by one redux.sync, the shortest step latency measured).  The other
// directions are throughput-bound and use G-lane groups with NP pairs.
template <int NP, int G, int NPH, int PF, int N>
__global__ void __launch_bounds__(kPathThreads)
sgm_paths_kernel(PairTable<N> pt, int W, int H, int P1, int P2, int paths)
{
    static_assert(G * 2 * NP == 32 * 2 * NPH, "both layouts cover the same padded range");
    const uint8_t* __restrict__ C = pt.p[blockIdx.z].cost;      // blockIdx.z = pair
    uint8_t* __restrict__ vol = pt.p[blockIdx.z].vol;
    const int r = blockIdx.y;
    int rx, ry;
    path_dir(r, rx, ry);
    if (ry == 0) walk<NPH, 32, PF>(C, W, H, P1, P2, paths, vol, r, rx, ry);
    else walk<NP, G, PF>(C, W, H, P1, P2, paths, vol, r, rx, ry);
}

template <int NP, int G, int NPH, int PF, int N>
cudaError_t paths_chunk(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    // blocks: enough for the non-horizontal directions (W + H - 1 scanlines at
    // most, 32/G per warp) and for the horizontal ones (H scanlines, 1 per warp)
    const int per_block = (kPathThreads / 32) * (32 / G);
    const int nb = (p.W + p.H - 1 + per_block - 1) / per_block;
    const int nbh = (p.H + kPathThreads / 32 - 1) / (kPathThreads / 32);
    dim3 grid(nb > nbh ? nb : nbh, p.paths, n);
    sgm_paths_kernel<NP, G, NPH, PF, N><<<grid, kPathThreads, 0, s>>>(pt, p.W, p.H, p.P1, p.P2, p.paths);
    return cudaGetLastError();
}

template <int NP, int G, int NPH, int N>
cudaError_t paths_pf(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, cudaStream_t s)
{
    switch (t.prefetch) {
        case 4: return paths_chunk<NP, G, NPH, 4, N>(p, pairs, n, s);
        case 12: return paths_chunk<NP, G, NPH, 12, N>(p, pairs, n, s);
        default: return paths_chunk<NP, G, NPH, 8, N>(p, pairs, n, s);
    }
}

template <int N>
cudaError_t paths_dp(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, cudaStream_t s)
{
    switch (p.Dp) {                            // lanes per scanline x 8 (or 6) disparities per lane
        case 64: return paths_pf<4, 8, 1, N>(p, pairs, n, t, s);
        case 128: return paths_pf<4, 16, 2, N>(p, pairs, n, t, s);
        case 192: return paths_pf<3, 32, 3, N>(p, pairs, n, t, s);
        case 256: return paths_pf<4, 32, 4, N>(p, pairs, n, t, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_paths(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        cudaError_t e = c == 1 ? paths_dp<1>(p, pairs + b, 1, t, s) : paths_dp<kMaxBatch>(p, pairs + b, c, t, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace simsense
