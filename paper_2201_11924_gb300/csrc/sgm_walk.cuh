// Device code of the SGM path aggregation shared by the path kernel and the
// fused batch kernel: scanline geometry, the cost ring, the recurrence on
// packed 16-bit pairs and the work-item numbering (the algorithm is described
// at the top of sgm_paths.cu).
#pragma once

#include "internal.h"
#include "simd.cuh"

namespace simsense {
namespace sgm {

constexpr int kPathThreads = 256;
constexpr uint32_t kInfPair = 0x3fff3fffu;

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

// Entry pixel of scanline `scan` of direction (rx, ry) and the number of
// pixels on it (0 if there is no such scanline).  Entry pixels are those whose
// predecessor p - r lies outside the image.  Diagonal scanlines 0 .. W-1 enter
// on the first row the path meets (x = scan), W .. W+H-2 on the first column.
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
    if (scan < W) {
        x = scan;
        y = ry > 0 ? 0 : H - 1;
    } else {
        const int k = scan - W + 1;
        x = rx > 0 ? 0 : W - 1;
        y = ry > 0 ? k : H - 1 - k;
    }
    const int nx = rx > 0 ? W - x : x + 1;
    const int ny = ry > 0 ? H - y : y + 1;
    return nx < ny ? nx : ny;
}

// Diagonal scanline of rank j (0 <= j < W + H - 1) in order of non-increasing
// length.  With m = min(W, H), M = max(W, H): M - m + 1 scanlines have length
// m, then every length l = m-1 .. 1 occurs twice, once entering on the first
// row (u = W - l steps from the path's starting corner) and once on the first
// column (k = H - l rows from it).
__device__ __forceinline__ int diag_scan(int j, int rx, int W, int H)
{
    const int m = W < H ? W : H;
    const int M = W < H ? H : W;
    const int full = M - m + 1;
    int u = -1, k = 0;
    if (j < full) {
        if (W >= H) u = j;
        else if (j == 0) u = 0;
        else k = j;
    } else {
        const int t = j - full;
        const int l = m - 1 - (t >> 1);
        if ((t & 1) == 0) u = W - l;
        else k = H - l;
    }
    if (u >= 0) return rx > 0 ? u : W - 1 - u;
    return W - 1 + k;
}

// Asynchronous copy of the lane's 4*NQ cost bytes into its shared-memory ring
// slot (skipped when pred is false), then a commit: every step commits one
// group, so "the copy of pixel i has landed" is "at most PF - 1 groups are
// still pending" (cp.async.wait_group PF - 1).
template <int NQ>
__device__ __forceinline__ void cp_cost(uint32_t dst, const uint8_t* src, bool pred)
{
    if (pred) {
        if constexpr (NQ == 1) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
        } else if constexpr (NQ == 2) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"(dst), "l"(src) : "memory");
        } else if constexpr (NQ == 3) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst), "l"(src) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst + 4), "l"(src + 4) : "memory");
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" :: "r"(dst + 8), "l"(src + 8) : "memory");
        } else {
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

template <int NQ>
__device__ __forceinline__ void lds_cost(uint32_t (&w)[NQ], uint32_t a)
{
    if constexpr (NQ == 1) {
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(w[0]) : "r"(a) : "memory");
    } else if constexpr (NQ == 2) {
        asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "r"(a) : "memory");
    } else if constexpr (NQ == 3) {
        asm volatile("ld.shared.b32 %0, [%3];\n\tld.shared.b32 %1, [%3+4];\n\tld.shared.b32 %2, [%3+8];"
                     : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]) : "r"(a) : "memory");
    } else {
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "r"(a) : "memory");
    }
}

// KEEP = false: streaming stores (the volume is read back only by a later
// launch, long after it has left L2); true: default stores, so that a reader
// soon after (the fused batch kernel's selection) can still find it in L2.
template <int NQ, bool KEEP = false>
__device__ __forceinline__ void store_words(uint8_t* p, const uint32_t (&w)[NQ])
{
    if constexpr (KEEP) {
        if constexpr (NQ == 1) {
            *reinterpret_cast<unsigned int*>(p) = w[0];
        } else if constexpr (NQ == 2) {
            *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        } else if constexpr (NQ == 3) {
            unsigned int* q = reinterpret_cast<unsigned int*>(p);
            q[0] = w[0];
            q[1] = w[1];
            q[2] = w[2];
        } else {
            *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else if constexpr (NQ == 1) {
        __stcs(reinterpret_cast<unsigned int*>(p), w[0]);
    } else if constexpr (NQ == 2) {
        __stcs(reinterpret_cast<uint2*>(p), make_uint2(w[0], w[1]));
    } else if constexpr (NQ == 3) {
        unsigned int* q = reinterpret_cast<unsigned int*>(p);
        __stcs(q, w[0]);
        __stcs(q + 1, w[1]);
        __stcs(q + 2, w[2]);
    } else {
        __stcs(reinterpret_cast<uint4*>(p), make_uint4(w[0], w[1], w[2], w[3]));
    }
}

// (m, m) with m the minimum over the group's cells: a three-input-min tree
// over the lane's 2*NQ pairs, the two halves, then the group.  For groups of
// 8 to 32 lanes, one whole-warp redux.sync per group, in which the other
// groups' lanes offer 0xffffffff: 32 / G independent reductions, a shorter
// chain than a butterfly of log2(G) dependent shuffles (the minimum m' is on
// the step-to-step chain of the recurrence); smaller groups use the
// butterfly.
template <int NQ, int G>
__device__ __forceinline__ uint32_t group_min(const uint32_t (&L)[2 * NQ])
{
    uint32_t mn;
    if constexpr (NQ == 1) {
        mn = vmin2(L[0], L[1]);
    } else if constexpr (NQ == 2) {
        mn = vmin2(vmin3(L[0], L[1], L[2]), L[3]);
    } else if constexpr (NQ == 3) {
        mn = vmin3(vmin3(L[0], L[1], L[2]), L[3], vmin3(L[4], L[5], L[5]));
    } else {
        mn = vmin3(vmin3(L[0], L[1], L[2]), vmin3(L[3], L[4], L[5]), vmin2(L[6], L[7]));
    }
    mn = vmin2(mn, __byte_perm(mn, 0, 0x1032));
    if constexpr (G >= 8) {
        constexpr int NG = 32 / G;
        const int grp = (threadIdx.x & 31) / G;
        uint32_t res = 0;
#pragma unroll
        for (int g = 0; g < NG; g++) {
            const uint32_t r = __reduce_min_sync(0xffffffffu, grp == g ? mn : 0xffffffffu);
            res = grp == g ? r : res;
        }
        return res;
    } else {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) mn = vmin2(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        return mn;
    }
}

// Steps base .. base + PF - 1 of a walk (fewer if the walk ends first).
// Guard = false: every lane's pixel i and prefetch target i + PF lie on its
// scanline, so loads and stores need no predicate; Guard = true: lanes whose
// scanline is shorter than the warp's longest stop loading and storing.
template <int NQ, int G, int PF, bool Guard, bool KEEP = false>
__device__ __forceinline__ void walk_steps(int base, int n, int len, uint32_t ring, const uint8_t*& cf,
                                           long long cstep, uint8_t*& op, long long ostep,
                                           uint32_t (&Lc)[2 * NQ], uint32_t (&Lp)[2 * NQ], uint32_t& mm,
                                           uint32_t& cap, uint32_t p1, uint32_t p2, uint32_t edge_lo,
                                           uint32_t edge_hi)
{
#pragma unroll
    for (int k = 0; k < PF; k++) {
        const int i = base + k;
        if (Guard && i >= n) break;            // uniform
        uint32_t cw[NQ];
        cp_wait<PF - 1>();                     // the copy of pixel i has landed
        lds_cost<NQ>(cw, ring + k * 512);
        // O pair of the quad below the lane's range, E pair above it
        const uint32_t o_below = __shfl_up_sync(0xffffffffu, Lp[2 * NQ - 1], 1, G) + edge_lo;
        const uint32_t e_above = __shfl_down_sync(0xffffffffu, Lp[0], 1, G) + edge_hi;
        uint32_t L[2 * NQ], out[NQ];
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            const uint32_t Oprev = q == 0 ? o_below : Lp[2 * q - 1];
            const uint32_t Enext = q == NQ - 1 ? e_above : Lp[2 * q + 2];
            // E = (d0, d2): d + 1 is O = (d1, d3), d - 1 is (d-1, d1)
            const uint32_t tE = vmin2(vmin3(Lc[2 * q], Lp[2 * q + 1], shift_pair(Oprev, Lp[2 * q + 1])), cap);
            // O = (d1, d3): d - 1 is E = (d0, d2), d + 1 is (d2, d4)
            const uint32_t tO = vmin2(vmin3(Lc[2 * q + 1], Lp[2 * q], shift_pair(Lp[2 * q], Enext)), cap);
            // cost bytes (c0, c1, c2, c3) -> (c1, c3) by a permute, and
            // (c0, c2) = word - 256 (c1, c3), folded into the sum as a
            // multiply-add (off the permute and minimum pipe, unlike a mask)
            const uint32_t cO = __byte_perm(cw[q], 0, 0x4341);
            L[2 * q] = tE + cw[q] - mm - cO * 256u;   // no borrow: every half of t is >= m'
            L[2 * q + 1] = tO + cO - mm;
            out[q] = L[2 * q + 1] * 256u + L[2 * q];            // bytes (L0, L1, L2, L3)
        }
        if (!Guard || i < len) store_words<NQ, KEEP>(op, out);
        op += ostep;
        // slot k is free again (its bytes were read above): pixel i + PF
        cp_cost<NQ>(ring + k * 512, cf, Guard ? i + PF < len : true);
        cf += cstep;
        mm = group_min<NQ, G>(L);
        cap = mm + p2;
#pragma unroll
        for (int k2 = 0; k2 < 2 * NQ; k2++) {
            Lc[k2] = L[k2];
            Lp[k2] = L[k2] + p1;
        }
    }
}

// Walks scanline `scan` of direction r with G lanes per scanline and NQ quads
// per lane.  The cost of the next PF pixels is in flight into the warp's
// shared-memory ring: slot k (a static index inside the PF-times unrolled
// loop) holds 16 bytes per lane, so the warp's ring is PF x 512 bytes.
template <int NQ, int G, int PF, bool KEEP = false>
__device__ __forceinline__ void walk(const uint8_t* __restrict__ C, int W, int H, int P1, int P2, int paths,
                                     uint8_t* __restrict__ vol, int r, int rx, int ry, int scan)
{
    constexpr int DPT = 4 * NQ;
    constexpr int Dp = G * DPT;
    constexpr int SPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    int x = 0, y = 0;
    const int len = scan_start(scan, rx, ry, W, H, x, y);
    const int n = SPW > 1 ? (int)__reduce_max_sync(0xffffffffu, (unsigned)len) : len;
    if (n == 0) return;                       // uniform across the warp
    const int nmin = SPW > 1 ? (int)__reduce_min_sync(0xffffffffu, (unsigned)len) : len;

    const uint32_t p1 = (uint32_t)P1 * 0x10001u;
    const uint32_t p2 = (uint32_t)P2 * 0x10001u;
    // the shuffled-in neighbour cells beyond the first and last lane become
    // larger than any candidate (adding to the lane's own value keeps every
    // half below 2^15)
    const uint32_t edge_lo = gl == 0 ? kInfPair : 0u;
    const uint32_t edge_hi = gl == G - 1 ? kInfPair : 0u;
    const long long pix0 = (long long)y * W + x;
    const long long step = (long long)ry * W + rx;      // pixel index increment along the path
    const long long cstep = step * Dp;
    const long long ostep = step * paths * Dp;
    const uint8_t* cf = C + pix0 * Dp + gl * DPT;        // cost of the next pixel to fetch
    uint8_t* op = vol + (pix0 * paths + r) * Dp + gl * DPT;

    extern __shared__ __align__(16) uint8_t path_smem[];
    const uint32_t ring = (uint32_t)__cvta_generic_to_shared(path_smem) + (threadIdx.x >> 5) * PF * 512 + lane * 16;
#pragma unroll
    for (int k = 0; k < PF; k++) {
        cp_cost<NQ>(ring + k * 512, cf, k < len);
        cf += cstep;
    }
    // State before the entry pixel: L' = 0 and m' = 0, which makes the
    // recurrence return exactly C there (the path's start condition).
    // Lc = L' and Lp = L' + P1 per pair, E pairs at even and O pairs at odd
    // indices; cap = m' + P2 is applied after the three-input minimum of
    // L'(d) and L'(d -+ 1) + P1, which keeps it off the step-to-step chain
    // (m' -> cap -> L -> m'): min is associative, the result is the same.
    uint32_t Lc[2 * NQ], Lp[2 * NQ];
#pragma unroll
    for (int k = 0; k < 2 * NQ; k++) {
        Lc[k] = 0;
        Lp[k] = p1;
    }
    uint32_t mm = 0;
    uint32_t cap = p2;                        // m' + P2, applied after the three-input minimum

    // steps whose pixel and prefetch target lie on every lane's scanline
    const int nmain = nmin > PF ? (nmin - PF) / PF * PF : 0;
    int base = 0;
    for (; base < nmain; base += PF)
        walk_steps<NQ, G, PF, false, KEEP>(base, n, len, ring, cf, cstep, op, ostep, Lc, Lp, mm, cap, p1, p2,
                                     edge_lo, edge_hi);
    for (; base < n; base += PF)
        walk_steps<NQ, G, PF, true, KEEP>(base, n, len, ring, cf, cstep, op, ostep, Lc, Lp, mm, cap, p1, p2,
                                    edge_lo, edge_hi);
}

// Work items of one launch: warp-sized groups of scanlines, longest first.
struct Items {
    int nh, nv, nd;          // groups per direction: horizontal, vertical, diagonal
    int cls_h, cls_v, cls_d; // items per class (all directions and pairs)
    int total;
    bool h_first;
};

__host__ __device__ inline Items make_items(int W, int H, int paths, int npairs, int spw, int spwh)
{
    Items it;
    it.nh = (H + spwh - 1) / spwh;
    it.nv = (W + spw - 1) / spw;
    it.nd = (W + H - 1 + spw - 1) / spw;
    it.cls_h = 2 * npairs * it.nh;
    it.cls_v = 2 * npairs * it.nv;
    it.cls_d = paths == 8 ? 4 * npairs * it.nd : 0;
    it.total = it.cls_h + it.cls_v + it.cls_d;
    it.h_first = W >= H;
    return it;
}

// Work item `i` of a single pair (the numbering of make_items with one pair):
// the warp walks its group of scanlines of one direction.  Rows use NQH quads
// and GH lanes per scanline, the other directions NQ and G.
template <int NQ, int G, int NQH, int GH, int PF, bool KEEP>
__device__ __forceinline__ void walk_item(const uint8_t* __restrict__ C, uint8_t* __restrict__ vol, int W, int H,
                                          int P1, int P2, int paths, int i)
{
    constexpr int SPW = 32 / G, SPWH = 32 / GH;
    const int lane = threadIdx.x & 31;
    const Items it = make_items(W, H, paths, 1, SPW, SPWH);
    if (i >= it.total) return;
    int cls;
    const int first = it.h_first ? it.cls_h : it.cls_v;
    if (i < first) {
        cls = it.h_first ? 0 : 1;
    } else if (i < it.cls_h + it.cls_v) {
        cls = it.h_first ? 1 : 0;
        i -= first;
    } else {
        cls = 2;
        i -= it.cls_h + it.cls_v;
    }
    const int ndir = cls == 2 ? 4 : 2;
    const int g = i / ndir;
    const int r = (cls == 0 ? 0 : cls == 1 ? 2 : 4) + i % ndir;
    int rx, ry;
    path_dir(r, rx, ry);
    if (cls == 0) {
        walk<NQH, GH, PF, KEEP>(C, W, H, P1, P2, paths, vol, r, rx, ry, g * SPWH + lane / GH);
    } else {
        const int j = g * SPW + lane / G;
        const int scan = cls == 1 ? j : (j < W + H - 1 ? diag_scan(j, rx, W, H) : W + H - 1);
        walk<NQ, G, PF, KEEP>(C, W, H, P1, P2, paths, vol, r, rx, ry, scan);
    }
}

}  // namespace sgm
}  // namespace simsense
