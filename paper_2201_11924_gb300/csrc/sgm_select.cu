// Selection and post-processing (arxiv 2201.11924 Sec. VI-D: best disparity
// candidates, uniqueness test, quadratic sub-pixel fitting, left-right
// consistency check, disparity to depth) fused into one kernel per image row.
//
// One block per row.  A group of G lanes takes one pixel (a warp takes 32 / G
// pixels side by side), each lane holding the same DPT consecutive
// disparities as in the path kernel.  A
// pixel's path costs are contiguous ([y][x][r][Dp]); a lane sums its bytes of
// every path with two masked 32-bit adds per word (even and odd bytes as
// packed 16-bit pairs; the sum of 8 bytes cannot carry out of a half).  Then
//   - d* = argmin S with the smallest d on ties: warp min-reduction of the key
//     (S << 9) | d;
//   - the uniqueness test against every d with |d - d*| > 1;
//   - every cell is offered to the right view: right pixel xr = x - d keeps
//     the minimum key over the cells mapping to it (shared-memory atomicMin),
//     which is argmin_d S(xr + d, d) with ties to the smallest d;
//   - the parabola through S(d*-1), S(d*), S(d*+1).
// When the whole row is in, each pixel's left-right check reads D_R(x - d*)
// and the depth f*b/d_f is written.
#include "internal.h"

namespace simsense {
namespace {

constexpr int kSelThreads = 512;
constexpr int kSelWarps = kSelThreads / 32;

// The lane's DPT bytes of one path, as words (2*NP bytes).
template <int NP>
struct Words { uint32_t w[(NP + 1) / 2]; };

// Loads the lane's bytes of one path when pred holds.  The predicate sits in
// the asm with the words as read-write operands, so the load lands in the
// buffer registers directly and is waited for only when the buffer is summed.
template <int NP>
__device__ __forceinline__ void load_words(Words<NP>& r, const uint8_t* p, bool pred)
{
    static_assert(NP == 3 || NP == 4, "lane groups hold 6 or 8 disparities");
    if constexpr (NP == 3) {
        asm volatile("{\n\t.reg .pred q;\n\t.reg .b16 a, b, c;\n\tsetp.ne.b32 q, %3, 0;\n\t"
                     "@q ld.global.cs.b16 a, [%2];\n\t"
                     "@q ld.global.cs.b16 b, [%2+2];\n\t"
                     "@q ld.global.cs.b16 c, [%2+4];\n\t"
                     "@q mov.b32 %0, {a, b};\n\t"
                     "@q cvt.u32.u16 %1, c;\n\t}"
                     : "+r"(r.w[0]), "+r"(r.w[1]) : "l"(p), "r"((int)pred));
    } else {
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t"
                     "@q ld.global.cs.v2.b32 {%0, %1}, [%2];\n\t}"
                     : "+r"(r.w[0]), "+r"(r.w[1]) : "l"(p), "r"((int)pred));
    }
}

template <int NP>
__device__ __forceinline__ void load_pixel(Words<NP> (&buf)[8], const uint8_t* src, int paths, int Dp, bool act)
{
#pragma unroll
    for (int r = 0; r < 8; r++) load_words<NP>(buf[r], src + r * Dp, act && r < paths);
}

// Sum of all paths for the lane's cells.  even[k] holds cells (4k, 4k+2),
// odd[k] cells (4k+1, 4k+3) of the lane's range, as 16-bit pairs.
template <int NP>
__device__ __forceinline__ void sum_paths(const Words<NP> (&buf)[8], int paths,
                                          uint32_t (&even)[(NP + 1) / 2], uint32_t (&odd)[(NP + 1) / 2])
{
    constexpr int NW = (NP + 1) / 2;
#pragma unroll
    for (int k = 0; k < NW; k++) { even[k] = 0; odd[k] = 0; }
#pragma unroll
    for (int r = 0; r < 8; r++) {
        if (r < paths) {
#pragma unroll
            for (int k = 0; k < NW; k++) {
                even[k] += buf[r].w[k] & 0x00ff00ffu;
                odd[k] += (buf[r].w[k] >> 8) & 0x00ff00ffu;
            }
        }
    }
}

// One pixel of the row for one lane group: sum, winner, uniqueness, offers to
// the right view, parabola.  buf holds the lane's bytes of every path.
template <int NP, int G>
__device__ __forceinline__ void select_pixel(const Words<NP> (&buf)[8], int x, bool act, int y, int W, int D,
                                             int paths, int uniq, uint32_t umagic, int subpixel, int gl,
                                             unsigned gmask, uint16_t* sw, uint32_t* keyR, float* dispf,
                                             int16_t* dstar, uint8_t* ufail, const SelectDebug& dbg)
{
    constexpr int DPT = 2 * NP;
    constexpr int Dp = G * DPT;
    constexpr int NW = (NP + 1) / 2;
    const int d0 = gl * DPT;
    const size_t pix = (size_t)y * W + x;
uint32_t even[NW], odd[NW];
sum_paths<NP>(buf, paths, even, odd);
    // cell j of the lane (d = d0 + j): word j/4, byte j%4
    uint32_t S[DPT];
#pragma unroll
    for (int j = 0; j < DPT; j++) {
        const uint32_t w = (j & 1) ? odd[j >> 2] : even[j >> 2];
        S[j] = (j & 2) ? (w >> 16) : (w & 0xffffu);
    }
    // every cell of the group is real and matches inside the image
    const bool interior = D == Dp && x >= Dp - 1;   // uniform per group
    uint32_t kmin = 0xffffffffu;
    if (interior) {
#pragma unroll
        for (int j = 0; j < DPT; j++) kmin = min(kmin, (S[j] << 9) | (uint32_t)(d0 + j));
    } else {
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int d = d0 + j;
            if (d < D) kmin = min(kmin, (S[j] << 9) | (uint32_t)d);
        }
    }
    kmin = __reduce_min_sync(gmask, kmin);
    const int ds = (int)(kmin & 511u);
    const uint32_t smin = kmin >> 9;

    // uniqueness: (100 - u) S(d) < 100 S(d*)  <=>  S(d) < T = ceil(100 S(d*) / (100 - u)),
    // the division done as a multiply-high by umagic = floor(2^32 / (100 - u)) + 1,
    // exact for numerators below 2^18; 100 - u = 1 (no magic in 32 bits) divides by one
    bool bad = false;
    if (uniq > 0) {
        const uint32_t num = 100u * smin + (uint32_t)(99 - uniq);
        const uint32_t T = uniq == 99 ? num : __umulhi(num, umagic);
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int d = d0 + j;
            if ((uint32_t)(d - ds + 1) > 2u && d < D && S[j] < T) bad = true;
        }
    }
    bad = (__ballot_sync(0xffffffffu, bad) & gmask) != 0;

    if (act) {
        if (interior) {
#pragma unroll
            for (int j = 0; j < DPT; j++) {
                sw[d0 + j] = (uint16_t)S[j];
                atomicMin(&keyR[x - d0 - j], (S[j] << 9) | (uint32_t)(d0 + j));
            }
        } else {
#pragma unroll
            for (int j = 0; j < DPT; j++) {
                const int d = d0 + j;
                if (d < D) {
                    sw[d] = (uint16_t)S[j];
                    if (d <= x) atomicMin(&keyR[x - d], (S[j] << 9) | (uint32_t)d);
                }
            }
        }
        if (dbg.aggregated) {
#pragma unroll
            for (int j = 0; j < DPT; j++)
                if (d0 + j < D) dbg.aggregated[pix * D + d0 + j] = (uint16_t)S[j];
        }
    }
    __syncwarp();
    if (gl == 0 && act) {
        float df = (float)ds;
        if (subpixel && ds >= 1 && ds <= D - 2) {
            const int sm = sw[ds - 1], sp = sw[ds + 1], s0 = (int)smin;
            df = (float)ds + __fdiv_rn((float)(sm - sp), (float)(2 * (sm + sp - 2 * s0)));
        }
        dispf[x] = df;
        dstar[x] = (int16_t)ds;
        ufail[x] = bad ? 1 : 0;
    }
    __syncwarp();
}

template <int NP, int G>
__global__ void __launch_bounds__(kSelThreads)
sgm_select_kernel(const uint8_t* __restrict__ vol, int paths, int W, int D, int uniq, uint32_t umagic,
                  int lr_max_diff, int subpixel, float fb, float* __restrict__ depth, SelectDebug dbg)
{
    constexpr int DPT = 2 * NP;
    constexpr int Dp = G * DPT;
    constexpr int SPW = 32 / G;               // pixels a warp takes at once
    constexpr int NW = (NP + 1) / 2;
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* keyR = reinterpret_cast<uint32_t*>(smem);              // W
    float* dispf = reinterpret_cast<float*>(keyR + W);               // W
    uint16_t* sbuf = reinterpret_cast<uint16_t*>(dispf + W);         // kSelWarps * SPW x Dp
    int16_t* dstar = reinterpret_cast<int16_t*>(sbuf + kSelWarps * SPW * Dp);  // W
    uint8_t* ufail = reinterpret_cast<uint8_t*>(dstar + W);          // W

    const int y = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, sub = lane / G;
    const unsigned gmask = SPW > 1 ? (((1u << G) - 1u) << (sub * G)) : 0xffffffffu;
    for (int i = threadIdx.x; i < W; i += kSelThreads) keyR[i] = 0xffffffffu;
    __syncthreads();

    const int d0 = gl * DPT;
    const size_t pstride = (size_t)paths * Dp;
    uint16_t* sw = sbuf + (warp * SPW + sub) * Dp;
    const uint8_t* row = vol + (size_t)y * W * pstride + d0;
    constexpr int kStride = kSelWarps * SPW;   // pixels the block takes per round
    Words<NP> bufA[8], bufB[8];
    const int x0 = warp * SPW + sub;
    load_pixel<NP>(bufA, row + (size_t)(x0 < W ? x0 : 0) * pstride, paths, Dp, x0 < W);
    for (int xb = warp * SPW; xb < W; xb += 2 * kStride) {     // uniform per warp
        const int xa = xb + sub, xbn = xa + kStride, xc = xa + 2 * kStride;
        load_pixel<NP>(bufB, row + (size_t)(xbn < W ? xbn : 0) * pstride, paths, Dp, xbn < W);
        select_pixel<NP, G>(bufA, xa, xa < W, y, W, D, paths, uniq, umagic, subpixel, gl, gmask, sw, keyR,
                            dispf, dstar, ufail, dbg);
        if (xb + kStride < W) {                                 // uniform per warp
            load_pixel<NP>(bufA, row + (size_t)(xc < W ? xc : 0) * pstride, paths, Dp, xc < W);
            select_pixel<NP, G>(bufB, xbn, xbn < W, y, W, D, paths, uniq, umagic, subpixel, gl, gmask, sw,
                                keyR, dispf, dstar, ufail, dbg);
        }
    }
    __syncthreads();

    for (int x = threadIdx.x; x < W; x += kSelThreads) {
        const size_t pix = (size_t)y * W + x;
        const int ds = dstar[x];
        int m = ufail[x];
        if (lr_max_diff >= 0) {
            const int xr = x - ds;
            if (xr < 0) {
                m |= 2;
            } else {
                const int dr = (int)(keyR[xr] & 511u);
                const int diff = ds > dr ? ds - dr : dr - ds;
                if (diff > lr_max_diff) m |= 2;
            }
        }
        const float df = dispf[x];
        if (!(df > 0.0f)) m |= 4;
        depth[pix] = m == 0 ? __fdiv_rn(fb, df) : 0.0f;
        if (dbg.disparity_int) dbg.disparity_int[pix] = (int16_t)ds;
        if (dbg.disparity) dbg.disparity[pix] = m == 0 ? df : -1.0f;
        if (dbg.mask) dbg.mask[pix] = (uint8_t)m;
    }
}

template <int NP, int G>
cudaError_t launch_t(const Params& p, const uint8_t* vol, float* depth, const SelectDebug& dbg,
                     cudaStream_t s)
{
    // keyR + dispf + dstar + ufail per pixel of the row, one S row per pixel group
    const size_t smem = (size_t)p.W * (4 + 4 + 2 + 1) + (size_t)kSelWarps * (32 / G) * p.Dp * 2 + 16;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sgm_select_kernel<NP, G>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const uint32_t umagic = (p.uniq > 0 && p.uniq < 99) ? (uint32_t)(0x100000000ull / (uint64_t)(100 - p.uniq)) + 1u : 0u;
    sgm_select_kernel<NP, G><<<p.H, kSelThreads, smem, s>>>(vol, p.paths, p.W, p.D, p.uniq, umagic,
                                                             p.lr_max_diff, p.subpixel, p.fb, depth, dbg);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_select(const Params& p, const uint8_t* paths, float* depth, const SelectDebug& dbg,
                          cudaStream_t s)
{
    switch (p.Dp) {                            // the path kernel's lane groups
        case 64: return launch_t<4, 8>(p, paths, depth, dbg, s);
        case 128: return launch_t<4, 16>(p, paths, depth, dbg, s);
        case 192: return launch_t<3, 32>(p, paths, depth, dbg, s);
        case 256: return launch_t<4, 32>(p, paths, depth, dbg, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace simsense
