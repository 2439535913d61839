// Hamming matching cost volume (arxiv 2201.11924 Sec. VI-D: "hamming distance
// as the cost function"; the section computes the cost from shared memory for
// data reuse).
//
// C(x, y, d) = popcount(cL(x, y) ^ cR(x - d, y)) for x - d >= 0, else nbits,
// stored once per cell as a byte, layout [y][x][Dp] (d fastest).  Every SGM
// path reads it instead of recomputing it: POPC issues at only 16 results per
// clock per SM on this GPU, so one evaluation per cell instead of one per path
// removes the dominant instruction of the aggregation.
//
// A block covers 64 pixels of one row; it stages their left codes and the
// right codes of [x0 - Dp + 1, x0 + 63] in shared memory.  Lane l of a warp
// handles d = l + 32 j, so the 32 lanes read 32 consecutive right codes
// (conflict-free) and write 32 consecutive bytes.  Disparities D <= d < Dp
// that pad the range get cost 255: with every real path cost at most
// nbits + P2 <= 255, a padded cell never becomes a strict minimum and never
// undercuts a real neighbour, so it behaves like the +infinity of the
// recurrence's boundary.
#include "internal.h"

namespace simsense {
namespace {

constexpr int kCostPix = 64;
constexpr int kCostThreads = 256;

__device__ __forceinline__ uint32_t popc(uint32_t v) { return __popc(v); }
__device__ __forceinline__ uint32_t popc(uint64_t v) { return __popcll(v); }

// blockIdx.z = pair.
template <typename CodeT, int DPT, int N>
__global__ void __launch_bounds__(kCostThreads)
cost_kernel(PairTable<N> pt, int W, int D, int nbits)
{
    constexpr int Dp = 32 * DPT;
    __shared__ CodeT sR[kCostPix + Dp];
    __shared__ CodeT sL[kCostPix];
    // fields read one by one: a reference to the parameter array element would
    // copy the table to local memory
    const CodeT* __restrict__ cL = static_cast<const CodeT*>(pt.p[blockIdx.z].codes_left);
    const CodeT* __restrict__ cR = static_cast<const CodeT*>(pt.p[blockIdx.z].codes_right);
    uint8_t* __restrict__ C = pt.p[blockIdx.z].cost;
    const int y = blockIdx.y, x0 = blockIdx.x * kCostPix;
    const CodeT* rowL = cL + (size_t)y * W;
    const CodeT* rowR = cR + (size_t)y * W;
    for (int i = threadIdx.x; i < kCostPix + Dp - 1; i += kCostThreads) {
        const int x = x0 - (Dp - 1) + i;
        sR[i] = (x >= 0 && x < W) ? rowR[x] : (CodeT)0;
    }
    for (int i = threadIdx.x; i < kCostPix; i += kCostThreads) {
        const int x = x0 + i;
        sL[i] = x < W ? rowL[x] : (CodeT)0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = warp; p < kCostPix; p += kCostThreads / 32) {
        const int x = x0 + p;
        if (x >= W) break;
        const CodeT cl = sL[p];
        uint8_t* out = C + ((size_t)y * W + x) * Dp + lane;
        const CodeT* sr = sR + p + Dp - 1 - lane;        // sr[-32 j] is cR(x - d), d = lane + 32 j
        if (x >= Dp - 1 && D == Dp) {                    // uniform: every cell is a real match
#pragma unroll
            for (int j = 0; j < DPT; j++) out[32 * j] = (uint8_t)popc(cl ^ sr[-32 * j]);
        } else {
#pragma unroll
            for (int j = 0; j < DPT; j++) {
                const int d = lane + 32 * j;
                uint32_t c;
                if (d >= D) c = 255u;
                else if (x < d) c = (uint32_t)nbits;
                else c = popc(cl ^ sr[-32 * j]);
                out[32 * j] = (uint8_t)c;
            }
        }
    }
}

template <typename CodeT, int N>
cudaError_t cost_chunk(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    dim3 grid((p.W + kCostPix - 1) / kCostPix, p.H, n);
    switch (p.dpt) {
        case 2: cost_kernel<CodeT, 2, N><<<grid, kCostThreads, 0, s>>>(pt, p.W, p.D, p.nbits); break;
        case 4: cost_kernel<CodeT, 4, N><<<grid, kCostThreads, 0, s>>>(pt, p.W, p.D, p.nbits); break;
        case 6: cost_kernel<CodeT, 6, N><<<grid, kCostThreads, 0, s>>>(pt, p.W, p.D, p.nbits); break;
        case 8: cost_kernel<CodeT, 8, N><<<grid, kCostThreads, 0, s>>>(pt, p.W, p.D, p.nbits); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int N>
cudaError_t cost_code(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    if (p.wide_codes) return cost_chunk<uint64_t, N>(p, pairs, n, s);
    return cost_chunk<uint32_t, N>(p, pairs, n, s);
}

// SGBM block cost (the variant Sec. VI-D describes: the Hamming distance
// between the local regions of the two pixels): the per-pixel cost volume
// `raw` averaged over the bw x bh block around each pixel (same d), over the
// block's pixels inside the image, rounded half up, into `out`.
// A block takes 32 pixels of one output row in two separable passes:
//   1. for every staged column (32 + bw - 1 pixels) and 4-byte word of the
//      disparity range, the sum over the bh input rows, kept in shared memory
//      as two 16-bit pairs (bytes 0 and 2, bytes 1 and 3; at most 49 x 255 <
//      2^16), so every input word is split into pairs once;
//   2. for every output pixel and word, the sum of the bw staged columns and
//      the division by the in-image pixel count n, a multiply-high by
//      floor(2^32 / n) + 1, exact for every numerator below 2^16 and n <= 81.
// Lanes take consecutive words of one pixel: coalesced loads, conflict-free
// shared-memory accesses.
constexpr int kBlkPix = 32;

struct Magic {
    uint32_t m[82];
};

// BW, BH (the block) and DP (the disparity pitch) are compile-time, so the
// taps unroll and the index arithmetic divides by constants.
template <int BW, int BH, int DP, int N>
__global__ void __launch_bounds__(256)
block_cost_kernel(PairTable<N> pt, int W, int H, Magic mg)
{
    constexpr int rx = BW / 2, ry = BH / 2;
    constexpr int span = kBlkPix + BW - 1;             // staged columns
    constexpr int words = DP / 4;                      // 4-byte words per pixel
    __shared__ uint2 col[span * words];                // column sums (even pairs, odd pairs)
    const uint32_t* __restrict__ raw = reinterpret_cast<const uint32_t*>(pt.p[blockIdx.z].vol);
    uint32_t* __restrict__ out = reinterpret_cast<uint32_t*>(pt.p[blockIdx.z].cost);
    const int y = blockIdx.y, x0 = blockIdx.x * kBlkPix;
    for (int i = threadIdx.x; i < span * words; i += blockDim.x) {
        const int w = i % words, px = i / words;
        const int xx = x0 - rx + px;
        uint32_t ev = 0, od = 0;
        if (xx >= 0 && xx < W) {
#pragma unroll
            for (int r = 0; r < BH; r++) {
                const int yy = y - ry + r;
                if (yy >= 0 && yy < H) {
                    const uint32_t v = __ldg(raw + ((size_t)yy * W + xx) * words + w);
                    ev += v & 0x00ff00ffu;
                    od += (v >> 8) & 0x00ff00ffu;
                }
            }
        }
        col[i] = make_uint2(ev, od);
    }
    __syncthreads();
    const int rows = min(y + ry, H - 1) - max(y - ry, 0) + 1;
    for (int i = threadIdx.x; i < kBlkPix * words; i += blockDim.x) {
        const int w = i % words, px = i / words;
        const int x = x0 + px;
        if (x >= W) break;                             // i grows with px
        uint32_t ev = 0, od = 0;
#pragma unroll
        for (int u = 0; u < BW; u++) {
            const uint2 c = col[(px + u) * words + w];
            ev += c.x;
            od += c.y;
        }
        const uint32_t n = (uint32_t)((min(x + rx, W - 1) - max(x - rx, 0) + 1) * rows);
        const uint32_t m = mg.m[n], h = n >> 1;
        const uint32_t c0 = __umulhi((ev & 0xffffu) + h, m), c2 = __umulhi((ev >> 16) + h, m);
        const uint32_t c1 = __umulhi((od & 0xffffu) + h, m), c3 = __umulhi((od >> 16) + h, m);
        out[((size_t)y * W + x) * words + w] = c0 | (c1 << 8) | (c2 << 16) | (c3 << 24);
    }
}

template <int N>
using K = void (*)(PairTable<N>, int, int, Magic);

template <int BW, int BH, int N>
K<N> block_kernel_dp(int Dp)
{
    switch (Dp) {
        case 64: return block_cost_kernel<BW, BH, 64, N>;
        case 128: return block_cost_kernel<BW, BH, 128, N>;
        case 192: return block_cost_kernel<BW, BH, 192, N>;
        default: return block_cost_kernel<BW, BH, 256, N>;
    }
}

// odd block sizes 1..7 in each direction
template <int N>
K<N> block_kernel_for(const Params& p)
{
    using F = K<N> (*)(int);
    static constexpr F table[4][4] = {
        {block_kernel_dp<1, 1, N>, block_kernel_dp<3, 1, N>, block_kernel_dp<5, 1, N>, block_kernel_dp<7, 1, N>},
        {block_kernel_dp<1, 3, N>, block_kernel_dp<3, 3, N>, block_kernel_dp<5, 3, N>, block_kernel_dp<7, 3, N>},
        {block_kernel_dp<1, 5, N>, block_kernel_dp<3, 5, N>, block_kernel_dp<5, 5, N>, block_kernel_dp<7, 5, N>},
        {block_kernel_dp<1, 7, N>, block_kernel_dp<3, 7, N>, block_kernel_dp<5, 7, N>, block_kernel_dp<7, 7, N>},
    };
    return table[p.block_h / 2][p.block_w / 2](p.Dp);
}

template <int N>
cudaError_t block_chunk(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    Magic mg{};
    for (uint32_t k = 1; k < 82; k++) mg.m[k] = (uint32_t)(0x100000000ull / k) + 1u;
    const K<N> kernel = block_kernel_for<N>(p);
    dim3 grid((p.W + kBlkPix - 1) / kBlkPix, p.H, n);
    kernel<<<grid, 256, 0, s>>>(pt, p.W, p.H, mg);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_block_cost(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        cudaError_t e = c == 1 ? block_chunk<1>(p, pairs + b, 1, s) : block_chunk<kMaxBatch>(p, pairs + b, c, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_cost(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        cudaError_t e = c == 1 ? cost_code<1>(p, pairs + b, 1, s) : cost_code<kMaxBatch>(p, pairs + b, c, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace simsense
