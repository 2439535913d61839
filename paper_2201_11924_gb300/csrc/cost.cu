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

}  // namespace

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
