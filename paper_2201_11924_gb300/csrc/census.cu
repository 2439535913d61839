// Census transform of both views (arxiv 2201.11924 Sec. VI-D: the census step,
// computed from a shared-memory tile for data reuse as the section describes).
//
// One thread per pixel.  A block stages its 32 x 8 pixel tile plus the window
// halo in shared memory; pixels outside the image are staged as 255, which is
// never smaller than a centre value, so they contribute 0 bits as the
// definition requires.  Bits are appended in raster order (dy outer, dx
// inner), which leaves the first offset in the most significant position.
#include "internal.h"

namespace simsense {
namespace {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kTileW = kTX + kMaxWin - 1;
constexpr int kTileH = kTY + kMaxWin - 1;

// WW, WH > 0: the window is a compile-time constant and the loops unroll;
// WW = WH = 0: the window comes from ww, wh at run time.
// blockIdx.z = 2 * pair + view (0 = left, 1 = right).
template <typename CodeT, int WW, int WH, int N>
__global__ void __launch_bounds__(kTX * kTY)
census_kernel(PairTable<N> pt, int W, int H, int ww_rt, int wh_rt)
{
    __shared__ uint8_t tile[kTileH * kTileW];
    const int ww = WW > 0 ? WW : ww_rt;
    const int wh = WH > 0 ? WH : wh_rt;
    // fields read one by one: a reference to the parameter array element would
    // copy the table to local memory
    const int pair = blockIdx.z >> 1;
    const uint8_t* img = (blockIdx.z & 1) ? pt.p[pair].right : pt.p[pair].left;
    CodeT* out = static_cast<CodeT*>((blockIdx.z & 1) ? pt.p[pair].codes_right : pt.p[pair].codes_left);
    const int rx = ww >> 1, ry = wh >> 1;
    const int tw = kTX + 2 * rx, th = kTY + 2 * ry;
    const int gx0 = blockIdx.x * kTX - rx, gy0 = blockIdx.y * kTY - ry;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    for (int i = tid; i < tw * th; i += kTX * kTY) {
        int tx = i % tw, ty = i / tw;
        int gx = gx0 + tx, gy = gy0 + ty;
        tile[ty * kTileW + tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * W + gx] : 255;
    }
    __syncthreads();
    const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kTY + threadIdx.y;
    if (x >= W || y >= H) return;
    const uint8_t* t = tile + threadIdx.y * kTileW + threadIdx.x;
    const int c = t[ry * kTileW + rx];
    // bit = [I(neighbour) < I(centre)] is the sign bit of the difference; the
    // code is built MSB first in raster order, the leading nbits - 32 bits
    // (64-bit codes) in the high word
    uint32_t hi = 0, lo = 0;
    if constexpr (WW > 0) {
        constexpr int nb = WW * WH - 1;
        int b = 0;
#pragma unroll
        for (int dy = 0; dy < WH; dy++) {
#pragma unroll
            for (int dx = 0; dx < WW; dx++) {
                if (dy == WH / 2 && dx == WW / 2) continue;
                const uint32_t bit = (uint32_t)((int)t[dy * kTileW + dx] - c) >> 31;
                if (nb - b > 32) hi = (hi << 1) | bit;
                else lo = (lo << 1) | bit;
                b++;
            }
        }
    } else {
        const int nb = ww * wh - 1;
        int b = 0;
        for (int dy = 0; dy < wh; dy++) {
            for (int dx = 0; dx < ww; dx++) {
                if (dy == ry && dx == rx) continue;
                const uint32_t bit = (uint32_t)((int)t[dy * kTileW + dx] - c) >> 31;
                if (nb - b > 32) hi = (hi << 1) | bit;
                else lo = (lo << 1) | bit;
                b++;
            }
        }
    }
    if constexpr (sizeof(CodeT) == 8) out[(size_t)y * W + x] = ((uint64_t)hi << 32) | lo;
    else out[(size_t)y * W + x] = lo;
}

__global__ void widen_kernel(const uint32_t* __restrict__ in, uint64_t* __restrict__ out, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

template <int N>
cudaError_t census_chunk(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    dim3 block(kTX, kTY);
    dim3 grid((p.W + kTX - 1) / kTX, (p.H + kTY - 1) / kTY, 2 * n);
    const int w = p.win_w, h = p.win_h;
    if (w == 7 && h == 7)
        census_kernel<uint64_t, 7, 7, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else if (w == 9 && h == 7)
        census_kernel<uint64_t, 9, 7, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else if (w == 5 && h == 5)
        census_kernel<uint32_t, 5, 5, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else if (p.wide_codes)
        census_kernel<uint64_t, 0, 0, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else
        census_kernel<uint32_t, 0, 0, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_census(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        cudaError_t e = c == 1 ? census_chunk<1>(p, pairs + b, 1, s) : census_chunk<kMaxBatch>(p, pairs + b, c, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_widen_codes(const Params& p, const void* codes, uint64_t* out, cudaStream_t s)
{
    size_t n = (size_t)p.W * p.H;
    if (p.wide_codes)
        return cudaMemcpyAsync(out, codes, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s);
    widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const uint32_t*)codes, out, n);
    return cudaGetLastError();
}

}  // namespace simsense
