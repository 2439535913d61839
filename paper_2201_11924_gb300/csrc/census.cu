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

template <typename CodeT>
__global__ void __launch_bounds__(kTX * kTY)
census_kernel(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right, int W, int H,
              int ww, int wh, CodeT* __restrict__ out_left, CodeT* __restrict__ out_right)
{
    __shared__ uint8_t tile[kTileH * kTileW];
    const uint8_t* img = blockIdx.z ? right : left;
    CodeT* out = blockIdx.z ? out_right : out_left;
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
    const uint8_t c = t[ry * kTileW + rx];
    CodeT code = 0;
    for (int dy = 0; dy < wh; dy++) {
        for (int dx = 0; dx < ww; dx++) {
            if (dy == ry && dx == rx) continue;
            code = (code << 1) | (CodeT)(t[dy * kTileW + dx] < c ? 1u : 0u);
        }
    }
    out[(size_t)y * W + x] = code;
}

__global__ void widen_kernel(const uint32_t* __restrict__ in, uint64_t* __restrict__ out, size_t n)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

}  // namespace

cudaError_t launch_census(const Params& p, const uint8_t* left, const uint8_t* right,
                          void* codes_left, void* codes_right, cudaStream_t s)
{
    dim3 block(kTX, kTY);
    dim3 grid((p.W + kTX - 1) / kTX, (p.H + kTY - 1) / kTY, 2);
    if (p.wide_codes)
        census_kernel<uint64_t><<<grid, block, 0, s>>>(left, right, p.W, p.H, p.win_w, p.win_h,
                                                       (uint64_t*)codes_left, (uint64_t*)codes_right);
    else
        census_kernel<uint32_t><<<grid, block, 0, s>>>(left, right, p.W, p.H, p.win_w, p.win_h,
                                                       (uint32_t*)codes_left, (uint32_t*)codes_right);
    return cudaGetLastError();
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
