// Census transform of both views (arxiv 2201.11924 Sec. VI-D: the census step,
// computed from a shared-memory tile for data reuse as the section describes).
//
// One thread per pixel.  A block stages its 32 x 8 pixel tile plus the window
// halo in shared memory.  Bits are appended in raster order (dy outer, dx
// inner), which leaves the first offset in the most significant position.
//  - Full census: bit = [I(p+o) < I(p)] for every offset o but the centre;
//    pixels outside the image are staged as 255, never smaller than a centre
//    value, so they contribute 0.
//  - Centre-symmetric census (CSCT, the variant Sec. VI-D names): bit =
//    [I(p+o) < I(p-o)] for the offsets o before the centre; a pair with a
//    pixel outside the image gives 0.  The first pixel of a pair is read from
//    a tile staged with 255 outside the image and the second from one staged
//    with 0, so either pixel outside makes the comparison false.
#include "internal.h"

#include <type_traits>

namespace simsense {
namespace {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kTileW = kTX + kMaxWin - 1;
constexpr int kTileH = kTY + kMaxWin - 1;

// WW, WH > 0: the window is a compile-time constant and the loops unroll;
// WW = WH = 0: the window comes from ww, wh at run time.  CS: centre-symmetric.
// blockIdx.z = 2 * pair + view (0 = left, 1 = right).
template <typename CodeT, int WW, int WH, bool CS, int N>
__global__ void __launch_bounds__(kTX * kTY)
census_kernel(PairTable<N> pt, int W, int H, int ww_rt, int wh_rt)
{
    __shared__ uint8_t tile[kTileH * kTileW];
    __shared__ uint8_t tile0[CS ? kTileH * kTileW : 1];   // CS: outside the image = 0
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
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        const uint8_t v = in ? img[(size_t)gy * W + gx] : 0;
        tile[ty * kTileW + tx] = in ? v : 255;
        if constexpr (CS) tile0[ty * kTileW + tx] = v;
    }
    __syncthreads();
    const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kTY + threadIdx.y;
    if (x >= W || y >= H) return;
    const uint8_t* t = tile + threadIdx.y * kTileW + threadIdx.x;
    const uint8_t* t0 = CS ? tile0 + threadIdx.y * kTileW + threadIdx.x : t;
    const int c = t[ry * kTileW + rx];
    // bit = [a < b] is the sign bit of a - b; the code is built MSB first in
    // raster order, the leading nbits - 32 bits (64-bit codes) in the high word
    uint32_t hi = 0, lo = 0;
    if constexpr (WW > 0) {
        constexpr int nb = CS ? (WW * WH - 1) / 2 : WW * WH - 1;
        int b = 0;
#pragma unroll
        for (int dy = 0; dy < WH; dy++) {
#pragma unroll
            for (int dx = 0; dx < WW; dx++) {
                if (dy == WH / 2 && dx == WW / 2) continue;
                if (CS && (dy > WH / 2 || (dy == WH / 2 && dx > WW / 2))) continue;
                const int other = CS ? (int)t0[(WH - 1 - dy) * kTileW + (WW - 1 - dx)] : c;
                const uint32_t bit = (uint32_t)((int)t[dy * kTileW + dx] - other) >> 31;
                if (nb - b > 32) hi = (hi << 1) | bit;
                else lo = (lo << 1) | bit;
                b++;
            }
        }
    } else {
        const int nb = CS ? (ww * wh - 1) / 2 : ww * wh - 1;
        int b = 0;
        for (int dy = 0; dy < wh; dy++) {
            for (int dx = 0; dx < ww; dx++) {
                if (dy == ry && dx == rx) continue;
                if (CS && (dy > ry || (dy == ry && dx > rx))) continue;
                const int other = CS ? (int)t0[(wh - 1 - dy) * kTileW + (ww - 1 - dx)] : c;
                const uint32_t bit = (uint32_t)((int)t[dy * kTileW + dx] - other) >> 31;
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

template <bool CS, int N>
cudaError_t census_launch(const Params& p, const PairTable<N>& pt, int n, cudaStream_t s)
{
    dim3 block(kTX, kTY);
    dim3 grid((p.W + kTX - 1) / kTX, (p.H + kTY - 1) / kTY, 2 * n);
    const int w = p.win_w, h = p.win_h;
    // the unrolled 7x7 and 9x7 windows: 48 / 62 bits (64-bit codes) for the
    // full census, 24 / 31 bits (32-bit codes) for the centre-symmetric one
    if (w == 7 && h == 7 && p.wide_codes == !CS)
        census_kernel<typename std::conditional<CS, uint32_t, uint64_t>::type, 7, 7, CS, N>
            <<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else if (w == 9 && h == 7 && p.wide_codes == !CS)
        census_kernel<typename std::conditional<CS, uint32_t, uint64_t>::type, 9, 7, CS, N>
            <<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else if (w == 5 && h == 5 && !p.wide_codes)
        census_kernel<uint32_t, 5, 5, CS, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else if (p.wide_codes)
        census_kernel<uint64_t, 0, 0, CS, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    else
        census_kernel<uint32_t, 0, 0, CS, N><<<grid, block, 0, s>>>(pt, p.W, p.H, w, h);
    return cudaGetLastError();
}

template <int N>
cudaError_t census_chunk(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    return p.census_cs ? census_launch<true, N>(p, pt, n, s) : census_launch<false, N>(p, pt, n, s);
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
