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
    pdl_wait();
    pdl_trigger();
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

// The unrolled windows (5x5, 7x7, 9x7) four pixels per thread, four
// comparisons per instruction sequence: byte j of a 32-bit word belongs to
// pixel x + j, so one word holds one window offset's neighbours of the four
// pixels.  For unsigned bytes a < b per byte: with d = (a | 0x80..) -
// (b & 0x7f..) no borrow crosses a byte, bit 7 of d is [low7(a) >= low7(b)],
// and a < b = (~a7 & b7) | (~(a7 ^ b7) & ~d7) -- one three-input logic op on
// the top bits.  Offsets go in reverse raster order into byte-wise shift
// registers (A = A >> 1 | lt & 0x80..: after eight offsets byte j of A holds
// eight bits of pixel j), which leaves bit b of the code on offset
// nbits - 1 - b, the MSB-first raster order of the one-pixel kernel above.
constexpr int kSwTX = 32;                   // threads per block row, 4 pixels each
constexpr int kSwTY = 8;                    // block rows
constexpr int kSwPix = 4 * kSwTX;           // pixels per block row
constexpr int kSwPad = 4;                   // tile bytes left of the block's first pixel (>= rx, word aligned)
constexpr int kSwRow = kSwPix + 2 * kSwPad; // tile bytes per row (34 words)

__device__ __forceinline__ uint32_t lt4(uint32_t a, uint32_t b, uint32_t d)
{
    return (~a & b) | (~(a ^ b) & ~d);      // valid in bits 7, 15, 23, 31
}

// tile words w and w + 1 from byte offset sh (0..3) on: bytes 4w + sh .. 4w + sh + 3
template <int SH>
__device__ __forceinline__ uint32_t word_at(const uint32_t* row, int w)
{
    if constexpr (SH == 0) return row[w];
    else return __funnelshift_r(row[w], row[w + 1], 8 * SH);
}

template <typename CodeT, int WW, int WH, bool CS, int N>
__global__ void __launch_bounds__(kSwTX * kSwTY)
census_swar_kernel(PairTable<N> pt, int W, int H)
{
    constexpr int rx = WW / 2, ry = WH / 2;
    constexpr int TH = kSwTY + 2 * ry;
    constexpr int RW = kSwRow / 4;                       // words per tile row
    constexpr int NB = CS ? (WW * WH - 1) / 2 : WW * WH - 1;
    constexpr int NG = (NB + 7) / 8;                     // byte groups of the code
    static_assert(rx <= kSwPad && NG <= 8 && NB <= 8 * (int)sizeof(CodeT), "window");
    __shared__ __align__(16) uint32_t tile[TH * RW];
    __shared__ __align__(16) uint32_t tile0[CS ? TH * RW : 1];
    pdl_wait();
    pdl_trigger();
    const int pair = blockIdx.z >> 1;
    const uint8_t* img = (blockIdx.z & 1) ? pt.p[pair].right : pt.p[pair].left;
    CodeT* out = static_cast<CodeT*>((blockIdx.z & 1) ? pt.p[pair].codes_right : pt.p[pair].codes_left);
    const int gx0 = blockIdx.x * kSwPix - kSwPad, gy0 = blockIdx.y * kSwTY - ry;
    // staged a word at a time when the rows are word aligned (W a multiple of
    // 4 and the image 4-byte aligned), byte by byte otherwise; outside the
    // image 255 (and 0 in the second tile)
    const bool words = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 3) == 0;
    for (int i = threadIdx.y * kSwTX + threadIdx.x; i < TH * RW; i += kSwTX * kSwTY) {
        const int w = i % RW, ty = i / RW;
        const int gx = gx0 + 4 * w, gy = gy0 + ty;
        uint32_t v = 0xffffffffu, v0 = 0u;
        if (gy >= 0 && gy < H) {
            const uint8_t* row = img + (size_t)gy * W;
            if (words && gx >= 0 && gx + 3 < W) {
                v = v0 = *reinterpret_cast<const uint32_t*>(row + gx);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (gx + j >= 0 && gx + j < W) {
                        const uint32_t b = row[gx + j];
                        v = (v & ~(0xffu << (8 * j))) | (b << (8 * j));
                        v0 |= b << (8 * j);
                    }
                }
            }
        }
        tile[i] = v;
        if constexpr (CS) tile0[i] = v0;
    }
    __syncthreads();
    const int x = blockIdx.x * kSwPix + 4 * threadIdx.x, y = blockIdx.y * kSwTY + threadIdx.y;
    if (x >= W || y >= H) return;
    const uint32_t* trow = tile + threadIdx.y * RW + threadIdx.x;   // + dy * RW: window row dy
    const uint32_t* t0row = CS ? tile0 + threadIdx.y * RW + threadIdx.x : trow;
    constexpr uint32_t H7 = 0x80808080u;
    const uint32_t c4 = trow[ry * RW + 1];               // the four centres
    const uint32_t cm = c4 & ~H7;
    uint32_t A[NG];
#pragma unroll
    for (int g = 0; g < NG; g++) A[g] = 0;
    int f = 0;                                           // offsets fed so far (a constant once unrolled)
#pragma unroll
    for (int k = WW * WH - 1; k >= 0; k--) {             // reverse raster order
        const int dy = k / WW, dx = k % WW;
        if (dy == ry && dx == rx) continue;
        if (CS && (dy > ry || (dy == ry && dx > rx))) continue;
        // pixel x + j + dx - rx sits at tile byte 4 tx + kSwPad + j + dx - rx
        const int b0 = kSwPad - rx + dx;
        uint32_t a;
        switch (b0 & 3) {
            case 0: a = word_at<0>(trow + dy * RW, b0 >> 2); break;
            case 1: a = word_at<1>(trow + dy * RW, b0 >> 2); break;
            case 2: a = word_at<2>(trow + dy * RW, b0 >> 2); break;
            default: a = word_at<3>(trow + dy * RW, b0 >> 2); break;
        }
        uint32_t lt;
        if constexpr (CS) {
            // the pair's second pixel p - o, read from the tile staged with 0
            const int b1 = kSwPad - rx + (WW - 1 - dx);
            const uint32_t* r0 = t0row + (WH - 1 - dy) * RW;
            uint32_t b;
            switch (b1 & 3) {
                case 0: b = word_at<0>(r0, b1 >> 2); break;
                case 1: b = word_at<1>(r0, b1 >> 2); break;
                case 2: b = word_at<2>(r0, b1 >> 2); break;
                default: b = word_at<3>(r0, b1 >> 2); break;
            }
            lt = lt4(a, b, (a | H7) - (b & ~H7));
        } else {
            lt = lt4(a, c4, (a | H7) - cm);
        }
        A[f >> 3] = (A[f >> 3] >> 1) | (lt & H7);
        f++;
    }
    if constexpr (NB % 8 != 0) A[NG - 1] >>= 8 - NB % 8;
    // byte j of A[g] is byte g of pixel j's code: a 4 x 4 byte transpose per
    // four groups
    uint32_t lo[4], hi[4] = {0u, 0u, 0u, 0u};
    {
        const uint32_t a0 = A[0], a1 = NG > 1 ? A[1] : 0u, a2 = NG > 2 ? A[2] : 0u, a3 = NG > 3 ? A[3] : 0u;
        const uint32_t s0 = __byte_perm(a0, a1, 0x5140), s1 = __byte_perm(a0, a1, 0x7362);
        const uint32_t s2 = __byte_perm(a2, a3, 0x5140), s3 = __byte_perm(a2, a3, 0x7362);
        lo[0] = __byte_perm(s0, s2, 0x5410);
        lo[1] = __byte_perm(s0, s2, 0x7632);
        lo[2] = __byte_perm(s1, s3, 0x5410);
        lo[3] = __byte_perm(s1, s3, 0x7632);
    }
    if constexpr (NG > 4) {
        const uint32_t a0 = A[4], a1 = NG > 5 ? A[5] : 0u, a2 = NG > 6 ? A[6] : 0u, a3 = NG > 7 ? A[7] : 0u;
        const uint32_t s0 = __byte_perm(a0, a1, 0x5140), s1 = __byte_perm(a0, a1, 0x7362);
        const uint32_t s2 = __byte_perm(a2, a3, 0x5140), s3 = __byte_perm(a2, a3, 0x7362);
        hi[0] = __byte_perm(s0, s2, 0x5410);
        hi[1] = __byte_perm(s0, s2, 0x7632);
        hi[2] = __byte_perm(s1, s3, 0x5410);
        hi[3] = __byte_perm(s1, s3, 0x7632);
    }
    CodeT* o = out + (size_t)y * W + x;
    if ((W & 3) == 0 && x + 3 < W) {                     // 16-byte aligned
        if constexpr (sizeof(CodeT) == 8) {
            reinterpret_cast<uint4*>(o)[0] = make_uint4(lo[0], hi[0], lo[1], hi[1]);
            reinterpret_cast<uint4*>(o)[1] = make_uint4(lo[2], hi[2], lo[3], hi[3]);
        } else {
            *reinterpret_cast<uint4*>(o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (x + j < W) {
                if constexpr (sizeof(CodeT) == 8) o[j] = ((uint64_t)hi[j] << 32) | lo[j];
                else o[j] = (CodeT)lo[j];
            }
        }
    }
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
    // full census, 24 / 31 bits (32-bit codes) for the centre-symmetric one;
    // 5x5: 24 / 12 bits
    dim3 sblock(kSwTX, kSwTY);
    dim3 sgrid((p.W + kSwPix - 1) / kSwPix, (p.H + kSwTY - 1) / kSwTY, 2 * n);
    using WideT = typename std::conditional<CS, uint32_t, uint64_t>::type;
    if (w == 7 && h == 7 && p.wide_codes == !CS)
        return launch_pdl(census_swar_kernel<WideT, 7, 7, CS, N>, sgrid, sblock, 0, s, pt, p.W, p.H);
    if (w == 9 && h == 7 && p.wide_codes == !CS)
        return launch_pdl(census_swar_kernel<WideT, 9, 7, CS, N>, sgrid, sblock, 0, s, pt, p.W, p.H);
    if (w == 5 && h == 5 && !p.wide_codes)
        return launch_pdl(census_swar_kernel<uint32_t, 5, 5, CS, N>, sgrid, sblock, 0, s, pt, p.W, p.H);
    if (p.wide_codes)
        return launch_pdl(census_kernel<uint64_t, 0, 0, CS, N>, grid, block, 0, s, pt, p.W, p.H, w, h);
    return launch_pdl(census_kernel<uint32_t, 0, 0, CS, N>, grid, block, 0, s, pt, p.W, p.H, w, h);
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
