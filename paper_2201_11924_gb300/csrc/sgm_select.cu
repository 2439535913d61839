// Selection and post-processing (arxiv 2201.11924 Sec. VI-D: best disparity
// candidates, uniqueness test, quadratic sub-pixel fitting, left-right
// consistency check, disparity to depth) fused into one kernel per image row.
//
// One block per row.  Each warp takes pixels x of the row in turn, its lanes
// holding the same disparities as in the path kernel.  Per pixel it
//   - sums the paths' L_r bytes into S(x, d) (<= 8 * 255, exact in 32 bits);
//   - finds d* = argmin S with the smallest d on ties by a warp min-reduction
//     of the key (S << 9) | d;
//   - runs the uniqueness test against every d with |d - d*| > 1;
//   - offers every cell to the right view: the right pixel xr = x - d keeps
//     the minimum key over the cells that map to it (a shared-memory atomicMin),
//     which is argmin_d S(xr + d, d) with ties to the smallest d;
//   - fits the parabola through S(d*-1), S(d*), S(d*+1).
// After the whole row is in, each pixel's left-right check reads D_R(x - d*)
// and the depth f*b/d_f is written.
#include "internal.h"

namespace simsense {
namespace {

constexpr int kSelThreads = 256;
constexpr int kSelWarps = kSelThreads / 32;

template <int DPT>
__device__ __forceinline__ void load_add(const uint8_t* src, uint32_t (&acc)[DPT])
{
    if constexpr (DPT == 2) {
        uint32_t v = *reinterpret_cast<const uint16_t*>(src);
        acc[0] += v & 0xff; acc[1] += v >> 8;
    } else if constexpr (DPT == 4) {
        uint32_t v = *reinterpret_cast<const uint32_t*>(src);
#pragma unroll
        for (int j = 0; j < 4; j++) acc[j] += (v >> (8 * j)) & 0xff;
    } else if constexpr (DPT == 6) {
        const uint16_t* s16 = reinterpret_cast<const uint16_t*>(src);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint32_t v = s16[k];
            acc[2 * k] += v & 0xff; acc[2 * k + 1] += v >> 8;
        }
    } else {
        uint2 v = *reinterpret_cast<const uint2*>(src);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[j] += (v.x >> (8 * j)) & 0xff;
            acc[4 + j] += (v.y >> (8 * j)) & 0xff;
        }
    }
}

template <int DPT>
__global__ void __launch_bounds__(kSelThreads)
sgm_select_kernel(const uint8_t* __restrict__ vol, int paths, int W, int H, int D, int Dp,
                  int uniq, int lr_max_diff, int subpixel, float fb, float* __restrict__ depth,
                  SelectDebug dbg)
{
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* keyR = reinterpret_cast<uint32_t*>(smem);          // W
    float* dispf = reinterpret_cast<float*>(keyR + W);           // W
    uint16_t* sbuf = reinterpret_cast<uint16_t*>(dispf + W);     // kSelWarps x Dp
    int16_t* dstar = reinterpret_cast<int16_t*>(sbuf + kSelWarps * Dp);  // W
    uint8_t* ufail = reinterpret_cast<uint8_t*>(dstar + W);      // W

    const int y = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < W; i += kSelThreads) keyR[i] = 0xffffffffu;
    __syncthreads();

    const size_t slice = (size_t)H * W * Dp;
    const int d0 = lane * DPT;
    uint16_t* sw = sbuf + warp * Dp;
    for (int x = warp; x < W; x += kSelWarps) {
        const size_t pix = (size_t)y * W + x;
        uint32_t S[DPT];
#pragma unroll
        for (int j = 0; j < DPT; j++) S[j] = 0;
        const uint8_t* src = vol + pix * Dp + d0;
        for (int r = 0; r < paths; r++) load_add<DPT>(src + r * slice, S);

        uint32_t key[DPT];
        uint32_t kmin = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int d = d0 + j;
            key[j] = d < D ? (S[j] << 9) | (uint32_t)d : 0xffffffffu;
            kmin = min(kmin, key[j]);
        }
        kmin = __reduce_min_sync(0xffffffffu, kmin);
        const int ds = (int)(kmin & 511u);
        const uint32_t smin = kmin >> 9;

        bool bad = false;
        if (uniq > 0) {
#pragma unroll
            for (int j = 0; j < DPT; j++) {
                const int d = d0 + j;
                const int diff = d > ds ? d - ds : ds - d;
                if (d < D && diff > 1 && (uint32_t)(100 - uniq) * S[j] < 100u * smin) bad = true;
            }
        }
        bad = __any_sync(0xffffffffu, bad);

#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int d = d0 + j;
            if (d < D) {
                sw[d] = (uint16_t)S[j];
                if (d <= x) atomicMin(&keyR[x - d], key[j]);
                if (dbg.aggregated) dbg.aggregated[pix * D + d] = (uint16_t)S[j];
            }
        }
        __syncwarp();
        if (lane == 0) {
            float df = (float)ds;
            if (subpixel && ds >= 1 && ds <= D - 2) {
                const int sm = sw[ds - 1], sp = sw[ds + 1], s0 = (int)smin;
                const int num = sm - sp;
                const int den = 2 * (sm + sp - 2 * s0);
                df = (float)ds + __fdiv_rn((float)num, (float)den);
            }
            dispf[x] = df;
            dstar[x] = (int16_t)ds;
            ufail[x] = bad ? 1 : 0;
        }
        __syncwarp();
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

template <int DPT>
cudaError_t launch_t(const Params& p, const uint8_t* vol, float* depth, const SelectDebug& dbg,
                     cudaStream_t s)
{
    const size_t smem = (size_t)p.W * (4 + 4 + 2 + 1) + (size_t)kSelWarps * p.Dp * 2 + 16;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sgm_select_kernel<DPT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    sgm_select_kernel<DPT><<<p.H, kSelThreads, smem, s>>>(vol, p.paths, p.W, p.H, p.D, p.Dp, p.uniq,
                                                          p.lr_max_diff, p.subpixel, p.fb, depth, dbg);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_select(const Params& p, const uint8_t* paths, float* depth, const SelectDebug& dbg,
                          cudaStream_t s)
{
    switch (p.dpt) {
        case 2: return launch_t<2>(p, paths, depth, dbg, s);
        case 4: return launch_t<4>(p, paths, depth, dbg, s);
        case 6: return launch_t<6>(p, paths, depth, dbg, s);
        case 8: return launch_t<8>(p, paths, depth, dbg, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace simsense
