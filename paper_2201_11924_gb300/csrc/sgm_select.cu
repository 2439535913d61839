// Selection and post-processing (arxiv 2201.11924 Sec. VI-D: best disparity
// candidates, uniqueness test, quadratic sub-pixel fitting, left-right
// consistency check, disparity to depth) fused into one kernel.
//
// Blocks are persistent over image rows.  A row's path costs are one
// contiguous run of W * paths * Dp bytes ([y][x][r][Dp]); the block streams it
// through a ring of shared-memory stages with TMA bulk copies
// (cp.async.bulk, completion counted on an mbarrier per stage), one thread
// issuing the copies a few stages ahead.  A stage holds one pixel for every
// lane group of the block (G lanes per pixel, each lane holding DPT
// consecutive disparities as in the path kernel).  Per pixel a group
//   - sums its bytes of every path with two masked 32-bit adds per word (even
//     and odd bytes as packed 16-bit pairs; 8 bytes cannot carry out of a half);
//   - finds d* = argmin S with the smallest d on ties: group min-reduction of
//     the key (S << 9) | d;
//   - runs the uniqueness test against every d with |d - d*| > 1;
//   - offers every cell to the right view: right pixel xr = x - d keeps the
//     minimum key over the cells mapping to it (shared-memory atomicMin),
//     which is argmin_d S(xr + d, d) with ties to the smallest d;
//   - fits the parabola through S(d*-1), S(d*), S(d*+1).
// When the whole row is in, each pixel's left-right check reads D_R(x - d*)
// and the depth f*b/d_f is written.  Every wait on a stage is bounded; a wait
// that gives up records SIMSENSE_ERR_TIMEOUT in the status word, drains the
// copies still in flight (again bounded) and ends the block.
#include <mutex>

#include "sgm_row.cuh"

namespace simsense {
namespace {

using namespace sgm;

// Shared-memory bytes of the block: per-row area and the stage barriers.
template <int NP, int G, int PATHS, int THREADS>
size_t select_smem(int W, int stages)
{
    return (RowShape<NP, G, PATHS, THREADS>::bytes(W, stages) + 15) / 16 * 16 + 8 * kMaxStages;
}

// Items are (pair, row); blocks are persistent over them.
template <int NP, int G, int PATHS, int THREADS, int N, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
sgm_select_kernel(PairTable<N> pt, int npairs, int W, int H, int D, int uniq, uint32_t umagic,
                  int lr_max_diff, int subpixel, float fb, SelectDebug dbg, int* __restrict__ status,
                  int kStages, int disp_mode)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        smem + (RowShape<NP, G, PATHS, THREADS>::bytes(W, kStages) + 15) / 16 * 16);
    __shared__ int abort_flag;
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        for (int k = 0; k < kStages; k++) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    __syncthreads();
    RingPos rp;
    constexpr size_t pbytes = RowShape<NP, G, PATHS, THREADS>::pbytes;
    for (int item = blockIdx.x; item < npairs * H; item += gridDim.x) {
        const int pair = item / H, y = item - pair * H;
        const int next = item + gridDim.x;
        const uint8_t* next_src = nullptr;
        if (next < npairs * H) {
            const int np = next / H, ny = next - np * H;
            next_src = pt.p[np].vol + (size_t)ny * W * pbytes;
        }
        if (!select_row<NP, G, PATHS, THREADS>(smem, bars, kStages, rp, &abort_flag, pt.p[pair].vol,
                                               pt.p[pair].depth, y, W, D, uniq, umagic, lr_max_diff, subpixel,
                                               fb, dbg, status, disp_mode, next_src))
            return;
    }
}

// MINB: blocks per SM (1024 / THREADS unless a layout needs the registers of
// a whole SM)
template <int NP, int G, int PATHS, int THREADS, int N, int MINB = 1024 / THREADS>
cudaError_t select_launch(const Params& p, const PairTable<N>& pt, int n, const SelectDebug& dbg, int* status,
                          cudaStream_t s)
{
    DevLimits lim;
    cudaError_t e = device_limits(lim);
    if (e != cudaSuccess) return e;
    // 1024 / THREADS blocks per SM with the deepest ring that lets them fit
    constexpr int blocks_per_sm = MINB;
    const size_t budget = blocks_per_sm == 1 ? (size_t)lim.optin : (size_t)lim.per_sm / blocks_per_sm - 1024;
    int stages = kMaxStages;
    while (stages > 2 && select_smem<NP, G, PATHS, THREADS>(p.W, stages) > budget) stages--;
    const size_t smem = select_smem<NP, G, PATHS, THREADS>(p.W, stages);
    if (smem > budget) return cudaErrorInvalidValue;
    auto kernel = sgm_select_kernel<NP, G, PATHS, THREADS, N, MINB>;
    e = ensure_smem(reinterpret_cast<const void*>(kernel), smem);
    if (e != cudaSuccess) return e;
    const int items = n * p.H;
    // persistent over rows: with r = ceil(items / slots) rows for the
    // busiest block, ceil(items / r) blocks take r rows each (the last one
    // fewer), where a full grid would leave some blocks one row short.  At
    // 1280 x 720 that is 144 blocks of 5 rows instead of 152 blocks of 4 or
    // 5, which took the selection from 167 to 164 us: the same longest block
    // with fewer blocks sharing the DRAM bandwidth.
    if (items <= 0) return cudaSuccess;
    int grid = items < blocks_per_sm * lim.nsm ? items : blocks_per_sm * lim.nsm;
    const int rows_per_block = (items + grid - 1) / grid;
    grid = (items + rows_per_block - 1) / rows_per_block;
    const uint32_t umagic = uniq_magic(p.uniq);
    return launch_pdl(kernel, dim3(grid), dim3(THREADS), smem, s, pt, n, p.W, p.H, p.D, p.uniq, umagic, p.lr_max_diff,
                      p.subpixel, p.fb, dbg, status, stages, p.median > 1 ? 1 : 0);
}

template <int NP, int G, int N>
cudaError_t select_chunk(const Params& p, const PairPtrs* pairs, int n, const Tuning& t,
                         const SelectDebug& dbg, int* status, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    // select_blocks 1: one block of 1024 threads per SM (rows spread over
    // fewer, faster blocks); 2: two blocks of 512 threads per SM
    if (p.paths == 4)
        return t.select_blocks == 1 ? select_launch<NP, G, 4, 1024, N>(p, pt, n, dbg, status, s)
                                    : select_launch<NP, G, 4, 512, N>(p, pt, n, dbg, status, s);
    return t.select_blocks == 1 ? select_launch<NP, G, 8, 1024, N>(p, pt, n, dbg, status, s)
                                : select_launch<NP, G, 8, 512, N>(p, pt, n, dbg, status, s);
}

// Dp = 64 and 256: G lanes a pixel with 16 disparities each, one 512-thread
// block per SM.  At 1920 x 1080, D = 256, 8 paths: 716 against 741 us for a
// whole warp a pixel with 8 disparities a lane in 1024-thread blocks; at
// 320 x 240, D = 64, 4 paths: 14.0 against 14.6 us for 8 lanes with 8
// disparities each.  (At Dp = 128 the same shape, 8 lanes with 16 each, took
// 180 against 175 us.)
template <int G, int N>
cudaError_t select_wide(const Params& p, const PairPtrs* pairs, int n, const SelectDebug& dbg, int* status,
                        cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    if (p.paths == 4) return select_launch<8, G, 4, 512, N, 1>(p, pt, n, dbg, status, s);
    return select_launch<8, G, 8, 512, N, 1>(p, pt, n, dbg, status, s);
}

template <int N>
cudaError_t select_dp(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, const SelectDebug& dbg,
                      int* status, cudaStream_t s)
{
    switch (p.Dp) {
        case 64: return select_wide<4, N>(p, pairs, n, dbg, status, s);
        case 128: return select_chunk<4, 16, N>(p, pairs, n, t, dbg, status, s);
        case 192: return select_chunk<3, 32, N>(p, pairs, n, t, dbg, status, s);
        case 256: return select_wide<16, N>(p, pairs, n, dbg, status, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t device_limits(DevLimits& out)
{
    constexpr int kMaxDev = 64;
    static DevLimits cache[kMaxDev];
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    DevLimits& c = cache[dev];
    if (c.nsm == 0) {
        e = cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c.per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e != cudaSuccess) {
            c = DevLimits{};
            return e;
        }
    }
    out = c;
    return cudaSuccess;
}

// Raises a kernel's dynamic shared-memory limit when a launch needs more than
// any earlier launch of that kernel on this device (setting it on every
// launch would put a function-attribute call between concurrent launches of
// other streams).  Entries are keyed by (device, kernel address).
cudaError_t ensure_smem(const void* kernel, size_t bytes)
{
    struct Entry {
        int dev;
        const void* fn;
        size_t bytes;
    };
    constexpr int kMaxEntries = 256;
    static Entry table[kMaxEntries];
    static int used = 0;
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    Entry* hit = nullptr;
    for (int i = 0; i < used; i++)
        if (table[i].dev == dev && table[i].fn == kernel) { hit = &table[i]; break; }
    if (hit && bytes <= hit->bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    // the kernels that stage through shared memory run with the largest
    // carve-out (for the path kernel 3% faster than the driver's choice)
    if (!hit) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    if (hit) hit->bytes = bytes;
    else if (used < kMaxEntries) table[used++] = Entry{dev, kernel, bytes};
    return cudaSuccess;
}

cudaError_t launch_select(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, const SelectDebug& dbg,
                          int* status, cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        const SelectDebug none{};
        cudaError_t e = c == 1 ? select_dp<1>(p, pairs + b, 1, t, n == 1 ? dbg : none, status, s)
                               : select_dp<kMaxBatch>(p, pairs + b, c, t, none, status, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace simsense
