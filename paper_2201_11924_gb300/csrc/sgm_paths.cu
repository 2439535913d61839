// SGM cost aggregation along scanline paths (arxiv 2201.11924 Sec. VI-D:
// semi-global matching on the Hamming cost, with the aggregation organised
// around warps).
//
// Every path direction r splits the image into independent scanlines (rows,
// columns or diagonals).  A group of G lanes walks one scanline (a warp walks
// 32 / G scanlines side by side); lane l of a group holds 4*NQ consecutive
// disparities of the padded range Dp, as NQ quads.  A quad's four cells
// d0..d3 live in two packed 16-bit pairs, E = (d0, d2) and O = (d1, d3), so
// that the neighbours d - 1 and d + 1 of one pair are mostly the other pair
// of the quad (only one byte permute per pair is needed for the rest).
//
// The recurrence L(p,d) = C(p,d) + min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m'+P2) - m'
// is evaluated with a three-input minimum (a DPX instruction on this GPU):
// the lane keeps, besides L' + P1, the clamped value min(L'(d), m' + P2), and
//   min(L'(d), m'+P2, L'(d-1)+P1, L'(d+1)+P1)
//     = min3(min(L'(d), m'+P2), L'(d-1)+P1, L'(d+1)+P1).
// Per pixel the group
//   1. takes C(p, .) from the byte cost volume and splits each word into its
//      even and odd cells.  The cost is copied PF pixels ahead into a ring
//      in shared memory with cp.async, so the DRAM latency overlaps PF steps
//      of the recurrence without holding the ring in registers;
//   2. evaluates the recurrence on the pairs (one shuffle from each
//      neighbouring lane supplies the cells beyond the lane's range);
//   3. stores L(p, .) as bytes (L <= nbits + P2 <= 255 for every real
//      disparity) into the path volume, layout [y][x][r][Dp], so that the
//      selection kernel reads one pixel's paths contiguously;
//   4. forms m = min_d L(p, d): a three-input-min tree over the lane's pairs,
//      then a reduction over the group (redux.sync for a whole warp, a
//      shuffle butterfly otherwise).
// All values stay below 2^15, so 32-bit adds of packed pairs never carry
// across the halves.  Padded disparities carry cost 255, which keeps their L
// at 255 or more: they never undercut a real candidate and never lower m.
//
// Scheduling: a warp takes one work item (a group of scanlines of one
// direction of one pair), numbered longest scanlines first: the longer of the
// horizontal and vertical directions, then the other, then the diagonals
// ranked by length.  The longest scanlines bound the kernel's duration, so
// they start first, and the short ones fill the SMs at the end.
#include "sgm_walk.cuh"

namespace simsense {
namespace {

using namespace sgm;

// Horizontal scanlines (rows) use NQH quads per lane and GH lanes per row,
// the other directions NQ and G (per disparity range, the layouts measured
// fastest on GB300: wider lanes mean fewer instructions per cell but more
// registers per thread).
//
// One warp per work item, item = blockIdx.x * warps + warp.  Items are
// numbered longest first, and blocks start in index order as earlier ones
// finish, so the long scanlines start at once and the short ones fill the
// SMs at the end.
template <int NQ, int G, int NQH, int GH, int PF, int N>
__global__ void __launch_bounds__(kPathThreads)
sgm_paths_kernel(PairTable<N> pt, int npairs, int W, int H, int P1, int P2, int paths)
{
    static_assert(G * 4 * NQ == GH * 4 * NQH, "both layouts cover the same padded range");
    constexpr int SPW = 32 / G, SPWH = 32 / GH;
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31;
    const Items it = make_items(W, H, paths, npairs, SPW, SPWH);
    int i = blockIdx.x * (kPathThreads / 32) + (threadIdx.x >> 5);
    if (i >= it.total) return;
    int cls;                                   // 0 horizontal, 1 vertical, 2 diagonal
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
    const int g = i / (ndir * npairs);         // group-major: every direction and pair advances together
    const int rem = i % (ndir * npairs);
    const int r = (cls == 0 ? 0 : cls == 1 ? 2 : 4) + rem % ndir;
    const int pair = rem / ndir;
    const uint8_t* __restrict__ C = pt.p[pair].cost;
    uint8_t* __restrict__ vol = pt.p[pair].vol;
    int rx, ry;
    path_dir(r, rx, ry);
    if (cls == 0) {
        walk<NQH, GH, PF>(C, W, H, P1, P2, paths, vol, r, rx, ry, g * SPWH + lane / GH);
    } else {
        const int j = g * SPW + lane / G;
        const int scan = cls == 1 ? j : (j < W + H - 1 ? diag_scan(j, rx, W, H) : W + H - 1);
        walk<NQ, G, PF>(C, W, H, P1, P2, paths, vol, r, rx, ry, scan);
    }
}

template <int NQ, int G, int NQH, int GH, int PF, int N>
cudaError_t paths_chunk(const Params& p, const PairPtrs* pairs, int n, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    const Items it = make_items(p.W, p.H, p.paths, n, 32 / G, 32 / GH);
    const int warps = kPathThreads / 32;
    const int blocks = (it.total + warps - 1) / warps;
    const size_t smem = (size_t)warps * PF * 512;
    auto kernel = sgm_paths_kernel<NQ, G, NQH, GH, PF, N>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kernel), smem);
    if (e != cudaSuccess) return e;
    // a plain launch: with programmatic stream serialisation after the cost
    // kernel (whether that kernel lets its dependents start at its beginning
    // or at its end) the 1280 x 720, D = 128 frame took 8% longer, cause not
    // found; the path kernel still lets the selection start early
    return launch_plain(kernel, dim3(blocks), dim3(kPathThreads), smem, s, pt, n, p.W, p.H, p.P1, p.P2, p.paths);
}

template <int NQ, int G, int NQH, int GH, int N>
cudaError_t paths_pf(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, cudaStream_t s)
{
    switch (t.prefetch) {
        case 8: return paths_chunk<NQ, G, NQH, GH, 8, N>(p, pairs, n, s);
        case 16: return paths_chunk<NQ, G, NQH, GH, 16, N>(p, pairs, n, s);
        default: return paths_chunk<NQ, G, NQH, GH, 12, N>(p, pairs, n, s);
    }
}

template <int N>
cudaError_t paths_dp(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, cudaStream_t s)
{
    switch (p.Dp) {                            // (quads per lane, lanes per scanline): other, horizontal
        case 64: return paths_pf<4, 4, 2, 8, N>(p, pairs, n, t, s);
        case 128: return paths_pf<4, 8, 2, 16, N>(p, pairs, n, t, s);
        case 192: return paths_pf<3, 16, 3, 16, N>(p, pairs, n, t, s);
        case 256: return paths_pf<4, 16, 2, 32, N>(p, pairs, n, t, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_unpack_paths(const Params& p, const uint8_t* vol, uint8_t* dbg_paths, cudaStream_t s)
{
    // plane r of every pixel ([y][x][r][Dp]) to [r][y][x][D]
    const size_t npx = (size_t)p.W * p.H;
    for (int r = 0; r < p.paths; r++) {
        cudaError_t e = cudaMemcpy2DAsync(dbg_paths + r * npx * p.D, p.D, vol + (size_t)r * p.Dp,
                                          (size_t)p.paths * p.Dp, p.D, npx, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_paths(const Params& p, const PairPtrs* pairs, int n, const Tuning& t, uint8_t* dbg_paths,
                         cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        cudaError_t e = c == 1 ? paths_dp<1>(p, pairs + b, 1, t, s) : paths_dp<kMaxBatch>(p, pairs + b, c, t, s);
        if (e != cudaSuccess) return e;
    }
    if (dbg_paths && n == 1) return launch_unpack_paths(p, pairs[0].vol, dbg_paths, s);
    return cudaSuccess;
}

}  // namespace simsense
