// Fused batch stage: one persistent launch for the SGM path aggregation and
// the selection (arxiv 2201.11924 Sec. VI-D: path costs aggregated around
// warps, then best disparity, uniqueness, sub-pixel fit, left-right check and
// depth) of every pair of a batch, whatever the pairs' sizes and disparity
// ranges.
//
// The work is a list of tasks in device memory, taken in list order by the
// blocks of a persistent grid through one atomic counter:
//  - a path task is 8 consecutive work items of one pair (the path kernel's
//    longest-first numbering): each warp of the block walks one item;
//  - a selection task is one image row of one pair, done by the whole block
//    with the selection kernel's TMA bulk-copy ring and row epilogue.
// A pair's rows may only be selected once all of its path tasks are done: a
// block that finishes a path task counts it on the pair's counter (release),
// and a block that takes a row waits (acquire, bounded) until the counter is
// complete.  The list puts the rows of the k-th pair after the path tasks of
// the (k + lag)-th, so while the last paths of a pair finish, blocks go on
// with the next pairs' paths, and the rows of a pair are selected soon after
// its paths were written (with the default L2 policy the selection can find
// much of a small pair's volume still in L2).  Tasks are only ever waited on
// after every task before them in the list has been taken by a running block,
// so the waits end whatever the number of resident blocks.  A wait that gives
// up records SIMSENSE_ERR_TIMEOUT and skips the row.
//
// Pair order, lag, cost prefetch depth and the store policy of the path
// volume are the schedule the batch autotuner chooses.
#include "sgm_row.cuh"
#include "sgm_walk.cuh"

namespace simsense {
namespace {

using namespace sgm;

constexpr int kFusedThreads = 256;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedStages = 4;               // stage barriers (the ring uses 2 .. 4 of them)
constexpr uint32_t kMaxDepPolls = 1u << 20;   // bound on polls of a pair's path counter (~1 s)

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int PF, bool KEEP>
__device__ __forceinline__ void path_task(const FusedPair& q, int item)
{
    switch (q.Dp) {                            // the path kernel's layouts per padded range
        case 64: walk_item<4, 4, 2, 8, PF, KEEP>(q.cost, q.vol, q.W, q.H, q.P1, q.P2, q.paths, item); break;
        case 128: walk_item<4, 8, 2, 16, PF, KEEP>(q.cost, q.vol, q.W, q.H, q.P1, q.P2, q.paths, item); break;
        case 192: walk_item<3, 16, 3, 16, PF, KEEP>(q.cost, q.vol, q.W, q.H, q.P1, q.P2, q.paths, item); break;
        default: walk_item<4, 16, 2, 32, PF, KEEP>(q.cost, q.vol, q.W, q.H, q.P1, q.P2, q.paths, item); break;
    }
}

template <int NP, int G>
__device__ __forceinline__ bool row_task(const FusedPair& q, int y, uint8_t* area, uint64_t* bars, int stages,
                                         RingPos& rp, int* abort_flag, int* status)
{
    const SelectDebug none{};
    if (q.paths == 4)
        return select_row<NP, G, 4, kFusedThreads>(area, bars, stages, rp, abort_flag, q.vol, q.depth, y, q.W, q.D,
                                                   q.uniq, q.umagic, q.lr_max_diff, q.subpixel, q.fb, none, status,
                                                   0);
    return select_row<NP, G, 8, kFusedThreads>(area, bars, stages, rp, abort_flag, q.vol, q.depth, y, q.W, q.D,
                                               q.uniq, q.umagic, q.lr_max_diff, q.subpixel, q.fb, none, status, 0);
}

// tasks[t] = (kind: 0 paths / 1 row / 2 nothing, pair, index); ctl[0] = next task,
// ctl[1 + p] = path tasks of pair p done (all zero at launch); the stage
// barriers sit at bars_off in dynamic shared memory, after the larger of the
// path rings and the selection's row area (a ring of `stages` stages).
template <int PF, bool KEEP>
__global__ void __launch_bounds__(kFusedThreads, 3)
sgm_fused_kernel(const FusedPair* __restrict__ pairs, const int4* __restrict__ tasks, int ntasks,
                 int* __restrict__ ctl, int* __restrict__ status, int bars_off, int stages)
{
    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + bars_off);
    __shared__ int task_sh, abort_flag, wait_failed;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kFusedStages; k++) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    RingPos rp;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) task_sh = atomicAdd(&ctl[0], 1);
        __syncthreads();
        const int t = task_sh;
        __syncthreads();                       // everyone has read it before thread 0 takes the next
        if (t >= ntasks) return;
        const int4 tk = tasks[t];
        const FusedPair& q = pairs[tk.y];
        if (tk.x == 2) continue;               // a placeholder (the test of the bounded waits)
        if (tk.x == 0) {
            path_task<PF, KEEP>(q, tk.z * kFusedWarps + warp);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();                   // the block's path bytes are all stored
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&ctl[1 + tk.y], 1);
            }
        } else {
            if (threadIdx.x == 0) {
                wait_failed = 1;
                for (uint32_t it = 0; it < kMaxDepPolls; it++) {
                    if (ld_acquire(&ctl[1 + tk.y]) >= q.path_tasks) {
                        wait_failed = 0;
                        break;
                    }
                    __nanosleep(256);
                }
                // the bulk copies (async proxy) read what other blocks stored
                asm volatile("fence.proxy.async.global;" ::: "memory");
                // and write the shared memory the path rings used (generic proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (wait_failed && status) atomicExch(status, SIMSENSE_ERR_TIMEOUT);
            }
            __syncthreads();
            if (wait_failed) continue;
            bool ok;
            switch (q.Dp) {
                case 64: ok = row_task<4, 8>(q, tk.z, smem, bars, stages, rp, &abort_flag, status); break;
                case 128: ok = row_task<4, 16>(q, tk.z, smem, bars, stages, rp, &abort_flag, status); break;
                case 192: ok = row_task<3, 32>(q, tk.z, smem, bars, stages, rp, &abort_flag, status); break;
                default: ok = row_task<4, 32>(q, tk.z, smem, bars, stages, rp, &abort_flag, status); break;
            }
            if (!ok) return;                   // a stage wait gave up: status recorded, ring drained
        }
    }
}

// Shared memory of the selection's row area for the padded range Dp.
size_t row_bytes(int Dp, int paths, int W, int stages)
{
    switch (Dp) {
        case 64: return paths == 4 ? RowShape<4, 8, 4, kFusedThreads>::bytes(W, stages)
                                   : RowShape<4, 8, 8, kFusedThreads>::bytes(W, stages);
        case 128: return paths == 4 ? RowShape<4, 16, 4, kFusedThreads>::bytes(W, stages)
                                    : RowShape<4, 16, 8, kFusedThreads>::bytes(W, stages);
        case 192: return paths == 4 ? RowShape<3, 32, 4, kFusedThreads>::bytes(W, stages)
                                    : RowShape<3, 32, 8, kFusedThreads>::bytes(W, stages);
        default: return paths == 4 ? RowShape<4, 32, 4, kFusedThreads>::bytes(W, stages)
                                   : RowShape<4, 32, 8, kFusedThreads>::bytes(W, stages);
    }
}

// Launches with the ring depth (2 .. 4 stages) that keeps the most blocks
// resident per SM, the deeper ring among equals.
template <int PF, bool KEEP>
cudaError_t fused_launch(const FusedPair* pairs, const int4* tasks, int ntasks, int* ctl, int* status,
                         const Params* cls, int ncls, cudaStream_t s)
{
    DevLimits lim;
    cudaError_t e = device_limits(lim);
    if (e != cudaSuccess) return e;
    auto kernel = sgm_fused_kernel<PF, KEEP>;
    const size_t path_ring = (size_t)kFusedWarps * PF * 512;
    int best_stages = 0, best_blocks = 0;
    size_t best_smem = 0, best_off = 0;
    for (int stages = kFusedStages; stages >= 2; stages--) {
        size_t area = path_ring;
        for (int c = 0; c < ncls; c++) {
            const size_t r = row_bytes(cls[c].Dp, cls[c].paths, cls[c].W, stages);
            if (r > area) area = r;
        }
        const size_t off = (area + 15) / 16 * 16;
        const size_t smem = off + 8 * kFusedStages;
        if (smem > (size_t)lim.optin) continue;
        e = ensure_smem(reinterpret_cast<const void*>(kernel), smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kFusedThreads, smem);
        if (e != cudaSuccess) return e;
        if (per_sm > best_blocks) {
            best_blocks = per_sm;
            best_stages = stages;
            best_smem = smem;
            best_off = off;
        }
    }
    if (best_blocks < 1) return cudaErrorInvalidValue;
    kernel<<<best_blocks * lim.nsm, kFusedThreads, best_smem, s>>>(pairs, tasks, ntasks, ctl, status, (int)best_off,
                                                                   best_stages);
    return cudaGetLastError();
}

}  // namespace

int fused_path_tasks(const Params& p)
{
    int spw = 0, spwh = 0;                     // scanlines per warp: other directions, rows
    switch (p.Dp) {                            // (32 / lanes per scanline of path_task's layouts)
        case 64: spw = 32 / 4; spwh = 32 / 8; break;
        case 128: spw = 32 / 8; spwh = 32 / 16; break;
        case 192: spw = 32 / 16; spwh = 32 / 16; break;
        default: spw = 32 / 16; spwh = 32 / 32; break;
    }
    const sgm::Items it = sgm::make_items(p.W, p.H, p.paths, 1, spw, spwh);
    return (it.total + kFusedWarps - 1) / kFusedWarps;
}

cudaError_t launch_fused(const FusedPair* pairs, const int4* tasks, int ntasks, int* ctl, int* status,
                         const Params* cls, int ncls, int keep, cudaStream_t s)
{
    return keep ? fused_launch<16, true>(pairs, tasks, ntasks, ctl, status, cls, ncls, s)
                : fused_launch<16, false>(pairs, tasks, ntasks, ctl, status, cls, ncls, s);
}

}  // namespace simsense
