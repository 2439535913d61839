// Hamming matching cost volume (arxiv 2201.11924 Sec. VI-D: the matching cost
// is the Hamming distance of the census codes; the section computes it from
// shared memory for data reuse).
//
// C(x, y, d) = popcount(cL(x, y) ^ cR(x - d, y)) for x - d >= 0, else nbits,
// stored once per cell as a byte, layout [y][x][Dp] (d fastest).  Every SGM
// path reads it instead of recomputing it.  Disparities D <= d < Dp that pad
// the range get cost 255: with every real path cost at most nbits + P2 <= 255,
// a padded cell never becomes a strict minimum and never undercuts a real
// neighbour, so it behaves like the +infinity of the recurrence's boundary.
//
// On the tensor cores.  With every census bit b mapped to s = 1 - 2 b (+1 or
// -1), the Hamming distance of two n-bit codes is (n - sum_k sL_k sR_k) / 2.
// For one image row the cost volume is therefore a band of the product of the
// left codes (pixels x bits) and the transposed right codes, a contraction
// the fifth-generation tensor cores run in e4m3 (+-1.0 exactly) with an f16
// accumulator (every partial sum is an integer of magnitude <= 64, exact).
// POPC, the alternative, issues 16 results per clock per SM on this GPU, two
// per cell for codes above 32 bits; here one tcgen05.mma per 32 code bits
// covers a whole 128-pixel tile, and the kernel is bound by turning the
// accumulators into bytes and writing the volume.
//
// A tile is 128 left pixels x0 .. x0 + 127 of one row.  A persistent block
// (one per SM: it holds all 512 TMEM columns) takes a contiguous range of
// tiles with three kinds of warps working on different tiles at once:
//  - 4 producer warps load the codes of the tile two ahead (prefetched two
//    tiles ahead) and expand the left codes (A, 128 x 32 KS bytes) and the right
//    codes of pixels x0 + 127 - n, n < Dp + 128 (B, descending, so that d
//    grows with n) to e4m3 in one of two operand buffers, in the K-major
//    core-matrix layout of the tensor-core descriptors (8 rows x 16 bytes per
//    core matrix; chunks 128 B apart along K, 8-row groups 8 * 32 KS bytes
//    apart).  Left bytes past nbits are 0.0, so the padding of the code words
//    adds nothing; for odd nbits the left byte nbits is +1.0 against the
//    right +1.0 there, which makes the sum even without changing H;
//  - 1 warp issues the MMAs (N <= 256 per instruction) of a tile into one of
//    two TMEM accumulators (one when Dp + 128 > 256) and commits them;
//  - 8 epilogue warps, two groups of 4 taking alternate tiles (group g reads
//    accumulator g), turn an accumulator into cost bytes.  D(m, n) holds
//    pixel x0 + m at d = m - 127 + n, in f16 (exact: |sum| <= 64).  The
//    thread of TMEM lane m reads columns 96 - 32 (m / 32) + s, s < Dp + 32,
//    two per register, so lane l of its warp holds d = s + l - 31.  One HFMA2
//    leaves two results H in the low mantissa bytes of 1536 + H, one byte
//    permute packs four consecutive s into a word, a funnel shift by the
//    lane's offset (31 - l) mod 4 aligns it to four consecutive d in the
//    pixel's staging row (pitch Dp + 16 spreads the lanes over the banks).
//    The warp's 32 rows, 32 consecutive pixels and so a contiguous run of the
//    volume, then go out as coalesced 16-byte stores (with an L2 evict-last
//    policy: the path kernel reads the volume next), the cells d >= D (255)
//    and x - d < 0 (nbits) rewritten in the chunks that have them.
// Operand buffers, accumulators and their hand-offs are tracked by mbarriers
// whose waits are all bounded: one that gives up records
// SIMSENSE_ERR_TIMEOUT in the status word and makes every warp leave its loop
// at its next tile; the block still waits (bounded) for its MMAs and frees
// the TMEM.
#include "internal.h"

#include <cuda_fp16.h>

#include <type_traits>

namespace simsense {
namespace {

constexpr int kTileM = 128;                 // left pixels per tile (the MMA's M)
constexpr int kEpiWarps = 8;                // two groups of 4; warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kProdWarps = 4;
constexpr int kCostThreads = 32 * (kEpiWarps + kProdWarps + 1);
constexpr int kIssuerWarp = kEpiWarps + kProdWarps;
constexpr uint32_t kOne4 = 0x38383838u;     // four e4m3 +1.0
constexpr uint32_t kSign4 = 0x80808080u;    // their sign bits
constexpr uint32_t kSpread = 0x10204080u;   // nibble bit i -> bit 8 i + 7
constexpr uint32_t kMaxTries = 1u << 20;    // bound on the tries of one mbarrier wait
constexpr uint32_t kStallTries = 1u << 11;  // the same under the wait test (SIMSENSE_OPT_TEST_STALL)
constexpr uint32_t kSuspendNs = 1000;       // suspend-time hint of one try

// per 4-byte group j of an expanded left code: 0xFF for the bytes below nbits
// rounded up to even, 0 past it
struct KMask {
    uint32_t keep[16];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void sts128(uint32_t a, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3)
{
    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(w0), "r"(w1), "r"(w2), "r"(w3) : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t a)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void sts32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// shared-memory matrix descriptor: K-major, no swizzle (core matrices of
// 8 rows x 16 B), lbo = byte step between core matrices along K, sbo = along
// the rows; bits 46-47 = 1 (this architecture's descriptor version)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f8f6f4: f16 accumulator (bits 4-5 = 0),
// A and B e4m3 (bits 7-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t mma_idesc(int n) { return ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24); }

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// try_wait suspends the waiting warp (up to the hint, in ns) instead of
// spinning, so waiting warps leave the issue slots to the working ones
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint32_t tries)
{
    for (uint32_t it = 0; it < tries; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(parity), "r"(kSuspendNs) : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes, two f16
// per register (columns 2 j and 2 j + 1 in register j)
__device__ __forceinline__ void tmem_ld32h(uint32_t (&r)[16], uint32_t taddr)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.pack::16b.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
}

// cells d0 .. d0 + 15 of pixel x: 255 for d >= D, nbits for x - d < 0
__device__ __forceinline__ uint4 fix_chunk(uint4 v, int x, int d0, int D, int nbits)
{
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int d = d0 + 4 * j;                       // bytes d .. d + 3 of word j
        const int kx = x - d + 1, kd = D - d;           // bytes below each bound
        const uint32_t keep_x = kx >= 4 ? 0xFFFFFFFFu : kx <= 0 ? 0u : 0xFFFFFFFFu >> (32 - 8 * kx);
        const uint32_t keep_d = kd >= 4 ? 0xFFFFFFFFu : kd <= 0 ? 0u : 0xFFFFFFFFu >> (32 - 8 * kd);
        w[j] = (w[j] & keep_x) | ((uint32_t)nbits * 0x01010101u & ~keep_x);
        w[j] |= ~keep_d;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <int KS, int DP>
struct TcShape {
    static constexpr int RB = 32 * KS;                  // expanded bytes per code (the K extent)
    static constexpr int SBO = 8 * RB;                  // bytes per 8-row core-matrix group
    static constexpr int NCOL = DP + kTileM;            // B rows = accumulator columns
    static constexpr int NBUF = NCOL <= 256 ? 2 : 1;    // TMEM accumulators (512 columns in all)
    static constexpr int TB = 512 / NBUF;               // columns per accumulator
    static constexpr int N0 = NCOL < 256 ? NCOL : 256;  // the first MMA's N
    static constexpr int N1 = NCOL - N0;                // the second one's (0: none)
    // staging row pitch: DP + 32 bytes is 8 or 24 words modulo the 32 banks,
    // which with the lanes' byte offsets (31 - lane) / 4 spreads a warp's 32
    // word stores over all 32 banks (DP + 16 put two lanes on each bank)
    static constexpr int SROW = DP + 32;
    static constexpr int OPS = (kTileM + NCOL) * RB;    // one operand buffer (A then B)
    static constexpr int S_OFF = 2 * OPS;               // staging rows of the two epilogue groups
    static constexpr int BAR_OFF = S_OFF + 2 * kTileM * SROW;
    static constexpr int BYTES = BAR_OFF + 8 * 8 + 16;     // mbarriers, TMEM address, flag
    // one block per SM (it allocates all 512 TMEM columns): at least 120 KB of
    // the 228 KB of shared memory
    static constexpr int SMEM = BYTES > 120 * 1024 ? BYTES : 120 * 1024;
    static constexpr int RPT = (NCOL + 127) / 128;      // right rows per producer thread
    static_assert(N0 % 16 == 0 && N1 % 16 == 0 && N0 <= 256 && N1 <= 256, "MMA N");
};

struct TileMap {
    int W, H, tx;                                       // tx = tiles per row
    // tile t -> (pair, row, first pixel); step() moves to tile t + 1
    struct Pos {
        int pair, y, x0;
    };
    __device__ __forceinline__ Pos at(int t) const
    {
        const int per = H * tx, pair = t / per, r = t - pair * per, y = r / tx;
        return Pos{pair, y, (r - y * tx) * kTileM};
    }
    __device__ __forceinline__ void step(Pos& q) const
    {
        q.x0 += kTileM;
        if (q.x0 >= W) {
            q.x0 = 0;
            if (++q.y == H) {
                q.y = 0;
                q.pair++;
            }
        }
    }
};

__device__ __forceinline__ uint32_t to_word(const uint32_t (&r)[16], int w, __half2 mh, __half2 bias)
{
    uint32_t h[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        __half2 v = *reinterpret_cast<const __half2*>(&r[2 * w + u]);
        v = __hfma2(v, mh, bias);
        h[u] = *reinterpret_cast<const uint32_t*>(&v);
    }
    return __byte_perm(h[0], h[1], 0x6420);
}

// stream word B (and B + 1) -> output word a = B - boff of the pixel's row
// at base + 4 B.  B is a constant once the callers' loops unroll, which folds
// the range test to the words at the two ends of the row.
template <int DP>
__device__ __forceinline__ void put_word(int B, uint32_t lo, uint32_t hi, uint32_t sh, int boff, uint32_t base)
{
    const int a = B - boff;
    if ((B >= 7 || a >= 0) && (B < DP / 4 || a < DP / 4)) sts32(base + 4u * (uint32_t)B, __funnelshift_r(lo, hi, sh));
}

// one tile's row of this thread: TMEM chunks of 32 columns, loaded in
// batches of up to 3 with one wait each (the accumulator is released after
// the last batch), turned into words with one word carried across chunks
// for the funnel shift
template <int DP>
__device__ __forceinline__ void row_to_staging(uint32_t taddr, uint32_t srow, int lane, __half2 bias, uint32_t acc_free)
{
    constexpr int NCH = DP / 32 + 1;                    // chunks: s < Dp + 32
    constexpr int NB = 3;                               // chunks per batch
    const __half2 mh = __float2half2_rn(-0.5f);
    const int o = 31 - lane;                            // d = s - o
    const uint32_t sh = 8u * (uint32_t)(o & 3);
    const int boff = o >> 2;                            // output word a = stream word b - boff
    const uint32_t base = srow - 4u * (uint32_t)boff;
    uint32_t carry = 0;
#pragma unroll
    for (int k0 = 0; k0 < NCH; k0 += NB) {
        uint32_t r[NB][16];
#pragma unroll
        for (int k = 0; k < NB; k++)
            if (k0 + k < NCH) tmem_ld32h(r[k], taddr + 32u * (uint32_t)(k0 + k));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (k0 + NB >= NCH) {
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            bar_arrive(acc_free);                       // the accumulator may take the next tile
        }
#pragma unroll
        for (int k = 0; k < NB; k++) {
            if (k0 + k < NCH) {
                const int kk = k0 + k;
                uint32_t P[8];
#pragma unroll
                for (int w = 0; w < 8; w++) P[w] = to_word(r[k], w, mh, bias);
                if (kk > 0) put_word<DP>(8 * kk - 1, carry, P[0], sh, boff, base);
#pragma unroll
                for (int w = 0; w < 7; w++) put_word<DP>(8 * kk + w, P[w], P[w + 1], sh, boff, base);
                carry = P[7];
            }
        }
    }
}

// one code (32 KS bits) -> its expanded row, four bits per word; LEFT rows
// keep only the bytes below nbits rounded up to even
template <int KS, bool LEFT, typename CodeT>
__device__ __forceinline__ void expand_code(uint32_t row, CodeT code, const KMask& km)
{
#pragma unroll
    for (int c = 0; c < 2 * KS; c++) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int j = 4 * c + u;
            w[u] = ((((uint32_t)(code >> (4 * j)) & 0xFu) * kSpread) & kSign4) | kOne4;
            if (LEFT) w[u] &= km.keep[j];
        }
        sts128(row + 128 * c, w[0], w[1], w[2], w[3]);
    }
}

template <typename CodeT>
__device__ __forceinline__ CodeT load_code(const CodeT* row, int x, int W)
{
    return (x >= 0 && x < W) ? row[x] : (CodeT)0;
}

// blockIdx.x takes tiles [t0, t1) of ntiles = pairs x rows x ceil(W / 128).
template <int KS, int DP, int N>
__global__ void __launch_bounds__(kCostThreads, 1)
cost_kernel(PairTable<N> pt, TileMap tm, int ntiles, int D, int nbits, KMask km, int* __restrict__ status,
            int stall)
{
    using CodeT = typename std::conditional<KS == 2, uint64_t, uint32_t>::type;
    using S = TcShape<KS, DP>;
    extern __shared__ __align__(128) uint8_t cost_smem[];
    pdl_wait();
    pdl_trigger();
    const uint32_t sbase = smem_u32(cost_smem);
    const uint32_t sS = sbase + S::S_OFF;
    const uint32_t bars = sbase + S::BAR_OFF;
    // mbarriers: ops_full[2], ops_free[2], acc_full[2], acc_free[2]
    const uint32_t ops_full = bars, ops_free = bars + 16, acc_full = bars + 32, acc_free = bars + 48;
    const uint32_t tslot = bars + 64;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(cost_smem + S::BAR_OFF + 68);
    // the block's tiles [t0, t1), walked in order by every role
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t tries = stall ? kStallTries : kMaxTries;
    const int t0 = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
    const int t1 = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x);

    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ops_full + 8 * b), "r"(32 * kProdWarps) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ops_free + 8 * b) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(acc_full + 8 * b) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(acc_free + 8 * b), "r"(16 * kEpiWarps) : "memory");
        }
        abort_flag[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(tslot) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t tmem;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(tslot) : "memory");

    if (warp >= kEpiWarps && warp < kIssuerWarp) {
        // ---- producers: thread p expands left pixel x0 + p and right rows p + 128 j
        const int p = tid - 32 * kEpiWarps;
        CodeT cl = 0, cr[S::RPT], nl = 0, nr[S::RPT], ml = 0, mr[S::RPT];
        TileMap::Pos q = tm.at(t0 < t1 ? t0 : 0);
        auto fetch = [&](const TileMap::Pos& at, CodeT& l, CodeT (&r)[S::RPT]) {
            const CodeT* rowL = static_cast<const CodeT*>(pt.p[at.pair].codes_left) + (size_t)at.y * tm.W;
            const CodeT* rowR = static_cast<const CodeT*>(pt.p[at.pair].codes_right) + (size_t)at.y * tm.W;
            l = load_code(rowL, at.x0 + p, tm.W);
#pragma unroll
            for (int j = 0; j < S::RPT; j++) {
                const int n = p + 128 * j;
                r[j] = n < S::NCOL ? load_code(rowR, at.x0 + kTileM - 1 - n, tm.W) : (CodeT)0;
            }
        };
        if (t0 < t1) fetch(q, cl, cr);
        if (t0 + 1 < t1) {
            tm.step(q);
            fetch(q, nl, nr);
        }
        for (int t = t0, i = 0; t < t1; t++, i++) {
            const int b = i & 1;
            // the codes two tiles ahead, in flight meanwhile (one tile ahead
            // left the producers waiting on the loads: 52 against 45 us for
            // the 1280 x 720, D = 128 volume)
            if (t + 2 < t1) {
                tm.step(q);
                fetch(q, ml, mr);
            }
            if (i >= 2 && !bar_wait(ops_free + 8 * b, ((i - 2) >> 1) & 1, tries)) {
                if (status) atomicExch(status, SIMSENSE_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            if (*abort_flag) break;
            const uint32_t sA = sbase + b * S::OPS, sB = sA + kTileM * S::RB;
            expand_code<KS, true>(sA + (p >> 3) * S::SBO + (p & 7) * 16, cl, km);
#pragma unroll
            for (int j = 0; j < S::RPT; j++) {
                const int n = p + 128 * j;
                if (S::NCOL % 128 == 0 || n < S::NCOL) expand_code<KS, false>(sB + (n >> 3) * S::SBO + (n & 7) * 16, cr[j], km);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_arrive(ops_full + 8 * b);
            cl = nl;
            nl = ml;
#pragma unroll
            for (int j = 0; j < S::RPT; j++) {
                cr[j] = nr[j];
                nr[j] = mr[j];
            }
        }
    } else if (warp == kIssuerWarp) {
        // ---- the MMA issuer (one thread)
        if (lane == 0) {
            int last = -1;
            for (int t = t0, i = 0; t < t1; t++, i++) {
                const int b = i & 1, ab = i % S::NBUF;
                bool ok = bar_wait(ops_full + 8 * b, (i >> 1) & 1, tries);
                // the accumulator's previous tile has been read (the mbarriers
                // go by tile parity, the epilogue group, whatever NBUF is, so
                // that no wait is ever a phase ahead of its barrier)
                if (ok && i >= S::NBUF) ok = bar_wait(acc_free + 8 * ((i - S::NBUF) & 1), ((i - S::NBUF) >> 1) & 1, tries);
                if (!ok) {
                    if (status) atomicExch(status, SIMSENSE_ERR_TIMEOUT);
                    *abort_flag = 1;
                }
                if (*abort_flag) break;
                if (stall) continue;                    // the wait test: nothing completes
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sA = sbase + b * S::OPS, sB = sA + kTileM * S::RB;
                const uint32_t d = tmem + (uint32_t)(ab * S::TB);
#pragma unroll
                for (int ks = 0; ks < KS; ks++) {
                    const uint64_t a = smem_desc(sA + 256 * ks, 128, S::SBO);
                    mma_f8(d, a, smem_desc(sB + 256 * ks, 128, S::SBO), mma_idesc(S::N0), ks);
                    if (S::N1 > 0)
                        mma_f8(d + S::N0, a, smem_desc(sB + (S::N0 / 8) * S::SBO + 256 * ks, 128, S::SBO),
                               mma_idesc(S::N1 > 0 ? S::N1 : 16), ks);
                }
                mma_commit(ops_free + 8 * b);           // the operand buffer may be refilled
                mma_commit(acc_full + 8 * b);           // the accumulator is ready for group b
                last = i;
            }
            if (last >= 0) bar_wait(acc_full + 8 * (last & 1), (last >> 1) & 1, kMaxTries);   // no MMA in flight
        }
        __syncwarp();
    } else {
        // ---- epilogue warps: group g = warp / 4 takes the tiles i = g, g + 2, ..
        const int g = warp >> 2, wq = warp & 3;
        const int m = 32 * wq + lane;                    // this thread's TMEM lane = pixel x0 + m
        const __half2 bias = __float2half2_rn(1536.0f + (float)((nbits + 1) >> 1));
        const uint32_t srow = sS + (uint32_t)((g * kTileM + m) * S::SROW);
        TileMap::Pos q = tm.at(t0 < t1 ? t0 : 0);
        constexpr int CPP = DP / 16;                     // 16-byte chunks per pixel
        for (int t = t0, i = 0; t < t1; t++, i++, tm.step(q)) {
            if ((i & 1) != g) continue;
            const int ab = S::NBUF == 2 ? g : 0;
            if (!bar_wait(acc_full + 8 * g, (uint32_t)(i >> 1) & 1u, tries)) {
                if (status) atomicExch(status, SIMSENSE_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            if (*abort_flag) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t taddr = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(ab * S::TB + 96 - 32 * wq);
            row_to_staging<DP>(taddr, srow, lane, bias, acc_free + 8 * g);
            __syncwarp();
            // the warp's 32 rows are 32 consecutive pixels: a contiguous run of
            // 32 Dp bytes, copied with 512 contiguous bytes per instruction
            const int xw = q.x0 + 32 * wq;
            const int nrow = tm.W - xw < 32 ? tm.W - xw : 32;
            uint8_t* dst = pt.p[q.pair].cost + ((size_t)q.y * tm.W + xw) * DP;
            const uint32_t wrow = srow - (uint32_t)(lane * S::SROW);
            // the volume is read next by every path: kept in L2 ahead of
            // other lines where it fits (measured 4 us less path time at
            // 1280 x 720, D = 128, whose 118 MB volume fits the 129 MB L2)
            uint64_t keep;
            asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
#pragma unroll 4
            for (int k = lane; k < 32 * CPP; k += 32) {
                const int rr = k / CPP, cc = k - rr * CPP;
                if (rr < nrow) {
                    uint4 v = lds128(wrow + rr * S::SROW + 16 * cc);
                    // cells d >= D (255) and x - d < 0 (nbits) of this chunk
                    if (16 * cc + 16 > D || 16 * cc + 15 > xw + rr) v = fix_chunk(v, xw + rr, 16 * cc, D, nbits);
                    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;"
                                 ::"l"(dst + (size_t)k * 16), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "l"(keep)
                                 : "memory");
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 1;
    }
    return n;
}

template <int KS, int DP, int N>
cudaError_t cost_launch(const Params& p, const PairTable<N>& pt, int n, int* status, cudaStream_t s)
{
    using S = TcShape<KS, DP>;
    KMask km{};
    const int nb2 = p.nbits + (p.nbits & 1);
    for (int j = 0; j < 16; j++) {
        const int lb = nb2 - 4 * j;                          // kept bytes of group j
        km.keep[j] = lb >= 4 ? 0xFFFFFFFFu : lb <= 0 ? 0u : (1u << (8 * lb)) - 1u;
    }
    const auto kernel = cost_kernel<KS, DP, N>;
    cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kernel), S::SMEM);
    if (e != cudaSuccess) return e;
    TileMap tm{p.W, p.H, (p.W + kTileM - 1) / kTileM};
    const int ntiles = n * p.H * tm.tx;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    e = launch_pdl(kernel, dim3(grid), dim3(kCostThreads), S::SMEM, s, pt, tm, ntiles, p.D, p.nbits, km, status,
                   p.test_stall);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
template <int KS, int N>
cudaError_t cost_dp(const Params& p, const PairTable<N>& pt, int n, int* status, cudaStream_t s)
{
    switch (p.Dp) {
        case 64: return cost_launch<KS, 64, N>(p, pt, n, status, s);
        case 128: return cost_launch<KS, 128, N>(p, pt, n, status, s);
        case 192: return cost_launch<KS, 192, N>(p, pt, n, status, s);
        case 256: return cost_launch<KS, 256, N>(p, pt, n, status, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int N>
cudaError_t cost_code(const Params& p, const PairPtrs* pairs, int n, int* status, cudaStream_t s)
{
    PairTable<N> pt{};
    for (int i = 0; i < n; i++) pt.p[i] = pairs[i];
    if (p.nbits < 1 || p.nbits > 64) return cudaErrorInvalidValue;
    return p.wide_codes ? cost_dp<2, N>(p, pt, n, status, s) : cost_dp<1, N>(p, pt, n, status, s);
}

// SGBM block cost (the variant Sec. VI-D describes, which matches
// neighbourhoods rather than single pixels): the per-pixel cost volume
// `raw` averaged over the bw x bh block around each pixel (same d), over the
// block's pixels inside the image, rounded half up, into `out`.
// A block takes 32 pixels of one output row in two separable passes:
//   1. for every staged column (32 + bw - 1 pixels) and 4-byte word of the
//      disparity range, the sum over the bh input rows, kept in shared memory
//      as two 16-bit pairs (bytes 0 and 2, bytes 1 and 3; at most 49 x 255 <
//      2^16), so every input word is split into pairs once;
//   2. for every output pixel and word, the sum of the bw staged columns and
//      the division by the in-image pixel count n, a multiply-high by
//      floor(2^32 / n) + 1, exact for every numerator below 2^16 and 2 <= n <= 81.
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
    // n = 1 (whose multiplier needs 33 bits) never reaches the kernel: such a
    // block is the per-pixel cost, which runs without it (block_active)
    Magic mg{};
    for (uint32_t k = 2; k < 82; k++) mg.m[k] = (uint32_t)(0x100000000ull / k) + 1u;
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

cudaError_t launch_cost(const Params& p, const PairPtrs* pairs, int n, int* status, cudaStream_t s)
{
    for (int b = 0; b < n; b += kMaxBatch) {
        const int c = n - b < kMaxBatch ? n - b : kMaxBatch;
        cudaError_t e = c == 1 ? cost_code<1>(p, pairs + b, 1, status, s)
                               : cost_code<kMaxBatch>(p, pairs + b, c, status, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace simsense
