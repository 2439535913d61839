// Device code of the selection and post-processing shared by the selection
// kernel and the fused batch kernel: the TMA bulk-copy stage ring, one
// pixel's sum / winner / uniqueness / right-view offers, and one whole row with
// its epilogue (the algorithm is described at the top of sgm_select.cu).
#pragma once

#include "internal.h"

namespace simsense {
namespace sgm {

constexpr int kMaxStages = 4;                // ring depth when shared memory allows
constexpr uint32_t kMaxPolls = 1u << 22;     // bound on polls of one stage barrier

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count) : "memory");
}

// One thread: expect `bytes` on the stage barrier and start the bulk copy.
__device__ __forceinline__ void stage_load(uint64_t* bar, void* dst, const void* src, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < kMaxPolls; it++) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// The lane's bytes of one path of one pixel in a stage, as words.
template <int NP>
__device__ __forceinline__ void lds_words(uint32_t (&w)[(NP + 1) / 2], const uint8_t* p)
{
    if constexpr (NP == 8) {
        const uint4 v = *reinterpret_cast<const uint4*>(p);
        w[0] = v.x;
        w[1] = v.y;
        w[2] = v.z;
        w[3] = v.w;
    } else if constexpr (NP == 4) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x;
        w[1] = v.y;
    } else {   // NP == 3: 6 bytes, 2-byte aligned
        const uint16_t* q = reinterpret_cast<const uint16_t*>(p);
        w[0] = (uint32_t)q[0] | ((uint32_t)q[1] << 16);
        w[1] = q[2];
    }
}

// keyR is padded with one word per 32: lanes whose cells map to right pixels
// 32 apart (lanes 4 apart in a 16-lane group hold disparities 32 apart) then
// hit different shared-memory banks.
__device__ __forceinline__ int kr(int xr) { return xr + (xr >> 5); }

// Minimum of a 32-bit value over the G lanes of a group: for 8 to 32 lanes
// one whole-warp redux.sync per group, the other groups' lanes offering
// 0xffffffff (fewer instructions than a shuffle butterfly), for smaller
// groups the butterfly.  Called by the whole warp.
template <int G>
__device__ __forceinline__ uint32_t group_min32(uint32_t v)
{
    if constexpr (G >= 8) {
        constexpr int NG = 32 / G;
        const int grp = (threadIdx.x & 31) / G;
        uint32_t res = 0;
#pragma unroll
        for (int g = 0; g < NG; g++) {
            const uint32_t r = __reduce_min_sync(0xffffffffu, grp == g ? v : 0xffffffffu);
            res = grp == g ? r : res;
        }
        return res;
    } else {
#pragma unroll
        for (int o = 1; o < G; o <<= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
}

// One pixel of the row for one lane group: sum, winner, uniqueness, offers to
// the right view, parabola.  src is the pixel's first path in the stage.
// DFULL: D equals the padded range, so every cell is a real disparity;
// otherwise `pad` marks the lane's padded cells (0xffff halves of the
// even / odd cell words).
template <int NP, int G, int PATHS, bool DFULL>
__device__ __forceinline__ void select_pixel(const uint8_t* src, int x, bool act, int y, int W, int D,
                                             int uniq, uint32_t umagic, int subpixel, int gl,
                                             uint16_t* sw, uint32_t* keyR, uint32_t* info, uint32_t* fit,
                                             const SelectDebug& dbg, const uint32_t (&pad)[2 * ((NP + 1) / 2)])
{
    constexpr int DPT = 2 * NP;
    constexpr int Dp = G * DPT;
    constexpr int NW = (NP + 1) / 2;
    // With two groups per warp, the second one takes its disparity chunks
    // rotated by half a group, so that the two groups' shared-memory reads of
    // their two pixels fall on disjoint banks.
    const int chunk = G == 16 ? (gl + 8 * ((threadIdx.x & 31) / 16)) % 16 : gl;
    const int d0 = chunk * DPT;
    const size_t pix = (size_t)y * W + x;
    // path sums: ev[k] holds cells (4k, 4k+2), od[k] cells (4k+1, 4k+3) as
    // 16-bit halves.  od sums the odd bytes (b1, b3) of every path word, one
    // permute each; a sum of at most 8 bytes (2040) never carries into the
    // upper half.  ev sums the whole words modulo 2^32 (carries between bytes
    // included) and then takes 256 * od off: sum(b0 + 2^8 b1 + 2^16 b2 +
    // 2^24 b3) - 2^8 sum(b1 + 2^16 b3) = sum(b0) + 2^16 sum(b2) < 2^32, so the
    // modular result is exact.  No byte mask: the adds and the one multiply-add
    // issue beside the permutes and minima instead of on their pipe.
    uint32_t ev[NW], od[NW];
#pragma unroll
    for (int r = 0; r < PATHS; r++) {
        uint32_t a[NW];
        lds_words<NP>(a, src + r * Dp + d0);
#pragma unroll
        for (int k = 0; k < NW; k++) {
            const uint32_t o = __byte_perm(a[k], 0, 0x4341);
            ev[k] = r == 0 ? a[k] : ev[k] + a[k];
            od[k] = r == 0 ? o : od[k] + o;
        }
    }
#pragma unroll
    for (int k = 0; k < NW; k++) ev[k] -= od[k] * 256u;
    // padded cells d >= D (their path bytes carry no meaning) read as
    // S = 0xffff: their keys lose to every real cell's (S <= 2040), in the
    // winner, in the right-view minimum (d = 0 is real for every right
    // pixel) and, with T capped at 0xffff below, in the uniqueness test
    if (!DFULL) {
#pragma unroll
        for (int k = 0; k < NW; k++) {
            ev[k] |= pad[2 * k];
            od[k] |= pad[2 * k + 1];
        }
    }
    // cell j of the lane (d = d0 + j): word j/4, parity j%2, half (j/2)%2
    uint32_t S[DPT];
#pragma unroll
    for (int j = 0; j < DPT; j++) {
        const uint32_t w = (j & 1) ? od[j >> 2] : ev[j >> 2];
        S[j] = (j & 2) ? (w >> 16) : (w & 0xffffu);
    }
    // winner: minimum key (S << 9) | d over the group, so ties go to the smallest d
    uint32_t key[DPT];
    uint32_t kmin = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < DPT; j++) key[j] = (S[j] << 9) + (uint32_t)(d0 + j);
    if constexpr (DPT == 8) {
        kmin = __vimin3_u32(__vimin3_u32(key[0], key[1], key[2]), __vimin3_u32(key[3], key[4], key[5]),
                            min(key[6], key[7]));
    } else {
        kmin = key[0];
#pragma unroll
        for (int j = 1; j + 1 < DPT; j += 2) kmin = __vimin3_u32(kmin, key[j], key[j + 1]);
        if constexpr (DPT % 2 == 0) kmin = min(kmin, key[DPT - 1]);
    }
    kmin = group_min32<G>(kmin);
    const int ds = (int)(kmin & 511u);
    const uint32_t smin = kmin >> 9;

    // uniqueness: (100 - u) S(d) < 100 S(d*)  <=>  S(d) < T = ceil(100 S(d*) / (100 - u)),
    // the division done as a multiply-high by umagic = floor(2^32 / (100 - u)) + 1,
    // exact for numerators below 2^18; 100 - u = 1 (no magic in 32 bits) divides by one.
    // The lane compares the minimum over its real cells at least 2 away from d*.
    bool bad = false;
    if (uniq > 0) {
        const uint32_t num = 100u * smin + (uint32_t)(99 - uniq);
        // capped at 0xffff: every real S is below it, a padded cell equals it
        const uint32_t T = min(uniq == 99 ? num : __umulhi(num, umagic), 0xffffu);
        uint32_t m = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < DPT; j++) {
            const int d = d0 + j;
            if ((uint32_t)(d - ds + 1) > 2u) m = min(m, S[j]);
        }
        bad = m < T;
    }
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G));
    bad = (__ballot_sync(0xffffffffu, bad) & gmask) != 0;

    if (act) {
        if constexpr (DPT % 8 == 0) {
#pragma unroll
            for (int k = 0; k < DPT / 4; k += 2)
                *reinterpret_cast<uint4*>(sw + d0 + 4 * k) =
                    make_uint4(__byte_perm(ev[k], od[k], 0x5410), __byte_perm(ev[k], od[k], 0x7632),
                               __byte_perm(ev[k + 1], od[k + 1], 0x5410), __byte_perm(ev[k + 1], od[k + 1], 0x7632));
        } else {
#pragma unroll
            for (int j = 0; j < DPT; j++) sw[d0 + j] = (uint16_t)S[j];
        }
        // offers to the right view: right pixel x - d keeps the minimum key
        if (x >= Dp - 1) {                     // every cell maps inside the image
            // kr(xr0 - j) = kr(xr0) - j - [j > xr0 mod 32] for j < 32: two
            // base addresses and a compile-time offset per cell
            const int xr0 = x - d0;
            const int c = xr0 & 31;
            uint32_t* const lo = keyR + kr(xr0);
            uint32_t* const hi = lo - 1;
#pragma unroll
            for (int j = 0; j < DPT; j++)
                atomicMin((j > c ? hi : lo) - j, key[j]);
        } else {
#pragma unroll
            for (int j = 0; j < DPT; j++) {
                const int d = d0 + j;
                if (d <= x) atomicMin(&keyR[kr(x - d)], key[j]);
            }
        }
        if (dbg.aggregated) {
#pragma unroll
            for (int j = 0; j < DPT; j++)
                if (d0 + j < D) dbg.aggregated[pix * D + d0 + j] = (uint16_t)S[j];
        }
    }
    __syncwarp();
    // the winner and the parabola's samples for the row's epilogue:
    // info = S(d*) << 16 | failed uniqueness << 15 | parabola fitted << 14 | d*,
    // fit = S(d*-1) | S(d*+1) << 16
    if (gl == 0 && act) {
        const bool para = subpixel && ds >= 1 && ds <= D - 2;
        info[x] = (smin << 16) | (bad ? 0x8000u : 0u) | (para ? 0x4000u : 0u) | (uint32_t)ds;
        if (para) fit[x] = (uint32_t)sw[ds - 1] | ((uint32_t)sw[ds + 1] << 16);
    }
    __syncwarp();
}


// Per-row shared memory of a block's selection: the stage ring (stages x
// kPix pixels x PATHS x Dp bytes), the pixels' S rows for the parabola, the
// right-view keys and the row's per-pixel results.  The stage barriers are
// kept elsewhere: they persist from row to row.
template <int NP, int G, int PATHS, int THREADS>
struct RowShape {
    static constexpr int DPT = 2 * NP;
    static constexpr int Dp = G * DPT;
    static constexpr int SPW = 32 / G;                  // pixels a warp takes per stage
    static constexpr int kPix = THREADS / 32 * SPW;     // pixels per stage
    static constexpr size_t pbytes = (size_t)PATHS * Dp;   // one pixel's path costs
    static constexpr size_t stage_bytes = kPix * pbytes;   // a multiple of 256
    static __host__ __device__ size_t bytes(int W, int stages)
    {
        return (size_t)stages * stage_bytes + (size_t)kPix * Dp * 2 + (size_t)(W + W / 32 + 2 * W) * 4 + 16;
    }
};

// Position of a block in its stage ring: stage number seq of the block lives
// in slot seq % stages with barrier phase (seq / stages) & 1, both advanced
// incrementally from row to row.  ahead: stages of the block's next row whose
// copies the previous row already started (thread 0's count).
struct RingPos {
    int slot = 0;
    uint32_t phase = 0;
    int ahead = 0;
};

// One image row y of one pair, by the whole block: every pixel's sum, winner,
// uniqueness and offers to the right view stage by stage, then the row
// epilogue (left-right check, parabola, depth).  area: RowShape::bytes of
// shared memory; bars: `stages` initialised stage barriers; abort_flag: a
// shared word, 0 on entry.  next_src: the path bytes of the row this block
// selects next (same W and layout), or null: as this row's last stages free
// their slots, the copies of the next row's first stages start, so that the
// row epilogue and the next row's start do not wait for DRAM.  Returns false
// if a stage wait gave up: the status word then holds SIMSENSE_ERR_TIMEOUT,
// the copies in flight have been drained (bounded) and the block must not
// touch the ring again.
template <int NP, int G, int PATHS, int THREADS>
__device__ bool select_row(uint8_t* area, uint64_t* bars, int stages, RingPos& rp, int* abort_flag,
                           const uint8_t* __restrict__ vol, float* __restrict__ depth, int y, int W, int D, int uniq,
                           uint32_t umagic, int lr_max_diff, int subpixel, float fb, const SelectDebug& dbg,
                           int* __restrict__ status, int disp_mode, const uint8_t* next_src = nullptr)
{
    using RS = RowShape<NP, G, PATHS, THREADS>;
    constexpr int DPT = RS::DPT;
    constexpr int Dp = RS::Dp;
    constexpr int SPW = RS::SPW;
    constexpr int kPix = RS::kPix;
    constexpr size_t pbytes = RS::pbytes;
    constexpr size_t stage_bytes = RS::stage_bytes;
    uint8_t* ring = area;
    uint16_t* sbuf = reinterpret_cast<uint16_t*>(ring + stages * stage_bytes);   // kPix x Dp, 16-byte aligned
    uint32_t* keyR = reinterpret_cast<uint32_t*>(sbuf + kPix * Dp);               // W + W/32 (padded)
    uint32_t* info = keyR + kr(W);                                                // W
    uint32_t* fit = info + W;                                                     // W

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gl = lane % G, sub = lane / G;
    const int slot_pix = warp * SPW + sub;      // this group's pixel within a stage
    // the lane's padded cells (its disparity chunk as select_pixel takes it)
    uint32_t pad[2 * ((NP + 1) / 2)];
    {
        const int chunk = G == 16 ? (gl + 8 * ((threadIdx.x & 31) / 16)) % 16 : gl;
        const int d0 = chunk * DPT;
#pragma unroll
        for (int k = 0; k < (NP + 1) / 2; k++) {
            pad[2 * k] = (d0 + 4 * k >= D ? 0xffffu : 0u) | (d0 + 4 * k + 2 >= D ? 0xffff0000u : 0u);
            pad[2 * k + 1] = (d0 + 4 * k + 1 >= D ? 0xffffu : 0u) | (d0 + 4 * k + 3 >= D ? 0xffff0000u : 0u);
        }
    }
    uint16_t* sw = sbuf + slot_pix * Dp;
    const int nst = (W + kPix - 1) / kPix;      // stages per row
    const uint8_t* rowsrc = vol + (size_t)y * W * pbytes;
    int slot = rp.slot;
    uint32_t phase = rp.phase;
    // thread 0's count of this row's stages whose copies have started, and
    // of the next row's
    int issued = 0, next_issued = 0;
    if (threadIdx.x == 0) {
        issued = min(rp.ahead, nst);
        int s = slot + issued;
        s = s >= stages ? s - stages : s;
        for (; issued < stages && issued < nst; issued++, s = s + 1 == stages ? 0 : s + 1) {
            const int x0 = issued * kPix, n = min(kPix, W - x0);
            stage_load(&bars[s], ring + s * stage_bytes, rowsrc + (size_t)x0 * pbytes, (uint32_t)(n * pbytes));
        }
    }
    for (int i = threadIdx.x; i < kr(W); i += THREADS) keyR[i] = 0xffffffffu;
    __syncthreads();
    for (int st = 0; st < nst; st++) {
        if (!stage_wait(&bars[slot], phase)) *abort_flag = 1;
        const int x = st * kPix + slot_pix;
        const uint8_t* src = ring + slot * stage_bytes + slot_pix * pbytes;
        if (D == Dp)
            select_pixel<NP, G, PATHS, true>(src, x, x < W, y, W, D, uniq, umagic, subpixel, gl, sw, keyR,
                                             info, fit, dbg, pad);
        else
            select_pixel<NP, G, PATHS, false>(src, x, x < W, y, W, D, uniq, umagic, subpixel, gl, sw, keyR,
                                              info, fit, dbg, pad);
        __syncthreads();                        // everyone is done with this slot
        if (*abort_flag) {
            if (threadIdx.x == 0) {
                if (status) atomicExch(status, SIMSENSE_ERR_TIMEOUT);
                // drain the copies still in flight into this block's ring
                // (bounded), this stage's own included: its wait may be
                // the one that gave up
                int s = slot;
                uint32_t ph = phase;
                for (int j = st; j < issued + next_issued; j++) {
                    stage_wait(&bars[s], ph);
                    if (++s == stages) { s = 0; ph ^= 1u; }
                }
            }
            return false;
        }
        if (threadIdx.x == 0) {
            // the slot just freed takes the stage `stages` ahead: of this
            // row while it has one, else of the next row (when this row has
            // fewer stages than the ring, the sequence positions of the two
            // rows' stages do not line up, and nothing is fetched ahead)
            if (issued < nst) {
                const int x0 = issued * kPix, n = min(kPix, W - x0);
                stage_load(&bars[slot], ring + slot * stage_bytes, rowsrc + (size_t)x0 * pbytes,
                           (uint32_t)(n * pbytes));
                issued++;
            } else if (next_src && next_issued < nst && st + stages == nst + next_issued) {
                const int x0 = next_issued * kPix, n = min(kPix, W - x0);
                stage_load(&bars[slot], ring + slot * stage_bytes, next_src + (size_t)x0 * pbytes,
                           (uint32_t)(n * pbytes));
                next_issued++;
            }
        }
        if (++slot == stages) { slot = 0; phase ^= 1u; }
    }
    rp.slot = slot;
    rp.phase = phase;
    rp.ahead = next_issued;
    for (int x = threadIdx.x; x < W; x += THREADS) {
        const size_t pix = (size_t)y * W + x;
        const uint32_t in = info[x];
        const int ds = (int)(in & 511u);
        int m = (in & 0x8000u) ? 1 : 0;
        float df = (float)ds;
        if (in & 0x4000u) {                    // parabola through S(d*-1), S(d*), S(d*+1)
            const uint32_t fv = fit[x];
            const int sm = (int)(fv & 0xffffu), sp = (int)(fv >> 16), s0 = (int)(in >> 16);
            df = (float)ds + __fdiv_rn((float)(sm - sp), (float)(2 * (sm + sp - 2 * s0)));
        }
        if (lr_max_diff >= 0) {
            const int xr = x - ds;
            if (xr < 0) {
                m |= 2;
            } else {
                const int dr = (int)(keyR[kr(xr)] & 511u);
                const int diff = ds > dr ? ds - dr : dr - ds;
                if (diff > lr_max_diff) m |= 2;
            }
        }
        if (!(df > 0.0f)) m |= 4;
        // disp_mode (a median filter follows): the disparity, 0 when invalid
        if (disp_mode) depth[pix] = m == 0 ? df : 0.0f;
        else depth[pix] = m == 0 ? __fdiv_rn(fb, df) : 0.0f;
        if (dbg.disparity_int) dbg.disparity_int[pix] = (int16_t)ds;
        if (dbg.disparity) dbg.disparity[pix] = m == 0 ? df : -1.0f;
        if (dbg.mask) dbg.mask[pix] = (uint8_t)m;
    }
    __syncthreads();                            // the row arrays are reused by the next row
    return true;
}

}  // namespace sgm
}  // namespace simsense
