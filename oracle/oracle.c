/*
 * Plain CPU oracle for the depth-estimation stage of an active-stereo
 * sensor simulator (arxiv 2201.11924, Sec. VI-D "Depth Generation by Stereo
 * Matching").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: it exists so that the tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against a slow,
 * obviously correct restatement of the method.  It shares no code, header,
 * table or helper with the CUDA sources.
 *
 * Sec. VI-D fixes the order of the steps: census transform, Hamming matching
 * cost, semi-global matching (SGM) cost aggregation along scanline paths,
 * best-disparity selection with a uniqueness test, quadratic sub-pixel
 * fitting, a left-right consistency check, and conversion of disparity to
 * depth.  Each function below is one step, written as plain nested loops in
 * int32 arithmetic (floating point only in the sub-pixel and depth steps,
 * where it is fp64).  There is no blocking, fusion or reordering.
 *
 * Readings of points the paper leaves open (all of them are listed in the
 * design notes of the repository):
 *  - census: full census over a w x h window without its centre,
 *    bit = [I(neighbour) < I(centre)], neighbours outside the image give 0,
 *    bits in raster order (dy outer, dx inner), first offset = most
 *    significant bit.  (Sec. VI-D names a centre-symmetric census; the
 *    bit counts of the configured windows, 24 / 48 / 62, are those of the
 *    full census.)
 *  - cost: C(x,y,d) = popcount(cL(x,y) xor cR(x-d,y)) when x-d >= 0, else
 *    nbits (the worst possible cost); d runs over 0..D-1.
 *  - SGM (Hirschmueller's recurrence, which Sec. VI-D cites):
 *      L_r(p,d) = C(p,d) + min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m'+P2) - m'
 *    with L' = L_r(p-r, .), m' = min_k L'(k), L'(-1) = L'(D) = +inf, and
 *    L_r(p,d) = C(p,d) where p-r is outside the image.  S = sum_r L_r.
 *    4 paths = {->, <-, down, up}; 8 paths add the four diagonals.
 *  - selection: d* = argmin_d S (smallest d on ties); uniqueness with an
 *    integer percentage u: unique iff for all d with |d-d*| > 1,
 *    (100-u) S(d) >= 100 S(d*)  (u = 0 disables it).
 *  - left-right check: D_R(xr) = argmin over d in [0, min(D-1, W-1-xr)] of
 *    S(xr+d, y, d) (smallest d on ties); valid iff x-d* >= 0 and
 *    |d* - D_R(x-d*)| <= lr_max_diff (lr_max_diff < 0 disables it).
 *  - sub-pixel: for 1 <= d* <= D-2, d_f = d* + (S- - S+) / (2 (S- + S+ - 2 S0)),
 *    else d_f = d*;  the checks above use the integer d*.
 *  - depth: Z = f b / d_f for a valid pixel with d_f > 0, else 0.
 *  - mask bits: 1 = uniqueness failed, 2 = left-right failed,
 *    4 = d_f <= 0.  A pixel is valid iff its mask is 0.
 *
 * Sensor noise (Sec. VI-C, the step before stereo matching):
 *    I_noisy = gamma * I_clean + n,  gamma ~ Gamma(k, theta),  n ~ N(mu, sigma^2),
 *  per pixel and view, then rounded half to even and clamped to [0, 255].
 *  Random numbers come from the counter-based Philox4x64-10 generator
 *  (Salmon et al., SC 2011) with counter (pixel, attempt, frame, view) and
 *  key (seed, 0); a 64-bit output r gives the uniform ((r >> 41) + 1/2) / 2^23.
 *  Normals by Box-Muller, gamma by Marsaglia and Tsang's squeeze-free
 *  rejection method (k >= 1), at most 16 attempts (if all are rejected,
 *  gamma = (k - 1/3) theta).
 *
 * Rectification and depth registration (Sec. VI-D: the stage starts by
 *  rectifying the pair onto one image plane and can end by registering the
 *  depth map to the frame of the RGB camera; the paper gives no camera
 *  model).  Readings:
 *  - rectification: for rectified pixel (u, v), the ray R^T ((u - rcx)/rfx,
 *    (v - rcy)/rfy, 1) in the raw camera, normalised by its z, distorted by
 *    the Brown-Conrady model (k1, k2, k3 radial, p1, p2 tangential) and
 *    projected with (fx, fy, cx, cy) gives the raw position (ur, vr), all in
 *    fp64 with + - * / only.  Fixed point: x0 = floor(ur), ax = the fraction
 *    times 256 rounded half to even (256 carries into x0 + 1), the same for
 *    y; the value is the 8-bit bilinear mix ((256-ax)(256-ay) I00 + ...
 *    + 32768) >> 16, taps outside the raw image reading 0.  A ray with
 *    z <= 0 gives 0.
 *  - registration: a valid depth pixel (u, v, Z) of the rectified left
 *    camera (fx, fy, cx, cy) is back-projected, moved by the rigid transform
 *    (R, t) into the RGB camera, projected with its intrinsics and splatted
 *    to the nearest RGB pixel (floor(u' + 1/2)), keeping the smallest Z' > 0
 *    there (a z-buffer); fp64 with + - * / only, Z' rounded to fp32; RGB
 *    pixels no depth pixel reaches stay 0.
 *
 * IR rendering of analytic scenes (Sec. VI-A/VI-B; the paper renders with
 *  ray tracing in Vulkan, here a direct-light ray caster states the same
 *  image formation).  Readings:
 *  - a rectified pinhole pair (left camera at the origin, right at
 *    (b, 0, 0), both looking along +z; f, cx, cy) casts one ray per pixel
 *    centre; the nearest hit among spheres and rectangles wins (ties to the
 *    lower index); no hit gives 0;
 *  - the projector is a textured spot light at a point with its own
 *    pinhole (pf, pcx, pcy) looking along +z; a lit point receives
 *    E = power * pattern / 255 * (n.i) / dist^2, pattern sampled at the
 *    nearest texel, 0 outside the texture or when a shadow ray to the
 *    projector meets another surface;
 *  - BSDF mix of Sec. VI-A: f = w_d f_d + (1 - w_d) f_s, w_d = (1 - metallic)
 *    (1 - transmission), f_d = albedo / pi (Lambert), f_s = the GGX
 *    microfacet term D F G / (4 (n.i)(n.o)) with alpha = roughness^2,
 *    D = alpha^2 / (pi ((n.h)^2 (alpha^2 - 1) + 1)^2), Smith G1(x) =
 *    2x / (x + sqrt(alpha^2 + (1 - alpha^2) x^2)), Schlick F with
 *    F0 = 0.04 (1 - metallic) + albedo * metallic; no refracted light;
 *  - radiance L = f E + ambient * albedo, pixel = gain * L rounded half to
 *    even and clamped to [0, 255];
 *  - all in fp64 with + - * / and sqrt only, in a fixed order.
 *  The two constants of the named approximations are pinned against the
 *  exact Fresnel equations for a dielectric of refractive index 1.5: F0 =
 *  0.04 is the reflectance at normal incidence ((n-1)/(n+1))^2, and with the
 *  exponent 5 Schlick's form stays within 0.04 of the exact reflectance from
 *  grazing to normal incidence (the exponents 4 and 6 do not).
 *
 * Variants Sec. VI-D also names (optional in the stage):
 *  - centre-symmetric census (CSCT): for every offset o of the window that
 *    precedes the centre in raster order, bit = [I(p+o) < I(p-o)]; a pair
 *    with a pixel outside the image gives 0; (w h - 1) / 2 bits, first
 *    offset = most significant bit.
 *  - SGBM block cost: the per-pixel Hamming cost averaged over a bw x bh
 *    block around the pixel (same d), over the block's pixels inside the
 *    image, rounded half up: Cb = floor((sum + n/2) / n).  The paper gives
 *    no normalisation; the mean keeps the cost within [0, nbits], the range
 *    the path costs are bounded with.
 *  - median filter: the k x k median of the disparity map after the checks
 *    (invalid pixels count as 0, borders replicated); the output pixel is
 *    valid iff the median is > 0, with depth f b / median.  The mask keeps
 *    the bits of the checks before the filter.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_ARG -1
#define ORACLE_NO_MEMORY -2

/* ---------------------------------------------------------------- census */

/* Census transform of one view (Sec. VI-D, first step after rectification).
 * img: H x W bytes, row-major.  codes: H x W uint64, row-major. */
int oracle_census(const uint8_t* img, int W, int H, int ww, int wh, uint64_t* codes)
{
    if (!img || !codes || W <= 0 || H <= 0) return ORACLE_BAD_ARG;
    if (ww < 1 || wh < 1 || (ww % 2) == 0 || (wh % 2) == 0) return ORACLE_BAD_ARG;
    if (ww * wh - 1 > 64) return ORACLE_BAD_ARG;
    int rx = ww / 2, ry = wh / 2;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int centre = img[y * W + x];
            uint64_t code = 0;
            for (int dy = -ry; dy <= ry; dy++) {
                for (int dx = -rx; dx <= rx; dx++) {
                    if (dx == 0 && dy == 0) continue;
                    int nx = x + dx, ny = y + dy;
                    int bit = 0;
                    if (nx >= 0 && nx < W && ny >= 0 && ny < H)
                        bit = img[ny * W + nx] < centre ? 1 : 0;
                    /* shifting before each new bit leaves the first offset in
                     * the most significant used position */
                    code = (code << 1) | (uint64_t)bit;
                }
            }
            codes[y * W + x] = code;
        }
    }
    return ORACLE_OK;
}

/* ----------------------------------------------------------- matching cost */

static int hamming64(uint64_t a, uint64_t b)
{
    uint64_t v = a ^ b;
    int n = 0;
    for (int k = 0; k < 64; k++) n += (int)((v >> k) & 1u);
    return n;
}

/* Hamming matching cost volume (Sec. VI-D: the matching cost is the Hamming
 * distance of the census codes).  C: H x W x D bytes, index (y*W + x)*D + d. */
int oracle_cost(const uint64_t* cL, const uint64_t* cR, int W, int H, int D, int nbits, uint8_t* C)
{
    if (!cL || !cR || !C || W <= 0 || H <= 0 || D <= 0 || nbits < 0 || nbits > 64) return ORACLE_BAD_ARG;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int d = 0; d < D; d++) {
                int c = nbits;
                if (x - d >= 0) c = hamming64(cL[y * W + x], cR[y * W + (x - d)]);
                C[((size_t)y * W + x) * D + d] = (uint8_t)c;
            }
    return ORACLE_OK;
}

/* --------------------------------------------------------------------- SGM */

/* One SGM path (Hirschmueller's recurrence, the SGM that Sec. VI-D cites),
 * along direction r = (rx, ry): the value at p comes from p - r.
 * L: H x W x D int32, index (y*W + x)*D + d. */
int oracle_path(const uint8_t* C, int W, int H, int D, int rx, int ry, int P1, int P2, int32_t* L)
{
    if (!C || !L || W <= 0 || H <= 0 || D <= 0) return ORACLE_BAD_ARG;
    if (rx < -1 || rx > 1 || ry < -1 || ry > 1 || (rx == 0 && ry == 0)) return ORACLE_BAD_ARG;
    if (P1 < 0 || P2 < P1) return ORACLE_BAD_ARG;
    /* visit pixels so that p - r is always visited before p */
    int y0 = ry >= 0 ? 0 : H - 1, y1 = ry >= 0 ? H : -1, ys = ry >= 0 ? 1 : -1;
    int x0 = rx >= 0 ? 0 : W - 1, x1 = rx >= 0 ? W : -1, xs = rx >= 0 ? 1 : -1;
    for (int y = y0; y != y1; y += ys) {
        for (int x = x0; x != x1; x += xs) {
            const uint8_t* c = C + ((size_t)y * W + x) * D;
            int32_t* l = L + ((size_t)y * W + x) * D;
            int qx = x - rx, qy = y - ry;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
                for (int d = 0; d < D; d++) l[d] = c[d];
                continue;
            }
            const int32_t* lp = L + ((size_t)qy * W + qx) * D;
            int32_t mprev = lp[0];
            for (int k = 1; k < D; k++)
                if (lp[k] < mprev) mprev = lp[k];
            for (int d = 0; d < D; d++) {
                int32_t best = lp[d];
                if (d - 1 >= 0 && lp[d - 1] + P1 < best) best = lp[d - 1] + P1;
                if (d + 1 < D && lp[d + 1] + P1 < best) best = lp[d + 1] + P1;
                if (mprev + P2 < best) best = mprev + P2;
                l[d] = (int32_t)c[d] + best - mprev;
            }
        }
    }
    return ORACLE_OK;
}

/* The path set: 4 paths = {->, <-, down, up}; 8 paths add the diagonals. */
static const int PATH_DIRS[8][2] = {
    {1, 0}, {-1, 0}, {0, 1}, {0, -1},
    {1, 1}, {-1, 1}, {1, -1}, {-1, -1},
};

/* Aggregated cost S = sum over the paths of L_r.  S: H x W x D int32. */
int oracle_aggregate(const uint8_t* C, int W, int H, int D, int paths, int P1, int P2, int32_t* S)
{
    if (!C || !S || W <= 0 || H <= 0 || D <= 0) return ORACLE_BAD_ARG;
    if (paths != 4 && paths != 8) return ORACLE_BAD_ARG;
    size_t n = (size_t)W * H * D;
    int32_t* L = (int32_t*)malloc(n * sizeof(int32_t));
    if (!L) return ORACLE_NO_MEMORY;
    memset(S, 0, n * sizeof(int32_t));
    for (int r = 0; r < paths; r++) {
        int rc = oracle_path(C, W, H, D, PATH_DIRS[r][0], PATH_DIRS[r][1], P1, P2, L);
        if (rc != ORACLE_OK) { free(L); return rc; }
        for (size_t i = 0; i < n; i++) S[i] += L[i];
    }
    free(L);
    return ORACLE_OK;
}

/* Direction vector of path index r (0..7), for callers that dump one path. */
int oracle_path_dir(int r, int* rx, int* ry)
{
    if (r < 0 || r > 7 || !rx || !ry) return ORACLE_BAD_ARG;
    *rx = PATH_DIRS[r][0];
    *ry = PATH_DIRS[r][1];
    return ORACLE_OK;
}

/* -------------------------------------------- selection and post-processing */

/* Best disparity, uniqueness test, left-right check, quadratic sub-pixel fit
 * and disparity-to-depth conversion (the remaining steps of Sec. VI-D).
 * S: H x W x D int32.  Outputs are H x W; any output pointer may be NULL
 * except dstar.  fb = focal length (px) times baseline (m). */
int oracle_select(const int32_t* S, int W, int H, int D, int uniq, int lr_max_diff,
                  int subpixel, double fb, int32_t* dstar, uint8_t* mask,
                  double* disp, double* depth)
{
    if (!S || !dstar || W <= 0 || H <= 0 || D <= 0 || uniq < 0 || uniq > 99) return ORACLE_BAD_ARG;
    /* pass 1: winner-take-all for every pixel */
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const int32_t* s = S + ((size_t)y * W + x) * D;
            int best = 0;
            for (int d = 1; d < D; d++)
                if (s[d] < s[best]) best = d;
            dstar[y * W + x] = best;
        }
    /* pass 2: checks, sub-pixel, depth */
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            const int32_t* s = S + ((size_t)y * W + x) * D;
            int ds = dstar[y * W + x];
            int m = 0;
            if (uniq > 0) {
                for (int d = 0; d < D; d++) {
                    int diff = d - ds;
                    if (diff < 0) diff = -diff;
                    if (diff <= 1) continue;
                    if ((int64_t)(100 - uniq) * s[d] < (int64_t)100 * s[ds]) { m |= 1; break; }
                }
            }
            if (lr_max_diff >= 0) {
                int xr = x - ds;
                if (xr < 0) {
                    m |= 2;
                } else {
                    int dmax = D - 1;
                    if (W - 1 - xr < dmax) dmax = W - 1 - xr;
                    int dr = 0;
                    int32_t sbest = S[((size_t)y * W + xr) * D + 0];
                    for (int d = 1; d <= dmax; d++) {
                        int32_t v = S[((size_t)y * W + (xr + d)) * D + d];
                        if (v < sbest) { sbest = v; dr = d; }
                    }
                    int diff = ds - dr;
                    if (diff < 0) diff = -diff;
                    if (diff > lr_max_diff) m |= 2;
                }
            }
            double df = (double)ds;
            if (subpixel && ds >= 1 && ds <= D - 2) {
                double sm = s[ds - 1], s0 = s[ds], sp = s[ds + 1];
                df = (double)ds + (sm - sp) / (2.0 * (sm + sp - 2.0 * s0));
            }
            if (!(df > 0.0)) m |= 4;
            if (mask) mask[y * W + x] = (uint8_t)m;
            if (disp) disp[y * W + x] = m == 0 ? df : -1.0;
            if (depth) depth[y * W + x] = m == 0 ? fb / df : 0.0;
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------- variants */

/* Centre-symmetric census transform of one view (the census variant Sec.
 * VI-D names).  img: H x W bytes; codes: H x W uint64. */
int oracle_census_cs(const uint8_t* img, int W, int H, int ww, int wh, uint64_t* codes)
{
    if (!img || !codes || W <= 0 || H <= 0) return ORACLE_BAD_ARG;
    if (ww < 1 || wh < 1 || (ww % 2) == 0 || (wh % 2) == 0) return ORACLE_BAD_ARG;
    if ((ww * wh - 1) / 2 > 64) return ORACLE_BAD_ARG;
    int rx = ww / 2, ry = wh / 2;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            uint64_t code = 0;
            for (int dy = -ry; dy <= ry; dy++) {
                for (int dx = -rx; dx <= rx; dx++) {
                    /* only the offsets before the centre: each pair once */
                    if (dy > 0 || (dy == 0 && dx >= 0)) continue;
                    int ax = x + dx, ay = y + dy;   /* p + o */
                    int bx = x - dx, by = y - dy;   /* p - o */
                    int bit = 0;
                    if (ax >= 0 && ax < W && ay >= 0 && ay < H && bx >= 0 && bx < W && by >= 0 && by < H)
                        bit = img[ay * W + ax] < img[by * W + bx] ? 1 : 0;
                    code = (code << 1) | (uint64_t)bit;
                }
            }
            codes[y * W + x] = code;
        }
    }
    return ORACLE_OK;
}

/* SGBM block cost (Sec. VI-D: the SGBM variant matches neighbourhoods, not
 * single pixels): the mean of C over the bw x bh block centred on each pixel, over
 * the block's pixels inside the image, rounded half up.
 * C, Cb: H x W x D bytes (Cb must not alias C). */
int oracle_cost_block(const uint8_t* C, int W, int H, int D, int bw, int bh, uint8_t* Cb)
{
    if (!C || !Cb || W <= 0 || H <= 0 || D <= 0) return ORACLE_BAD_ARG;
    if (bw < 1 || bh < 1 || (bw % 2) == 0 || (bh % 2) == 0) return ORACLE_BAD_ARG;
    int rx = bw / 2, ry = bh / 2;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int d = 0; d < D; d++) {
                int sum = 0, n = 0;
                for (int v = -ry; v <= ry; v++)
                    for (int u = -rx; u <= rx; u++) {
                        int xx = x + u, yy = y + v;
                        if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                        sum += C[((size_t)yy * W + xx) * D + d];
                        n++;
                    }
                Cb[((size_t)y * W + x) * D + d] = (uint8_t)((sum + n / 2) / n);
            }
    return ORACLE_OK;
}

/* k x k median of a disparity map with replicated borders (Sec. VI-D lists
 * median filtering among the disparity post-processing steps).
 * in, out: H x W doubles (out must not alias in). */
int oracle_median(const double* in, int W, int H, int k, double* out)
{
    if (!in || !out || W <= 0 || H <= 0 || k < 1 || (k % 2) == 0 || k > 9) return ORACLE_BAD_ARG;
    int r = k / 2;
    double win[81];
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            int n = 0;
            for (int v = -r; v <= r; v++)
                for (int u = -r; u <= r; u++) {
                    int xx = x + u, yy = y + v;
                    if (xx < 0) xx = 0;
                    if (xx >= W) xx = W - 1;
                    if (yy < 0) yy = 0;
                    if (yy >= H) yy = H - 1;
                    win[n++] = in[yy * W + xx];
                }
            /* insertion sort; the median is the middle of the k*k values */
            for (int i = 1; i < n; i++) {
                double t = win[i];
                int j = i - 1;
                while (j >= 0 && win[j] > t) { win[j + 1] = win[j]; j--; }
                win[j + 1] = t;
            }
            out[y * W + x] = win[n / 2];
        }
    return ORACLE_OK;
}

/* ---------------------------------------------------------- sensor noise */

/* Philox4x64-10: ten rounds of two 64x64->128-bit multiplies with the key
 * bumped by the Weyl constants between rounds. */
void oracle_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        unsigned __int128 p0 = (unsigned __int128)M0 * x0;
        unsigned __int128 p1 = (unsigned __int128)M1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in (0, 1) from the top 23 bits: (2m + 1) / 2^24, exact in single precision too */
static double unit23(uint64_t r) { return ((double)(r >> 41) + 0.5) / 8388608.0; }

/* Sensor noise of one view (Sec. VI-C).  clean, noisy: H x W bytes.  value
 * (may be NULL): the noisy intensity before rounding.  margin (may be NULL):
 * the smallest distance of a decision to its threshold (the rounding of
 * value and every acceptance test evaluated), for comparisons with a
 * single-precision implementation. */
int oracle_noise(const uint8_t* clean, int W, int H, double mu, double sigma, double k, double theta,
                 uint64_t seed, uint32_t frame, uint32_t view, double* value, uint8_t* noisy, double* margin)
{
    if (!clean || !noisy || W <= 0 || H <= 0 || !(k >= 1.0) || !(theta > 0.0) || !(sigma >= 0.0))
        return ORACLE_BAD_ARG;
    const double PI = 3.14159265358979323846;
    const double d = k - 1.0 / 3.0, c = 1.0 / (3.0 * sqrt(d));
    const uint64_t key[2] = {seed, 0};
    for (int i = 0; i < W * H; i++) {
        double gamma = d * theta, z1 = 0.0, m = 1e300;
        for (int attempt = 0; attempt < 16; attempt++) {
            const uint64_t ctr[4] = {(uint64_t)i, (uint64_t)attempt, frame, view};
            uint64_t r[4];
            oracle_philox4x64(ctr, key, r);
            double u0 = unit23(r[0]), u1 = unit23(r[1]), u2 = unit23(r[2]);
            double rad = sqrt(-2.0 * log(u0));
            double z0 = rad * cos(2.0 * PI * u1);
            z1 = rad * sin(2.0 * PI * u1);
            double t = 1.0 + c * z0;
            if (!(t > 0.0)) continue;
            double v = t * t * t;
            double lhs = log(u2), rhs = 0.5 * z0 * z0 + d - d * v + d * log(v);
            double gap = fabs(lhs - rhs);
            if (gap < m) m = gap;
            if (lhs < rhs) {
                gamma = d * v * theta;
                break;
            }
        }
        double val = gamma * (double)clean[i] + (mu + sigma * z1);
        double q = nearbyint(val);            /* round half to even (default mode) */
        double bgap = fabs(val - (floor(val) + 0.5));
        if (bgap < m) m = bgap;
        if (q < 0.0) q = 0.0;
        if (q > 255.0) q = 255.0;
        noisy[i] = (uint8_t)q;
        if (value) value[i] = val;
        if (margin) margin[i] = m;
    }
    return ORACLE_OK;
}

/* -------------------------------------------- rectification, registration */

/* Camera of one raw view and its rectified counterpart. */
typedef struct {
    double fx, fy, cx, cy;        /* raw intrinsics */
    double k1, k2, p1, p2, k3;    /* Brown-Conrady distortion */
    double R[9];                  /* rectified ray = R * raw ray, row-major */
    double rfx, rfy, rcx, rcy;    /* rectified intrinsics */
} oracle_camera;

/* Fixed-point source position of rectified pixel (u, v): x0, y0 and the
 * 1/256 fractions ax, ay; returns 0 when the ray points behind the camera. */
static int rect_source(const oracle_camera* c, int u, int v, int* x0, int* y0, int* ax, int* ay)
{
    double xr = ((double)u - c->rcx) / c->rfx;
    double yr = ((double)v - c->rcy) / c->rfy;
    /* raw ray = R^T (xr, yr, 1) */
    double X = c->R[0] * xr + c->R[3] * yr + c->R[6];
    double Y = c->R[1] * xr + c->R[4] * yr + c->R[7];
    double Z = c->R[2] * xr + c->R[5] * yr + c->R[8];
    if (!(Z > 0.0)) return 0;
    double x = X / Z, y = Y / Z;
    double r2 = x * x + y * y;
    double radial = 1.0 + c->k1 * r2 + c->k2 * r2 * r2 + c->k3 * r2 * r2 * r2;
    double xd = x * radial + 2.0 * c->p1 * x * y + c->p2 * (r2 + 2.0 * x * x);
    double yd = y * radial + c->p1 * (r2 + 2.0 * y * y) + 2.0 * c->p2 * x * y;
    double ur = c->fx * xd + c->cx, vr = c->fy * yd + c->cy;
    if (!(fabs(ur) < 1e9) || !(fabs(vr) < 1e9)) return 0;
    double fxl = floor(ur), fyl = floor(vr);
    int a = (int)nearbyint((ur - fxl) * 256.0), b = (int)nearbyint((vr - fyl) * 256.0);
    int xi = (int)fxl, yi = (int)fyl;
    if (a == 256) { a = 0; xi++; }
    if (b == 256) { b = 0; yi++; }
    *x0 = xi; *y0 = yi; *ax = a; *ay = b;
    return 1;
}

/* Rectification of one view (raw and rectified images both W x H bytes). */
int oracle_rectify(const uint8_t* raw, int W, int H, const double* cam, uint8_t* out)
{
    if (!raw || !out || !cam || W <= 0 || H <= 0) return ORACLE_BAD_ARG;
    oracle_camera c;
    memcpy(&c, cam, sizeof(c));
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++) {
            int x0, y0, ax, ay;
            uint32_t val = 0;
            if (rect_source(&c, u, v, &x0, &y0, &ax, &ay)) {
                uint32_t t[4] = {0, 0, 0, 0};   /* taps (x0,y0) (x0+1,y0) (x0,y0+1) (x0+1,y0+1) */
                for (int k = 0; k < 4; k++) {
                    int xx = x0 + (k & 1), yy = y0 + (k >> 1);
                    if (xx >= 0 && xx < W && yy >= 0 && yy < H) t[k] = raw[yy * W + xx];
                }
                uint32_t bx = 256 - (uint32_t)ax, by = 256 - (uint32_t)ay;
                val = (bx * by * t[0] + (uint32_t)ax * by * t[1] + bx * (uint32_t)ay * t[2] +
                       (uint32_t)ax * (uint32_t)ay * t[3] + 32768u) >> 16;
            }
            out[v * W + u] = (uint8_t)val;
        }
    return ORACLE_OK;
}

/* Registration of a depth map (W x H, 0 = invalid) of the camera
 * (fx, fy, cx, cy) into an RGB camera: reg = {fx2, fy2, cx2, cy2, R[9], t[3]}.
 * out: W2 x H2 floats. */
int oracle_register(const float* depth, int W, int H, double fx, double fy, double cx, double cy,
                    const double* reg, float* out, int W2, int H2)
{
    if (!depth || !reg || !out || W <= 0 || H <= 0 || W2 <= 0 || H2 <= 0) return ORACLE_BAD_ARG;
    const double fx2 = reg[0], fy2 = reg[1], cx2 = reg[2], cy2 = reg[3];
    const double* R = reg + 4;
    const double* t = reg + 13;
    for (int i = 0; i < W2 * H2; i++) out[i] = 0.0f;
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++) {
            double Z = depth[v * W + u];
            if (!(Z > 0.0)) continue;
            double X = ((double)u - cx) / fx * Z, Y = ((double)v - cy) / fy * Z;
            double X2 = R[0] * X + R[1] * Y + R[2] * Z + t[0];
            double Y2 = R[3] * X + R[4] * Y + R[5] * Z + t[1];
            double Z2 = R[6] * X + R[7] * Y + R[8] * Z + t[2];
            if (!(Z2 > 0.0)) continue;
            double u2 = fx2 * (X2 / Z2) + cx2, v2 = fy2 * (Y2 / Z2) + cy2;
            double pu = floor(u2 + 0.5), pv = floor(v2 + 0.5);
            if (!(pu >= 0.0 && pu < (double)W2 && pv >= 0.0 && pv < (double)H2)) continue;
            int k = (int)pv * W2 + (int)pu;
            float z = (float)Z2;
            if (out[k] == 0.0f || z < out[k]) out[k] = z;
        }
    return ORACLE_OK;
}

/* ---------------------------------------------------------- IR rendering */

typedef struct {
    int kind;                       /* 0 sphere (c, radius), 1 rectangle (c, half-axes u, v) */
    int pad;
    double c[3], u[3], v[3], radius;
    double albedo, metallic, roughness, transmission;
} oracle_prim;

typedef struct {
    int W, H;
    double f, cx, cy, baseline;     /* rectified camera pair */
    double proj[3];                 /* projector centre */
    double pf, pcx, pcy;            /* projector intrinsics */
    int PW, PH;                     /* pattern size */
    double power, ambient, gain;
} oracle_render_params;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Ray o + t d against one primitive: the smallest t > eps, else -1. */
static double hit_prim(const oracle_prim* q, const double* o, const double* d)
{
    const double eps = 1e-9;
    if (q->kind == 0) {
        double oc[3] = {o[0] - q->c[0], o[1] - q->c[1], o[2] - q->c[2]};
        double a = dot3(d, d), b = 2.0 * dot3(d, oc), cc = dot3(oc, oc) - q->radius * q->radius;
        double disc = b * b - 4.0 * a * cc;
        if (disc < 0.0) return -1.0;
        double sq = sqrt(disc);
        double t = (-b - sq) / (2.0 * a);
        if (t > eps) return t;
        t = (-b + sq) / (2.0 * a);
        return t > eps ? t : -1.0;
    }
    double n[3] = {q->u[1] * q->v[2] - q->u[2] * q->v[1], q->u[2] * q->v[0] - q->u[0] * q->v[2],
                   q->u[0] * q->v[1] - q->u[1] * q->v[0]};
    double den = dot3(d, n);
    if (den == 0.0) return -1.0;
    double co[3] = {q->c[0] - o[0], q->c[1] - o[1], q->c[2] - o[2]};
    double t = dot3(co, n) / den;
    if (!(t > eps)) return -1.0;
    double p[3] = {o[0] + t * d[0] - q->c[0], o[1] + t * d[1] - q->c[1], o[2] + t * d[2] - q->c[2]};
    double s = dot3(p, q->u) / dot3(q->u, q->u), w = dot3(p, q->v) / dot3(q->v, q->v);
    if (s < -1.0 || s > 1.0 || w < -1.0 || w > 1.0) return -1.0;
    return t;
}

static double shade(const oracle_prim* prims, int n, const oracle_render_params* rp, const uint8_t* pattern,
                    const double* o, const double* d)
{
    const double PI = 3.14159265358979323846;
    int best = -1;
    double tb = 0.0;
    for (int k = 0; k < n; k++) {
        double t = hit_prim(&prims[k], o, d);
        if (t > 0.0 && (best < 0 || t < tb)) { best = k; tb = t; }
    }
    if (best < 0) return 0.0;
    const oracle_prim* q = &prims[best];
    double p[3] = {o[0] + tb * d[0], o[1] + tb * d[1], o[2] + tb * d[2]};
    double nn[3];
    if (q->kind == 0) {
        nn[0] = (p[0] - q->c[0]) / q->radius; nn[1] = (p[1] - q->c[1]) / q->radius; nn[2] = (p[2] - q->c[2]) / q->radius;
    } else {
        double m[3] = {q->u[1] * q->v[2] - q->u[2] * q->v[1], q->u[2] * q->v[0] - q->u[0] * q->v[2],
                       q->u[0] * q->v[1] - q->u[1] * q->v[0]};
        double len = sqrt(dot3(m, m));
        nn[0] = m[0] / len; nn[1] = m[1] / len; nn[2] = m[2] / len;
        if (dot3(nn, d) > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
    }
    double L = rp->ambient * q->albedo;
    /* projector light */
    double li[3] = {rp->proj[0] - p[0], rp->proj[1] - p[1], rp->proj[2] - p[2]};
    double dist2 = dot3(li, li), dist = sqrt(dist2);
    double iv[3] = {li[0] / dist, li[1] / dist, li[2] / dist};
    double ni = dot3(nn, iv);
    double X[3] = {p[0] - rp->proj[0], p[1] - rp->proj[1], p[2] - rp->proj[2]};
    if (ni > 0.0 && X[2] > 0.0) {
        int lit = 1;
        for (int k = 0; k < n && lit; k++) {
            if (k == best) continue;
            double t = hit_prim(&prims[k], p, li);
            if (t > 0.0 && t < 1.0) lit = 0;
        }
        double up = rp->pf * (X[0] / X[2]) + rp->pcx, vp = rp->pf * (X[1] / X[2]) + rp->pcy;
        double fu = floor(up + 0.5), fv = floor(vp + 0.5);
        double pat = 0.0;
        if (fu >= 0.0 && fu < (double)rp->PW && fv >= 0.0 && fv < (double)rp->PH)
            pat = (double)pattern[(int)fv * rp->PW + (int)fu] / 255.0;
        if (lit && pat > 0.0) {
            double E = rp->power * pat * ni / dist2;
            double ov[3] = {o[0] - p[0], o[1] - p[1], o[2] - p[2]};
            double ol = sqrt(dot3(ov, ov));
            ov[0] = ov[0] / ol; ov[1] = ov[1] / ol; ov[2] = ov[2] / ol;
            double no = dot3(nn, ov);
            double wd = (1.0 - q->metallic) * (1.0 - q->transmission);
            double fd = q->albedo / PI;
            double fs = 0.0;
            if (no > 0.0) {
                double hv[3] = {iv[0] + ov[0], iv[1] + ov[1], iv[2] + ov[2]};
                double hl = sqrt(dot3(hv, hv));
                hv[0] = hv[0] / hl; hv[1] = hv[1] / hl; hv[2] = hv[2] / hl;
                double a = q->roughness * q->roughness, a2 = a * a;
                double nh = dot3(nn, hv);
                double den = nh * nh * (a2 - 1.0) + 1.0;
                double D = a2 / (PI * den * den);
                double g1i = 2.0 * ni / (ni + sqrt(a2 + (1.0 - a2) * ni * ni));
                double g1o = 2.0 * no / (no + sqrt(a2 + (1.0 - a2) * no * no));
                double F0 = 0.04 * (1.0 - q->metallic) + q->albedo * q->metallic;
                double vh = dot3(ov, hv);
                double m1 = 1.0 - vh, m2 = m1 * m1;
                double F = F0 + (1.0 - F0) * (m2 * m2 * m1);
                fs = D * F * (g1i * g1o) / (4.0 * ni * no);
            }
            L = L + (wd * fd + (1.0 - wd) * fs) * E;
        }
    }
    return rp->gain * L;
}

/* IR images of both cameras.  prims: n primitives; pattern: PH x PW bytes;
 * left, right: H x W bytes; left_f, right_f (may be NULL): gain * L before
 * rounding. */
int oracle_render(const oracle_prim* prims, int n, const oracle_render_params* rp, const uint8_t* pattern,
                  uint8_t* left, uint8_t* right, double* left_f, double* right_f)
{
    if (!prims || n < 0 || !rp || !pattern || !left || !right || rp->W <= 0 || rp->H <= 0) return ORACLE_BAD_ARG;
    for (int view = 0; view < 2; view++) {
        double o[3] = {view ? rp->baseline : 0.0, 0.0, 0.0};
        uint8_t* img = view ? right : left;
        double* imf = view ? right_f : left_f;
        for (int v = 0; v < rp->H; v++)
            for (int u = 0; u < rp->W; u++) {
                double d[3] = {((double)u - rp->cx) / rp->f, ((double)v - rp->cy) / rp->f, 1.0};
                double val = shade(prims, n, rp, pattern, o, d);
                double qv = nearbyint(val);
                if (qv < 0.0) qv = 0.0;
                if (qv > 255.0) qv = 255.0;
                img[v * rp->W + u] = (uint8_t)qv;
                if (imf) imf[v * rp->W + u] = val;
            }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------ whole stage */

/* The whole depth stage for one rectified pair, with the optional variants:
 * census_cs = 1 selects the centre-symmetric census, bw x bh > 1 x 1 the SGBM
 * block cost, median_k > 1 the median filter.  Every output except depth may
 * be NULL.  codes: H x W; S: H x W x D int32. */
int oracle_compute_ex(const uint8_t* left, const uint8_t* right, int W, int H, int D,
                      int ww, int wh, int P1, int P2, int paths, int uniq, int lr_max_diff,
                      int subpixel, double f, double baseline, int census_cs, int bw, int bh, int median_k,
                      double* depth, double* disp, int32_t* dstar, uint8_t* mask,
                      uint64_t* codes_left, uint64_t* codes_right, int32_t* S_out)
{
    if (!left || !right || !depth || W <= 0 || H <= 0 || D <= 0) return ORACLE_BAD_ARG;
    if (bw < 1 || bh < 1 || median_k < 0) return ORACLE_BAD_ARG;
    int nbits = census_cs ? (ww * wh - 1) / 2 : ww * wh - 1;
    size_t npx = (size_t)W * H, nvol = npx * (size_t)D;
    uint64_t* cl = codes_left ? codes_left : (uint64_t*)malloc(npx * sizeof(uint64_t));
    uint64_t* cr = codes_right ? codes_right : (uint64_t*)malloc(npx * sizeof(uint64_t));
    uint8_t* C = (uint8_t*)malloc(nvol);
    int32_t* S = S_out ? S_out : (int32_t*)malloc(nvol * sizeof(int32_t));
    int32_t* ds = dstar ? dstar : (int32_t*)malloc(npx * sizeof(int32_t));
    int rc = ORACLE_OK;
    if (!cl || !cr || !C || !S || !ds) { rc = ORACLE_NO_MEMORY; goto done; }
    if (census_cs) {
        rc = oracle_census_cs(left, W, H, ww, wh, cl);
        if (rc == ORACLE_OK) rc = oracle_census_cs(right, W, H, ww, wh, cr);
    } else {
        rc = oracle_census(left, W, H, ww, wh, cl);
        if (rc == ORACLE_OK) rc = oracle_census(right, W, H, ww, wh, cr);
    }
    if (rc == ORACLE_OK) rc = oracle_cost(cl, cr, W, H, D, nbits, C);
    if (rc == ORACLE_OK && (bw > 1 || bh > 1)) {
        uint8_t* Cb = (uint8_t*)malloc(nvol);
        if (!Cb) { rc = ORACLE_NO_MEMORY; goto done; }
        rc = oracle_cost_block(C, W, H, D, bw, bh, Cb);
        memcpy(C, Cb, nvol);
        free(Cb);
    }
    if (rc == ORACLE_OK) rc = oracle_aggregate(C, W, H, D, paths, P1, P2, S);
    if (rc == ORACLE_OK) {
        double* dsp = (double*)malloc(npx * sizeof(double));
        uint8_t* msk = (uint8_t*)malloc(npx);
        if (!dsp || !msk) {
            free(dsp);
            free(msk);
            rc = ORACLE_NO_MEMORY;
            goto done;
        }
        rc = oracle_select(S, W, H, D, uniq, lr_max_diff, subpixel, f * baseline, ds, msk, dsp, depth);
        if (rc == ORACLE_OK && median_k > 1) {
            /* invalid pixels enter the filter as 0 */
            double* d0 = (double*)malloc(npx * sizeof(double));
            if (!d0) {
                rc = ORACLE_NO_MEMORY;
            } else {
                for (size_t i = 0; i < npx; i++) d0[i] = msk[i] == 0 ? dsp[i] : 0.0;
                rc = oracle_median(d0, W, H, median_k, dsp);
                for (size_t i = 0; i < npx && rc == ORACLE_OK; i++) {
                    depth[i] = dsp[i] > 0.0 ? f * baseline / dsp[i] : 0.0;
                    if (!(dsp[i] > 0.0)) dsp[i] = -1.0;
                }
                free(d0);
            }
        }
        if (disp) memcpy(disp, dsp, npx * sizeof(double));
        if (mask) memcpy(mask, msk, npx);
        free(dsp);
        free(msk);
    }
done:
    if (!codes_left) free(cl);
    if (!codes_right) free(cr);
    free(C);
    if (!S_out) free(S);
    if (!dstar) free(ds);
    return rc;
}

/* The plain stage (full census, per-pixel cost, no median filter). */
int oracle_compute(const uint8_t* left, const uint8_t* right, int W, int H, int D,
                   int ww, int wh, int P1, int P2, int paths, int uniq, int lr_max_diff,
                   int subpixel, double f, double baseline,
                   double* depth, double* disp, int32_t* dstar, uint8_t* mask,
                   uint64_t* codes_left, uint64_t* codes_right, int32_t* S_out)
{
    return oracle_compute_ex(left, right, W, H, D, ww, wh, P1, P2, paths, uniq, lr_max_diff, subpixel, f,
                             baseline, 0, 1, 1, 0, depth, disp, dstar, mask, codes_left, codes_right, S_out);
}
