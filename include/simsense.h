/*
 * simsense.h — C ABI of the GB300 (sm_103a) depth stage of an active-stereo
 * sensor simulator: rectified left/right IR pair in, depth map out.
 *
 * The stage follows arxiv 2201.11924, Sec. VI-D ("Depth Generation by Stereo
 * Matching"): census transform of both views, Hamming matching cost, semi-
 * global matching (SGM) cost aggregation along 4 or 8 scanline paths with
 * penalties P1/P2, winner-take-all with a uniqueness test, a left-right
 * consistency check, quadratic (parabolic) sub-pixel refinement and the
 * conversion of disparity d to depth Z = f * b / d.  Sec. VI-D also states
 * that the module's key parameters are adjustable per sensor; they are the
 * arguments of simsense_create().
 *
 * Definitions (the readings of points the paper leaves open):
 *  - census over a w x h window without its centre, bit = [I(nbr) < I(ctr)],
 *    neighbours outside the image give 0, bits in raster order with the first
 *    offset as the most significant bit; nbits = w*h - 1.
 *  - cost C(x,y,d) = popcount(cL(x,y) ^ cR(x-d,y)) for x-d >= 0, else nbits;
 *    d = 0 .. D-1.
 *  - SGM: L_r(p,d) = C(p,d) + min(L'(d), L'(d+-1)+P1, m'+P2) - m' with
 *    L' = L_r(p-r,.), m' = min L'; L_r = C where p-r is outside the image;
 *    S = sum over the paths of L_r.  4 paths: -> <- down up; 8 paths add the
 *    diagonals.
 *  - d* = argmin_d S (smallest d on ties).  Uniqueness (u = uniq_ratio in
 *    percent, 0 disables): unique iff (100-u) S(d) >= 100 S(d*) for every d
 *    with |d-d*| > 1.
 *  - left-right check (lr_max_diff < 0 disables): D_R(xr) = argmin over
 *    d <= min(D-1, W-1-xr) of S(xr+d, y, d) (smallest d on ties); the pixel
 *    passes iff x-d* >= 0 and |d* - D_R(x-d*)| <= lr_max_diff.
 *  - sub-pixel (on by default): for 1 <= d* <= D-2,
 *    d_f = d* + (S- - S+) / (2 (S- + S+ - 2 S0)) in IEEE fp32 (one
 *    round-to-nearest division of the two exact integers), else d_f = d*.
 *  - depth: Z = fb / d_f (fp32, round to nearest) with fb = (float)(f * b)
 *    formed in double; Z = 0 for a pixel that failed a check or has d_f <= 0.
 *
 * Conventions for every call:
 *  - images are contiguous row-major with pitch W (no padding): uint8 H x W
 *    for the views, float32 H x W for depth; caller-owned; inputs and outputs
 *    must not overlap.  Device buffers belong to the GPU that was current
 *    when the handle was created (the calls switch to it); the library does
 *    not check a pointer's GPU, the Python binding does.
 *  - the library owns its scratch memory: it is allocated by simsense_create
 *    and released by simsense_destroy; simsense_compute allocates nothing.
 *  - compute calls are asynchronous on the given CUDA stream (NULL = the
 *    legacy default stream); results are ready once the stream has been
 *    synchronised.  One handle must not be used by two streams at once (its
 *    scratch is shared by its calls).
 *  - every call returns a status code (SIMSENSE_OK or a negative error);
 *    nothing aborts, traps or prints.  simsense_last_cuda_error() returns the
 *    CUDA error code behind the most recent SIMSENSE_ERR_CUDA of a handle.
 */
#ifndef SIMSENSE_H
#define SIMSENSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;                       /* = cudaStream_t */
typedef struct simsense_ctx* simsense_t;

/* status codes */
#define SIMSENSE_OK                 0
#define SIMSENSE_ERR_INVALID_ARG   -1     /* an argument is out of range or NULL */
#define SIMSENSE_ERR_OOM           -2     /* scratch allocation failed */
#define SIMSENSE_ERR_CUDA          -3     /* a CUDA call or launch failed */
#define SIMSENSE_ERR_TIMEOUT       -4     /* a bounded device-side wait gave up */

/* options for simsense_set_option */
#define SIMSENSE_OPT_SUBPIXEL       1     /* value 0/1, default 1 */
#define SIMSENSE_OPT_PROFILE        2     /* value 0/1, default 0: time each stage */
/*
 * Variants of the stage that Sec. VI-D names (arxiv 2201.11924): a
 * centre-symmetric census, semi-global block matching (SGBM), whose cost
 * compares the regions around the two pixels by Hamming distance, and a
 * median filter among the disparity post-processing steps.  The paper
 * defines none of them; the library's readings:
 *  CENSUS_CS  value 0/1, default 0.  1: for every window offset o before the
 *             centre in raster order, bit = [I(p+o) < I(p-o)], a pair with a
 *             pixel outside the image gives 0; (w*h-1)/2 bits, first offset
 *             = most significant bit.
 *  BLOCK      value bw | bh << 8 (odd, 1..7 each), default 1 | 1 << 8 (per-
 *             pixel cost).  Otherwise the cost of (x, y, d) is the per-pixel
 *             Hamming cost averaged over the bw x bh block around (x, y) at
 *             the same d, over the block's pixels inside the image, rounded
 *             half up (the mean keeps the cost within [0, nbits]).
 *  MEDIAN     value 0, 3 or 5, default 0.  k x k median of the disparity map
 *             after the checks (invalid pixels count as 0, borders
 *             replicated); a pixel is valid iff the median is > 0, depth =
 *             f*b / median.  The debug disparity is the filtered one; the
 *             debug mask keeps the bits of the checks before the filter.
 * Out-of-range values return SIMSENSE_ERR_INVALID_ARG and change nothing.
 * The batch and no-allocation entry points run the plain stage only.
 */
#define SIMSENSE_OPT_CENSUS_CS      3
#define SIMSENSE_OPT_BLOCK          4
#define SIMSENSE_OPT_MEDIAN         5

/*
 * SIMSENSE_OPT_TEST_STALL (value 0/1, default 0): a test of the bounded
 * device-side waits.  While 1, the cost stage's MMA-issuing thread issues no
 * tensor-core work, so the waits on its completions run out (each after a
 * limit of 2048 short tries instead of the normal ~1 s): the stage gives up,
 * frees its tensor memory and returns, simsense_device_status then reports
 * SIMSENSE_ERR_TIMEOUT, the depth of that call is undefined, and the handle
 * and the CUDA context stay usable.  Nothing faults, traps or hangs.
 */
#define SIMSENSE_OPT_TEST_STALL     6

/* stages timed under SIMSENSE_OPT_PROFILE, in launch order */
#define SIMSENSE_STAGE_CENSUS       0     /* census transform of both views */
#define SIMSENSE_STAGE_COST         1     /* Hamming matching cost volume */
#define SIMSENSE_STAGE_PATHS        2     /* SGM path aggregation */
#define SIMSENSE_STAGE_SELECT       3     /* sum of paths, WTA, checks, sub-pixel, depth */
#define SIMSENSE_NUM_STAGES         4

/* census_win packs the window as w | (h << 8); h = 0 means a square w x w. */
#define SIMSENSE_WIN(w, h) ((w) | ((h) << 8))

/*
 * Create a matcher for W x H pairs with disparities 0 .. D-1 (Sec. VI-D:
 * the stage's adjustable parameters).
 *   census_win   SIMSENSE_WIN(w, h) with odd w, h <= 15 and 1 <= w*h - 1 <= 64
 *                (e.g. 5x5 -> 24 bits, 7x7 -> 48, 9x7 -> 62)
 *   P1, P2       SGM penalties, 0 <= P1 <= P2 and nbits + P2 <= 255
 *   paths        4 or 8
 *   uniq_ratio   0 .. 99 (percent; 0 disables the uniqueness test)
 *   lr_max_diff  < 0 disables the left-right check
 *   f, baseline  focal length in pixels and baseline in metres, both > 0
 * Limits: 1 <= D <= 256, D <= W, w <= W <= 8192 and h <= H <= 16384.
 * Returns SIMSENSE_ERR_INVALID_ARG for anything outside these ranges,
 * SIMSENSE_ERR_OOM if the scratch memory cannot be allocated on the current
 * device (the handle is bound to that device).  On success *out owns the
 * handle; release it with simsense_destroy.
 */
int simsense_create(simsense_t* out, int W, int H, int D, int census_win, int P1, int P2,
                    int paths, int uniq_ratio, int lr_max_diff, float f, float baseline);

/*
 * Depth of one rectified pair (the whole of Sec. VI-D after rectification).
 *   left_u8, right_u8   device pointers, H x W uint8
 *   depth_f32           device pointer, H x W float32 (written in full)
 *   stream              CUDA stream the kernels are enqueued on
 */
int simsense_compute(simsense_t h, const uint8_t* left_u8, const uint8_t* right_u8,
                     float* depth_f32, struct CUstream_st* stream);

/*
 * Same as simsense_compute for HOST buffers: copies both views from host
 * memory into the handle's device staging buffers, runs the stage and copies
 * the depth map back, all enqueued on stream.  Page-locked host buffers make
 * the copies asynchronous; with pageable ones the copies block the host.
 * The depth buffer is complete once the stream has been synchronised.
 */
int simsense_compute_host(simsense_t h, const uint8_t* left_host, const uint8_t* right_host,
                          float* depth_host, struct CUstream_st* stream);

/*
 * Intermediate results of one compute call, all DEVICE pointers; any member
 * may be NULL to skip it.  They are written by the same kernels that run in
 * simsense_compute (no separate code path).
 *   census_left/right  H x W uint64 codes (always widened to 64 bits)
 *   aggregated         H x W x D uint16, S(x, y, d) at (y*W + x)*D + d
 *   disparity_int      H x W int16, the winner d*
 *   disparity          H x W float32, d_f of a valid pixel, -1.0f otherwise
 *   mask               H x W uint8, bit 1 = uniqueness failed,
 *                      bit 2 = left-right check failed, bit 4 = d_f <= 0
 *   cost               H x W x D uint8, the matching cost C(x, y, d) at
 *                      (y*W + x)*D + d (the block cost with SIMSENSE_OPT_BLOCK)
 *   paths              paths x H x W x D uint8, L_r(x, y, d) of direction r
 *                      at ((r*H + y)*W + x)*D + d, r in the order ->, <-,
 *                      down, up, down-right, down-left, up-right, up-left
 *                      (each path cost is at most nbits + P2 <= 255), copied
 *                      from the path volume the path kernel wrote
 */
typedef struct simsense_debug {
    uint64_t* census_left;
    uint64_t* census_right;
    uint16_t* aggregated;
    int16_t* disparity_int;
    float* disparity;
    uint8_t* mask;
    uint8_t* cost;
    uint8_t* paths;
} simsense_debug_t;

/* simsense_compute plus the intermediate results named in *dbg (device
 * pointers, see simsense_debug_t).  dbg may be NULL. */
int simsense_compute_debug(simsense_t h, const uint8_t* left_u8, const uint8_t* right_u8,
                           float* depth_f32, const simsense_debug_t* dbg,
                           struct CUstream_st* stream);

/*
 * No-allocation variant of simsense_compute (the paper has no counterpart;
 * this is a deployment aid).  For callers that may not allocate device memory
 * at all: a plugin whose host application owns all device memory through its
 * own pool, a real-time loop that bans allocation after start-up because
 * cudaMalloc can block the host and synchronise the device, or a process whose
 * memory is already held by another framework's caching allocator.  Such a
 * caller cannot use simsense_create, which allocates the handle's scratch.
 *
 * This call takes the parameters of simsense_create (same ranges) plus the
 * sub-pixel switch (0/1) and the device buffers of one pair, and runs the same
 * kernels as simsense_compute on a fixed scratch array that is part of the
 * library image (SIMSENSE_NOALLOC_SCRATCH_BYTES on every GPU that loads the
 * library's code, held until the process exits).  It calls no cudaMalloc,
 * cudaFree or allocating library routine.
 *   - The problem must fit: 2 * round256(W*H*code bytes)
 *     + round256(W*H*Dp) + paths*W*H*Dp <= SIMSENSE_NOALLOC_SCRATCH_BYTES,
 *     with code bytes = 4 when w*h - 1 <= 32 else 8, and Dp = 64 * ceil(D/64).  Larger problems, like
 *     any other out-of-range argument, return SIMSENSE_ERR_INVALID_ARG.
 *     (320x240, D = 64, 4 paths fits; 1280x720 does not.)
 *   - The first call on a device looks up the array's device address with
 *     that device current (a one-time set-up per device).  With lazy module
 *     loading (the CUDA default) that lookup also loads the library's device
 *     code on the device, which is when the array is reserved: a caller whose
 *     memory pool takes the rest of the device should make this first call at
 *     start-up, before the pool grows and before any stream capture.  The
 *     cached address is not refreshed after cudaDeviceReset.
 *   - All calls share the one array: calls whose kernels overlap on the GPU
 *     (different streams or threads) race; order them, e.g. on one stream.
 *     Nothing in the array needs clearing between calls, since every byte a
 *     call reads is written earlier in the same call.
 *   - Bounded device-side waits that give up record SIMSENSE_ERR_TIMEOUT in a
 *     status word of the same kind (one per GPU, in the library image, zero
 *     at load); simsense_noalloc_status reads it.
 * Asynchronous on stream like simsense_compute; SIMSENSE_ERR_CUDA reports a
 * failed launch (there is no handle to keep the CUDA error code; the error is
 * cleared so that it does not reach the caller's next CUDA call).
 */
#define SIMSENSE_NOALLOC_SCRATCH_BYTES (32u << 20)
int simsense_compute_noalloc(const uint8_t* left_u8, const uint8_t* right_u8, float* depth_f32,
                             int W, int H, int D, int census_win, int P1, int P2, int paths,
                             int uniq_ratio, int lr_max_diff, float f, float baseline,
                             int subpixel, struct CUstream_st* stream);

/*
 * Device-side status of the no-allocation calls on the current GPU (the
 * paper has no counterpart): like simsense_device_status, synchronises
 * `stream`, returns SIMSENSE_OK or the status recorded since the last read
 * (SIMSENSE_ERR_TIMEOUT if a bounded wait of a call gave up; that call's depth
 * is then undefined) and clears it.  Allocates nothing (the word lives next to
 * the scratch array); SIMSENSE_ERR_CUDA if the copy fails.
 */
int simsense_noalloc_status(struct CUstream_st* stream);

/*
 * IR sensor noise (arxiv 2201.11924 Sec. VI-C): I_noisy = gamma * I_clean + n
 * per pixel, gamma ~ Gamma(k, theta) (laser speckle), n ~ N(mu, sigma^2)
 * (thermal noise); the D415 values Sec. VII estimates are mu = -0.231,
 * sigma = 0.83, k = 3.98, theta = 0.254.  The result is rounded half to even
 * and clamped to [0, 255].  Random numbers: Philox4x64-10 with counter
 * (pixel index y*W + x, attempt, frame, view) and key (seed, 0); a 64-bit
 * output r gives the uniform ((r >> 41) + 1/2) / 2^23; normals by Box-Muller,
 * gamma by Marsaglia-Tsang rejection (k >= 1, at most 16 attempts).  The paper
 * fixes neither the generator nor the sampling method.
 *
 * simsense_set_noise: enable (1) or disable (0) the noise on both views of
 * every later compute call of h (views 0 = left, 1 = right); the n-th call
 * after this one uses frame n.  Requires k >= 1, theta > 0, sigma >= 0, all
 * finite, when enabling; else SIMSENSE_ERR_INVALID_ARG.  The batch and
 * no-allocation entry points run without noise.
 *
 * simsense_add_noise: the same noise on one device image: clean and noisy
 * are W x H device bytes (row-major; they may be the same buffer), frame and
 * view select the generator stream.  Asynchronous on stream;
 * SIMSENSE_ERR_INVALID_ARG for NULL buffers, W or H < 1, W*H > 2^30 or the
 * parameter ranges above, SIMSENSE_ERR_CUDA for a failed launch.
 */
int simsense_set_noise(simsense_t h, int enable, float mu, float sigma, float k, float theta,
                       unsigned long long seed);
int simsense_add_noise(const uint8_t* clean, uint8_t* noisy, int W, int H, float mu, float sigma, float k,
                       float theta, unsigned long long seed, unsigned int frame, unsigned int view,
                       struct CUstream_st* stream);

/*
 * Stereo rectification and depth registration (arxiv 2201.11924 Sec. VI-D:
 * the stage starts by rectifying the pair onto one image plane and can end by
 * registering the depth map to the frame of the RGB camera).  The paper gives
 * no camera model; the library's reading:
 *  - camera of one view: raw intrinsics (fx, fy, cx, cy) in pixels, Brown-
 *    Conrady distortion (k1, k2, k3 radial, p1, p2 tangential), rectifying
 *    rotation R (row-major; rectified ray = R * raw ray) and rectified
 *    intrinsics (rfx, rfy, rcx, rcy).  Rectified pixel (u, v) samples the raw
 *    image at (fx x_d + cx, fy y_d + cy), where (x, y) is the raw ray
 *    R^T ((u - rcx)/rfx, (v - rcy)/rfy, 1) divided by its z and
 *    x_d = x (1 + k1 r^2 + k2 r^4 + k3 r^6) + 2 p1 x y + p2 (r^2 + 2 x^2),
 *    y_d = y (1 + k1 r^2 + k2 r^4 + k3 r^6) + p1 (r^2 + 2 y^2) + 2 p2 x y;
 *    computed in fp64 without fused multiply-adds, quantised to 1/256 px
 *    (half to even) and resampled by 8-bit fixed-point bilinear
 *    interpolation; taps outside the raw image read 0, rays with z <= 0 give 0.
 *    Raw and rectified images have the same size W x H.
 *  - registration: every depth pixel (u, v) with Z > 0 of the camera
 *    (fx, fy, cx, cy) goes to X = (u - cx)/fx Z, Y = (v - cy)/fy Z, then
 *    P' = R (X, Y, Z) + t in the RGB camera (fx2, fy2, cx2, cy2), which
 *    projects it to the nearest pixel floor(fx2 X'/Z' + cx2 + 1/2), ...;
 *    each RGB pixel keeps the smallest Z' > 0 (fp32), others are 0.
 *
 * simsense_set_rectify: rectify both raw views (after the sensor noise,
 * before the census) in every later compute call of h; NULL, NULL switches
 * it off.  Computes the two per-pixel maps once (8 bytes per pixel each,
 * allocated here, freed by simsense_destroy or the next call).  Returns
 * SIMSENSE_ERR_INVALID_ARG for one NULL camera or a non-finite or zero focal
 * length, SIMSENSE_ERR_OOM, SIMSENSE_ERR_CUDA.
 * simsense_rectify: one view, map and resampling in one launch; raw and out
 * are W x H device bytes (not the same buffer).
 * simsense_register_depth: depth is W x H device floats (0 = invalid), out is
 * reg->W2 x reg->H2 device floats, cleared here.  Both asynchronous on
 * stream; SIMSENSE_ERR_INVALID_ARG for NULL pointers, sizes outside
 * 1..32000 or non-finite parameters.
 */
typedef struct {
    double fx, fy, cx, cy;
    double k1, k2, p1, p2, k3;
    double R[9];
    double rfx, rfy, rcx, rcy;
} simsense_camera_t;

typedef struct {
    double fx, fy, cx, cy;        /* the depth map's camera */
    double fx2, fy2, cx2, cy2;    /* the RGB camera */
    double R[9];                  /* depth camera -> RGB camera, row-major */
    double t[3];                  /* metres */
    int W2, H2;                   /* RGB image size */
} simsense_registration_t;

int simsense_set_rectify(simsense_t h, const simsense_camera_t* left, const simsense_camera_t* right);
int simsense_rectify(const uint8_t* raw, uint8_t* out, int W, int H, const simsense_camera_t* cam,
                     struct CUstream_st* stream);
int simsense_register_depth(const float* depth, int W, int H, const simsense_registration_t* reg, float* out,
                            struct CUstream_st* stream);

/*
 * IR image formation of analytic scenes (arxiv 2201.11924 Sec. VI-A/VI-B: the
 * projector is a spot light that throws a texture, surfaces use the BSDF mix
 * f = w_d f_d + (1 - w_d) f_s with w_d = (1 - metallic)(1 - transmission),
 * f_d Lambertian, f_s GGX, plus a weak ambient light).  The paper renders with
 * a Vulkan path tracer; the library's reading is a direct-light ray caster:
 *  - cameras: a rectified pinhole pair (f, cx, cy in pixels), the left at the
 *    origin and the right at (baseline, 0, 0), both looking along +z; one ray
 *    per pixel centre, the nearest hit among the primitives (ties to the lower
 *    index), 0 where nothing is hit;
 *  - primitives: kind 0 sphere (centre c, radius), kind 1 rectangle (centre
 *    c, half-axes u and v, assumed orthogonal); albedo, metallic, roughness,
 *    transmission in [0, 1];
 *  - projector at proj looking along +z, pinhole (pf, pcx, pcy), texture
 *    pattern PH x PW bytes sampled at the nearest texel; a point receives
 *    E = power * pattern / 255 * (n.i) / dist^2 unless the texel lies outside
 *    the texture or another primitive is between it and the projector;
 *  - f_s = D F G / (4 (n.i)(n.o)), alpha = roughness^2, D GGX, Smith G1,
 *    Schlick F with F0 = 0.04 (1 - metallic) + albedo metallic; no refracted
 *    or indirect light;
 *  - pixel = gain * (f E + ambient * albedo), rounded half to even, clamped
 *    to [0, 255]; fp64 with correctly rounded + - * / and sqrt in a fixed
 *    order.
 * prims: n (0..4096) device primitives; pattern, left, right: device bytes;
 * rp: host pointer.  Asynchronous on stream; SIMSENSE_ERR_INVALID_ARG for
 * NULL pointers, sizes outside 1..16384, non-finite parameters or a zero
 * focal length.
 */
typedef struct {
    int kind;                       /* 0 sphere, 1 rectangle */
    int pad;
    double c[3], u[3], v[3], radius;
    double albedo, metallic, roughness, transmission;
} simsense_primitive_t;

typedef struct {
    int W, H;
    double f, cx, cy, baseline;
    double proj[3];
    double pf, pcx, pcy;
    int PW, PH;
    double power, ambient, gain;
} simsense_render_t;

int simsense_render_ir(const simsense_primitive_t* prims, int n, const simsense_render_t* rp,
                       const uint8_t* pattern, uint8_t* left, uint8_t* right, struct CUstream_st* stream);

/* Set an option (SIMSENSE_OPT_*).  Takes effect at the next compute call. */
int simsense_set_option(simsense_t h, int opt, int value);

/*
 * Stage timings.  While SIMSENSE_OPT_PROFILE is 1, every compute call records
 * CUDA events around each stage on its stream (up to 4096 calls are kept).
 * simsense_profile_read waits for the recorded events, writes into
 * stage_ms[0 .. SIMSENSE_NUM_STAGES-1] the summed duration of each stage over
 * the recorded calls, sets *n_calls to their number and clears the record.
 * Either pointer may be NULL.
 */
int simsense_profile_read(simsense_t h, double* stage_ms, int* n_calls);

/* Name of stage i (SIMSENSE_STAGE_*), or NULL. */
const char* simsense_stage_name(int i);

/*
 * Device-side status of the handle's kernels since the last call: waits
 * inside the kernels are bounded, and one that gives up records
 * SIMSENSE_ERR_TIMEOUT instead of hanging (its output is then undefined).
 * Synchronises `stream`, returns SIMSENSE_OK or the recorded status, and
 * clears it.
 */
int simsense_device_status(simsense_t h, struct CUstream_st* stream);

/* Bytes of device scratch memory the handle holds (for admission control). */
size_t simsense_scratch_bytes(simsense_t h);

/* Release the handle and its scratch memory.  NULL is accepted. */
int simsense_destroy(simsense_t h);

/*
 * Completion notice for a request loop (a serving aid; the paper has no
 * counterpart): once all work enqueued on `stream` before this call has
 * finished, the 8 bytes of `tag` are written to the file descriptor fd
 * (typically the write end of a pipe), from the CUDA driver's callback thread.
 * A loop can then block in poll/select on the read end until its earliest
 * request is done instead of querying events in a spin.  The write is a single
 * write of 8 bytes (atomic on a pipe); fd must stay open until the notice has
 * been written, and a full pipe blocks the stream's later work until it is
 * read.  SIMSENSE_ERR_INVALID_ARG for fd < 0, SIMSENSE_ERR_CUDA if the host
 * function cannot be enqueued.
 */
int simsense_notify_on_completion(struct CUstream_st* stream, int fd, unsigned long long tag);

/* ------------------------------------------------------------------ batches */

/*
 * Parameters of one pair of a batch: the arguments of simsense_create (same
 * ranges) plus the sub-pixel switch (0/1).
 */
typedef struct simsense_pair_params {
    int W, H, D;
    int census_win;          /* SIMSENSE_WIN(w, h) */
    int P1, P2;
    int paths;               /* 4 or 8 */
    int uniq_ratio;          /* 0 .. 99 */
    int lr_max_diff;         /* < 0 disables */
    int subpixel;            /* 0 or 1 */
    float f, baseline;
} simsense_pair_params_t;

typedef struct simsense_batch* simsense_batch_t;

#define SIMSENSE_BATCH_OPT_GRAPH    1     /* 1 (default): capture/replay a CUDA graph; 0: launch directly */
/*
 * SIMSENSE_BATCH_OPT_TEST_STALL (value 0/1, default 0): a test of the fused
 * launch's bounded waits.  While 1, the task list leaves out the path work of
 * pair 0, so the selection of each of its rows waits for a count that never
 * completes and gives up after its limit (~0.3 s): the launch records
 * SIMSENSE_ERR_TIMEOUT (simsense_batch_device_status), pair 0's depth is
 * undefined, the other pairs are computed as usual and the batch stays
 * usable.  Nothing faults, traps or hangs.
 */
#define SIMSENSE_BATCH_OPT_TEST_STALL 2

/*
 * A batch of n pairs of possibly different sizes, disparity ranges and
 * parameters, computed together (the same four stages as simsense_compute:
 * census and cost one launch per class of pairs with identical parameters,
 * the classes running concurrently, then path aggregation and selection of
 * every pair in one persistent launch, see simsense_batch_schedule_t).
 * Allocates all scratch memory once, on the current device.  Errors as
 * simsense_create.
 */
int simsense_batch_create(simsense_batch_t* out, const simsense_pair_params_t* pairs, int n);

/*
 * Depth of every pair of the batch.  left, right, depth: HOST arrays of n
 * DEVICE pointers (pair i: H_i x W_i uint8 views, H_i x W_i float32 depth).
 * Asynchronous on stream.  The first call records the work into a CUDA graph
 * and later calls with the same pointers replay it (new pointers re-record).
 */
int simsense_batch_compute(simsense_batch_t b, const uint8_t* const* left, const uint8_t* const* right,
                           float* const* depth, struct CUstream_st* stream);

/* Set a batch option (SIMSENSE_BATCH_OPT_*). */
int simsense_batch_set_option(simsense_batch_t b, int opt, int value);

/* Number of classes (groups of pairs with identical parameters). */
int simsense_batch_num_classes(simsense_batch_t b);

/* Parameters and pair count of class c; either pointer may be NULL. */
int simsense_batch_class_info(simsense_batch_t b, int c, simsense_pair_params_t* params, int* npairs);

/*
 * Launch choices of class c: prefetch = pixels of cost in flight per
 * scanline of the path kernel (8, 12 or 16), select_blocks = selection-kernel
 * blocks per SM (1: one block of 1024 threads, 2: two blocks of 512 threads).
 * Results do not depend on them.
 */
int simsense_batch_get_tuning(simsense_batch_t b, int c, int* prefetch, int* select_blocks);
int simsense_batch_set_tuning(simsense_batch_t b, int c, int prefetch, int select_blocks);

/*
 * Schedule of the batch (Sec. VI-D's parallel scheme applied to many pairs):
 *   fused       1 (default): one persistent launch runs the path aggregation
 *               and the selection of every pair of the batch from a task list
 *               (census and cost stay one launch per class); 0: every class
 *               runs its own path and selection launches
 *   prefetch    pixels of cost in flight per scanline in the fused launch (16)
 *   keep_paths  fused: 1 = the path volume is stored with the default L2
 *               policy, so a pair's selection soon after its paths can find
 *               part of it in L2; 0 = streaming stores
 *   lag         fused: the selection rows of the k-th pair (in the order
 *               below) follow the path work of the (k + lag)-th, 1 or 2
 *   order       fused: pairs as given (0), largest first (1), smallest first
 *               (2), by W * H * D
 * Results do not depend on the schedule.  Defaults {1, 16, 1, 1, 1}.
 * simsense_batch_set_schedule returns SIMSENSE_ERR_INVALID_ARG for values
 * outside these sets and waits for the device when the task list changes.
 */
typedef struct simsense_batch_schedule {
    int fused;
    int prefetch;
    int keep_paths;
    int lag;
    int order;
} simsense_batch_schedule_t;

int simsense_batch_get_schedule(simsense_batch_t b, simsense_batch_schedule_t* out);
int simsense_batch_set_schedule(simsense_batch_t b, const simsense_batch_schedule_t* sc);

/*
 * Autotuner: for every class, runs its stages with each candidate launch
 * choice `reps` times (1 .. 100) on the given buffers, timed with CUDA events
 * on `stream`, and keeps the fastest; then times whole batches in the
 * per-class form and in every fused schedule (3 pair orders x 2 lags x 2
 * store policies) and keeps the fastest schedule.  Synchronises the stream.
 */
int simsense_batch_tune(simsense_batch_t b, const uint8_t* const* left, const uint8_t* const* right,
                        float* const* depth, int reps, struct CUstream_st* stream);

/* Device scratch bytes held by the batch. */
size_t simsense_batch_scratch_bytes(simsense_batch_t b);

/* As simsense_device_status, for a batch. */
int simsense_batch_device_status(simsense_batch_t b, struct CUstream_st* stream);

/* CUDA error code behind the batch's last SIMSENSE_ERR_CUDA. */
int simsense_batch_last_cuda_error(simsense_batch_t b);

/* Release the batch and its memory.  NULL is accepted. */
int simsense_batch_destroy(simsense_batch_t b);

/* Static description of a status code. */
const char* simsense_strerror(int code);

/* CUDA error code (cudaError_t) behind the handle's last SIMSENSE_ERR_CUDA. */
int simsense_last_cuda_error(simsense_t h);

/*
 * Test hook for the out-of-memory paths: the nth device allocation the library
 * makes from now on (1 = the next one) fails as if the device were out of
 * memory, and the ones after it succeed again; 0 (or less) disarms it.  The
 * allocations are those of simsense_create (the scratch buffers, in a fixed
 * order: codes left and right, cost volume, path volume, status word, the
 * two input and the depth staging buffers), simsense_set_rectify (map and
 * image of the left view, then of the right) and simsense_batch_create
 * (scratch, status word).  The failing call returns SIMSENSE_ERR_OOM and
 * frees what it had allocated: a create leaves *out NULL, simsense_set_rectify
 * leaves rectification off.  Process-wide; for tests, not for production use.
 */
void simsense_test_fail_allocation(int nth);

#ifdef __cplusplus
}
#endif

#endif /* SIMSENSE_H */
