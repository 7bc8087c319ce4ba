/*
 * lenia.h - C ABI of the GB300 Lenia step library (liblenia.so).
 *
 * The library advances a multi-channel Lenia world with localized genes by
 * one or more steps on one NVIDIA GB300 (sm_103a), following "Towards
 * Large-Scale Simulations of Open-Ended Evolution in Continuous Cellular
 * Automata" (Chan, arXiv 2304.05639):
 *   - phenospace A in R^{c x y x x}, values in [0, 1], toroidal grid (Section 2.1, 2.2);
 *   - genospace P in R^{p x k x y x x} holding per-site growth genes (Section 2.2);
 *   - kernels K_k, normalised K~ = K / (K * 1) (Algorithm 1, note after Algorithm 2),
 *     kernel k reading channel src(k) and writing channel dst(k) (Section 2.1);
 *   - growth mapping and clipped update A_i -> [A_i + dt sum_k G_k(K~_k * A_j)]_0^1
 *     (Section 2.1, Algorithm 2), with dt and the signed growth
 *     2 exp(-(u-m)^2 / 2s^2) - 1 of the original Lenia;
 *   - gene maintenance: genospace diffusion (Section 2.3) and the alpha mask
 *     P -> P (.) alpha, alpha = Delta_all(U) AND Delta_all(P) (Section 2.2).
 *
 * Conventions for every entry point:
 *   - Layout: A is float32 [C][H][W]; P is float32 [n_p][K][H][W] with the
 *     gene planes in the order mu, sigma, h (only the localized ones), then
 *     the kernel genes r1, w1, b1, r2, w2, b2 with LENIA_LOC_KERNEL;
 *     U is float32 [K][H][W].  All contiguous, row-major, x fastest.
 *   - Pointers named *_in / *_out / A / P / U / stats_out are DEVICE pointers
 *     unless the entry point's name ends in _host.  The caller owns them.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Work is enqueued on it and is asynchronous; results are valid after the
 *     stream is synchronised.  A context is not thread-safe.
 *   - The library owns the context and all scratch memory (kernel spectra,
 *     FFT intermediates, potentials, stats partials), allocated in lenia_init
 *     and freed in lenia_destroy.  After lenia_init only lenia_set_walls,
 *     the first lenia_step_evolve and the first host-buffer step allocate
 *     device memory (as documented there), and lenia_measure_fp32_peak
 *     its own small buffer; instantiating the CUDA graphs of lenia_rollout
 *     and lenia_backward lets the driver reserve memory for them;
 *     lenia_stats_noalloc allocates nothing at all.
 *   - Errors: every entry point returns a status; nothing aborts and nothing
 *     is thrown.  Arguments are validated before any launch; a CUDA error
 *     seen after a launch returns LENIA_ECUDA.  lenia_last_error() gives a
 *     one-line description of the last failure on that context.
 */
#ifndef LENIA_H
#define LENIA_H

#include <stdint.h>

#if defined(__GNUC__)
#define LENIA_API __attribute__((visibility("default")))
#else
#define LENIA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lenia_ctx lenia_ctx;

typedef enum {
    LENIA_OK = 0,
    LENIA_EINVAL = 1,    /* invalid argument, shape, or aliasing */
    LENIA_ENOMEM = 2,    /* device or host allocation failed in lenia_init */
    LENIA_ECUDA = 3,     /* a CUDA call or kernel launch failed */
    LENIA_ETIMEOUT = 4,  /* a device-side bounded wait gave up */
    LENIA_ENOTSUP = 5    /* valid request this build does not implement */
} lenia_status;

enum { LENIA_KERNEL_SHELLS = 0, LENIA_KERNEL_BUMPS = 1 };
enum { LENIA_GROWTH_SIGNED = 0, LENIA_GROWTH_PAPER = 1 };
/* LENIA_LOC_KERNEL: ring-wise kernel genes (Section 2.4), six planes r1, w1,
 * b1, r2, w2, b2 after the growth planes; needs n_rings > 0. */
enum { LENIA_LOC_MU = 1, LENIA_LOC_SIGMA = 2, LENIA_LOC_H = 4, LENIA_LOC_KERNEL = 8 };
/* Convolution routes: AUTO picks FFT for power-of-two worlds with R > 6,
 * else DIRECT (FP32 sums).  DIRECT_BF16 and DIRECT_BF16X3 run the direct
 * convolution on the tensor cores as banded Toeplitz products (tcgen05,
 * FP32 accumulation): BF16 operands (8 significant bits: a potential moves
 * by at most (2^-7 + 2^-16) of its value), or both operands split into BF16
 * high and low parts and three products summed (at most about 3 2^-16 of
 * the value); both need H % 256 == 0, W % 32 == 0 and R <= 100, and are not
 * available to lenia_backward. */
enum { LENIA_CONV_AUTO = 0, LENIA_CONV_FFT = 1, LENIA_CONV_DIRECT = 2, LENIA_CONV_DIRECT_BF16 = 3,
       LENIA_CONV_DIRECT_BF16X3 = 4 };

/* One kernel k (Section 2.1: kernels with their growth mappings).
 *   src_channel, dst_channel: the channel convolved and the channel updated.
 *   radius R >= 1 pixels; 2R+1 <= min(H, W).
 *   form LENIA_KERNEL_SHELLS: K(d) = beta[floor(B rho)] core(B rho mod 1),
 *     rho = |d|_2 / R < 1, B = n_shells in 1..4, core(q) = exp(4 - 1/(q(1-q)))
 *     (the original Lenia kernel shell; Section 1.2 cites it).
 *   form LENIA_KERNEL_BUMPS: K(d) = sum_{i=0,1} b_i exp(-(rho - r_i)^2 / (2 w_i^2))
 *     for rho < 1, bump = {r1, w1, b1, r2, w2, b2} (Section 2.1 and 2.4).
 *   h, mu, sigma: global growth genes (used for every gene not localized). */
typedef struct {
    int32_t src_channel;
    int32_t dst_channel;
    int32_t radius;
    int32_t form;
    int32_t n_shells;
    double beta[4];
    double bump[6];
    float h, mu, sigma;
} lenia_kernel_desc;

/* World configuration.
 *   height H, width W: W % 4 == 0, H, W >= 8.  The FFT path needs H and W
 *     powers of two in [64, 4096].
 *   n_channels C in 1..8, n_kernels K in 1..64.
 *   dt: time step multiplying the growth sum (the paper's update is dt = 1).
 *   growth_form: LENIA_GROWTH_SIGNED, h (2g - 1); LENIA_GROWTH_PAPER, h g
 *     (Section 2.4), g = exp(-(u - m)^2 / (2 s^2)) and g = 0 where s <= 0.
 *   localized: OR of LENIA_LOC_* - the genes read per site from P.  P holds
 *     the localized growth genes mu, sigma, h (in that order), then with
 *     LENIA_LOC_KERNEL the kernel genes r1, w1, b1, r2, w2, b2.
 *   maintain_genes: 1 runs diffusion (Section 2.3) and the alpha mask
 *     (Section 2.2); needs localized != 0.
 *   eps_u: alpha threshold on the growth h g (or on U when alpha_on = 1);
 *   eps_p: gene threshold of Delta_same / Delta_all (strict '>').
 *   r_diff: radius of the diffusion disk |d|_2 <= r_diff, 0..8.
 *   conv_path: LENIA_CONV_* (AUTO picks FFT for power-of-two worlds).
 *     The tensor-core routes (LENIA_CONV_DIRECT_BF16, _BF16X3) are chosen only
 *     on request.
 *   max_rollout_steps, ckpt_every: adjoint buffers for lenia_backward (0 = none;
 *     global genes only); states kept every ckpt_every steps (0 -> 8); with
 *     ckpt_every = 1 every state and every step's potentials are kept
 *     (max_rollout_steps x (C + K) planes) and nothing is recomputed.
 *   n_rings: with LENIA_LOC_KERNEL, the ring decomposition of Section 2.4
 *     (0 otherwise): every kernel has the same radius R; ring r holds the
 *     offsets with r <= n_rings |d|_2 / R < r + 1 and |d|_2 < R; at each site
 *     kernel k's potential is sum_r k_r (K_r * A_src) / sum_r k_r (K_r * 1)
 *     with k_r = sum_i b_i exp(-(r / n_rings - r_i)^2 / (2 w_i^2)) from the
 *     site's diffused kernel genes (a term is 0 where w_i <= 0; U = 0 where
 *     the denominator is <= 0).  1 <= n_rings <= 64, n_channels * n_rings <= 256.
 *     The convolution stage then produces the ring potentials K_r * A_c,
 *     [C][n_rings][H][W] (lenia_potentials returns those). */
typedef struct {
    int32_t height, width, n_channels, n_kernels;
    float dt;
    int32_t growth_form;
    int32_t localized;
    int32_t maintain_genes;
    float eps_u, eps_p;
    int32_t r_diff;
    int32_t alpha_on;
    int32_t conv_path;
    int32_t max_rollout_steps, ckpt_every;
    int32_t n_rings;
} lenia_config;

/* Validate cfg and kernels[0..n_kernels), build the normalised kernels in
 * FP64 (Algorithm 1 pre-calculation; Algorithm 2 "pre-calculate kernel"),
 * their FP32 spectra for the FFT path, and all scratch.  Work for the spectra
 * runs on `stream` and is complete when lenia_init returns.  On success *out
 * holds a new context; on failure *out is NULL. */
LENIA_API lenia_status lenia_init(const lenia_config* cfg, const lenia_kernel_desc* kernels,
                        void* stream, lenia_ctx** out);

/* One step (Algorithm 2, diffuse .. update): reads A_in [C][H][W] and, when
 * localized != 0, P_in [n_p][K][H][W]; writes A_out and P_out (P_out may be
 * NULL only when localized == 0).  stats_out (nullable, device, C*3 floats)
 * receives mass, circular-mean centre y and centre x of each channel of
 * A_out.  In and out buffers must not overlap (EINVAL).  One-channel,
 * one-kernel worlds whose width is a multiple of 128 take the tiled update
 * kernel when stats_out is NULL and the streaming one otherwise; the two
 * agree to FP32 rounding, not bit for bit. */
LENIA_API lenia_status lenia_step(lenia_ctx* ctx, const float* A_in, const float* P_in,
                        float* A_out, float* P_out, float* stats_out, void* stream);

/* n_steps steps in place on A (and P): the state ping-pongs through
 * library-owned buffers and ends in the caller's.  stats_out (nullable,
 * device) receives n_steps * C * 3 floats, step s at offset s*C*3.
 * Without stats_out and with n_steps >= 4, pairs of steps replay a CUDA
 * graph that the context captures for its (A, P) pointers and genes (the
 * first such call captures it; calls with other buffers capture again).
 * Small worlds with global genes on the direct route (conv_path
 * LENIA_CONV_DIRECT, no gene maps, H and W multiples of 8, H W <= 128 x 128)
 * instead run a rollout without stats_out of n_steps >= 2 as one cooperative
 * launch: every block keeps an 8 x 8 tile for the whole rollout and the
 * blocks meet at a bounded grid barrier after each step; its results equal
 * repeated lenia_step calls to FP32 rounding (direct sums in the same order,
 * the growth through expf).  The smallest of them (H W <= 8192, W a multiple
 * of 32, H a multiple of 16 or 8, kernel radius <= 16, A 16-byte aligned) run
 * in one thread-block cluster of 16 (or 8) blocks that keep the world in
 * shared memory and meet at the cluster barrier: dense (2R+1)^2 sums in
 * another order, equal to repeated lenia_step calls to FP32 rounding.
 * lenia_rollout_route tells which form a context uses. */
LENIA_API lenia_status lenia_rollout(lenia_ctx* ctx, float* A, float* P, int32_t n_steps,
                           float* stats_out, void* stream);

/* Adjoint of an n_steps rollout from A0 for worlds with global genes
 * (localized == 0; no gene maps, so no alpha decisions).  Needs a context made
 * with max_rollout_steps >= n_steps; states are checkpointed every
 * ckpt_every steps (default 8) and recomputed segment by segment.
 * Given gA_T = dL/dA_T (device, [C][H][W]) it writes gA0 = dL/dA_0 (device,
 * nullable) and g_genes = [K][3] (device, nullable): dL/dmu_k, dL/dsigma_k,
 * dL/dh_k.  Per step (Section 2.1 update, Algorithm 2 growth and clip):
 * clip subgradient 1 iff 0 < pre-clip < 1, growth derivative, and the
 * transposed convolution, which for the point-symmetric K~ is the same
 * convolution.  P0 must be NULL.  Returns LENIA_ENOTSUP when the context has
 * no adjoint buffers or has gene maps.  A0 and gA_T are copied into library
 * buffers first and the results copied out last; the pass between runs as a
 * CUDA graph captured once per (n_steps, genes) and replayed afterwards. */
LENIA_API lenia_status lenia_backward(lenia_ctx* ctx, const float* A0, const float* P0, int32_t n_steps,
                            const float* gA_T, float* gA0, float* g_genes, void* stream);

/* Replace the global growth genes: genes is a HOST array [K][3] of
 * (mu, sigma, h) per kernel (sigma > 0 unless sigma is localized).  The
 * kernels' shapes and spectra are unchanged.  Takes effect for work
 * enqueued after the call (graphs captured with the old genes are redone). */
LENIA_API lenia_status lenia_set_genes(lenia_ctx* ctx, const float* genes);

/* Mass, circular-mean centre y, centre x of each channel of A: out is a
 * device array of C*3 floats.  Sums run in a fixed order (deterministic),
 * block records and their reduction in compensated FP32 pairs (hi + lo),
 * the arctangents in FP64. */
LENIA_API lenia_status lenia_stats(lenia_ctx* ctx, const float* A, float* out, void* stream);

/* Potentials U_k = K~_k * A_src(k) for every kernel (Algorithm 2, convolve
 * and normalised sum; note after Algorithm 2 for the FFT route) into U_out
 * [K][H][W], through the context's convolution path.  With n_rings > 0 the
 * ring potentials K_r * A_c instead, [C][n_rings][H][W] (Section 2.4). */
LENIA_API lenia_status lenia_potentials(lenia_ctx* ctx, const float* A_in, float* U_out, void* stream);

/* The step after the convolution: diffusion, growth, alpha mask, masking and
 * clipped update (Sections 2.2-2.4, Algorithm 2) from given potentials
 * U_in [K][H][W] (ring potentials [C][n_rings][H][W] with n_rings > 0).
 * alpha_out (nullable) receives one byte per site. */
LENIA_API lenia_status lenia_update_from_potentials(lenia_ctx* ctx, const float* A_in, const float* P_in,
                                          const float* U_in, float* A_out, float* P_out,
                                          uint8_t* alpha_out, void* stream);

/* ---- Evolutionary lines of Algorithm 2 (Sections 2.5-2.7).
 * The random choices of one step, drawn by the caller (any generator can drive
 * them, and a step is reproducible from its events):
 *   mutation (Section 2.5): gene plane mut_plane (index among the localized
 *     planes mu, sigma, h in that order; -1 = off), kernel mut_kernel, delta
 *     mut_delta and the periodic square x in [mut_x0 - mut_half, mut_x0 +
 *     mut_half), y likewise: P += gamma_mut * mut_delta there where alpha = 1.
 *   penalisation (Section 2.6): plane pen_plane (-1 = off), kernel pen_kernel
 *     and pen_delta (the caller picks its sign: > 0 on a mu plane, < 0 on a
 *     sigma plane): P += gamma_pen * pen_delta where E_pen > eps_pen and
 *     alpha = 1, with E_oxy = (1 - Delta_sum(U)) * K_oxy, E_pen = (1 - E_oxy)
 *     * K_oxy and K_oxy the disk |d|_2 <= r_oxy (1..32) over its point count.
 *     Delta_sum(U) thresholds the sum over kernels of the per-kernel alpha
 *     test (h_k g_k, or U_k with alpha_on) at eps_u. */
typedef struct {
    int32_t mut_plane, mut_kernel, mut_x0, mut_y0, mut_half;
    double mut_delta, gamma_mut;
    int32_t pen_plane, pen_kernel;
    double pen_delta, gamma_pen, eps_pen;
    int32_t r_oxy;
} lenia_events;

/* Walls (Section 2.7): mask is a HOST array [H][W] of bytes, non-zero at wall
 * sites, or NULL to remove every wall.  Synchronous; the context keeps a
 * device list of the wall sites. */
LENIA_API lenia_status lenia_set_walls(lenia_ctx* ctx, const uint8_t* mask);

/* One step of Algorithm 2 with its evolutionary lines, in its order:
 * (1) the walls zero A and P at their sites IN PLACE (A, P: the current
 * state, device); (2) the step of lenia_step from (A, P) into (A_out, P_out);
 * (3) E_pen from that step's Delta_sum(U); (4) mutation and (5) penalisation
 * of P_out as `ev` (host) describes.  stats_out (C*3 floats), alpha_out
 * ([H][W] bytes) and epen_out ([H][W] floats, E_pen) are nullable device
 * outputs.  Without gene maps both operators must be off.  The first call
 * allocates 4 bytes of scratch per site (synchronously). */
LENIA_API lenia_status lenia_step_evolve(lenia_ctx* ctx, float* A, float* P, float* A_out, float* P_out,
                                         const lenia_events* ev, float* stats_out, uint8_t* alpha_out,
                                         float* epen_out, void* stream);

/* Waits for `stream` and reads the context's device status word: returns
 * LENIA_ETIMEOUT (and clears the word) if a kernel gave up a bounded
 * device-side wait since the last check, else LENIA_OK.  lenia_step_host
 * calls it before returning. */
LENIA_API lenia_status lenia_check(lenia_ctx* ctx, void* stream);

/* Failure-path self-test (no counterpart in the paper): enqueue one block whose
 * mbarrier wait nothing completes, bounded by limit_mcycles million SM clock
 * cycles (1..4000); when the bound runs out it sets the device status word as
 * a streaming kernel would, so the next lenia_check returns LENIA_ETIMEOUT.
 * Nothing faults or traps; the context stays usable. */
LENIA_API lenia_status lenia_selftest_wait_timeout(lenia_ctx* ctx, int32_t limit_mcycles, void* stream);

/* Failure-injection test hook (no counterpart in the paper; for testing the
 * error paths without a GPU fault).  Arms a process-wide countdown over the
 * library's checked CUDA calls: after n_calls further calls succeed, the next
 * one - which itself runs normally - is reported as failed
 * (cudaErrorLaunchOutOfResources), so the entry point in progress returns
 * LENIA_ECUDA with " (injected)" in lenia_last_error; the hook then disarms
 * itself.  n_calls < 0 disarms it.  The device and the context are left
 * consistent: the work enqueued before the reported failure runs, the rest
 * of that call is not enqueued, and later calls work normally (a host-buffer
 * step waits for its copies before returning the error; a rollout whose
 * graph capture fails falls back to direct launches and succeeds). */
LENIA_API lenia_status lenia_debug_fail_after(int32_t n_calls);

/* Measurement helper (no counterpart in the paper): the FP32 throughput of
 * the current device's CUDA cores in TFLOP/s, as the best of five timed
 * launches of independent fused multiply-add chains on every SM, scalar
 * (scalar_tflops) and on packed FP32 pairs (pair_tflops; one packed FMA
 * counts four flops).  It is the denominator of the FP32-pipe fractions the
 * benchmark reports beside the HBM roofline.  Synchronous: it allocates and
 * frees a small device buffer and waits for `stream`.  Both outputs are host
 * pointers and must be non-null (LENIA_EINVAL otherwise). */
LENIA_API lenia_status lenia_measure_fp32_peak(double* scalar_tflops, double* pair_tflops, void* stream);

/* lenia_step with HOST buffers: copies A_in/P_in host->device into library
 * buffers, steps, and copies A_out/P_out (and stats_out, C*3 floats, nullable)
 * back; returns after the copies have finished (lenia_step_host_async
 * followed by lenia_host_wait).  Page-locked host memory makes the copies
 * fast; pageable memory works. */
LENIA_API lenia_status lenia_step_host(lenia_ctx* ctx, const float* A_in, const float* P_in,
                             float* A_out, float* P_out, float* stats_out, void* stream);

/* The same step enqueued without waiting, for independent host worlds in a
 * row (a serving loop).  Alternate calls use two sets of device staging
 * buffers: a call's uploads (on a library stream) wait only until the call
 * before last has finished reading its set, so they run under the previous
 * call's step and downloads; the step runs on `stream`; the downloads run on
 * another library stream.  The first host-buffer step (this or
 * lenia_step_host) allocates the second set, (2 C + 2 n_p K) floats per site
 * (synchronously).  Host buffers must stay valid and unmodified (inputs) /
 * unread (outputs) until lenia_host_wait returns.  Each call's inputs must
 * not be a previous call's pending outputs. */
LENIA_API lenia_status lenia_step_host_async(lenia_ctx* ctx, const float* A_in, const float* P_in,
                                             float* A_out, float* P_out, float* stats_out, void* stream);
/* Waits for every enqueued host step (downloads included), then lenia_check. */
LENIA_API lenia_status lenia_host_wait(lenia_ctx* ctx, void* stream);

/* Per-launch timing for benchmarks.  lenia_profile_start makes the library
 * record a CUDA event pair on the launching stream around each of its next
 * max_launches kernel launches (event creation only; no device memory).
 * lenia_profile_stop waits for those events and fills total_ms[kind] (summed
 * milliseconds) and counts[kind] for the launch kinds 0..LENIA_PROFILE_KINDS-1
 * (names from lenia_profile_kind_name), then turns recording off. */
#define LENIA_PROFILE_KINDS 9
LENIA_API lenia_status lenia_profile_start(lenia_ctx* ctx, int32_t max_launches);
LENIA_API lenia_status lenia_profile_stop(lenia_ctx* ctx, float* total_ms, int32_t* counts);
LENIA_API const char* lenia_profile_kind_name(int32_t kind);

/* lenia_stats without a context and without any allocation (the paper has
 * no counterpart; this is a deployment aid).  Same output as lenia_stats:
 * out (device, C*3 floats) = mass, circular-mean centre y, centre x of each
 * channel of the device array A [C][H][W].
 *
 * For callers that cannot call cudaMalloc: code whose device memory is all
 * owned by another allocator (a framework that reserves the GPU up front,
 * so a raw cudaMalloc fails or fragments its pool), code that must not pay
 * the device-wide synchronisation of cudaMalloc/cudaFree in the middle of
 * its work, and host applications that forbid plug-ins from allocating.
 *
 * Scratch: a file-scope static __device__ array of 2.75 MB inside
 * liblenia.so, held on every GPU that loads the library until the process
 * exits.  Limits: 1 <= C <= 8, 1 <= H, W <= 8192 and
 * ceil(W/32) * ceil(H/32) * C <= 65536 (blocks of 32 x 32 sites times
 * channels; for example 2048 x 2048 with 3 channels, or 8192 x 8192 with
 * one); larger requests return LENIA_EINVAL with a message on stderr before
 * any launch.
 * Each call made outside stream capture looks the array's device address up
 * in the current context (cudaGetSymbolAddress, with that device current; a
 * lookup, no allocation), so a context that was reset (cudaDeviceReset) or
 * replaced since the previous call is handled.  A call whose stream is
 * capturing reuses the address of the device's last lookup: make the first
 * call on each device before any stream capture.  All calls share the one
 * array and it keeps the last call's contents; every value a call reads is
 * written earlier in the same call, so nothing needs clearing.  Calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race on the array: serialise them.  The result equals lenia_stats to
 * rounding, not bit for bit (its sine/cosine tables are computed on the
 * device here and on the host there).  Returns LENIA_ECUDA if a launch
 * fails. */
LENIA_API lenia_status lenia_stats_noalloc(const float* A, int32_t n_channels, int32_t height,
                                           int32_t width, float* out, void* stream);

/* The normalised FP64 kernel k, (2R+1)^2 values row-major over dy, dx in
 * -R..R, copied to the HOST buffer out. */
LENIA_API lenia_status lenia_kernel_weights(const lenia_ctx* ctx, int32_t k, double* out);

/* Convolution path in use: LENIA_CONV_FFT, _DIRECT, _DIRECT_BF16 or _DIRECT_BF16X3. */
LENIA_API int32_t lenia_conv_path(const lenia_ctx* ctx);

/* Form of lenia_rollout (without stats_out, n_steps >= 2) for this context:
 * LENIA_ROUTE_STEPS (launches per step, pairs of steps replayed from a CUDA
 * graph), LENIA_ROUTE_COOPERATIVE (one cooperative launch) or
 * LENIA_ROUTE_CLUSTER (one thread-block cluster; a caller's A that is not
 * 16-byte aligned takes the cooperative launch instead); -1 for NULL. */
#define LENIA_ROUTE_STEPS 0
#define LENIA_ROUTE_COOPERATIVE 1
#define LENIA_ROUTE_CLUSTER 2
LENIA_API int32_t lenia_rollout_route(const lenia_ctx* ctx);

/* Number of CUDA kernel launches one lenia_step enqueues (with stats). */
LENIA_API int32_t lenia_launches_per_step(const lenia_ctx* ctx);

/* ---- Batched worlds (many independent worlds of uneven sizes and genotypes;
 * the scale-out of the paper's Section 1.4 on one GPU; not a construct of the
 * paper itself).
 * lenia_batch_init makes one context per world from cfgs[0..n_worlds) and
 * kernels (world w's n_kernels descriptors follow world w-1's).  With
 * autotune != 0, worlds whose conv_path is AUTO take the FFT path when several
 * worlds share their (size, channels, kernels, genes) - so that they can step
 * as a group, see lenia_batch_group_of - and otherwise the faster of the FFT
 * and direct paths, timed once per distinct (size, channels, kernels, genes,
 * largest radius).  All scratch is allocated here.
 * lenia_batch_rollout advances every world n_steps in place: A and P are HOST
 * arrays of n_worlds DEVICE pointers (P[w] may be NULL for worlds without gene
 * maps; P itself may be NULL if no world has them).  The steps of all worlds
 * are captured once per pointer set into a CUDA graph whose branches run the
 * groups and the remaining worlds concurrently; one graph launch advances
 * every world two steps.  The
 * work is ordered after earlier work on `stream` and before later work.
 * Worlds must not share buffers.  No statistics are computed. */
typedef struct lenia_batch lenia_batch;
LENIA_API lenia_status lenia_batch_init(int32_t n_worlds, const lenia_config* cfgs,
                                        const lenia_kernel_desc* kernels, int32_t autotune,
                                        void* stream, lenia_batch** out);
LENIA_API lenia_status lenia_batch_rollout(lenia_batch* batch, float* const* A, float* const* P,
                                           int32_t n_steps, void* stream);
/* Group of world w (worlds on the FFT path of one size whose configuration and
 * kernel topology are identical - kernel shapes may differ, and global genes
 * that the gene maps replace are ignored - step together:
 * one launch per stage for the whole group, the worlds along the launch's
 * planes or grid z), or -1 when it steps on its own (or w is out of range).
 * A grouped world's epilogue is the tiled kernel (FP32 division and expf),
 * which can differ in the last bits from the streaming kernel a world of
 * width 256 k uses on its own when that kernel is chosen (steps with
 * statistics, several kernels or channels). */
LENIA_API int32_t lenia_batch_group_of(const lenia_batch* batch, int32_t world);
/* Epilogue shape of world w's group: 0 = the tiled kernel, *param = rows per
 * thread (1, 2 or 4); 2 = the tiled kernel with four adjacent columns per
 * thread (float4 loads; one-kernel worlds of width 128 k with 16-byte aligned
 * state buffers), *param = rows per thread (1 or 2); 1 = the streaming kernel
 * in one persistent launch over
 * a device work queue of (world, 256-column chunk, band) items, with every
 * world's tensor maps in device memory, *param = bands per world (widths of
 * 256 k only); -1 when w steps on its own.  With autotune, lenia_batch_rollout
 * times every candidate once per group (on the caller's state, writing only
 * the batch's own buffers) the first time it sees a pointer set, and keeps the
 * fastest.  param may be NULL. */
LENIA_API int32_t lenia_batch_epilogue_shape(const lenia_batch* batch, int32_t world, int32_t* param);
/* Sets the epilogue shape of world w's group (kind and param as above; the
 * autotuner then leaves that group alone).  LENIA_EINVAL for a world without
 * a group or a shape the group cannot take (the streaming kernel before the
 * group's tensor maps exist, i.e. before the first rollout, or for widths not
 * a multiple of 256). */
LENIA_API lenia_status lenia_batch_set_epilogue_shape(lenia_batch* batch, int32_t world, int32_t kind,
                                                      int32_t param);
/* Convolution path chosen for world w (LENIA_CONV_FFT or LENIA_CONV_DIRECT), or -1. */
LENIA_API int32_t lenia_batch_conv_path(const lenia_batch* batch, int32_t world);
/* lenia_check over every world's context after synchronising `stream`. */
LENIA_API lenia_status lenia_batch_check(lenia_batch* batch, void* stream);
LENIA_API void lenia_batch_destroy(lenia_batch* batch);

LENIA_API const char* lenia_last_error(const lenia_ctx* ctx);
LENIA_API const char* lenia_status_string(lenia_status s);
LENIA_API void lenia_destroy(lenia_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LENIA_H */
