// Internal declarations shared by the CUDA translation units of liblenia.
#pragma once
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace lenia {

constexpr int kMaxKernels = 64;
constexpr int kMaxChannels = 8;
constexpr int kMaxPlanes = 9;   // mu, sigma, h, then the ring-wise kernel genes r1, w1, b1, r2, w2, b2
constexpr int kMaxRings = 64;
constexpr int kMaxConvPlanes = 256;   // convolution outputs: kernels, or channels x rings
constexpr int ROW_RMAX = 32;     // largest radix of the row transforms (column transforms: 16)

// Raises kernel Kern's dynamic shared-memory limit to `bytes` the first time a
// launch needs it on the current device; the attribute persists, so later
// launches skip the driver call.
template <auto Kern>
inline cudaError_t smem_limit(size_t bytes)
{
    static std::atomic<int> done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (done[dev].load(std::memory_order_relaxed) >= (int)bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) {
        int cur = done[dev].load();
        while (cur < (int)bytes && !done[dev].compare_exchange_weak(cur, (int)bytes)) {
        }
    }
    return e;
}

// Programmatic dependent launch: the kernels of the step's chain (the FFT
// passes, the direct convolution and the epilogues) are launched with the
// programmatic-serialization attribute, so that the launch of each one is
// prepared while its predecessor in the stream still runs and its blocks
// start as soon as the predecessor's last block exits.  Each of them starts
// with pdl_enter(), which waits until the predecessor has completed and its
// writes are visible, so no block touches global memory before the work it
// depends on is done.  (No kernel signals its dependents early: letting them
// be scheduled once all of a grid's blocks run made the step slower.)
// Launched without the attribute, pdl_enter() returns at once.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Compensated FP32 sums for the statistics' block records and their final
// reduction.  A value is the unevaluated pair hi + lo; each addition keeps
// its rounding error with Knuth's two-sum (exact in round-to-nearest) and
// renormalises, so a fixed-order sum of pairs is deterministic and accurate
// to about 2^-44 of the summed magnitudes, on the FP32 pipe (FP64
// arithmetic runs at a small fraction of the FP32 rate on sm_103).
__device__ __forceinline__ float2 ff_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bv = s - a.x;
    const float e = (a.x - (s - bv)) + (b.x - bv);
    const float t = e + (a.y + b.y);
    const float hi = s + t;
    return make_float2(hi, t - (hi - s));
}

__device__ __forceinline__ float2 ff_shfl_down(float2 v, int off)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off));
}

// One channel's outputs from its five reduced sums tot[c * 5 + (M, S_y,
// C_y, S_x, C_x)]: axis 0 (y) also writes the mass; each axis writes the
// circular-mean centre atan2(S, C) n / (2 pi) wrapped to [0, n), in FP64 on
// the pairs' values.  One thread per (channel, axis), so that the two
// arctangents of a channel run side by side.
__device__ __forceinline__ void stats_centre(const float2* tot, int c, int axis, int H, int W, float* out)
{
    constexpr double kInv2Pi = 0.15915494309189533576888376337251;
    const float2* t = tot + c * 5;
    const int n = axis ? W : H;
    const double s = (double)t[1 + 2 * axis].x + (double)t[1 + 2 * axis].y;
    const double co = (double)t[2 + 2 * axis].x + (double)t[2 + 2 * axis].y;
    double centre = atan2(s, co) * ((double)n * kInv2Pi);
    if (centre < 0.0) centre += n;
    out[c * 3 + 1 + axis] = (float)centre;
    if (axis == 0) out[c * 3] = t[0].x + t[0].y;
}

// Per-kernel scalars, passed by value to the kernels that need them.
struct KernelTable {
    int K, C;
    int src[kMaxKernels], dst[kMaxKernels];
    float h[kMaxKernels], mu[kMaxKernels], sigma[kMaxKernels];
};

// Growth, alpha mask, masking and clipped update (plus stats partials).
struct EpiParams {
    const float* A;
    const float* P;
    const float* U;
    float* A_out;
    float* P_out;
    uint8_t* alpha_out;
    uint8_t* empty_out;        // 1 where sum_k t_k <= eps_u (not Delta_sum(U)), or null
    float2* partials;          // [n_blocks][C][5] compensated (hi, lo) sums, or null
    float* stats_out;          // [C][3]; when set, the last block reduces the partials (streaming kernel)
    unsigned int* ticket;      // completion counter for that reduction (0 between launches)
    const float* sin_y;
    const float* cos_y;
    const float* sin_x;
    const float* cos_x;
    int H, W, n_p;
    int p_mu, p_sigma, p_h;    // plane index of each localized gene or -1
    int maintain, growth_form, alpha_on, r_diff;
    float dt, eps_u, eps_p;
    // growth sum of channel c at sites where alpha = 0 (genes masked to zero):
    // -sum_{dst(k)=c} h_k for the signed form with global h, else 0
    float acc0[kMaxChannels];
    // worlds batched in one launch (tiled epilogue only): world blockIdx.z reads
    // A_list / P_list and writes Aout_list / Pout_list, its potentials at
    // U + world * u_stride (null lists: a single world at A, P, A_out, P_out)
    const float* const* A_list;
    const float* const* P_list;
    float* const* Aout_list;
    float* const* Pout_list;
    size_t u_stride;
    // ring decomposition (Section 2.4): U holds the ring potentials
    // [C][n_rings][H][W]; the kernel genes start at plane p_kern
    int n_rings, p_kern;
    float ring_cnt[kMaxRings];  // K_r * 1 (pixels per ring)
    float ring_x[kMaxRings];    // r / n_rings, where the kernel function is evaluated
    KernelTable kt;
};

// Walls, penalising area, mutation and penalisation (Sections 2.5-2.7).
constexpr int kMaxROxy = 32;
struct EvoParams {
    const uint8_t* empty;      // [H][W] 1 where Delta_sum(U) is false
    const uint8_t* alpha;      // [H][W] alpha mask of the step
    float* P;                  // P' [n_p K][H][W], updated in place
    float* epen_out;           // [H][W] E_pen or null
    int H, W, r_oxy, n_disk;
    double n_disk2;            // n_disk^2
    int half_width[kMaxROxy + 1];   // largest w with w^2 + dy^2 <= r^2, per |dy|
    int mut_plane, pen_plane;  // plane p K + k, or -1 (operator off)
    int mut_x0, mut_y0, mut_half;
    float mut_add, pen_add;    // gamma delta, rounded once from FP64
    long long pen_thresh;      // penalise where M > pen_thresh
};

// Direct periodic convolution of every kernel.
struct ConvParams {
    const float* A;
    float* U;
    const float* w;            // dense FP32 kernels, transposed [dx][dy], back to back
    const int* w_off;          // offset of kernel k in w
    const int* yr;             // per kernel, per dx: largest |dy| with a non-zero tap (-1: none)
    const int* yr_off;         // offset of kernel k in yr
    int H, W, C, K;
    int R[kMaxConvPlanes];
    int kcount[kMaxChannels];
    int klist[kMaxChannels][kMaxKernels];
    int* status;               // device status word (bounded TMA waits)
    int tma;                   // set by the launcher: interior tiles staged by TMA
};

// Direct convolution on the tensor cores (conv_tc.cu): BF16 Toeplitz blocks,
// FP32 accumulation in tensor memory.
constexpr int TC_NT = 32;       // output columns per block
constexpr int TC_NG = 4;        // kernels per block (its accumulators: 2 x TC_NG x TC_NT TMEM columns)
struct TcConvParams {
    uint16_t* Ap_hi;            // [C][Hp][Wp] BF16 padded copy of A (periodic halo of R)
    uint16_t* Ap_lo;            // low parts A - hi (TERMS = 3) or null
    const unsigned char* B;     // Toeplitz blocks [plane][dy + R][KP / 8][TC_NT][8] BF16 (high parts)
    size_t B_lo_off;            // byte offset of the low parts
    const int2* ks;             // [plane][dy + R]: first and last K step (16 columns) with a non-zero tap
    const int* grp;             // per block z: channel, kernel count, up to TC_NG kernels
    const int* has_taps;        // [plane]: 0 for a kernel without any non-zero tap
    float* U;
    int* status;
    int H, W, C, R, Hp, Wp, KP, rows_pad, n_dy, n_groups, terms;
};
bool tc_conv_supported(int H, int W, int max_R);
size_t tc_block_bytes_host(int kp);
cudaError_t launch_conv_tc(const TcConvParams& p, const float* A, cudaStream_t s);

// Rollouts of small worlds with global genes in one cooperative launch
// (small_rollout.cu); tap tables as in ConvParams.
struct SmallRolloutParams {
    float* A;                  // [C][H][W], in and out
    float* buf;                // second state
    const int2* taps;          // non-zero taps of every kernel: ((dy + 1024) 2048 + dx + 1024, weight bits)
    int tap_off[kMaxKernels + 1];   // kernel k's taps: tap_off[k] .. tap_off[k + 1] - 1
    int n_taps;
    KernelTable kt;
    int H, W, C, maxR, growth_form, n_steps;
    float dt;
    unsigned* count;           // grid barrier counter (zeroed by the launcher)
    int* status;
};
// Rollouts of small worlds with global genes in one thread-block cluster
// (the world in the blocks' shared memory).
struct ClusterRolloutParams {
    float* A;                  // [C][H][W], in and out (16-byte aligned)
    const float* w;            // dense kernels [K][2 maxR + 1][2 maxR + 1] (row dy, column dx), zero-padded
    KernelTable kt;
    int H, W, C, maxR, growth_form, n_steps;
    int Q;                     // blocks in the cluster (16 or 8)
    float dt;
};
// Blocks of the cluster the world can run on (16 or 8), or 0 if it cannot.
int cluster_rollout_blocks(int H, int W, int C, int K, int maxR);
// true when the dense [K][2 maxR + 1]^2 weights are zero wherever the
// cluster rollout skips them (outside the disk |d| < maxR, row group by row group)
bool cluster_rollout_weights_fit(const float* w, int K, int maxR);
size_t cluster_rollout_smem(int H, int W, int C, int K, int maxR, int Q);
cudaError_t launch_cluster_rollout(const ClusterRolloutParams& p, cudaStream_t s);

size_t small_rollout_smem(int C, int maxR, int n_taps);
bool small_rollout_supported(int H, int W, int C, int K, int maxR, int n_taps);
cudaError_t launch_small_rollout(const SmallRolloutParams& p, cudaStream_t s);

// Spectral (FFT) convolution.
struct FftParams {
    const float* A;            // [C][H][W]
    float2* Ahat;              // [C][M][H] row spectra, column-major, M = W/2, kx = 0 packs (DC, Nyquist)
    float2* Uhat;              // [K][M][H] per-kernel column-inverse spectra, same layout and packing
    float* U;                  // [K][H][W] potentials
    const float* S;            // [K][M+1][H/2+1] real kernel spectra / (H W)
    const float2* tw_M;        // per-pass twiddle tables of the length-M row transforms
    const float2* tw_W;        // exp(-2 pi i m / W), m <= M  (real-signal packing)
    const float2* tw_H;        // per-pass twiddle tables of the length-H column transforms
    int H, W, C, K;
    int k_base;                // the column pass writes Uhat plane k - k_base (0 for the forward step)
    const float* add;          // inverse row pass: added to its output, same layout as U (nullable)
    int* status;               // device status word for bounded waits (nullable)
    // worlds batched in one launch (identical shapes and kernels): plane y of the
    // row pass is channel y % cw of world y / cw, read from A_list[world] when
    // A_list is set; the column pass writes Uhat plane world * kpw + k.  A
    // single world has cw = C and any kpw.
    const float* const* A_list;
    const float* const* S_list;  // per-world kernel spectra (world = plane / cw), else S
    int cw, kpw;
    int list_aligned;          // every A_list pointer is 16-byte aligned
    int kcount[kMaxChannels];
    int klist[kMaxChannels][kMaxKernels];
};

// Adjoint of one step with global genes.
struct AdjParams {
    const float* A;            // step input A_t [C][H][W]
    const float* U;            // potentials of A_t [K][H][W]
    const float* gA_next;      // dL/dA_{t+1} [C][H][W]
    float* gpre;               // clip-masked dL/dA_{t+1} [C][H][W]
    float* gU;                 // dL/dU [K][H][W]
    const float* V;            // K~_k (x) gU_k [K][H][W], or summed per source channel [C][H][W]
    int v_per_channel;         // 1: V holds sum_{src(k) = c} K~_k (x) gU_k per channel c
    float* gA_out;             // dL/dA_t [C][H][W]
    float2* gene_partials;     // [K][3][blocks], compensated (hi, lo) sums
    float2* gene_acc;          // [K][3]: d/dmu, d/dsigma, d/dh, compensated (hi, lo) sums
    int H, W, growth_form;
    float dt;
    KernelTable kt;
};

// Launchers (return the cudaError_t of the launch).
cudaError_t launch_direct_conv(const ConvParams& p, int max_R, cudaStream_t s);
cudaError_t launch_fft_rows_r2c(const FftParams& p, cudaStream_t s);
cudaError_t launch_fft_cols(const FftParams& p, cudaStream_t s);
// transposed column pass: Uhat plane c = inv( sum_{k in klist[c]} S_k fwd(Ahat plane k) ), grid (M, C)
cudaError_t launch_fft_cols_adj(const FftParams& p, cudaStream_t s);
cudaError_t launch_fft_rows_c2r(const FftParams& p, cudaStream_t s);
cudaError_t launch_epilogue(const EpiParams& p, cudaStream_t s, int* n_blocks);
cudaError_t launch_stats_partials(const float* A, int C, int H, int W, const float* sin_y,
                                  const float* cos_y, const float* sin_x, const float* cos_x,
                                  float2* partials, cudaStream_t s, int* n_blocks);
cudaError_t launch_stats_final(const float2* partials, int n_blocks, int C, int H, int W,
                               float* out, cudaStream_t s);
cudaError_t launch_spectra(const double* Kd, int R, int H, int W, const double* cos_H,
                           const double* cos_W, double* T_scratch, float* S_out, cudaStream_t s);
cudaError_t launch_selftest_wait(long long limit_cycles, int* status, cudaStream_t s);
int adjoint_blocks(int H, int W);
cudaError_t launch_adjoint_epilogue(const AdjParams& p, cudaStream_t s);
cudaError_t measure_fp32_peak(cudaStream_t s, double* scalar_tflops, double* pair_tflops);
cudaError_t launch_adjoint_gather(const AdjParams& p, cudaStream_t s);
cudaError_t launch_adjoint_gene_out(const float2* gene_acc, int nv, float* out, cudaStream_t s);
bool epilogue_rows_supported(const EpiParams& p);
// The streaming epilogue over the worlds of a batched group (one persistent
// launch; work items taken from a device queue): one world's tensor maps and
// outputs, in device memory.
struct QueueWorld {             // aligned as CUtensorMap
    CUtensorMap tm_p, tm_u, tm_a, tm_h;
    float* A_out;
    float* P_out;
};
// p: the group's shared parameters (shape, genes, thresholds); single-channel
// single-kernel worlds of width 256 k with r_diff 1.
bool epilogue_queue_supported(const EpiParams& p);
bool epilogue_queue_world(QueueWorld* out, const EpiParams& p, const float* A, const float* P, const float* U,
                          float* A_out, float* P_out);
// n_bands bands per world; ctas_per_sm 0 = as many as fit.  `counter` (one
// int of device memory) is zeroed on `s` before the launch.
cudaError_t launch_epilogue_queue(const EpiParams& p, const QueueWorld* worlds, int n_worlds, int n_bands,
                                  int ctas_per_sm, int* counter, int* status, cudaStream_t s);
// cuTensorMapEncodeTiled through the runtime's driver entry point (null if
// the driver does not provide it).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
cudaError_t launch_epilogue_rows(const EpiParams& p, int num_sms, int* status, cudaStream_t s, int* n_blocks);
bool fft_size_supported(int H, int W);
int epilogue_blocks(int H, int W);
// The batched-worlds runner's view of a context: its convolution and epilogue
// parameters (false unless the context is on the FFT path).
struct lenia_ctx_view {
    FftParams fp;
    EpiParams ep;
    size_t N;
    int C, K;
};
}  // namespace lenia
struct lenia_ctx;
namespace lenia {
bool ctx_view(lenia_ctx* c, lenia_ctx_view* v);
// batched worlds: one tiled-epilogue launch over n_worlds (grid z), pointer lists in EpiParams
bool epilogue_batch_supported(const EpiParams& p);
// br: rows per thread of the one-kernel tiled epilogue (1, 2 or 4)
cudaError_t launch_epilogue_batch(const EpiParams& p, int n_worlds, cudaStream_t s, int br = 2);
int ring_epilogue_blocks(int H, int W);   // stats records of the ring epilogue
// pass 1: Delta_sum complement -> counts; pass 2: E_pen, mutation, penalisation
// both passes in one launch (counts kept in shared memory)
cudaError_t launch_disk_fused(const EvoParams& p, cudaStream_t s);
cudaError_t launch_walls_zero(const int* idx, int n, float* A, int C, float* P, int npk, size_t N,
                              cudaStream_t s);

}  // namespace lenia
