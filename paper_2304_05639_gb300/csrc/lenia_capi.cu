// C ABI of liblenia (declared in include/lenia.h): validation, the FP64
// kernel builder, scratch allocation, and the per-step launch sequence.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <array>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lenia.h"
#include "lenia_internal.cuh"

using namespace lenia;

struct lenia_ctx {
    lenia_config cfg;
    std::vector<lenia_kernel_desc> kd;
    std::vector<std::vector<double>> kw;   // normalised FP64 kernels, row-major dy, dx
    // what the convolution stage computes: the kernels, or (ring decomposition)
    // one binary ring mask per (channel, ring), plane c * n_rings + r
    std::vector<std::vector<double>> conv_w;
    std::vector<int> conv_src, conv_R;
    std::vector<double> ring_cnt;          // K_r * 1 per ring
    int path = LENIA_CONV_DIRECT;
    int n_p = 0, p_mu = -1, p_sigma = -1, p_h = -1, p_kern = -1;
    int max_R = 0;
    size_t N = 0;                          // sites
    // device scratch (library-owned)
    float* d_w = nullptr;
    int* d_w_off = nullptr;
    // small worlds with global genes: rollouts in one cooperative launch
    bool small = false;
    unsigned* d_small_count = nullptr;
    int2* d_small_taps = nullptr;
    std::vector<int> small_tap_off;
    // the smallest of them: rollouts in one thread-block cluster (cr_Q blocks)
    int cr_Q = 0;
    float* d_cr_w = nullptr;
    // tensor-core route (LENIA_CONV_DIRECT_BF16 / _BF16X3)
    uint16_t* d_tc_hi = nullptr;
    uint16_t* d_tc_lo = nullptr;
    unsigned char* d_tc_B = nullptr;
    int2* d_tc_ks = nullptr;
    int* d_tc_grp = nullptr;
    int* d_tc_has = nullptr;
    TcConvParams tp;
    int* d_yr = nullptr;
    int* d_yr_off = nullptr;
    float* d_S = nullptr;
    float2* d_twM = nullptr;
    float2* d_twW = nullptr;
    float2* d_twH = nullptr;
    float2* d_Ahat = nullptr;
    float2* d_Uhat = nullptr;
    float* d_U = nullptr;
    float2* d_partials = nullptr;
    float* d_trig = nullptr;               // sin_y, cos_y, sin_x, cos_x
    float* d_A2 = nullptr;
    float* d_P2 = nullptr;
    float* d_A3 = nullptr;
    float* d_P3 = nullptr;
    float* d_stats = nullptr;
    int* d_status = nullptr;               // device status word (bounded-wait failures)
    unsigned int* d_ticket = nullptr;      // last-block ticket of the fused stats reduction
    int num_sms = 0;
    int n_part_blocks = 0;
    ConvParams cp;
    FftParams fp;
    KernelTable kt;
    std::string err;
    // adjoint (lenia_backward): checkpoints, segment states, gradients
    bool adj = false;
    int ckpt = 0, max_steps = 0;
    float* d_ckpt = nullptr;               // [n_ckpt][C][H][W]
    float* d_seg = nullptr;                // [max(ckpt, 2)][C][H][W]
    float* d_Useg = nullptr;               // [ckpt][K][H][W] potentials of the segment's states
    float* d_gA[2] = {nullptr, nullptr};
    float* d_gpre = nullptr;
    float* d_gU = nullptr;
    float* d_V = nullptr;
    float2* d_gene_part = nullptr;    // compensated FP32 (hi, lo) pairs
    float2* d_gene_acc = nullptr;
    float2* d_Ahat_t = nullptr;            // spectra of the K gradient planes (transposed conv)
    float2* d_Uhat_t = nullptr;
    // evolutionary operators (lenia_set_walls, lenia_step_evolve)
    int* d_walls = nullptr;                // wall site indices
    int n_walls = 0;
    uint8_t* d_alpha_e = nullptr;          // [H][W] alpha of the evolving step
    uint8_t* d_empty = nullptr;            // [H][W] not Delta_sum(U)
    // host-buffer steps (lenia_step_host[_async]): a stream for gene uploads and
    // one for downloads, and the events that order them against the compute
    // host-buffer pipeline (lenia_step_host_async): two staging sets used by
    // alternate steps; set 0 is d_A2/d_P2 (in) and d_A3/d_P3 (out), set 1 is
    // allocated on first use
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr}, ev_down[2] = {nullptr, nullptr};
    float *d_hA_in1 = nullptr, *d_hP_in1 = nullptr, *d_hA_out1 = nullptr, *d_hP_out1 = nullptr;
    float* d_hstats = nullptr;             // [2][C][3]
    int host_set = 0;                      // staging set of the next host step
    bool host_pending = false;             // a download has been enqueued since the last wait
    // optional per-launch timing (lenia_profile_start / lenia_profile_stop)
    bool prof = false;
    // rollouts and backward passes as CUDA graphs, captured on a private
    // stream and replayed while the call's arguments and the genes are
    // unchanged (kernel parameters carry the genes and the pointers)
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        std::array<uintptr_t, 7> key{};
    };
    cudaStream_t cap_stream = nullptr;
    GraphSlot g_rollout, g_backward;
    uint64_t genes_version = 0;            // bumped by lenia_set_genes
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    size_t ev_used = 0;
};

// names of the launch kinds the profiler distinguishes
static const char* kKindNames[] = {"rows_r2c", "cols_conv", "rows_c2r", "direct_conv", "epilogue",
                                   "stats_partials", "stats_final", "walls", "pen_disk"};
enum { KIND_R2C, KIND_COLS, KIND_C2R, KIND_DIRECT, KIND_EPI, KIND_STATS_P, KIND_STATS_F, KIND_WALLS,
       KIND_PEN, KIND_COUNT };
static_assert(KIND_COUNT == LENIA_PROFILE_KINDS, "profile kinds and the header disagree");
static_assert(sizeof(kKindNames) / sizeof(kKindNames[0]) == KIND_COUNT, "one name per profile kind");

namespace {

const double kTwoPi = 6.283185307179586476925286766559;

lenia_status fail(lenia_ctx* c, lenia_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

// Failure injection (lenia_debug_fail_after, a test hook): while armed, a
// countdown of checked CUDA calls; the call that takes it below zero is
// reported as failed (cudaErrorLaunchOutOfResources) after it has run, and
// the hook disarms itself.
std::atomic<int> g_fail_after{-1};

cudaError_t checked(cudaError_t e, bool* injected)
{
    *injected = false;
    int v = g_fail_after.load(std::memory_order_relaxed);
    while (v >= 0 && !g_fail_after.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) {
    }
    if (v != 0 || e != cudaSuccess) return e;
    *injected = true;
    return cudaErrorLaunchOutOfResources;
}

#define CUDA_OR_FAIL(ctx, call)                                                      \
    do {                                                                             \
        bool inj_ = false;                                                           \
        cudaError_t e_ = checked((call), &inj_);                                     \
        if (e_ != cudaSuccess)                                                       \
            return fail(ctx, LENIA_ECUDA,                                            \
                        std::string(#call) + ": " + cudaGetErrorString(e_) + (inj_ ? " (injected)" : "")); \
    } while (0)

// Kernel shell of the original Lenia: beta[floor(B rho)] core(B rho mod 1),
// core(q) = exp(4 - 1/(q (1 - q))); or the paper's two-bump kernel function.
double kernel_at(const lenia_kernel_desc& k, int dy, int dx)
{
    const double rho = sqrt((double)(dy * dy + dx * dx)) / (double)k.radius;
    if (!(rho < 1.0)) return 0.0;
    if (k.form == LENIA_KERNEL_SHELLS) {
        const double br = rho * k.n_shells;
        const double fl = floor(br);
        const double q = br - fl;
        const double core = (q > 0.0 && q < 1.0) ? exp(4.0 - 1.0 / (q * (1.0 - q))) : 0.0;
        return k.beta[(int)fl] * core;
    }
    double v = 0.0;
    for (int b = 0; b < 2; b++) {
        const double d = rho - k.bump[3 * b];
        const double w = k.bump[3 * b + 1];
        v += k.bump[3 * b + 2] * exp(-d * d / (2.0 * w * w));
    }
    return v;
}

bool build_kernel(const lenia_kernel_desc& k, std::vector<double>& out)
{
    const int R = k.radius, n = 2 * R + 1;
    out.assign((size_t)n * n, 0.0);
    double total = 0.0;
    for (int dy = -R; dy <= R; dy++)
        for (int dx = -R; dx <= R; dx++) {
            const double v = kernel_at(k, dy, dx);
            out[(size_t)(dy + R) * n + (dx + R)] = v;
            total += v;
        }
    if (!(total > 0.0) || !isfinite(total)) return false;
    for (double& v : out) v /= total;
    return true;
}

lenia_status validate(const lenia_config* c, const lenia_kernel_desc* ks, std::string& why)
{
    auto bad = [&](const char* m) { why = m; return LENIA_EINVAL; };
    if (!c || !ks) return bad("null config or kernels");
    if (c->height < 8 || c->width < 8) return bad("height and width must be >= 8");
    if (c->width % 4) return bad("width must be a multiple of 4");
    if ((long long)c->height * c->width > (1LL << 30)) return bad("world larger than 2^30 sites");
    if (c->n_channels < 1 || c->n_channels > kMaxChannels) return bad("n_channels must be 1..8");
    if (c->n_kernels < 1 || c->n_kernels > kMaxKernels) return bad("n_kernels must be 1..64");
    if (!isfinite(c->dt) || c->dt < 0.f) return bad("dt must be finite and >= 0");
    if (c->growth_form != LENIA_GROWTH_SIGNED && c->growth_form != LENIA_GROWTH_PAPER)
        return bad("unknown growth_form");
    if (c->localized & ~15) return bad("localized has unknown bits");
    if ((c->localized & LENIA_LOC_KERNEL) != 0) {
        if (c->n_rings < 1 || c->n_rings > kMaxRings) return bad("n_rings must be 1..64 with LENIA_LOC_KERNEL");
        if (c->n_channels * c->n_rings > kMaxConvPlanes) return bad("n_channels * n_rings must be <= 256");
        for (int k = 1; k < c->n_kernels; k++)
            if (ks[k].radius != ks[0].radius) return bad("the ring decomposition needs one radius for every kernel");
    } else if (c->n_rings != 0) {
        return bad("n_rings needs LENIA_LOC_KERNEL");
    }
    if (c->maintain_genes != 0 && c->maintain_genes != 1) return bad("maintain_genes must be 0 or 1");
    if (c->maintain_genes && !c->localized) return bad("maintain_genes needs localized genes");
    if (c->r_diff < 0 || c->r_diff > 8 || 2 * c->r_diff + 1 > c->height || 2 * c->r_diff + 1 > c->width)
        return bad("r_diff must be 0..8 and 2 r_diff + 1 <= min(H, W)");
    if (!isfinite(c->eps_u) || !isfinite(c->eps_p)) return bad("eps must be finite");
    if (c->alpha_on != 0 && c->alpha_on != 1) return bad("alpha_on must be 0 or 1");
    if (c->conv_path < LENIA_CONV_AUTO || c->conv_path > LENIA_CONV_DIRECT_BF16X3) return bad("unknown conv_path");
    if ((c->conv_path == LENIA_CONV_DIRECT_BF16 || c->conv_path == LENIA_CONV_DIRECT_BF16X3) &&
        c->max_rollout_steps > 0)
        return bad("the adjoint needs the FFT or the FP32 direct path");
    if (c->conv_path == LENIA_CONV_FFT && !fft_size_supported(c->height, c->width))
        return bad("FFT path needs H and W powers of two in [64, 4096]");
    for (int k = 0; k < c->n_kernels; k++) {
        const lenia_kernel_desc& d = ks[k];
        if (d.src_channel < 0 || d.src_channel >= c->n_channels || d.dst_channel < 0 ||
            d.dst_channel >= c->n_channels)
            return bad("kernel channel index out of range");
        if (d.radius < 1 || 2 * d.radius + 1 > c->height || 2 * d.radius + 1 > c->width)
            return bad("kernel radius must be >= 1 and 2R + 1 <= min(H, W)");
        if (d.radius > 64) return bad("kernel radius must be <= 64");
        if (d.form == LENIA_KERNEL_SHELLS) {
            if (d.n_shells < 1 || d.n_shells > 4) return bad("n_shells must be 1..4");
            for (int i = 0; i < d.n_shells; i++)
                if (!isfinite(d.beta[i])) return bad("beta must be finite");
        } else if (d.form == LENIA_KERNEL_BUMPS) {
            for (int i = 0; i < 6; i++)
                if (!isfinite(d.bump[i])) return bad("bump parameters must be finite");
            if (!(d.bump[1] > 0.0) || !(d.bump[4] > 0.0)) return bad("bump widths must be > 0");
        } else {
            return bad("unknown kernel form");
        }
        if (!isfinite(d.h) || !isfinite(d.mu) || !isfinite(d.sigma)) return bad("genes must be finite");
        if (!(c->localized & LENIA_LOC_SIGMA) && !(d.sigma > 0.f)) return bad("global sigma must be > 0");
    }
    return LENIA_OK;
}

bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb)
{
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    return pa < pb + nb && pb < pa + na;
}

// BF16 bit pattern of x rounded to nearest, ties to even (the upper 16 bits
// of the FP32 pattern after adding half an ulp of BF16; NaN kept quiet), and
// the value of a BF16 bit pattern.
uint16_t bf16_bits(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7FFFFFFFu) > 0x7F800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

template <class T>
lenia_status dalloc(lenia_ctx* c, T** p, size_t n)
{
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(c, LENIA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return LENIA_OK;
}

// Per-pass Stockham twiddle tables of a length-n transform (passes of radix
// rmax while at least rmax remains, then the rest), each laid out [r - 1][k]:
// exp(-2 pi i r k / (Ns R)), computed in FP64 and rounded once.
std::vector<float2> pass_twiddles(int n, int rmax)
{
    std::vector<float2> t;
    for (int ns = 1; ns < n;) {
        const int R = n / ns >= rmax ? rmax : n / ns;
        if (ns > 1)
            for (int r = 1; r < R; r++)
                for (int k = 0; k < ns; k++) {
                    const double a = kTwoPi * (double)r * k / ((double)ns * R);
                    t.push_back(make_float2((float)cos(a), (float)-sin(a)));
                }
        ns *= R;
    }
    if (t.empty()) t.push_back(make_float2(1.f, 0.f));
    return t;
}

std::vector<float2> twiddles(int n, int count)
{
    std::vector<float2> t((size_t)count);
    for (int m = 0; m < count; m++) {
        const double a = kTwoPi * (double)m / (double)n;
        t[m] = make_float2((float)cos(a), (float)-sin(a));
    }
    return t;
}

// Records an event pair around each launch while profiling is on.
struct ProfScope {
    lenia_ctx* c;
    cudaStream_t s;
    bool on;
    ProfScope(lenia_ctx* c_, int kind, cudaStream_t s_) : c(c_), s(s_), on(false)
    {
        nvtxRangePushA(kKindNames[kind]);        // named range per launch kind (no-op without a tool)
        if (c->prof && c->ev_used + 2 <= c->ev.size()) {
            on = true;
            c->ev_kind[c->ev_used / 2] = kind;
            cudaEventRecord(c->ev[c->ev_used], s);
        }
    }
    ~ProfScope()
    {
        nvtxRangePop();
        if (on) {
            cudaEventRecord(c->ev[c->ev_used + 1], s);
            c->ev_used += 2;
        }
    }
};

lenia_status potentials(lenia_ctx* c, const float* A, float* U, cudaStream_t s)
{
    if (c->path == LENIA_CONV_FFT) {
        FftParams fp = c->fp;
        fp.A = A;
        fp.U = U;
        {
            ProfScope ps(c, KIND_R2C, s);
            CUDA_OR_FAIL(c, launch_fft_rows_r2c(fp, s));
        }
        {
            ProfScope ps(c, KIND_COLS, s);
            CUDA_OR_FAIL(c, launch_fft_cols(fp, s));
        }
        {
            ProfScope ps(c, KIND_C2R, s);
            CUDA_OR_FAIL(c, launch_fft_rows_c2r(fp, s));
        }
    } else if (c->path == LENIA_CONV_DIRECT_BF16 || c->path == LENIA_CONV_DIRECT_BF16X3) {
        TcConvParams tp = c->tp;
        tp.U = U;
        ProfScope ps(c, KIND_DIRECT, s);
        CUDA_OR_FAIL(c, launch_conv_tc(tp, A, s));
    } else {
        ConvParams cp = c->cp;
        cp.A = A;
        cp.U = U;
        ProfScope ps(c, KIND_DIRECT, s);
        CUDA_OR_FAIL(c, launch_direct_conv(cp, c->max_R, s));
    }
    return LENIA_OK;
}

EpiParams epi_params(lenia_ctx* c)
{
    EpiParams ep;
    memset(&ep, 0, sizeof(ep));
    ep.sin_y = c->d_trig;
    ep.cos_y = c->d_trig + c->cfg.height;
    ep.sin_x = c->d_trig + 2 * c->cfg.height;
    ep.cos_x = c->d_trig + 2 * c->cfg.height + c->cfg.width;
    ep.H = c->cfg.height;
    ep.W = c->cfg.width;
    ep.n_p = c->n_p;
    ep.p_mu = c->p_mu;
    ep.p_sigma = c->p_sigma;
    ep.p_h = c->p_h;
    ep.maintain = c->cfg.maintain_genes;
    ep.growth_form = c->cfg.growth_form;
    ep.alpha_on = c->cfg.alpha_on;
    ep.r_diff = c->cfg.r_diff;
    ep.dt = c->cfg.dt;
    ep.eps_u = c->cfg.eps_u;
    ep.eps_p = c->cfg.eps_p;
    ep.kt = c->kt;
    ep.n_rings = c->cfg.n_rings;
    ep.p_kern = c->p_kern;
    for (int r = 0; r < c->cfg.n_rings; r++) {
        ep.ring_cnt[r] = (float)c->ring_cnt[r];
        ep.ring_x[r] = (float)((double)r / (double)c->cfg.n_rings);
    }
    for (int ch = 0; ch < c->cfg.n_channels; ch++) {
        float a0 = 0.f;
        if (c->cfg.growth_form == LENIA_GROWTH_SIGNED && c->p_h < 0)
            for (int k = 0; k < c->cfg.n_kernels; k++)
                if (c->kd[k].dst_channel == ch) a0 -= c->kd[k].h;   // h (2*0 - 1), in kernel order
        ep.acc0[ch] = a0;
    }
    return ep;
}

lenia_status check_state_args(lenia_ctx* c, const float* A_in, const float* P_in, const float* A_out,
                              const float* P_out)
{
    if (!c) return LENIA_EINVAL;
    const size_t abytes = c->N * c->cfg.n_channels * sizeof(float);
    const size_t pbytes = c->N * c->n_p * c->cfg.n_kernels * sizeof(float);
    if (!A_in || !A_out) return fail(c, LENIA_EINVAL, "A_in and A_out must be non-null");
    if (c->n_p && (!P_in || !P_out)) return fail(c, LENIA_EINVAL, "P_in and P_out are required with localized genes");
    if (ranges_overlap(A_in, abytes, A_out, abytes)) return fail(c, LENIA_EINVAL, "A_in and A_out overlap");
    if (c->n_p) {
        if (ranges_overlap(P_in, pbytes, P_out, pbytes)) return fail(c, LENIA_EINVAL, "P_in and P_out overlap");
        if (ranges_overlap(A_out, abytes, P_out, pbytes) || ranges_overlap(A_out, abytes, P_in, pbytes) ||
            ranges_overlap(A_in, abytes, P_out, pbytes))
            return fail(c, LENIA_EINVAL, "A and P buffers overlap");
    }
    return LENIA_OK;
}

lenia_status step_impl(lenia_ctx* c, const float* A_in, const float* P_in, float* A_out, float* P_out,
                       float* stats_out, uint8_t* alpha_out, const float* U_given, cudaStream_t s,
                       uint8_t* empty_out = nullptr)
{
    if (!U_given) {
        lenia_status st = potentials(c, A_in, c->d_U, s);
        if (st != LENIA_OK) return st;
    }
    EpiParams ep = epi_params(c);
    ep.A = A_in;
    ep.P = P_in;
    ep.U = U_given ? U_given : c->d_U;
    ep.A_out = A_out;
    ep.P_out = c->n_p ? P_out : nullptr;
    ep.alpha_out = alpha_out;
    ep.empty_out = empty_out;
    ep.partials = stats_out ? c->d_partials : nullptr;
    int nb = 0;
    bool fused_stats = false;
    {
        ProfScope ps(c, KIND_EPI, s);
        const bool aligned = ((uintptr_t)ep.A % 16 == 0) && ((uintptr_t)ep.U % 16 == 0) &&
                             (!ep.P || (uintptr_t)ep.P % 16 == 0);
        // one-kernel worlds without statistics: the tiled kernel with four
        // columns per thread (float4 rows; 1024^2: 21.5 against 25.6 us per
        // step with the streaming kernel, whose pipelines are short here)
        const bool aligned_out = ((uintptr_t)ep.A_out % 16 == 0) && (!ep.P_out || (uintptr_t)ep.P_out % 16 == 0);
        if (!stats_out && !alpha_out && !empty_out && ep.kt.K == 1 && ep.kt.C == 1 && ep.W % 128 == 0 &&
            ep.H % 8 == 0 && epilogue_batch_supported(ep) && aligned && aligned_out) {
            CUDA_OR_FAIL(c, launch_epilogue_batch(ep, 1, s, -1));
        } else if (aligned && epilogue_rows_supported(ep)) {
            ep.stats_out = stats_out;        // reduced by the kernel's last block
            ep.ticket = c->d_ticket;
            fused_stats = stats_out != nullptr;
            CUDA_OR_FAIL(c, launch_epilogue_rows(ep, c->num_sms, c->d_status, s, &nb));
        } else {
            CUDA_OR_FAIL(c, launch_epilogue(ep, s, &nb));
        }
    }
    if (stats_out && !fused_stats) {
        ProfScope ps(c, KIND_STATS_F, s);
        CUDA_OR_FAIL(c, launch_stats_final(c->d_partials, nb, c->cfg.n_channels, c->cfg.height,
                                           c->cfg.width, stats_out, s));
    }
    return LENIA_OK;
}

// The transpose of the convolution stage (the kernels are point symmetric, so
// each kernel's transpose is the same convolution).  FFT path: per source
// channel c, V_c = sum_{k: src(k) = c} K~_k (x) gU_k, summed in the frequency
// domain (forward transforms of the K gradient planes, one inverse transform
// per channel); returns true in *per_channel, and with `out` writes
// out_c = add_c + V_c instead of V.  Direct path: V_k for every kernel, in
// groups of at most kMaxChannels kernels treated as channels.
lenia_status transposed_conv(lenia_ctx* c, const float* gU, float* V, cudaStream_t s, bool* per_channel,
                             const float* add = nullptr, float* out = nullptr)
{
    const int K = c->cfg.n_kernels;
    if (c->path == LENIA_CONV_FFT) {
        FftParams fp = c->fp;
        fp.A = gU;
        fp.U = out ? out : V;          // with out: out_c = add_c + V_c in the inverse row pass
        fp.add = out ? add : nullptr;
        fp.Ahat = c->d_Ahat_t;        // K planes
        fp.Uhat = c->d_Uhat_t;        // C planes
        fp.C = K;                      // the row pass transforms every gradient plane
        CUDA_OR_FAIL(c, launch_fft_rows_r2c(fp, s));
        fp.C = c->cfg.n_channels;      // one column block row per source channel
        CUDA_OR_FAIL(c, launch_fft_cols_adj(fp, s));
        fp.K = c->cfg.n_channels;      // inverse row pass of the C summed planes
        CUDA_OR_FAIL(c, launch_fft_rows_c2r(fp, s));
        *per_channel = true;
        return LENIA_OK;
    }
    for (int k0 = 0; k0 < K; k0 += kMaxChannels) {
        const int g = std::min(kMaxChannels, K - k0);
        ConvParams cp = c->cp;
        cp.A = gU + (size_t)k0 * c->N;
        cp.U = V;   // kernel k writes plane k
        cp.C = g;
        for (int j = 0; j < kMaxChannels; j++) cp.kcount[j] = 0;
        for (int j = 0; j < g; j++) {
            cp.kcount[j] = 1;
            cp.klist[j][0] = k0 + j;
        }
        CUDA_OR_FAIL(c, launch_direct_conv(cp, c->max_R, s));
    }
    *per_channel = false;
    return LENIA_OK;
}

}  // namespace

namespace lenia {
// For the batched-worlds runner (lenia_batch.cu): the parameters one step of
// this context launches with; false unless it is on the FFT path.
bool ctx_view(lenia_ctx* c, lenia_ctx_view* v)
{
    if (!c || !v || c->path != LENIA_CONV_FFT) return false;
    v->fp = c->fp;
    v->ep = epi_params(c);
    v->N = c->N;
    v->C = c->cfg.n_channels;
    v->K = (int)c->conv_w.size();
    return true;
}
}  // namespace lenia

extern "C" {

const char* lenia_status_string(lenia_status s)
{
    switch (s) {
        case LENIA_OK: return "ok";
        case LENIA_EINVAL: return "invalid argument";
        case LENIA_ENOMEM: return "out of memory";
        case LENIA_ECUDA: return "CUDA error";
        case LENIA_ETIMEOUT: return "device wait timed out";
        case LENIA_ENOTSUP: return "not supported";
    }
    return "unknown status";
}

lenia_status lenia_debug_fail_after(int32_t n_calls)
{
    g_fail_after.store(n_calls < 0 ? -1 : n_calls, std::memory_order_relaxed);
    return LENIA_OK;
}

const char* lenia_last_error(const lenia_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int32_t lenia_conv_path(const lenia_ctx* ctx) { return ctx ? ctx->path : -1; }

int32_t lenia_rollout_route(const lenia_ctx* ctx)
{
    if (!ctx) return -1;
    return ctx->cr_Q ? LENIA_ROUTE_CLUSTER : (ctx->small ? LENIA_ROUTE_COOPERATIVE : LENIA_ROUTE_STEPS);
}

int32_t lenia_launches_per_step(const lenia_ctx* ctx)
{
    if (!ctx) return -1;
    EpiParams ep = epi_params(const_cast<lenia_ctx*>(ctx));
    const bool fused = epilogue_rows_supported(ep);   // stats reduced inside the epilogue
    const int conv = ctx->path == LENIA_CONV_FFT ? 3 : (ctx->path == LENIA_CONV_DIRECT ? 1 : 2);
    return conv + (fused ? 1 : 2);
}

void lenia_destroy(lenia_ctx* c)
{
    if (!c) return;
    void* ptrs[] = {c->d_w, c->d_w_off, c->d_yr, c->d_yr_off, c->d_S, c->d_twM, c->d_twW, c->d_twH,
                    c->d_Ahat, c->d_Uhat, c->d_U, c->d_partials, c->d_trig, c->d_A2, c->d_P2,
                    c->d_A3, c->d_P3, c->d_stats, c->d_status, c->d_ckpt, c->d_seg, c->d_gA[0],
                    c->d_gA[1], c->d_gpre, c->d_gU, c->d_V, c->d_gene_part, c->d_gene_acc,
                    c->d_Ahat_t, c->d_Uhat_t, c->d_ticket, c->d_walls, c->d_alpha_e, c->d_empty,
                    c->d_Useg, c->d_hA_in1, c->d_hP_in1, c->d_hA_out1,
                    c->d_hP_out1, c->d_hstats, c->d_tc_hi, c->d_tc_lo, c->d_tc_B, c->d_tc_ks,
                    c->d_tc_grp, c->d_tc_has, c->d_small_count, c->d_small_taps, c->d_cr_w};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (int b = 0; b < 2; b++)
        for (cudaEvent_t e : {c->ev_up[b], c->ev_done[b], c->ev_down[b]})
            if (e) cudaEventDestroy(e);
    for (cudaGraphExec_t g : {c->g_rollout.exec, c->g_backward.exec})
        if (g) cudaGraphExecDestroy(g);
    for (cudaStream_t t : {c->up_stream, c->down_stream, c->cap_stream})
        if (t) cudaStreamDestroy(t);
    delete c;
}

lenia_status lenia_init(const lenia_config* cfg, const lenia_kernel_desc* kernels, void* stream,
                        lenia_ctx** out)
{
    if (!out) return LENIA_EINVAL;
    *out = nullptr;
    std::string why;
    lenia_status st = validate(cfg, kernels, why);
    if (st != LENIA_OK) {
        fprintf(stderr, "lenia_init: %s\n", why.c_str());
        return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    lenia_ctx* c = new lenia_ctx();
    c->cfg = *cfg;
    c->kd.assign(kernels, kernels + cfg->n_kernels);
    const int H = cfg->height, W = cfg->width, C = cfg->n_channels, K = cfg->n_kernels;
    c->N = (size_t)H * W;
    const int loc = cfg->localized;
    c->n_p = ((loc & LENIA_LOC_MU) != 0) + ((loc & LENIA_LOC_SIGMA) != 0) + ((loc & LENIA_LOC_H) != 0);
    c->p_mu = (loc & LENIA_LOC_MU) ? 0 : -1;
    c->p_sigma = (loc & LENIA_LOC_SIGMA) ? ((loc & LENIA_LOC_MU) ? 1 : 0) : -1;
    c->p_h = (loc & LENIA_LOC_H) ? c->n_p - 1 : -1;
    if (loc & LENIA_LOC_KERNEL) {
        c->p_kern = c->n_p;
        c->n_p += 6;
    }
    const int n_rings = cfg->n_rings;

    // kernels in FP64, normalised to sum 1 (with rings the kernels are made per
    // site from the ring masks instead)
    c->kw.resize(K);
    for (int k = 0; k < K; k++) {
        if (!n_rings && !build_kernel(c->kd[k], c->kw[k])) {
            lenia_destroy(c);
            fprintf(stderr, "lenia_init: kernel %d sums to zero\n", k);
            return LENIA_EINVAL;
        }
        c->max_R = std::max(c->max_R, c->kd[k].radius);
    }
    if (n_rings) {
        // ring r holds the offsets with r <= n |d| / R < r + 1, |d| < R, decided in
        // integers: the largest m with m^2 R^2 <= n^2 |d|^2
        const int R = c->kd[0].radius, nw = 2 * R + 1;
        c->conv_w.assign((size_t)C * n_rings, std::vector<double>((size_t)nw * nw, 0.0));
        c->ring_cnt.assign(n_rings, 0.0);
        for (int dy = -R; dy <= R; dy++)
            for (int dx = -R; dx <= R; dx++) {
                const long long q = (long long)dy * dy + (long long)dx * dx;
                if (q >= (long long)R * R) continue;
                int m = 0;
                while ((long long)(m + 1) * (m + 1) * R * R <= (long long)n_rings * n_rings * q) m++;
                c->ring_cnt[m] += 1.0;
                for (int ch = 0; ch < C; ch++) c->conv_w[(size_t)ch * n_rings + m][(size_t)(dy + R) * nw + (dx + R)] = 1.0;
            }
        for (int ch = 0; ch < C; ch++)
            for (int r = 0; r < n_rings; r++) {
                c->conv_src.push_back(ch);
                c->conv_R.push_back(R);
            }
    } else {
        c->conv_w = c->kw;
        for (int k = 0; k < K; k++) {
            c->conv_src.push_back(c->kd[k].src_channel);
            c->conv_R.push_back(c->kd[k].radius);
        }
    }
    const int NC = (int)c->conv_w.size();      // convolution output planes
    memset(&c->kt, 0, sizeof(c->kt));
    c->kt.K = K;
    c->kt.C = C;
    for (int k = 0; k < K; k++) {
        c->kt.src[k] = c->kd[k].src_channel;
        c->kt.dst[k] = c->kd[k].dst_channel;
        c->kt.h[k] = c->kd[k].h;
        c->kt.mu[k] = c->kd[k].mu;
        c->kt.sigma[k] = c->kd[k].sigma;
    }

    // path choice: spectral for power-of-two worlds unless the kernels are small
    int path = cfg->conv_path;
    if (path == LENIA_CONV_AUTO)
        path = (fft_size_supported(H, W) && c->max_R > 6) ? LENIA_CONV_FFT : LENIA_CONV_DIRECT;
    if (path == LENIA_CONV_DIRECT && (size_t)(38 + 2 * c->max_R) * (32 + 2 * c->max_R) * 4 + 128 > 200 * 1024) {
        lenia_destroy(c);
        fprintf(stderr, "lenia_init: radius too large for the direct path\n");
        return LENIA_EINVAL;
    }
    const bool tc = path == LENIA_CONV_DIRECT_BF16 || path == LENIA_CONV_DIRECT_BF16X3;
    if (tc && !tc_conv_supported(H, W, c->max_R)) {
        lenia_destroy(c);
        fprintf(stderr, "lenia_init: the tensor-core path needs H %% 256 == 0, W %% 32 == 0 and R <= 100\n");
        return LENIA_EINVAL;
    }
    c->path = path;

#define ALLOC(ptr, n)                                  \
    do {                                               \
        lenia_status a_ = dalloc(c, &(ptr), (n));      \
        if (a_ != LENIA_OK) {                          \
            fprintf(stderr, "lenia_init: %s\n", c->err.c_str()); \
            lenia_destroy(c);                          \
            return a_;                                 \
        }                                              \
    } while (0)
#define CK_INIT(call)                                                         \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            fprintf(stderr, "lenia_init: %s: %s\n", #call, cudaGetErrorString(e_)); \
            lenia_destroy(c);                                                 \
            return LENIA_ECUDA;                                               \
        }                                                                     \
    } while (0)

    const size_t nA = c->N * C, nP = c->N * c->n_p * K;
    ALLOC(c->d_U, c->N * NC);
    ALLOC(c->d_A2, nA);
    ALLOC(c->d_A3, nA);
    if (nP) {
        ALLOC(c->d_P2, nP);
        ALLOC(c->d_P3, nP);
    }
    ALLOC(c->d_stats, (size_t)C * 3);
    ALLOC(c->d_status, 1);
    CK_INIT(cudaMemset(c->d_status, 0, sizeof(int)));
    ALLOC(c->d_ticket, 1);
    CK_INIT(cudaMemset(c->d_ticket, 0, sizeof(unsigned int)));
    {
        int dev = 0;
        CK_INIT(cudaGetDevice(&dev));
        CK_INIT(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // stats records: the larger of the tiled epilogue's blocks and one per SM-resident CTA
    c->n_part_blocks = std::max(std::max(epilogue_blocks(H, W), ring_epilogue_blocks(H, W)), 8 * c->num_sms);
    ALLOC(c->d_partials, (size_t)c->n_part_blocks * C * 5);

    // circular-mean tables
    {
        std::vector<float> trig(2 * (size_t)H + 2 * (size_t)W);
        for (int y = 0; y < H; y++) {
            trig[y] = (float)sin(kTwoPi * y / H);
            trig[H + y] = (float)cos(kTwoPi * y / H);
        }
        for (int x = 0; x < W; x++) {
            trig[2 * H + x] = (float)sin(kTwoPi * x / W);
            trig[2 * H + W + x] = (float)cos(kTwoPi * x / W);
        }
        ALLOC(c->d_trig, trig.size());
        CK_INIT(cudaMemcpy(c->d_trig, trig.data(), trig.size() * sizeof(float), cudaMemcpyHostToDevice));
    }

    // per-channel lists of the convolution planes each channel feeds
    int kcount[kMaxChannels] = {0};
    int klist[kMaxChannels][kMaxKernels];
    for (int k = 0; k < NC; k++) {
        const int sc = c->conv_src[k];
        klist[sc][kcount[sc]++] = k;
    }

    // small worlds with global genes on the direct route: their rollouts run
    // as one cooperative launch over every kernel's non-zero taps (in the
    // direct route's order: tap columns dx, then rows dy)
    if (c->n_p == 0 && !cfg->maintain_genes && c->cfg.n_rings == 0 && cfg->conv_path == LENIA_CONV_DIRECT &&
        NC == K) {
        std::vector<int2> taps;
        c->small_tap_off.assign(1, 0);
        for (int k = 0; k < NC; k++) {
            const int R = c->conv_R[k], n = 2 * R + 1;
            for (int dx = -R; dx <= R; dx++)
                for (int dy = -R; dy <= R; dy++) {
                    const double v = c->conv_w[k][(size_t)(dy + R) * n + (dx + R)];
                    if (v == 0.0) continue;
                    const float f = (float)v;
                    int bits;
                    memcpy(&bits, &f, 4);
                    taps.push_back(make_int2((dy + 1024) * 2048 + (dx + 1024), bits));
                }
            c->small_tap_off.push_back((int)taps.size());
        }
        c->small = small_rollout_supported(H, W, C, NC, c->max_R, (int)taps.size());
        if (c->small) {
            ALLOC(c->d_small_count, 1);
            ALLOC(c->d_small_taps, taps.size());
            CK_INIT(cudaMemcpy(c->d_small_taps, taps.data(), taps.size() * sizeof(int2), cudaMemcpyHostToDevice));
        }
        // dense (2 maxR + 1)^2 kernels, each centred, for the cluster rollout
        c->cr_Q = cluster_rollout_blocks(H, W, C, NC, c->max_R);
        if (c->cr_Q) {
            const int KW = 2 * c->max_R + 1;
            std::vector<float> dense((size_t)NC * KW * KW, 0.f);
            for (int k = 0; k < NC; k++) {
                const int R = c->conv_R[k], n = 2 * R + 1, o = c->max_R - R;
                for (int dy = 0; dy < n; dy++)
                    for (int dx = 0; dx < n; dx++)
                        dense[((size_t)k * KW + dy + o) * KW + dx + o] = (float)c->conv_w[k][(size_t)dy * n + dx];
            }
            if (cluster_rollout_weights_fit(dense.data(), NC, c->max_R)) {
                ALLOC(c->d_cr_w, dense.size());
                CK_INIT(cudaMemcpy(c->d_cr_w, dense.data(), dense.size() * sizeof(float), cudaMemcpyHostToDevice));
            } else {
                c->cr_Q = 0;
            }
        }
    }
    if (path == LENIA_CONV_DIRECT) {
        std::vector<float> w;
        std::vector<int> woff(NC), yr, yroff(NC);
        for (int k = 0; k < NC; k++) {
            const int R = c->conv_R[k], n = 2 * R + 1;
            woff[k] = (int)w.size();
            yroff[k] = (int)yr.size();
            for (int dx = -R; dx <= R; dx++) {
                int r = -1;
                for (int dy = -R; dy <= R; dy++) {
                    const double v = c->conv_w[k][(size_t)(dy + R) * n + (dx + R)];
                    w.push_back((float)v);
                    if (v != 0.0) r = std::max(r, std::abs(dy));
                }
                yr.push_back(r);
            }
        }
        ALLOC(c->d_w, w.size());
        ALLOC(c->d_w_off, (size_t)NC);
        ALLOC(c->d_yr, yr.size());
        ALLOC(c->d_yr_off, (size_t)NC);
        CK_INIT(cudaMemcpy(c->d_w, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_w_off, woff.data(), NC * sizeof(int), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_yr, yr.data(), yr.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_yr_off, yroff.data(), NC * sizeof(int), cudaMemcpyHostToDevice));
        memset(&c->cp, 0, sizeof(c->cp));
        c->cp.w = c->d_w;
        c->cp.w_off = c->d_w_off;
        c->cp.yr = c->d_yr;
        c->cp.yr_off = c->d_yr_off;
        c->cp.H = H;
        c->cp.W = W;
        c->cp.C = C;
        c->cp.K = NC;
        c->cp.status = c->d_status;
        for (int k = 0; k < NC; k++) c->cp.R[k] = c->conv_R[k];
        memcpy(c->cp.kcount, kcount, sizeof(kcount));
        memcpy(c->cp.klist, klist, sizeof(klist));
    }
    if (tc) {
        // Toeplitz blocks of every plane and row offset dy (BF16 high and low
        // parts), K-step ranges, and the blocks' kernel groups
        const int Rm = c->max_R, nt = TC_NT, n_dy = 2 * Rm + 1;
        const int kp = (nt + 2 * Rm + 15) / 16 * 16;
        const size_t blk = tc_block_bytes_host(kp);              // bytes of one block
        const size_t n_el = blk / 2;
        std::vector<uint16_t> Bt(2 * (size_t)NC * n_dy * n_el, 0);
        std::vector<int2> ksr((size_t)NC * n_dy);
        std::vector<int> has(NC, 0);
        const size_t lo_off = (size_t)NC * n_dy * n_el;
        for (int k = 0; k < NC; k++) {
            const int Rk = c->conv_R[k], nk = 2 * Rk + 1;
            for (int dyi = 0; dyi < n_dy; dyi++) {
                const int dy = dyi - Rm;
                int dmin = 1 << 30, dmax = -(1 << 30);
                if (std::abs(dy) <= Rk)
                    for (int dx = -Rk; dx <= Rk; dx++)
                        if (c->conv_w[k][(size_t)(dy + Rk) * nk + (dx + Rk)] != 0.0) {
                            dmin = std::min(dmin, dx);
                            dmax = std::max(dmax, dx);
                        }
                if (dmax < dmin) {
                    ksr[(size_t)k * n_dy + dyi] = make_int2(1, 0);
                    continue;
                }
                has[k] = 1;
                ksr[(size_t)k * n_dy + dyi] = make_int2((dmin + Rm) / 16, (dmax + Rm + nt - 1) / 16);
                uint16_t* bh = Bt.data() + ((size_t)k * n_dy + dyi) * n_el;
                uint16_t* bl = bh + lo_off;
                for (int kc = 0; kc < kp / 8; kc++)
                    for (int x = 0; x < nt; x++)
                        for (int e8 = 0; e8 < 8; e8++) {
                            const int dx = 8 * kc + e8 - x - Rm;
                            if (std::abs(dx) > Rk) continue;
                            const double w = c->conv_w[k][(size_t)(dy + Rk) * nk + (dx + Rk)];
                            const size_t o = ((size_t)kc * nt + x) * 8 + e8;
                            bh[o] = bf16_bits((float)w);
                            bl[o] = bf16_bits((float)(w - (double)bf16_value(bh[o])));
                        }
            }
        }
        std::vector<int> grp;
        for (int ch = 0; ch < C; ch++)
            for (int t0 = 0; t0 < kcount[ch]; t0 += TC_NG) {
                const int n = std::min(TC_NG, kcount[ch] - t0);
                grp.push_back(ch);
                grp.push_back(n);
                for (int t = 0; t < TC_NG; t++) grp.push_back(t < n ? klist[ch][t0 + t] : 0);
            }
        const int Hp = H + 2 * Rm, Wp = (W + 2 * Rm + 7) / 8 * 8;
        ALLOC(c->d_tc_hi, (size_t)C * Hp * Wp);
        if (path == LENIA_CONV_DIRECT_BF16X3) ALLOC(c->d_tc_lo, (size_t)C * Hp * Wp);
        ALLOC(c->d_tc_B, Bt.size() * 2);
        ALLOC(c->d_tc_ks, ksr.size());
        ALLOC(c->d_tc_grp, grp.size());
        ALLOC(c->d_tc_has, has.size());
        CK_INIT(cudaMemcpy(c->d_tc_B, Bt.data(), Bt.size() * 2, cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_tc_ks, ksr.data(), ksr.size() * sizeof(int2), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_tc_grp, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_tc_has, has.data(), has.size() * sizeof(int), cudaMemcpyHostToDevice));
        memset(&c->tp, 0, sizeof(c->tp));
        c->tp.Ap_hi = c->d_tc_hi;
        c->tp.Ap_lo = c->d_tc_lo;
        c->tp.B = c->d_tc_B;
        c->tp.B_lo_off = lo_off * 2;
        c->tp.ks = c->d_tc_ks;
        c->tp.grp = c->d_tc_grp;
        c->tp.has_taps = c->d_tc_has;
        c->tp.status = c->d_status;
        c->tp.H = H;
        c->tp.W = W;
        c->tp.C = C;
        c->tp.R = Rm;
        c->tp.Hp = Hp;
        c->tp.Wp = Wp;
        c->tp.KP = kp;
        c->tp.rows_pad = (256 + 2 * Rm + 15) / 16 * 16;
        c->tp.n_dy = n_dy;
        c->tp.n_groups = (int)grp.size() / (2 + TC_NG);
        c->tp.terms = path == LENIA_CONV_DIRECT_BF16X3 ? 3 : 1;
    } else if (path == LENIA_CONV_FFT) {
        const int M = W / 2, HS = H / 2 + 1;
        ALLOC(c->d_Ahat, (size_t)C * H * M);
        ALLOC(c->d_Uhat, (size_t)NC * H * M);
        ALLOC(c->d_S, (size_t)NC * (M + 1) * HS);
        std::vector<float2> twM = pass_twiddles(M, ROW_RMAX), twW = twiddles(W, M + 1), twH = pass_twiddles(H, 16);
        ALLOC(c->d_twM, twM.size());
        ALLOC(c->d_twW, twW.size());
        ALLOC(c->d_twH, twH.size());
        CK_INIT(cudaMemcpy(c->d_twM, twM.data(), twM.size() * sizeof(float2), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_twW, twW.data(), twW.size() * sizeof(float2), cudaMemcpyHostToDevice));
        CK_INIT(cudaMemcpy(c->d_twH, twH.data(), twH.size() * sizeof(float2), cudaMemcpyHostToDevice));
        // FP64 spectra of every kernel on the device, rounded once to FP32
        std::vector<double> cosH(H), cosW(W);
        for (int m = 0; m < H; m++) cosH[m] = cos(kTwoPi * m / H);
        for (int m = 0; m < W; m++) cosW[m] = cos(kTwoPi * m / W);
        double *d_cosH = nullptr, *d_cosW = nullptr, *d_Kd = nullptr, *d_T = nullptr;
        const size_t kmax = (size_t)(2 * c->max_R + 1) * (2 * c->max_R + 1);
        bool ok = cudaMalloc(&d_cosH, H * sizeof(double)) == cudaSuccess &&
                  cudaMalloc(&d_cosW, W * sizeof(double)) == cudaSuccess &&
                  cudaMalloc(&d_Kd, kmax * sizeof(double)) == cudaSuccess &&
                  cudaMalloc(&d_T, (size_t)(2 * c->max_R + 1) * (M + 1) * sizeof(double)) == cudaSuccess;
        cudaError_t e = ok ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemcpy(d_cosH, cosH.data(), H * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_cosW, cosW.data(), W * sizeof(double), cudaMemcpyHostToDevice);
        for (int k = 0; k < NC && e == cudaSuccess; k++) {
            e = cudaMemcpyAsync(d_Kd, c->conv_w[k].data(), c->conv_w[k].size() * sizeof(double),
                                cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess)
                e = launch_spectra(d_Kd, c->conv_R[k], H, W, d_cosH, d_cosW, d_T,
                                   c->d_S + (size_t)k * (M + 1) * HS, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        cudaFree(d_cosH);
        cudaFree(d_cosW);
        cudaFree(d_Kd);
        cudaFree(d_T);
        CK_INIT(e);
        memset(&c->fp, 0, sizeof(c->fp));
        c->fp.Ahat = c->d_Ahat;
        c->fp.Uhat = c->d_Uhat;
        c->fp.S = c->d_S;
        c->fp.tw_M = c->d_twM;
        c->fp.tw_W = c->d_twW;
        c->fp.tw_H = c->d_twH;
        c->fp.H = H;
        c->fp.W = W;
        c->fp.C = C;
        c->fp.K = NC;
        c->fp.status = c->d_status;
        c->fp.cw = C;
        c->fp.kpw = NC;
        memcpy(c->fp.kcount, kcount, sizeof(kcount));
        memcpy(c->fp.klist, klist, sizeof(klist));
    }
    // adjoint buffers (global genes only; gene maps make alpha decisions)
    if (cfg->max_rollout_steps > 0 && c->n_p == 0 && !cfg->maintain_genes) {
        c->adj = true;
        c->max_steps = cfg->max_rollout_steps;
        c->ckpt = cfg->ckpt_every > 0 ? cfg->ckpt_every : 8;
        const int n_ckpt = (c->max_steps + c->ckpt - 1) / c->ckpt;
        const size_t nA1 = c->N * C;
        ALLOC(c->d_ckpt, (size_t)n_ckpt * nA1);
        ALLOC(c->d_seg, (size_t)std::max(c->ckpt, 2) * nA1);
        // every state kept (ckpt_every = 1): the forward pass also keeps every
        // step's potentials, so the reverse pass recomputes nothing
        ALLOC(c->d_Useg, (size_t)(c->ckpt == 1 ? c->max_steps : c->ckpt) * K * c->N);
        ALLOC(c->d_gA[0], nA1);
        ALLOC(c->d_gA[1], nA1);
        ALLOC(c->d_gpre, nA1);
        ALLOC(c->d_gU, c->N * K);
        ALLOC(c->d_V, c->N * K);
        ALLOC(c->d_gene_part, (size_t)adjoint_blocks(H, W) * K * 3);
        ALLOC(c->d_gene_acc, (size_t)K * 3);
        if (path == LENIA_CONV_FFT) {
            ALLOC(c->d_Ahat_t, (size_t)K * (W / 2) * H);     // spectra of the K gradient planes
            ALLOC(c->d_Uhat_t, (size_t)C * (W / 2) * H);     // their per-channel sums
        }
    }
    CK_INIT(cudaStreamSynchronize(s));
    CK_INIT(cudaGetLastError());
#undef ALLOC
#undef CK_INIT
    *out = c;
    return LENIA_OK;
}

lenia_status lenia_step(lenia_ctx* c, const float* A_in, const float* P_in, float* A_out, float* P_out,
                        float* stats_out, void* stream)
{
    lenia_status st = check_state_args(c, A_in, P_in, A_out, P_out);
    if (st != LENIA_OK) return st;
    return step_impl(c, A_in, P_in, A_out, P_out, stats_out, nullptr, nullptr, (cudaStream_t)stream);
}

// Runs body(stream) as a CUDA graph: captured once on the private stream for
// a key (the call's arguments and the genes version), then launched on s.
// Capturing enqueues nothing.  While per-launch profiling is on, or if a
// capture fails, body runs directly on s.
extern "C++" {
template <class Body>
static lenia_status run_graph(lenia_ctx* c, lenia_ctx::GraphSlot& slot, const std::array<uintptr_t, 7>& key,
                              cudaStream_t s, Body body)
{
    if (c->prof) return body(s);
    if (!(slot.exec && slot.key == key)) {
        if (slot.exec) {
            cudaGraphExecDestroy(slot.exec);
            slot.exec = nullptr;
        }
        if (!c->cap_stream) CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const lenia_status st = body(c->cap_stream);
            ok = cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && st == LENIA_OK && g;
            if (ok) ok = cudaGraphInstantiate(&slot.exec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
        }
        if (!ok) {
            slot.exec = nullptr;
            (void)cudaGetLastError();
            c->err.clear();
            return body(s);
        }
        slot.key = key;
    }
    CUDA_OR_FAIL(c, cudaGraphLaunch(slot.exec, s));
    return LENIA_OK;
}
}  // extern "C++"

static lenia_status rollout_body(lenia_ctx* c, float* A, float* P, int32_t n_steps, float* stats_out, cudaStream_t s)
{
    const size_t stride = (size_t)c->cfg.n_channels * 3;
    for (int t = 0; t < n_steps; t++) {
        const bool even = (t % 2) == 0;
        const float* Ai = even ? A : c->d_A2;
        const float* Pi = even ? P : c->d_P2;
        float* Ao = even ? c->d_A2 : A;
        float* Po = even ? c->d_P2 : P;
        lenia_status st = step_impl(c, Ai, c->n_p ? Pi : nullptr, Ao, c->n_p ? Po : nullptr,
                                    stats_out ? stats_out + t * stride : nullptr, nullptr, nullptr, s);
        if (st != LENIA_OK) return st;
    }
    if (n_steps % 2) {
        CUDA_OR_FAIL(c, cudaMemcpyAsync(A, c->d_A2, c->N * c->cfg.n_channels * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s));
        if (c->n_p)
            CUDA_OR_FAIL(c, cudaMemcpyAsync(P, c->d_P2, c->N * c->n_p * c->cfg.n_kernels * sizeof(float),
                                            cudaMemcpyDeviceToDevice, s));
    }
    return LENIA_OK;
}

lenia_status lenia_rollout(lenia_ctx* c, float* A, float* P, int32_t n_steps, float* stats_out, void* stream)
{
    if (!c) return LENIA_EINVAL;
    if (n_steps < 0) return fail(c, LENIA_EINVAL, "n_steps must be >= 0");
    if (!A || (c->n_p && !P)) return fail(c, LENIA_EINVAL, "A (and P with localized genes) must be non-null");
    if (n_steps == 0) return LENIA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->cr_Q && !stats_out && n_steps >= 2 && ((uintptr_t)A & 15) == 0) {
        // the whole rollout in one thread-block cluster (the smallest worlds)
        ClusterRolloutParams cp;
        memset(&cp, 0, sizeof(cp));
        cp.A = A;
        cp.w = c->d_cr_w;
        cp.kt = c->kt;
        cp.H = c->cfg.height;
        cp.W = c->cfg.width;
        cp.C = c->cfg.n_channels;
        cp.maxR = c->max_R;
        cp.growth_form = c->cfg.growth_form;
        cp.n_steps = n_steps;
        cp.Q = c->cr_Q;
        cp.dt = c->cfg.dt;
        ProfScope ps(c, KIND_DIRECT, s);
        CUDA_OR_FAIL(c, launch_cluster_rollout(cp, s));
        return LENIA_OK;
    }
    if (c->small && !stats_out && n_steps >= 2) {
        // one cooperative launch for the whole rollout (small world, global genes)
        SmallRolloutParams sp;
        memset(&sp, 0, sizeof(sp));
        sp.A = A;
        sp.buf = c->d_A2;
        sp.taps = c->d_small_taps;
        for (int k = 0; k <= c->cfg.n_kernels; k++) sp.tap_off[k] = c->small_tap_off[k];
        sp.n_taps = c->small_tap_off.back();
        sp.kt = c->kt;
        sp.H = c->cfg.height;
        sp.W = c->cfg.width;
        sp.C = c->cfg.n_channels;
        sp.maxR = c->max_R;
        sp.growth_form = c->cfg.growth_form;
        sp.dt = c->cfg.dt;
        sp.n_steps = n_steps;
        sp.count = c->d_small_count;
        sp.status = c->d_status;
        ProfScope ps(c, KIND_DIRECT, s);
        CUDA_OR_FAIL(c, launch_small_rollout(sp, s));
        return LENIA_OK;
    }
    // per-step statistics go to per-step addresses, and short rollouts do not
    // repay a capture: launch directly
    if (stats_out || n_steps < 4) return rollout_body(c, A, P, n_steps, stats_out, s);
    // otherwise pairs of steps replay one cached two-step graph (the state is
    // back in A, P after each pair); an odd last step runs directly
    const std::array<uintptr_t, 7> key{(uintptr_t)A, (uintptr_t)P, (uintptr_t)c->genes_version, 2, 0, 0, 0};
    for (int i = 0; i < n_steps / 2; i++) {
        const lenia_status st =
            run_graph(c, c->g_rollout, key, s, [&](cudaStream_t t) { return rollout_body(c, A, P, 2, nullptr, t); });
        if (st != LENIA_OK) return st;
    }
    return (n_steps % 2) ? rollout_body(c, A, P, 1, nullptr, s) : LENIA_OK;
}

// The backward's work, enqueued on s (a fixed sequence of launches and
// copies for given arguments: no host decision depends on device data).
// Reads A_0 from the first checkpoint slot and dL/dA_T from d_gA[0]; leaves
// dL/dA_0 in d_gA[n_steps % 2] (one buffer swap per reversed step) and the
// gene gradients in d_gene_acc (compensated FP32 pairs), so that it touches
// library buffers only.
static lenia_status backward_body(lenia_ctx* c, int32_t n_steps, cudaStream_t s)
{
    const int C = c->cfg.n_channels, K = c->cfg.n_kernels, L = c->ckpt;
    const size_t nA = c->N * C;
    auto ckpt = [&](int j) { return c->d_ckpt + (size_t)j * nA; };
    auto seg = [&](int j) { return c->d_seg + (size_t)j * nA; };

    // forward pass, keeping the states at multiples of the checkpoint interval
    const float* prev = ckpt(0);
    if (L == 1) {
        // every state and every step's potentials kept: reverse directly
        auto uall = [&](int t) { return c->d_Useg + (size_t)t * K * c->N; };
        for (int t = 0; t < n_steps; t++) {
            lenia_status st = potentials(c, ckpt(t), uall(t), s);
            if (st == LENIA_OK && t + 1 < n_steps)
                st = step_impl(c, ckpt(t), nullptr, ckpt(t + 1), nullptr, nullptr, nullptr, uall(t), s);
            if (st != LENIA_OK) return st;
        }
        CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_gene_acc, 0, (size_t)K * 3 * sizeof(float2), s));
        int cur = 0;
        for (int t = n_steps - 1; t >= 0; t--) {
            AdjParams ap;
            memset(&ap, 0, sizeof(ap));
            ap.A = ckpt(t);
            ap.U = uall(t);
            ap.gA_next = c->d_gA[cur];
            ap.gpre = c->d_gpre;
            ap.gU = c->d_gU;
            ap.V = c->d_V;
            ap.gA_out = c->d_gA[cur ^ 1];
            ap.gene_partials = c->d_gene_part;
            ap.gene_acc = c->d_gene_acc;
            ap.H = c->cfg.height;
            ap.W = c->cfg.width;
            ap.growth_form = c->cfg.growth_form;
            ap.dt = c->cfg.dt;
            ap.kt = c->kt;
            CUDA_OR_FAIL(c, launch_adjoint_epilogue(ap, s));
            bool per_channel = false;
            lenia_status st = transposed_conv(c, c->d_gU, c->d_V, s, &per_channel, c->d_gpre, c->d_gA[cur ^ 1]);
            if (st != LENIA_OK) return st;
            if (!per_channel) CUDA_OR_FAIL(c, launch_adjoint_gather(ap, s));
            cur ^= 1;
        }
        return LENIA_OK;
    }
    for (int t = 0; t + 1 < n_steps; t++) {
        float* dst = ((t + 1) % L == 0) ? ckpt((t + 1) / L) : seg((t + 1) & 1);
        lenia_status st = step_impl(c, prev, nullptr, dst, nullptr, nullptr, nullptr, nullptr, s);
        if (st != LENIA_OK) return st;
        prev = dst;
    }
    // backward, segment by segment from the last: recompute the segment's
    // states and their potentials from its checkpoint, then apply the step
    // adjoint in reverse
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->d_gene_acc, 0, (size_t)K * 3 * sizeof(float2), s));
    auto useg = [&](int j) { return c->d_Useg + (size_t)j * K * c->N; };
    int cur = 0;
    const int n_seg = (n_steps + L - 1) / L;
    for (int sg = n_seg - 1; sg >= 0; sg--) {
        const int s0 = sg * L, s1 = std::min(n_steps, s0 + L);
        for (int j = 0; j < s1 - s0; j++) {
            const float* Aj = j == 0 ? ckpt(sg) : seg(j);
            lenia_status st = potentials(c, Aj, useg(j), s);
            if (st == LENIA_OK && j + 1 < s1 - s0)
                st = step_impl(c, Aj, nullptr, seg(j + 1), nullptr, nullptr, nullptr, useg(j), s);
            if (st != LENIA_OK) return st;
        }
        for (int t = s1 - 1; t >= s0; t--) {
            const float* At = t == s0 ? ckpt(sg) : seg(t - s0);
            AdjParams ap;
            memset(&ap, 0, sizeof(ap));
            ap.A = At;
            ap.U = useg(t - s0);
            ap.gA_next = c->d_gA[cur];
            ap.gpre = c->d_gpre;
            ap.gU = c->d_gU;
            ap.V = c->d_V;
            ap.gA_out = c->d_gA[cur ^ 1];
            ap.gene_partials = c->d_gene_part;
            ap.gene_acc = c->d_gene_acc;
            ap.H = c->cfg.height;
            ap.W = c->cfg.width;
            ap.growth_form = c->cfg.growth_form;
            ap.dt = c->cfg.dt;
            ap.kt = c->kt;
            CUDA_OR_FAIL(c, launch_adjoint_epilogue(ap, s));
            bool per_channel = false;
            lenia_status st = transposed_conv(c, c->d_gU, c->d_V, s, &per_channel, c->d_gpre, c->d_gA[cur ^ 1]);
            if (st != LENIA_OK) return st;
            if (!per_channel) CUDA_OR_FAIL(c, launch_adjoint_gather(ap, s));
            cur ^= 1;
        }
    }
    return LENIA_OK;
}

lenia_status lenia_backward(lenia_ctx* c, const float* A0, const float* P0, int32_t n_steps, const float* gA_T,
                            float* gA0, float* g_genes, void* stream)
{
    if (!c) return LENIA_EINVAL;
    if (!c->adj)
        return fail(c, LENIA_ENOTSUP,
                    "lenia_backward needs global genes and a context made with max_rollout_steps > 0");
    if (!A0 || !gA_T) return fail(c, LENIA_EINVAL, "A0 and gA_T must be non-null");
    if (P0) return fail(c, LENIA_EINVAL, "P0 must be NULL: the adjoint covers global genes only");
    if (n_steps < 1 || n_steps > c->max_steps) return fail(c, LENIA_EINVAL, "n_steps must be 1..max_rollout_steps");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = c->cfg.n_kernels;
    const size_t nA = c->N * c->cfg.n_channels;
    // the arguments go in and out by copies on s, so that the graph of the
    // pass itself depends only on n_steps and the genes
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_ckpt, A0, nA * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->d_gA[0], gA_T, nA * sizeof(float), cudaMemcpyDeviceToDevice, s));
    const std::array<uintptr_t, 7> key{(uintptr_t)n_steps, (uintptr_t)c->genes_version, 1, 0, 0, 0, 0};
    const lenia_status st =
        run_graph(c, c->g_backward, key, s, [&](cudaStream_t t) { return backward_body(c, n_steps, t); });
    if (st != LENIA_OK) return st;
    const int cur = n_steps & 1;
    if (gA0) CUDA_OR_FAIL(c, cudaMemcpyAsync(gA0, c->d_gA[cur], nA * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (g_genes) CUDA_OR_FAIL(c, launch_adjoint_gene_out(c->d_gene_acc, K * 3, g_genes, s));
    return LENIA_OK;
}

lenia_status lenia_set_genes(lenia_ctx* c, const float* genes)
{
    if (!c || !genes) return LENIA_EINVAL;
    const int K = c->cfg.n_kernels;
    for (int k = 0; k < K; k++) {
        const float mu = genes[3 * k], sg = genes[3 * k + 1], h = genes[3 * k + 2];
        if (!isfinite(mu) || !isfinite(sg) || !isfinite(h)) return fail(c, LENIA_EINVAL, "genes must be finite");
        if (!(c->cfg.localized & LENIA_LOC_SIGMA) && !(sg > 0.f)) return fail(c, LENIA_EINVAL, "sigma must be > 0");
    }
    for (int k = 0; k < K; k++) {
        c->kd[k].mu = c->kt.mu[k] = genes[3 * k];
        c->kd[k].sigma = c->kt.sigma[k] = genes[3 * k + 1];
        c->kd[k].h = c->kt.h[k] = genes[3 * k + 2];
    }
    c->genes_version++;                    // kernels captured with the old genes are stale
    return LENIA_OK;
}

lenia_status lenia_stats(lenia_ctx* c, const float* A, float* out, void* stream)
{
    if (!c) return LENIA_EINVAL;
    if (!A || !out) return fail(c, LENIA_EINVAL, "A and out must be non-null");
    cudaStream_t s = (cudaStream_t)stream;
    const int H = c->cfg.height, W = c->cfg.width, C = c->cfg.n_channels;
    int nb = 0;
    CUDA_OR_FAIL(c, launch_stats_partials(A, C, H, W, c->d_trig, c->d_trig + H, c->d_trig + 2 * H,
                                          c->d_trig + 2 * H + W, c->d_partials, s, &nb));
    CUDA_OR_FAIL(c, launch_stats_final(c->d_partials, nb, C, H, W, out, s));
    return LENIA_OK;
}

lenia_status lenia_potentials(lenia_ctx* c, const float* A_in, float* U_out, void* stream)
{
    if (!c) return LENIA_EINVAL;
    if (!A_in || !U_out) return fail(c, LENIA_EINVAL, "A_in and U_out must be non-null");
    if (ranges_overlap(A_in, c->N * c->cfg.n_channels * sizeof(float), U_out,
                       c->N * c->cfg.n_kernels * sizeof(float)))
        return fail(c, LENIA_EINVAL, "A_in and U_out overlap");
    return potentials(c, A_in, U_out, (cudaStream_t)stream);
}

lenia_status lenia_update_from_potentials(lenia_ctx* c, const float* A_in, const float* P_in, const float* U_in,
                                          float* A_out, float* P_out, uint8_t* alpha_out, void* stream)
{
    lenia_status st = check_state_args(c, A_in, P_in, A_out, P_out);
    if (st != LENIA_OK) return st;
    if (!U_in) return fail(c, LENIA_EINVAL, "U_in must be non-null");
    return step_impl(c, A_in, P_in, A_out, P_out, nullptr, alpha_out, U_in, (cudaStream_t)stream);
}

lenia_status lenia_set_walls(lenia_ctx* c, const uint8_t* mask)
{
    if (!c) return LENIA_EINVAL;
    std::vector<int> idx;
    if (mask)
        for (size_t i = 0; i < c->N; i++)
            if (mask[i]) idx.push_back((int)i);
    if (c->d_walls) {
        CUDA_OR_FAIL(c, cudaFree(c->d_walls));
        c->d_walls = nullptr;
    }
    c->n_walls = 0;
    if (idx.empty()) return LENIA_OK;
    lenia_status st = dalloc(c, &c->d_walls, idx.size());
    if (st != LENIA_OK) return st;
    CUDA_OR_FAIL(c, cudaMemcpy(c->d_walls, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
    c->n_walls = (int)idx.size();
    return LENIA_OK;
}

lenia_status lenia_step_evolve(lenia_ctx* c, float* A, float* P, float* A_out, float* P_out,
                               const lenia_events* ev, float* stats_out, uint8_t* alpha_out, float* epen_out,
                               void* stream)
{
    lenia_status st = check_state_args(c, A, P, A_out, P_out);
    if (st != LENIA_OK) return st;
    if (!ev) return fail(c, LENIA_EINVAL, "ev must be non-null");
    const int H = c->cfg.height, W = c->cfg.width, K = c->cfg.n_kernels;
    if (ev->r_oxy < 1 || ev->r_oxy > kMaxROxy || 2 * ev->r_oxy + 1 > std::min(H, W))
        return fail(c, LENIA_EINVAL, "r_oxy must be 1..32 and 2 r_oxy + 1 <= min(H, W)");
    if (!isfinite(ev->mut_delta) || !isfinite(ev->gamma_mut) || !isfinite(ev->pen_delta) ||
        !isfinite(ev->gamma_pen) || !isfinite(ev->eps_pen))
        return fail(c, LENIA_EINVAL, "event deltas, rates and eps_pen must be finite");
    if (ev->mut_plane < -1 || ev->mut_plane >= c->n_p || ev->pen_plane < -1 || ev->pen_plane >= c->n_p)
        return fail(c, LENIA_EINVAL, "mut_plane and pen_plane must be -1 or a localized gene plane");
    if (ev->mut_plane >= 0 &&
        (ev->mut_kernel < 0 || ev->mut_kernel >= K || ev->mut_x0 < 0 || ev->mut_x0 >= W || ev->mut_y0 < 0 ||
         ev->mut_y0 >= H || ev->mut_half < 0 || 2 * ev->mut_half > std::min(H, W)))
        return fail(c, LENIA_EINVAL, "mutation kernel, centre or half-size out of range");
    if (ev->pen_plane >= 0 && (ev->pen_kernel < 0 || ev->pen_kernel >= K))
        return fail(c, LENIA_EINVAL, "pen_kernel out of range");
    if (!c->d_empty) {
        st = dalloc(c, &c->d_alpha_e, c->N);
        if (st == LENIA_OK) st = dalloc(c, &c->d_empty, c->N);
        if (st != LENIA_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // (1) environment: walls remove material from the current state
    if (c->n_walls > 0) {
        ProfScope ps(c, KIND_WALLS, s);
        CUDA_OR_FAIL(c, launch_walls_zero(c->d_walls, c->n_walls, A, c->cfg.n_channels, P, c->n_p * K, c->N, s));
    }
    // (2) the step, with its alpha and not-Delta_sum(U) masks
    uint8_t* alpha = alpha_out ? alpha_out : c->d_alpha_e;
    st = step_impl(c, A, P, A_out, P_out, stats_out, alpha, nullptr, s, c->d_empty);
    if (st != LENIA_OK) return st;
    // (3)-(5) penalising area, mutation, penalisation
    EvoParams e;
    memset(&e, 0, sizeof(e));
    e.empty = c->d_empty;
    e.alpha = alpha;
    e.P = c->n_p ? P_out : nullptr;
    e.epen_out = epen_out;
    e.H = H;
    e.W = W;
    e.r_oxy = ev->r_oxy;
    int n = 0;
    for (int dy = 0; dy <= ev->r_oxy; dy++) {
        int w = 0;
        while ((w + 1) * (w + 1) + dy * dy <= ev->r_oxy * ev->r_oxy) w++;
        e.half_width[dy] = w;
        n += (dy == 0 ? 1 : 2) * (2 * w + 1);
    }
    e.n_disk = n;
    e.n_disk2 = (double)n * n;
    e.mut_plane = ev->mut_plane >= 0 ? ev->mut_plane * K + ev->mut_kernel : -1;
    e.pen_plane = ev->pen_plane >= 0 ? ev->pen_plane * K + ev->pen_kernel : -1;
    e.mut_x0 = ev->mut_x0;
    e.mut_y0 = ev->mut_y0;
    e.mut_half = ev->mut_half;
    e.mut_add = (float)(ev->gamma_mut * ev->mut_delta);
    e.pen_add = (float)(ev->gamma_pen * ev->pen_delta);
    // E_pen > eps_pen  <=>  M > eps_pen n^2  <=>  M > floor(eps_pen n^2) for integer M
    const double t = floor(ev->eps_pen * e.n_disk2);
    e.pen_thresh = t < -1.0 ? -1LL : (t > e.n_disk2 ? (long long)e.n_disk2 : (long long)t);
    if (!c->n_p) e.mut_plane = e.pen_plane = -1;
    {
        // both disk passes in one launch (kind "pen_disk")
        ProfScope ps(c, KIND_PEN, s);
        CUDA_OR_FAIL(c, launch_disk_fused(e, s));
    }
    return LENIA_OK;
}

lenia_status lenia_check(lenia_ctx* c, void* stream)
{
    if (!c) return LENIA_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_OR_FAIL(c, cudaStreamSynchronize(s));
    int st = 0;
    CUDA_OR_FAIL(c, cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        CUDA_OR_FAIL(c, cudaMemset(c->d_status, 0, sizeof(int)));
        // a block that gave up never took its stats ticket: re-arm the counter
        CUDA_OR_FAIL(c, cudaMemset(c->d_ticket, 0, sizeof(unsigned int)));
        return fail(c, LENIA_ETIMEOUT, "a device-side wait gave up (status " + std::to_string(st) + ")");
    }
    return LENIA_OK;
}

lenia_status lenia_selftest_wait_timeout(lenia_ctx* c, int32_t limit_mcycles, void* stream)
{
    if (!c || limit_mcycles < 1 || limit_mcycles > 4000) return LENIA_EINVAL;
    CUDA_OR_FAIL(c, launch_selftest_wait((long long)limit_mcycles * 1000000LL, c->d_status, (cudaStream_t)stream));
    return LENIA_OK;
}

static lenia_status host_step_enqueue(lenia_ctx* c, const float* A_in, const float* P_in, float* A_out,
                                      float* P_out, float* stats_out, void* stream)
{
    if (!c) return LENIA_EINVAL;
    if (!A_in || !A_out || (c->n_p && (!P_in || !P_out)))
        return fail(c, LENIA_EINVAL, "host A (and P with localized genes) must be non-null");
    const int C = c->cfg.n_channels;
    const size_t nA = c->N * C, nP = c->N * c->n_p * c->cfg.n_kernels;
    if (!c->up_stream) {
        lenia_status a = LENIA_OK;
        if (!c->d_hA_in1) a = dalloc(c, &c->d_hA_in1, nA);
        if (a == LENIA_OK && !c->d_hA_out1) a = dalloc(c, &c->d_hA_out1, nA);
        if (a == LENIA_OK && nP && !c->d_hP_in1) a = dalloc(c, &c->d_hP_in1, nP);
        if (a == LENIA_OK && nP && !c->d_hP_out1) a = dalloc(c, &c->d_hP_out1, nP);
        if (a == LENIA_OK && !c->d_hstats) a = dalloc(c, &c->d_hstats, (size_t)2 * C * 3);
        if (a != LENIA_OK) return a;
        // streams and events are made into locals and kept only once all exist
        cudaStream_t up = nullptr, down = nullptr;
        cudaEvent_t evs[6] = {};
        auto make = [&]() -> lenia_status {
            CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking));
            CUDA_OR_FAIL(c, cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking));
            for (int i = 0; i < 6; i++) CUDA_OR_FAIL(c, cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming));
            // nothing recorded yet: record once so that the first waits are no-ops
            for (int b = 0; b < 2; b++) {
                CUDA_OR_FAIL(c, cudaEventRecord(evs[2 + b], (cudaStream_t)stream));
                CUDA_OR_FAIL(c, cudaEventRecord(evs[4 + b], (cudaStream_t)stream));
            }
            return LENIA_OK;
        };
        const lenia_status ms = make();
        if (ms != LENIA_OK) {
            for (cudaEvent_t e : evs)
                if (e) cudaEventDestroy(e);
            if (up) cudaStreamDestroy(up);
            if (down) cudaStreamDestroy(down);
            return ms;
        }
        c->up_stream = up;
        c->down_stream = down;
        for (int b = 0; b < 2; b++) {
            c->ev_up[b] = evs[b];
            c->ev_done[b] = evs[2 + b];
            c->ev_down[b] = evs[4 + b];
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int b = c->host_set;
    float* dA_in = b ? c->d_hA_in1 : c->d_A2;
    float* dP_in = b ? c->d_hP_in1 : c->d_P2;
    float* dA_out = b ? c->d_hA_out1 : c->d_A3;
    float* dP_out = b ? c->d_hP_out1 : c->d_P3;
    float* dstats = c->d_hstats + (size_t)b * C * 3;
    const size_t ab = nA * sizeof(float), pb = nP * sizeof(float);
    // uploads on their own stream, into the set the step before last has
    // finished reading: they run ahead, under the previous step's compute
    // and downloads
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(c->up_stream, c->ev_done[b], 0));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(dA_in, A_in, ab, cudaMemcpyHostToDevice, c->up_stream));
    if (pb) CUDA_OR_FAIL(c, cudaMemcpyAsync(dP_in, P_in, pb, cudaMemcpyHostToDevice, c->up_stream));
    CUDA_OR_FAIL(c, cudaEventRecord(c->ev_up[b], c->up_stream));
    // the step, once its inputs landed and the download of the step before
    // last is done with this set's outputs
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(s, c->ev_up[b], 0));
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(s, c->ev_down[b], 0));
    lenia_status st = step_impl(c, dA_in, c->n_p ? dP_in : nullptr, dA_out, c->n_p ? dP_out : nullptr,
                                stats_out ? dstats : nullptr, nullptr, nullptr, s);
    if (st != LENIA_OK) return st;
    CUDA_OR_FAIL(c, cudaEventRecord(c->ev_done[b], s));
    // downloads on their own stream, overlapping the next steps' uploads
    CUDA_OR_FAIL(c, cudaStreamWaitEvent(c->down_stream, c->ev_done[b], 0));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(A_out, dA_out, ab, cudaMemcpyDeviceToHost, c->down_stream));
    if (pb) CUDA_OR_FAIL(c, cudaMemcpyAsync(P_out, dP_out, pb, cudaMemcpyDeviceToHost, c->down_stream));
    if (stats_out)
        CUDA_OR_FAIL(c, cudaMemcpyAsync(stats_out, dstats, C * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                                        c->down_stream));
    CUDA_OR_FAIL(c, cudaEventRecord(c->ev_down[b], c->down_stream));
    c->host_set = b ^ 1;
    c->host_pending = true;
    return LENIA_OK;
}

lenia_status lenia_step_host_async(lenia_ctx* c, const float* A_in, const float* P_in, float* A_out, float* P_out,
                                   float* stats_out, void* stream)
{
    const lenia_status st = host_step_enqueue(c, A_in, P_in, A_out, P_out, stats_out, stream);
    if (st != LENIA_OK && st != LENIA_EINVAL && c && c->up_stream) {
        // a failure after part of the step was enqueued: let every copy that
        // touches the caller's host buffers finish before returning, so that
        // none of them runs after the caller has reused its buffers
        cudaStreamSynchronize(c->up_stream);
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaStreamSynchronize(c->down_stream);
        (void)cudaGetLastError();
        c->host_pending = false;
    }
    return st;
}

lenia_status lenia_host_wait(lenia_ctx* c, void* stream)
{
    if (!c) return LENIA_EINVAL;
    if (c->host_pending) {
        CUDA_OR_FAIL(c, cudaStreamSynchronize(c->down_stream));
        c->host_pending = false;
    }
    return lenia_check(c, stream);
}

lenia_status lenia_step_host(lenia_ctx* c, const float* A_in, const float* P_in, float* A_out, float* P_out,
                             float* stats_out, void* stream)
{
    lenia_status st = lenia_step_host_async(c, A_in, P_in, A_out, P_out, stats_out, stream);
    if (st != LENIA_OK) return st;
    return lenia_host_wait(c, stream);
}

lenia_status lenia_profile_start(lenia_ctx* c, int32_t max_launches)
{
    if (!c || max_launches < 1 || max_launches > (1 << 20)) return LENIA_EINVAL;
    const size_t need = 2 * (size_t)max_launches;
    while (c->ev.size() < need) {
        cudaEvent_t e;
        CUDA_OR_FAIL(c, cudaEventCreate(&e));
        c->ev.push_back(e);
    }
    c->ev_kind.assign(max_launches, 0);
    c->ev_used = 0;
    c->prof = true;
    return LENIA_OK;
}

lenia_status lenia_profile_stop(lenia_ctx* c, float* total_ms, int32_t* counts)
{
    if (!c || !total_ms || !counts) return LENIA_EINVAL;
    c->prof = false;
    for (int k = 0; k < KIND_COUNT; k++) {
        total_ms[k] = 0.f;
        counts[k] = 0;
    }
    for (size_t i = 0; i < c->ev_used; i += 2) {
        CUDA_OR_FAIL(c, cudaEventSynchronize(c->ev[i + 1]));
        float ms = 0.f;
        CUDA_OR_FAIL(c, cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
        const int k = c->ev_kind[i / 2];
        total_ms[k] += ms;
        counts[k] += 1;
    }
    c->ev_used = 0;
    return LENIA_OK;
}

const char* lenia_profile_kind_name(int32_t kind)
{
    return (kind >= 0 && kind < KIND_COUNT) ? kKindNames[kind] : nullptr;
}

lenia_status lenia_kernel_weights(const lenia_ctx* c, int32_t k, double* out)
{
    if (!c || !out || k < 0 || k >= c->cfg.n_kernels) return LENIA_EINVAL;
    if (c->cfg.n_rings) return LENIA_ENOTSUP;     // kernels are made per site from the rings
    memcpy(out, c->kw[k].data(), c->kw[k].size() * sizeof(double));
    return LENIA_OK;
}

}  // extern "C"
