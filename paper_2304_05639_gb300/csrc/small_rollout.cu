// Rollouts of small worlds with global genes in one cooperative launch
// (Algorithm 2's step repeated: convolve, growth, clipped update; no gene
// maps, so no diffusion or alpha mask).
//
// A world of a few thousand sites cannot fill the GPU with one launch per
// stage: every step of the regular route is four or five short launches, and
// their start-up latency, not the arithmetic, sets the step time.  Here every
// block owns an 8 x 8 tile of sites for the whole rollout (four threads per
// site).  Per step it
// stages the tile's neighbourhood of every channel (radius maxR, periodic)
// from the current state into shared memory, computes each kernel's
// potential at its sites as a direct sum over the kernel's non-zero taps (in
// the order of the direct route: tap columns dx, then rows dy), the growth G = h (2 g - 1) or h g with g = exp(-(U - mu)^2 /
// 2 sigma^2), and the clipped update, writes the next state, and meets the
// other blocks at a grid barrier.  The barrier is a counter in device memory
// (zeroed before the launch) that each block increments once per step and
// then waits for, bounded in time: a wait that gives up writes the status
// word and the block leaves (the others then give up at their own next
// wait).  The launch is cooperative, so every block is resident.
#include <math.h>

#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

namespace {

constexpr int SR_T = 8;                 // tile side (one site per thread)

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every block arrives once; returns false if the wait gave up.
__device__ bool grid_barrier(unsigned* count, unsigned target, int* status)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        ok = 1;
        const long long t0 = clock64();
        while (ld_acquire(count) < target) {
            if (clock64() - t0 > kWaitLimitCycles) {
                ok = 0;
                atomicExch(status, kStatusWaitTimeout);
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Four threads per site (consecutive lanes), each summing every fourth tap
// of each kernel with four alternating accumulators; the four partial sums
// meet in a shuffle tree, and the first thread of the site forms the growth
// and the update.  The non-zero taps of every kernel (offset in the staged
// tile, weight) are copied into shared memory once per rollout, so the tap
// loop reads shared memory only.
constexpr int SR_Q = 4;
constexpr int SR_THREADS = SR_T * SR_T * SR_Q;

__global__ void __launch_bounds__(SR_THREADS) k_small_rollout(SmallRolloutParams p)
{
    extern __shared__ float smem_f[];
    const int R = p.maxR, TP = SR_T + 2 * R;
    const int H = p.H, W = p.W, C = p.C;
    const size_t N = (size_t)H * W;
    float* tiles = smem_f;                               // [C][TP * TP]
    float* tw = tiles + (size_t)C * TP * TP;             // [n_taps] weights
    int* toff = reinterpret_cast<int*>(tw + p.n_taps);   // [n_taps] offsets dy TP + dx
    for (int i = threadIdx.x; i < p.n_taps; i += SR_THREADS) {
        const int2 t = __ldg(&p.taps[i]);                // ((dy + 1024) 2048 + dx + 1024, weight bits)
        const int dy = t.x / 2048 - 1024, dx = t.x % 2048 - 1024;
        toff[i] = dy * TP + dx;
        tw[i] = __int_as_float(t.y);
    }
    const int tiles_x = W / SR_T;
    const int x0 = (blockIdx.x % tiles_x) * SR_T, y0 = (blockIdx.x / tiles_x) * SR_T;
    const int tid = threadIdx.x, site = tid / SR_Q, q = tid % SR_Q;
    const int tx = site % SR_T, ty = site / SR_T;
    const int x = x0 + tx, y = y0 + ty;
    for (int t = 0; t < p.n_steps; t++) {
        const float* src = (t % 2 == 0) ? p.A : p.buf;
        float* dst = (t % 2 == 0) ? p.buf : p.A;
#pragma unroll 4
        for (int u = tid; u < C * TP * TP; u += SR_THREADS) {
            const int c = u / (TP * TP), r = u % (TP * TP);
            int yy = y0 - R + r / TP, xx = x0 - R + r % TP;
            yy = yy < 0 ? yy + H : (yy >= H ? yy - H : yy);
            xx = xx < 0 ? xx + W : (xx >= W ? xx - W : xx);
            tiles[u] = __ldcg(&src[(size_t)c * N + (size_t)yy * W + xx]);
        }
        __syncthreads();
        float acc[kMaxChannels];
        for (int c = 0; c < C; c++) acc[c] = 0.f;
        for (int k = 0; k < p.kt.K; k++) {
            const float* tl = tiles + (size_t)p.kt.src[k] * TP * TP + (ty + R) * TP + (tx + R);
            const int i0 = p.tap_off[k], i1 = p.tap_off[k + 1];
            float u0 = 0.f, u1 = 0.f, u2 = 0.f, u3 = 0.f;
            int i = i0 + q;
            for (; i + 3 * SR_Q < i1; i += 4 * SR_Q) {
                u0 = fmaf(tw[i], tl[toff[i]], u0);
                u1 = fmaf(tw[i + SR_Q], tl[toff[i + SR_Q]], u1);
                u2 = fmaf(tw[i + 2 * SR_Q], tl[toff[i + 2 * SR_Q]], u2);
                u3 = fmaf(tw[i + 3 * SR_Q], tl[toff[i + 3 * SR_Q]], u3);
            }
            for (; i < i1; i += SR_Q) u0 = fmaf(tw[i], tl[toff[i]], u0);
            float u = (u0 + u1) + (u2 + u3);
            u += __shfl_xor_sync(0xffffffffu, u, 1);
            u += __shfl_xor_sync(0xffffffffu, u, 2);
            const float sg = p.kt.sigma[k], h = p.kt.h[k];
            const float z = (u - p.kt.mu[k]) / sg;
            const float g = sg > 0.f ? expf(-0.5f * z * z) : 0.f;
            acc[p.kt.dst[k]] += p.growth_form == 0 ? h * (2.f * g - 1.f) : h * g;
        }
        if (q == 0) {
            const size_t i = (size_t)y * W + x;
            for (int c = 0; c < C; c++) {
                const float a = tiles[(size_t)c * TP * TP + (ty + R) * TP + (tx + R)] + p.dt * acc[c];
                dst[(size_t)c * N + i] = fminf(fmaxf(a, 0.f), 1.f);
            }
        }
        if (!grid_barrier(p.count, (unsigned)(t + 1) * gridDim.x, p.status)) return;
    }
    if (p.n_steps % 2 && q == 0) {
        // the last step wrote the second buffer: this block's sites back to A
        const size_t i = (size_t)y * W + x;
        for (int c = 0; c < C; c++) p.A[(size_t)c * N + i] = __ldcg(&p.buf[(size_t)c * N + i]);
    }
}

}  // namespace

size_t small_rollout_smem(int C, int maxR, int n_taps)
{
    const size_t tp = SR_T + 2 * (size_t)maxR;
    return (size_t)C * tp * tp * sizeof(float) + (size_t)n_taps * 8;
}

bool small_rollout_supported(int H, int W, int C, int K, int maxR, int n_taps)
{
    if (H % SR_T || W % SR_T || (long long)H * W > 128 * 128 || C > kMaxChannels || K > kMaxKernels) return false;
    if (small_rollout_smem(C, maxR, n_taps) > 160 * 1024) return false;
    int dev = 0, n_sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    const size_t smem = small_rollout_smem(C, maxR, n_taps);
    if (cudaFuncSetAttribute(k_small_rollout, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_rollout, SR_THREADS, smem) != cudaSuccess)
        return false;
    return (long long)(H / SR_T) * (W / SR_T) <= (long long)per_sm * n_sms;
}

cudaError_t launch_small_rollout(const SmallRolloutParams& p, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(p.count, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const size_t smem = small_rollout_smem(p.C, p.maxR, p.n_taps);
    e = cudaFuncSetAttribute(k_small_rollout, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    SmallRolloutParams q = p;
    void* args[] = {&q};
    const dim3 grid((p.H / SR_T) * (p.W / SR_T)), block(SR_THREADS);
    return cudaLaunchCooperativeKernel((const void*)k_small_rollout, grid, block, args, smem, s);
}

}  // namespace lenia
