// Adjoint of the Lenia step with global genes (no gene maps, no alpha):
//   U_k  = K~_k * A_src(k)
//   g_k  = exp(-(U_k - mu_k)^2 / (2 sigma_k^2)),  F(g) = 2g - 1 (signed) or g (paper form)
//   pre_c = A_c + dt sum_{k: dst(k)=c} h_k F(g_k),   A'_c = clip(pre_c, 0, 1)
// Given dL/dA' this computes, per site,
//   gpre_c = dL/dA'_c [0 < pre_c < 1]                (clip subgradient)
//   gU_k   = gpre_dst(k) dt h_k F'(g) g (-(U - mu) / sigma^2)
// and the per-kernel gene gradients
//   dL/dmu_k    = sum gpre dt h_k F' g (U - mu) / sigma^2
//   dL/dsigma_k = sum gpre dt h_k F' g (U - mu)^2 / sigma^3
//   dL/dh_k     = sum gpre dt F(g)
// as block partials in compensated FP32 pairs (hi + lo), reduced in a fixed
// order by a second small kernel (one block per value).  The transposed convolution (gA_src += K~_k (x) gU_k; K~ is
// point symmetric, so it is the same convolution) runs on the forward
// machinery; its inverse row pass adds gpre (FFT path) or k_adjoint_gather
// adds it (direct path).
#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

constexpr int ADJ_THREADS = 256;
constexpr float ADJ_HALF_LOG2E = 0.721347520444481703680f;   // 0.5 log2(e)

// One site per thread; the growth is recomputed with the same arithmetic as
// the forward streaming epilogue so that clip decisions match.
__global__ void __launch_bounds__(ADJ_THREADS) k_adjoint_epilogue(AdjParams p)
{
    pdl_enter();
    const int K = p.kt.K, C = p.kt.C;
    const size_t N = (size_t)p.H * p.W;
    const size_t i = (size_t)blockIdx.x * ADJ_THREADS + threadIdx.x;
    const bool valid = i < N;
    __shared__ float red[ADJ_THREADS / 32][kMaxKernels * 3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    float pre[kMaxChannels];
    float gpre[kMaxChannels];
    if (valid) {
        for (int c = 0; c < C; c++) pre[c] = 0.f;
        for (int k = 0; k < K; k++) {
            const float u = __ldg(&p.U[(size_t)k * N + i]);
            const float z = (u - p.kt.mu[k]) * rcp_approx(p.kt.sigma[k]);
            const float g = ex2_approx(-ADJ_HALF_LOG2E * (z * z));
            const float h = p.kt.h[k];
            pre[p.kt.dst[k]] += p.growth_form == 0 ? fmaf(2.f * g, h, -h) : h * g;
        }
        for (int c = 0; c < C; c++) {
            const float a = __ldg(&p.A[(size_t)c * N + i]) + p.dt * pre[c];
            const float gA = __ldg(&p.gA_next[(size_t)c * N + i]);
            gpre[c] = (a > 0.f && a < 1.f) ? gA : 0.f;
            p.gpre[(size_t)c * N + i] = gpre[c];
        }
    }
    // kernel by kernel: potential gradient and this block's gene partials
    for (int k = 0; k < K; k++) {
        float dmu = 0.f, dsg = 0.f, dh = 0.f;
        if (valid) {
            const float u = __ldg(&p.U[(size_t)k * N + i]);
            const float mu = p.kt.mu[k], sg = p.kt.sigma[k], h = p.kt.h[k];
            const float d = u - mu;
            const float z = d * rcp_approx(sg);
            const float g = ex2_approx(-ADJ_HALF_LOG2E * (z * z));
            const float fp = p.growth_form == 0 ? 2.f : 1.f;          // F'(g)
            const float gG = gpre[p.kt.dst[k]] * p.dt * h;             // dL/dF
            const float w = gG * fp * g;                               // dL/d(exp term)
            const float inv_s2 = 1.f / (sg * sg);
            p.gU[(size_t)k * N + i] = -w * d * inv_s2;
            dmu = w * d * inv_s2;
            dsg = w * d * d * inv_s2 / sg;
            dh = gpre[p.kt.dst[k]] * p.dt * (p.growth_form == 0 ? 2.f * g - 1.f : g);
        }
        float v[3] = {dmu, dsg, dh};
#pragma unroll
        for (int j = 0; j < 3; j++) {
            float t = v[j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
            if (lane == 0) red[warp][k * 3 + j] = t;
        }
    }
    __syncthreads();
    // value-major partials [K * 3][blocks]: the reduction kernel reads them coalesced
    for (int v = threadIdx.x; v < K * 3; v += ADJ_THREADS) {
        float2 s = make_float2(0.f, 0.f);
        for (int w = 0; w < ADJ_THREADS / 32; w++) s = ff_add(s, make_float2(red[w][v], 0.f));
        p.gene_partials[(size_t)v * gridDim.x + blockIdx.x] = s;
    }
}

// gene_acc[v] += sum over the nb block partials of value v (block v): thread t
// sums blocks t, t + 256, ... in order, then a fixed shuffle / shared tree,
// so every launch adds in the same order.
constexpr int ADJ_RED_THREADS = 256;
__global__ void __launch_bounds__(ADJ_RED_THREADS) k_adjoint_gene_reduce(const float2* partials, int nb,
                                                                      float2* gene_acc)
{
    pdl_enter();
    __shared__ float2 wsum[ADJ_RED_THREADS / 32];
    const int v = blockIdx.x;
    const float2* src = partials + (size_t)v * nb;
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
    int b = threadIdx.x;
    for (; b + ADJ_RED_THREADS < nb; b += 2 * ADJ_RED_THREADS) {
        s0 = ff_add(s0, src[b]);
        s1 = ff_add(s1, src[b + ADJ_RED_THREADS]);
    }
    if (b < nb) s0 = ff_add(s0, src[b]);
    float2 s = ff_add(s0, s1);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s = ff_add(s, ff_shfl_down(s, off));
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < ADJ_RED_THREADS / 32; w++) t = ff_add(t, wsum[w]);
        gene_acc[v] = ff_add(gene_acc[v], t);
    }
}

// gA_c = gpre_c + sum_{k: src(k) = c} V_k  (V_k = K~_k (x) gU_k, in kernel order),
// or gpre_c + V_c when the sum over kernels was taken in the frequency domain
__global__ void __launch_bounds__(256) k_adjoint_gather(AdjParams p)
{
    pdl_enter();
    const size_t N = (size_t)p.H * p.W;
    const size_t i = (size_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < p.kt.C; c++) {
        float s = __ldg(&p.gpre[(size_t)c * N + i]);
        if (p.v_per_channel) {
            s += __ldg(&p.V[(size_t)c * N + i]);
        } else {
            for (int k = 0; k < p.kt.K; k++)
                if (p.kt.src[k] == c) s += __ldg(&p.V[(size_t)k * N + i]);
        }
        p.gA_out[(size_t)c * N + i] = s;
    }
}

__global__ void k_adjoint_gene_out(const float2* gene_acc, int nv, float* out)
{
    pdl_enter();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) out[v] = gene_acc[v].x + gene_acc[v].y;
}

int adjoint_blocks(int H, int W) { return (int)(((size_t)H * W + ADJ_THREADS - 1) / ADJ_THREADS); }

cudaError_t launch_adjoint_epilogue(const AdjParams& p, cudaStream_t s)
{
    const int nb = adjoint_blocks(p.H, p.W);
    launch_pdl(k_adjoint_epilogue, nb, ADJ_THREADS, 0, s, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    launch_pdl(k_adjoint_gene_reduce, p.kt.K * 3, ADJ_RED_THREADS, 0, s, p.gene_partials, nb, p.gene_acc);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gather(const AdjParams& p, cudaStream_t s)
{
    const size_t N = (size_t)p.H * p.W;
    launch_pdl(k_adjoint_gather, (unsigned)((N + 255) / 256), 256, 0, s, p);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gene_out(const float2* gene_acc, int nv, float* out, cudaStream_t s)
{
    launch_pdl(k_adjoint_gene_out, (nv + 63) / 64, 64, 0, s, gene_acc, nv, out);
    return cudaGetLastError();
}

}  // namespace lenia
