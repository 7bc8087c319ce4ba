// Direct periodic convolution, the fused growth / gene-maintenance / update
// epilogue, and per-channel statistics (arXiv 2304.05639, Sections 2.1-2.4,
// Algorithm 2).
#include <math.h>

#include "lenia_internal.cuh"

namespace lenia {

__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------- direct convolution
// U_k(y, x) = sum_d K~_k(d) A_src(k)(y + d, x + d), periodic (K~ is point
// symmetric, so this is the convolution K~ * A).  A block computes a 32 x 32
// output tile of one channel for every kernel reading that channel.  Each
// thread owns one column x and four rows; for each tap column dx it slides a
// four-row register window down the non-zero taps of that column.
constexpr int DC_TX = 32, DC_TY = 32, DC_ROWS = 4;

__global__ void __launch_bounds__(256) k_direct_conv(ConvParams p, int maxR)
{
    extern __shared__ float tile[];
    const int c = blockIdx.z;
    const int x0 = blockIdx.x * DC_TX, y0 = blockIdx.y * DC_TY;
    const int pitch = DC_TX + 2 * maxR;
    const int rows = DC_TY + 2 * maxR;
    const float* A = p.A + (size_t)c * p.H * p.W;
    for (int u = threadIdx.y * 32 + threadIdx.x; u < rows * pitch; u += 256) {
        const int ty = u / pitch, tx = u % pitch;
        tile[u] = __ldg(&A[(size_t)wrapi(y0 - maxR + ty, p.H) * p.W + wrapi(x0 - maxR + tx, p.W)]);
    }
    __syncthreads();
    const int tx = threadIdx.x;
    const int ty = threadIdx.y * DC_ROWS;
    const int x = x0 + tx;
    for (int t = 0; t < p.kcount[c]; t++) {
        const int k = p.klist[c][t];
        const int R = p.R[k];
        const float* w = p.w + p.w_off[k];       // [dx + R][dy + R]
        const int* yr = p.yr + p.yr_off[k];
        float acc[DC_ROWS] = {0.f, 0.f, 0.f, 0.f};
        for (int dx = -R; dx <= R; dx++) {
            const int r = __ldg(&yr[dx + R]);
            if (r < 0) continue;
            const float* col = tile + (size_t)(ty + maxR) * pitch + (tx + maxR + dx);
            const float* wc = w + (dx + R) * (2 * R + 1) + R;
            float v[DC_ROWS];
#pragma unroll
            for (int o = 0; o < DC_ROWS - 1; o++) v[o] = col[(o - r) * pitch];
            for (int dy = -r; dy <= r; dy++) {
                v[DC_ROWS - 1] = col[(dy + DC_ROWS - 1) * pitch];
                const float wv = __ldg(&wc[dy]);
#pragma unroll
                for (int o = 0; o < DC_ROWS; o++) acc[o] = fmaf(wv, v[o], acc[o]);
#pragma unroll
                for (int o = 0; o < DC_ROWS - 1; o++) v[o] = v[o + 1];
            }
        }
        if (x < p.W) {
#pragma unroll
            for (int o = 0; o < DC_ROWS; o++) {
                const int y = y0 + ty + o;
                if (y < p.H) p.U[((size_t)k * p.H + y) * p.W + x] = acc[o];
            }
        }
    }
}

cudaError_t launch_direct_conv(const ConvParams& p, int max_R, cudaStream_t s)
{
    const size_t smem = (size_t)(DC_TX + 2 * max_R) * (DC_TY + 2 * max_R) * sizeof(float);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(k_direct_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((p.W + DC_TX - 1) / DC_TX, (p.H + DC_TY - 1) / DC_TY, p.C);
    k_direct_conv<<<grid, dim3(32, DC_TY / DC_ROWS), smem, s>>>(p, max_R);
    return cudaGetLastError();
}

// ------------------------------------------------------------- epilogue
// Per site, in the order of Algorithm 2:
//   diffuse every gene plane (Section 2.3):
//     P^ = clip( sum_{|d|<=r} P / #{|d|<=r : P > eps_p}, 0, 1 ), 0 if the count is 0;
//   growth bump g_k = exp(-(U_k - m)^2 / (2 s^2)), g = 0 where s <= 0;
//   alpha = AND_k [h_k g_k > eps_u] AND AND_{p,k} [P^ > eps_p] (Section 2.2;
//     alpha_on = 1 tests U_k > eps_u instead of the growth);
//   P' = P^ . alpha;
//   A'_c = clip(A_c + dt sum_{k: dst(k)=c} h'_k G(g'_k), 0, 1) with the
//     masked genes (g' = 0 and localized h' = 0 where alpha = 0) and
//     G = 2g - 1 (signed) or g (paper form).
// Block: 32 x 8 sites, one per thread.  Optional per-block stats partials
// (sum A, sum A sin/cos of the y and x angles) in a fixed reduction order.
constexpr int EP_TX = 32, EP_TY = 8;

template <int KT, int CT, int NPT>
__global__ void __launch_bounds__(256) k_epilogue(EpiParams p)
{
    const int K = KT ? KT : p.kt.K;
    const int C = CT ? CT : p.kt.C;
    const int n_p = NPT >= 0 ? NPT : p.n_p;
    constexpr int KA = KT ? KT : kMaxKernels;
    constexpr int CA = CT ? CT : kMaxChannels;
    constexpr int PA = (NPT >= 0 ? NPT : kMaxPlanes) * KA;

    const int x = blockIdx.x * EP_TX + threadIdx.x;
    const int y = blockIdx.y * EP_TY + threadIdx.y;
    const bool valid = x < p.W && y < p.H;
    const size_t N = (size_t)p.H * p.W;
    const size_t i = (size_t)y * p.W + x;

    float acc[CA];
#pragma unroll
    for (int c = 0; c < CA; c++) acc[c] = 0.f;
    float anew[CA];

    if (valid) {
        float ph[PA > 0 ? PA : 1];
        bool alpha = true;
        const int npk = n_p * K;
#pragma unroll
        for (int pk = 0; pk < PA; pk++) {
            if (pk >= npk) break;
            const float* pl = p.P + (size_t)pk * N;
            float v;
            if (p.maintain) {
                float s = 0.f;
                int cnt = 0;
                const int r = p.r_diff;
                for (int dy = -r; dy <= r; dy++) {
                    const float* row = pl + (size_t)wrapi(y + dy, p.H) * p.W;
                    for (int dx = -r; dx <= r; dx++) {
                        if (dy * dy + dx * dx > r * r) continue;
                        const float q = __ldg(&row[wrapi(x + dx, p.W)]);
                        s += q;
                        cnt += q > p.eps_p;
                    }
                }
                v = 0.f;
                if (cnt > 0) v = fminf(fmaxf(s / (float)cnt, 0.f), 1.f);
                alpha = alpha && (v > p.eps_p);
            } else {
                v = __ldg(&pl[i]);
            }
            ph[pk] = v;
        }
        float g[KA];
        float hk[KA];
#pragma unroll
        for (int k = 0; k < KA; k++) {
            if (k >= K) break;
            const float u = __ldg(&p.U[(size_t)k * N + i]);
            const float m = p.p_mu >= 0 ? ph[p.p_mu * K + k] : p.kt.mu[k];
            const float sg = p.p_sigma >= 0 ? ph[p.p_sigma * K + k] : p.kt.sigma[k];
            const float hh = p.p_h >= 0 ? ph[p.p_h * K + k] : p.kt.h[k];
            float gk = 0.f;
            if (sg > 0.f) {
                const float z = (u - m) / sg;
                gk = expf(-0.5f * z * z);
            }
            if (p.maintain) {
                const float t = p.alpha_on ? u : hh * gk;
                alpha = alpha && (t > p.eps_u);
            }
            g[k] = gk;
            hk[k] = hh;
        }
        if (!p.maintain) alpha = true;
#pragma unroll
        for (int k = 0; k < KA; k++) {
            if (k >= K) break;
            const float gm = alpha ? g[k] : 0.f;
            const float hm = (p.p_h >= 0 && !alpha) ? 0.f : hk[k];
            const float G = p.growth_form == 0 ? hm * (2.f * gm - 1.f) : hm * gm;
            const int d = p.kt.dst[k];
#pragma unroll
            for (int c = 0; c < CA; c++)
                if (c == d) acc[c] += G;
        }
#pragma unroll
        for (int c = 0; c < CA; c++) {
            if (c >= C) break;
            const float a = __ldg(&p.A[(size_t)c * N + i]) + p.dt * acc[c];
            anew[c] = fminf(fmaxf(a, 0.f), 1.f);
            p.A_out[(size_t)c * N + i] = anew[c];
        }
        if (p.P_out) {
#pragma unroll
            for (int pk = 0; pk < PA; pk++) {
                if (pk >= npk) break;
                p.P_out[(size_t)pk * N + i] = (p.maintain && !alpha) ? 0.f : ph[pk];
            }
        }
        if (p.alpha_out) p.alpha_out[i] = alpha ? 1 : 0;
    }

    if (p.partials) {
        // five sums per channel, reduced warp by warp then across warps
        __shared__ float red[EP_TY][kMaxChannels * 5];
        const int lane = threadIdx.x;
        for (int c = 0; c < C; c++) {
            float a = valid ? anew[c] : 0.f;
            float sy = valid ? __ldg(&p.sin_y[y]) : 0.f, cy = valid ? __ldg(&p.cos_y[y]) : 0.f;
            float sx = valid ? __ldg(&p.sin_x[x]) : 0.f, cx = valid ? __ldg(&p.cos_x[x]) : 0.f;
            float v[5] = {a, a * sy, a * cy, a * sx, a * cx};
#pragma unroll
            for (int j = 0; j < 5; j++) {
                float t = v[j];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
                if (lane == 0) red[threadIdx.y][c * 5 + j] = t;
            }
        }
        __syncthreads();
        const int tid = threadIdx.y * EP_TX + threadIdx.x;
        if (tid < C * 5) {
            double s = 0.0;
            for (int w = 0; w < EP_TY; w++) s += (double)red[w][tid];
            const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
            p.partials[blk * C * 5 + tid] = s;
        }
    }
}

int epilogue_blocks(int H, int W)
{
    return ((W + EP_TX - 1) / EP_TX) * ((H + EP_TY - 1) / EP_TY);
}

cudaError_t launch_epilogue(const EpiParams& p, cudaStream_t s, int* n_blocks)
{
    dim3 grid((p.W + EP_TX - 1) / EP_TX, (p.H + EP_TY - 1) / EP_TY);
    dim3 block(EP_TX, EP_TY);
    if (n_blocks) *n_blocks = grid.x * grid.y;
    const int K = p.kt.K, C = p.kt.C;
    if (K == 1 && C == 1 && p.n_p == 2) k_epilogue<1, 1, 2><<<grid, block, 0, s>>>(p);
    else if (K == 1 && C == 1 && p.n_p == 0) k_epilogue<1, 1, 0><<<grid, block, 0, s>>>(p);
    else if (K == 15 && C == 3 && p.n_p == 2) k_epilogue<15, 3, 2><<<grid, block, 0, s>>>(p);
    else if (K == 15 && C == 3 && p.n_p == 0) k_epilogue<15, 3, 0><<<grid, block, 0, s>>>(p);
    else k_epilogue<0, 0, -1><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- statistics
// Block partials of (sum A, sum A sin(2 pi y/H), sum A cos(2 pi y/H), sum A
// sin(2 pi x/W), sum A cos(2 pi x/W)) per channel, same tiling and reduction
// order as the epilogue.
__global__ void __launch_bounds__(256) k_stats_partials(const float* A, int C, int H, int W,
                                                        const float* sin_y, const float* cos_y,
                                                        const float* sin_x, const float* cos_x,
                                                        double* partials)
{
    __shared__ float red[EP_TY][kMaxChannels * 5];
    const int x = blockIdx.x * EP_TX + threadIdx.x;
    const int y = blockIdx.y * EP_TY + threadIdx.y;
    const bool valid = x < W && y < H;
    const int lane = threadIdx.x;
    for (int c = 0; c < C; c++) {
        float a = valid ? __ldg(&A[((size_t)c * H + y) * W + x]) : 0.f;
        float sy = valid ? __ldg(&sin_y[y]) : 0.f, cy = valid ? __ldg(&cos_y[y]) : 0.f;
        float sx = valid ? __ldg(&sin_x[x]) : 0.f, cx = valid ? __ldg(&cos_x[x]) : 0.f;
        float v[5] = {a, a * sy, a * cy, a * sx, a * cx};
#pragma unroll
        for (int j = 0; j < 5; j++) {
            float t = v[j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
            if (lane == 0) red[threadIdx.y][c * 5 + j] = t;
        }
    }
    __syncthreads();
    const int tid = threadIdx.y * EP_TX + threadIdx.x;
    if (tid < C * 5) {
        double s = 0.0;
        for (int w = 0; w < EP_TY; w++) s += (double)red[w][tid];
        const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        partials[blk * C * 5 + tid] = s;
    }
}

cudaError_t launch_stats_partials(const float* A, int C, int H, int W, const float* sin_y,
                                  const float* cos_y, const float* sin_x, const float* cos_x,
                                  double* partials, cudaStream_t s, int* n_blocks)
{
    dim3 grid((W + EP_TX - 1) / EP_TX, (H + EP_TY - 1) / EP_TY);
    if (n_blocks) *n_blocks = grid.x * grid.y;
    k_stats_partials<<<grid, dim3(EP_TX, EP_TY), 0, s>>>(A, C, H, W, sin_y, cos_y, sin_x, cos_x, partials);
    return cudaGetLastError();
}

// Final reduction: one block; thread t sums blocks t, t+256, ... in FP64, then
// a fixed tree.  out[c] = (mass, centre y, centre x), centres from the
// circular mean atan2(sum A sin, sum A cos) scaled to [0, n).
__global__ void __launch_bounds__(256) k_stats_final(const double* partials, int n_blocks, int C,
                                                     int H, int W, float* out)
{
    __shared__ double red[256];
    __shared__ double tot[kMaxChannels * 5];
    for (int v = 0; v < C * 5; v++) {
        double s = 0.0;
        for (int b = threadIdx.x; b < n_blocks; b += 256) s += partials[(size_t)b * C * 5 + v];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) tot[v] = red[0];
        __syncthreads();
    }
    if (threadIdx.x < C) {
        const int c = threadIdx.x;
        const double two_pi = 6.283185307179586476925286766559;
        const double m = tot[c * 5 + 0];
        double ty = atan2(tot[c * 5 + 1], tot[c * 5 + 2]) * H / two_pi;
        double tx = atan2(tot[c * 5 + 3], tot[c * 5 + 4]) * W / two_pi;
        if (ty < 0.0) ty += H;
        if (tx < 0.0) tx += W;
        out[c * 3 + 0] = (float)m;
        out[c * 3 + 1] = (float)ty;
        out[c * 3 + 2] = (float)tx;
    }
}

cudaError_t launch_stats_final(const double* partials, int n_blocks, int C, int H, int W,
                               float* out, cudaStream_t s)
{
    k_stats_final<<<1, 256, 0, s>>>(partials, n_blocks, C, H, W, out);
    return cudaGetLastError();
}

}  // namespace lenia
