// Direct periodic convolution, the fused growth / gene-maintenance / update
// epilogue, and per-channel statistics (arXiv 2304.05639, Sections 2.1-2.4,
// Algorithm 2).
#include <math.h>
#include <string.h>

#include <mutex>
#include <utility>
#include <vector>

#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

// Periodic index for any integer i (modulo; used off the per-site hot loops).
__device__ __forceinline__ int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// ------------------------------------------------------- direct convolution
// U_k(y, x) = sum_d K~_k(d) A_src(k)(y + d, x + d), periodic (K~ is point
// symmetric, so this is the convolution K~ * A).  A block of 32 x 8 threads
// computes a (32 CX) x (8 RY) output tile of one kernel (grid z runs over the
// kernels, so that small worlds still fill the GPU); thread (tx, ty) owns
// columns tx + 32 j (j < CX, so that a warp's shared loads are contiguous)
// and rows RY ty .. RY ty + RY - 1 of its tile.  The input tile with its R
// halo is staged in shared memory: by one tiled TMA box (the mbarrier wait is
// bounded) when it lies inside the world, else - at the torus edges, where it
// wraps - by plain loads.  Box columns start at a multiple of 4 floats (16
// bytes), so the tile carries up to 3 extra columns on the left: `off`.  For
// each tap column dx the thread slides an RY-row register window down the
// non-zero taps of that column: per tap, CX shared loads and one weight load
// feed CX x RY fused multiply-adds.
template <int CX, int RY>
struct DcTile {
    static constexpr int TW = 32 * CX, TH = 8 * RY;
    __host__ __device__ static constexpr int pitch(int maxR) { return (TW + 2 * maxR + 3 + 3) / 4 * 4; }
    __host__ __device__ static constexpr int rows(int maxR) { return TH + 2 * maxR; }
    static size_t smem(int maxR) { return (size_t)pitch(maxR) * rows(maxR) * sizeof(float) + 128; }
};

template <int CX, int RY>
__global__ void __launch_bounds__(256) k_direct_conv(ConvParams p, int maxR, const __grid_constant__ CUtensorMap tm_a)
{
    pdl_enter();
    using T = DcTile<CX, RY>;
    extern __shared__ __align__(128) unsigned char dc_raw[];
    float* tile = reinterpret_cast<float*>(dc_raw + ((128 - (smem_addr(dc_raw) & 127)) & 127));
    __shared__ __align__(8) uint64_t bar;
    // grid z enumerates (channel, kernel of that channel) pairs
    int c = 0, t = blockIdx.z;
    while (c < p.C - 1 && t >= p.kcount[c]) t -= p.kcount[c++];
    const int k = p.klist[c][t];
    const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
    const int pitch = T::pitch(maxR), rows = T::rows(maxR);
    const int xs = (x0 - maxR) & ~3;                 // first staged column (may be negative)
    const int off = x0 - maxR - xs;                  // 0..3
    const int ys = y0 - maxR;
    const bool inside = p.tma && xs >= 0 && xs + pitch <= p.W && ys >= 0 && ys + rows <= p.H;
    const float* A = p.A + (size_t)c * p.H * p.W;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (inside) {
        if (tid == 0) {
            mbar_init(&bar, 1);
            mbar_fence_init();
            mbar_arrive_expect_tx(&bar, (uint32_t)(pitch * rows * 4));
            tma_load_3d(tile, &tm_a, xs, ys, c, &bar);
        }
        __syncthreads();
        if (!__syncthreads_and(mbar_wait_bounded(&bar, 0))) {
            if (tid == 0) {
                atomicExch(p.status, kStatusWaitTimeout);
                mbar_wait_bounded(&bar, 0);
            }
            return;
        }
    } else {
        for (int u = tid; u < rows * pitch; u += 256) {
            const int ty = u / pitch, tx = u % pitch;
            tile[u] = __ldg(&A[(size_t)wrapi(ys + ty, p.H) * p.W + wrapi(xs + tx, p.W)]);
        }
        __syncthreads();
    }
    const int tx = threadIdx.x;
    const int ty = threadIdx.y * RY;
    const int R = p.R[k];
    const float* w = p.w + p.w_off[k];       // [dx + R][dy + R]
    const int* yr = p.yr + p.yr_off[k];
    float acc[CX][RY];
#pragma unroll
    for (int j = 0; j < CX; j++)
#pragma unroll
        for (int o = 0; o < RY; o++) acc[j][o] = 0.f;
    for (int dx = -R; dx <= R; dx++) {
        const int r = __ldg(&yr[dx + R]);
        if (r < 0) continue;
        const float* col = tile + (size_t)(ty + maxR) * pitch + (tx + off + maxR + dx);
        const float* wc = w + (dx + R) * (2 * R + 1) + R;
        float v[CX][RY];
#pragma unroll
        for (int j = 0; j < CX; j++)
#pragma unroll
            for (int o = 0; o < RY - 1; o++) v[j][o] = col[(o - r) * pitch + 32 * j];
#pragma unroll 4
        for (int dy = -r; dy <= r; dy++) {
            const float wv = __ldg(&wc[dy]);
#pragma unroll
            for (int j = 0; j < CX; j++) {
                v[j][RY - 1] = col[(dy + RY - 1) * pitch + 32 * j];
#pragma unroll
                for (int o = 0; o < RY; o++) acc[j][o] = fmaf(wv, v[j][o], acc[j][o]);
#pragma unroll
                for (int o = 0; o < RY - 1; o++) v[j][o] = v[j][o + 1];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CX; j++) {
        const int x = x0 + tx + 32 * j;
        if (x >= p.W) continue;
#pragma unroll
        for (int o = 0; o < RY; o++) {
            const int y = y0 + ty + o;
            if (y < p.H) p.U[((size_t)k * p.H + y) * p.W + x] = acc[j][o];
        }
    }
}

// Tensor map of a phenospace [C][H][W] (FP32) with boxes of the direct
// convolution's staged tile; cached by argument.
static bool dc_map(CUtensorMap* out, const float* base, int W, int H, int C, int bx, int by)
{
    struct Key {
        const void* base;
        int W, H, C, bx, by;
        bool operator==(const Key& o) const
        {
            return base == o.base && W == o.W && H == o.H && C == o.C && bx == o.bx && by == o.by;
        }
    };
    static std::mutex mu;
    static std::vector<std::pair<Key, CUtensorMap>> cache;
    const Key key{base, W, H, C, bx, by};
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : cache)
        if (e.first == key) {
            *out = e.second;
            return true;
        }
    auto fn = tensor_map_encoder();
    if (!fn || ((uintptr_t)base & 15) != 0 || W % 4 != 0 || bx > 256 || by > 256) return false;
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)C};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 4, (cuuint64_t)W * H * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cache.insert(cache.begin(), {key, m});
    if (cache.size() > 32) cache.pop_back();
    *out = m;
    return true;
}

template <int CX, int RY>
static cudaError_t launch_dc(const ConvParams& p, int max_R, int planes, cudaStream_t s)
{
    using T = DcTile<CX, RY>;
    const size_t smem = T::smem(max_R);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = smem_limit<k_direct_conv<CX, RY>>(smem);
    if (e != cudaSuccess) return e;
    ConvParams q = p;
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    const int pitch = T::pitch(max_R), rows = T::rows(max_R);
    // worlds too narrow or short for an interior tile use plain loads only
    q.tma = p.W >= pitch && p.H >= rows && dc_map(&tm, p.A, p.W, p.H, p.C, pitch, rows);
    dim3 grid((p.W + T::TW - 1) / T::TW, (p.H + T::TH - 1) / T::TH, planes);
    launch_pdl(k_direct_conv<CX, RY>, grid, dim3(32, 8), smem, s, q, max_R, tm);
    return cudaGetLastError();
}

// 64 x 64 tiles (2 x 8 outputs per thread) when they give at least two blocks
// per SM, else 32 x 32 (1 x 4) or 32 x 16 (1 x 2) tiles for parallelism.
cudaError_t launch_direct_conv(const ConvParams& p, int max_R, cudaStream_t s)
{
    int planes = 0;
    for (int c = 0; c < p.C; c++) planes += p.kcount[c];
    if (planes == 0) return cudaSuccess;
    static int n_sms = 0;
    if (n_sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n_sms = 148;
    }
    auto blocks = [&](int tw, int th) { return (long long)((p.W + tw - 1) / tw) * ((p.H + th - 1) / th) * planes; };
    if (blocks(64, 64) >= 2LL * n_sms && DcTile<2, 8>::smem(max_R) <= 200 * 1024)
        return launch_dc<2, 8>(p, max_R, planes, s);
    if (blocks(32, 32) >= 2LL * n_sms) return launch_dc<1, 4>(p, max_R, planes, s);
    return launch_dc<1, 2>(p, max_R, planes, s);
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
//     G = 2g - 1 (signed) or g (paper form).  Where alpha = 0 the sum is the
//     per-channel constant acc0 computed on the host.
// Optional per-block stats partials: sum A, sum A sin/cos(2 pi y/H), sum A
// sin/cos(2 pi x/W) per channel, reduced in a fixed order.
constexpr int EP_TX = 32, EP_TY = 8, EP_RY = 4;    // block: 32 x 8 threads, 4 rows each

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Block reduction of per-thread stats (CA channels x 5 sums) into one record
// per block (compensated pairs, warp order); every thread of the block must
// call it.
template <int CA>
__device__ __forceinline__ void block_stats(const float* st, int C, float2* partials)
{
    __shared__ float red[EP_TY][kMaxChannels * 5];
    const int lane = threadIdx.x;
#pragma unroll
    for (int v = 0; v < CA * 5; v++) {
        if (v >= C * 5) break;
        float t = st[v];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
        if (lane == 0) red[threadIdx.y][v] = t;
    }
    __syncthreads();
    const int tid = threadIdx.y * EP_TX + threadIdx.x;
    if (tid < C * 5) {
        float2 s = make_float2(0.f, 0.f);
        for (int w = 0; w < EP_TY; w++) s = ff_add(s, make_float2(red[w][tid], 0.f));
        const size_t blk = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        partials[blk * C * 5 + tid] = s;
    }
}

// Fast path: diffusion radius 1 (the 5-site plus), compile-time kernel count,
// channel count and gene layout.  Each thread owns one column x and rows
// y0 + 8 j (j < EP_RY); wrapped neighbour indices are formed once per row.
template <int KT, int CT, int LOC, int RY = EP_RY>
__global__ void __launch_bounds__(256, 3) k_epilogue_r1(EpiParams p)
{
    pdl_enter();
    constexpr int NP = ((LOC & 1) != 0) + ((LOC & 2) != 0) + ((LOC & 4) != 0);
    constexpr int PMU = (LOC & 1) ? 0 : -1;
    constexpr int PSG = (LOC & 2) ? ((LOC & 1) ? 1 : 0) : -1;
    constexpr int PH = (LOC & 4) ? NP - 1 : -1;
    constexpr int NPK = NP * KT;
    const int H = p.H, W = p.W;
    const size_t N = (size_t)H * W;
    const int x = blockIdx.x * EP_TX + threadIdx.x;
    const bool xin = x < W;
    const int xc = xin ? x : W - 1;
    const int xm = xc == 0 ? W - 1 : xc - 1;
    const int xp = xc == W - 1 ? 0 : xc + 1;
    const float eps_p = p.eps_p, eps_u = p.eps_u;
    // world blockIdx.z of a batched launch (lists set), else the single world
    const int wz = blockIdx.z;
    const float* pA = p.A_list ? p.A_list[wz] : p.A;
    const float* pP = p.P_list ? p.P_list[wz] : p.P;
    float* pAo = p.Aout_list ? p.Aout_list[wz] : p.A_out;
    float* pPo = p.Pout_list ? p.Pout_list[wz] : p.P_out;
    const float* pU = p.U + (size_t)wz * p.u_stride;

    float st[CT * 5];
#pragma unroll
    for (int v = 0; v < CT * 5; v++) st[v] = 0.f;

    for (int j = 0; j < RY; j++) {
        const int y = blockIdx.y * (EP_TY * RY) + j * EP_TY + threadIdx.y;
        if (y >= H) break;
        const size_t rc = (size_t)y * W;
        const size_t ru = (size_t)(y == 0 ? H - 1 : y - 1) * W;
        const size_t rd = (size_t)(y == H - 1 ? 0 : y + 1) * W;
        const size_t i = rc + xc;

        float ph[NPK > 0 ? NPK : 1];
        bool alpha = true;
#pragma unroll
        for (int pk = 0; pk < NPK; pk++) {
            const float* pl = pP + (size_t)pk * N;
            if (p.maintain) {
                // disk |d| <= 1 in the order (-1,0), (0,-1), (0,0), (0,1), (1,0)
                const float v0 = __ldg(pl + ru + xc);
                const float v1 = __ldg(pl + rc + xm);
                const float v2 = __ldg(pl + rc + xc);
                const float v3 = __ldg(pl + rc + xp);
                const float v4 = __ldg(pl + rd + xc);
                const float s = (((v0 + v1) + v2) + v3) + v4;
                const int n = (v0 > eps_p) + (v1 > eps_p) + (v2 > eps_p) + (v3 > eps_p) + (v4 > eps_p);
                const float v = n > 0 ? fminf(fmaxf(s / (float)n, 0.f), 1.f) : 0.f;
                alpha = alpha && (v > eps_p);
                ph[pk] = v;
            } else {
                ph[pk] = __ldg(pl + i);
            }
        }
        float acc[CT];
        float tsum = 0.f;                  // sum of the alpha tests (Delta_sum)
#pragma unroll
        for (int c = 0; c < CT; c++) acc[c] = 0.f;
#pragma unroll
        for (int k = 0; k < KT; k++) {
            const float u = __ldg(&pU[(size_t)k * N + i]);
            const float m = PMU >= 0 ? ph[(PMU >= 0 ? PMU : 0) * KT + k] : p.kt.mu[k];
            const float sg = PSG >= 0 ? ph[(PSG >= 0 ? PSG : 0) * KT + k] : p.kt.sigma[k];
            const float hh = PH >= 0 ? ph[(PH >= 0 ? PH : 0) * KT + k] : p.kt.h[k];
            float gk = 0.f;
            if (sg > 0.f) {
                const float z = (u - m) / sg;
                gk = expf(-0.5f * z * z);
            }
            const float t = p.alpha_on ? u : hh * gk;
            tsum += t;
            if (p.maintain) alpha = alpha && (t > eps_u);
            const float G = p.growth_form == 0 ? hh * (2.f * gk - 1.f) : hh * gk;
            const int d = p.kt.dst[k];
#pragma unroll
            for (int c = 0; c < CT; c++)
                if (c == d) acc[c] += G;
        }
        if (!p.maintain) alpha = true;
        if (xin) {
#pragma unroll
            for (int c = 0; c < CT; c++) {
                const float a = __ldg(&pA[(size_t)c * N + i]) + p.dt * (alpha ? acc[c] : p.acc0[c]);
                const float an = fminf(fmaxf(a, 0.f), 1.f);
                pAo[(size_t)c * N + i] = an;
                if (p.partials) {
                    const float sy = __ldg(&p.sin_y[y]), cy = __ldg(&p.cos_y[y]);
                    const float sx = __ldg(&p.sin_x[x]), cx = __ldg(&p.cos_x[x]);
                    st[c * 5 + 0] += an;
                    st[c * 5 + 1] += an * sy;
                    st[c * 5 + 2] += an * cy;
                    st[c * 5 + 3] += an * sx;
                    st[c * 5 + 4] += an * cx;
                }
            }
            if (pPo) {
#pragma unroll
                for (int pk = 0; pk < NPK; pk++)
                    pPo[(size_t)pk * N + i] = (p.maintain && !alpha) ? 0.f : ph[pk];
            }
            if (p.alpha_out) p.alpha_out[i] = alpha ? 1 : 0;
            if (p.empty_out) p.empty_out[i] = tsum > eps_u ? 0 : 1;
        }
    }
    if (p.partials) block_stats<CT>(st, CT, p.partials);
}

// Potential of kernel k at site i from the ring potentials (Section 2.4):
//   k_r = sum_i b_i exp(-(r/n - r_i)^2 / (2 w_i^2))  (a term is 0 where w_i <= 0),
//   U = sum_r k_r (K_r * A_src) / sum_r k_r (K_r * 1),  0 where the denominator is <= 0,
// with the site's diffused kernel genes ph (planes p_kern .. p_kern + 5).
__device__ float ring_potential(const EpiParams& p, const float* ph, int K, int k, size_t i, size_t N)
{
    const int kb = p.p_kern;
    const float r1 = ph[(kb + 0) * K + k], w1 = ph[(kb + 1) * K + k], b1 = ph[(kb + 2) * K + k];
    const float r2 = ph[(kb + 3) * K + k], w2 = ph[(kb + 4) * K + k], b2 = ph[(kb + 5) * K + k];
    const bool on1 = w1 > 0.f, on2 = w2 > 0.f;
    const float c1 = on1 ? 0.5f / (w1 * w1) : 0.f, c2 = on2 ? 0.5f / (w2 * w2) : 0.f;
    const int n = p.n_rings;
    const float* V = p.U + (size_t)p.kt.src[k] * n * N + i;
    float num = 0.f, den = 0.f;
    for (int r = 0; r < n; r++) {
        const float x = (float)r / (float)n;
        const float d1 = x - r1, d2 = x - r2;
        const float kr = (on1 ? b1 * expf(-(d1 * d1) * c1) : 0.f) + (on2 ? b2 * expf(-(d2 * d2) * c2) : 0.f);
        num = fmaf(kr, __ldg(V + (size_t)r * N), num);
        den = fmaf(kr, p.ring_cnt[r], den);
    }
    return den > 0.f ? num / den : 0.f;
}

// General path: any diffusion radius, kernel count, channel count and gene
// layout, and the ring decomposition (runtime loops; per-site arrays may
// live in local memory).
__global__ void __launch_bounds__(256) k_epilogue_generic(EpiParams p)
{
    pdl_enter();
    const int K = p.kt.K, C = p.kt.C, n_p = p.n_p;
    const int H = p.H, W = p.W;
    const size_t N = (size_t)H * W;
    const int x = blockIdx.x * EP_TX + threadIdx.x;
    const bool xin = x < W;
    const int xc = xin ? x : W - 1;
    const int r = p.r_diff;
    float st[kMaxChannels * 5];
    for (int v = 0; v < kMaxChannels * 5; v++) st[v] = 0.f;

    for (int j = 0; j < EP_RY; j++) {
        const int y = blockIdx.y * (EP_TY * EP_RY) + j * EP_TY + threadIdx.y;
        if (y >= H) break;
        const size_t i = (size_t)y * W + xc;
        float ph[kMaxPlanes * kMaxKernels];
        bool alpha = true;
        const int npk = n_p * K;
        for (int pk = 0; pk < npk; pk++) {
            const float* pl = p.P + (size_t)pk * N;
            float v;
            if (p.maintain) {
                float s = 0.f;
                int cnt = 0;
                for (int dy = -r; dy <= r; dy++) {
                    const float* row = pl + (size_t)wrap1(y + dy, H) * W;
                    for (int dx = -r; dx <= r; dx++) {
                        if (dy * dy + dx * dx > r * r) continue;
                        const float q = __ldg(&row[wrap1(xc + dx, W)]);
                        s += q;
                        cnt += q > p.eps_p;
                    }
                }
                v = cnt > 0 ? fminf(fmaxf(s / (float)cnt, 0.f), 1.f) : 0.f;
                alpha = alpha && (v > p.eps_p);
            } else {
                v = __ldg(&pl[i]);
            }
            ph[pk] = v;
        }
        float acc[kMaxChannels];
        float tsum = 0.f;                  // sum of the alpha tests (Delta_sum)
        for (int c = 0; c < C; c++) acc[c] = 0.f;
        for (int k = 0; k < K; k++) {
            const float u = p.n_rings > 0 ? ring_potential(p, ph, K, k, i, N) : __ldg(&p.U[(size_t)k * N + i]);
            const float m = p.p_mu >= 0 ? ph[p.p_mu * K + k] : p.kt.mu[k];
            const float sg = p.p_sigma >= 0 ? ph[p.p_sigma * K + k] : p.kt.sigma[k];
            const float hh = p.p_h >= 0 ? ph[p.p_h * K + k] : p.kt.h[k];
            float gk = 0.f;
            if (sg > 0.f) {
                const float z = (u - m) / sg;
                gk = expf(-0.5f * z * z);
            }
            const float t = p.alpha_on ? u : hh * gk;
            tsum += t;
            if (p.maintain) alpha = alpha && (t > p.eps_u);
            acc[p.kt.dst[k]] += p.growth_form == 0 ? hh * (2.f * gk - 1.f) : hh * gk;
        }
        if (!p.maintain) alpha = true;
        if (xin) {
            for (int c = 0; c < C; c++) {
                const float a = __ldg(&p.A[(size_t)c * N + i]) + p.dt * (alpha ? acc[c] : p.acc0[c]);
                const float an = fminf(fmaxf(a, 0.f), 1.f);
                p.A_out[(size_t)c * N + i] = an;
                if (p.partials) {
                    st[c * 5 + 0] += an;
                    st[c * 5 + 1] += an * __ldg(&p.sin_y[y]);
                    st[c * 5 + 2] += an * __ldg(&p.cos_y[y]);
                    st[c * 5 + 3] += an * __ldg(&p.sin_x[x]);
                    st[c * 5 + 4] += an * __ldg(&p.cos_x[x]);
                }
            }
            if (p.P_out)
                for (int pk = 0; pk < npk; pk++)
                    p.P_out[(size_t)pk * N + i] = (p.maintain && !alpha) ? 0.f : ph[pk];
            if (p.alpha_out) p.alpha_out[i] = alpha ? 1 : 0;
            if (p.empty_out) p.empty_out[i] = tsum > p.eps_u ? 0 : 1;
        }
    }
    if (p.partials) block_stats<kMaxChannels>(st, C, p.partials);
}

// Ring decomposition fast path (Section 2.4): diffusion radius 1, compile-time
// kernel and channel counts, ring count and gene layout; one site per thread
// (32 x 8 sites per block).  Kernels are taken in order of their source
// channel; each kernel's NP gene planes over the block's tile with a one-site
// halo (RG_TILE_H x RG_TILE_W) are copied into shared memory with cp.async
// while the previous kernel is computed (double buffer), and the 5-point
// diffusion reads them there.  The kernel's ring weights come from its
// diffused kernel genes with the hardware base-2 exponential,
// k_r = sum_i b_i 2^(-(r/n - r_i)^2 log2(e) / (2 w_i^2)), and its potential
// from the channel's ring potentials, which each thread copies for its own
// site with cp.async into dynamic shared memory (n_rings x 256 floats) once
// per channel, right after the previous channel's last use.  The maintained genes are written as soon as they are diffused;
// a site that ends without alpha rewrites them with zeros.  Needs
// W >= RG_TILE_W and H >= RG_TILE_H (one wrap per halo coordinate).
// One Gaussian bump's share of a ring-recombined potential (Section 2.4):
// adds w_r V_r and w_r |K_r| over the NR rings to num and den, with
// w_r = b exp(-(r/NR - c)^2 / (2 w^2)) (nothing where w <= 0).  With
// x_r = r / NR equally spaced (D = 1/NR), the base-2 exponent
// L(r) = a (x_r - c)^2, a = -log2(e) / (2 w^2) <= 0, steps by
// L(r + 1) - L(r) = a D (D + 2 (x_r - c)), itself growing by 2 a D^2 per ring:
//   w_{r+1} = w_r q_r,  q_{r+1} = q_r s,  s = 2^(2 a D^2)   (walking up),
//   w_{r-1} = w_r q'_r, q'_{r-1} = q'_r s                   (walking down),
// so four exponentials per bump replace one per ring.  The walks start at
// the ring nearest c (w there is the bump's largest) and go outwards, where
// every ratio is <= 1: no value overflows, an underflow only cuts off a
// decaying tail, and the rounding of the products grows with the distance
// from the peak, where the weights are small.  A walk stops once its weight
// falls below 2^-40 of the peak's (its remaining terms are below FP32
// resolution of the sums).  The four exponentials are the accurate exp2f,
// since their rounding is carried along each walk.
// Each walk takes its rings in pairs on packed FP32 pairs (sm_100 family
// f32x2 instructions): {w_r, w_(r+1)} steps by {q_r q_(r+1), q_(r+1) q_(r+2)},
// which itself steps by s^4, and two partial sums per accumulator (num and
// den are the sums of the pairs' halves) -- two multiplies and two
// multiply-adds per pair of rings instead of eight scalar operations; a
// pair is taken while its first (larger) weight is at least the stop value.
template <int NR>
__device__ __forceinline__ void ring_walk(float e0, float q0, float s, float stop, int r0, int step,
                                          const float* v, const float* cnt, float2& num, float2& den)
{
    float2 E = make_float2(e0, e0 * q0);
    const float qs = q0 * q0 * s;
    float2 Q = make_float2(qs, qs * s * s);
    const float s4 = (s * s) * (s * s);
    const float2 S4 = make_float2(s4, s4);
    int r = r0;
    for (; r + step >= 0 && r + step < NR && E.x >= stop; r += 2 * step) {
        num = __ffma2_rn(E, make_float2(v[r * 256], v[(r + step) * 256]), num);
        den = __ffma2_rn(E, make_float2(cnt[r], cnt[r + step]), den);
        E = __fmul2_rn(E, Q);
        Q = __fmul2_rn(Q, S4);
    }
    if (r >= 0 && r < NR && E.x >= stop) {
        num.x = fmaf(E.x, v[r * 256], num.x);
        den.x = fmaf(E.x, cnt[r], den.x);
    }
}

template <int NR>
__device__ __forceinline__ void ring_bump(float c, float w, float b, const float* v, const float* cnt,
                                          float2& num, float2& den)
{
    if (!(w > 0.f) || b == 0.f) return;
    constexpr float LOG2E = 1.4426950408889634f;
    constexpr float D = 1.f / (float)NR;
    const float a = -0.5f * LOG2E / (w * w);
    int rs = __float2int_rn(c * (float)NR);
    rs = rs < 0 ? 0 : (rs > NR - 1 ? NR - 1 : rs);
    const float d = (float)rs * D - c;
    const float e0 = b * exp2f(a * (d * d));
    const float aD = a * D;
    const float s = exp2f(2.f * aD * D);
    const float stop = e0 * 9.094947e-13f;             // 2^-40 of the peak weight
    // up from the peak ring, then down from the ring below it
    ring_walk<NR>(e0, exp2f(aD * (D + 2.f * d)), s, stop, rs, 1, v, cnt, num, den);
    const float qd = exp2f(aD * (D - 2.f * d));
    ring_walk<NR>(e0 * qd, qd * s, s, stop, rs - 1, -1, v, cnt, num, den);
}

constexpr int RG_TY = 8;     // rows per block of the ring epilogue (one site per thread)
constexpr int RG_TILE_W = EP_TX + 2, RG_TILE_H = RG_TY + 2;

// Three blocks per SM (72 registers): 0.2585 ms on the paper's configuration
// against 0.2613 at four blocks (64 registers) and 0.2592 at two (80); gene
// tiles three buffers deep (two kernels ahead) measured 0.2608.
template <int KT, int CT, int NR, int LOC>
__global__ void __launch_bounds__(256, 3) k_epilogue_rings(EpiParams p)
{
    pdl_enter();
    constexpr int NG = ((LOC & 1) != 0) + ((LOC & 2) != 0) + ((LOC & 4) != 0);
    constexpr int NP = NG + 6;
    constexpr int PMU = (LOC & 1) ? 0 : -1;
    constexpr int PSG = (LOC & 2) ? ((LOC & 1) ? 1 : 0) : -1;
    constexpr int PH = (LOC & 4) ? NG - 1 : -1;
    constexpr int PK = NG;
    constexpr float LOG2E = 1.4426950408889634f;
    constexpr int TP = RG_TILE_H * RG_TILE_W;           // floats per staged plane
    __shared__ float tile[2][NP * TP];
    __shared__ int ord[KT];
    __shared__ float cnt_s[NR];
    extern __shared__ float vst[];                      // [NR][256]: each thread's own ring potentials
    const int H = p.H, W = p.W;
    const size_t N = (size_t)H * W;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * EP_TX, y0 = blockIdx.y * RG_TY;
    const int x = x0 + tx;
    const int y = y0 + ty;
    const bool in = x < W && y < H;
    const int xc = x < W ? x : W - 1, yc = y < H ? y : H - 1;
    const float eps_p = p.eps_p, eps_u = p.eps_u;
    const size_t i = (size_t)yc * W + xc;
    // this thread's staged elements: tile rows ty (and 8 + ty for ty < 2),
    // tile columns tx (and 32 + tx for tx < 2), as wrapped global offsets
    auto wrapx = [&](int v) { return v < 0 ? v + W : (v >= W ? v - W : v); };
    auto wrapy = [&](int v) { return v < 0 ? v + H : (v >= H ? v - H : v); };
    const size_t g_r0 = (size_t)wrapy(y0 - 1 + ty) * W;
    const size_t g_r1 = (size_t)wrapy(y0 + RG_TY - 1 + ty) * W;
    const int g_c0 = wrapx(x0 - 1 + tx), g_c1 = wrapx(x0 + EP_TX - 1 + tx);
    const bool hr = ty < RG_TILE_H - RG_TY, hc = tx < RG_TILE_W - EP_TX;
    auto stage = [&](int k, float* buf) {
#pragma unroll
        for (int pp = 0; pp < NP; pp++) {
            const float* base = p.P + (size_t)(pp * KT + k) * N;
            float* t = buf + pp * TP;
            cp_async4(&t[ty * RG_TILE_W + tx], base + g_r0 + g_c0);
            if (hc) cp_async4(&t[ty * RG_TILE_W + EP_TX + tx], base + g_r0 + g_c1);
            if (hr) {
                cp_async4(&t[(RG_TY + ty) * RG_TILE_W + tx], base + g_r1 + g_c0);
                if (hc) cp_async4(&t[(RG_TY + ty) * RG_TILE_W + EP_TX + tx], base + g_r1 + g_c1);
            }
        }
        cp_async_commit();
    };
    // kernels in order of their source channel (the order of the sums below)
    if (ty == 0)
        for (int r = tx; r < NR; r += EP_TX) cnt_s[r] = p.ring_cnt[r];
    if (tx == 0 && ty == 0) {
        int n = 0;
        for (int c = 0; c < CT; c++)
            for (int k = 0; k < KT; k++)
                if (p.kt.src[k] == c) ord[n++] = k;
    }
    __syncthreads();
    const int tid = ty * EP_TX + tx;
    // the thread's own ring potentials of one channel (no block barrier needed:
    // the thread that copies them is the one that reads them)
    auto stage_v = [&](int c) {
        const float* Vc = p.U + (size_t)c * NR * N + i;
#pragma unroll
        for (int r = 0; r < NR; r++) cp_async4(&vst[r * 256 + tid], Vc + (size_t)r * N);
        cp_async_commit();
    };
    stage_v(p.kt.src[ord[0]]);
    stage(ord[0], tile[0]);

    bool alpha = true;
    bool wrote_nz = false;         // a non-zero gene value was stored before alpha was known
    float tsum = 0.f;
    float acc[CT];
#pragma unroll
    for (int c = 0; c < CT; c++) acc[c] = 0.f;
    const int o = (ty + 1) * RG_TILE_W + tx + 1;        // the site in the tile
#pragma unroll 1
    for (int j = 0; j < KT; j++) {
        const int k = ord[j];
        const int c = p.kt.src[k];
        cp_async_wait_all();
        __syncthreads();            // kernel j staged; every thread is done with kernel j - 1's buffer
        if (j + 1 < KT) stage(ord[j + 1], tile[(j + 1) & 1]);
        const float* T = tile[j & 1];
        float g[NP];
#pragma unroll
        for (int pp = 0; pp < NP; pp++) {
            const float* t = T + pp * TP;
            float val;
            if (p.maintain) {
                // disk |d| <= 1 in the order (-1,0), (0,-1), (0,0), (0,1), (1,0)
                const float v0 = t[o - RG_TILE_W], v1 = t[o - 1], v2 = t[o], v3 = t[o + 1], v4 = t[o + RG_TILE_W];
                const float sm = (((v0 + v1) + v2) + v3) + v4;
                const float n = (float)(v0 > eps_p) + (float)(v1 > eps_p) + (float)(v2 > eps_p) +
                                (float)(v3 > eps_p) + (float)(v4 > eps_p);
                val = n > 0.f ? __saturatef(sm * rcp_approx(n)) : 0.f;
            } else {
                val = t[o];
            }
            alpha = alpha && (!p.maintain || val > eps_p);
            g[pp] = val;
        }
        // the kernel's maintained genes go out now, while they are in
        // registers (zeros once alpha is known false); a site that ends
        // without alpha rewrites its planes with zeros below
        if (in && p.P_out) {
#pragma unroll
            for (int pp = 0; pp < NP; pp++) {
                const float val = alpha ? g[pp] : 0.f;
                wrote_nz = wrote_nz || val != 0.f;
                p.P_out[(size_t)(pp * KT + k) * N + i] = val;
            }
        }
        // ring weights and the potential: each bump's weights over the rings,
        // walked outwards from its peak ring (recurrence below), summed
        // against the channel's ring potentials staged in shared memory
        float2 num2 = make_float2(0.f, 0.f), den2 = make_float2(0.f, 0.f);
        ring_bump<NR>(g[PK + 0], g[PK + 1], g[PK + 2], vst + tid, cnt_s, num2, den2);
        ring_bump<NR>(g[PK + 3], g[PK + 4], g[PK + 5], vst + tid, cnt_s, num2, den2);
        const float num = num2.x + num2.y, den = den2.x + den2.y;
        // the channel's last kernel: fetch the next channel's potentials now
        if (j + 1 < KT && p.kt.src[ord[j + 1]] != c) stage_v(p.kt.src[ord[j + 1]]);
        const float u = den > 0.f ? num * rcp_approx(den) : 0.f;
        // growth (the streaming epilogue's arithmetic: hardware reciprocal and exponential)
        const float m = PMU >= 0 ? g[PMU >= 0 ? PMU : 0] : p.kt.mu[k];
        const float sg = PSG >= 0 ? g[PSG >= 0 ? PSG : 0] : p.kt.sigma[k];
        const float hh = PH >= 0 ? g[PH >= 0 ? PH : 0] : p.kt.h[k];
        float gk = 0.f;
        if (sg > 0.f) {
            const float z = (u - m) * rcp_approx(sg);
            gk = ex2_approx(-0.721347520444481703680f * (z * z));
        }
        const float t = p.alpha_on ? u : hh * gk;
        tsum += t;
        if (p.maintain) alpha = alpha && (t > eps_u);
        const float G = p.growth_form == 0 ? hh * (2.f * gk - 1.f) : hh * gk;
        const int d = p.kt.dst[k];
#pragma unroll
        for (int cc = 0; cc < CT; cc++)
            if (cc == d) acc[cc] += G;
    }
    if (!p.maintain) alpha = true;
    float st[CT * 5];
#pragma unroll
    for (int v = 0; v < CT * 5; v++) st[v] = 0.f;
    if (in) {
        // a later store from this thread to the same address wins
        if (p.P_out && !alpha && wrote_nz) {
#pragma unroll 1
            for (int pk = 0; pk < NP * KT; pk++) p.P_out[(size_t)pk * N + i] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < CT; c++) {
            const float a = __ldg(&p.A[(size_t)c * N + i]) + p.dt * (alpha ? acc[c] : p.acc0[c]);
            const float an = fminf(fmaxf(a, 0.f), 1.f);
            p.A_out[(size_t)c * N + i] = an;
            if (p.partials) {
                st[c * 5 + 0] = an;
                st[c * 5 + 1] = an * __ldg(&p.sin_y[y]);
                st[c * 5 + 2] = an * __ldg(&p.cos_y[y]);
                st[c * 5 + 3] = an * __ldg(&p.sin_x[x]);
                st[c * 5 + 4] = an * __ldg(&p.cos_x[x]);
            }
        }
        if (p.alpha_out) p.alpha_out[i] = alpha ? 1 : 0;
        if (p.empty_out) p.empty_out[i] = tsum > eps_u ? 0 : 1;
    }
    if (p.partials) block_stats<CT>(st, CT, p.partials);
}

int ring_epilogue_blocks(int H, int W) { return ((W + EP_TX - 1) / EP_TX) * ((H + RG_TY - 1) / RG_TY); }

// Batched worlds of one channel and one kernel: the tiled epilogue's
// arithmetic in the same order (so a world gives the same bits as on its own
// through k_epilogue_r1), but each thread takes BR rows of one column and
// issues every load of its rows before the first row's arithmetic: a group's
// blocks are short-lived, and this keeps more loads in flight per thread
// (two rows measured best on the 256-world batch: 1, 2, 4, 8 rows gave 0.375,
// 0.364, 0.424, 0.511 ms per step).
// Needs W % 32 == 0 and H % (8 BR) == 0; no statistics, alpha or empty output.
template <int LOC, int BR>
__global__ void __launch_bounds__(256) k_epilogue_batch11(EpiParams p)
{
    pdl_enter();
    constexpr int NP = ((LOC & 1) != 0) + ((LOC & 2) != 0) + ((LOC & 4) != 0);
    constexpr int PMU = (LOC & 1) ? 0 : -1;
    constexpr int PSG = (LOC & 2) ? ((LOC & 1) ? 1 : 0) : -1;
    constexpr int PH = (LOC & 4) ? NP - 1 : -1;
    const int H = p.H, W = p.W;
    const size_t N = (size_t)H * W;
    const int x = blockIdx.x * EP_TX + threadIdx.x;
    const int xm = x == 0 ? W - 1 : x - 1;
    const int xp = x == W - 1 ? 0 : x + 1;
    const float eps_p = p.eps_p, eps_u = p.eps_u;
    const int wz = blockIdx.z;
    const float* pA = p.A_list[wz];
    const float* pP = p.P_list ? p.P_list[wz] : nullptr;
    float* pAo = p.Aout_list[wz];
    float* pPo = p.Pout_list ? p.Pout_list[wz] : nullptr;
    const float* pU = p.U + (size_t)wz * p.u_stride;

    float v[BR][NP > 0 ? NP : 1][5];
    float u[BR], a[BR];
    size_t ic[BR];
#pragma unroll
    for (int j = 0; j < BR; j++) {
        const int y = blockIdx.y * (EP_TY * BR) + j * EP_TY + threadIdx.y;
        const size_t rc = (size_t)y * W;
        const size_t ru = (size_t)(y == 0 ? H - 1 : y - 1) * W;
        const size_t rd = (size_t)(y == H - 1 ? 0 : y + 1) * W;
        ic[j] = rc + x;
#pragma unroll
        for (int pk = 0; pk < NP; pk++) {
            const float* pl = pP + (size_t)pk * N;
            if (p.maintain) {
                v[j][pk][0] = __ldg(pl + ru + x);
                v[j][pk][1] = __ldg(pl + rc + xm);
                v[j][pk][2] = __ldg(pl + rc + x);
                v[j][pk][3] = __ldg(pl + rc + xp);
                v[j][pk][4] = __ldg(pl + rd + x);
            } else {
                v[j][pk][2] = __ldg(pl + ic[j]);
            }
        }
        u[j] = __ldg(pU + ic[j]);
        a[j] = __ldg(pA + ic[j]);
    }
#pragma unroll
    for (int j = 0; j < BR; j++) {
        float ph[NP > 0 ? NP : 1];
        bool alpha = true;
#pragma unroll
        for (int pk = 0; pk < NP; pk++) {
            if (p.maintain) {
                const float v0 = v[j][pk][0], v1 = v[j][pk][1], v2 = v[j][pk][2], v3 = v[j][pk][3], v4 = v[j][pk][4];
                const float s = (((v0 + v1) + v2) + v3) + v4;
                const int n = (v0 > eps_p) + (v1 > eps_p) + (v2 > eps_p) + (v3 > eps_p) + (v4 > eps_p);
                const float vv = n > 0 ? fminf(fmaxf(s / (float)n, 0.f), 1.f) : 0.f;
                alpha = alpha && (vv > eps_p);
                ph[pk] = vv;
            } else {
                ph[pk] = v[j][pk][2];
            }
        }
        float acc = 0.f;
        {
            const float m = PMU >= 0 ? ph[PMU >= 0 ? PMU : 0] : p.kt.mu[0];
            const float sg = PSG >= 0 ? ph[PSG >= 0 ? PSG : 0] : p.kt.sigma[0];
            const float hh = PH >= 0 ? ph[PH >= 0 ? PH : 0] : p.kt.h[0];
            float gk = 0.f;
            if (sg > 0.f) {
                const float z = (u[j] - m) / sg;
                gk = expf(-0.5f * z * z);
            }
            const float t = p.alpha_on ? u[j] : hh * gk;
            if (p.maintain) alpha = alpha && (t > eps_u);
            const float G = p.growth_form == 0 ? hh * (2.f * gk - 1.f) : hh * gk;
            acc += G;
        }
        if (!p.maintain) alpha = true;
        const float an = fminf(fmaxf(a[j] + p.dt * (alpha ? acc : p.acc0[0]), 0.f), 1.f);
        pAo[ic[j]] = an;
        if (pPo) {
#pragma unroll
            for (int pk = 0; pk < NP; pk++) pPo[(size_t)pk * N + ic[j]] = (p.maintain && !alpha) ? 0.f : ph[pk];
        }
    }
}

// The same per-site arithmetic with four adjacent columns per thread: every
// row of a gene plane, the potential and the phenospace come in as float4
// loads (the diffusion's left and right neighbours of the four columns as two
// scalar loads), so a thread issues 12 loads for four sites instead of 48.
// A block of 32 x 8 threads covers 128 columns x 8 BR rows.  Needs
// W % 128 == 0 and H % (8 BR) == 0; results are those of k_epilogue_batch11.
template <int LOC, int BR, bool LISTS = true>
__global__ void __launch_bounds__(256) k_epilogue_batch11v(EpiParams p)
{
    pdl_enter();
    constexpr int NP = ((LOC & 1) != 0) + ((LOC & 2) != 0) + ((LOC & 4) != 0);
    constexpr int PMU = (LOC & 1) ? 0 : -1;
    constexpr int PSG = (LOC & 2) ? ((LOC & 1) ? 1 : 0) : -1;
    constexpr int PH = (LOC & 4) ? NP - 1 : -1;
    const int H = p.H, W = p.W;
    const size_t N = (size_t)H * W;
    const int x = (blockIdx.x * EP_TX + threadIdx.x) * 4;        // first of the thread's four columns
    const int xm = x == 0 ? W - 1 : x - 1;
    const int xp = x + 4 == W ? 0 : x + 4;
    const float eps_p = p.eps_p, eps_u = p.eps_u;
    const int wz = blockIdx.z;
    // LISTS: world blockIdx.z of a batched launch; else the single world
    const float* pA = LISTS ? p.A_list[wz] : p.A;
    const float* pP = LISTS ? (p.P_list ? p.P_list[wz] : nullptr) : p.P;
    float* pAo = LISTS ? p.Aout_list[wz] : p.A_out;
    float* pPo = LISTS ? (p.Pout_list ? p.Pout_list[wz] : nullptr) : p.P_out;
    const float* pU = p.U + (size_t)wz * p.u_stride;

    float4 up[BR][NP > 0 ? NP : 1], ce[BR][NP > 0 ? NP : 1], dn[BR][NP > 0 ? NP : 1];
    float lf[BR][NP > 0 ? NP : 1], rt[BR][NP > 0 ? NP : 1];
    float4 u[BR], a[BR];
    size_t ic[BR];
#pragma unroll
    for (int j = 0; j < BR; j++) {
        const int y = blockIdx.y * (EP_TY * BR) + j * EP_TY + threadIdx.y;
        const size_t rc = (size_t)y * W;
        const size_t ru = (size_t)(y == 0 ? H - 1 : y - 1) * W;
        const size_t rd = (size_t)(y == H - 1 ? 0 : y + 1) * W;
        ic[j] = rc + x;
#pragma unroll
        for (int pk = 0; pk < NP; pk++) {
            const float* pl = pP + (size_t)pk * N;
            ce[j][pk] = __ldg(reinterpret_cast<const float4*>(pl + rc + x));
            if (p.maintain) {
                up[j][pk] = __ldg(reinterpret_cast<const float4*>(pl + ru + x));
                dn[j][pk] = __ldg(reinterpret_cast<const float4*>(pl + rd + x));
                lf[j][pk] = __ldg(pl + rc + xm);
                rt[j][pk] = __ldg(pl + rc + xp);
            }
        }
        u[j] = __ldg(reinterpret_cast<const float4*>(pU + ic[j]));
        a[j] = __ldg(reinterpret_cast<const float4*>(pA + ic[j]));
    }
#pragma unroll
    for (int j = 0; j < BR; j++) {
        float outA[4], outP[4][NP > 0 ? NP : 1];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float ph[NP > 0 ? NP : 1];
            bool alpha = true;
#pragma unroll
            for (int pk = 0; pk < NP; pk++) {
                const float* cv = reinterpret_cast<const float*>(&ce[j][pk]);
                if (p.maintain) {
                    const float v0 = reinterpret_cast<const float*>(&up[j][pk])[c];
                    const float v1 = c == 0 ? lf[j][pk] : cv[c - 1];
                    const float v2 = cv[c];
                    const float v3 = c == 3 ? rt[j][pk] : cv[c + 1];
                    const float v4 = reinterpret_cast<const float*>(&dn[j][pk])[c];
                    const float sm = (((v0 + v1) + v2) + v3) + v4;
                    const int n = (v0 > eps_p) + (v1 > eps_p) + (v2 > eps_p) + (v3 > eps_p) + (v4 > eps_p);
                    const float vv = n > 0 ? fminf(fmaxf(sm / (float)n, 0.f), 1.f) : 0.f;
                    alpha = alpha && (vv > eps_p);
                    ph[pk] = vv;
                } else {
                    ph[pk] = cv[c];
                }
            }
            const float uu = reinterpret_cast<const float*>(&u[j])[c];
            float acc = 0.f;
            {
                const float m = PMU >= 0 ? ph[PMU >= 0 ? PMU : 0] : p.kt.mu[0];
                const float sg = PSG >= 0 ? ph[PSG >= 0 ? PSG : 0] : p.kt.sigma[0];
                const float hh = PH >= 0 ? ph[PH >= 0 ? PH : 0] : p.kt.h[0];
                float gk = 0.f;
                if (sg > 0.f) {
                    const float z = (uu - m) / sg;
                    gk = expf(-0.5f * z * z);
                }
                const float tt = p.alpha_on ? uu : hh * gk;
                if (p.maintain) alpha = alpha && (tt > eps_u);
                const float G = p.growth_form == 0 ? hh * (2.f * gk - 1.f) : hh * gk;
                acc += G;
            }
            if (!p.maintain) alpha = true;
            outA[c] = fminf(fmaxf(reinterpret_cast<const float*>(&a[j])[c] + p.dt * (alpha ? acc : p.acc0[0]), 0.f),
                            1.f);
#pragma unroll
            for (int pk = 0; pk < NP; pk++) outP[c][pk] = (p.maintain && !alpha) ? 0.f : ph[pk];
        }
        *reinterpret_cast<float4*>(pAo + ic[j]) = make_float4(outA[0], outA[1], outA[2], outA[3]);
        if (pPo) {
#pragma unroll
            for (int pk = 0; pk < NP; pk++)
                *reinterpret_cast<float4*>(pPo + (size_t)pk * N + ic[j]) =
                    make_float4(outP[0][pk], outP[1][pk], outP[2][pk], outP[3][pk]);
        }
    }
}

// One launch over n_worlds batched worlds of the same shape (tiled epilogue;
// EpiParams carries the pointer lists).  False if the shape has no tiled kernel.
bool epilogue_batch_supported(const EpiParams& p)
{
    const int loc = (p.p_mu >= 0 ? 1 : 0) | (p.p_sigma >= 0 ? 2 : 0) | (p.p_h >= 0 ? 4 : 0);
    const int K = p.kt.K, C = p.kt.C;
    return (p.r_diff == 1 || !p.maintain) && p.n_rings == 0 &&
           ((K == 15 && C == 3 && (loc == 3 || loc == 0)) || (K == 1 && C == 1 && (loc == 3 || loc == 0)));
}

cudaError_t launch_epilogue_batch(const EpiParams& p, int n_worlds, cudaStream_t s, int br)
{
    if (!epilogue_batch_supported(p) || n_worlds < 1 || n_worlds > 65535) return cudaErrorInvalidValue;
    const int loc = (p.p_mu >= 0 ? 1 : 0) | (p.p_sigma >= 0 ? 2 : 0) | (p.p_h >= 0 ? 4 : 0);
    const int K = p.kt.K;
    if (p.partials || p.alpha_out || p.empty_out) return cudaErrorInvalidValue;
    // the batched forms read every world's buffers through the lists; a single
    // world (null lists) takes the four-column form or the one-row-per-thread kernel
    const bool lists = p.A_list && p.Aout_list && (p.n_p == 0 || (p.P_list && p.Pout_list));
    dim3 block(EP_TX, EP_TY);
    // br < 0: four columns per thread, |br| rows (float4 form; widths of 128 k)
    if ((br == -1 || br == -2) && K == 1 && p.W % (4 * EP_TX) == 0 && p.H % (EP_TY * -br) == 0) {
        dim3 g4(p.W / (4 * EP_TX), p.H / (EP_TY * -br), n_worlds);
        if (br == -1 && !lists) {           // one world, its own buffers
            if (loc == 3) launch_pdl(k_epilogue_batch11v<3, 1, false>, g4, block, 0, s, p);
            else launch_pdl(k_epilogue_batch11v<0, 1, false>, g4, block, 0, s, p);
        } else if (!lists) {
            return cudaErrorInvalidValue;
        } else if (br == -1) {
            if (loc == 3) launch_pdl(k_epilogue_batch11v<3, 1>, g4, block, 0, s, p);
            else launch_pdl(k_epilogue_batch11v<0, 1>, g4, block, 0, s, p);
        } else {
            if (loc == 3) launch_pdl(k_epilogue_batch11v<3, 2>, g4, block, 0, s, p);
            else launch_pdl(k_epilogue_batch11v<0, 2>, g4, block, 0, s, p);
        }
        return cudaGetLastError();
    }
    if (br != 1 && br != 2 && br != 4) br = 2;
    if (lists && K == 1 && p.W % EP_TX == 0 && p.H % (EP_TY * br) == 0) {
        dim3 g4(p.W / EP_TX, p.H / (EP_TY * br), n_worlds);
        if (br == 1) {
            if (loc == 3) launch_pdl(k_epilogue_batch11<3, 1>, g4, block, 0, s, p);
            else launch_pdl(k_epilogue_batch11<0, 1>, g4, block, 0, s, p);
        } else if (br == 2) {
            if (loc == 3) launch_pdl(k_epilogue_batch11<3, 2>, g4, block, 0, s, p);
            else launch_pdl(k_epilogue_batch11<0, 2>, g4, block, 0, s, p);
        } else {
            if (loc == 3) launch_pdl(k_epilogue_batch11<3, 4>, g4, block, 0, s, p);
            else launch_pdl(k_epilogue_batch11<0, 4>, g4, block, 0, s, p);
        }
        return cudaGetLastError();
    }
    // one row per thread: the worlds of a group are often small, so the grid
    // needs the extra blocks (no statistics are gathered here)
    dim3 grid((p.W + EP_TX - 1) / EP_TX, (p.H + EP_TY - 1) / EP_TY, n_worlds);
    if (K == 15 && loc == 3) launch_pdl(k_epilogue_r1<15, 3, 3, 1>, grid, block, 0, s, p);
    else if (K == 15) launch_pdl(k_epilogue_r1<15, 3, 0, 1>, grid, block, 0, s, p);
    else if (loc == 3) launch_pdl(k_epilogue_r1<1, 1, 3, 1>, grid, block, 0, s, p);
    else launch_pdl(k_epilogue_r1<1, 1, 0, 1>, grid, block, 0, s, p);
    return cudaGetLastError();
}

int epilogue_blocks(int H, int W)
{
    return ((W + EP_TX - 1) / EP_TX) * ((H + EP_TY * EP_RY - 1) / (EP_TY * EP_RY));
}

cudaError_t launch_epilogue(const EpiParams& p, cudaStream_t s, int* n_blocks)
{
    dim3 grid((p.W + EP_TX - 1) / EP_TX, (p.H + EP_TY * EP_RY - 1) / (EP_TY * EP_RY));
    dim3 block(EP_TX, EP_TY);
    if (n_blocks) *n_blocks = grid.x * grid.y;
    const int K = p.kt.K, C = p.kt.C;
    const int loc = (p.p_mu >= 0 ? 1 : 0) | (p.p_sigma >= 0 ? 2 : 0) | (p.p_h >= 0 ? 4 : 0);
    const bool rd1 = p.r_diff == 1 || !p.maintain;
    const bool r1 = rd1 && p.n_rings == 0;
    const int locr = loc | (p.p_kern >= 0 ? 8 : 0);
    if (rd1 && p.n_rings > 0 && locr == 15 && p.W >= RG_TILE_W && p.H >= RG_TILE_H &&
        ((p.n_rings == 24 && K == 15 && C == 3) || (p.n_rings == 24 && K == 1 && C == 1) ||
         (p.n_rings == 12 && K == 15 && C == 3))) {
        const dim3 rgrid((p.W + EP_TX - 1) / EP_TX, (p.H + RG_TY - 1) / RG_TY);
        if (n_blocks) *n_blocks = rgrid.x * rgrid.y;
        const dim3 rblock(EP_TX, RG_TY);
        const size_t vb = (size_t)p.n_rings * 256 * sizeof(float);
        cudaError_t e = cudaSuccess;
        if (p.n_rings == 24 && K == 15) {
            e = smem_limit<k_epilogue_rings<15, 3, 24, 15>>(vb);
            if (e == cudaSuccess) launch_pdl(k_epilogue_rings<15, 3, 24, 15>, rgrid, rblock, vb, s, p);
        } else if (p.n_rings == 24) {
            e = smem_limit<k_epilogue_rings<1, 1, 24, 15>>(vb);
            if (e == cudaSuccess) launch_pdl(k_epilogue_rings<1, 1, 24, 15>, rgrid, rblock, vb, s, p);
        } else {
            e = smem_limit<k_epilogue_rings<15, 3, 12, 15>>(vb);
            if (e == cudaSuccess) launch_pdl(k_epilogue_rings<15, 3, 12, 15>, rgrid, rblock, vb, s, p);
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (r1 && K == 15 && C == 3 && loc == 3) launch_pdl(k_epilogue_r1<15, 3, 3>, grid, block, 0, s, p);
    else if (r1 && K == 15 && C == 3 && loc == 0) launch_pdl(k_epilogue_r1<15, 3, 0>, grid, block, 0, s, p);
    else if (r1 && K == 1 && C == 1 && loc == 3) launch_pdl(k_epilogue_r1<1, 1, 3>, grid, block, 0, s, p);
    else if (r1 && K == 1 && C == 1 && loc == 0) launch_pdl(k_epilogue_r1<1, 1, 0>, grid, block, 0, s, p);
    else launch_pdl(k_epilogue_generic, grid, block, 0, s, p);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- statistics
// Block partials of (sum A, sum A sin(2 pi y/H), sum A cos(2 pi y/H), sum A
// sin(2 pi x/W), sum A cos(2 pi x/W)) per channel, same tiling and reduction
// order as the epilogue.
__global__ void __launch_bounds__(256) k_stats_partials(const float* A, int C, int H, int W,
                                                        const float* sin_y, const float* cos_y,
                                                        const float* sin_x, const float* cos_x,
                                                        float2* partials)
{
    pdl_enter();
    const int x = blockIdx.x * EP_TX + threadIdx.x;
    float st[kMaxChannels * 5];
    for (int v = 0; v < kMaxChannels * 5; v++) st[v] = 0.f;
    if (x < W) {
        for (int j = 0; j < EP_RY; j++) {
            const int y = blockIdx.y * (EP_TY * EP_RY) + j * EP_TY + threadIdx.y;
            if (y >= H) break;
            for (int c = 0; c < C; c++) {
                const float a = __ldg(&A[((size_t)c * H + y) * W + x]);
                st[c * 5 + 0] += a;
                st[c * 5 + 1] += a * __ldg(&sin_y[y]);
                st[c * 5 + 2] += a * __ldg(&cos_y[y]);
                st[c * 5 + 3] += a * __ldg(&sin_x[x]);
                st[c * 5 + 4] += a * __ldg(&cos_x[x]);
            }
        }
    }
    block_stats<kMaxChannels>(st, C, partials);
}

cudaError_t launch_stats_partials(const float* A, int C, int H, int W, const float* sin_y,
                                  const float* cos_y, const float* sin_x, const float* cos_x,
                                  float2* partials, cudaStream_t s, int* n_blocks)
{
    dim3 grid((W + EP_TX - 1) / EP_TX, (H + EP_TY * EP_RY - 1) / (EP_TY * EP_RY));
    if (n_blocks) *n_blocks = grid.x * grid.y;
    launch_pdl(k_stats_partials, grid, dim3(EP_TX, EP_TY), 0, s, A, C, H, W, sin_y, cos_y, sin_x, cos_x, partials);
    return cudaGetLastError();
}

// Final reduction, one block of 1024 threads: for each of the C*5 sums,
// 64 threads stride over the block records (fixed order), then two fixed
// shuffle trees and one add, all in compensated FP32 pairs.  out[c] = (mass,
// centre y, centre x), centres from the circular mean atan2(sum A sin, sum A
// cos) scaled to [0, n) (FP64, on the pairs' values).
__global__ void __launch_bounds__(1024) k_stats_final(const float2* partials, int n_blocks, int C,
                                                      int H, int W, float* out)
{
    pdl_enter();
    __shared__ float2 part[32];
    __shared__ float2 tot[kMaxChannels * 5];
    const int nv = C * 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v0 = 0; v0 < nv; v0 += 16) {
        const int v = v0 + (threadIdx.x >> 6);     // 16 values per pass, 64 threads each
        const int stripe = threadIdx.x & 63;
        float2 s = make_float2(0.f, 0.f);
        if (v < nv)
            for (int b = stripe; b < n_blocks; b += 64 * 8) {
                // eight records in flight per thread, added in block order
                float2 x[8];
#pragma unroll
                for (int u = 0; u < 8; u++)
                    x[u] = b + 64 * u < n_blocks ? partials[(size_t)(b + 64 * u) * nv + v] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 8; u++) s = ff_add(s, x[u]);
            }
        for (int off = 16; off > 0; off >>= 1) s = ff_add(s, ff_shfl_down(s, off));
        if (lane == 0) part[warp] = s;
        __syncthreads();
        if (threadIdx.x < 16 && v0 + threadIdx.x < nv)
            tot[v0 + threadIdx.x] = ff_add(part[2 * threadIdx.x], part[2 * threadIdx.x + 1]);
        __syncthreads();
    }
    if (threadIdx.x < 2 * C) stats_centre(tot, threadIdx.x >> 1, threadIdx.x & 1, H, W, out);
}

cudaError_t launch_stats_final(const float2* partials, int n_blocks, int C, int H, int W,
                               float* out, cudaStream_t s)
{
    launch_pdl(k_stats_final, 1, 1024, 0, s, partials, n_blocks, C, H, W, out);
    return cudaGetLastError();
}

}  // namespace lenia
