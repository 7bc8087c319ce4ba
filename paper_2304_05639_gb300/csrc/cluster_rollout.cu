// Rollouts of small worlds with global genes in one thread-block cluster
// (Algorithm 2's step repeated: convolve, growth, clipped update; no gene
// maps, so no diffusion or alpha mask).
//
// The Q blocks of one cluster (16 where the part allows it, else 8) keep the
// world in shared memory for the whole rollout.  Block q owns the rows
// q H/Q .. (q + 1) H/Q - 1 of every channel, in two buffers (the state of
// even and odd steps).  Per step it gathers the rows it needs (its own and R
// above and below, periodic) from the owners' buffers through distributed
// shared memory into a tile with a periodic column halo, computes its sites'
// potentials, growth and clipped update into its other buffer, and meets the
// other blocks at the cluster barrier (hardware, with release / acquire
// ordering of the shared-memory writes).  A block reads a peer's buffer of
// step t only between the barriers that end steps t - 1 and t, and the peer
// writes that buffer again only after the barrier that ends step t + 1, so
// one barrier per step suffices.  Nothing leaves the cluster until the last
// step is done: the state is read from A before the first step and written
// back after the last.
//
// The convolution sums each kernel over the disk |d| < R of its support (R
// at compile time): a thread takes a strip of 8 sites of one row and every
// eighth kernel row dy (row group g: dy + R = g, g + 8, ...), keeps the
// strip's input window for that row in registers and adds 8 products per
// weight; the 8 row groups of a strip sit in neighbouring lanes and meet in
// a reduce-scatter of shuffles, after which lane g holds the potential of
// the strip's site g.  The lanes of a warp take kernel rows 8j .. 8j + 7
// together, so each pass j spans only the columns where one of those rows
// has support (a compile-time range); the weights outside it are zero (the
// host checks this before it picks the route), and the sums are the dense
// sums without their zero terms.  A warp takes four
// strips 8 columns apart and the tile's row pitch is 1 modulo 32, so its 32
// lanes (8 consecutive rows, four strips) read 32 different banks.  (Sixteen
// warps with 16 row groups measured the same.)
#include <cooperative_groups.h>
#include <math.h>

#include "lenia_internal.cuh"

namespace lenia {

namespace {

namespace cg = cooperative_groups;

constexpr int CR_XS = 8;          // sites per strip
constexpr int CR_G = 8;           // kernel-row groups per strip (lane bits 0..2)
constexpr int CR_THREADS = 256;
constexpr int CR_MIN_R = 1, CR_MAX_R = 16;

// Half-width of the support of kernel row dy (|d| < R): the largest h with
// h^2 + dy^2 < R^2, or -1 for an empty row.
__host__ __device__ constexpr int cr_row_hw(int R, int dy)
{
    int h = -1;
    while ((h + 1) * (h + 1) + dy * dy < R * R) h++;
    return h;
}

// The widest half-width among kernel rows CR_G J .. CR_G J + CR_G - 1 (row
// index dy + R), or -1 when none of them has support.
__host__ __device__ constexpr int cr_group_hw(int R, int J)
{
    int m = -1;
    for (int r = CR_G * J; r < CR_G * J + CR_G && r <= 2 * R; r++) {
        const int h = cr_row_hw(R, r - R);
        m = h > m ? h : m;
    }
    return m;
}

// Pass J of a lane's kernel rows: row CR_G J + g over the group's column
// range, then the next pass.
template <int R, int J>
__device__ __forceinline__ void cr_row_passes(int g, const float* tk, const float* wk, int yl, int TW,
                                              float (&acc)[CR_XS])
{
    constexpr int KW = 2 * R + 1;
    if constexpr (CR_G * J < KW) {
        constexpr int HW = cr_group_hw(R, J);
        if constexpr (HW >= 0) {
            constexpr int LO = R - HW, NDX = 2 * HW + 1;
            const int dyi = CR_G * J + g;
            if (dyi < KW) {
                const float* trow = tk + (size_t)(yl + dyi) * TW + LO;
                const float* wrow = wk + dyi * KW + LO;
                float v[NDX + CR_XS - 1];
#pragma unroll
                for (int j = 0; j < NDX + CR_XS - 1; j++) v[j] = trow[j];
#pragma unroll
                for (int dx = 0; dx < NDX; dx++) {
                    const float wv = wrow[dx];
#pragma unroll
                    for (int s = 0; s < CR_XS; s++) acc[s] = fmaf(wv, v[dx + s], acc[s]);
                }
            }
        }
        cr_row_passes<R, J + 1>(g, tk, wk, yl, TW, acc);
    }
}

// Shared-memory layout (floats): own[2][C][HS][W], tile[C][TH][TW],
// weights[K][KW][KW].  Tile column R + x holds column x of the world
// (x = -R .. W + R - 1, periodic); TW = 1 mod 32.
struct CrLayout {
    int HS, TH, TW, KW;
    size_t own, tile, wts;
    __host__ __device__ CrLayout(int H, int W, int C, int K, int R, int Q)
    {
        HS = H / Q;
        KW = 2 * R + 1;
        TH = HS + 2 * R;
        TW = (W + 2 * R + 30) / 32 * 32 + 1;
        own = (size_t)C * HS * W;
        tile = (size_t)C * TH * TW;
        wts = (size_t)K * KW * KW;
    }
    __host__ __device__ size_t bytes() const { return (2 * own + tile + wts) * sizeof(float); }
};

template <int R>
__global__ void __launch_bounds__(CR_THREADS, 1) k_cluster_rollout(ClusterRolloutParams p)
{
    constexpr int KW = 2 * R + 1;
    cg::cluster_group cl = cg::this_cluster();
    const int Q = (int)cl.num_blocks(), q = (int)cl.block_rank();
    const int H = p.H, W = p.W, C = p.C, K = p.kt.K;
    const CrLayout L(H, W, C, K, R, Q);
    const int HS = L.HS, TH = L.TH, TW = L.TW;
    extern __shared__ float4 cr_sm4[];
    float* own0 = reinterpret_cast<float*>(cr_sm4);
    float* own1 = own0 + L.own;
    float* tile = own1 + L.own;
    float* wt = tile + L.tile;
    const int tid = threadIdx.x;
    const size_t N = (size_t)H * W;
    for (int i = tid; i < K * KW * KW; i += CR_THREADS) wt[i] = __ldg(&p.w[i]);
    // this block's rows of every channel (W is a multiple of 32: float4 rows)
    const int W4 = W / 4;
    for (int u = tid; u < C * HS * W4; u += CR_THREADS) {
        const int c = u / (HS * W4), r = u % (HS * W4);
        const int yl = r / W4, x4 = r % W4;
        reinterpret_cast<float4*>(own0)[u] =
            __ldcg(reinterpret_cast<const float4*>(p.A + (size_t)c * N + (size_t)(q * HS + yl) * W) + x4);
    }
    cl.sync();

    const int lane = tid & 31, warp = tid >> 5;
    const int g = lane & (CR_G - 1), ss = lane >> 3;     // row group, strip of the warp's four
    const int quads = W / (4 * CR_XS);                   // four-strip groups per row
    const int n_items = HS * quads;
    // gather: a warp takes whole tile rows, lpr lanes per row (W / 4 = 8, 16: several rows per warp)
    const int lpr = (W4 < 32 && 32 % W4 == 0) ? W4 : 32;
    const int rpw = 32 / lpr, sub = lane / lpr, xl = lane % lpr;
    for (int t = 0; t < p.n_steps; t++) {
        const float* cur = (t & 1) ? own1 : own0;
        float* nxt = (t & 1) ? own0 : own1;
        // rows -R .. HS + R - 1 (relative to this block's first row) from their
        // owners, each value also into the periodic column halo
        for (int rr = warp * rpw + sub; rr < C * TH; rr += (CR_THREADS / 32) * rpw) {
            const int c = rr / TH, row = rr - c * TH;
            int y = (q * HS + row - R) % H;
            if (y < 0) y += H;
            const int owner = y / HS, ly = y - owner * HS;
            const float4* src = reinterpret_cast<const float4*>(
                cl.map_shared_rank(const_cast<float*>(cur), owner) + ((size_t)c * HS + ly) * W);
            float* trow = tile + ((size_t)c * TH + row) * TW + R;
            for (int x4 = xl; x4 < W4; x4 += lpr) {
                const float4 v4 = src[x4];
                const float v[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int x = 4 * x4 + e;
                    trow[x] = v[e];
                    if (x < R) trow[W + x] = v[e];
                    if (x >= W - R) trow[x - W] = v[e];
                }
            }
        }
        __syncthreads();
        for (int it = warp; it < n_items; it += CR_THREADS / 32) {
            const int yl = it / quads, qd = it % quads;
            const int x0 = (qd * 4 + ss) * CR_XS;
            float gsum[kMaxChannels];
#pragma unroll
            for (int c = 0; c < kMaxChannels; c++) gsum[c] = 0.f;
            for (int k = 0; k < K; k++) {
                const float* tk = tile + (size_t)p.kt.src[k] * TH * TW + x0;
                const float* wk = wt + (size_t)k * KW * KW;
                float acc[CR_XS];
#pragma unroll
                for (int s = 0; s < CR_XS; s++) acc[s] = 0.f;
                cr_row_passes<R, 0>(g, tk, wk, yl, TW, acc);     // kernel rows g, g + 8, ... (dy = row - R)
                // reduce-scatter over the 8 row groups: lane g ends with site x0 + g
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const bool hi = g & 4;
                    const float send = hi ? acc[i] : acc[i + 4], keep = hi ? acc[i + 4] : acc[i];
                    acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                }
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    const bool hi = g & 2;
                    const float send = hi ? acc[i] : acc[i + 2], keep = hi ? acc[i + 2] : acc[i];
                    acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
                }
                float u;
                {
                    const bool hi = g & 1;
                    const float send = hi ? acc[0] : acc[1], keep = hi ? acc[1] : acc[0];
                    u = keep + __shfl_xor_sync(0xffffffffu, send, 1);
                }
                const float sg = p.kt.sigma[k], h = p.kt.h[k];
                const float z = (u - p.kt.mu[k]) / sg;
                const float gk = sg > 0.f ? expf(-0.5f * z * z) : 0.f;
                const float G = p.growth_form == 0 ? h * (2.f * gk - 1.f) : h * gk;
                const int d = p.kt.dst[k];
#pragma unroll
                for (int c = 0; c < kMaxChannels; c++)
                    if (c == d) gsum[c] += G;
            }
            const int x = x0 + g;
#pragma unroll
            for (int c = 0; c < kMaxChannels; c++) {
                if (c >= C) break;
                const float a = tile[((size_t)c * TH + yl + R) * TW + R + x] + p.dt * gsum[c];
                nxt[((size_t)c * HS + yl) * W + x] = fminf(fmaxf(a, 0.f), 1.f);
            }
        }
        cl.sync();
    }
    const float* fin = (p.n_steps & 1) ? own1 : own0;
    for (int u = tid; u < C * HS * W4; u += CR_THREADS) {
        const int c = u / (HS * W4), r = u % (HS * W4);
        const int yl = r / W4, x4 = r % W4;
        reinterpret_cast<float4*>(p.A + (size_t)c * N + (size_t)(q * HS + yl) * W)[x4] =
            reinterpret_cast<const float4*>(fin)[u];
    }
}

using CrKernel = void (*)(ClusterRolloutParams);

template <int R>
CrKernel cr_pick(int r)
{
    if constexpr (R > CR_MAX_R) {
        (void)r;
        return nullptr;
    } else {
        return r == R ? k_cluster_rollout<R> : cr_pick<R + 1>(r);
    }
}

cudaLaunchConfig_t cr_config(const ClusterRolloutParams& p, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.Q);
    cfg.blockDim = dim3(CR_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t cr_prepare(CrKernel fn, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace

bool cluster_rollout_weights_fit(const float* w, int K, int maxR)
{
    const int KW = 2 * maxR + 1;
    for (int k = 0; k < K; k++)
        for (int r = 0; r < KW; r++) {
            const int hw = cr_group_hw(maxR, r / CR_G);
            for (int dx = 0; dx < KW; dx++) {
                const int off = dx - maxR < 0 ? maxR - dx : dx - maxR;
                if (off > hw && w[((size_t)k * KW + r) * KW + dx] != 0.f) return false;
            }
        }
    return true;
}

size_t cluster_rollout_smem(int H, int W, int C, int K, int maxR, int Q)
{
    return CrLayout(H, W, C, K, maxR, Q).bytes();
}

int cluster_rollout_blocks(int H, int W, int C, int K, int maxR)
{
    if (maxR < CR_MIN_R || maxR > CR_MAX_R || C < 1 || C > kMaxChannels || K < 1 || K > kMaxKernels) return 0;
    if (W % (4 * CR_XS) || (long long)H * W > 8192 || maxR >= H || maxR >= W) return 0;
    CrKernel fn = cr_pick<CR_MIN_R>(maxR);
    if (!fn) return 0;
    for (int Q : {16, 8}) {
        if (H % Q) continue;
        const size_t smem = cluster_rollout_smem(H, W, C, K, maxR, Q);
        if (smem > 160 * 1024) continue;
        if (cr_prepare(fn, smem) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        ClusterRolloutParams p = {};
        p.Q = Q;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cr_config(p, smem, nullptr, attr);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, (const void*)fn, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (n >= 1) return Q;
    }
    return 0;
}

cudaError_t launch_cluster_rollout(const ClusterRolloutParams& p, cudaStream_t s)
{
    CrKernel fn = cr_pick<CR_MIN_R>(p.maxR);
    if (!fn || p.Q < 1 || p.H % p.Q) return cudaErrorInvalidValue;
    const size_t smem = cluster_rollout_smem(p.H, p.W, p.C, p.kt.K, p.maxR, p.Q);
    cudaError_t e = cr_prepare(fn, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cr_config(p, smem, s, attr);
    return cudaLaunchKernelEx(&cfg, fn, p);
}

}  // namespace lenia
