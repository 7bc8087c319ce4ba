// The evolutionary lines of Algorithm 2 around the Lenia step:
//   environment (Section 2.7): walls remove A and P at their sites before the step;
//   penalising area (Section 2.6): E_oxy = (1 - Delta_sum(U)) * K_oxy,
//     E_pen = (1 - E_oxy) * K_oxy, K_oxy the disk |d| <= r_oxy over its point count n;
//   mutation (Section 2.5): P_{pk} += gamma_mut delta on a periodic square AND alpha;
//   penalisation (Section 2.6): P_{pk} += gamma_pen delta on [E_pen > eps_pen] AND alpha.
//
// Both disk averages are taken on integer counts, so they are exact:
//   c(x) = #{empty sites in the disk at x}        (E_oxy = c / n)
//   M(x) = sum over the disk of (n - c)           (E_pen = M / n^2)
// and the penalising test E_pen > eps_pen is M > floor(eps_pen n^2), decided
// on the host in FP64 once per step.
//
// One kernel takes both disk averages per 32 x 32 tile: it loads the tile's
// empty bytes with a periodic halo of 2 r into shared memory, turns every row
// into exclusive prefix sums, forms n - c over the tile plus a halo of r (for
// each of the 2 r + 1 rows of the disk, the difference of two prefix sums),
// takes those rows' prefix sums, and sums M over each output site's disk.
#include "lenia_internal.cuh"

namespace lenia {

constexpr int DK_T = 32;        // output tile side
constexpr int DK_THREADS = 256; // 32 x 8 threads, 4 output rows each

// Periodic index; indices already inside [0, n) (all but the halo near the
// world's edges) skip the division.
__device__ __forceinline__ int wrap_i(int v, int n)
{
    if (v >= 0 && v < n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

// Exclusive prefix sums of S rows of `pre` (row pitch SP, entries 1..S hold
// the values, entry 0 receives 0), one warp per row: each lane owns up to
// MAXPER consecutive entries, then a warp scan of the lanes' totals.
template <int MAXPER>
__device__ __forceinline__ void row_scans(int* pre, int S, int SP)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (S + 31) / 32;
    for (int row = warp; row < S; row += DK_THREADS / 32) {
        int* q = pre + row * SP;
        int part[MAXPER];
        int sum = 0;
#pragma unroll
        for (int t = 0; t < MAXPER; t++) {
            const int j = lane * per + t;
            sum += (t < per && j < S) ? q[j + 1] : 0;
            part[t] = sum;
        }
        int incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += n;
        }
        const int excl = incl - sum;
#pragma unroll
        for (int t = 0; t < MAXPER; t++) {
            const int j = lane * per + t;
            if (t < per && j < S) q[j + 1] = excl + part[t];
        }
        if (lane == 0) q[0] = 0;
    }
}

// Both disk passes in one kernel: the block loads the Delta_sum complement
// bytes of its 32 x 32 tile with a halo of 2 r, takes their row prefix sums,
// forms n - c on the tile plus a halo of r (c = empty sites in each disk),
// takes those rows' prefix sums, and sums M over each output site's disk; the
// counts never leave shared memory.  The same arithmetic as the two passes
// (integer, exact).
__global__ void __launch_bounds__(DK_THREADS) k_disk_fused(EvoParams p)
{
    pdl_enter();
    extern __shared__ int sm_i[];
    const int r = p.r_oxy;
    const int E = DK_T + 4 * r, EP = E + 1;     // empty bytes: tile + 2 r halo
    const int S = DK_T + 2 * r, SP = S + 1;     // n - c: tile + r halo
    int* preE = sm_i;                           // [E][EP]
    int* preM = sm_i + E * EP;                  // [S][SP]
    const int by = blockIdx.y * DK_T, bx = blockIdx.x * DK_T;
    for (int ty = threadIdx.x >> 5; ty < E; ty += DK_THREADS / 32) {
        const size_t row = (size_t)wrap_i(by - 2 * r + ty, p.H) * p.W;
        for (int tx = threadIdx.x & 31; tx < E; tx += 32)
            preE[ty * EP + tx + 1] = (int)p.empty[row + wrap_i(bx - 2 * r + tx, p.W)];
    }
    __syncthreads();
    row_scans<5>(preE, E, EP);
    __syncthreads();
    // n - c at region coordinates (cy, cx) = the disk centred on empty-region (cy + r, cx + r)
    for (int u = threadIdx.x; u < S * S; u += DK_THREADS) {
        const int cy = u / S, cx = u % S;
        int c = 0;
        for (int dy = -r; dy <= r; dy++) {
            const int hw = p.half_width[dy < 0 ? -dy : dy];
            const int* q = preE + (cy + r + dy) * EP;
            c += q[cx + r + hw + 1] - q[cx + r - hw];
        }
        preM[cy * SP + cx + 1] = p.n_disk - c;
    }
    __syncthreads();
    row_scans<3>(preM, S, SP);
    __syncthreads();
    const int tx = threadIdx.x & 31, tyb = threadIdx.x >> 5;
    const int x = bx + tx;
    if (x >= p.W) return;
    const size_t N = (size_t)p.H * p.W;
    for (int j = 0; j < DK_T / 8; j++) {
        const int ty = tyb + 8 * j;
        const int y = by + ty;
        if (y >= p.H) break;
        int s = 0;
        for (int dy = -r; dy <= r; dy++) {
            const int hw = p.half_width[dy < 0 ? -dy : dy];
            const int* q = preM + (ty + r + dy) * SP;
            s += q[tx + r + hw + 1] - q[tx + r - hw];
        }
        const size_t i = (size_t)y * p.W + x;
        if (p.epen_out) p.epen_out[i] = (float)((double)s / p.n_disk2);
        if (p.alpha[i]) {
            if (p.mut_plane >= 0 && wrap_i(x - p.mut_x0 + p.mut_half, p.W) < 2 * p.mut_half &&
                wrap_i(y - p.mut_y0 + p.mut_half, p.H) < 2 * p.mut_half)
                p.P[(size_t)p.mut_plane * N + i] += p.mut_add;
            if (p.pen_plane >= 0 && (long long)s > p.pen_thresh) p.P[(size_t)p.pen_plane * N + i] += p.pen_add;
        }
    }
}

// Half-width of the disk |d| <= R at row offset dy: the largest w with
// w^2 + dy^2 <= R^2 (the host's definition of the same disk).
__host__ __device__ constexpr int disk_hw(int R, int dy)
{
    int w = 0;
    while ((w + 1) * (w + 1) + dy * dy <= R * R) w++;
    return w;
}

template <int R>
struct DiskRows {
    int hw[2 * R + 1];
    constexpr DiskRows() : hw()
    {
        for (int dy = -R; dy <= R; dy++) hw[dy + R] = disk_hw(R, dy < 0 ? -dy : dy);
    }
};

// Exclusive prefix sums of `rows` rows of LEN values (entries 1..LEN of each
// row, row pitch SP; entry 0 receives 0), one thread per row, in order.
template <int LEN>
__device__ __forceinline__ void row_scans_seq(int* pre, int rows, int SP)
{
    for (int row = threadIdx.x; row < rows; row += DK_THREADS) {
        int* q = pre + row * SP;
        int sum = 0;
        q[0] = 0;
#pragma unroll 8
        for (int j = 1; j <= LEN; j++) {
            sum += q[j];
            q[j] = sum;
        }
    }
}

// k_disk_fused for a disk radius known at compile time: the same integer
// arithmetic with the disk's row half-widths as constants (every prefix-sum
// difference is a shared load at a fixed offset), one thread per row for the
// prefix sums (a row of at most 64 entries), and the interior blocks' tile
// loads without the periodic wrap.
template <int R>
__global__ void __launch_bounds__(DK_THREADS) k_disk_fused_t(EvoParams p)
{
    pdl_enter();
    constexpr int E = DK_T + 4 * R, EP = E + 1;     // empty bytes: tile + 2 R halo
    constexpr int S = DK_T + 2 * R, SP = S + 1;     // n - c: tile + R halo
    constexpr DiskRows<R> D{};
    __shared__ int preE[E * EP];
    __shared__ int preM[S * SP];
    const int H = p.H, W = p.W;
    const int by = blockIdx.y * DK_T, bx = blockIdx.x * DK_T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int any = 0, all = 1;
    if (by >= 2 * R && by + DK_T + 2 * R <= H && bx >= 2 * R && bx + DK_T + 2 * R <= W && W % 4 == 0) {
        // interior tile: 4-byte words covering each row segment (bx is a
        // multiple of 32, so the segment starts OFF bytes into its first
        // word), every load of a thread issued before its stores
        constexpr int OFF = (4 - (2 * R) % 4) % 4;
        constexpr int NWD = (OFF + E + 3) / 4;                 // words per row
        constexpr int PER = (E * NWD + DK_THREADS - 1) / DK_THREADS;
        const unsigned* src =
            reinterpret_cast<const unsigned*>(p.empty + (size_t)(by - 2 * R) * W + (bx - 2 * R - OFF));
        const int W4 = W / 4;
        unsigned wv[PER];
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const int u = threadIdx.x + i * DK_THREADS;
            wv[i] = u < E * NWD ? __ldg(&src[(size_t)(u / NWD) * W4 + u % NWD]) : 0u;
        }
#pragma unroll
        for (int i = 0; i < PER; i++) {
            const int u = threadIdx.x + i * DK_THREADS;
            if (u >= E * NWD) break;
            const int ty = u / NWD, x0 = 4 * (u % NWD) - OFF;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int tx = x0 + b;
                if (tx < 0 || tx >= E) continue;
                const int v = (int)((wv[i] >> (8 * b)) & 0xffu);
                any |= v;
                all &= v;
                preE[ty * EP + tx + 1] = v;
            }
        }
    } else {
        for (int ty = warp; ty < E; ty += DK_THREADS / 32) {
            const size_t row = (size_t)wrap_i(by - 2 * R + ty, H) * W;
            for (int tx = lane; tx < E; tx += 32) {
                const int v = (int)p.empty[row + wrap_i(bx - 2 * R + tx, W)];
                any |= v;
                all &= v;
                preE[ty * EP + tx + 1] = v;
            }
        }
    }
    // a tile whose whole 2 R neighbourhood is one value has the same M at
    // every site: n^2 with no empty site (c = 0), 0 with every site empty
    any = __syncthreads_or(any);
    all = __syncthreads_and(all);
    const bool uniform = !any || all;
    if (!uniform) {
        row_scans_seq<E>(preE, E, EP);
        __syncthreads();
        // n - c at region coordinates (cy, cx) = the disk centred on empty-region (cy + R, cx + R)
        for (int u = threadIdx.x; u < S * S; u += DK_THREADS) {
            const int cy = u / S, cx = u % S;
            const int* q = preE + (cy + R) * EP + cx + R;
            int c = 0;
#pragma unroll
            for (int dy = -R; dy <= R; dy++) c += q[dy * EP + D.hw[dy + R] + 1] - q[dy * EP - D.hw[dy + R]];
            preM[cy * SP + cx + 1] = p.n_disk - c;
        }
        __syncthreads();
        row_scans_seq<S>(preM, S, SP);
        __syncthreads();
    }
    const int x = bx + lane;
    if (x >= W) return;
    const size_t N = (size_t)H * W;
    const bool mut_x = p.mut_plane >= 0 && wrap_i(x - p.mut_x0 + p.mut_half, W) < 2 * p.mut_half;
    uint8_t al[DK_T / 8];
#pragma unroll
    for (int j = 0; j < DK_T / 8; j++) {
        const int y = by + warp + 8 * j;
        al[j] = y < H ? __ldg(&p.alpha[(size_t)y * W + x]) : 0;
    }
#pragma unroll
    for (int j = 0; j < DK_T / 8; j++) {
        const int ty = warp + 8 * j;
        const int y = by + ty;
        if (y >= H) break;
        int s = any ? 0 : p.n_disk * p.n_disk;
        if (!uniform) {
            const int* q = preM + (ty + R) * SP + lane + R;
#pragma unroll
            for (int dy = -R; dy <= R; dy++) s += q[dy * SP + D.hw[dy + R] + 1] - q[dy * SP - D.hw[dy + R]];
        }
        const size_t i = (size_t)y * W + x;
        if (p.epen_out) p.epen_out[i] = (float)((double)s / p.n_disk2);
        if (al[j]) {
            if (mut_x && wrap_i(y - p.mut_y0 + p.mut_half, H) < 2 * p.mut_half)
                p.P[(size_t)p.mut_plane * N + i] += p.mut_add;
            if (p.pen_plane >= 0 && (long long)s > p.pen_thresh) p.P[(size_t)p.pen_plane * N + i] += p.pen_add;
        }
    }
}

template <int R>
static cudaError_t launch_disk_t(const EvoParams& p, cudaStream_t s)
{
    const dim3 grid((p.W + DK_T - 1) / DK_T, (p.H + DK_T - 1) / DK_T);
    launch_pdl(k_disk_fused_t<R>, grid, DK_THREADS, 0, s, p);
    return cudaGetLastError();
}

size_t disk_fused_smem(int r)
{
    const size_t E = DK_T + 4 * (size_t)r, S = DK_T + 2 * (size_t)r;
    return (E * (E + 1) + S * (S + 1)) * sizeof(int);
}

cudaError_t launch_disk_fused(const EvoParams& p, cudaStream_t s)
{
    switch (p.r_oxy) {
        case 1: return launch_disk_t<1>(p, s);
        case 2: return launch_disk_t<2>(p, s);
        case 3: return launch_disk_t<3>(p, s);
        case 4: return launch_disk_t<4>(p, s);
        case 5: return launch_disk_t<5>(p, s);
        case 6: return launch_disk_t<6>(p, s);
        case 7: return launch_disk_t<7>(p, s);
        case 8: return launch_disk_t<8>(p, s);
    }
    const size_t smem = disk_fused_smem(p.r_oxy);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = smem_limit<k_disk_fused>(smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((p.W + DK_T - 1) / DK_T, (p.H + DK_T - 1) / DK_T);
    launch_pdl(k_disk_fused, grid, DK_THREADS, smem, s, p);
    return cudaGetLastError();
}

// A and P are zeroed at each listed wall site (in place): one thread per
// (plane, wall site), sites fastest, so a warp writes neighbouring wall sites
// of one plane together (the list is in increasing site order).
__global__ void k_walls_zero(const int* idx, int n, float* A, int C, float* P, int npk, size_t N)
{
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * (C + npk)) return;
    const int plane = t / n, j = t - plane * n;
    const size_t i = (size_t)__ldg(&idx[j]);
    if (plane < C)
        A[(size_t)plane * N + i] = 0.f;
    else
        P[(size_t)(plane - C) * N + i] = 0.f;
}

cudaError_t launch_walls_zero(const int* idx, int n, float* A, int C, float* P, int npk, size_t N,
                              cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const long long total = (long long)n * (C + npk);
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    launch_pdl(k_walls_zero, (int)((total + 255) / 256), 256, 0, s, idx, n, A, C, P, npk, N);
    return cudaGetLastError();
}

}  // namespace lenia
