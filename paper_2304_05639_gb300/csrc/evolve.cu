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
// Each disk pass loads a (32 + 2r)^2 tile with its periodic halo into shared
// memory, turns every tile row into exclusive prefix sums, and adds, for each
// of the 2r + 1 rows of the disk, the difference of two prefix sums.
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

// PASS 1: empty (0/1 bytes) -> c.  PASS 2: c -> M, then mutation, penalisation
// and the optional E_pen output at each site.
template <int PASS>
__global__ void __launch_bounds__(DK_THREADS) k_disk_pass(EvoParams p)
{
    extern __shared__ int pre[];                // [S][S + 1] exclusive row prefix sums
    const int r = p.r_oxy;
    const int S = DK_T + 2 * r;
    const int SP = S + 1;                       // odd row pitch: the row scans hit distinct banks
    const int y0 = blockIdx.y * DK_T - r, x0 = blockIdx.x * DK_T - r;
    for (int ty = threadIdx.x >> 5; ty < S; ty += DK_THREADS / 32) {
        const size_t row = (size_t)wrap_i(y0 + ty, p.H) * p.W;
        for (int tx = threadIdx.x & 31; tx < S; tx += 32) {
            const size_t gi = row + wrap_i(x0 + tx, p.W);
            pre[ty * SP + tx + 1] = PASS == 1 ? (int)p.empty[gi] : p.n_disk - (int)p.cnt_in[gi];
        }
    }
    __syncthreads();
    // prefix sums, one warp per tile row: each lane owns up to 3 consecutive
    // entries (S <= 96), then a warp scan of the lanes' totals
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int per = (S + 31) / 32;
        for (int row = warp; row < S; row += DK_THREADS / 32) {
            int* q = pre + row * SP;
            int part[3];
            int sum = 0;
#pragma unroll
            for (int t = 0; t < 3; t++) {
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
            for (int t = 0; t < 3; t++) {
                const int j = lane * per + t;
                if (t < per && j < S) q[j + 1] = excl + part[t];
            }
            if (lane == 0) q[0] = 0;
        }
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, tyb = threadIdx.x >> 5;
    const int x = blockIdx.x * DK_T + tx;
    if (x >= p.W) return;
    const size_t N = (size_t)p.H * p.W;
    for (int j = 0; j < DK_T / 8; j++) {
        const int ty = tyb + 8 * j;
        const int y = blockIdx.y * DK_T + ty;
        if (y >= p.H) break;
        int s = 0;
        for (int dy = -r; dy <= r; dy++) {
            const int hw = p.half_width[dy < 0 ? -dy : dy];
            const int* q = pre + (ty + r + dy) * SP;
            s += q[tx + r + hw + 1] - q[tx + r - hw];
        }
        const size_t i = (size_t)y * p.W + x;
        if (PASS == 1) {
            p.cnt_out[i] = (uint16_t)s;
        } else {
            if (p.epen_out) p.epen_out[i] = (float)((double)s / p.n_disk2);
            if (p.alpha[i]) {
                if (p.mut_plane >= 0 && wrap_i(x - p.mut_x0 + p.mut_half, p.W) < 2 * p.mut_half &&
                    wrap_i(y - p.mut_y0 + p.mut_half, p.H) < 2 * p.mut_half)
                    p.P[(size_t)p.mut_plane * N + i] += p.mut_add;
                if (p.pen_plane >= 0 && (long long)s > p.pen_thresh)
                    p.P[(size_t)p.pen_plane * N + i] += p.pen_add;
            }
        }
    }
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

size_t disk_fused_smem(int r)
{
    const size_t E = DK_T + 4 * (size_t)r, S = DK_T + 2 * (size_t)r;
    return (E * (E + 1) + S * (S + 1)) * sizeof(int);
}

cudaError_t launch_disk_fused(const EvoParams& p, cudaStream_t s)
{
    const size_t smem = disk_fused_smem(p.r_oxy);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = smem_limit<k_disk_fused>(smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((p.W + DK_T - 1) / DK_T, (p.H + DK_T - 1) / DK_T);
    k_disk_fused<<<grid, DK_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

// A and P are zeroed at each listed wall site (in place).
__global__ void k_walls_zero(const int* idx, int n, float* A, int C, float* P, int npk, size_t N)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const size_t i = (size_t)idx[t];
    for (int c = 0; c < C; c++) A[(size_t)c * N + i] = 0.f;
    for (int pk = 0; pk < npk; pk++) P[(size_t)pk * N + i] = 0.f;
}

size_t disk_pass_smem(int r)
{
    const int S = DK_T + 2 * r;
    return (size_t)S * (S + 1) * sizeof(int);
}

cudaError_t launch_disk_pass(const EvoParams& p, int pass, cudaStream_t s)
{
    // at most (32 + 64) x 97 ints = 37 KB for r_oxy = 32: no opt-in needed
    const size_t smem = disk_pass_smem(p.r_oxy);
    const dim3 grid((p.W + DK_T - 1) / DK_T, (p.H + DK_T - 1) / DK_T);
    if (pass == 1)
        k_disk_pass<1><<<grid, DK_THREADS, smem, s>>>(p);
    else
        k_disk_pass<2><<<grid, DK_THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_walls_zero(const int* idx, int n, float* A, int C, float* P, int npk, size_t N,
                              cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_walls_zero<<<(n + 255) / 256, 256, 0, s>>>(idx, n, A, C, P, npk, N);
    return cudaGetLastError();
}

}  // namespace lenia
