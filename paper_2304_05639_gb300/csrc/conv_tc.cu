// Direct periodic convolution U_k = K~_k * A_src(k) on the tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulation in tensor memory).
//
// Convolution route of Algorithm 2 ("convolve"), written as a sum of banded
// Toeplitz products: for every kernel row offset dy,
//   U[y, x0 + n] += sum_j A[y + dy, x0 - R + j] T_dy[j, n],
//   T_dy[j, n] = K~[dy, j - n - R]  (0 outside |j - n - R| <= R_k),
// i.e. one GEMM per dy with M = output rows, N = NT output columns and
// K = NT + 2R input columns (padded to KP, a multiple of 16).  The input
// operand of offset dy is the staged input tile shifted down by dy rows: the
// tile is stored as 8-column chunks with every row at a 16-byte stride, so a
// row shift is a 16-byte shift of the operand's start address (the canonical
// K-major layout without swizzle: 8 x 16-byte core matrices, SBO = 128 bytes
// between 8-row groups, LBO = one chunk between the two K halves of an
// instruction).  The Toeplitz blocks are built once on the host (BF16, in
// the same chunked layout) and streamed per (kernel, dy) through a ring of
// shared-memory slots by bulk copies.
//
// Block: one channel, 256 output rows (two M = 128 accumulators) x NT output
// columns, up to TC_NG kernels of that channel; its accumulators, 2 x TC_NG x
// NT FP32 columns, live in tensor memory.  Warp 0 lane 0 loads (TMA for the
// input tile, bulk copies for the Toeplitz blocks), warp 1 lane 0 issues the
// MMAs and commits them to the slots' "empty" barriers, then all four warps
// move the accumulators to U.  Every wait is bounded.
//
// BF16 keeps 8 significant bits (rounding error <= 2^-8 relative).  TERMS = 1
// uses A_hi T_hi alone: each product is off by at most 2^-7 + 2^-16 of its
// value, and so is the potential (all terms are non-negative).  TERMS = 3
// splits both operands into BF16 high and low parts, x = x_hi + x_lo + e with
// |e| <= 2^-16 |x|, and sums A_hi T_hi + A_lo T_hi + A_hi T_lo (the dropped
// A_lo T_lo is <= 2^-16 relative): at most about 3 2^-16 relative, for three
// times the tensor work.
#include <cuda_bf16.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

namespace {

constexpr int TC_ROWS_OUT = 256;      // output rows per block (two M = 128 MMAs)
constexpr int TC_THREADS = 128;
constexpr int TC_NS = 6;              // Toeplitz-block ring slots

// Shared-memory matrix descriptor of tcgen05 (K-major, no swizzle).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// Arrives on `bar` once every MMA this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// v[0..31] <- 32 consecutive columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Bytes of one staged input tile (KP / 8 chunks of rows_pad rows x 16 bytes)
// and of one Toeplitz block (KP / 8 chunks of NT rows x 16 bytes).
__host__ __device__ constexpr size_t tc_tile_bytes(int kp, int rows_pad) { return (size_t)(kp / 8) * rows_pad * 16; }
__host__ __device__ constexpr size_t tc_block_bytes(int kp, int nt) { return (size_t)(kp / 8) * nt * 16; }

template <int NT, int TERMS>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_tc(TcConvParams p, const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo)
{
    pdl_enter();
    constexpr int NA = TERMS == 1 ? 1 : 2;          // input tiles (hi, lo)
    constexpr int NB = TERMS == 1 ? 1 : 2;          // Toeplitz blocks per slot (hi, lo)
    constexpr int NCOLS = 2 * TC_NG * NT;           // accumulator columns
    static_assert(NCOLS == 32 || NCOLS == 64 || NCOLS == 128 || NCOLS == 256 || NCOLS == 512, "TMEM columns");
    constexpr uint32_t IDESC = umma_idesc_bf16(NT);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
    __shared__ __align__(8) uint64_t a_full, done;
    __shared__ __align__(8) uint64_t b_full[TC_NS], b_empty[TC_NS];
    __shared__ uint32_t tmem_base;
    __shared__ int blk_failed;

    const int KP = p.KP, rows_pad = p.rows_pad, nch = KP / 8;
    const size_t tile_b = tc_tile_bytes(KP, rows_pad);
    const size_t blk_b = tc_block_bytes(KP, NT);
    unsigned char* At = smem;                                   // [NA][nch][rows_pad][16 B]
    unsigned char* Bs = smem + NA * tile_b;                     // [TC_NS][NB][nch][NT][16 B]

    const int* grp = p.grp + 6 * blockIdx.z;        // channel, kernel count, up to four kernels
    const int c = grp[0], ng = grp[1];
    const int x0 = blockIdx.x * NT, y0 = blockIdx.y * TC_ROWS_OUT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        mbar_init(&a_full, 1);
        mbar_init(&done, 1);
        for (int s = 0; s < TC_NS; s++) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        mbar_fence_init();
        blk_failed = 0;
    }
    if (warp == 0) {
        tmem_alloc<NCOLS>(&tmem_base);
        tmem_fence_before_sync();
    }
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ loads
        if (lane == 0) {
            bool ok = true;
            const int half = rows_pad / 2;
            mbar_arrive_expect_tx(&a_full, (uint32_t)(NA * tile_b));
            for (int kc = 0; kc < nch; kc++)
                for (int h = 0; h < 2; h++) {
                    unsigned char* dst = At + ((size_t)kc * rows_pad + (size_t)h * half) * 16;
                    tma_load_3d(dst, &tm_hi, x0 + 8 * kc, y0 + h * half, c, &a_full);
                    if (NA == 2) tma_load_3d(dst + tile_b, &tm_lo, x0 + 8 * kc, y0 + h * half, c, &a_full);
                }
            int it = 0;
            for (int gi = 0; ok && gi < ng; gi++) {
                const int k = grp[2 + gi];
                for (int dyi = 0; ok && dyi < p.n_dy; dyi++) {
                    const int2 r = p.ks[k * p.n_dy + dyi];
                    if (r.y < r.x) continue;
                    const int s = it % TC_NS;
                    if (it >= TC_NS && !mbar_wait_bounded(&b_empty[s], ((it - TC_NS) / TC_NS) & 1)) {
                        ok = false;
                        break;
                    }
                    unsigned char* dst = Bs + (size_t)s * NB * blk_b;
                    const unsigned char* src = p.B + ((size_t)k * p.n_dy + dyi) * blk_b;
                    mbar_arrive_expect_tx(&b_full[s], (uint32_t)(NB * blk_b));
                    bulk_g2s(dst, src, (uint32_t)blk_b, &b_full[s]);
                    if (NB == 2) bulk_g2s(dst + blk_b, src + p.B_lo_off, (uint32_t)blk_b, &b_full[s]);
                    it++;
                }
            }
            if (!ok) {
                blk_failed = 1;
                atomicExch(p.status, kStatusWaitTimeout);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            bool ok = mbar_wait_bounded(&a_full, 0);
            tmem_fence_after_sync();
            const uint32_t a0 = smem_addr(At);
            const uint32_t b0 = smem_addr(Bs);
            const uint32_t lbo_a = (uint32_t)rows_pad * 16, lbo_b = NT * 16;
            int it = 0;
            for (int gi = 0; ok && gi < ng; gi++) {
                const int k = grp[2 + gi];
                uint32_t acc = 0;
                for (int dyi = 0; ok && dyi < p.n_dy; dyi++) {
                    const int2 r = p.ks[k * p.n_dy + dyi];
                    if (r.y < r.x) continue;
                    const int s = it % TC_NS;
                    if (!mbar_wait_bounded(&b_full[s], (it / TC_NS) & 1)) {
                        ok = false;
                        break;
                    }
                    tmem_fence_after_sync();
                    const uint32_t bs = b0 + (uint32_t)(s * NB * blk_b);
                    for (int kk = r.x; kk <= r.y; kk++) {
                        const uint64_t bh = umma_desc(bs + (uint32_t)(2 * kk) * lbo_b, lbo_b, 128);
                        const uint64_t bl = umma_desc(bs + (uint32_t)blk_b + (uint32_t)(2 * kk) * lbo_b, lbo_b, 128);
#pragma unroll
                        for (int mt = 0; mt < 2; mt++) {
                            // tile row of output row 0 of this M tile: mt 128 + dy + R
                            const uint32_t ao = (uint32_t)(2 * kk) * lbo_a + (uint32_t)(mt * 128 + dyi) * 16;
                            const uint32_t d = tbase + (uint32_t)((gi * 2 + mt) * NT);
                            umma_bf16(d, umma_desc(a0 + ao, lbo_a, 128), bh, IDESC, acc);
                            if (TERMS == 3) {
                                umma_bf16(d, umma_desc(a0 + (uint32_t)tile_b + ao, lbo_a, 128), bh, IDESC, 1u);
                                umma_bf16(d, umma_desc(a0 + ao, lbo_a, 128), bl, IDESC, 1u);
                            }
                        }
                        acc = 1u;
                    }
                    umma_commit(&b_empty[s]);
                    it++;
                }
            }
            if (!ok) {
                blk_failed = 1;
                atomicExch(p.status, kStatusWaitTimeout);
            }
            umma_commit(&done);        // every MMA issued above, whatever happened
        }
        __syncwarp();
    }

    // ------------------------------------------------ accumulators -> U
    const bool fin = mbar_wait_bounded(&done, 0);
    tmem_fence_after_sync();
    if (fin) {
        const int H = p.H, W = p.W;
        for (int gi = 0; gi < ng; gi++) {
            const int k = grp[2 + gi];
            const bool has = p.has_taps[k] != 0;
            for (int mt = 0; mt < 2; mt++) {
                float v[32];
                if (NT == 32) {
                    tmem_ld32(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)((gi * 2 + mt) * NT), v);
                } else {
                    tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)((gi * 2 + mt) * NT), v);
                }
                const int y = y0 + mt * 128 + warp * 32 + lane;
                float4* dst = reinterpret_cast<float4*>(p.U + ((size_t)k * H + y) * W + x0);
#pragma unroll
                for (int q = 0; q < NT / 4; q++)
                    dst[q] = has ? make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3])
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    } else if (tid == 0) {
        atomicExch(p.status, kStatusWaitTimeout);
    }
    tmem_fence_before_sync();
    __syncthreads();
    if (!fin && tid == 0) mbar_wait_bounded(&done, 0);      // a last bounded chance for in-flight MMAs
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after_sync();
        tmem_dealloc<NCOLS>(tbase);
    }
}

// Padded BF16 copy of the phenospace for the tensor-core route: plane c, row
// q, column r holds A[c][(q - R) mod H][(r - R) mod W] for r < W + 2R (0
// beyond, up to the 8-aligned row pitch Wp); with lo != null also the low
// part A - hi.
__global__ void k_tc_pad(const float* A, int C, int H, int W, int R, int Hp, int Wp, __nv_bfloat16* hi,
                         __nv_bfloat16* lo)
{
    pdl_enter();
    const size_t n = (size_t)C * Hp * Wp;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i % Wp);
        const size_t t = i / Wp;
        const int q = (int)(t % Hp);
        const int c = (int)(t / Hp);
        float v = 0.f;
        if (r < W + 2 * R) {
            int y = q - R, x = r - R;
            y = y < 0 ? y + H : (y >= H ? y - H : y);
            x = x < 0 ? x + W : (x >= W ? x - W : x);
            v = __ldg(&A[((size_t)c * H + y) * W + x]);
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i] = h;
        if (lo) lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// Tensor map of the padded planes [C][Hp][Wp] (BF16), boxes of 8 columns x
// box_rows rows x 1 plane; cached by argument.
bool tc_map(CUtensorMap* out, const void* base, int Wp, int Hp, int C, int box_rows)
{
    struct Key {
        const void* base;
        int Wp, Hp, C, br;
        bool operator==(const Key& o) const
        {
            return base == o.base && Wp == o.Wp && Hp == o.Hp && C == o.C && br == o.br;
        }
    };
    static std::mutex mu;
    static std::vector<std::pair<Key, CUtensorMap>> cache;
    const Key key{base, Wp, Hp, C, box_rows};
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : cache)
        if (e.first == key) {
            *out = e.second;
            return true;
        }
    auto fn = tensor_map_encoder();
    if (!fn || ((uintptr_t)base & 15) != 0) return false;
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)Wp, (cuuint64_t)Hp, (cuuint64_t)C};
    const cuuint64_t strides[2] = {(cuuint64_t)Wp * 2, (cuuint64_t)Wp * Hp * 2};
    const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cache.insert(cache.begin(), {key, m});
    if (cache.size() > 32) cache.pop_back();
    *out = m;
    return true;
}

template <int NT, int TERMS>
cudaError_t launch_tc(const TcConvParams& p, cudaStream_t s)
{
    constexpr int NA = TERMS == 1 ? 1 : 2, NB = NA;
    // at least 80 KB, so that at most two blocks (2 x 256 TMEM columns) share an SM
    const size_t smem = std::max<size_t>(
        NA * tc_tile_bytes(p.KP, p.rows_pad) + (size_t)TC_NS * NB * tc_block_bytes(p.KP, NT) + 1024, 80 * 1024);
    cudaError_t e = smem_limit<k_conv_tc<NT, TERMS>>(smem);
    if (e != cudaSuccess) return e;
    CUtensorMap th, tl;
    memset(&tl, 0, sizeof(tl));
    if (!tc_map(&th, p.Ap_hi, p.Wp, p.Hp, p.C, p.rows_pad / 2)) return cudaErrorInvalidValue;
    if (TERMS == 3 && !tc_map(&tl, p.Ap_lo, p.Wp, p.Hp, p.C, p.rows_pad / 2)) return cudaErrorInvalidValue;
    const dim3 grid(p.W / NT, p.H / TC_ROWS_OUT, p.n_groups);
    launch_pdl(k_conv_tc<NT, TERMS>, grid, TC_THREADS, smem, s, p, th, tl);
    return cudaGetLastError();
}

}  // namespace

size_t tc_block_bytes_host(int kp) { return tc_block_bytes(kp, TC_NT); }

bool tc_conv_supported(int H, int W, int max_R)
{
    const int rows_pad = (TC_ROWS_OUT + 2 * max_R + 15) / 16 * 16;
    const int kp = (TC_NT + 2 * max_R + 15) / 16 * 16;
    return H % TC_ROWS_OUT == 0 && W % TC_NT == 0 && rows_pad / 2 <= 256 &&
           2 * tc_tile_bytes(kp, rows_pad) + (size_t)TC_NS * 2 * tc_block_bytes(kp, TC_NT) + 1024 <= 227 * 1024;
}

cudaError_t launch_conv_tc(const TcConvParams& p, const float* A, cudaStream_t s)
{
    int blocks = (int)std::min<size_t>(((size_t)p.C * p.Hp * p.Wp + 255) / 256, 4096);
    launch_pdl(k_tc_pad, blocks, 256, 0, s, A, p.C, p.H, p.W, p.R, p.Hp, p.Wp, reinterpret_cast<__nv_bfloat16*>(p.Ap_hi),
                                    p.terms == 3 ? reinterpret_cast<__nv_bfloat16*>(p.Ap_lo) : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return p.terms == 3 ? launch_tc<TC_NT, 3>(p, s) : launch_tc<TC_NT, 1>(p, s);
}

}  // namespace lenia
