// Spectral convolution U_k = K~_k * A_src(k) for all kernels (convolution
// theorem, note after Algorithm 2 of arXiv 2304.05639; cached kernel
// spectra, Section 2.4).
//
// Three passes over the world, each a set of shared-memory FFTs:
//   rows_r2c  : real row FFT of every channel row (length-W real signal as a
//               length-W/2 complex FFT plus the standard even/odd split),
//               NB rows per block.  Spectra are stored column-major,
//               [channel][kx][y], kx < W/2; element kx = 0 packs the two real
//               values X[0] (DC) and X[W/2] (Nyquist) as (re, im).
//   cols_conv : one spectrum column per block: forward column FFT, then for
//               each kernel reading that channel the product with the real
//               kernel spectrum and the inverse column FFT, stored
//               [kernel][kx][y].  Column 0 holds the packed DC and Nyquist
//               columns (both real along y), which are separated, multiplied
//               by their own spectra and re-packed in one step.
//   rows_c2r  : inverse real row FFT of every kernel row -> U_k, NB rows per
//               block, staged from the column-major spectra by tiled TMA loads.
// Forward and inverse transforms are unnormalised; 1/(H W) is folded into
// the stored kernel spectra.
#include <mutex>
#include <utility>
#include <vector>

#include "fft_core.cuh"
#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

// ---------------------------------------------------------------- rows R2C
// BULK: the block's NB rows are contiguous in A; one bulk copy stages them,
// unswizzled, at the start of the work buffer, and the first pass reads them
// from there (its stores follow the pass's barrier, so the two layouts may
// share the buffer).  Otherwise the first pass reads A directly.
// Where every pass has 32 butterflies per row (M = 1024: two radix-32
// passes) and a block has one warp per row, each row instead gets its own
// bulk copy and mbarrier and lands at its work pitch, and its warp
// transforms it in place as soon as it arrives, synchronising only itself;
// the block meets once, before the even/odd split that mixes rows.
template <int M, int T, int NB, bool BULK>
__global__ void __launch_bounds__(T, 3) k_rows_r2c(FftParams p)
{
    pdl_enter();
    extern __shared__ float4 sm4[];
    float2* sm = reinterpret_cast<float2*>(sm4);
    constexpr int SZ = row_pitch(M);
    const int c = blockIdx.y;
    const int y0 = blockIdx.x * NB;
    const int W = 2 * M;
    const float* plane = p.A_list ? p.A_list[c / p.cw] + (size_t)(c % p.cw) * p.H * W : p.A + (size_t)c * p.H * W;
    const float2* src = reinterpret_cast<const float2*>(plane + (size_t)y0 * W);
    auto sld = [&](int b, int i) { return sm[b * SZ + swz32(i)]; };
    auto sst = [&](int b, int i, float2 v) { sm[b * SZ + swz32(i)] = v; };
    // two radix-32 passes of 32 butterflies per row, one warp per row
    constexpr bool ROWPIPE = BULK && ROW_RMAX == 32 && M == 32 * 32 && T == 32 * NB;
    if constexpr (ROWPIPE) {
        __shared__ uint64_t bars[NB];
        if (threadIdx.x == 0) {
            for (int b = 0; b < NB; b++) mbar_init(&bars[b], 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int b = 0; b < NB; b++) {
                mbar_arrive_expect_tx(&bars[b], (uint32_t)M * sizeof(float2));
                bulk_g2s(sm + (size_t)b * SZ, src + (size_t)b * M, (uint32_t)M * sizeof(float2), &bars[b]);
            }
        }
        const bool landed = mbar_wait_bounded(&bars[threadIdx.x >> 5], 0);    // this warp's row
        auto ld_s = [&](int b, int i) { return sm[b * SZ + i]; };
        fft_run<M, NB, T, false, false, ROW_RMAX, 1, false, true>(p.tw_M, ld_s, sld, sst, sst);
        if (!__syncthreads_and(landed)) {
            if (threadIdx.x == 0) {
                if (p.status) atomicExch(p.status, kStatusWaitTimeout);
                for (int b = 0; b < NB; b++) mbar_wait_bounded(&bars[b], 0);
            }
            return;
        }
    } else if constexpr (BULK) {
        __shared__ uint64_t bar;
        constexpr uint32_t bytes = (uint32_t)NB * M * sizeof(float2);
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&bar, bytes);
            bulk_g2s(sm, src, bytes, &bar);
        }
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0));
        if (!ok) {
            // the copy did not land in time: report it, give it a last bounded
            // chance to finish before the block's shared memory is released
            if (threadIdx.x == 0) {
                if (p.status) atomicExch(p.status, kStatusWaitTimeout);
                mbar_wait_bounded(&bar, 0);
            }
            return;
        }
        auto ld_s = [&](int b, int i) { return sm[b * M + i]; };
        fft_run<M, NB, T, false, false, ROW_RMAX>(p.tw_M, ld_s, sld, sst, sst);
    } else {
        auto ld_g = [&](int b, int i) { return __ldg(&src[(size_t)b * M + i]); };
        fft_run<M, NB, T, false, false, ROW_RMAX>(p.tw_M, ld_g, sld, sst, sst);
    }

    // X[k] = E[k] + w_W^k O[k], E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / 2i
    // Output column kx holds rows y0 .. y0 + NB - 1 contiguously (b fastest).
    float2* outc = p.Ahat + (size_t)c * M * p.H + y0;
    // four pairs per thread in flight (their twiddle loads overlap): 0.035 ->
    // 0.033 ms at 2048^2, although the registers rise from 80 to 90
#pragma unroll 4
    for (int u = threadIdx.x; u < NB * (M / 2 + 1); u += T) {
        const int b = u % NB;
        const int k = u / NB;
        if (k == 0) {
            float2 z = sm[b * SZ + swz32(0)];
            outc[b] = make_float2(z.x + z.y, z.x - z.y);
            continue;
        }
        const float2 zk = sm[b * SZ + swz32(k)];
        const float2 zm = sm[b * SZ + swz32(M - k)];
        {
            float2 e = cscale(cadd(zk, cconj(zm)), 0.5f);
            float2 d = cscale(csub(zk, cconj(zm)), 0.5f);
            float2 o = make_float2(d.y, -d.x);               // d / i
            outc[(size_t)k * p.H + b] = cadd(e, cmul(__ldg(&p.tw_W[k]), o));
        }
        if (k != M - k) {
            float2 e = cscale(cadd(zm, cconj(zk)), 0.5f);
            float2 d = cscale(csub(zm, cconj(zk)), 0.5f);
            float2 o = make_float2(d.y, -d.x);
            outc[(size_t)(M - k) * p.H + b] = cadd(e, cmul(__ldg(&p.tw_W[M - k]), o));
        }
    }
}

// Tensor map of a column-major spectrum stack [planes][M][H] of float2,
// viewed as (H, M, planes) 8-byte elements, with boxes of box_y x box_x x 1.
// Encoded maps are cached by argument (most recent first).
static bool spectrum_map(CUtensorMap* out, const float2* base, int H, int M, int planes, int box_y, int box_x)
{
    struct Key {
        const void* base;
        int H, M, planes, by, bx;
        bool operator==(const Key& o) const
        {
            return base == o.base && H == o.H && M == o.M && planes == o.planes && by == o.by && bx == o.bx;
        }
    };
    static std::mutex mu;
    static std::vector<std::pair<Key, CUtensorMap>> cache;
    const Key key{base, H, M, planes, box_y, box_x};
    std::lock_guard<std::mutex> lock(mu);
    for (size_t i = 0; i < cache.size(); i++)
        if (cache[i].first == key) {
            *out = cache[i].second;
            return true;
        }
    auto fn = tensor_map_encoder();
    if (!fn || ((uintptr_t)base & 15) != 0) return false;
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)H, (cuuint64_t)M, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)H * 8, (cuuint64_t)M * H * 8};
    const cuuint32_t box[3] = {(cuuint32_t)box_y, (cuuint32_t)box_x, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cache.insert(cache.begin(), {key, m});
    if (cache.size() > 64) cache.pop_back();
    *out = m;
    return true;
}

// ---------------------------------------------------------------- rows C2R
// Tiled TMA loads stage the block's NB rows of a kernel's column-major
// spectrum: boxes of NB rows x C2R_BOX columns, landing as [kx][b] in the
// work buffer (128-byte aligned).  The first radix-32 pass reads X[q] and
// X[M - q] from there, forms
//   Z'[q] = (X[q] + conj X[M-q]) + i w_W^{-q} (X[q] - conj X[M-q])   (= 2 Z[q]),
// and, after its barrier, writes the swizzled work layout over the staged
// data.  Lanes take consecutive rows first, so each warp's staged reads
// cover 256 contiguous bytes.
constexpr int C2R_BOX = 256;                   // spectrum columns per TMA box (the box limit)

template <int M, int T, int NB>
__global__ void __launch_bounds__(T, (512 / T) < 8 ? (512 / T) : 8)
    k_rows_c2r(FftParams p, const __grid_constant__ CUtensorMap tm_uhat)
{
    pdl_enter();
    constexpr int R = fft_radix(M, ROW_RMAX);
    static_assert(R == 32 || R == M, "first inverse row pass is radix 32");
    constexpr int BX = M < C2R_BOX ? M : C2R_BOX;
    extern __shared__ float4 sm4[];
    __shared__ uint64_t bar;
    float2* sm = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(sm4) +
                                           ((128 - (smem_addr(sm4) & 127)) & 127));
    constexpr int SZ = row_pitch(M);
    const int k = blockIdx.y;
    const int y0 = blockIdx.x * NB;
    const int W = 2 * M;

    constexpr uint32_t bytes = (uint32_t)NB * M * sizeof(float2);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, bytes);
#pragma unroll
        for (int i = 0; i < M / BX; i++) tma_load_3d(sm + (size_t)i * BX * NB, &tm_uhat, y0, i * BX, k, &bar);
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0));
    if (!ok) {
        if (threadIdx.x == 0) {
            if (p.status) atomicExch(p.status, kStatusWaitTimeout);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }

    float2* out = reinterpret_cast<float2*>(p.U + ((size_t)k * p.H + y0) * W);
    const float2* addp = p.add ? reinterpret_cast<const float2*>(p.add + ((size_t)k * p.H + y0) * W) : nullptr;
    auto st_g = [&](int b, int i, float2 v) {
        if (addp) {
            const float2 a = __ldg(&addp[(size_t)b * M + i]);
            v = make_float2(a.x + v.x, a.y + v.y);
        }
        out[(size_t)b * M + i] = v;
    };
    auto sld = [&](int b, int i) { return sm[b * SZ + swz32(i)]; };
    auto sst = [&](int b, int i, float2 v) { sm[b * SZ + swz32(i)] = v; };
    auto stg = [&](int b, int q) { return sm[q * NB + b]; };      // staged element (row b, column q)

    constexpr int JB = M / R;                        // butterflies per row
    constexpr int NBF = NB * JB;
    constexpr int PER = (NBF + T - 1) / T;
    float2 v[PER][R];
#pragma unroll
    for (int it = 0; it < PER; it++) {
        const int u = threadIdx.x + it * T;
        if (NBF % T == 0 || u < NBF) {
            const int b = u % NB, j = u / NB;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int q = j + r * JB;
                const float2 xk = stg(b, q);
                if (q == 0) {                                  // (DC, Nyquist)
                    v[it][r] = make_float2(xk.x + xk.y, xk.x - xk.y);
                } else {
                    const float2 xm = stg(b, M - q);
                    const float2 sp = cadd(xk, cconj(xm));
                    const float2 d = cmulc(csub(xk, cconj(xm)), __ldg(&p.tw_W[q]));
                    v[it][r] = make_float2(sp.x - d.y, sp.y + d.x);   // s + i d
                }
            }
            DFT<R, true>::run(v[it]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < PER; it++) {
        const int u = threadIdx.x + it * T;
        if (NBF % T == 0 || u < NBF) {
            const int b = u % NB, j = u / NB;
#pragma unroll
            for (int q = 0; q < R; q++) {
                if constexpr (R == M) st_g(b, j * R + q, v[it][q]);
                else sst(b, j * R + q, v[it][q]);
            }
        }
    }
    if constexpr (R < M) {
        __syncthreads();
        fft_run<M, NB, T, true, false, ROW_RMAX, R>(p.tw_M, sld, sld, sst, st_g);
    }
}

// ------------------------------------------------------- columns: fwd, x K^, inv
// The column transforms use packed FP32-pair butterflies (PK = true; 7%
// faster on a 2048^2 world); the row transforms, whose radix-32 butterflies
// are register-bound, run faster with scalar ones.
// PERK: one block per (column, channel, kernel of that channel), grid z = the
// longest kernel list: shorter serial chains for small grids, at the cost of
// repeating the forward column transform for every kernel of a channel.
// Column passes of H >= 2048 keep each thread's share of the forward column
// spectrum in tensor memory (TMEM) instead of a second shared-memory buffer:
// one H-element work buffer and one kernel-spectrum column per block, so that
// eight blocks fit on an SM.
template <int H>
__host__ __device__ constexpr bool cols_tmem() { return H >= 2048; }
__host__ __device__ constexpr int cols_spec_floats(int H) { return (H / 2 + 1 + 3) / 4 * 4; }
template <int H>
__host__ __device__ constexpr size_t cols_smem_bytes()
{
    return (cols_tmem<H>() ? 1 : 2) * (size_t)H * 8 + (size_t)cols_spec_floats(H) * 4;
}

// Column 0 of the packed spectrum holds the DC and Nyquist columns (both
// real along y): out = f a + conj(f(-ky)) b with a, b from the two kernel
// spectra.  It runs in one H-element buffer, repeating the forward
// transform for each kernel (one block in M), and out of line so that its
// registers do not weigh on the other columns' code.
template <int H, int T>
__device__ __noinline__ void cols_conv_dc(const FftParams& p, float2* Bf, int plane, int c, int w, int t0, int nk,
                                          const float* Sw)
{
    const int M = p.W / 2;
    const int HS = H / 2 + 1;
    const float2* src = p.Ahat + (size_t)plane * M * H;
    auto ld_g = [&](int, int i) { return __ldg(&src[i]); };
    auto sld = [&](int, int i) { return Bf[swx(i)]; };
    auto sst = [&](int, int i, float2 v) { Bf[swx(i)] = v; };
    for (int t = t0; t < nk; t++) {
        fft_run<H, 1, T, false, false, 16, 1, true, false, true>(p.tw_H, ld_g, sld, sst, sst);
        const int k = p.klist[c][t];
        const float* Sk = Sw + (size_t)k * (M + 1) * HS;
        // the first inverse pass reads every input before its barrier, so it
        // may write the same buffer
        auto ld_mul = [&](int, int i) {
            const int kyr = i <= H / 2 ? i : H - i;
            const float2 f = Bf[swx(i)];
            const float s0 = __ldg(&Sk[kyr]);
            const float sn = __ldg(&Sk[(size_t)M * HS + kyr]);
            const float2 fm = cconj(Bf[swx((H - i) & (H - 1))]);
            const float a = 0.5f * (s0 + sn), bb = 0.5f * (s0 - sn);
            return make_float2(f.x * a + fm.x * bb, f.y * a + fm.y * bb);
        };
        float2* dst = p.Uhat + ((size_t)(w * p.kpw + k - p.k_base) * M) * H;
        auto st_g = [&](int, int i, float2 v) { dst[i] = v; };
        fft_run<H, 1, T, true, false, 16, 1, true, false, true>(p.tw_H, ld_mul, sld, sst, st_g);
    }
}

// One-warp blocks (columns of at most 512 points) are held to 128 registers,
// 16 blocks per SM: the 256-world batch steps in 0.254 instead of 0.267 ms
// (167-181 registers left 11 per SM; 80 registers measured 0.266 ms).
template <int H, int T, bool PERK>
__global__ void __launch_bounds__(T, T == 32 ? 16 : (1024 / T < 8 ? 1024 / T : 8)) k_cols_conv(FftParams p)
{
    pdl_enter();
    constexpr bool TM = cols_tmem<H>();
    extern __shared__ float2 sm[];
    float2* F = sm;                                         // forward spectrum (smem variant)
    float2* Wk = TM ? sm : sm + H;                          // inverse work buffer
    float* Sb = reinterpret_cast<float*>(sm + (TM ? H : 2 * H));   // the current kernel's spectrum column
    const int plane = blockIdx.y;              // Ahat plane: channel c of world w
    const int c = plane % p.cw, w = plane / p.cw;
    const int kx = blockIdx.x;
    const int M = p.W / 2;
    const int HS = H / 2 + 1;
    if (PERK && (int)blockIdx.z >= p.kcount[c]) return;     // uniform over the block
    const int t0 = PERK ? (int)blockIdx.z : 0;
    const int nk = PERK ? t0 + 1 : p.kcount[c];
    const float* Sw = p.S_list ? p.S_list[w] : p.S;
    if (kx == 0) {
        cols_conv_dc<H, T>(p, sm, plane, c, w, t0, nk, Sw);
        return;
    }

    const float2* src = p.Ahat + ((size_t)plane * M + kx) * H;
    auto ld_g = [&](int, int i) { return __ldg(&src[i]); };
    auto sldF = [&](int, int i) { return F[swx(i)]; };
    auto sstF = [&](int, int i, float2 v) { F[swx(i)] = v; };
    auto sldW = [&](int, int i) { return Wk[swx(i)]; };
    auto sstW = [&](int, int i, float2 v) { Wk[swx(i)] = v; };

    // Each kernel's spectrum column is copied asynchronously into Sb while
    // the previous transform runs (the first one during the forward
    // transform); the product with it is the first inverse pass's load.
    auto fetch_s = [&](int t) {
        const float* Sc = Sw + (size_t)p.klist[c][t] * (M + 1) * HS + (size_t)kx * HS;
        for (int i = threadIdx.x; i < HS; i += T) cp_async4(&Sb[i], &Sc[i]);
        cp_async_commit();
    };
    constexpr int R1 = fft_radix(H, 16);
    if constexpr (!TM) {
        if (t0 < nk) fetch_s(t0);
        fft_run<H, 1, T, false, false, 16, 1, true, false, true>(p.tw_H, ld_g, sldF, sstF, sstF);
        auto ld_mul = [&](int, int i) { return cscale(F[swx(i)], Sb[i <= H / 2 ? i : H - i]); };
        for (int t = t0; t < nk; t++) {
            const int k = p.klist[c][t];
            cp_async_wait_all();
            __syncthreads();
            float2* dst = p.Uhat + ((size_t)(w * p.kpw + k - p.k_base) * M + kx) * H;
            auto st_g = [&](int, int i, float2 v) { dst[i] = v; };
            // first pass (reads Sb, then a barrier), then the next column's copy
            fft_pass<H, R1, 1, T, true, false, true>(1, p.tw_H, ld_mul, sstW);
            if (t + 1 < nk) fetch_s(t + 1);
            fft_run<H, 1, T, true, false, 16, R1, true, false, true>(p.tw_H, sldW, sldW, sstW, st_g);
        }
    } else {
        // The first inverse pass (radix 16, one butterfly per thread) takes
        // elements j + r H/16 of the forward spectrum, the same for every
        // kernel: thread j keeps those 16 values in its TMEM lane.
        constexpr int TS = H / R1;
        static_assert(R1 == 16 && TS == T && T % 128 == 0, "one first-pass butterfly per thread");
        constexpr int NCOLS = 32 * (T / 128);
        __shared__ uint32_t tmem_base;
        const int warp = threadIdx.x >> 5, j = threadIdx.x;
        if (warp == 0) {
            tmem_alloc<NCOLS>(&tmem_base);
            tmem_fence_before_sync();
        }
        if (t0 < nk) fetch_s(t0);
        // The forward transform's last pass (sub-transforms of 256, radix
        // H / 256) leaves butterfly p of thread j with outputs j + p T + q 256
        // (q < H / 256), which are exactly this thread's elements j + r TS,
        // r = p + q (256 / T): they go from registers to TMEM, not through
        // shared memory.
        static_assert(H / 256 <= 16 && (H / 256) * (256 / T) * T == H && 256 % T == 0, "last forward pass layout");
        constexpr int PL = 256 / T;                           // butterflies per thread in the last pass
        float fv[32];
        auto st_reg = [&](int, int, float2 v, int pp, int q) {
            fv[2 * (pp + q * PL)] = v.x;
            fv[2 * (pp + q * PL) + 1] = v.y;
        };
        fft_run<H, 1, T, false, false, 16, 1, true, false, true>(p.tw_H, ld_g, sldF, sstF, st_reg);   // ends with a barrier
        tmem_fence_after_sync();
        const uint32_t taddr = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
        tmem_st16(taddr, fv);
        tmem_st16(taddr + 16, fv + 16);
        tmem_wait_st();
        for (int t = t0; t < nk; t++) {
            const int k = p.klist[c][t];
            cp_async_wait_all();
            __syncthreads();          // Sb landed; every read of the work buffer is done
            float fv[32];
            tmem_ld16(taddr, fv);
            tmem_ld16(taddr + 16, fv + 16);
            float2 v[16];
#pragma unroll
            for (int r = 0; r < 16; r++) {
                const int ky = j + r * TS;
                v[r] = cscale(make_float2(fv[2 * r], fv[2 * r + 1]), Sb[ky <= H / 2 ? ky : H - ky]);
            }
            DFT<16, true, true>::run(v);
#pragma unroll
            for (int q = 0; q < 16; q++) Wk[swx(j * 16 + q)] = v[q];
            __syncthreads();
            if (t + 1 < nk) fetch_s(t + 1);
            float2* dst = p.Uhat + ((size_t)(w * p.kpw + k - p.k_base) * M + kx) * H;
            auto st_g = [&](int, int i, float2 v) { dst[i] = v; };
            fft_run<H, 1, T, true, false, 16, R1, true, false, true>(p.tw_H, sldW, sldW, sstW, st_g);
        }
        tmem_fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            tmem_fence_after_sync();
            tmem_dealloc<NCOLS>(tmem_base);
        }
    }
}

// ---------------------------------- columns, transposed: sum_k K^_k x fwd(col_k), inv
// The adjoint of the convolution stage for every source channel c at once:
// V_c = sum_{k: src(k) = c} K~_k (x) G_k.  Per spectrum column: forward column
// FFT of each kernel's gradient plane (Ahat plane k), times the kernel's real
// spectrum, accumulated in the frequency domain; one inverse column FFT per
// channel (Uhat plane c).  Same packed (DC, Nyquist) handling as k_cols_conv.
template <int H, int T>
__global__ void __launch_bounds__(T, 1024 / T < 8 ? 1024 / T : 8) k_cols_adj(FftParams p)
{
    pdl_enter();
    extern __shared__ float2 sm[];
    float2* F = sm;
    float2* Acc = sm + H;
    const int c = blockIdx.y;
    const int kx = blockIdx.x;
    const int M = p.W / 2;
    const int HS = H / 2 + 1;
    for (int i = threadIdx.x; i < H; i += T) Acc[swx(i)] = make_float2(0.f, 0.f);
    auto sldF = [&](int, int i) { return F[swx(i)]; };
    auto sstF = [&](int, int i, float2 v) { F[swx(i)] = v; };
    const int nk = p.kcount[c];
    for (int t = 0; t < nk; t++) {
        const int k = p.klist[c][t];
        const float2* src = p.Ahat + ((size_t)k * M + kx) * H;
        auto ld_g = [&](int, int i) { return __ldg(&src[i]); };
        fft_run<H, 1, T, false, false, 16, 1, true, false, true>(p.tw_H, ld_g, sldF, sstF, sstF);
        const float* Sk = p.S + (size_t)k * (M + 1) * HS;
        // each thread updates its own entries of Acc (no barrier needed between
        // the zeroing and the updates); F is complete after fft_run's barrier
        for (int i = threadIdx.x; i < H; i += T) {
            const int kyr = i <= H / 2 ? i : H - i;
            const float2 f = F[swx(i)];
            float2 v;
            if (kx == 0) {
                const float s0 = __ldg(&Sk[kyr]);
                const float sn = __ldg(&Sk[(size_t)M * HS + kyr]);
                const float2 fm = cconj(F[swx((H - i) & (H - 1))]);
                const float a = 0.5f * (s0 + sn), bb = 0.5f * (s0 - sn);
                v = make_float2(f.x * a + fm.x * bb, f.y * a + fm.y * bb);
            } else {
                v = cscale(f, __ldg(&Sk[(size_t)kx * HS + kyr]));
            }
            Acc[swx(i)] = cadd(Acc[swx(i)], v);
        }
    }
    __syncthreads();
    float2* dst = p.Uhat + ((size_t)c * M + kx) * H;
    auto ld_acc = [&](int, int i) { return Acc[swx(i)]; };
    auto st_g = [&](int, int i, float2 v) { dst[i] = v; };
    fft_run<H, 1, T, true, false, 16, 1, true, false, true>(p.tw_H, ld_acc, sldF, sstF, st_g);
}

// ------------------------------------------------------------ dispatch
template <int M, int NB>
static cudaError_t rows_launch_nb(const FftParams& p, cudaStream_t s, bool inverse)
{
    constexpr int T0 = NB * M / ROW_RMAX;
    constexpr int T1 = T0 < 32 ? 32 : (T0 < 512 ? T0 : 512);
    constexpr int TI = T1;
    const size_t smem = (size_t)NB * row_pitch(M) * sizeof(float2);
    if (p.H % NB) return cudaErrorInvalidValue;
    if (!inverse) {
        // bulk staging needs 16-byte aligned rows (always, for 16-byte aligned A;
        // a batched launch's caller checks every listed pointer)
        if (p.A_list ? p.list_aligned != 0 : ((uintptr_t)p.A & 15) == 0) {
            cudaError_t e = smem_limit<k_rows_r2c<M, T1, NB, true>>(smem);
            if (e != cudaSuccess) return e;
            launch_pdl(k_rows_r2c<M, T1, NB, true>, dim3(p.H / NB, p.C), T1, smem, s, p);
        } else {
            cudaError_t e = smem_limit<k_rows_r2c<M, T1, NB, false>>(smem);
            if (e != cudaSuccess) return e;
            launch_pdl(k_rows_r2c<M, T1, NB, false>, dim3(p.H / NB, p.C), T1, smem, s, p);
        }
    } else {
        // column-major spectrum [plane][kx][y] as (y, kx, plane) of 8-byte elements
        CUtensorMap tm;
        constexpr int BX = M < C2R_BOX ? M : C2R_BOX;
        if (!spectrum_map(&tm, p.Uhat, p.H, M, p.K, NB, BX)) return cudaErrorInvalidValue;
        cudaError_t e = smem_limit<k_rows_c2r<M, TI, NB>>(smem + 128);
        if (e != cudaSuccess) return e;
        launch_pdl(k_rows_c2r<M, TI, NB>, dim3(p.H / NB, p.K), TI, smem + 128, s, p, tm);
    }
    return cudaGetLastError();
}

template <int M>
static cudaError_t rows_launch(const FftParams& p, cudaStream_t s, bool inverse)
{
    // at least 8 rows per block (64-byte runs of the column-major spectra) and
    // at least 4096 complex values; one radix-ROW_RMAX butterfly per thread.
    // Grids that would have fewer than 256 blocks (small worlds, few planes)
    // take 8 rows per block instead, for parallelism.
    constexpr int NB0 = (4096 / M) > 8 ? (4096 / M) : 8;
    constexpr int NB = NB0 < 64 ? NB0 : 64;
    const int planes = inverse ? p.K : p.C;
    if (NB > 8 && (p.H / NB) * planes < 256) return rows_launch_nb<M, 8>(p, s, inverse);
    return rows_launch_nb<M, NB>(p, s, inverse);
}

template <int H>
static cudaError_t cols_launch(const FftParams& p, cudaStream_t s, bool transposed = false)
{
    // one radix-16 butterfly per thread, at least one warp (a 64-thread
    // minimum left half the threads idle in the radix-16 passes of 512-point
    // columns: 4.7% slower on the 256-world batch)
    constexpr int T = H / 16 >= 32 ? H / 16 : 32;
    const size_t smem = cols_smem_bytes<H>();
    const int M = p.W / 2;
    if (transposed) {
        const size_t smem = 2 * (size_t)H * 8;
        cudaError_t e = smem_limit<k_cols_adj<H, T>>(smem);
        if (e != cudaSuccess) return e;
        launch_pdl(k_cols_adj<H, T>, dim3(M, p.C), T, smem, s, p);
        return cudaGetLastError();
    }
    int kmax = 0;
    for (int c = 0; c < p.cw && c < kMaxChannels; c++) kmax = p.kcount[c] > kmax ? p.kcount[c] : kmax;
    // fewer than ~4 blocks per SM of a 152-SM part: one block per kernel
    if (M * p.C < 608 && kmax > 1) {
        cudaError_t e = smem_limit<k_cols_conv<H, T, true>>(smem);
        if (e != cudaSuccess) return e;
        launch_pdl(k_cols_conv<H, T, true>, dim3(M, p.C, kmax), T, smem, s, p);
    } else {
        cudaError_t e = smem_limit<k_cols_conv<H, T, false>>(smem);
        if (e != cudaSuccess) return e;
        launch_pdl(k_cols_conv<H, T, false>, dim3(M, p.C), T, smem, s, p);
    }
    return cudaGetLastError();
}

static cudaError_t rows_dispatch(const FftParams& p, cudaStream_t s, bool inverse)
{
    switch (p.W / 2) {
        case 32: return rows_launch<32>(p, s, inverse);
        case 64: return rows_launch<64>(p, s, inverse);
        case 128: return rows_launch<128>(p, s, inverse);
        case 256: return rows_launch<256>(p, s, inverse);
        case 512: return rows_launch<512>(p, s, inverse);
        case 1024: return rows_launch<1024>(p, s, inverse);
        case 2048: return rows_launch<2048>(p, s, inverse);
    }
    return cudaErrorInvalidValue;
}

static cudaError_t cols_dispatch(const FftParams& p, cudaStream_t s, bool transposed = false)
{
    switch (p.H) {
        case 64: return cols_launch<64>(p, s, transposed);
        case 128: return cols_launch<128>(p, s, transposed);
        case 256: return cols_launch<256>(p, s, transposed);
        case 512: return cols_launch<512>(p, s, transposed);
        case 1024: return cols_launch<1024>(p, s, transposed);
        case 2048: return cols_launch<2048>(p, s, transposed);
        case 4096: return cols_launch<4096>(p, s, transposed);
    }
    return cudaErrorInvalidValue;
}

bool fft_size_supported(int H, int W)
{
    auto pow2 = [](int n) { return n > 0 && (n & (n - 1)) == 0; };
    return pow2(H) && pow2(W) && H >= 64 && H <= 4096 && W >= 64 && W <= 4096;
}

cudaError_t launch_fft_rows_r2c(const FftParams& p, cudaStream_t s) { return rows_dispatch(p, s, false); }
cudaError_t launch_fft_cols(const FftParams& p, cudaStream_t s) { return cols_dispatch(p, s); }
cudaError_t launch_fft_cols_adj(const FftParams& p, cudaStream_t s) { return cols_dispatch(p, s, true); }
cudaError_t launch_fft_rows_c2r(const FftParams& p, cudaStream_t s) { return rows_dispatch(p, s, true); }

// ------------------------------------------------------- kernel spectra (FP64)
// S(ky, kx) = (1 / (H W)) sum_{dy,dx} K~(dy, dx) cos(2 pi ky dy / H) cos(2 pi kx dx / W):
// the DFT of the kernel placed on the torus; it is real and even in each axis
// because K~ depends on |d| only.  Computed in two separable FP64 sums.
__global__ void k_spec_rows(const double* Kd, int R, int W, const double* cos_W, double* T)
{
    // T[dy + R][kx] = sum_dx K(dy, dx) cos(2 pi kx dx / W), kx in 0..W/2
    const int M1 = W / 2 + 1;
    const int n = 2 * R + 1;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n * M1; u += gridDim.x * blockDim.x) {
        const int r = u / M1, kx = u % M1;
        double acc = 0.0;
        for (int dx = -R; dx <= R; dx++) {
            const int m = (int)(((long long)kx * (dx + W)) % W);
            acc += Kd[r * n + dx + R] * cos_W[m];
        }
        T[u] = acc;
    }
}

__global__ void k_spec_cols(const double* T, int R, int H, int W, const double* cos_H, float* S)
{
    // S[kx][ky] for ky in 0..H/2
    const int M1 = W / 2 + 1;
    const int HS = H / 2 + 1;
    const double scale = 1.0 / ((double)H * (double)W);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < M1 * HS; u += gridDim.x * blockDim.x) {
        const int kx = u / HS, ky = u % HS;
        double acc = 0.0;
        for (int dy = -R; dy <= R; dy++) {
            const int m = (int)(((long long)ky * (dy + H)) % H);
            acc += T[(dy + R) * M1 + kx] * cos_H[m];
        }
        S[u] = (float)(acc * scale);
    }
}

cudaError_t launch_spectra(const double* Kd, int R, int H, int W, const double* cos_H,
                           const double* cos_W, double* T_scratch, float* S_out, cudaStream_t s)
{
    const int n = 2 * R + 1;
    const int M1 = W / 2 + 1;
    int blocks = (n * M1 + 255) / 256;
    k_spec_rows<<<blocks, 256, 0, s>>>(Kd, R, W, cos_W, T_scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    blocks = (M1 * (H / 2 + 1) + 255) / 256;
    k_spec_cols<<<blocks, 256, 0, s>>>(T_scratch, R, H, W, cos_H, S_out);
    return cudaGetLastError();
}

}  // namespace lenia
