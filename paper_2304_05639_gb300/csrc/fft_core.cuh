// Shared-memory FFT building blocks for the spectral convolution route
// (convolution theorem, note after Algorithm 2 of arXiv 2304.05639:
// X * Y = F^-1(F X . F Y)).
//
// A length-N complex FFT (N a power of two) runs as a sequence of Stockham
// decimation-in-time passes.  In one pass of radix R with sub-transform size
// Ns, butterfly j (0 <= j < N/R) reads x[j + r N/R] (r < R), multiplies by
// w^{r k} with k = j mod Ns and w = exp(-+2 pi i / (Ns R)), takes an R-point
// DFT in registers and writes y_q to position (j - k) R + k + q Ns.  After
// the passes (Ns = 1, R, R^2, ...) the output is in natural order.
//
// Each pass reads all of a thread's butterfly inputs into registers, waits at
// a block barrier, then writes, so a single shared buffer serves as source and
// destination.  The first pass can read through a caller-supplied functor
// (global memory, or a spectral product) and the last pass can write through
// one, which saves two shared-memory round trips per transform.
//
// Twiddles come from FP32 tables built in FP64 on the host and rounded once.
// Each pass with Ns > 1 has its own table laid out [r - 1][k]:
// tw[(r - 1) Ns + k] = exp(-2 pi i r k / (Ns R)), so the lanes of a warp
// (consecutive k) read consecutive entries.  The passes' tables are stored
// back to back in plan order (fft_tw_offset).  A butterfly loads w^b (b < 4)
// and w^(4a) and forms w^(4a + b) as their product: 6 loads instead of 15
// at radix 16, one more rounding on 9 of the twiddles (the rms error of a
// 512^2, 15-kernel convolution moves from 9.7e-9 to 1.1e-8).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace lenia {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// The same sums on packed FP32 pairs (sm_100 family f32x2 instructions, one
// instruction per complex add; round-to-nearest like the scalar forms, so
// the results are identical).  PK selects them in the butterflies below.
template <bool PK>
__device__ __forceinline__ float2 cadd_(float2 a, float2 b)
{
    if constexpr (PK) return __fadd2_rn(a, b);
    else return cadd(a, b);
}
template <bool PK>
__device__ __forceinline__ float2 csub_(float2 a, float2 b)
{
    if constexpr (PK) return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
    else return csub(a, b);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(pi q / 16) and sin(pi q / 16) for q = 0..15 (decimal expansions of
// cos(pi/16), cos(pi/8), cos(3 pi/16), sqrt(2)/2 and their complements).
struct C32 {
    static constexpr float k1 = 0.980785280403230449126f;   // cos(pi/16)
    static constexpr float k2 = 0.923879532511286756128f;   // cos(pi/8)
    static constexpr float k3 = 0.831469612302545237079f;   // cos(3 pi/16)
    static constexpr float k4 = 0.707106781186547524401f;   // cos(pi/4)
    static constexpr float k5 = 0.555570233019602224743f;   // cos(5 pi/16) = sin(3 pi/16)
    static constexpr float k6 = 0.382683432365089771728f;   // cos(3 pi/8)  = sin(pi/8)
    static constexpr float k7 = 0.195090322016128267848f;   // cos(7 pi/16) = sin(pi/16)
    __host__ __device__ static constexpr float cosq(int q)
    {
        return q == 0 ? 1.f : q == 1 ? k1 : q == 2 ? k2 : q == 3 ? k3 : q == 4 ? k4 : q == 5 ? k5 : q == 6 ? k6
             : q == 7 ? k7 : q == 8 ? 0.f : -cosq(16 - q);
    }
    __host__ __device__ static constexpr float sinq(int q) { return q <= 8 ? cosq(8 - q) : cosq(q - 8); }
};

// w_R^q = exp(-+2 pi i q / R) applied to a, for q < R/2 (compile-time).
template <int R, int Q, bool INV, bool PK = false>
__device__ __forceinline__ float2 rot(float2 a)
{
    static_assert(R == 2 || R == 4 || R == 8 || R == 16 || R == 32, "radix");
    constexpr int q32 = Q * (32 / R);   // angle in units of 2 pi / 32 = pi / 16
    if constexpr (q32 == 0) return a;
    else if constexpr (q32 == 8) return mul_mi<INV>(a);
    else {
        constexpr float c = C32::cosq(q32);
        constexpr float s = C32::sinq(q32);
        // forward: multiply by (c - i s); inverse by (c + i s)
        if constexpr (PK)
            return INV ? __ffma2_rn(make_float2(a.y, a.x), make_float2(-s, s), __fmul2_rn(a, make_float2(c, c)))
                       : __ffma2_rn(make_float2(a.y, a.x), make_float2(s, -s), __fmul2_rn(a, make_float2(c, c)));
        else
            return INV ? make_float2(a.x * c - a.y * s, a.x * s + a.y * c)
                       : make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
    }
}

// In-register R-point DFT, natural-order input and output (radix-2 split).
template <int R, bool INV, bool PK = false>
struct DFT {
    template <int Q>
    __device__ __forceinline__ static void combine(float2* v, const float2* e, const float2* o)
    {
        if constexpr (Q < R / 2) {
            float2 t = rot<R, Q, INV, PK>(o[Q]);
            v[Q] = cadd_<PK>(e[Q], t);
            v[Q + R / 2] = csub_<PK>(e[Q], t);
            combine<Q + 1>(v, e, o);
        }
    }
    __device__ __forceinline__ static void run(float2* v)
    {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; i++) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        DFT<R / 2, INV, PK>::run(e);
        DFT<R / 2, INV, PK>::run(o);
        combine<0>(v, e, o);
    }
};
template <bool INV, bool PK>
struct DFT<2, INV, PK> {
    __device__ __forceinline__ static void run(float2* v)
    {
        float2 a = v[0], b = v[1];
        v[0] = cadd_<PK>(a, b);
        v[1] = csub_<PK>(a, b);
    }
};
template <bool INV, bool PK>
struct DFT<1, INV, PK> {
    __device__ __forceinline__ static void run(float2*) {}
};

// Radix plan: passes of radix RMAX while at least RMAX remains, then the rest.
__host__ __device__ constexpr int fft_radix(int remaining, int rmax = 16)
{
    return remaining >= rmax ? rmax : remaining;
}

// Offset of the twiddle table of the pass with sub-transform size NS in the
// concatenated per-pass tables of a length-N transform; fft_tw_offset(N, N)
// is the total length.
__host__ __device__ constexpr int fft_tw_offset(int N, int NS, int rmax = 16)
{
    int off = 0;
    for (int ns = 1; ns < NS && ns < N; ns *= fft_radix(N / ns, rmax))
        if (ns > 1) off += (fft_radix(N / ns, rmax) - 1) * ns;
    return off;
}

// One Stockham pass over NB independent length-N transforms held by a block of
// T threads.  Element i of transform b is read with ld(b, i) and written with
// st(b, i, v).  BFAST: consecutive threads take consecutive transforms b
// (interleaved layouts), else consecutive butterflies j.  SW: each warp's
// butterflies and shared-memory elements belong to the warp alone (one
// transform per warp), so the pass synchronises the warp, not the block.
// TWC: only w and w^4 come from the table; w^2, w^3 and w^(4a) for a > 1 are
// products of them (squarings first, at most three roundings deep), which
// trades table loads through L1 for multiplies.
template <int N, int R, int NB, int T, bool INV, bool BFAST, bool PK = false, bool SW = false, bool TWC = false,
          class LD, class ST>
__device__ __forceinline__ void fft_pass(int Ns, const float2* __restrict__ twp, LD ld, ST st)
{
    constexpr int NBF = NB * (N / R);
    constexpr int PER = (NBF + T - 1) / T;
    float2 v[PER][R];
    const int tstep = N / R;
#pragma unroll
    for (int p = 0; p < PER; p++) {
        const int u = threadIdx.x + p * T;
        if (NBF % T == 0 || u < NBF) {
            const int b = BFAST ? (u % NB) : (u / (N / R));
            const int j = BFAST ? (u / NB) : (u % (N / R));
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; r++) v[p][r] = ld(b, j + r * tstep);
            if (Ns > 1) {
                // w^r for r = 4a + b: w^b (b < 4) and w^(4a) from the table,
                // their product for the others (one rounding more)
                float2 wb[4], wa[R / 4 > 0 ? R / 4 : 1];
                if constexpr (TWC && R >= 8) {
                    wb[1] = __ldg(&twp[k]);
                    wa[1] = __ldg(&twp[3 * Ns + k]);
                    wb[2] = cmul(wb[1], wb[1]);
                    wb[3] = cmul(wb[2], wb[1]);
                    if constexpr (R >= 16) {
                        wa[2] = cmul(wa[1], wa[1]);
                        wa[3] = cmul(wa[2], wa[1]);
                    }
                    if constexpr (R >= 32) {
                        wa[4] = cmul(wa[2], wa[2]);
                        wa[5] = cmul(wa[4], wa[1]);
                        wa[6] = cmul(wa[4], wa[2]);
                        wa[7] = cmul(wa[6], wa[1]);
                    }
                } else {
#pragma unroll
                    for (int b2 = 1; b2 < 4 && b2 < R; b2++) wb[b2] = __ldg(&twp[(b2 - 1) * Ns + k]);
#pragma unroll
                    for (int a = 1; a < R / 4; a++) wa[a] = __ldg(&twp[(4 * a - 1) * Ns + k]);
                }
#pragma unroll
                for (int r = 1; r < R; r++) {
                    const int a = r / 4, b2 = r % 4;
                    const float2 w = a == 0 ? wb[b2] : (b2 == 0 ? wa[a] : cmul(wa[a], wb[b2]));
                    v[p][r] = INV ? cmulc(v[p][r], w) : cmul(v[p][r], w);
                }
            }
            DFT<R, INV, PK>::run(v[p]);
        }
    }
    if constexpr (SW) __syncwarp();
    else __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; p++) {
        const int u = threadIdx.x + p * T;
        if (NBF % T == 0 || u < NBF) {
            const int b = BFAST ? (u % NB) : (u / (N / R));
            const int j = BFAST ? (u / NB) : (u % (N / R));
            const int k = j & (Ns - 1);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int q = 0; q < R; q++) {
                // a writer that also takes (p, q) can place the output in registers
                if constexpr (std::is_invocable_v<ST, int, int, float2, int, int>) st(b, base + q * Ns, v[p][q], p, q);
                else st(b, base + q * Ns, v[p][q]);
            }
        }
    }
    if constexpr (SW) __syncwarp();
    else __syncthreads();
}

// Full transform: pass 1 reads with ld_first, middle passes use the shared
// accessors sld/sst, the last pass writes with st_last.  With a single pass
// the first reader and the last writer are used together.
template <int N, int NB, int T, bool INV, bool BFAST, int RMAX = 16, int NS = 1, bool PK = false, bool SW = false,
          bool TWC = false, class LF, class SL, class SS, class STL>
__device__ __forceinline__ void fft_run(const float2* __restrict__ tw, LF ld_first, SL sld, SS sst, STL st_last)
{
    constexpr int R = fft_radix(N / NS, RMAX);
    constexpr bool first = (NS == 1);
    constexpr bool last = (NS * R == N);
    const float2* twp = tw + fft_tw_offset(N, NS, RMAX);
    if constexpr (first && last) {
        fft_pass<N, R, NB, T, INV, BFAST, PK, SW, TWC>(NS, twp, ld_first, st_last);
    } else if constexpr (first) {
        fft_pass<N, R, NB, T, INV, BFAST, PK, SW, TWC>(NS, twp, ld_first, sst);
        fft_run<N, NB, T, INV, BFAST, RMAX, NS * R, PK, SW, TWC>(tw, ld_first, sld, sst, st_last);
    } else if constexpr (last) {
        fft_pass<N, R, NB, T, INV, BFAST, PK, SW, TWC>(NS, twp, sld, st_last);
    } else {
        fft_pass<N, R, NB, T, INV, BFAST, PK, SW, TWC>(NS, twp, sld, sst);
        fft_run<N, NB, T, INV, BFAST, RMAX, NS * R, PK, SW, TWC>(tw, ld_first, sld, sst, st_last);
    }
}

// Shared-memory index swizzle: one float2 of padding per 16 (per 32 for the
// radix-32 row transforms, whose first pass writes with stride 32) keeps the
// power-of-two strides of the first passes off a single bank.
__device__ __forceinline__ int swz(int i) { return i + (i >> 4); }
// XOR form without padding (column transforms): element i of each aligned
// group of 16 moves to slot (i mod 16) xor (i / 16 mod 16), which spreads the
// stride-16 stores of the first two radix-16 passes over all 16 bank pairs.
__device__ __forceinline__ int swx(int i) { return i ^ ((i >> 4) & 15); }
__host__ __device__ constexpr int swz_size(int n) { return n + (n >> 4) + 1; }
__device__ __forceinline__ int swz32(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int swz32_size(int n) { return n + (n >> 5) + 1; }
// Pitch of one row transform when several rows are walked row-fastest
// (8 rows x 2 columns per half-warp): a pitch of 2 (mod 16) float2 puts those
// 16 accesses on 16 distinct bank pairs.
__host__ __device__ constexpr int row_pitch(int n) { return (swz32_size(n) + 15) / 16 * 16 + 2; }

}  // namespace lenia
