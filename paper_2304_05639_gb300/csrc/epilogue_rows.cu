// Streaming growth / gene-maintenance / update epilogue (the same per-site
// rule as step_kernels.cu: Sections 2.2-2.4 and Algorithm 2 of arXiv
// 2304.05639) for diffusion radius 1 and worlds whose width is a multiple of
// 256.
//
// Persistent layout: CTA b owns the 256-column chunk (b mod n_chunks) of a
// band of consecutive rows and walks down it.  Bulk asynchronous copies keep
// the rows it needs in shared memory, ahead of use:
//   - a 4-slot ring of gene rows: every gene plane, 256 columns plus a
//     4-column halo on each side (periodic), rows y-1, y, y+1 and y+2 in
//     flight;
//   - a 2-slot ring of potential rows (K planes) and phenospace rows (C).
// Each copy group completes on its slot's mbarrier; every wait is bounded.
// Each thread computes one column; the 5-site diffusion disk is read from
// the ring, so every gene value is fetched from global memory once.
#include <cudaTypedefs.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "lenia_internal.cuh"
#include "ptx_util.cuh"

namespace lenia {

constexpr int ER_CH = 256;             // columns per CTA
constexpr int ER_PW = ER_CH + 8;       // gene row with 4-column halos

// 0.5 * log2(e): exp(-z^2 / 2) = exp2(-C_HALF_LOG2E * z^2)
constexpr float C_HALF_LOG2E = 0.721347520444481703680f;
constexpr int ER_GROUPS = 2;                  // consumer warp groups, alternate rows
constexpr int ER_WPG = ER_CH / 32;            // warps per group, 32 columns each
constexpr int ER_CONSUMERS = ER_GROUPS * ER_WPG;
constexpr int ER_THREADS = ER_CONSUMERS * 32 + 32;   // plus one producer warp
constexpr int ER_NP = 5;                      // gene-row ring: rows i-1 .. i+2 in use, one ahead
constexpr int ER_NU = 3;                      // ring depth of potential / phenospace rows

constexpr int ALIGN_F = 32;                   // 128-byte alignment of TMA destinations, in floats
__host__ __device__ constexpr size_t round_f(size_t n) { return (n + ALIGN_F - 1) / ALIGN_F * ALIGN_F; }

// Shared-memory layout.  A gene slot holds every gene plane's row, 264
// floats each (4-column halos on both sides), as one TMA box of 132 8-byte
// elements x 1 row x NPK planes; a halo slot holds the 4 columns beyond each
// edge of the world (NPK x 4 floats per side) for the chunks at the edges.
template <int KT, int CT, int LOC, int NPD = ER_NP, int NUD = ER_NU>
struct ErLayout {
    static constexpr int NP = ((LOC & 1) != 0) + ((LOC & 2) != 0) + ((LOC & 4) != 0);
    static constexpr int NPK = NP * KT;
    static constexpr size_t p_slot = round_f((size_t)NPK * ER_PW);
    static constexpr size_t h_slot = round_f((size_t)NPK * 4);
    static constexpr size_t u_slot = (size_t)KT * ER_CH;
    static constexpr size_t a_slot = (size_t)CT * ER_CH;
    static constexpr size_t p_floats = NPD * p_slot;
    static constexpr size_t h_floats = NPD * 2 * h_slot;
    static constexpr size_t u_floats = NUD * u_slot;
    static constexpr size_t a_floats = NUD * a_slot;
    // + 128 bytes to align the base of the dynamic shared memory to 128
    static constexpr size_t bytes = (p_floats + h_floats + u_floats + a_floats) * 4 + 2 * (NPD + NUD) * 8 + 128;
};

// Destination channel of kernel k in the paper's 15-kernel topology: 3 self
// kernels per channel, then (0,1), (1,0), (0,2), (2,0), (1,2), (2,1).
__host__ __device__ constexpr int paper_dst(int k)
{
    return k < 9 ? k / 3 : (k == 9 ? 1 : k == 10 ? 0 : k == 11 ? 2 : k == 12 ? 0 : k == 13 ? 2 : 1);
}

// Warp-specialised pipeline.  The producer warp fills the rings with bulk
// copies; each slot has a "full" barrier (copy bytes landed) and an "empty"
// barrier (every consumer warp is done with it).  Two groups of consumer
// warps take alternate rows; warp w of a group computes 32 columns of its
// row, all kernels, and never waits for another consumer warp.  Local gene
// row l (global row r0 - 1 + l) is used by rows l - 2, l - 1 and l; a group
// releases rows i and i + 1 after computing row i, so each gene slot is
// released once by each group.
// TOPO = 1: kernels route to channels as in the paper's topology (checked on
// the host).  EPS0 = 1: eps_p == 0, where a zero neighbour count forces a
// non-positive sum and the saturated quotient is already 0.
//
// er_band runs this pipeline over rows r0 .. r1 - 1 of the chunk starting at
// column x0, reading through the tensor maps tm_* (generic addresses: kernel
// parameters or global memory) and writing A_out / P_out; every barrier must
// be freshly initialised.  If a bounded wait gives up it sets *blk_failed and
// the status word; last_gene / last_pot record the producer's last issued
// rows for the drain after a failure.
template <int KT, int CT, int LOC, int TOPO, int EPS0, int NPD = ER_NP, int NUD = ER_NU>
__device__ __forceinline__ void er_band(const EpiParams& p, const CUtensorMap* tm_p, const CUtensorMap* tm_u,
                                        const CUtensorMap* tm_a, const CUtensorMap* tm_h, float* A_out,
                                        float* P_out, int x0, int r0, int r1, float* Pring, float* Hring,
                                        float* Uring, float* Aring, uint64_t* full_p, uint64_t* empty_p,
                                        uint64_t* full_u, uint64_t* empty_u, float* st, int* blk_failed,
                                        int& last_gene, int& last_pot, int* status)
{
    using L = ErLayout<KT, CT, LOC, NPD, NUD>;
    constexpr int NPK = L::NPK, NP = L::NP;
    constexpr int PMU = (LOC & 1) ? 0 : -1;
    constexpr int PSG = (LOC & 2) ? ((LOC & 1) ? 1 : 0) : -1;
    constexpr int PH = (LOC & 4) ? NP - 1 : -1;
    const int H = p.H, W = p.W;
    const unsigned N = (unsigned)H * (unsigned)W;        // sites; n_p K N < 2^31 (host check)
    const int nrows = r1 - r0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool edge_l = x0 == 0, edge_r = x0 + ER_CH == W;

    if (warp == ER_CONSUMERS) {
        // ------------------------------------------------ producer warp
        // One lane issues TMA boxes; x coordinates count 8-byte elements (two
        // floats), so the gene box at x0/2 - 2 spans columns x0 - 4 .. x0 + 259.
        auto genes = [&](int l) -> bool {                      // local gene row l = global r0 - 1 + l
            if (NPK == 0) return true;
            const int slot = l % NPD;
            if (l >= NPD && !mbar_wait_bounded(&empty_p[slot], ((l - NPD) / NPD) & 1)) return false;
            int r = r0 - 1 + l;
            r = r < 0 ? r + H : (r >= H ? r - H : r);
            last_gene = l;
            if (lane == 0) {
                fence_proxy_async_shared();
                const uint32_t bytes = NPK * ER_PW * 4 + (edge_l ? NPK * 16 : 0) + (edge_r ? NPK * 16 : 0);
                mbar_arrive_expect_tx(&full_p[slot], bytes);
                tma_load_3d(Pring + slot * L::p_slot, tm_p, x0 / 2 - 2, r, 0, &full_p[slot]);
                // periodic halos of the edge chunks (the main box reads zeros there)
                if (edge_l) tma_load_3d(Hring + (slot * 2 + 0) * L::h_slot, tm_h, W / 2 - 2, r, 0, &full_p[slot]);
                if (edge_r) tma_load_3d(Hring + (slot * 2 + 1) * L::h_slot, tm_h, 0, r, 0, &full_p[slot]);
            }
            return true;
        };
        auto pot = [&](int i) -> bool {                        // potentials + phenospace of local row i
            const int slot = i % NUD;
            if (i >= NUD && !mbar_wait_bounded(&empty_u[slot], ((i - NUD) / NUD) & 1)) return false;
            const int r = r0 + i;
            last_pot = i;
            if (lane == 0) {
                mbar_arrive_expect_tx(&full_u[slot], (KT + CT) * ER_CH * 4);
                tma_load_3d(Uring + slot * L::u_slot, tm_u, x0 / 2, r, 0, &full_u[slot]);
                tma_load_3d(Aring + slot * L::a_slot, tm_a, x0 / 2, r, 0, &full_u[slot]);
            }
            return true;
        };
        // issue in order of need: row i wants gene rows up to l = i + 2 and U/A row i
        bool ok = nrows <= 0 || (genes(0) && genes(1));
        for (int i = 0; ok && i < nrows; i++) ok = genes(i + 2) && pot(i);
        if (!ok && lane == 0) {
            *blk_failed = 1;
            atomicExch(status, kStatusWaitTimeout);
        }
        // on success no copy is left in flight: the consumers waited for all of them
    } else {
        // ------------------------------------------------ consumer warps
        const int grp = warp / ER_WPG;
        const int t = (warp % ER_WPG) * 32 + lane;       // column within the chunk
        const int x = x0 + t;
        const float eps_p = p.eps_p, eps_u = p.eps_u;
        const bool stats = p.partials != nullptr;
        const float sx = stats ? __ldg(&p.sin_x[x]) : 0.f, cx = stats ? __ldg(&p.cos_x[x]) : 0.f;
        // gene row l = 0 is used by row 0 only: group 1 releases it up front
        // so that its slot, like every other, collects one release per group
        if (grp == 1 && lane == 0 && NPK > 0 && nrows > 0) mbar_arrive(&empty_p[0]);
        for (int i = grp; i < nrows; i += ER_GROUPS) {
            bool ok = true;
            if (NPK > 0)
                for (int l = i; l <= i + 2; l++) ok = ok && mbar_wait_bounded(&full_p[l % NPD], (l / NPD) & 1);
            ok = ok && mbar_wait_bounded(&full_u[i % NUD], (i / NUD) & 1);
            if (!ok) {
                if (lane == 0) {
                    *blk_failed = 1;
                    atomicExch(status, kStatusWaitTimeout);
                }
                break;
            }
            const int y = r0 + i;
            // the row's trigonometric weights, fetched before the row's arithmetic
            const float sy = stats ? __ldg(&p.sin_y[y]) : 0.f, cy = stats ? __ldg(&p.cos_y[y]) : 0.f;
            const float* Pu = Pring + (size_t)(i % NPD) * L::p_slot;
            float* Pcw = Pring + (size_t)((i + 1) % NPD) * L::p_slot;
            const float* Pc = Pcw;
            const float* Pd = Pring + (size_t)((i + 2) % NPD) * L::p_slot;
            const float* Ur = Uring + (size_t)(i % NUD) * L::u_slot;
            const float* Ar = Aring + (size_t)(i % NUD) * L::a_slot;
            // The centre row's halo column beyond a world edge arrived in the
            // halo slot; the one lane that reads it moves it into place.
            if (NPK > 0 && p.maintain && ((edge_l && t == 0) || (edge_r && t == ER_CH - 1))) {
                const int side = t == 0 ? 0 : 1;
                const float* hs = Hring + (((i + 1) % NPD) * 2 + side) * L::h_slot;
                for (int pk = 0; pk < NPK; pk++)
                    Pcw[pk * ER_PW + (side == 0 ? 3 : 4 + ER_CH)] = hs[pk * 4 + (side == 0 ? 3 : 0)];
                fence_proxy_async_shared();   // before the slot is refilled by TMA
            }

            float ph[NPK > 0 ? NPK : 1];
            float pmin = 1.f;                  // min over the diffused genes
            float tmin = 3.4e38f;              // min over the alpha tests (h g, or U)
            float tsum = 0.f;                  // their sum (Delta_sum)
            float acc[CT];
#pragma unroll
            for (int c = 0; c < CT; c++) acc[c] = 0.f;
#pragma unroll
            for (int k = 0; k < KT; k++) {
                if constexpr (NP == 2) {
                    // the kernel's two gene planes side by side on packed FP32
                    // pairs: the same additions and products, lane by lane
                    const int o0 = k * ER_PW + t + 4, o1 = (KT + k) * ER_PW + t + 4;
                    float2 v;
                    if (p.maintain) {
                        // disk |d| <= 1 in the order (-1,0), (0,-1), (0,0), (0,1), (1,0)
                        const float2 v0 = make_float2(Pu[o0], Pu[o1]), v1 = make_float2(Pc[o0 - 1], Pc[o1 - 1]),
                                     v2 = make_float2(Pc[o0], Pc[o1]), v3 = make_float2(Pc[o0 + 1], Pc[o1 + 1]),
                                     v4 = make_float2(Pd[o0], Pd[o1]);
                        const float2 s = __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(v0, v1), v2), v3), v4);
                        auto ind = [&](float2 a) { return make_float2((float)(a.x > eps_p), (float)(a.y > eps_p)); };
                        const float2 n = __fadd2_rn(
                            __fadd2_rn(__fadd2_rn(__fadd2_rn(ind(v0), ind(v1)), ind(v2)), ind(v3)), ind(v4));
                        const float2 q = __fmul2_rn(s, make_float2(rcp_approx(n.x), rcp_approx(n.y)));
                        v = make_float2(__saturatef(q.x), __saturatef(q.y));
                        if (!EPS0) v = make_float2(n.x > 0.f ? v.x : 0.f, n.y > 0.f ? v.y : 0.f);
                        pmin = fminf(pmin, fminf(v.x, v.y));
                    } else {
                        v = make_float2(Pc[o0], Pc[o1]);
                    }
                    ph[k] = v.x;
                    ph[KT + k] = v.y;
                } else {
#pragma unroll
                    for (int pp = 0; pp < NP; pp++) {
                        const int o = (pp * KT + k) * ER_PW + t + 4;
                        float v;
                        if (p.maintain) {
                            // disk |d| <= 1 in the order (-1,0), (0,-1), (0,0), (0,1), (1,0)
                            const float v0 = Pu[o], v1 = Pc[o - 1], v2 = Pc[o], v3 = Pc[o + 1], v4 = Pd[o];
                            const float s = (((v0 + v1) + v2) + v3) + v4;
                            const float n = (float)(v0 > eps_p) + (float)(v1 > eps_p) + (float)(v2 > eps_p) +
                                            (float)(v3 > eps_p) + (float)(v4 > eps_p);
                            v = __saturatef(s * rcp_approx(n));
                            if (!EPS0) v = n > 0.f ? v : 0.f;
                            pmin = fminf(pmin, v);
                        } else {
                            v = Pc[o];
                        }
                        ph[pp * KT + k] = v;
                    }
                }
            }
            // growth, two kernels at a time on packed FP32 pairs (the same
            // operations, lane by lane; sums and minima in kernel order)
            auto gene = [&](int pl, int k, const float* bank) {
                return pl >= 0 ? ph[(pl >= 0 ? pl : 0) * KT + k] : bank[k];
            };
            auto add_growth = [&](int k, float G) {
                const int d = TOPO ? paper_dst(k) : p.kt.dst[k];
#pragma unroll
                for (int c = 0; c < CT; c++)
                    if (c == d) acc[c] += G;
            };
#pragma unroll
            for (int k = 0; k < KT; k += 2) {
                if (k + 1 < KT) {
                    const float2 u = make_float2(Ur[k * ER_CH + t], Ur[(k + 1) * ER_CH + t]);
                    const float2 m = make_float2(gene(PMU, k, p.kt.mu), gene(PMU, k + 1, p.kt.mu));
                    const float2 sg = make_float2(gene(PSG, k, p.kt.sigma), gene(PSG, k + 1, p.kt.sigma));
                    const float2 hh = make_float2(gene(PH, k, p.kt.h), gene(PH, k + 1, p.kt.h));
                    const float2 z = __fmul2_rn(__fadd2_rn(u, make_float2(-m.x, -m.y)),
                                                make_float2(rcp_approx(sg.x), rcp_approx(sg.y)));
                    const float2 e = __fmul2_rn(make_float2(-C_HALF_LOG2E, -C_HALF_LOG2E), __fmul2_rn(z, z));
                    const float2 gk = make_float2(sg.x > 0.f ? ex2_approx(e.x) : 0.f, sg.y > 0.f ? ex2_approx(e.y) : 0.f);
                    const float2 tk = p.alpha_on ? u : __fmul2_rn(hh, gk);
                    tmin = fminf(fminf(tmin, tk.x), tk.y);
                    tsum += tk.x;
                    tsum += tk.y;
                    const float2 G = p.growth_form == 0
                                         ? __ffma2_rn(__fmul2_rn(make_float2(2.f, 2.f), gk), hh, make_float2(-hh.x, -hh.y))
                                         : __fmul2_rn(hh, gk);
                    add_growth(k, G.x);
                    add_growth(k + 1, G.y);
                } else {
                    const float u = Ur[k * ER_CH + t];
                    const float m = gene(PMU, k, p.kt.mu), sg = gene(PSG, k, p.kt.sigma), hh = gene(PH, k, p.kt.h);
                    const float z = (u - m) * rcp_approx(sg);
                    const float gk = sg > 0.f ? ex2_approx(-C_HALF_LOG2E * (z * z)) : 0.f;
                    const float tk = p.alpha_on ? u : hh * gk;
                    tmin = fminf(tmin, tk);
                    tsum += tk;
                    add_growth(k, p.growth_form == 0 ? fmaf(2.f * gk, hh, -hh) : hh * gk);
                }
            }
            const bool alpha = !p.maintain || ((NPK == 0 || pmin > eps_p) && tmin > eps_u);
            const unsigned gi = (unsigned)y * (unsigned)W + (unsigned)x;
#pragma unroll
            for (int c = 0; c < CT; c++) {
                const float an = __saturatef(Ar[c * ER_CH + t] + p.dt * (alpha ? acc[c] : p.acc0[c]));
                A_out[(unsigned)c * N + gi] = an;
                // the column's weights (sin, cos of x) are applied to the
                // column's mass once, at the end of the band
                st[c * 5 + 0] += an;
                st[c * 5 + 1] += an * sy;
                st[c * 5 + 2] += an * cy;
            }
            if (p.alpha_out) p.alpha_out[gi] = alpha ? 1 : 0;
            if (p.empty_out) p.empty_out[gi] = tsum > eps_u ? 0 : 1;
            if (P_out) {
                // kept genes, or zeros (one branch per site instead of a select per plane)
                float* Po = P_out + gi;
                if (!p.maintain || alpha) {
#pragma unroll
                    for (int pk = 0; pk < NPK; pk++) Po[(unsigned)pk * N] = ph[pk];
                } else {
#pragma unroll
                    for (int pk = 0; pk < NPK; pk++) Po[(unsigned)pk * N] = 0.f;
                }
            }
            // this warp is done with gene rows l = i, i + 1 and U/A row i
            __syncwarp();
            if (lane == 0) {
                if (NPK > 0) {
                    mbar_arrive(&empty_p[i % NPD]);
                    mbar_arrive(&empty_p[(i + 1) % NPD]);
                }
                mbar_arrive(&empty_u[i % NUD]);
            }
        }
        // sum A sin(2 pi x / W), sum A cos(2 pi x / W) of this column's rows
#pragma unroll
        for (int c = 0; c < CT; c++) {
            st[c * 5 + 3] = st[c * 5 + 0] * sx;
            st[c * 5 + 4] = st[c * 5 + 0] * cx;
        }
    }
}

// After a failed band: the producer gives the copies it issued last a
// bounded chance to land before the block's shared memory is released.
template <int NPD = ER_NP, int NUD = ER_NU>
__device__ __forceinline__ void er_drain(int last_gene, int last_pot, uint64_t* full_p, uint64_t* full_u)
{
    if ((threadIdx.x >> 5) == ER_CONSUMERS && (threadIdx.x & 31) == 0) {
        for (int l = last_gene - (NPD - 1) < 0 ? 0 : last_gene - (NPD - 1); l <= last_gene; l++)
            mbar_wait_bounded(&full_p[l % NPD], (l / NPD) & 1);
        for (int i = last_pot - (NUD - 1) < 0 ? 0 : last_pot - (NUD - 1); i <= last_pot; i++)
            mbar_wait_bounded(&full_u[i % NUD], (i / NUD) & 1);
    }
}

// Shared-memory carve-up of the streaming epilogue.
template <int KT, int CT, int LOC, int NPD = ER_NP, int NUD = ER_NU>
struct ErSmem {
    float *Pring, *Hring, *Uring, *Aring;
    uint64_t *full_p, *empty_p, *full_u, *empty_u;
    __device__ explicit ErSmem(unsigned char* smem)
    {
        using L = ErLayout<KT, CT, LOC, NPD, NUD>;
        Pring = reinterpret_cast<float*>(smem);
        Hring = Pring + L::p_floats;                   // [slot][left, right][NPK][4]
        Uring = Hring + L::h_floats;
        Aring = Uring + L::u_floats;
        full_p = reinterpret_cast<uint64_t*>(Aring + L::a_floats);
        empty_p = full_p + NPD;
        full_u = empty_p + NPD;
        empty_u = full_u + NUD;
    }
    // (re-)initialise every barrier; `reuse`: they served an earlier item and
    // are invalidated first (no thread waits on them and no copy is pending)
    __device__ void init(bool reuse = false) const
    {
        if (reuse) {
            for (int b = 0; b < NPD; b++) {
                mbar_inval(&full_p[b]);
                mbar_inval(&empty_p[b]);
            }
            for (int b = 0; b < NUD; b++) {
                mbar_inval(&full_u[b]);
                mbar_inval(&empty_u[b]);
            }
        }
        for (int b = 0; b < NPD; b++) {
            mbar_init(&full_p[b], 1);
            mbar_init(&empty_p[b], ER_CONSUMERS);
        }
        for (int b = 0; b < NUD; b++) {
            mbar_init(&full_u[b], 1);
            mbar_init(&empty_u[b], ER_WPG);
        }
        mbar_fence_init();
    }
};

template <int KT, int CT, int LOC, int TOPO, int EPS0>
__global__ void __launch_bounds__(ER_THREADS, 1)
    k_epilogue_rows(EpiParams p, const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_u,
                    const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_h, int n_chunks, int n_bands,
                    int* status)
{
    pdl_enter();
    static_assert(TOPO == 0 || (KT == 15 && CT == 3), "paper topology has 15 kernels, 3 channels");
    static_assert(CT * 5 <= ER_THREADS / 32, "one warp per statistics sum");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    const ErSmem<KT, CT, LOC> sm(smem);
    __shared__ float red[ER_CONSUMERS][CT * 5];
    __shared__ int blk_failed;

    const int H = p.H;
    const int chunk = blockIdx.x % n_chunks, band = blockIdx.x / n_chunks;
    const int x0 = chunk * ER_CH;
    const int r0 = (int)((long long)band * H / n_bands);
    const int r1 = (int)((long long)(band + 1) * H / n_bands);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        sm.init();
        blk_failed = 0;
    }
    __syncthreads();

    float st[CT * 5];
#pragma unroll
    for (int v = 0; v < CT * 5; v++) st[v] = 0.f;
    int last_gene = -1, last_pot = -1;      // producer: last rows whose copies were issued
    er_band<KT, CT, LOC, TOPO, EPS0>(p, &tm_p, &tm_u, &tm_a, &tm_h, p.A_out, p.P_out, x0, r0, r1, sm.Pring,
                                     sm.Hring, sm.Uring, sm.Aring, sm.full_p, sm.empty_p, sm.full_u, sm.empty_u,
                                     st, &blk_failed, last_gene, last_pot, status);

    // Every warp reaches this point (all waits are bounded).
    __syncthreads();
    if (blk_failed) {
        er_drain<>(last_gene, last_pot, sm.full_p, sm.full_u);
        return;
    }
    if (p.partials) {
        if (warp < ER_CONSUMERS) {
#pragma unroll
            for (int v = 0; v < CT * 5; v++) {
                float s = st[v];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
                if (lane == 0) red[warp][v] = s;
            }
        }
        __syncthreads();
        // The producer warp writes the block's record: it has no global
        // stores of its own in flight, so its fence waits only for the record
        // (the consumers' streaming stores drain meanwhile, unfenced).
        const bool writer = warp == ER_CONSUMERS && lane < CT * 5;
        if (writer) {
            float2 s = make_float2(0.f, 0.f);
            for (int w = 0; w < ER_CONSUMERS; w++) s = ff_add(s, make_float2(red[w][lane], 0.f));
            p.partials[(size_t)blockIdx.x * CT * 5 + lane] = s;
        }
        if (p.stats_out) {
            // The last block to finish reduces every block's record in block
            // order (deterministic) and re-arms the ticket for the next launch.
            // Each record writer fences, the block meets, then one writer
            // takes the ticket.
            __shared__ unsigned int ticket;
            if (writer) __threadfence();
            __syncthreads();
            if (warp == ER_CONSUMERS && lane == 0) ticket = atomicAdd(p.ticket, 1u);
            __syncthreads();
            if (ticket == gridDim.x - 1) {
                __threadfence();
                __shared__ float2 tot[CT * 5];
                // one warp per sum: lanes stride over the block records, then a
                // fixed shuffle tree (deterministic; compensated FP32 pairs)
                if (warp < CT * 5) {
                    float2 s = make_float2(0.f, 0.f);
                    for (unsigned b = lane; b < gridDim.x; b += 32 * 4) {
                        // four records in flight per lane, added in block order
                        float2 r[4];
#pragma unroll
                        for (int u = 0; u < 4; u++)
                            r[u] = b + 32 * u < gridDim.x ? __ldcg(&p.partials[(size_t)(b + 32 * u) * CT * 5 + warp])
                                                          : make_float2(0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < 4; u++) s = ff_add(s, r[u]);
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) s = ff_add(s, ff_shfl_down(s, off));
                    if (lane == 0) tot[warp] = s;
                }
                __syncthreads();
                if (tid < 2 * CT) stats_centre(tot, tid >> 1, tid & 1, H, p.W, p.stats_out);
                if (tid == 0) *p.ticket = 0u;
            }
        }
    }
}

// Many worlds of one shape (a batched group) in one persistent launch: work
// items (world, chunk, band) are taken from a device work queue (an atomic
// counter) by every block until none is left; each item runs the streaming
// pipeline above with that world's tensor maps, read from global memory.
// Between items the block waits at a barrier (every copy of the last item
// has been consumed, every release has arrived) and re-initialises its
// barriers.  No statistics, alpha or empty outputs.
// Ring depths of the queued kernel: its one-kernel rows are small (about
// 4 KB of genes, potential and phenospace per row), so it keeps many more of
// them in flight than the 15-kernel pipeline.
constexpr int EQ_NP = 16, EQ_NU = 12;

template <int LOC, int EPS0>
__global__ void __launch_bounds__(ER_THREADS, 1)
    k_epilogue_queue(EpiParams p, const QueueWorld* __restrict__ worlds, int n_items, int n_chunks, int n_bands,
                     int* counter, int* status)
{
    pdl_enter();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127);
    const ErSmem<1, 1, LOC, EQ_NP, EQ_NU> sm(smem);
    __shared__ int blk_failed, item;
    const int H = p.H, tid = threadIdx.x;
    float st[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (tid == 0) blk_failed = 0;
    int last_gene = -1, last_pot = -1;
    for (int n = 0;; n++) {
        __syncthreads();                       // the previous item is done everywhere
        if (tid == 0) {
            item = atomicAdd(counter, 1);
            sm.init(n > 0);
        }
        __syncthreads();
        const int it = item;
        if (it >= n_items || blk_failed) break;
        const int w = it / (n_chunks * n_bands);
        const int rest = it - w * (n_chunks * n_bands);
        const int band = rest / n_chunks, chunk = rest - band * n_chunks;
        const QueueWorld* qw = worlds + w;
        const int r0 = (int)((long long)band * H / n_bands);
        const int r1 = (int)((long long)(band + 1) * H / n_bands);
        last_gene = last_pot = -1;
        er_band<1, 1, LOC, 0, EPS0, EQ_NP, EQ_NU>(p, &qw->tm_p, &qw->tm_u, &qw->tm_a, &qw->tm_h, qw->A_out, qw->P_out,
                                    chunk * ER_CH, r0, r1, sm.Pring, sm.Hring, sm.Uring, sm.Aring, sm.full_p,
                                    sm.empty_p, sm.full_u, sm.empty_u, st, &blk_failed, last_gene, last_pot,
                                    status);
    }
    __syncthreads();
    if (blk_failed) er_drain<EQ_NP, EQ_NU>(last_gene, last_pot, sm.full_p, sm.full_u);
}

// ------------------------------------------------------------ tensor maps
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

namespace {

struct MapKey {
    const void* base;
    int W, H, planes, box_x, box_planes;
    bool operator==(const MapKey& o) const
    {
        return base == o.base && W == o.W && H == o.H && planes == o.planes && box_x == o.box_x &&
               box_planes == o.box_planes;
    }
};

// A plane stack [planes][H][W] of floats viewed as (W/2 8-byte elements, H
// rows, planes); boxes of box_x elements x 1 row x box_planes.  Encoded maps
// are cached by argument (most recent first).
bool plane_map(CUtensorMap* out, const float* base, int W, int H, int planes, int box_x, int box_planes)
{
    static std::mutex mu;
    static std::vector<std::pair<MapKey, CUtensorMap>> cache;
    const MapKey key{base, W, H, planes, box_x, box_planes};
    std::lock_guard<std::mutex> lock(mu);
    for (size_t i = 0; i < cache.size(); i++)
        if (cache[i].first == key) {
            *out = cache[i].second;
            return true;
        }
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    CUtensorMap m;
    const cuuint64_t dims[3] = {(cuuint64_t)W / 2, (cuuint64_t)H, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 4, (cuuint64_t)W * H * 4};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, 1, (cuuint32_t)box_planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    cache.insert(cache.begin(), {key, m});
    if (cache.size() > 32) cache.pop_back();
    *out = m;
    return true;
}

}  // namespace

// Shared-memory limit and resident CTAs per SM of one instantiation, found
// once per device.
template <auto Kern>
static cudaError_t rows_occupancy(size_t bytes, int* per_sm)
{
    static std::atomic<int> occ[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    int v = occ[dev].load(std::memory_order_relaxed);
    if (v > 0) {
        *per_sm = v;
        return cudaSuccess;
    }
    cudaError_t e = smem_limit<Kern>(bytes);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, Kern, ER_THREADS, bytes);
    if (e != cudaSuccess) return e;
    occ[dev].store(v);
    *per_sm = v;
    return cudaSuccess;
}

template <int KT, int CT, int LOC, int TOPO = 0>
static cudaError_t launch_rows(const EpiParams& p, int num_sms, int* status, cudaStream_t s, int* n_blocks)
{
    using L = ErLayout<KT, CT, LOC>;
    auto kern = p.eps_p == 0.f ? k_epilogue_rows<KT, CT, LOC, TOPO, 1> : k_epilogue_rows<KT, CT, LOC, TOPO, 0>;
    int per_sm = 1;
    cudaError_t e = p.eps_p == 0.f ? rows_occupancy<k_epilogue_rows<KT, CT, LOC, TOPO, 1>>(L::bytes, &per_sm)
                                   : rows_occupancy<k_epilogue_rows<KT, CT, LOC, TOPO, 0>>(L::bytes, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int n_chunks = p.W / ER_CH;
    int n_bands = (num_sms * per_sm) / n_chunks;
    if (n_bands < 1) n_bands = 1;
    if (n_bands > p.H) n_bands = p.H;
    if (n_blocks) *n_blocks = n_chunks * n_bands;
    CUtensorMap tp, tu, ta, th;
    memset(&tp, 0, sizeof(tp));
    memset(&th, 0, sizeof(th));
    if (L::NPK > 0 && (!plane_map(&tp, p.P, p.W, p.H, L::NPK, ER_PW / 2, L::NPK) ||
                       !plane_map(&th, p.P, p.W, p.H, L::NPK, 2, L::NPK)))
        return cudaErrorInvalidValue;
    if (!plane_map(&tu, p.U, p.W, p.H, KT, ER_CH / 2, KT) || !plane_map(&ta, p.A, p.W, p.H, CT, ER_CH / 2, CT))
        return cudaErrorInvalidValue;
    launch_pdl(kern, n_chunks * n_bands, ER_THREADS, L::bytes, s, p, tp, tu, ta, th, n_chunks, n_bands, status);
    return cudaGetLastError();
}

// A plane stack as plane_map describes it, encoded without the cache (the
// queued epilogue stores its maps in device memory).
static bool plane_map_direct(CUtensorMap* out, const float* base, int W, int H, int planes, int box_x,
                             int box_planes)
{
    auto fn = tensor_map_encoder();
    if (!fn || ((uintptr_t)base & 15) != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)W / 2, (cuuint64_t)H, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)W * 4, (cuuint64_t)W * H * 4};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, 1, (cuuint32_t)box_planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(out, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int queue_loc(const EpiParams& p)
{
    return (p.p_mu >= 0 ? 1 : 0) | (p.p_sigma >= 0 ? 2 : 0) | (p.p_h >= 0 ? 4 : 0);
}

bool epilogue_queue_supported(const EpiParams& p)
{
    const int loc = queue_loc(p);
    return p.kt.K == 1 && p.kt.C == 1 && p.n_rings == 0 && (loc == 3 || loc == 0) && p.W % ER_CH == 0 &&
           (!p.maintain || p.r_diff == 1) && (long long)p.H * p.W * 2 < (1LL << 31) && !p.partials &&
           !p.alpha_out && !p.empty_out;
}

bool epilogue_queue_world(QueueWorld* q, const EpiParams& p, const float* A, const float* P, const float* U,
                          float* A_out, float* P_out)
{
    memset(q, 0, sizeof(*q));
    const int npk = queue_loc(p) == 3 ? 2 : 0;
    if (npk > 0 && (!plane_map_direct(&q->tm_p, P, p.W, p.H, npk, ER_PW / 2, npk) ||
                    !plane_map_direct(&q->tm_h, P, p.W, p.H, npk, 2, npk)))
        return false;
    if (!plane_map_direct(&q->tm_u, U, p.W, p.H, 1, ER_CH / 2, 1) ||
        !plane_map_direct(&q->tm_a, A, p.W, p.H, 1, ER_CH / 2, 1))
        return false;
    q->A_out = A_out;
    q->P_out = P_out;
    return true;
}

template <int LOC, int EPS0>
static cudaError_t launch_queue(const EpiParams& p, const QueueWorld* worlds, int n_worlds, int n_bands,
                                int ctas_per_sm, int* counter, int* status, cudaStream_t s)
{
    using L = ErLayout<1, 1, LOC, EQ_NP, EQ_NU>;
    int per_sm = 1;
    cudaError_t e = rows_occupancy<k_epilogue_queue<LOC, EPS0>>(L::bytes, &per_sm);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    static int n_sms = 0;
    if (n_sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n_sms = 148;
    }
    const int n_chunks = p.W / ER_CH;
    const int n_items = n_worlds * n_chunks * n_bands;
    const int grid = std::min(n_items, n_sms * per_sm);
    e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    launch_pdl(k_epilogue_queue<LOC, EPS0>, grid, ER_THREADS, L::bytes, s, p, worlds, n_items, n_chunks, n_bands, counter,
                                                                    status);
    return cudaGetLastError();
}

cudaError_t launch_epilogue_queue(const EpiParams& p, const QueueWorld* worlds, int n_worlds, int n_bands,
                                  int ctas_per_sm, int* counter, int* status, cudaStream_t s)
{
    if (!epilogue_queue_supported(p) || n_worlds < 1 || n_bands < 1 || n_bands > p.H) return cudaErrorInvalidValue;
    const bool e0 = p.eps_p == 0.f;
    if (queue_loc(p) == 3)
        return e0 ? launch_queue<3, 1>(p, worlds, n_worlds, n_bands, ctas_per_sm, counter, status, s)
                  : launch_queue<3, 0>(p, worlds, n_worlds, n_bands, ctas_per_sm, counter, status, s);
    return e0 ? launch_queue<0, 1>(p, worlds, n_worlds, n_bands, ctas_per_sm, counter, status, s)
              : launch_queue<0, 0>(p, worlds, n_worlds, n_bands, ctas_per_sm, counter, status, s);
}

bool epilogue_rows_supported(const EpiParams& p)
{
    if (p.W % ER_CH != 0 || (p.maintain && p.r_diff != 1) || p.n_rings > 0) return false;
    // 32-bit site indexing of every plane
    const long long N = (long long)p.H * p.W;
    if (N * (p.n_p * p.kt.K > p.kt.K ? p.n_p * p.kt.K : p.kt.K) >= (1LL << 31) || N * p.kt.C >= (1LL << 31))
        return false;
    const int loc = (p.p_mu >= 0 ? 1 : 0) | (p.p_sigma >= 0 ? 2 : 0) | (p.p_h >= 0 ? 4 : 0);
    const int K = p.kt.K, C = p.kt.C;
    return (K == 15 && C == 3 && (loc == 3 || loc == 0)) || (K == 1 && C == 1 && (loc == 3 || loc == 0));
}

cudaError_t launch_epilogue_rows(const EpiParams& p, int num_sms, int* status, cudaStream_t s, int* n_blocks)
{
    const int loc = (p.p_mu >= 0 ? 1 : 0) | (p.p_sigma >= 0 ? 2 : 0) | (p.p_h >= 0 ? 4 : 0);
    const int K = p.kt.K, C = p.kt.C;
    bool paper = K == 15 && C == 3;
    for (int k = 0; paper && k < K; k++) paper = p.kt.dst[k] == paper_dst(k);
    if (paper && loc == 3) return launch_rows<15, 3, 3, 1>(p, num_sms, status, s, n_blocks);
    if (paper && loc == 0) return launch_rows<15, 3, 0, 1>(p, num_sms, status, s, n_blocks);
    if (K == 15 && C == 3 && loc == 3) return launch_rows<15, 3, 3>(p, num_sms, status, s, n_blocks);
    if (K == 15 && C == 3 && loc == 0) return launch_rows<15, 3, 0>(p, num_sms, status, s, n_blocks);
    if (K == 1 && C == 1 && loc == 3) return launch_rows<1, 1, 3>(p, num_sms, status, s, n_blocks);
    if (K == 1 && C == 1 && loc == 0) return launch_rows<1, 1, 0>(p, num_sms, status, s, n_blocks);
    return cudaErrorInvalidValue;
}

}  // namespace lenia
