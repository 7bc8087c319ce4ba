/*
 * FP64 CPU oracle for one step of Lenia with localized genes.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant with the CUDA library: every formula is
 * written out here again from the paper (arXiv 2304.05639) and from the
 * original Lenia definitions that paper builds on.
 *
 * Plain, slow, obviously correct: direct periodic (toroidal) convolution,
 * loops in the order the definitions are written, double precision
 * throughout, OpenMP only across independent output rows (each output is
 * computed by one thread in a fixed order, so results do not depend on the
 * thread count).
 *
 * Step order follows Algorithm 2 (intrinsic evolution loop): diffuse the
 * genospace, convolve the phenospace, compute alpha, mask the genospace,
 * growth mapping and clipped update.  oracle_evolve_step adds the other lines
 * of Algorithm 2: environment (walls), E_pen, mutation and penalisation.
 *
 * Readings where the paper is silent or ambiguous (each one is also listed in
 * the design notes):
 *  R1 growth: signed form h*(2*exp(-(u-m)^2/(2 s^2)) - 1) (form 0) or the
 *     paper's h*exp(...) (form 1, Section 2.4).
 *  R2 dt multiplies the growth sum; the paper's update is dt = 1.
 *  R3 kernel: rho = |d|_2 / R, zero for rho >= 1.  Shell form
 *     beta[floor(B rho)] * core(B rho mod 1), core(q) = exp(4 - 1/(q(1-q))),
 *     core(0) = 0.  Bump form sum_i b_i exp(-(rho - r_i)^2 / (2 w_i^2)).
 *  R5 alpha tests h_k*g_k > eps_u (g in [0,1]), AND over k, and every gene
 *     plane > eps_p (Delta_all); alpha_on = 1 tests U_k > eps_u instead.
 *  R6 eps_u and eps_p are separate thresholds, strict '>'.
 *  R7 K_diff is the disk |d|_2 <= r_diff.
 *  R8 diffusion with no neighbour above eps_p gives 0.
 *  R9 g = 0 where the gene sigma is 0; the update uses the masked genes, so
 *     where alpha = 0 the growth is h*(2*0 - 1) = -h (form 0) or 0 (form 1).
 *  R14 walls zero A and P at the wall sites before the step (the environment
 *     line comes first in Algorithm 2); the step's own output is not masked.
 *  R15 K_oxy is the disk |d|_2 <= r_oxy divided by its point count (like
 *     K_diff, Section 2.3); Delta_sum(U) sums the per-kernel alpha tests of R5.
 *  R16 "(x,y) in E_pen" reads E_pen > eps_pen, a parameter (default 0.5: at
 *     the straight edge of a large body E_pen is 1/2).
 *  R17 the mutation square is x in [x0 - s, x0 + s), y in [y0 - s, y0 + s),
 *     periodic; delta and the centre are inputs (drawn by the caller).
 *  R18 penalisation: p is the mu or the sigma plane, delta > 0 for mu and
 *     delta < 0 for sigma (Figure 3's arrows); no clip after either operator
 *     (the next step's diffusion clips to [0, 1]).
 *  R19 rings (Section 2.4): ring r of a radius-R kernel in n rings holds the
 *     offsets with r <= n |d|_2 / R < r + 1 and |d|_2 < R (binary masks, so
 *     K_r * 1 is the ring's point count); every kernel shares one radius.
 *  R20 the ring weight evaluates the kernel function at r / n (the ring's
 *     inner radius), as written; k(x; r, w, b) = 0 where w <= 0.
 *  R21 the weighted sum uses the diffused, unmasked kernel genes (it comes
 *     between diffusion and alpha in Algorithm 2); U = 0 where the
 *     normalising sum is <= 0.
 *  R22 gene planes: m, s, h (the localized ones), then r1, w1, b1, r2, w2, b2;
 *     all of them take part in diffusion, Delta_all(P) and masking.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LOC_MU 1
#define LOC_SIGMA 2
#define LOC_H 4
#define LOC_KERNEL 8      /* ring-wise kernel genes r1, w1, b1, r2, w2, b2 (Section 2.4) */
#define MAX_PK 576        /* 9 gene types x 64 kernels */

/* Lenia kernel core (original Lenia, cited in Section 1.2): a smooth bump on
 * (0,1) with value 1 at q = 1/2 and limit 0 at both ends. */
static double kernel_core(double q)
{
    if (q <= 0.0 || q >= 1.0) return 0.0;
    return exp(4.0 - 1.0 / (q * (1.0 - q)));
}

/* Unnormalised kernel value at pixel offset (dy, dx). */
static double kernel_value(int R, int form, int n_shells, const double* beta,
                           const double* bump, int dy, int dx)
{
    double rho = sqrt((double)dy * dy + (double)dx * dx) / (double)R;
    if (rho >= 1.0) return 0.0;
    if (form == 0) {
        double br = n_shells * rho;
        int i = (int)floor(br);
        return beta[i] * kernel_core(br - i);
    }
    /* Section 2.4: kernel function k(x; r, w, b) = b exp(-(x - r)^2 / 2 w^2),
     * two bumps (r1, w1, b1, r2, w2, b2). */
    double v = 0.0;
    for (int i = 0; i < 2; i++) {
        double r = bump[3 * i], w = bump[3 * i + 1], b = bump[3 * i + 2];
        v += b * exp(-(rho - r) * (rho - r) / (2.0 * w * w));
    }
    return v;
}

/* Normalised kernel K~ = K / (K * 1), Algorithm 1 pre-calculation and the
 * note after Algorithm 2 (K * 1 = sum over the kernel).  out has (2R+1)^2
 * entries, row-major over dy = -R..R, dx = -R..R.  Returns 0, or -1 if the
 * kernel sums to zero. */
int oracle_kernel(int R, int form, int n_shells, const double* beta,
                  const double* bump, double* out)
{
    int n = 2 * R + 1;
    double sum = 0.0;
    for (int dy = -R; dy <= R; dy++)
        for (int dx = -R; dx <= R; dx++) {
            double v = kernel_value(R, form, n_shells, beta, bump, dy, dx);
            out[(dy + R) * n + (dx + R)] = v;
            sum += v;
        }
    if (!(sum > 0.0)) return -1;
    for (int i = 0; i < n * n; i++) out[i] /= sum;
    return 0;
}

static inline int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* Periodic convolution U = K~ * A on an H x W torus (Section 2.1, toroidal
 * world; Algorithm 1 "convolve the phenotype with kernels"):
 *   U(y, x) = sum_{dy,dx} K~(dy, dx) A(y - dy, x - dx).
 * Zero kernel taps are skipped (adding an exact zero changes nothing).
 * With extended != 0 the sum is accumulated in long double, to measure the
 * oracle's own rounding error. */
void oracle_potential(int H, int W, const double* A, int R, const double* K,
                      double* U, int extended)
{
    int n = 2 * R + 1;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            long double sl = 0.0L;
            for (int dy = -R; dy <= R; dy++) {
                const double* krow = K + (dy + R) * n;
                const double* arow = A + (size_t)wrap(y - dy, H) * W;
                for (int dx = -R; dx <= R; dx++) {
                    double k = krow[dx + R];
                    if (k == 0.0) continue;
                    double a = arow[wrap(x - dx, W)];
                    if (extended) sl += (long double)k * (long double)a;
                    else s += k * a;
                }
            }
            U[(size_t)y * W + x] = extended ? (double)sl : s;
        }
    }
}

/* Genospace diffusion of one gene plane (Section 2.3):
 *   P -> clip( (P * K_diff) / (Delta_same(P) * K_diff), 0, 1 )
 * K_diff the disk |d| <= r_diff (R7), Delta_same(P) = [P > eps_p] (Section
 * 2.2), 0 where no disk site is above eps_p (R8). */
void oracle_diffuse(int H, int W, const double* P, int r_diff, double eps_p, double* out)
{
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            int cnt = 0;
            for (int dy = -r_diff; dy <= r_diff; dy++)
                for (int dx = -r_diff; dx <= r_diff; dx++) {
                    if (dy * dy + dx * dx > r_diff * r_diff) continue;
                    double v = P[(size_t)wrap(y + dy, H) * W + wrap(x + dx, W)];
                    s += v;
                    if (v > eps_p) cnt++;
                }
            double r = 0.0;
            if (cnt > 0) {
                r = s / (double)cnt;
                if (r < 0.0) r = 0.0;
                if (r > 1.0) r = 1.0;
            }
            out[(size_t)y * W + x] = r;
        }
    }
}

/* Gaussian bump of the growth mapping, g in [0, 1]; 0 where s <= 0 (R9). */
static double growth_bump(double u, double m, double s)
{
    if (!(s > 0.0)) return 0.0;
    double z = (u - m) / s;
    return exp(-0.5 * z * z);
}

typedef struct {
    int H, W, C, K;
    double dt;
    int growth_form, localized, maintain, r_diff, alpha_on;
    double eps_u, eps_p;
    int n_rings;          /* > 0 with LOC_KERNEL: ring decomposition, Section 2.4 */
} oracle_cfg;

/* Gene planes in P, in this order: the localized growth genes m, s, h, then
 * (LOC_KERNEL) the six kernel genes r1, w1, b1, r2, w2, b2 of Section 2.1. */
typedef struct {
    int n_p, p_mu, p_sigma, p_h, p_kern;
} plane_map;

static plane_map planes_of(int loc)
{
    plane_map m;
    m.n_p = ((loc & LOC_MU) != 0) + ((loc & LOC_SIGMA) != 0) + ((loc & LOC_H) != 0);
    m.p_mu = (loc & LOC_MU) ? 0 : -1;
    m.p_sigma = (loc & LOC_SIGMA) ? ((loc & LOC_MU) ? 1 : 0) : -1;
    m.p_h = (loc & LOC_H) ? m.n_p - 1 : -1;
    m.p_kern = -1;
    if (loc & LOC_KERNEL) {
        m.p_kern = m.n_p;
        m.n_p += 6;
    }
    return m;
}

/* Ring of offset (dy, dx) for a radius-R kernel cut into n rings
 * (Section 2.4): the ring index r with r <= n |d|_2 / R < r + 1, for
 * |d|_2 < R; -1 outside.  Decided in integers: r = max{m : m^2 R^2 <= n^2 |d|^2}. */
static int ring_of(int dy, int dx, int R, int n)
{
    const long long q = (long long)dy * dy + (long long)dx * dx;
    if (q >= (long long)R * R) return -1;
    int m = (int)floor((double)n * sqrt((double)q) / (double)R);
    while ((long long)(m + 1) * (m + 1) * R * R <= (long long)n * n * q) m++;
    while (m > 0 && (long long)m * m * R * R > (long long)n * n * q) m--;
    return m;
}

/* Pixel count of every ring, K_r * 1 = sum over the ring (Section 2.4). */
void oracle_ring_counts(int R, int n, double* cnt)
{
    for (int r = 0; r < n; r++) cnt[r] = 0.0;
    for (int dy = -R; dy <= R; dy++)
        for (int dx = -R; dx <= R; dx++) {
            int r = ring_of(dy, dx, R, n);
            if (r >= 0) cnt[r] += 1.0;
        }
}

/* Ring potentials K_r * A of one plane for every ring r (Section 2.4,
 * "the rings are convolved with the phenospace"): V[r][y][x] =
 * sum_{d in ring r} A(y - dy, x - dx), periodic.  One pass over the disk per
 * site, each tap added to its ring's sum. */
void oracle_ring_potentials(int H, int W, const double* A, int R, int n, double* V)
{
    const size_t N = (size_t)H * W;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++) {
        double acc[256];
        for (int x = 0; x < W; x++) {
            for (int r = 0; r < n; r++) acc[r] = 0.0;
            for (int dy = -R; dy <= R; dy++) {
                const double* arow = A + (size_t)wrap(y - dy, H) * W;
                for (int dx = -R; dx <= R; dx++) {
                    int r = ring_of(dy, dx, R, n);
                    if (r < 0) continue;
                    acc[r] += arow[wrap(x - dx, W)];
                }
            }
            for (int r = 0; r < n; r++) V[(size_t)r * N + (size_t)y * W + x] = acc[r];
        }
    }
}

/* Kernel function of Section 2.4, k(x; r, w, b) = b exp(-(x - r)^2 / 2 w^2);
 * 0 where w <= 0 (as for a zero growth width, R9). */
static double kernel_fn(double x, double r, double w, double b)
{
    if (!(w > 0.0)) return 0.0;
    return b * exp(-(x - r) * (x - r) / (2.0 * w * w));
}

/* Potential of kernel k at one site from the ring potentials (Section 2.4):
 *   k_r = sum_i k(r / n_ring; r_i, w_i, b_i) with the site's kernel genes,
 *   U = sum_r k_r (K_r * A) / sum_r k_r (K_r * 1),  0 where the denominator is <= 0.
 * vr[r] holds (K_r * A_src(k)) at the site; ph the site's (diffused) genes. */
static double ring_recombine(int n, const double* vr, const double* cnt, const double* ph,
                             plane_map pm, int K, int k)
{
    const double r1 = ph[(pm.p_kern + 0) * K + k], w1 = ph[(pm.p_kern + 1) * K + k];
    const double b1 = ph[(pm.p_kern + 2) * K + k], r2 = ph[(pm.p_kern + 3) * K + k];
    const double w2 = ph[(pm.p_kern + 4) * K + k], b2 = ph[(pm.p_kern + 5) * K + k];
    double num = 0.0, den = 0.0;
    for (int r = 0; r < n; r++) {
        const double x = (double)r / (double)n;
        const double kr = kernel_fn(x, r1, w1, b1) + kernel_fn(x, r2, w2, b2);
        num += kr * vr[r];
        den += kr * cnt[r];
    }
    return den > 0.0 ? num / den : 0.0;
}

/* Growth, alpha mask, genospace masking and clipped update at one site.
 *  u[k]: potentials; ph[pk]: the site's genes after diffusion (pk = p*K + k);
 *  a_in[c]: the site's state.  Writes a_out[c], p_out[pk] and returns alpha. */
static int site_update(const oracle_cfg* cfg, plane_map pm, const int* dst, const double* h,
                       const double* mu, const double* sigma, const double* u, const double* ph,
                       const double* a_in, double* a_out, double* p_out, double* tsum_out)
{
    const int K = cfg->K;
    double g[64];
    double hk[64];
    int alpha = 1;
    double tsum = 0.0;
    for (int k = 0; k < K; k++) {
        double m = pm.p_mu >= 0 ? ph[pm.p_mu * K + k] : mu[k];
        double s = pm.p_sigma >= 0 ? ph[pm.p_sigma * K + k] : sigma[k];
        hk[k] = pm.p_h >= 0 ? ph[pm.p_h * K + k] : h[k];
        g[k] = growth_bump(u[k], m, s);
        /* the per-kernel test of alpha (R5): growth h g, or the potential */
        double t = cfg->alpha_on ? u[k] : hk[k] * g[k];
        tsum += t;
        if (cfg->maintain) {
            /* Section 2.2: alpha = Delta_all(U) AND Delta_all(P) (R5). */
            if (!(t > cfg->eps_u)) alpha = 0;
        }
    }
    if (tsum_out) *tsum_out = tsum;
    if (cfg->maintain)
        for (int pk = 0; pk < pm.n_p * K; pk++)
            if (!(ph[pk] > cfg->eps_p)) alpha = 0;

    /* Mask the genospace: P -> P (.) alpha. */
    if (p_out)
        for (int pk = 0; pk < pm.n_p * K; pk++)
            p_out[pk] = alpha ? ph[pk] : 0.0;

    /* Growth mapping and clipped update with the masked genes (R1, R2, R9):
     * A_i -> [A_i + dt sum_{k: dst(k) = i} G_k(U_k)]_0^1. */
    for (int c = 0; c < cfg->C; c++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) {
            if (dst[k] != c) continue;
            double gm = alpha ? g[k] : 0.0;
            double hm = (pm.p_h >= 0 && !alpha) ? 0.0 : hk[k];
            double G = cfg->growth_form == 0 ? hm * (2.0 * gm - 1.0) : hm * gm;
            acc += G;
        }
        double a = a_in[c] + cfg->dt * acc;
        if (a < 0.0) a = 0.0;
        if (a > 1.0) a = 1.0;
        a_out[c] = a;
    }
    return alpha;
}

/* The step after the convolution on the whole grid: diffusion (or plain
 * genes), then site_update everywhere.  Without rings U holds the potentials
 * U[K][H][W]; with rings (ring_cnt != NULL) it holds the ring potentials
 * V[C][n_rings][H][W] and each site's U_k is recombined from them with the
 * site's diffused kernel genes (Algorithm 2: the weighted sum comes after the
 * diffusion and before alpha).  U_out (nullable) receives U_k. */
static int update_grid(const oracle_cfg* cfg, const int* src, const int* dst, const double* h,
                       const double* mu, const double* sigma, const double* A, const double* P,
                       const double* U, const double* ring_cnt, double* A_out, double* P_out,
                       double* U_out, unsigned char* alpha_out, double* tsum_out)
{
    const int H = cfg->H, W = cfg->W, C = cfg->C, K = cfg->K, n = cfg->n_rings;
    const size_t N = (size_t)H * W;
    const plane_map pm = planes_of(cfg->localized);
    if (K > 64 || C > 64 || pm.n_p * K > MAX_PK) return -1;
    if (ring_cnt && (pm.p_kern < 0 || n < 1 || n > 256 || !src)) return -1;

    /* Algorithm 2: diffuse the genospace. */
    double* Ph = NULL;
    if (pm.n_p > 0) {
        Ph = (double*)malloc(sizeof(double) * (size_t)pm.n_p * K * N);
        for (int pk = 0; pk < pm.n_p * K; pk++) {
            if (cfg->maintain)
                oracle_diffuse(H, W, P + (size_t)pk * N, cfg->r_diff, cfg->eps_p, Ph + (size_t)pk * N);
            else
                memcpy(Ph + (size_t)pk * N, P + (size_t)pk * N, sizeof(double) * N);
        }
    }
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)N; i++) {
        double u[64], ph[MAX_PK], a_in[64], a_out[64], p_out[MAX_PK], vr[256];
        for (int pk = 0; pk < pm.n_p * K; pk++) ph[pk] = Ph[(size_t)pk * N + i];
        for (int k = 0; k < K; k++) {
            if (ring_cnt) {
                for (int r = 0; r < n; r++) vr[r] = U[((size_t)src[k] * n + r) * N + i];
                u[k] = ring_recombine(n, vr, ring_cnt, ph, pm, K, k);
            } else {
                u[k] = U[(size_t)k * N + i];
            }
        }
        for (int c = 0; c < C; c++) a_in[c] = A[(size_t)c * N + i];
        double ts = 0.0;
        int alpha = site_update(cfg, pm, dst, h, mu, sigma, u, ph, a_in, a_out, p_out, &ts);
        for (int c = 0; c < C; c++) A_out[(size_t)c * N + i] = a_out[c];
        if (P_out)
            for (int pk = 0; pk < pm.n_p * K; pk++) P_out[(size_t)pk * N + i] = p_out[pk];
        if (U_out)
            for (int k = 0; k < K; k++) U_out[(size_t)k * N + i] = u[k];
        if (alpha_out) alpha_out[i] = (unsigned char)alpha;
        if (tsum_out) tsum_out[i] = ts;
    }
    free(Ph);
    return 0;
}

/* The step after the convolution from given potentials U[K][H][W]. */
int oracle_update(const oracle_cfg* cfg, const int* dst, const double* h, const double* mu,
                  const double* sigma, const double* A, const double* P, const double* U,
                  double* A_out, double* P_out, unsigned char* alpha_out, double* tsum_out)
{
    if (cfg->localized & LOC_KERNEL) return -1;
    return update_grid(cfg, NULL, dst, h, mu, sigma, A, P, U, NULL, A_out, P_out, NULL, alpha_out,
                       tsum_out);
}

/* Ring potentials of every channel, V[C][n_rings][H][W]. */
static double* ring_potentials_all(const oracle_cfg* cfg, int R, const double* A)
{
    const size_t N = (size_t)cfg->H * cfg->W;
    const int n = cfg->n_rings;
    double* V = (double*)malloc(sizeof(double) * (size_t)cfg->C * n * N);
    for (int c = 0; c < cfg->C; c++)
        oracle_ring_potentials(cfg->H, cfg->W, A + (size_t)c * N, R, n, V + (size_t)c * n * N);
    return V;
}

/* The step after the ring convolutions, from given ring potentials
 * V[C][n_rings][H][W] of a radius-R kernel set (Section 2.4). */
int oracle_ring_update(const oracle_cfg* cfg, const int* src, const int* dst, int R, const double* h,
                       const double* mu, const double* sigma, const double* A, const double* P,
                       const double* V, double* A_out, double* P_out, double* U_out,
                       unsigned char* alpha_out, double* tsum_out)
{
    double cnt[256];
    if (cfg->n_rings < 1 || cfg->n_rings > 256) return -1;
    oracle_ring_counts(R, cfg->n_rings, cnt);
    return update_grid(cfg, src, dst, h, mu, sigma, A, P, V, cnt, A_out, P_out, U_out, alpha_out,
                       tsum_out);
}

/* One full step with ring-wise localized kernel genes (Algorithm 2 with the
 * ring decomposition of Section 2.4): every kernel has radius R; the kernel
 * of kernel k at a site is sum_r k_r K_r with the site's genes. */
int oracle_ring_step(const oracle_cfg* cfg, const int* src, const int* dst, int R, const double* h,
                     const double* mu, const double* sigma, const double* A, const double* P,
                     double* A_out, double* P_out, double* U_out, unsigned char* alpha_out)
{
    if (cfg->n_rings < 1 || cfg->n_rings > 256 || !(cfg->localized & LOC_KERNEL)) return -1;
    double* V = ring_potentials_all(cfg, R, A);
    int rc = oracle_ring_update(cfg, src, dst, R, h, mu, sigma, A, P, V, A_out, P_out, U_out, alpha_out, NULL);
    free(V);
    return rc;
}

/* One full step.
 *  A[C][H][W] in, A_out out; P[n_p][K][H][W] in (NULL when no gene maps),
 *  P_out out (NULL allowed); U_out[K][H][W], alpha_out[H][W] optional.
 *  Kernels: src[k], dst[k], R[k], h/mu/sigma[k] global genes; Kw holds the
 *  normalised kernels back to back, kernel k at offset kw_off[k].
 * Order of Algorithm 2: diffuse, convolve (the weighted ring sum collapses
 * to one normalised kernel when kernel genes are global), alpha, mask,
 * update.  Returns 0. */
int oracle_step(const oracle_cfg* cfg, const int* src, const int* dst, const int* R,
                const double* h, const double* mu, const double* sigma,
                const double* Kw, const long* kw_off,
                const double* A, const double* P, double* A_out, double* P_out,
                double* U_out, unsigned char* alpha_out)
{
    const int H = cfg->H, W = cfg->W, K = cfg->K;
    const size_t N = (size_t)H * W;
    if (cfg->localized & LOC_KERNEL) return -1;
    double* U = (double*)malloc(sizeof(double) * (size_t)K * N);
    for (int k = 0; k < K; k++)
        oracle_potential(H, W, A + (size_t)src[k] * N, R[k], Kw + kw_off[k], U + (size_t)k * N, 0);
    int rc = oracle_update(cfg, dst, h, mu, sigma, A, P, U, A_out, P_out, alpha_out, NULL);
    if (U_out) memcpy(U_out, U, sizeof(double) * (size_t)K * N);
    free(U);
    return rc;
}

/* The same step evaluated only at n listed sites (ys[i], xs[i]): the
 * potential by its direct sum, diffusion of each gene plane over the disk,
 * then site_update.  Outputs are [C][n], [n_p K][n], [K][n], the diffused
 * unmasked genes [n_p K][n] and alpha [n]. */
int oracle_step_sites(const oracle_cfg* cfg, const int* src, const int* dst, const int* R,
                      const double* h, const double* mu, const double* sigma,
                      const double* Kw, const long* kw_off, const float* A, const float* P,
                      long n, const int* ys, const int* xs, double* A_out, double* P_out,
                      double* U_out, double* Ph_out, unsigned char* alpha_out)
{
    const int H = cfg->H, W = cfg->W, C = cfg->C, K = cfg->K;
    const size_t N = (size_t)H * W;
    const plane_map pm = planes_of(cfg->localized);
    const int rd = cfg->r_diff;
    if (K > 64 || C > 64 || (cfg->localized & LOC_KERNEL)) return -1;
    #pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < n; i++) {
        const int y = ys[i], x = xs[i];
        double u[64], ph[MAX_PK], a_in[64], a_out[64], p_out[MAX_PK];
        for (int k = 0; k < K; k++) {
            const int r = R[k], nn = 2 * r + 1;
            const double* Kk = Kw + kw_off[k];
            const float* Ac = A + (size_t)src[k] * N;
            double s = 0.0;
            for (int dy = -r; dy <= r; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    double kv = Kk[(dy + r) * nn + (dx + r)];
                    if (kv == 0.0) continue;
                    s += kv * (double)Ac[(size_t)wrap(y - dy, H) * W + wrap(x - dx, W)];
                }
            u[k] = s;
        }
        for (int pk = 0; pk < pm.n_p * K; pk++) {
            const float* pl = P + (size_t)pk * N;
            if (!cfg->maintain) {
                ph[pk] = (double)pl[(size_t)y * W + x];
                continue;
            }
            double s = 0.0;
            int cnt = 0;
            for (int dy = -rd; dy <= rd; dy++)
                for (int dx = -rd; dx <= rd; dx++) {
                    if (dy * dy + dx * dx > rd * rd) continue;
                    double v = (double)pl[(size_t)wrap(y + dy, H) * W + wrap(x + dx, W)];
                    s += v;
                    if (v > cfg->eps_p) cnt++;
                }
            double r = 0.0;
            if (cnt > 0) {
                r = s / (double)cnt;
                if (r < 0.0) r = 0.0;
                if (r > 1.0) r = 1.0;
            }
            ph[pk] = r;
        }
        for (int c = 0; c < C; c++) a_in[c] = (double)A[(size_t)c * N + (size_t)y * W + x];
        int alpha = site_update(cfg, pm, dst, h, mu, sigma, u, ph, a_in, a_out, p_out, NULL);
        for (int c = 0; c < C; c++) A_out[(size_t)c * n + i] = a_out[c];
        if (P_out)
            for (int pk = 0; pk < pm.n_p * K; pk++) P_out[(size_t)pk * n + i] = p_out[pk];
        if (U_out)
            for (int k = 0; k < K; k++) U_out[(size_t)k * n + i] = u[k];
        if (Ph_out)
            for (int pk = 0; pk < pm.n_p * K; pk++) Ph_out[(size_t)pk * n + i] = ph[pk];
        if (alpha_out) alpha_out[i] = (unsigned char)alpha;
    }
    return 0;
}

/* Normalised disk average over |d|_2 <= r (periodic):
 * out(x) = sum_{|d| <= r} in(x + d) / #{|d| <= r}. */
void oracle_disk_mean(int H, int W, const double* in, int r, double* out)
{
    int n = 0;
    for (int dy = -r; dy <= r; dy++)
        for (int dx = -r; dx <= r; dx++)
            if (dy * dy + dx * dx <= r * r) n++;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            for (int dy = -r; dy <= r; dy++)
                for (int dx = -r; dx <= r; dx++) {
                    if (dy * dy + dx * dx > r * r) continue;
                    s += in[(size_t)wrap(y + dy, H) * W + wrap(x + dx, W)];
                }
            out[(size_t)y * W + x] = s / (double)n;
        }
}

/* Random choices of one step of Algorithm 2's evolutionary operators (drawn
 * by the caller, so both implementations see the same ones):
 *   mutation (Section 2.5): plane mut_p, kernel mut_k, delta mut_delta, square
 *     of side 2 mut_half with corner (x0 - s, y0 - s), i.e. x in [x0 - s, x0 + s);
 *   penalisation (Section 2.6): plane pen_p, kernel pen_k, delta pen_delta
 *     (its sign chosen by the caller from the plane).
 * A plane index < 0 switches that operator off. */
typedef struct {
    int mut_p, mut_k, mut_x0, mut_y0, mut_half;
    double mut_delta;
    int pen_p, pen_k;
    double pen_delta;
    double gamma_mut, gamma_pen, eps_pen;
    int r_oxy;
} oracle_evo;

/* One step with Algorithm 2's remaining lines:
 *   line 158: walls (walls[i] != 0) remove A and P before the step (Section 2.7);
 *   lines 159-165: diffuse, convolve, alpha, mask, update (oracle_step);
 *   line 164: E_oxy = (1 - Delta_sum(U)) * K_oxy, E_pen = (1 - E_oxy) * K_oxy,
 *     Delta_sum(U) = [sum_k t_k > eps_u] with t_k the per-kernel alpha test,
 *     K_oxy the normalised disk of radius r_oxy (Section 2.6);
 *   line 166: P[mut_p, mut_k] += gamma_mut delta on the square AND alpha;
 *   line 167: P[pen_p, pen_k] += gamma_pen delta on [E_pen > eps_pen] AND alpha.
 * epen_out and tsum_out (nullable) receive E_pen and sum_k t_k. */
int oracle_evolve_step(const oracle_cfg* cfg, const int* src, const int* dst, const int* R,
                       const double* h, const double* mu, const double* sigma,
                       const double* Kw, const long* kw_off, const unsigned char* walls,
                       const oracle_evo* ev, const double* A, const double* P,
                       double* A_out, double* P_out, unsigned char* alpha_out, double* epen_out,
                       double* tsum_out)
{
    const int H = cfg->H, W = cfg->W, C = cfg->C, K = cfg->K;
    const size_t N = (size_t)H * W;
    const plane_map pm = planes_of(cfg->localized);
    const size_t nP = (size_t)pm.n_p * K * N;
    double* Aw = (double*)malloc(sizeof(double) * C * N);
    double* Pw = nP ? (double*)malloc(sizeof(double) * nP) : NULL;
    for (size_t i = 0; i < C * N; i++) Aw[i] = (walls && walls[i % N]) ? 0.0 : A[i];
    for (size_t i = 0; i < nP; i++) Pw[i] = (walls && walls[i % N]) ? 0.0 : P[i];
    unsigned char* al = (unsigned char*)malloc(N);
    double* tsum = (double*)malloc(sizeof(double) * N);
    double* U = NULL;
    int rc;
    if (cfg->n_rings > 0) {
        U = ring_potentials_all(cfg, R[0], Aw);
        rc = oracle_ring_update(cfg, src, dst, R[0], h, mu, sigma, Aw, Pw, U, A_out, P_out, NULL, al, tsum);
    } else {
        U = (double*)malloc(sizeof(double) * (size_t)K * N);
        for (int k = 0; k < K; k++)
            oracle_potential(H, W, Aw + (size_t)src[k] * N, R[k], Kw + kw_off[k], U + (size_t)k * N, 0);
        rc = oracle_update(cfg, dst, h, mu, sigma, Aw, Pw, U, A_out, P_out, al, tsum);
    }
    double* empty = (double*)malloc(sizeof(double) * N);
    double* eoxy = (double*)malloc(sizeof(double) * N);
    double* epen = (double*)malloc(sizeof(double) * N);
    for (size_t i = 0; i < N; i++) empty[i] = (tsum[i] > cfg->eps_u) ? 0.0 : 1.0;
    oracle_disk_mean(H, W, empty, ev->r_oxy, eoxy);
    for (size_t i = 0; i < N; i++) empty[i] = 1.0 - eoxy[i];
    oracle_disk_mean(H, W, empty, ev->r_oxy, epen);
    if (P_out && pm.n_p && ev->mut_p >= 0) {
        double* mp = P_out + ((size_t)ev->mut_p * K + ev->mut_k) * N;
        for (int dy = -ev->mut_half; dy < ev->mut_half; dy++)
            for (int dx = -ev->mut_half; dx < ev->mut_half; dx++) {
                size_t i = (size_t)wrap(ev->mut_y0 + dy, H) * W + wrap(ev->mut_x0 + dx, W);
                if (al[i]) mp[i] += ev->gamma_mut * ev->mut_delta;
            }
    }
    if (P_out && pm.n_p && ev->pen_p >= 0) {
        double* pp = P_out + ((size_t)ev->pen_p * K + ev->pen_k) * N;
        for (size_t i = 0; i < N; i++)
            if (al[i] && epen[i] > ev->eps_pen) pp[i] += ev->gamma_pen * ev->pen_delta;
    }
    if (alpha_out) memcpy(alpha_out, al, N);
    if (epen_out) memcpy(epen_out, epen, sizeof(double) * N);
    if (tsum_out) memcpy(tsum_out, tsum, sizeof(double) * N);
    free(Aw); free(Pw); free(U); free(al); free(tsum); free(empty); free(eoxy); free(epen);
    return rc;
}

/* Per-channel mass and circular-mean centroid:
 *   M = sum A,  centre_y = atan2(sum A sin(2 pi y / H), sum A cos(2 pi y / H)) H / (2 pi)
 * wrapped to [0, H); same for x.  out[C][3] = (mass, centre_y, centre_x). */
void oracle_stats(int C, int H, int W, const double* A, double* out)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int c = 0; c < C; c++) {
        double m = 0.0, sy = 0.0, cy = 0.0, sx = 0.0, cx = 0.0;
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                double a = A[((size_t)c * H + y) * W + x];
                m += a;
                sy += a * sin(two_pi * y / H);
                cy += a * cos(two_pi * y / H);
                sx += a * sin(two_pi * x / W);
                cx += a * cos(two_pi * x / W);
            }
        double ty = atan2(sy, cy) * H / two_pi;
        double tx = atan2(sx, cx) * W / two_pi;
        if (ty < 0.0) ty += H;
        if (tx < 0.0) tx += W;
        out[c * 3 + 0] = m;
        out[c * 3 + 1] = ty;
        out[c * 3 + 2] = tx;
    }
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
