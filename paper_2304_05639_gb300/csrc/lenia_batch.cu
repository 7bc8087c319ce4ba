// Batched worlds: many independent Lenia worlds of uneven sizes, radii and
// genotypes advanced together.  Each world keeps its own context (kernels,
// spectra, scratch).  Worlds on the FFT path of the same size whose
// configuration and kernel topology are identical (they may differ in kernel
// shapes, genotypes and state) form a group that steps in one launch per
// stage: the row and column transforms treat the group's worlds as extra
// planes (the column pass reads each world's kernel spectra through a list),
// and the tiled epilogue takes the worlds along grid z, each reading and
// writing through per-world pointer lists.  The steps of
// all groups and remaining worlds are captured once into a CUDA graph whose
// branches run concurrently on worker streams, and the graph is replayed, so
// a rollout costs one graph launch per two steps.  Sizes shared by several
// worlds take the FFT path (so that they group); an autotuner times the FFT
// and direct paths once for every other shape and keeps the faster one.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/lenia.h"
#include "lenia_internal.cuh"

namespace {

constexpr int kWorkers = 16;   // concurrent graph branches

struct ShapeKey {
    int H, W, C, K, loc, maintain, rmax;
    bool operator<(const ShapeKey& o) const
    {
        return std::tie(H, W, C, K, loc, maintain, rmax) < std::tie(o.H, o.W, o.C, o.K, o.loc, o.maintain, o.rmax);
    }
};

}  // namespace

// Worlds stepped together (identical configuration and kernel topology, FFT
// path; kernel shapes may differ, each world's spectra come from a list).
struct Group {
    std::vector<int> worlds;
    lenia::lenia_ctx_view v;               // the first world's parameters
    float2* Ahat = nullptr;                // [n][C][M][H]
    float2* Uhat = nullptr;                // [n][K][M][H]
    float* U = nullptr;                    // [n][K][H][W]
    const float** S = nullptr;             // per-world kernel spectra (worlds may differ in kernels)
    // per-world pointer lists for the two ping-pong directions:
    // [0] caller's state -> batch state, [1] batch state -> caller's state
    const float** Ain[2] = {nullptr, nullptr};
    const float** Pin[2] = {nullptr, nullptr};
    float** Aout[2] = {nullptr, nullptr};
    float** Pout[2] = {nullptr, nullptr};
    bool aligned = false;                  // every listed A pointer is 16-byte aligned
    bool aligned_all = false;              // every listed A and P pointer is 16-byte aligned
    // epilogue: 0 = tiled kernel (br rows per thread), 1 = streaming kernel over
    // a device work queue (`bands` bands per world; per-world tensor maps in qw)
    lenia::QueueWorld* qw[2] = {nullptr, nullptr};
    int* counter = nullptr;                // the queue's work counter
    int epi = 0, br = 2, bands = 1;
    bool tuned = false;                    // epilogue shape chosen by the autotuner
    float tune_ms[8] = {};                 // the timed candidates (for lenia_batch_epilogue_choice)
};

struct lenia_batch {
    int n = 0;
    bool autotune = false;
    std::vector<lenia_ctx*> ctx;
    std::vector<Group> groups;
    std::vector<int> group_of;             // world -> group index or -1
    std::vector<size_t> abytes, pbytes;
    std::vector<float*> A2, P2;            // library-owned second state per world
    cudaStream_t origin = nullptr;
    cudaStream_t workers[kWorkers] = {};
    cudaEvent_t fork = nullptr, join[kWorkers] = {}, done = nullptr;
    cudaGraphExec_t g2 = nullptr;          // two steps: user -> A2 -> user
    cudaGraphExec_t g1 = nullptr;          // one step user -> A2, copy back
    std::vector<const void*> key2, key1;   // pointers the graphs were captured with
};

namespace {

lenia_status bfail(const char* msg)
{
    fprintf(stderr, "lenia_batch: %s\n", msg);
    return LENIA_EINVAL;
}

// Time `reps` steps of a fresh context with the given path on zero-filled
// state (the arithmetic does not depend on the values).
float time_path(const lenia_config& cfg0, const lenia_kernel_desc* ks, int path, cudaStream_t s)
{
    lenia_config cfg = cfg0;
    cfg.conv_path = path;
    cfg.max_rollout_steps = 0;
    lenia_ctx* c = nullptr;
    if (lenia_init(&cfg, ks, s, &c) != LENIA_OK) return INFINITY;
    const size_t N = (size_t)cfg.height * cfg.width;
    const int n_p = ((cfg.localized & 1) != 0) + ((cfg.localized & 2) != 0) + ((cfg.localized & 4) != 0);
    float *A = nullptr, *P = nullptr;
    float ms = INFINITY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    if (cudaMalloc(&A, N * cfg.n_channels * sizeof(float)) == cudaSuccess &&
        (n_p == 0 || cudaMalloc(&P, N * n_p * cfg.n_kernels * sizeof(float)) == cudaSuccess)) {
        cudaMemsetAsync(A, 0, N * cfg.n_channels * sizeof(float), s);
        if (P) cudaMemsetAsync(P, 0, N * n_p * cfg.n_kernels * sizeof(float), s);
        bool ok = lenia_rollout(c, A, P, 2, nullptr, s) == LENIA_OK;    // warm-up
        cudaEventRecord(e0, s);
        ok = ok && lenia_rollout(c, A, P, 6, nullptr, s) == LENIA_OK;
        cudaEventRecord(e1, s);
        if (ok && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (A) cudaFree(A);
    if (P) cudaFree(P);
    lenia_destroy(c);
    return ms;
}

void free_group(Group& g)
{
    void* ptrs[] = {g.Ahat, g.Uhat, g.U, g.S, g.Ain[0], g.Ain[1], g.Pin[0], g.Pin[1], g.Aout[0], g.Aout[1],
                    g.Pout[0], g.Pout[1], g.qw[0], g.qw[1], g.counter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

// The epilogue parameters of a group for direction `dir`.
lenia::EpiParams group_epi(const Group& g, int dir)
{
    lenia::EpiParams ep = g.v.ep;
    ep.A = ep.P = nullptr;
    ep.A_out = ep.P_out = nullptr;
    ep.A_list = g.Ain[dir];
    ep.P_list = g.Pin[dir];
    ep.Aout_list = g.Aout[dir];
    ep.Pout_list = g.Pout[dir];
    ep.U = g.U;
    ep.u_stride = (size_t)g.v.K * g.v.N;
    ep.partials = nullptr;
    ep.stats_out = nullptr;
    ep.alpha_out = ep.empty_out = nullptr;
    return ep;
}

// The group's epilogue in the chosen shape.
cudaError_t group_epilogue(const Group& g, int dir, cudaStream_t s)
{
    const lenia::EpiParams ep = group_epi(g, dir);
    const int n = (int)g.worlds.size();
    if (g.epi == 1) return lenia::launch_epilogue_queue(ep, g.qw[dir], n, g.bands, 0, g.counter, g.v.fp.status, s);
    // the four-column form needs 16-byte aligned state buffers
    return lenia::launch_epilogue_batch(ep, n, s, g.br < 0 && !g.aligned_all ? 2 : g.br);
}

// One step of every world of a group: A/P lists of direction `dir`.
lenia_status group_step(const Group& g, int dir, cudaStream_t s)
{
    const int n = (int)g.worlds.size();
    lenia::FftParams fp = g.v.fp;
    fp.A = nullptr;
    fp.A_list = g.Ain[dir];
    fp.S_list = g.S;
    fp.list_aligned = g.aligned ? 1 : 0;
    fp.Ahat = g.Ahat;
    fp.Uhat = g.Uhat;
    fp.U = g.U;
    fp.cw = g.v.C;
    fp.kpw = g.v.K;
    fp.C = n * g.v.C;                      // planes of the row and column passes
    fp.K = n * g.v.K;                      // planes of the inverse row pass
    if (lenia::launch_fft_rows_r2c(fp, s) != cudaSuccess) return LENIA_ECUDA;
    if (lenia::launch_fft_cols(fp, s) != cudaSuccess) return LENIA_ECUDA;
    if (lenia::launch_fft_rows_c2r(fp, s) != cudaSuccess) return LENIA_ECUDA;
    return group_epilogue(g, dir, s) == cudaSuccess ? LENIA_OK : LENIA_ECUDA;
}

// Autotuner of the epilogue's shape: times every candidate on direction 0
// (the caller's state in, the batch's buffers out: the caller's data are not
// changed) and keeps the fastest.  Candidates: the tiled kernel with 1, 2 or
// 4 rows per thread, and - for widths of 256 k - the queued streaming kernel
// with 1, 2, 4 or 8 bands per world.
lenia_status tune_epilogue(Group& g, cudaStream_t s)
{
    const lenia::EpiParams ep = group_epi(g, 0);
    struct Cand {
        int epi, br, bands;
    };
    std::vector<Cand> cands = {{0, 1, 1}, {0, 2, 1}, {0, 4, 1}};
    // four columns per thread (float4 loads; widths of 128 k, every listed pointer 16-byte aligned)
    if (g.v.K == 1 && g.v.C == 1 && g.v.fp.W % 128 == 0 && g.aligned_all)
        for (int b : {-1, -2})
            if (g.v.fp.H % (8 * -b) == 0) cands.push_back({0, b, 1});
    if (g.qw[0])
        for (int b : {1, 2, 4, 8})
            if (b <= g.v.fp.H) cands.push_back({1, 2, b});
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LENIA_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LENIA_ECUDA;
    }
    // each candidate timed in three rounds of five launches (rounds interleaved
    // over the candidates), its best round kept: single rounds of candidates
    // within ~20% of each other ordered them differently from run to run
    std::vector<float> t_best(cands.size(), INFINITY);
    for (int round = 0; round < 3; round++) {
        for (size_t ci = 0; ci < cands.size(); ci++) {
            Group t = g;
            t.epi = cands[ci].epi;
            t.br = cands[ci].br;
            t.bands = cands[ci].bands;
            bool ok = true;
            for (int r = 0; ok && r < 2; r++) ok = group_epilogue(t, 0, s) == cudaSuccess;     // warm-up
            ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
            for (int r = 0; ok && r < 5; r++) ok = group_epilogue(t, 0, s) == cudaSuccess;
            ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
            float ms = INFINITY;
            if (ok) cudaEventElapsedTime(&ms, e0, e1);
            else (void)cudaGetLastError();
            t_best[ci] = std::min(t_best[ci], ms);
        }
    }
    float best = INFINITY;
    Cand pick = {0, 2, 1};
    for (size_t ci = 0; ci < cands.size(); ci++) {
        if (ci < 8) g.tune_ms[ci] = t_best[ci] / 5;
        if (t_best[ci] < best) {
            best = t_best[ci];
            pick = cands[ci];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g.epi = pick.epi;
    g.br = pick.br;
    g.bands = pick.bands;
    g.tuned = true;
    return best < INFINITY ? LENIA_OK : LENIA_ECUDA;
}

void destroy_graphs(lenia_batch* b)
{
    if (b->g2) cudaGraphExecDestroy(b->g2);
    if (b->g1) cudaGraphExecDestroy(b->g1);
    b->g2 = b->g1 = nullptr;
    b->key2.clear();
    b->key1.clear();
}

// Capture `steps` steps of every world (ping-pong between the caller's
// buffers and the batch's), worlds spread over the worker streams.
lenia_status capture(lenia_batch* b, float* const* A, float* const* P, int steps, bool copy_back,
                     cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LENIA_ECUDA;
    lenia_status st = LENIA_OK;
    cudaEventRecord(b->fork, b->origin);
    for (int w = 0; w < kWorkers; w++) cudaStreamWaitEvent(b->workers[w], b->fork, 0);
    int lane = 0;
    for (size_t gi = 0; gi < b->groups.size() && st == LENIA_OK; gi++) {
        Group& g = b->groups[gi];
        cudaStream_t s = b->workers[lane++ % kWorkers];
        for (int t = 0; t < steps && st == LENIA_OK; t++) st = group_step(g, t % 2, s);
        for (int i : g.worlds) {
            if (st != LENIA_OK || !copy_back || !(steps % 2)) break;
            if (cudaMemcpyAsync(A[i], b->A2[i], b->abytes[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                st = LENIA_ECUDA;
            if (b->pbytes[i] &&
                cudaMemcpyAsync(P[i], b->P2[i], b->pbytes[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                st = LENIA_ECUDA;
        }
    }
    for (int i = 0; i < b->n && st == LENIA_OK; i++) {
        if (b->group_of[i] >= 0) continue;
        cudaStream_t s = b->workers[lane++ % kWorkers];
        const bool hasP = b->pbytes[i] > 0;
        for (int t = 0; t < steps && st == LENIA_OK; t++) {
            const bool even = (t % 2) == 0;
            float* ai = even ? A[i] : b->A2[i];
            float* ao = even ? b->A2[i] : A[i];
            float* pi = hasP ? (even ? P[i] : b->P2[i]) : nullptr;
            float* po = hasP ? (even ? b->P2[i] : P[i]) : nullptr;
            st = lenia_step(b->ctx[i], ai, pi, ao, po, nullptr, s);
        }
        if (st == LENIA_OK && copy_back && (steps % 2)) {
            if (cudaMemcpyAsync(A[i], b->A2[i], b->abytes[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                st = LENIA_ECUDA;
            if (hasP && cudaMemcpyAsync(P[i], b->P2[i], b->pbytes[i], cudaMemcpyDeviceToDevice, s) != cudaSuccess)
                st = LENIA_ECUDA;
        }
    }
    for (int w = 0; w < kWorkers; w++) {
        cudaEventRecord(b->join[w], b->workers[w]);
        cudaStreamWaitEvent(b->origin, b->join[w], 0);
    }
    cudaError_t e = cudaStreamEndCapture(b->origin, &g);
    if (st != LENIA_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != LENIA_OK ? st : LENIA_ECUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e == cudaSuccess ? LENIA_OK : LENIA_ECUDA;
}

std::vector<const void*> key_of(lenia_batch* b, float* const* A, float* const* P)
{
    std::vector<const void*> k;
    for (int i = 0; i < b->n; i++) {
        k.push_back(A[i]);
        k.push_back(P ? P[i] : nullptr);
    }
    return k;
}

// Launch the graph on the batch's origin stream, ordered after `stream`'s
// earlier work and before its later work.
lenia_status run_graph(lenia_batch* b, cudaGraphExec_t g, cudaStream_t stream)
{
    if (cudaEventRecord(b->done, stream) != cudaSuccess) return LENIA_ECUDA;
    if (cudaStreamWaitEvent(b->origin, b->done, 0) != cudaSuccess) return LENIA_ECUDA;
    if (cudaGraphLaunch(g, b->origin) != cudaSuccess) return LENIA_ECUDA;
    if (cudaEventRecord(b->done, b->origin) != cudaSuccess) return LENIA_ECUDA;
    if (cudaStreamWaitEvent(stream, b->done, 0) != cudaSuccess) return LENIA_ECUDA;
    return LENIA_OK;
}

}  // namespace

extern "C" {

void lenia_batch_destroy(lenia_batch* b)
{
    if (!b) return;
    destroy_graphs(b);
    for (Group& g : b->groups) free_group(g);
    for (lenia_ctx* c : b->ctx) lenia_destroy(c);
    for (float* p : b->A2)
        if (p) cudaFree(p);
    for (float* p : b->P2)
        if (p) cudaFree(p);
    for (int w = 0; w < kWorkers; w++) {
        if (b->workers[w]) cudaStreamDestroy(b->workers[w]);
        if (b->join[w]) cudaEventDestroy(b->join[w]);
    }
    if (b->origin) cudaStreamDestroy(b->origin);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    delete b;
}

lenia_status lenia_batch_init(int32_t n_worlds, const lenia_config* cfgs, const lenia_kernel_desc* kernels,
                              int32_t autotune, void* stream, lenia_batch** out)
{
    if (!out) return LENIA_EINVAL;
    *out = nullptr;
    if (n_worlds < 1 || n_worlds > 65536 || !cfgs || !kernels) return bfail("n_worlds, cfgs and kernels");
    cudaStream_t s = (cudaStream_t)stream;
    lenia_batch* b = new lenia_batch();
    b->n = n_worlds;
    b->autotune = autotune != 0;
    bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess;
    for (int w = 0; ok && w < kWorkers; w++)
        ok = cudaStreamCreateWithFlags(&b->workers[w], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[w], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        lenia_batch_destroy(b);
        return LENIA_ECUDA;
    }
    std::map<ShapeKey, int> tuned;   // shape -> chosen path
    // shapes shared by several worlds take the FFT path when it exists: their
    // worlds can then step as one group (one launch per stage for all of them)
    std::map<ShapeKey, int> shape_count;
    {
        size_t ko = 0;
        for (int i = 0; i < n_worlds; i++) {
            const lenia_kernel_desc* ks = kernels + ko;
            if (cfgs[i].n_kernels < 1 || cfgs[i].n_kernels > 64) break;      // reported below
            ko += cfgs[i].n_kernels;
            int rmax = 0;
            for (int k = 0; k < cfgs[i].n_kernels; k++) rmax = rmax > ks[k].radius ? rmax : ks[k].radius;
            (void)rmax;
            shape_count[ShapeKey{cfgs[i].height, cfgs[i].width, cfgs[i].n_channels, cfgs[i].n_kernels,
                                 cfgs[i].localized, cfgs[i].maintain_genes, 0}]++;
        }
    }
    size_t koff = 0;
    for (int i = 0; i < n_worlds; i++) {
        lenia_config cfg = cfgs[i];
        cfg.max_rollout_steps = 0;
        const lenia_kernel_desc* ks = kernels + koff;
        if (cfg.n_kernels < 1 || cfg.n_kernels > 64) {
            lenia_batch_destroy(b);
            return bfail("n_kernels out of range");
        }
        koff += cfg.n_kernels;
        if (autotune && cfg.conv_path == LENIA_CONV_AUTO) {
            int rmax = 0;
            for (int k = 0; k < cfg.n_kernels; k++) rmax = rmax > ks[k].radius ? rmax : ks[k].radius;
            const ShapeKey key{cfg.height, cfg.width, cfg.n_channels, cfg.n_kernels, cfg.localized,
                               cfg.maintain_genes, rmax};
            auto it = tuned.find(key);
            if (it == tuned.end()) {
                const ShapeKey size_key{key.H, key.W, key.C, key.K, key.loc, key.maintain, 0};
                if (shape_count[size_key] > 1 && lenia::fft_size_supported(cfg.height, cfg.width) && cfg.n_rings == 0) {
                    it = tuned.emplace(key, LENIA_CONV_FFT).first;
                } else {
                    const float t_direct = time_path(cfg, ks, LENIA_CONV_DIRECT, s);
                    const float t_fft = time_path(cfg, ks, LENIA_CONV_FFT, s);   // inf when unsupported
                    it = tuned.emplace(key, t_fft < t_direct ? LENIA_CONV_FFT : LENIA_CONV_DIRECT).first;
                }
            }
            cfg.conv_path = it->second;
        }
        lenia_ctx* c = nullptr;
        lenia_status st = lenia_init(&cfg, ks, s, &c);
        if (st != LENIA_OK) {
            lenia_batch_destroy(b);
            return st;
        }
        b->ctx.push_back(c);
        const size_t N = (size_t)cfg.height * cfg.width;
        const int n_p = ((cfg.localized & 1) != 0) + ((cfg.localized & 2) != 0) + ((cfg.localized & 4) != 0);
        b->abytes.push_back(N * cfg.n_channels * sizeof(float));
        b->pbytes.push_back(N * n_p * cfg.n_kernels * sizeof(float));
        float *a2 = nullptr, *p2 = nullptr;
        if (cudaMalloc(&a2, b->abytes.back()) != cudaSuccess ||
            (b->pbytes.back() && cudaMalloc(&p2, b->pbytes.back()) != cudaSuccess)) {
            if (a2) cudaFree(a2);
            lenia_batch_destroy(b);
            return LENIA_ENOMEM;
        }
        b->A2.push_back(a2);
        b->P2.push_back(p2);
    }
    // groups: worlds on the FFT path with a tiled epilogue whose configuration
    // and kernels are identical field by field
    b->group_of.assign(n_worlds, -1);
    {
        std::map<std::vector<double>, std::vector<int>> members;
        size_t ko = 0;
        for (int i = 0; i < n_worlds; i++) {
            const lenia_config& c0 = cfgs[i];
            const lenia_kernel_desc* ks = kernels + ko;
            ko += c0.n_kernels;
            lenia::lenia_ctx_view v;
            if (!lenia::ctx_view(b->ctx[i], &v) || !lenia::epilogue_batch_supported(v.ep)) continue;
            std::vector<double> key = {(double)c0.height, (double)c0.width, (double)c0.n_channels,
                                       (double)c0.n_kernels, c0.dt, (double)c0.growth_form, (double)c0.localized,
                                       (double)c0.maintain_genes, c0.eps_u, c0.eps_p, (double)c0.r_diff,
                                       (double)c0.alpha_on, (double)c0.n_rings};
            // kernel shapes may differ (each world's spectra are read through a list)
            for (int k = 0; k < c0.n_kernels; k++) {
                const lenia_kernel_desc& d = ks[k];
                key.push_back((double)d.src_channel);
                key.push_back((double)d.dst_channel);
                // global genes matter only where they are not read from the gene maps
                key.push_back((c0.localized & LENIA_LOC_H) ? 0.0 : (double)d.h);
                key.push_back((c0.localized & LENIA_LOC_MU) ? 0.0 : (double)d.mu);
                key.push_back((c0.localized & LENIA_LOC_SIGMA) ? 0.0 : (double)d.sigma);
            }
            members[key].push_back(i);
        }
        for (auto& kv : members) {
            if (kv.second.size() < 2) continue;
            Group g;
            g.worlds = kv.second;
            lenia::ctx_view(b->ctx[g.worlds[0]], &g.v);
            const size_t n = g.worlds.size();
            const size_t H = cfgs[g.worlds[0]].height, W = cfgs[g.worlds[0]].width, M = W / 2;
            bool okg = cudaMalloc(&g.Ahat, n * g.v.C * M * H * sizeof(float2)) == cudaSuccess &&
                       cudaMalloc(&g.Uhat, n * g.v.K * M * H * sizeof(float2)) == cudaSuccess &&
                       cudaMalloc(&g.U, n * g.v.K * g.v.N * sizeof(float)) == cudaSuccess &&
                       cudaMalloc(&g.S, n * sizeof(float*)) == cudaSuccess;
            if (okg) {
                std::vector<const float*> spec(n);
                for (size_t j = 0; j < n; j++) {
                    lenia::lenia_ctx_view vj;
                    lenia::ctx_view(b->ctx[g.worlds[j]], &vj);
                    spec[j] = vj.fp.S;
                }
                okg = cudaMemcpy(g.S, spec.data(), n * sizeof(float*), cudaMemcpyHostToDevice) == cudaSuccess;
            }
            for (int d = 0; okg && d < 2; d++)
                okg = cudaMalloc(&g.Ain[d], n * sizeof(float*)) == cudaSuccess &&
                      cudaMalloc(&g.Pin[d], n * sizeof(float*)) == cudaSuccess &&
                      cudaMalloc(&g.Aout[d], n * sizeof(float*)) == cudaSuccess &&
                      cudaMalloc(&g.Pout[d], n * sizeof(float*)) == cudaSuccess;
            if (!okg) {
                free_group(g);
                lenia_batch_destroy(b);
                return LENIA_ENOMEM;
            }
            if (okg && lenia::epilogue_queue_supported(group_epi(g, 0))) {
                okg = cudaMalloc(&g.qw[0], n * sizeof(lenia::QueueWorld)) == cudaSuccess &&
                      cudaMalloc(&g.qw[1], n * sizeof(lenia::QueueWorld)) == cudaSuccess &&
                      cudaMalloc(&g.counter, sizeof(int)) == cudaSuccess;
                if (!okg) {
                    free_group(g);
                    lenia_batch_destroy(b);
                    return LENIA_ENOMEM;
                }
            }
            for (int i : g.worlds) b->group_of[i] = (int)b->groups.size();
            b->groups.push_back(g);
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        lenia_batch_destroy(b);
        return LENIA_ECUDA;
    }
    *out = b;
    return LENIA_OK;
}

int32_t lenia_batch_epilogue_shape(const lenia_batch* b, int32_t world, int32_t* param)
{
    if (!b || world < 0 || world >= b->n || b->group_of[world] < 0) return -1;
    const Group& g = b->groups[b->group_of[world]];
    if (param) *param = g.epi == 1 ? g.bands : (g.br < 0 ? -g.br : g.br);
    return g.epi == 1 ? 1 : (g.br < 0 ? 2 : 0);
}

lenia_status lenia_batch_set_epilogue_shape(lenia_batch* b, int32_t world, int32_t kind, int32_t param)
{
    if (!b || world < 0 || world >= b->n || b->group_of[world] < 0) return LENIA_EINVAL;
    Group& g = b->groups[b->group_of[world]];
    if (kind == 0 && (param == 1 || param == 2 || param == 4) && g.v.fp.H % (8 * param) == 0) {
        g.epi = 0;
        g.br = param;
    } else if (kind == 2 && (param == 1 || param == 2) && g.v.K == 1 && g.v.C == 1 && g.v.fp.W % 128 == 0 &&
               g.v.fp.H % (8 * param) == 0) {
        g.epi = 0;
        g.br = -param;
    } else if (kind == 1 && param >= 1 && param <= g.v.fp.H && g.qw[0]) {
        g.epi = 1;
        g.bands = param;
    } else {
        return LENIA_EINVAL;
    }
    g.tuned = true;
    destroy_graphs(b);
    return LENIA_OK;
}

lenia_status lenia_batch_rollout(lenia_batch* b, float* const* A, float* const* P, int32_t n_steps, void* stream)
{
    if (!b || !A || n_steps < 0) return LENIA_EINVAL;
    for (int i = 0; i < b->n; i++)
        if (!A[i] || (b->pbytes[i] && (!P || !P[i]))) return bfail("state pointers");
    if (n_steps == 0) return LENIA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const std::vector<const void*> key = key_of(b, A, P);
    if ((n_steps >= 2 && b->key2 != key) || ((n_steps % 2) && b->key1 != key)) {
        // the groups' pointer lists for these buffers (read when the graphs run)
        if (cudaStreamSynchronize(b->origin) != cudaSuccess) return LENIA_ECUDA;
        for (Group& g : b->groups) {
            const size_t n = g.worlds.size();
            std::vector<const float*> a0(n), p0(n), a1(n), p1(n);
            std::vector<float*> ao0(n), po0(n), ao1(n), po1(n);
            g.aligned = true;
            g.aligned_all = true;
            for (size_t j = 0; j < n; j++) {
                const int i = g.worlds[j];
                a0[j] = A[i];
                p0[j] = P ? P[i] : nullptr;
                ao0[j] = b->A2[i];
                po0[j] = b->P2[i];
                a1[j] = b->A2[i];
                p1[j] = b->P2[i];
                ao1[j] = A[i];
                po1[j] = P ? P[i] : nullptr;
                g.aligned = g.aligned && ((uintptr_t)A[i] % 16 == 0) && ((uintptr_t)b->A2[i] % 16 == 0);
                g.aligned_all = g.aligned_all && ((uintptr_t)A[i] % 16 == 0) && ((uintptr_t)b->A2[i] % 16 == 0) &&
                                ((uintptr_t)(P ? P[i] : nullptr) % 16 == 0) && ((uintptr_t)b->P2[i] % 16 == 0);
            }
            const size_t pb = n * sizeof(float*);
            bool ok = cudaMemcpy(g.Ain[0], a0.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Pin[0], p0.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Aout[0], ao0.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Pout[0], po0.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Ain[1], a1.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Pin[1], p1.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Aout[1], ao1.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess &&
                      cudaMemcpy(g.Pout[1], po1.data(), pb, cudaMemcpyHostToDevice) == cudaSuccess;
            if (!ok) return LENIA_ECUDA;
            if (g.qw[0]) {
                // per-world tensor maps of the queued streaming epilogue, both directions
                const lenia::EpiParams ep = group_epi(g, 0);
                for (int d = 0; d < 2; d++) {
                    std::vector<lenia::QueueWorld> q(n);
                    for (size_t j = 0; j < n && ok; j++)
                        ok = lenia::epilogue_queue_world(&q[j], ep, d ? a1[j] : a0[j], d ? p1[j] : p0[j],
                                                         g.U + j * g.v.K * g.v.N, d ? ao1[j] : ao0[j],
                                                         d ? po1[j] : po0[j]);
                    ok = ok && cudaMemcpy(g.qw[d], q.data(), n * sizeof(lenia::QueueWorld),
                                          cudaMemcpyHostToDevice) == cudaSuccess;
                }
                if (!ok) {
                    // maps cannot be encoded for these buffers: the tiled kernel only
                    cudaFree(g.qw[0]);
                    cudaFree(g.qw[1]);
                    g.qw[0] = g.qw[1] = nullptr;
                    if (g.epi == 1) g.epi = 0;
                    ok = true;
                }
            }
            if (b->autotune && !g.tuned) {
                const lenia_status ts = tune_epilogue(g, b->origin);
                if (ts != LENIA_OK) return ts;
            }
        }
        destroy_graphs(b);
    }
    if (n_steps >= 2 && (!b->g2 || b->key2 != key)) {
        if (b->g2) cudaGraphExecDestroy(b->g2);
        b->g2 = nullptr;
        lenia_status st = capture(b, A, P, 2, false, &b->g2);
        if (st != LENIA_OK) return st;
        b->key2 = key;
    }
    if ((n_steps % 2) && (!b->g1 || b->key1 != key)) {
        if (b->g1) cudaGraphExecDestroy(b->g1);
        b->g1 = nullptr;
        lenia_status st = capture(b, A, P, 1, true, &b->g1);
        if (st != LENIA_OK) return st;
        b->key1 = key;
    }
    for (int t = 0; t + 1 < n_steps; t += 2) {
        lenia_status st = run_graph(b, b->g2, s);
        if (st != LENIA_OK) return st;
    }
    if (n_steps % 2) return run_graph(b, b->g1, s);
    return LENIA_OK;
}

int32_t lenia_batch_group_of(const lenia_batch* b, int32_t world)
{
    if (!b || world < 0 || world >= b->n) return -1;
    return b->group_of[world];
}

int32_t lenia_batch_conv_path(const lenia_batch* b, int32_t world)
{
    if (!b || world < 0 || world >= b->n) return -1;
    return lenia_conv_path(b->ctx[world]);
}

lenia_status lenia_batch_check(lenia_batch* b, void* stream)
{
    if (!b) return LENIA_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LENIA_ECUDA;
    for (lenia_ctx* c : b->ctx) {
        lenia_status st = lenia_check(c, nullptr);
        if (st != LENIA_OK) return st;
    }
    return LENIA_OK;
}

}  // extern "C"
