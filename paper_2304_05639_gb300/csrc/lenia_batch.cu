// Batched worlds: many independent Lenia worlds of uneven sizes, radii and
// genotypes advanced together.  Each world keeps its own context (kernels,
// spectra, scratch); the steps of all worlds are captured once into a CUDA
// graph whose branches run the worlds concurrently on worker streams, and the
// graph is replayed, so a rollout costs one graph launch per two steps.  An
// autotuner times the FFT and direct paths once per distinct world shape and
// keeps the faster one.
#include <math.h>
#include <stdio.h>
#include <string.h>

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

struct lenia_batch {
    int n = 0;
    std::vector<lenia_ctx*> ctx;
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
    for (int i = 0; i < b->n && st == LENIA_OK; i++) {
        cudaStream_t s = b->workers[i % kWorkers];
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
                const float t_direct = time_path(cfg, ks, LENIA_CONV_DIRECT, s);
                const float t_fft = time_path(cfg, ks, LENIA_CONV_FFT, s);   // inf when unsupported
                it = tuned.emplace(key, t_fft < t_direct ? LENIA_CONV_FFT : LENIA_CONV_DIRECT).first;
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
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        lenia_batch_destroy(b);
        return LENIA_ECUDA;
    }
    *out = b;
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
