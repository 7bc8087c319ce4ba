// lenia_stats_noalloc: the per-channel mass / centroid reduction of
// lenia_stats for callers that cannot allocate device memory.  Its scratch
// (block partial sums and the sine/cosine tables) lives in one file-scope
// static device array of fixed size instead of context-owned cudaMalloc
// memory; nothing here allocates.
#include <stdio.h>

#include <mutex>

#include "../../include/lenia.h"
#include "lenia_internal.cuh"

using namespace lenia;

namespace {

// Limits of the static scratch: (stats blocks x channels) partial records of
// five compensated (hi, lo) FP32 pairs, 8 bytes each, and sine/cosine tables
// for H, W <= 8192; the array is declared in 8-byte slots.
constexpr int kNoAllocMaxRecords = 65536;
constexpr int kNoAllocMaxSide = 8192;
constexpr size_t kPartialSlots = (size_t)kNoAllocMaxRecords * 5;
constexpr size_t kTrigFloats = 4 * (size_t)kNoAllocMaxSide;
constexpr size_t kScratchDoubles = kPartialSlots + kTrigFloats / 2;   // 2.75 MB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array in the current device's current context.  The
// address is looked up again (cudaGetSymbolAddress: a lookup, no allocation)
// on every call whose stream is not capturing, so a context that was reset
// (cudaDeviceReset) or replaced since the last call gets its own address; a
// capturing stream reuses the address of the device's last such lookup, which
// is why the first call on a device must come before any capture.
cudaError_t scratch_address(cudaStream_t s, void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// sin/cos of 2 pi y / H and 2 pi x / W, the tables the stats kernels read.
__global__ void k_noalloc_trig(float* trig, int H, int W)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < H + W; i += gridDim.x * blockDim.x) {
        if (i < H) {
            double s, c;
            sincospi(2.0 * i / H, &s, &c);
            trig[i] = (float)s;
            trig[H + i] = (float)c;
        } else {
            const int x = i - H;
            double s, c;
            sincospi(2.0 * x / W, &s, &c);
            trig[2 * H + x] = (float)s;
            trig[2 * H + W + x] = (float)c;
        }
    }
}

}  // namespace

extern "C" lenia_status lenia_stats_noalloc(const float* A, int32_t n_channels, int32_t height, int32_t width,
                                            float* out, void* stream)
{
    if (!A || !out) {
        fprintf(stderr, "lenia_stats_noalloc: A and out must be non-null\n");
        return LENIA_EINVAL;
    }
    if (n_channels < 1 || n_channels > kMaxChannels || height < 1 || width < 1 ||
        height > kNoAllocMaxSide || width > kNoAllocMaxSide) {
        fprintf(stderr, "lenia_stats_noalloc: need 1 <= channels <= %d and 1 <= height, width <= %d\n",
                kMaxChannels, kNoAllocMaxSide);
        return LENIA_EINVAL;
    }
    const long long records = (long long)epilogue_blocks(height, width) * n_channels;
    if (records > kNoAllocMaxRecords) {
        fprintf(stderr,
                "lenia_stats_noalloc: world too large for the static scratch "
                "(ceil(W/32) * ceil(H/32) * channels = %lld > %d)\n",
                records, kNoAllocMaxRecords);
        return LENIA_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void* base = nullptr;
    cudaError_t e = scratch_address(s, &base);
    if (e != cudaSuccess) {
        fprintf(stderr, "lenia_stats_noalloc: scratch address lookup: %s\n", cudaGetErrorString(e));
        return LENIA_ECUDA;
    }
    float2* partials = (float2*)base;
    float* trig = (float*)(partials + kPartialSlots);
    const int H = height, W = width, C = n_channels;
    k_noalloc_trig<<<(H + W + 255) / 256, 256, 0, s>>>(trig, H, W);
    e = cudaGetLastError();
    int nb = 0;
    if (e == cudaSuccess)
        e = launch_stats_partials(A, C, H, W, trig, trig + H, trig + 2 * H, trig + 2 * H + W, partials, s, &nb);
    if (e == cudaSuccess) e = launch_stats_final(partials, nb, C, H, W, out, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "lenia_stats_noalloc: launch failed: %s\n", cudaGetErrorString(e));
        return LENIA_ECUDA;
    }
    return LENIA_OK;
}
