// mqr_noalloc.cu -- mqr_sort_objects_noalloc: the Morton-key computation and
// radix sort of the objects, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: embedders that own all device memory
// (a fixed budget or their own pool) and latency-critical loops that cannot
// afford the device-wide synchronisation cudaMalloc / cudaFree may cause.
// This entry point needs no allocation at all: its scratch (sort ping-pong
// buffers, digit histograms, look-back status) is one file-scope __device__
// array of fixed size (about 4.3 MB for MQR_NOALLOC_MAX_OBJECTS objects),
// which every GPU that loads the library holds until the process exits.  The
// caller passes only inputs and outputs.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mqr.h"
#include "mqr_internal.cuh"

using namespace mqr;

namespace {

constexpr uint32_t kMaxN = MQR_NOALLOC_MAX_OBJECTS;
constexpr uint32_t kTiles = (kMaxN + kSortTile - 1) / kSortTile;

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t kOffKeysA = 0;
constexpr size_t kOffKeysB = kOffKeysA + (size_t)kMaxN * 8;
constexpr size_t kOffHist = kOffKeysB + (size_t)kMaxN * 8;            // 4 x 256 u32
constexpr size_t kOffCounters = kOffHist + 4 * 256 * 4;                // 4 tile counters + error word
constexpr size_t kOffStatus = kOffCounters + 256;                      // 4 x 256 x kTiles u32
constexpr size_t kZeroBytes = kOffStatus + (size_t)4 * 256 * kTiles * 4 - kOffHist;
constexpr size_t kScratchBytes = kOffStatus + (size_t)4 * 256 * kTiles * 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_dev_ptr[kMaxDevices] = {};

mqr_status nfail(mqr_status s, const std::string &m) {
    set_last_error(m);   // reported by mqr_last_error()
    return s;
}

// Morton keys of objects 0..n-1 (all present) packed as (key << 32 | id),
// plus the digit histograms of the four 8-bit passes over bits 32..63.
__global__ void noalloc_keys_kernel(const float2 *__restrict__ xy, uint32_t n, float x0, float y0, float sx,
                                    float sy, unsigned char *scratch) {
    __shared__ uint32_t s_hist[4 * 256];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch + kOffKeysA);
    uint32_t *hist = reinterpret_cast<uint32_t *>(scratch + kOffHist);
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 p = xy[i];
        const uint32_t k = morton2(cell_of(p.x, x0, sx), cell_of(p.y, y0, sy));
        keys[i] = ((unsigned long long)k << 32) | i;
        atomicAdd(&s_hist[k & 255u], 1u);
        atomicAdd(&s_hist[256 + ((k >> 8) & 255u)], 1u);
        atomicAdd(&s_hist[512 + ((k >> 16) & 255u)], 1u);
        atomicAdd(&s_hist[768 + (k >> 24)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x)
        if (s_hist[i]) atomicAdd(hist + i, s_hist[i]);
}

__global__ void noalloc_split_kernel(const unsigned long long *__restrict__ sorted, uint32_t n,
                                     uint32_t *__restrict__ keys_out, uint32_t *__restrict__ ids_out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned long long k = sorted[i];
        keys_out[i] = (uint32_t)(k >> 32);
        ids_out[i] = (uint32_t)k;
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress must run with that device current).
mqr_status scratch_ptr(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(MQR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(MQR_ERR_INTERNAL, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return nfail(MQR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return MQR_OK;
}

}  // namespace

extern "C" mqr_status mqr_sort_objects_noalloc(mqr_rect bounds, const float *xy_dev, uint32_t n,
                                               uint32_t *keys_out_dev, uint32_t *ids_out_dev,
                                               void *cuda_stream) {
    if (n > kMaxN)
        return nfail(MQR_ERR_INVALID_ARG, "n exceeds MQR_NOALLOC_MAX_OBJECTS (" + std::to_string(kMaxN) + ")");
    if (n > 0 && (!xy_dev || !keys_out_dev || !ids_out_dev))
        return nfail(MQR_ERR_INVALID_ARG, "xy_dev / keys_out_dev / ids_out_dev is NULL");
    if (!(bounds.xmax > bounds.xmin) || !(bounds.ymax > bounds.ymin))
        return nfail(MQR_ERR_INVALID_ARG, "bounds must have xmax > xmin and ymax > ymin");
    if (n > 0 && ((reinterpret_cast<uintptr_t>(xy_dev) & 7u) ||
                  ((reinterpret_cast<uintptr_t>(keys_out_dev) | reinterpret_cast<uintptr_t>(ids_out_dev)) & 3u)))
        return nfail(MQR_ERR_INVALID_ARG, "xy_dev must be 8-byte and keys_out_dev / ids_out_dev 4-byte aligned");
    if (n == 0) return MQR_OK;
    unsigned char *s = nullptr;
    mqr_status st = scratch_ptr(&s);
    if (st != MQR_OK) return st;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    volatile float wx = bounds.xmax - bounds.xmin, wy = bounds.ymax - bounds.ymin;
    volatile float sx = 32768.0f / wx, sy = 32768.0f / wy;

    // The array keeps the previous call's contents: clear the histograms, the
    // tile counters, the error word and the look-back status.
    cudaError_t e = cudaMemsetAsync(s + kOffHist, 0, kZeroBytes, stream);
    if (e != cudaSuccess) return nfail(MQR_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    uint32_t grid = (n + 4095) / 4096;
    noalloc_keys_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const float2 *>(xy_dev), n, bounds.xmin,
                                                  bounds.ymin, sx, sy, s);
    unsigned long long *a = reinterpret_cast<unsigned long long *>(s + kOffKeysA);
    unsigned long long *b = reinterpret_cast<unsigned long long *>(s + kOffKeysB);
    uint32_t *hist = reinterpret_cast<uint32_t *>(s + kOffHist);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(s + kOffCounters);
    unsigned long long *err = reinterpret_cast<unsigned long long *>(s + kOffCounters + 64);
    uint32_t *status = reinterpret_cast<uint32_t *>(s + kOffStatus);
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    for (int p = 0; p < 4; ++p) {
        launch_onesweep_pass(stream, a, b, n, 32 + 8 * p, hist + 256 * p, status + (size_t)256 * tiles * p,
                             ctr + p, err, false, nullptr, nullptr, nullptr, nullptr);
        unsigned long long *t = a; a = b; b = t;
    }
    noalloc_split_kernel<<<grid, 256, 0, stream>>>(a, n, keys_out_dev, ids_out_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(MQR_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    unsigned long long herr = 0;
    e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return nfail(MQR_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    if (herr & kErrTimeout) return nfail(MQR_ERR_TIMEOUT, "a device-side wait exceeded its deadline");
    if (herr) return nfail(MQR_ERR_INTERNAL, "device index out of range in the sort");
    return MQR_OK;
}
