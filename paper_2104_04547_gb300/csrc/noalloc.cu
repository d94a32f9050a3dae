// CNN dense layer with a fixed, library-owned scratch area: an entry point
// that allocates no memory of any kind.
//
// Who needs it: a caller that runs under a device-memory budget it does not
// own (for example a serving process that admits work against a fixed HBM
// budget, or a host application whose allocator owns all device memory), or a
// caller in a latency-bound request loop that cannot afford the implicit
// device synchronisation and unbounded latency that cudaMalloc / cudaFree may
// bring.  Such a caller provides its inputs and outputs and gets the same
// result as the split-K dense layer of fusion_score, with the split partials
// kept in the static array below instead of a model workspace.
//
// The scratch array lives in every GPU that loads this library, for the
// lifetime of the process (8 MiB).  Host code cannot use the array's name as a
// device address, so the address is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current; that
// first call should therefore come before any stream capture.  The looked-up
// address is kept for the life of the process: it does not survive a
// cudaDeviceReset of that device, after which this entry point must not be
// called again in the same process.  All calls share
// the one array: calls whose kernels overlap on the GPU (different streams, or
// different host threads on one device) race on it and must be serialised by
// the caller.  Nothing in the array needs to start at zero: every partial the
// reduction reads is written earlier in the same call.
#include "fusion_internal.cuh"

#include <cstdint>
#include <mutex>
#include <string>

#define FUSION_NOALLOC_MAX_DEVICES 64

// splits x B x N partial sums, FUSION_NOALLOC_MAX_PARTIALS floats (8 MiB)
static __device__ __align__(256) float g_dense_scratch[FUSION_NOALLOC_MAX_PARTIALS];

namespace {

std::mutex g_noalloc_mu;
void *g_scratch_addr[FUSION_NOALLOC_MAX_DEVICES] = {};

int noalloc_fail(int code, const std::string &m) { return fusion::set_last_error(code, m.c_str()); }

}  // namespace

extern "C" int fusion_cnn_dense_noalloc(const float *x, const float *w, const float *bias, int32_t B, int32_t N,
                                        int32_t K, int32_t relu, float *y, void *cuda_stream) {
    if (!x || !w || !bias || !y) return noalloc_fail(FUSION_EINVAL, "NULL pointer argument");
    // x and w are read 16 bytes at a time (rows of K floats, K a multiple of 8, stay aligned), bias and y
    // one float at a time: an offset view would make the kernel fault and lose the caller's context
    if (((uintptr_t)x | (uintptr_t)w) & 15u)
        return noalloc_fail(FUSION_EINVAL, "x and w must be 16-byte aligned");
    if (((uintptr_t)bias | (uintptr_t)y) & 3u)
        return noalloc_fail(FUSION_EINVAL, "bias and y must be 4-byte aligned");
    if (B < 1 || N < 1 || K < 8 || K % 8 != 0)
        return noalloc_fail(FUSION_EINVAL, "need B >= 1, N >= 1 and K a positive multiple of 8");
    const int splits = fusion::dense_splits(K);
    const long long need = (long long)splits * B * N;
    if (need > FUSION_NOALLOC_MAX_PARTIALS)
        return noalloc_fail(FUSION_EINVAL, "splits x B x N = " + std::to_string(need) +
                                               " partials exceed the fixed scratch of " +
                                               std::to_string(FUSION_NOALLOC_MAX_PARTIALS) + " floats");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(FUSION_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= FUSION_NOALLOC_MAX_DEVICES) return noalloc_fail(FUSION_EINVAL, "device index too large");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_dense_scratch);
            if (e != cudaSuccess)
                return noalloc_fail(FUSION_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    // an error left pending by earlier work would otherwise be reported below as this call's launch failure
    e = cudaPeekAtLastError();
    if (e != cudaSuccess)
        return noalloc_fail(FUSION_ECUDA, std::string("a CUDA error was pending before this call (nothing launched): ") +
                                              cudaGetErrorString(e));
    fusion::DenseArgs a{x, w, bias, static_cast<float *>(scratch), y, B, N, K, splits, 0, relu ? 1 : 0};
    fusion::launch_dense(a, static_cast<cudaStream_t>(cuda_stream));
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FUSION_ECUDA, std::string("dense launch: ") + cudaGetErrorString(e));
    return FUSION_OK;
}
