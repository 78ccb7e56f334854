// scwp_background_noalloc: the background FFT step (spectrum update + inverse
// 2-D FFT) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a host
// callback or a real-time render/audio thread where an allocation would
// synchronise the device, runtimes that hand out only pre-registered
// buffers, or plug-ins whose host application owns every allocation.  This
// entry point lets them evolve and transform a background spectrum they
// already hold in device memory.  Its scratch (the row-pass intermediate and
// the twiddle tables) lives in one file-scope __device__ array below, sized
// for grids up to kNoAllocMaxN x kNoAllocMaxN; every GPU that loads this
// library holds that array (3 x 257 x 512 + 512 complex floats, about
// 3.0 MiB) until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "../../include/scwp.h"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxN = 512;
constexpr size_t kInterElems = 3 * (size_t)(kNoAllocMaxN / 2 + 1) * kNoAllocMaxN;
constexpr size_t kScratchElems = kInterElems + kNoAllocMaxN;

// [0, kInterElems): row-pass output (H1, Dx1, Dy1 of the rows k_y <= N/2);
// [kInterElems, kScratchElems): the twiddle tables of every grid N = 8 ..
// kNoAllocMaxN, one after another (tw_offset(N)); together they take 480 of
// the kNoAllocMaxN entries.
static __device__ __align__(256) float2 g_noalloc_scratch[kScratchElems];

// offset of grid N's twiddle table in the twiddle area
size_t tw_offset(int n) {
    size_t o = 0;
    for (int m = 8; m < n; m *= 2) o += scwp::background_twiddle_elems(m);
    return o;
}

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
float2* g_scratch_ptr[kMaxDevices] = {};

// One-time set-up per device (the caller's current device): look up the
// array's device address and fill the twiddle tables.  Runs on the first
// call on that device; the copy below is a synchronous cudaMemcpy, so that
// first call must not happen inside a stream capture.
cudaError_t setup_device(int dev, float2** out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_ptr[dev]) {
        *out = g_scratch_ptr[dev];
        return cudaSuccess;
    }
    float2* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (tw_offset(2 * kNoAllocMaxN) > (size_t)kNoAllocMaxN) return cudaErrorInvalidValue;   // the tables fit
    static float2 tw[kNoAllocMaxN];   // host staging, no heap allocation
    for (int n = 8; n <= kNoAllocMaxN; n *= 2) scwp::build_background_twiddles(n, tw + tw_offset(n));
    e = cudaMemcpy(ptr + kInterElems, tw, kNoAllocMaxN * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = ptr;
    *out = ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" scwp_status scwp_background_noalloc(const float* h0, const float* omega, int32_t n,
                                               double fft_L, double choppiness, double t, float* out,
                                               void* stream) {
    if (!h0 || !omega || !out || !(fft_L > 0)) return SCWP_E_INVALID;
    if (n < 8 || n > kNoAllocMaxN || (n & (n - 1)) != 0) return SCWP_E_INVALID;
    // h0 and omega are read as 8-byte float pairs: an address off that
    // alignment would fault the kernel, so it is refused here
    if ((((uintptr_t)h0 | (uintptr_t)omega) & 7u) != 0 || ((uintptr_t)out & 3u) != 0) return SCWP_E_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SCWP_E_CUDA;
    }
    float2* scratch = nullptr;
    if (setup_device(dev, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return SCWP_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const float2* tw = scratch + kInterElems + tw_offset(n);
    scwp::BgDev bg;
    bg.N = n;
    bg.h0 = reinterpret_cast<const float2*>(h0);
    bg.omega = reinterpret_cast<const float2*>(omega);
    bg.tw = tw;
    bg.I = scratch;
    bg.out = out;
    bg.lam = (float)choppiness;
    bg.dk = (float)(2.0 * M_PI / fft_L);
    if (scwp::launch_background(bg, t, st) != cudaSuccess) return SCWP_E_CUDA;
    return SCWP_OK;
}
