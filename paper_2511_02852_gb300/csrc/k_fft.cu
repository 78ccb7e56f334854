// FFT background of the hybrid ocean (sm_103a): spectrum update fused with
// the row pass of a shared-memory Stockham inverse FFT, then the column pass.
// (Sec. 3.1 / Sec. 4.1: the conventional spectral evolution and inverse FFT.)
//
//   h~(k,t) = h0(k) e^{i w t} + conj(h0(-k)) e^{-i w t}
//   D~(k,t) = -i lambda_c (k/|k|) h~(k,t)
//   h(x) + i Dx(x) = IFFT2(h~ + i D~x),   Dy(x) = IFFT2(D~y)     (both real)
//
// The inverse transform is unnormalised: f[j] = sum_m F[m] e^{+2 pi i m j / N}.
// Stockham autosort, radix 4 (one radix-2 stage when log2 N is odd), batched
// transforms interleaved in shared memory (element (t, m) at m*T + t) so that
// consecutive threads touch consecutive words.  Twiddles come from a float
// table of e^{2 pi i m / N} computed in float64 on the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scwp {
namespace {

constexpr int kThreads = 512;    // upper bound of a launch's block

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }  // i a

// Inverse FFT of T interleaved length-N transforms in shared memory.
// Returns the buffer holding the result (a or b).
__device__ float2* fft_inverse_smem(float2* a, float2* b, int N, int T, const float2* tw) {
    float2* src = a;
    float2* dst = b;
    for (int Ns = 1; Ns < N;) {
        const int R = (N / Ns >= 4) ? 4 : 2;
        const int nbf = N / R;
        const int step = N / (Ns * R);
        for (int w = threadIdx.x; w < nbf * T; w += blockDim.x) {
            const int t = w % T, j = w / T;
            const int k = j & (Ns - 1);
            const int idxD = (j - k) * R + k;
            if (R == 4) {
                float2 v0 = src[(j) * T + t];
                float2 v1 = cmul(src[(j + nbf) * T + t], tw[(1 * k * step) & (N - 1)]);
                float2 v2 = cmul(src[(j + 2 * nbf) * T + t], tw[(2 * k * step) & (N - 1)]);
                float2 v3 = cmul(src[(j + 3 * nbf) * T + t], tw[(3 * k * step) & (N - 1)]);
                const float2 a0 = cadd(v0, v2), a1 = csub(v0, v2);
                const float2 a2 = cadd(v1, v3), a3 = cmuli(csub(v1, v3));
                dst[(idxD) * T + t] = cadd(a0, a2);
                dst[(idxD + Ns) * T + t] = cadd(a1, a3);
                dst[(idxD + 2 * Ns) * T + t] = csub(a0, a2);
                dst[(idxD + 3 * Ns) * T + t] = csub(a1, a3);
            } else {
                const float2 v0 = src[(j) * T + t];
                const float2 v1 = cmul(src[(j + nbf) * T + t], tw[(k * step) & (N - 1)]);
                dst[(idxD) * T + t] = cadd(v0, v1);
                dst[(idxD + Ns) * T + t] = csub(v0, v1);
            }
        }
        __syncthreads();
        float2* tmp = src;
        src = dst;
        dst = tmp;
        Ns *= R;
    }
    return src;
}

// Rows pass: spectrum update (a1) + inverse FFT along x of h~ + i D~x and D~y.
// One CTA handles `rpc` consecutive rows (2 rpc interleaved transforms).
__global__ void __launch_bounds__(kThreads) k_spectrum_rows(BgDev bg, double t_arg, const double* t_dev, int rpc) {
    const double t = t_dev ? *t_dev : t_arg;
    extern __shared__ float2 sm[];
    const int N = bg.N;
    const int T = 2 * rpc;
    float2* tw = sm;
    float2* a = sm + N;
    float2* b = a + (size_t)N * T;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = bg.tw[i];
    const int row0 = blockIdx.x * rpc;
    const double two_pi = 6.283185307179586476925286766559;
    for (int w = threadIdx.x; w < N * rpc; w += blockDim.x) {
        const int r = w / N, mx = w - r * N;
        const int my = row0 + r;
        const int nx = mx < N / 2 ? mx : mx - N;
        const int ny = my < N / 2 ? my : my - N;
        const size_t idx = (size_t)my * N + mx;
        const size_t idm = (size_t)((N - my) & (N - 1)) * N + ((N - mx) & (N - 1));
        const float2 h0a = bg.h0[idx], h0b = bg.h0[idm];
        double ph = bg.omega[idx] * t;
        ph -= two_pi * rint(ph * (1.0 / two_pi));
        float s, c;
        sincosf((float)ph, &s, &c);
        // q = h0(-k) e^{i w t};  h~ = h0(k) e^{i w t} + conj(q)
        const float2 q = make_float2(h0b.x * c - h0b.y * s, h0b.x * s + h0b.y * c);
        const float2 ht = make_float2(h0a.x * c - h0a.y * s + q.x, h0a.x * s + h0a.y * c - q.y);
        const float kx = bg.dk * (float)nx, ky = bg.dk * (float)ny;
        const float kk = sqrtf(kx * kx + ky * ky);
        float ux = 0.f, uy = 0.f;
        if (kk > 0.f) {
            ux = kx / kk;
            uy = ky / kk;
        }
        // -i h~ = (h~.y, -h~.x)
        const float2 mi = make_float2(ht.y, -ht.x);
        const float2 dxt = make_float2(bg.lam * ux * mi.x, bg.lam * ux * mi.y);
        const float2 dyt = make_float2(bg.lam * uy * mi.x, bg.lam * uy * mi.y);
        a[(size_t)mx * T + 2 * r] = make_float2(ht.x - dxt.y, ht.y + dxt.x);  // h~ + i D~x
        a[(size_t)mx * T + 2 * r + 1] = dyt;
    }
    __syncthreads();
    const float2* res = fft_inverse_smem(a, b, N, T, tw);
    const size_t plane = (size_t)N * N;
    for (int w = threadIdx.x; w < N * T; w += blockDim.x) {
        const int tt = w / N, jx = w - tt * N;
        const int r = tt >> 1, p = tt & 1;
        bg.G[p * plane + (size_t)(row0 + r) * N + jx] = res[(size_t)jx * T + tt];
    }
}

// Columns pass: inverse FFT along y of `cw` columns of plane blockIdx.y per
// CTA; writes h = Re, Dx = Im (plane 0) and Dy = Re (plane 1).
__global__ void __launch_bounds__(kThreads) k_fft_cols(BgDev bg, int cw) {
    extern __shared__ float2 sm[];
    const int N = bg.N;
    float2* tw = sm;
    float2* a = sm + N;
    float2* b = a + (size_t)N * cw;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = bg.tw[i];
    const int c0 = blockIdx.x * cw, p = blockIdx.y;
    const size_t plane = (size_t)N * N;
    for (int w = threadIdx.x; w < N * cw; w += blockDim.x) {
        const int m = w / cw, c = w - m * cw;
        a[w] = bg.G[p * plane + (size_t)m * N + c0 + c];
    }
    __syncthreads();
    const float2* res = fft_inverse_smem(a, b, N, cw, tw);
    for (int w = threadIdx.x; w < N * cw; w += blockDim.x) {
        const int jy = w / cw, c = w - jy * cw;
        const float2 v = res[w];
        const size_t o = (size_t)jy * N + c0 + c;
        if (p == 0) {
            bg.out[o] = v.x;
            bg.out[plane + o] = v.y;
        } else {
            bg.out[2 * plane + o] = v.x;
        }
    }
}

}  // namespace

cudaError_t launch_background(const BgDev& bg, double t, cudaStream_t st, const double* t_dev) {
    const int N = bg.N;
    int rpc = N >= 512 ? 1 : 512 / N;
    if (rpc > N) rpc = N;
    const size_t smr = sizeof(float2) * ((size_t)N + 2 * (size_t)N * 2 * rpc);
    cudaError_t e = cudaFuncSetAttribute(k_spectrum_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smr);
    if (e != cudaSuccess) return e;
    // 512 threads from N = 512 up (more warps to hide the shared-memory
    // stages; measured best against 256 and 1024), 256 below
    const int threads = N >= 512 ? 512 : 256;
    k_spectrum_rows<<<N / rpc, threads, smr, st>>>(bg, t, t_dev, rpc);
    // enough column groups to fill the SMs (both planes: 2 N / cw CTAs), at
    // least 4 columns (one 32-byte sector of each row) where shared memory
    // (twiddles + two buffers of N x cw) still leaves two CTAs per SM
    int cw = 2048 / N;
    if (cw > 16) cw = 16;
    if (cw < 4) cw = 4;
    while (cw > 1 && sizeof(float2) * ((size_t)N + 2 * (size_t)N * cw) > 110 * 1024) cw >>= 1;   // two CTAs per SM
    if (cw > N) cw = N;
    const size_t smc = sizeof(float2) * ((size_t)N + 2 * (size_t)N * cw);
    e = cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
    if (e != cudaSuccess) return e;
    k_fft_cols<<<dim3(N / cw, 2), threads, smc, st>>>(bg, cw);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace scwp
