// Layered-texture synthesis variant of the hybrid ocean (sm_103a), the
// paper's own description of the WP accumulation (Sec. 4.2): particles
// accumulate into one layer texture per frequency bucket, each layer is
// smoothed by two separable passes along x and y, and the layers are summed.
//
// Per bucket i (bucket after bucket, into one float accumulator, so the sum
// order is fixed):
//   splat   each binned bump's signed amplitude is deposited bilinearly at
//           texel resolution (position (X - Q/2)/Q) into a layer that extends
//           the patch by K + 2 texels, K = floor((R_i - 1)/Q); deposits are
//           int64 fixed point (2^-32 m), so the integer atomics make the
//           layer exact and independent of the deposit order;
//   x pass  Lx = L * k, Ls = L * (lam/2) s along x for every layer row
//           (k(n) = 1/2(1 + cos(pi n Q/R)), s(n) = sin(pi n Q/R), |n| <= K);
//   y pass  h += Lx * k, Dx += Ls * k, Dy += Lx * (lam/2) s along y.
// Then the blend epilogue of the gather path.  Bumps exactly at texel
// centres give exactly the gather result; elsewhere the bilinear splat is a
// second-order approximation of it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scwp {
namespace {

constexpr int32_t kQi = 65536, kHalfi = 32768;
constexpr double kFix = 4294967296.0;   // 2^32 fixed-point units per metre

struct LayerGeom {
    int K;          // taps on each side
    int M;          // layer margin (K + 2)
    int Lw, Lh;     // layer size
    int32_t R;
    float lamh;
};

__global__ void k_layer_splat(const BumpRec* rec, const uint32_t* offsets, int key0, int key1,
                              unsigned long long* layer, LayerGeom g) {
    const int e0 = (int)offsets[key0], e1 = (int)offsets[key1];
    for (int e = e0 + blockIdx.x * blockDim.x + threadIdx.x; e < e1; e += gridDim.x * blockDim.x) {
        const BumpRec r = rec[e];
        const int64_t px = (int64_t)r.x - kHalfi, py = (int64_t)r.y - kHalfi;
        const int x0 = (int)(px >> 16), y0 = (int)(py >> 16);
        const double fx = (double)(px & 0xFFFF) * (1.0 / 65536.0);
        const double fy = (double)(py & 0xFFFF) * (1.0 / 65536.0);
        const double a = (double)r.amp;
        const double w[4] = {(1.0 - fx) * (1.0 - fy), fx * (1.0 - fy), (1.0 - fx) * fy, fx * fy};
        const int ox[4] = {0, 1, 0, 1}, oy[4] = {0, 0, 1, 1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int gx = x0 + ox[k] + g.M, gy = y0 + oy[k] + g.M;
            if (gx < 0 || gx >= g.Lw || gy < 0 || gy >= g.Lh) continue;
            const long long v = __double2ll_rn(a * w[k] * kFix);
            if (v) atomicAdd(&layer[(size_t)gy * g.Lw + gx], (unsigned long long)v);
        }
    }
}

// x pass over every layer row; output columns are the patch's 0..W-1
__global__ void __launch_bounds__(256) k_layer_xpass(const unsigned long long* layer, float* Lx, float* Ls,
                                                     int W, LayerGeom g) {
    extern __shared__ float sm[];
    const int K = g.K, T = 2 * K + 1;
    float* tk = sm;            // k(n), n = -K..K
    float* ts = sm + T;        // (lam/2) s(n)
    float* seg = sm + 2 * T;   // 256 + 2K layer values
    for (int j = threadIdx.x; j < T; j += blockDim.x) {
        const int n = j - K;
        float s, c;
        sincospif((float)((double)n * kQi / (double)g.R), &s, &c);
        tk[j] = 0.5f + 0.5f * c;
        ts[j] = g.lamh * s;
    }
    const int row = blockIdx.y;
    const int x0 = blockIdx.x * 256;
    // layer column of patch column x is x + M; need layer columns x0 - K + M ..
    for (int j = threadIdx.x; j < 256 + 2 * K; j += blockDim.x) {
        const int lc = x0 - K + g.M + j;
        float v = 0.f;
        if (lc >= 0 && lc < g.Lw) v = (float)(long long)layer[(size_t)row * g.Lw + lc] * (float)(1.0 / kFix);
        seg[j] = v;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= W) return;
    // out(x) = sum_n L(x - n) t(n): seg index of x - n is threadIdx.x + K - n
    float a = 0.f, b = 0.f;
    for (int j = 0; j < T; ++j) {
        const float v = seg[threadIdx.x + 2 * K - j];   // n = j - K
        a = fmaf(v, tk[j], a);
        b = fmaf(v, ts[j], b);
    }
    Lx[(size_t)row * W + x] = a;
    Ls[(size_t)row * W + x] = b;
}

// y pass: 8 output rows of one column per thread, accumulated into acc
__global__ void __launch_bounds__(256) k_layer_ypass(const float* Lx, const float* Ls, float* acc, int W,
                                                     int H, LayerGeom g) {
    extern __shared__ float sm[];
    const int K = g.K, T = 2 * K + 1;
    float* tk = sm;
    float* ts = sm + T;
    for (int j = threadIdx.x; j < T; j += blockDim.x) {
        const int n = j - K;
        float s, c;
        sincospif((float)((double)n * kQi / (double)g.R), &s, &c);
        tk[j] = 0.5f + 0.5f * c;
        ts[j] = g.lamh * s;
    }
    __syncthreads();
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y0 = (blockIdx.y * 8 + (threadIdx.x >> 5)) * 8;
    if (x >= W || y0 >= H) return;
    float oh[8], ox[8], oy[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) oh[r] = ox[r] = oy[r] = 0.f;
    // output row y0 + r takes layer row (y0 + r - n) + M, |n| <= K; rows
    // past the patch's last row are not needed
    const int s_end = min(K + 8, (H - y0) + K);
    for (int s = -K; s < s_end; ++s) {
        const int lr = y0 + s + g.M;
        const float vx = Lx[(size_t)lr * W + x];
        const float vs = Ls[(size_t)lr * W + x];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int n = r - s;       // tap index n = (y0 + r) - (y0 + s)
            if (n >= -K && n <= K) {
                oh[r] = fmaf(vx, tk[n + K], oh[r]);
                ox[r] = fmaf(vs, tk[n + K], ox[r]);
                oy[r] = fmaf(vx, ts[n + K], oy[r]);
            }
        }
    }
    const size_t plane = (size_t)W * H;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int y = y0 + r;
        if (y >= H) break;
        const size_t o = (size_t)y * W + x;
        acc[o] += oh[r];
        acc[plane + o] += ox[r];
        acc[2 * plane + o] += oy[r];
    }
}

// the float accumulator [3][H][W], rounded up so the int64 layer after it
// stays 256-byte aligned
size_t acc_bytes(const PatchDev& p) { return ((size_t)3 * p.W * p.H * 4 + 255) & ~(size_t)255; }

}  // namespace

size_t layered_scratch_bytes(const PatchDev& p, const int32_t* R_host) {
    size_t best = 0;
    for (int i = 0; i < p.nb; ++i) {
        const int K = (int)((R_host[i] - 1) >> 16), M = K + 2;
        const size_t Lw = (size_t)p.W + 2 * M, Lh = (size_t)p.H + 2 * M;
        const size_t b = Lw * Lh * 8 + 2 * Lh * (size_t)p.W * 4;
        if (b > best) best = b;
    }
    return best + acc_bytes(p);
}

cudaError_t launch_layered(const PatchDev& p, const SynthParams& sp, const int32_t* R_host,
                           const int* base_host, const int* nbins_host, cudaStream_t st) {
    const size_t plane = (size_t)p.W * p.H;
    float* acc = p.layers;
    unsigned char* scratch = reinterpret_cast<unsigned char*>(p.layers) + acc_bytes(p);
    cudaError_t e = cudaMemsetAsync(acc, 0, 3 * plane * sizeof(float), st);
    if (e != cudaSuccess) return e;
    int launches = 0;
    for (int i = 0; i < p.nb; ++i) {
        LayerGeom g;
        g.R = R_host[i];
        g.K = (int)((g.R - 1) >> 16);
        g.M = g.K + 2;
        g.Lw = p.W + 2 * g.M;
        g.Lh = p.H + 2 * g.M;
        g.lamh = sp.lam_half;
        unsigned long long* layer = reinterpret_cast<unsigned long long*>(scratch);
        float* Lx = reinterpret_cast<float*>(scratch + (size_t)g.Lw * g.Lh * 8);
        float* Ls = Lx + (size_t)g.Lh * p.W;
        e = cudaMemsetAsync(layer, 0, (size_t)g.Lw * g.Lh * 8, st);
        if (e != cudaSuccess) return e;
        k_layer_splat<<<152 * 4, 256, 0, st>>>(p.rec, p.offsets, base_host[i], base_host[i] + nbins_host[i],
                                                layer, g);
        const int T = 2 * g.K + 1;
        const size_t smx = (size_t)(2 * T + 256 + 2 * g.K) * sizeof(float);
        e = cudaFuncSetAttribute(k_layer_xpass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx);
        if (e != cudaSuccess) return e;
        k_layer_xpass<<<dim3((p.W + 255) / 256, g.Lh), 256, smx, st>>>(layer, Lx, Ls, p.W, g);
        const size_t smy = (size_t)2 * T * sizeof(float);
        e = cudaFuncSetAttribute(k_layer_ypass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smy);
        if (e != cudaSuccess) return e;
        k_layer_ypass<<<dim3((p.W + 31) / 32, (p.H + 63) / 64), 256, smy, st>>>(Lx, Ls, acc, p.W, p.H, g);
        launches += 3;
    }
    count_launches(launches);
    return launch_blend(p, sp, acc, 1, st);
}

}  // namespace scwp
