// Blend of one synthesised texel into the background (Sec. 4.2 last
// step, reading O15: smoothstep weight over the band, bilinear periodic
// background sample), shared by the synthesis kernels that blend in their
// epilogue.
#pragma once
#include "internal.h"

namespace scwp {

// blend weight at (ix, iy) and the bilinear background sample of one field
__device__ __forceinline__ float blend1(const SynthParams& sp, int ix, int iy, int f, float wp) {
    const float d = fminf(fminf((float)ix + 0.5f, (float)sp.W - (float)ix - 0.5f),
                          fminf((float)iy + 0.5f, (float)sp.H - (float)iy - 0.5f));
    const float t = fminf(fmaxf(d / sp.band, 0.f), 1.f);
    const float w = t * t * (3.f - 2.f * t);
    if (w >= 1.f) return wp;
    const int N = sp.N;
    const float fx = sp.fx0 + (float)ix * sp.fsx, fy = sp.fy0 + (float)iy * sp.fsx;
    const float flx = floorf(fx), fly = floorf(fy);
    const float a = fx - flx, b = fy - fly;
    int x0 = (int)flx % N, y0 = (int)fly % N;
    if (x0 < 0) x0 += N;
    if (y0 < 0) y0 += N;
    const int x1 = (x0 + 1) % N, y1 = (y0 + 1) % N;
    const float* g = sp.bg + (size_t)f * N * N;
    const float bg = (1.f - a) * (1.f - b) * g[(size_t)y0 * N + x0] + a * (1.f - b) * g[(size_t)y0 * N + x1] +
                     (1.f - a) * b * g[(size_t)y1 * N + x0] + a * b * g[(size_t)y1 * N + x1];
    return w * wp + (1.f - w) * bg;
}

}  // namespace scwp
