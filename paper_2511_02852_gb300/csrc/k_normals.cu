// Normals of a patch's blended maps by finite differences (Sec. 4.2: the
// normals are derived from the height maps by finite differences).  The
// paper gives no formula; with choppy displacement the surface is the
// displaced grid p(i, j) = (i c + Dx, j c + Dy, h) (c the cell size), and its
// normal is the normalised cross product of the two finite-difference
// tangents: central differences inside the patch, one-sided at its edges.
#include <cuda_runtime.h>

#include "internal.h"

namespace scwp {
namespace {

__global__ void __launch_bounds__(256) k_normals(const float* maps, int W, int H, float cell, float* dst) {
    const size_t plane = (size_t)W * H;
    const float* h = maps;
    const float* dx = maps + plane;
    const float* dy = maps + 2 * plane;
    for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < plane; o += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(o / W), i = (int)(o - (size_t)j * W);
        const int il = i > 0 ? i - 1 : i, ir = i < W - 1 ? i + 1 : i;
        const int jl = j > 0 ? j - 1 : j, jr = j < H - 1 ? j + 1 : j;
        const size_t a = (size_t)j * W + il, b = (size_t)j * W + ir;
        const size_t c = (size_t)jl * W + i, d = (size_t)jr * W + i;
        // tangents along i and j (each scaled by its own step count, which
        // does not change the normal's direction)
        float tx0 = (float)(ir - il) * cell + dx[b] - dx[a], tx1 = dy[b] - dy[a], tx2 = h[b] - h[a];
        float ty0 = dx[d] - dx[c], ty1 = (float)(jr - jl) * cell + dy[d] - dy[c], ty2 = h[d] - h[c];
        if (ir == il) { tx0 = cell; tx1 = tx2 = 0.f; }   // one-texel-wide patch
        if (jr == jl) { ty1 = cell; ty0 = ty2 = 0.f; }
        const float nx = tx1 * ty2 - tx2 * ty1;
        const float ny = tx2 * ty0 - tx0 * ty2;
        const float nz = tx0 * ty1 - tx1 * ty0;
        const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
        dst[o] = nx * inv;
        dst[plane + o] = ny * inv;
        dst[2 * plane + o] = nz * inv;
    }
}

}  // namespace

cudaError_t launch_normals(const float* maps, int W, int H, float cell, float* dst, cudaStream_t st) {
    const size_t n = (size_t)W * H;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_normals<<<blocks, 256, 0, st>>>(maps, W, H, cell, dst);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace scwp
