// Wave-particle synthesis of the hybrid ocean (sm_103a), Sec. 4.2:
// per-bucket accumulation of the particle kernels into the patch height map,
// displacement from the kernel gradient, and the distance-weighted blend into
// the FFT background.
//
// Tile gather.  One CTA owns a 64 x 64 texel tile and keeps its h, Dx, Dy
// sums in registers (4 x 4 texels per thread).  For each bucket it walks the
// integer bins that can reach the tile; the bump records of each bin row are
// contiguous in memory and are staged into shared memory with bulk async
// copies (cp.async.bulk, completion on an mbarrier), double-buffered so the
// copy of the next chunk overlaps the arithmetic of the current one.
//
// The bump kernel is separable, K = k(u) k(v), k(u) = 1/2 (1 + cos(pi u/R)),
// so for each staged bump the CTA evaluates k and sin once per tile column and
// once per tile row (shared memory), and each thread does the outer product:
//   h  += (A k(v)) * k(u)                 Dx += (A k(v)) * (lam/2) sin(pi u/R)
//   Dy += (A (lam/2) sin(pi v/R)) * k(u)
// i.e. 3 FMAs per bump-texel.  A warp skips bumps whose support misses its
// 16 x 32 sub-tile.  The epilogue applies the smoothstep blend weight and the
// bilinear background sample and writes the three maps (no atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scwp {
namespace {

constexpr int kT = 64;             // tile side (texels)
constexpr int kThreads = 256;
constexpr int kCH = 64;            // bumps per staged chunk
constexpr int kMaxRanges = 64;     // bin rows per bucket batch
constexpr int32_t kQi = 65536, kHalfi = 32768;
constexpr long long kSpinLimit = 1ll << 26;

struct SynthSmem {
    int4 rec[2][kCH];              // staged bump records (16-byte aligned)
    unsigned long long bar[2];     // mbarriers
    float kx[kCH][kT];             // k(u) per column
    float kd[kCH][kT];             // (lam/2) sin(pi u / R) per column
    float ay[kCH][kT];             // A k(v) per row
    float cy[kCH][kT];             // A (lam/2) sin(pi v / R) per row
    uint32_t mask[kCH];            // warps whose sub-tile the bump reaches
    int rstart[kMaxRanges];        // bin-row ranges of the current bucket batch
    int rlen[kMaxRanges];
    int cpre[kMaxRanges + 1];      // chunk prefix per range
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// bounded wait on an mbarrier phase; on timeout records the error and
// returns false (the caller abandons the tile).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity,
                                                  unsigned long long* err) {
    for (long long it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(err, (unsigned long long)kErrTimeout);
    return false;
}

__device__ __forceinline__ int span_lo(int32_t C, int32_t R) {
    return (int)((((int64_t)C - R - kHalfi) >> 16) + 1);
}
__device__ __forceinline__ int span_hi(int32_t C, int32_t R) {
    return (int)(((int64_t)C + R - kHalfi - 1) >> 16);
}

__global__ void __launch_bounds__(kThreads, 2) k_synth_gather(PatchDev p, SynthParams sp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SynthSmem& S = *reinterpret_cast<SynthSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = blockIdx.x * kT, ty0 = blockIdx.y * kT;
    const int tc = 8 * (warp & 1) + (lane & 7);     // column quad 0..15
    const int tr = 4 * (warp >> 1) + (lane >> 3);   // row quad 0..15

    float h[4][4], dx[4][4], dy[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) h[r][c] = dx[r][c] = dy[r][c] = 0.f;

    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    bool aborted = false;   // block-uniform (decided by __syncthreads_or)
    const int32_t Xlo = tx0 * kQi + kHalfi, Xhi = (tx0 + kT - 1) * kQi + kHalfi;
    const int32_t Ylo = ty0 * kQi + kHalfi, Yhi = (ty0 + kT - 1) * kQi + kHalfi;
    const float lamh = sp.lam_half;

    for (int bi = 0; bi < sp.nb && !aborted; ++bi) {
        const BucketDev bk = p.bk[bi];
        int bx_lo = (int)(((int64_t)Xlo) / bk.C);
        int bx_hi = (int)(((int64_t)Xhi + 2 * (int64_t)bk.R - 1) / bk.C);
        int by_lo = (int)(((int64_t)Ylo) / bk.C);
        int by_hi = (int)(((int64_t)Yhi + 2 * (int64_t)bk.R - 1) / bk.C);
        if (bx_lo < 0) bx_lo = 0;
        if (by_lo < 0) by_lo = 0;
        if (bx_hi > bk.nbx - 1) bx_hi = bk.nbx - 1;
        if (by_hi > bk.nby - 1) by_hi = bk.nby - 1;
        if (bx_lo > bx_hi || by_lo > by_hi) continue;
        const float invR = bk.invR;
        for (int byb = by_lo; byb <= by_hi && !aborted; byb += kMaxRanges) {
            const int nr = min(kMaxRanges, by_hi - byb + 1);
            for (int k = tid; k < nr; k += kThreads) {
                const int key0 = bk.base + (byb + k) * bk.nbx;
                const int s = (int)p.offsets[key0 + bx_lo];
                const int e = (int)p.offsets[key0 + bx_hi + 1];
                S.rstart[k] = s;
                S.rlen[k] = e - s;
            }
            __syncthreads();
            if (tid == 0) {
                int acc = 0;
                for (int k = 0; k < nr; ++k) {
                    S.cpre[k] = acc;
                    acc += (S.rlen[k] + kCH - 1) / kCH;
                }
                S.cpre[nr] = acc;
            }
            __syncthreads();
            const int nchunks = S.cpre[nr];
            if (nchunks == 0) continue;
            // chunk c -> (source offset, count), computable by any thread
            auto chunk = [&](int c, int& off, int& n) {
                int k = 0;
                while (S.cpre[k + 1] <= c) ++k;
                off = S.rstart[k] + (c - S.cpre[k]) * kCH;
                n = min(kCH, S.rstart[k] + S.rlen[k] - off);
            };
            if (tid == 0) {
                int off, n;
                chunk(0, off, n);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_expect(&S.bar[0], (uint32_t)n * 16u);
                bulk_g2s(&S.rec[0][0], p.rec + off, (uint32_t)n * 16u, &S.bar[0]);
            }
            for (int c = 0; c < nchunks; ++c) {
                const int slot = c & 1;
                int off, n;
                chunk(c, off, n);
                const bool late = !mbar_wait_bounded(&S.bar[slot], parity[slot], p.stats + 2);
                parity[slot] ^= 1u;
                if (__syncthreads_or(late)) {
                    aborted = true;
                    break;
                }
                if (tid == 0 && c + 1 < nchunks) {
                    int off2, n2;
                    chunk(c + 1, off2, n2);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive_expect(&S.bar[slot ^ 1], (uint32_t)n2 * 16u);
                    bulk_g2s(&S.rec[slot ^ 1][0], p.rec + off2, (uint32_t)n2 * 16u, &S.bar[slot ^ 1]);
                }
                // per-bump axis factors for this tile
                for (int it = tid; it < n * 2 * kT; it += kThreads) {
                    const int b = it / (2 * kT), a = it - b * (2 * kT);
                    const int4 rc = S.rec[slot][b];
                    if (a < kT) {
                        const int32_t u = (tx0 + a) * kQi + kHalfi - rc.x;
                        float kv = 0.f, dv = 0.f;
                        if (u > -bk.R && u < bk.R) {
                            float sn, cs;
                            sincospif((float)u * invR, &sn, &cs);
                            kv = 0.5f + 0.5f * cs;
                            dv = lamh * sn;
                        }
                        S.kx[b][a] = kv;
                        S.kd[b][a] = dv;
                    } else {
                        const int rr = a - kT;
                        const int32_t v = (ty0 + rr) * kQi + kHalfi - rc.y;
                        float av = 0.f, cv = 0.f;
                        if (v > -bk.R && v < bk.R) {
                            float sn, cs;
                            sincospif((float)v * invR, &sn, &cs);
                            const float A = __int_as_float(rc.z);
                            av = A * (0.5f + 0.5f * cs);
                            cv = A * lamh * sn;
                        }
                        S.ay[b][rr] = av;
                        S.cy[b][rr] = cv;
                    }
                }
                if (tid < n) {
                    const int4 rc = S.rec[slot][tid];
                    const int xl = span_lo(rc.x, bk.R) - tx0, xh = span_hi(rc.x, bk.R) - tx0;
                    const int yl = span_lo(rc.y, bk.R) - ty0, yh = span_hi(rc.y, bk.R) - ty0;
                    uint32_t m = 0;
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        const int c0 = 32 * (w & 1), r0 = 16 * (w >> 1);
                        if (xl <= c0 + 31 && xh >= c0 && yl <= r0 + 15 && yh >= r0) m |= 1u << w;
                    }
                    S.mask[tid] = m;
                }
                __syncthreads();
                for (int b = 0; b < n; ++b) {
                    if (!((S.mask[b] >> warp) & 1u)) continue;
                    const float4 kx4 = *reinterpret_cast<const float4*>(&S.kx[b][4 * tc]);
                    const float4 kd4 = *reinterpret_cast<const float4*>(&S.kd[b][4 * tc]);
                    const float4 ay4 = *reinterpret_cast<const float4*>(&S.ay[b][4 * tr]);
                    const float4 cy4 = *reinterpret_cast<const float4*>(&S.cy[b][4 * tr]);
                    const float kxv[4] = {kx4.x, kx4.y, kx4.z, kx4.w};
                    const float kdv[4] = {kd4.x, kd4.y, kd4.z, kd4.w};
                    const float ayv[4] = {ay4.x, ay4.y, ay4.z, ay4.w};
                    const float cyv[4] = {cy4.x, cy4.y, cy4.z, cy4.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            h[r][cc] = fmaf(ayv[r], kxv[cc], h[r][cc]);
                            dx[r][cc] = fmaf(ayv[r], kdv[cc], dx[r][cc]);
                            dy[r][cc] = fmaf(cyv[r], kxv[cc], dy[r][cc]);
                        }
                }
                __syncthreads();
            }
        }
    }

    // ---- epilogue: blend with the background, store -----------------------------
    const size_t plane = (size_t)sp.W * sp.H;
    const size_t nplane = (size_t)sp.N * sp.N;
    const int N = sp.N;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int iy = ty0 + 4 * tr + r;
        if (iy >= sp.H) continue;
        float o[3][4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int ix = tx0 + 4 * tc + cc;
            const float d = fminf(fminf((float)ix + 0.5f, (float)sp.W - (float)ix - 0.5f),
                                  fminf((float)iy + 0.5f, (float)sp.H - (float)iy - 0.5f));
            const float t = fminf(fmaxf(d / sp.band, 0.f), 1.f);
            const float w = t * t * (3.f - 2.f * t);
            float bh = 0.f, bx = 0.f, byv = 0.f;
            if (w < 1.f) {
                const float fx = sp.fx0 + (float)ix * sp.fsx;
                const float fy = sp.fy0 + (float)iy * sp.fsx;
                const float flx = floorf(fx), fly = floorf(fy);
                const float a = fx - flx, bb = fy - fly;
                int x0 = (int)flx % N, y0 = (int)fly % N;
                if (x0 < 0) x0 += N;
                if (y0 < 0) y0 += N;
                const int x1 = (x0 + 1) % N, y1 = (y0 + 1) % N;
                const float w00 = (1.f - a) * (1.f - bb), w01 = a * (1.f - bb);
                const float w10 = (1.f - a) * bb, w11 = a * bb;
                const size_t i00 = (size_t)y0 * N + x0, i01 = (size_t)y0 * N + x1;
                const size_t i10 = (size_t)y1 * N + x0, i11 = (size_t)y1 * N + x1;
                bh = w00 * sp.bg[i00] + w01 * sp.bg[i01] + w10 * sp.bg[i10] + w11 * sp.bg[i11];
                const float* g1 = sp.bg + nplane;
                bx = w00 * g1[i00] + w01 * g1[i01] + w10 * g1[i10] + w11 * g1[i11];
                const float* g2 = sp.bg + 2 * nplane;
                byv = w00 * g2[i00] + w01 * g2[i01] + w10 * g2[i10] + w11 * g2[i11];
            }
            o[0][cc] = w * h[r][cc] + (1.f - w) * bh;
            o[1][cc] = w * dx[r][cc] + (1.f - w) * bx;
            o[2][cc] = w * dy[r][cc] + (1.f - w) * byv;
        }
        const int ix0 = tx0 + 4 * tc;
        const size_t rowo = (size_t)iy * sp.W;
        if ((sp.W & 3) == 0 && ix0 + 3 < sp.W) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
                *reinterpret_cast<float4*>(p.out + f * plane + rowo + ix0) =
                    make_float4(o[f][0], o[f][1], o[f][2], o[f][3]);
        } else {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                if (ix0 + cc < sp.W)
#pragma unroll
                    for (int f = 0; f < 3; ++f) p.out[f * plane + rowo + ix0 + cc] = o[f][cc];
        }
    }
}

}  // namespace

cudaError_t launch_synth_gather(const PatchDev& p, const SynthParams& sp, cudaStream_t st) {
    const size_t sm = sizeof(SynthSmem);
    cudaError_t e = cudaFuncSetAttribute(k_synth_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((p.W + kT - 1) / kT, (p.H + kT - 1) / kT);
    k_synth_gather<<<grid, kThreads, sm, st>>>(p, sp);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace scwp
