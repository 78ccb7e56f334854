// Wave-particle synthesis of the hybrid ocean (sm_103a), Sec. 4.2:
// per-bucket accumulation of the particle kernels into the patch height map,
// displacement from the kernel gradient, and the distance-weighted blend into
// the FFT background.
//
// Tile gather.  One CTA (4 warps) owns a 64 x 64 texel tile and keeps its
// h, Dx, Dy sums in registers (8 x 4 texels per thread).  For each bucket it walks the
// integer bins that can reach the tile; the bump records of each bin row are
// contiguous in memory and are staged into shared memory with bulk async
// copies (cp.async.bulk, completion on an mbarrier), double-buffered so the
// copy of the next chunk overlaps the arithmetic of the current one.
//
// The bump kernel is separable, K = k(u) k(v), k(u) = 1/2 (1 + cos(pi u/R)),
// so for each staged bump the CTA evaluates k and sin once per tile column and
// once per tile row (shared memory) — one accurate sincospi per bump and
// axis at the tile's first texel, then the angle-addition rotation by the
// bucket's per-texel phase step e^{i pi Q / R} (a 64-entry float64-built
// table) — and each thread does the outer product:
//   h  += (A k(v)) * k(u)                 Dx += (A k(v)) * (lam/2) sin(pi u/R)
//   Dy += (A (lam/2) sin(pi v/R)) * k(u)
// i.e. 3 FMAs per bump-texel.  A warp skips bumps whose support misses its
// 32 x 32 sub-tile.  The epilogue applies the smoothstep blend weight and the
// bilinear background sample and writes the three maps (no atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace scwp {
namespace {

constexpr int kRPT = 8;            // texel rows per thread
constexpr int kCPT = 4;            // texel columns per thread
constexpr int kWR = 4 * kRPT;      // warp sub-tile: 4 x 8 threads
constexpr int kWC = 8 * kCPT;
constexpr int kTY = 2 * kWR;       // CTA tile: 2 x 2 warps (64 rows)
constexpr int kTX = 2 * kWC;       //                       (64 columns)
constexpr int kSlots = kTX + kTY;  // axis samples per bump
constexpr int kThreads = 128;
constexpr int kCH = 32;            // bumps per staged chunk
constexpr int kMaxRanges = 64;     // bin rows per bucket batch
constexpr int32_t kQi = 65536, kHalfi = 32768;
constexpr long long kSpinLimit = 1ll << 26;

struct BumpBase {                  // per bump and axis
    float c0, s0;                  // cos, sin of pi u0 / R at the tile's first texel
    int32_t u0;                    // first texel centre minus bump centre (Q16.16)
    float amp;                     // signed amplitude (rows), 1 (columns)
};

struct SynthSmem {
    int4 rec[2][kCH];              // staged bump records (16-byte aligned)
    unsigned long long bar[2];     // mbarriers
    BumpBase base[kCH][2];
    float kx[kCH][kTX];            // k(u) per column
    float kd[kCH][kTX];            // (lam/2) sin(pi u / R) per column
    float ay[kCH][kTY];            // A k(v) per row
    float cy[kCH][kTY];            // A (lam/2) sin(pi v / R) per row
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

// smoothstep blend weight of texel (ix, iy) and the bilinear, periodic
// background sample (h, Dx, Dy) there (skipped where the weight is 1)
__device__ __forceinline__ float blend_at(const SynthParams& sp, int ix, int iy, float bgv[3]) {
    const float d = fminf(fminf((float)ix + 0.5f, (float)sp.W - (float)ix - 0.5f),
                          fminf((float)iy + 0.5f, (float)sp.H - (float)iy - 0.5f));
    const float t = fminf(fmaxf(d / sp.band, 0.f), 1.f);
    const float w = t * t * (3.f - 2.f * t);
    bgv[0] = bgv[1] = bgv[2] = 0.f;
    if (w < 1.f) {
        const int N = sp.N;
        const size_t nplane = (size_t)N * N;
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
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const float* gp = sp.bg + f * nplane;
            bgv[f] = w00 * gp[i00] + w01 * gp[i01] + w10 * gp[i10] + w11 * gp[i11];
        }
    }
    return w;
}

// store 4 consecutive texels of row iy for the three fields
__device__ __forceinline__ void store_row4(float* out, size_t plane, int W, int iy, int ix0,
                                           const float o[3][4]) {
    const size_t rowo = (size_t)iy * W;
    if ((W & 3) == 0 && ix0 + 3 < W) {
#pragma unroll
        for (int f = 0; f < 3; ++f)
            *reinterpret_cast<float4*>(out + f * plane + rowo + ix0) =
                make_float4(o[f][0], o[f][1], o[f][2], o[f][3]);
    } else {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
            if (ix0 + cc < W)
#pragma unroll
                for (int f = 0; f < 3; ++f) out[f * plane + rowo + ix0 + cc] = o[f][cc];
    }
}

// sum of the bucket-group partials (in group order) and the blend
__global__ void __launch_bounds__(256) k_blend_groups(PatchDev p, SynthParams sp, const float* partial,
                                                      int groups) {
    const size_t plane = (size_t)sp.W * sp.H;
    const int qw = (sp.W + 3) / 4;
    const int nq = qw * sp.H;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const int iy = q / qw, ix0 = 4 * (q - iy * qw);
        float acc[3][4];
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) acc[f][cc] = 0.f;
        const size_t rowo = (size_t)iy * sp.W;
        const bool vec = (sp.W & 3) == 0 && ix0 + 3 < sp.W;
        for (int g = 0; g < groups; ++g) {
            const float* src = partial + (size_t)g * 3 * plane;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                if (vec) {
                    const float4 v = *reinterpret_cast<const float4*>(src + f * plane + rowo + ix0);
                    acc[f][0] += v.x;
                    acc[f][1] += v.y;
                    acc[f][2] += v.z;
                    acc[f][3] += v.w;
                } else {
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (ix0 + cc < sp.W) acc[f][cc] += src[f * plane + rowo + ix0 + cc];
                }
            }
        }
        float o[3][4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            float bgv[3];
            const float w = blend_at(sp, ix0 + cc, iy, bgv);
#pragma unroll
            for (int f = 0; f < 3; ++f) o[f][cc] = w * acc[f][cc] + (1.f - w) * bgv[f];
        }
        store_row4(p.out, plane, sp.W, iy, ix0, o);
    }
}

__global__ void __launch_bounds__(kThreads, 3) k_synth_gather(PatchDev p, SynthParams sp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SynthSmem& S = *reinterpret_cast<SynthSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = blockIdx.x * kTX, ty0 = blockIdx.y * kTY;
    // warp w covers rows kWR (w >> 1) .. +kWR, columns kWC (w & 1) .. +kWC
    const int tc = 8 * (warp & 1) + (lane & 7);     // column group 0..15
    const int tr = 4 * (warp >> 1) + (lane >> 3);   // row group 0..7

    float h[kRPT][kCPT], dx[kRPT][kCPT], dy[kRPT][kCPT];
#pragma unroll
    for (int r = 0; r < kRPT; ++r)
#pragma unroll
        for (int c = 0; c < kCPT; ++c) h[r][c] = dx[r][c] = dy[r][c] = 0.f;

    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    bool aborted = false;   // block-uniform (decided by __syncthreads_or)
    const int32_t Xlo = tx0 * kQi + kHalfi, Xhi = (tx0 + kTX - 1) * kQi + kHalfi;
    const int32_t Ylo = ty0 * kQi + kHalfi, Yhi = (ty0 + kTY - 1) * kQi + kHalfi;
    const float lamh = sp.lam_half;
    // this thread's sample slots in the generation phase: slot s < kTX is
    // column s, slot s >= kTX is row s - kTX; thread t owns slots t, t + 128
    constexpr int kSlotsPT = (kSlots + kThreads - 1) / kThreads;

    // bucket group of this CTA: buckets [b_begin, b_end)
    const int G = gridDim.z, g = blockIdx.z;
    const int b_begin = (g * sp.nb) / G, b_end = ((g + 1) * sp.nb) / G;
    for (int bi = b_begin; bi < b_end && !aborted; ++bi) {
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
        const int32_t R = bk.R;
        // rotation steps of this thread's sample slots: e^{i pi n Q / R}
        float2 rot[kSlotsPT];
#pragma unroll
        for (int q = 0; q < kSlotsPT; ++q) {
            const int sl = tid + q * kThreads;
            rot[q] = sl < kSlots ? p.rot[bi * kRotN + (sl < kTX ? sl : sl - kTX)] : make_float2(1.f, 0.f);
        }
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
                // (1) per bump and axis: the phase at the tile's first texel;
                //     per bump: which warps' sub-tiles its support reaches
                if (tid < 2 * n) {
                    const int b = tid >> 1, ax = tid & 1;
                    const int4 rc = S.rec[slot][b];
                    const int32_t u0 = ax ? Ylo - rc.y : Xlo - rc.x;
                    float sn, cs;
                    sincospif((float)u0 * invR, &sn, &cs);
                    BumpBase bb;
                    bb.c0 = cs;
                    bb.s0 = sn;
                    bb.u0 = u0;
                    bb.amp = ax ? __int_as_float(rc.z) : 1.f;
                    S.base[b][ax] = bb;
                } else if (tid >= 64 && tid < 64 + n) {
                    const int b = tid - 64;
                    const int4 rc = S.rec[slot][b];
                    const int xl = span_lo(rc.x, R) - tx0, xh = span_hi(rc.x, R) - tx0;
                    const int yl = span_lo(rc.y, R) - ty0, yh = span_hi(rc.y, R) - ty0;
                    uint32_t m = 0;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const int c0 = kWC * (w & 1), r0 = kWR * (w >> 1);
                        if (xl <= c0 + kWC - 1 && xh >= c0 && yl <= r0 + kWR - 1 && yh >= r0) m |= 1u << w;
                    }
                    S.mask[b] = m;
                }
                __syncthreads();
                // (2) samples by phase rotation of the bump's base phase
                for (int b = 0; b < n; ++b) {
#pragma unroll
                    for (int q = 0; q < kSlotsPT; ++q) {
                        const int sl = tid + q * kThreads;
                        if (sl >= kSlots) break;
                        const bool col = sl < kTX;
                        const int k = col ? sl : sl - kTX;
                        const BumpBase bb = S.base[b][col ? 0 : 1];
                        const int32_t u = bb.u0 + k * kQi;
                        const bool in = u > -R && u < R;
                        const float cs = bb.c0 * rot[q].x - bb.s0 * rot[q].y;
                        const float sn = bb.s0 * rot[q].x + bb.c0 * rot[q].y;
                        const float kv = in ? bb.amp * (0.5f + 0.5f * cs) : 0.f;
                        const float dv = in ? bb.amp * lamh * sn : 0.f;
                        if (col) {
                            S.kx[b][k] = kv;
                            S.kd[b][k] = dv;
                        } else {
                            S.ay[b][k] = kv;
                            S.cy[b][k] = dv;
                        }
                    }
                }
                uint32_t todo = __ballot_sync(0xffffffffu, lane < n && ((S.mask[lane] >> warp) & 1u));
                __syncthreads();
                // (3) outer products: kRPT x kCPT texels x 3 fields per thread
                while (todo) {
                    const int b = __ffs(todo) - 1;
                    todo &= todo - 1;
                    float kxv[kCPT], kdv[kCPT], ayv[kRPT], cyv[kRPT];
#pragma unroll
                    for (int q = 0; q < kCPT / 4; ++q) {
                        const float4 a = *reinterpret_cast<const float4*>(&S.kx[b][kCPT * tc + 4 * q]);
                        const float4 d = *reinterpret_cast<const float4*>(&S.kd[b][kCPT * tc + 4 * q]);
                        kxv[4 * q] = a.x; kxv[4 * q + 1] = a.y; kxv[4 * q + 2] = a.z; kxv[4 * q + 3] = a.w;
                        kdv[4 * q] = d.x; kdv[4 * q + 1] = d.y; kdv[4 * q + 2] = d.z; kdv[4 * q + 3] = d.w;
                    }
#pragma unroll
                    for (int q = 0; q < kRPT / 4; ++q) {
                        const float4 a = *reinterpret_cast<const float4*>(&S.ay[b][kRPT * tr + 4 * q]);
                        const float4 c = *reinterpret_cast<const float4*>(&S.cy[b][kRPT * tr + 4 * q]);
                        ayv[4 * q] = a.x; ayv[4 * q + 1] = a.y; ayv[4 * q + 2] = a.z; ayv[4 * q + 3] = a.w;
                        cyv[4 * q] = c.x; cyv[4 * q + 1] = c.y; cyv[4 * q + 2] = c.z; cyv[4 * q + 3] = c.w;
                    }
#pragma unroll
                    for (int r = 0; r < kRPT; ++r)
#pragma unroll
                        for (int cc = 0; cc < kCPT; ++cc) {
                            h[r][cc] = fmaf(ayv[r], kxv[cc], h[r][cc]);
                            dx[r][cc] = fmaf(ayv[r], kdv[cc], dx[r][cc]);
                            dy[r][cc] = fmaf(cyv[r], kxv[cc], dy[r][cc]);
                        }
                }
                __syncthreads();
            }
        }
    }

    // ---- epilogue ------------------------------------------------------------------
    const size_t plane = (size_t)sp.W * sp.H;
    if (G > 1) {
        // raw sums of this bucket group; k_blend_groups adds the groups in
        // order and blends
        float* dst = p.partial + (size_t)g * 3 * plane;
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const int iy = ty0 + kRPT * tr + r;
            if (iy >= sp.H) continue;
#pragma unroll
            for (int q = 0; q < kCPT / 4; ++q) {
                const float o[3][4] = {{h[r][4 * q], h[r][4 * q + 1], h[r][4 * q + 2], h[r][4 * q + 3]},
                                       {dx[r][4 * q], dx[r][4 * q + 1], dx[r][4 * q + 2], dx[r][4 * q + 3]},
                                       {dy[r][4 * q], dy[r][4 * q + 1], dy[r][4 * q + 2], dy[r][4 * q + 3]}};
                store_row4(dst, plane, sp.W, iy, tx0 + kCPT * tc + 4 * q, o);
            }
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int iy = ty0 + kRPT * tr + r;
        if (iy >= sp.H) continue;
#pragma unroll
        for (int q = 0; q < kCPT / 4; ++q) {
            float o[3][4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int ix = tx0 + kCPT * tc + 4 * q + cc;
                float bgv[3];
                const float w = blend_at(sp, ix, iy, bgv);
                o[0][cc] = w * h[r][4 * q + cc] + (1.f - w) * bgv[0];
                o[1][cc] = w * dx[r][4 * q + cc] + (1.f - w) * bgv[1];
                o[2][cc] = w * dy[r][4 * q + cc] + (1.f - w) * bgv[2];
            }
            store_row4(p.out, plane, sp.W, iy, tx0 + kCPT * tc + 4 * q, o);
        }
    }
}

}  // namespace

cudaError_t launch_synth_gather(const PatchDev& p, const SynthParams& sp, cudaStream_t st) {
    const size_t sm = sizeof(SynthSmem);
    cudaError_t e = cudaFuncSetAttribute(k_synth_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int G = p.groups > 1 && p.partial ? p.groups : 1;
    dim3 grid((p.W + kTX - 1) / kTX, (p.H + kTY - 1) / kTY, G);
    k_synth_gather<<<grid, kThreads, sm, st>>>(p, sp);
    count_launches(1);
    if (G > 1) return launch_blend(p, sp, p.partial, G, st);
    return cudaGetLastError();
}

cudaError_t launch_blend(const PatchDev& p, const SynthParams& sp, const float* src, int groups,
                         cudaStream_t st) {
    const int nq = ((p.W + 3) / 4) * p.H;
    int blocks = (nq + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_blend_groups<<<blocks, 256, 0, st>>>(p, sp, src, groups);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace scwp
