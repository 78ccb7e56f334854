// Wave-particle synthesis of the hybrid ocean (sm_103a), Sec. 4.2:
// per-bucket accumulation of the particle kernels into the patch height map,
// displacement from the kernel gradient, and the distance-weighted blend into
// the FFT background.
//
// Tile gather, warp-specialised.  One CTA owns a 64 x 64 texel tile (and one
// group of its buckets) with six warps:
//   * two producer warps walk the integer bins that can reach the tile, stage
//     each chunk of 32 bump records into shared memory with a bulk async copy
//     (cp.async.bulk, completion on an mbarrier), and turn it into the
//     separable kernel factors of the tile: per bump one accurate sincospi
//     per axis at the tile's first texel, then the angle-addition rotation by
//     the bucket's per-texel phase step e^{i pi n Q / R} (a float64-built
//     table), giving per column k(u), (lam/2) sin(pi u/R) and per row
//     A k(v), A (lam/2) sin(pi v/R), plus a mask of the warps whose
//     32 x 32 sub-tile the bump reaches;
//   * four consumer warps keep the tile's h, Dx, Dy sums in registers
//     (8 x 4 texels per thread) and do the outer products
//       h  += (A k(v)) k(u)    Dx += (A k(v)) (lam/2) sin(pi u/R)
//       Dy += (A (lam/2) sin(pi v/R)) k(u)
//     i.e. 3 FMAs per bump-texel, skipping bumps outside their sub-tile.
// Producers and consumers meet in a ring of factor slots guarded by
// full/empty mbarriers (no block-wide barrier in the steady state).  Every
// wait is bounded in time; a timeout sets an error flag and the CTA stops.
// The epilogue writes the group's partial sums, or (one group) applies the
// smoothstep blend weight and the bilinear background sample (no atomics).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "internal.h"

namespace scwp {
namespace {

constexpr int kRPT = 8;            // texel rows per consumer thread
constexpr int kCPT = 4;            // texel columns per consumer thread
constexpr int kWR = 4 * kRPT;      // consumer warp sub-tile: 4 x 8 threads
constexpr int kWC = 8 * kCPT;
constexpr int kTY = 2 * kWR;       // CTA tile: 2 x 2 consumer warps (64 rows)
constexpr int kTX = 2 * kWC;       //                                (64 columns)
constexpr int kConsumers = 4;      // warps
constexpr int kProducers = 2;      // warps
constexpr int kPThreads = 32 * kProducers;
constexpr int kThreads = 32 * (kConsumers + kProducers);
constexpr int kCH = 32;            // bumps per chunk
constexpr int kSlotsRing = 3;      // factor slots in flight
constexpr int kMaxRanges = 64;     // bin rows per bucket batch
constexpr int32_t kQi = 65536, kHalfi = 32768;
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

struct __align__(16) FactorSlot {
    float kx[kCH][kTX];            // k(u) per column
    float kd[kCH][kTX];            // (lam/2) sin(pi u / R) per column
    float ay[kCH][kTY];            // A k(v) per row
    float cy[kCH][kTY];            // A (lam/2) sin(pi v / R) per row
    uint32_t mask[kCH];            // consumer warps whose sub-tile the bump reaches
    int n;                         // bumps in the slot; -1 ends the stream
};

struct BumpBase {                  // per bump and axis
    float c0, s0;                  // cos, sin of pi u0 / R at the tile's first texel
    int32_t u0;                    // first texel centre minus bump centre (Q16.16)
    float amp;                     // signed amplitude (rows), 1 (columns)
};

struct SynthSmem {
    FactorSlot slot[kSlotsRing];
    BumpRec rec[2][kCH];           // staged bump records (16-byte aligned)
    unsigned long long rbar[2];    // record copies: complete_tx
    unsigned long long full[kSlotsRing];   // producers -> consumers (kPThreads arrivals)
    unsigned long long empty[kSlotsRing];  // consumers -> producers (kConsumers arrivals)
    BumpBase base[kCH][2];
    int rstart[kMaxRanges];        // bin-row ranges of the current bucket batch
    int rlen[kMaxRanges];
    int cpre[kMaxRanges + 1];      // chunk prefix per range
    int stop;                      // producers: a wait timed out
};
// float4 loads from every slot and bulk copies into rec need 16-byte alignment
static_assert(sizeof(FactorSlot) % 16 == 0, "factor slot alignment");
static_assert(offsetof(SynthSmem, rec) % 16 == 0, "record staging alignment");
static_assert(offsetof(SynthSmem, rbar) % 8 == 0 && offsetof(SynthSmem, full) % 8 == 0 &&
                  offsetof(SynthSmem, empty) % 8 == 0,
              "mbarrier alignment");
static_assert(offsetof(FactorSlot, kd) % 16 == 0 && offsetof(FactorSlot, ay) % 16 == 0 &&
                  offsetof(FactorSlot, cy) % 16 == 0,
              "factor array alignment");

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
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(err, (unsigned long long)kErrTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// named barrier among the producer warps only
__device__ __forceinline__ void producer_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kPThreads) : "memory");
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

// sum of the bucket-group partials (in group order) and the blend of quad q
// (texels 4 (q mod qw) .. + 3 of row q / qw)
__device__ __forceinline__ void blend_quad(const PatchDev& p, const SynthParams& sp, const float* partial,
                                           int groups, int q) {
    const size_t plane = (size_t)sp.W * sp.H;
    const int qw = (sp.W + 3) / 4;
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

__global__ void __launch_bounds__(256) k_blend_groups(PatchDev p, SynthParams sp, const float* partial,
                                                      int groups) {
    const int nq = ((sp.W + 3) / 4) * sp.H;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x)
        blend_quad(p, sp, partial, groups, q);
}

// the same over spans of any patches: one CTA per span
__global__ void __launch_bounds__(256) k_blend_spans(const BlendSpan* spans, const PatchDev* pdevs,
                                                     const SynthParams* sps) {
    pdl_enter();
    const BlendSpan sn = spans[blockIdx.x];
    const PatchDev& p = pdevs[sn.patch];
    const SynthParams& sp = sps[sn.patch];
    for (int q = sn.q0 + threadIdx.x; q < sn.q1; q += blockDim.x) blend_quad(p, sp, p.partial, sn.groups, q);
}

__global__ void __launch_bounds__(kThreads, 2) k_synth_gather(PatchDev p, SynthParams sp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SynthSmem& S = *reinterpret_cast<SynthSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx0 = blockIdx.x * kTX, ty0 = blockIdx.y * kTY;
    const int G = gridDim.z, g = blockIdx.z;
    const int b_begin = (g * sp.nb) / G, b_end = ((g + 1) * sp.nb) / G;

    if (tid == 0) {
        mbar_init(&S.rbar[0], 1);
        mbar_init(&S.rbar[1], 1);
        for (int k = 0; k < kSlotsRing; ++k) {
            mbar_init(&S.full[k], kPThreads);
            mbar_init(&S.empty[k], kConsumers);
        }
        S.stop = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    if (warp >= kConsumers) {
        // ======================= producers ===================================
        const int ptid = tid - 32 * kConsumers;
        const int32_t Xlo = tx0 * kQi + kHalfi, Xhi = (tx0 + kTX - 1) * kQi + kHalfi;
        const int32_t Ylo = ty0 * kQi + kHalfi, Yhi = (ty0 + kTY - 1) * kQi + kHalfi;
        const float lamh = sp.lam_half;
        uint32_t rpar[2] = {0u, 0u};
        int produced = 0;                  // chunks pushed into the ring
        bool dead = false;
        for (int bi = b_begin; bi < b_end && !dead; ++bi) {
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
            // rotation steps of this thread's column and row: e^{i pi n Q / R}
            const float2 rot = p.rot[bi * kRotN + ptid];
            for (int byb = by_lo; byb <= by_hi && !dead; byb += kMaxRanges) {
                const int nr = min(kMaxRanges, by_hi - byb + 1);
                for (int k = ptid; k < nr; k += kPThreads) {
                    const int key0 = bk.base + (byb + k) * bk.nbx;
                    const int s = (int)p.offsets[key0 + bx_lo];
                    const int e = (int)p.offsets[key0 + bx_hi + 1];
                    S.rstart[k] = s;
                    S.rlen[k] = e - s;
                }
                producer_sync();
                if (ptid == 0) {
                    int acc = 0;
                    for (int k = 0; k < nr; ++k) {
                        S.cpre[k] = acc;
                        acc += (S.rlen[k] + kCH - 1) / kCH;
                    }
                    S.cpre[nr] = acc;
                }
                producer_sync();
                const int nchunks = S.cpre[nr];
                if (nchunks == 0) continue;
                auto chunk = [&](int c, int& off, int& n) {
                    int k = 0;
                    while (S.cpre[k + 1] <= c) ++k;
                    off = S.rstart[k] + (c - S.cpre[k]) * kCH;
                    n = min(kCH, S.rstart[k] + S.rlen[k] - off);
                };
                if (ptid == 0) {
                    int off, n;
                    chunk(0, off, n);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive_expect(&S.rbar[0], (uint32_t)(n * sizeof(BumpRec)));
                    bulk_g2s(&S.rec[0][0], p.rec + off, (uint32_t)(n * sizeof(BumpRec)), &S.rbar[0]);
                }
                for (int c = 0; c < nchunks; ++c) {
                    const int rs = c & 1;
                    int off, n;
                    chunk(c, off, n);
                    const bool ok_r = mbar_wait_bounded(&S.rbar[rs], rpar[rs], p.stats + 2);
                    rpar[rs] ^= 1u;
                    if (!ok_r) S.stop = 1;
                    // bases (warp 0 of the producers: x, warp 1: y) and masks
                    if (lane < n && !S.stop) {
                        const BumpRec rc = S.rec[rs][lane];
                        const int ax = ptid >> 5;
                        const int32_t u0 = ax ? Ylo - rc.y : Xlo - rc.x;
                        float sn, cs;
                        sincospif((float)u0 * invR, &sn, &cs);
                        BumpBase bb;
                        bb.c0 = cs;
                        bb.s0 = sn;
                        bb.u0 = u0;
                        bb.amp = ax ? rc.amp : 1.f;
                        S.base[lane][ax] = bb;
                    }
                    const int fs = produced % kSlotsRing;
                    const uint32_t epar = ((produced / kSlotsRing) & 1u) ^ 1u;
                    const bool ok_e = mbar_wait_bounded(&S.empty[fs], epar, p.stats + 2);
                    if (!ok_e) S.stop = 1;
                    FactorSlot& F = S.slot[fs];
                    if (ptid < n && !S.stop) {
                        const BumpRec rc = S.rec[rs][ptid];
                        const int xl = span_lo(rc.x, R) - tx0, xh = span_hi(rc.x, R) - tx0;
                        const int yl = span_lo(rc.y, R) - ty0, yh = span_hi(rc.y, R) - ty0;
                        uint32_t m = 0;
#pragma unroll
                        for (int w = 0; w < kConsumers; ++w) {
                            const int c0 = kWC * (w & 1), r0 = kWR * (w >> 1);
                            if (xl <= c0 + kWC - 1 && xh >= c0 && yl <= r0 + kWR - 1 && yh >= r0) m |= 1u << w;
                        }
                        F.mask[ptid] = m;
                    }
                    producer_sync();   // bases visible; record slot rs free
                    if (S.stop) {
                        dead = true;
                        break;
                    }
                    if (ptid == 0 && c + 1 < nchunks) {
                        int off2, n2;
                        chunk(c + 1, off2, n2);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        mbar_arrive_expect(&S.rbar[rs ^ 1], (uint32_t)(n2 * sizeof(BumpRec)));
                        bulk_g2s(&S.rec[rs ^ 1][0], p.rec + off2, (uint32_t)(n2 * sizeof(BumpRec)), &S.rbar[rs ^ 1]);
                    }
                    // factors: column ptid and row ptid of every bump
                    for (int b = 0; b < n; ++b) {
                        {
                            const BumpBase bb = S.base[b][0];
                            const int32_t u = bb.u0 + ptid * kQi;
                            const bool in = u > -R && u < R;
                            const float cs = bb.c0 * rot.x - bb.s0 * rot.y;
                            const float sn = bb.s0 * rot.x + bb.c0 * rot.y;
                            F.kx[b][ptid] = in ? 0.5f + 0.5f * cs : 0.f;
                            F.kd[b][ptid] = in ? lamh * sn : 0.f;
                        }
                        {
                            const BumpBase bb = S.base[b][1];
                            const int32_t v = bb.u0 + ptid * kQi;
                            const bool in = v > -R && v < R;
                            const float cs = bb.c0 * rot.x - bb.s0 * rot.y;
                            const float sn = bb.s0 * rot.x + bb.c0 * rot.y;
                            F.ay[b][ptid] = in ? bb.amp * (0.5f + 0.5f * cs) : 0.f;
                            F.cy[b][ptid] = in ? bb.amp * lamh * sn : 0.f;
                        }
                    }
                    if (ptid == 0) F.n = n;
                    mbar_arrive(&S.full[fs]);
                    ++produced;
                    producer_sync();   // every producer done with S.base before the next chunk
                }
            }
        }
        // end of stream (also after a timeout, so the consumers stop)
        const int fs = produced % kSlotsRing;
        const uint32_t epar = ((produced / kSlotsRing) & 1u) ^ 1u;
        mbar_wait_bounded(&S.empty[fs], epar, p.stats + 2);
        if (ptid == 0) S.slot[fs].n = -1;
        mbar_arrive(&S.full[fs]);
        return;
    }

    // ========================= consumers =======================================
    const int tc = 8 * (warp & 1) + (lane & 7);     // column group 0..15
    const int tr = 4 * (warp >> 1) + (lane >> 3);   // row group 0..7
    float h[kRPT][kCPT], dx[kRPT][kCPT], dy[kRPT][kCPT];
#pragma unroll
    for (int r = 0; r < kRPT; ++r)
#pragma unroll
        for (int c = 0; c < kCPT; ++c) h[r][c] = dx[r][c] = dy[r][c] = 0.f;
    for (int k = 0;; ++k) {
        const int fs = k % kSlotsRing;
        const uint32_t fpar = (k / kSlotsRing) & 1u;
        if (!mbar_wait_bounded(&S.full[fs], fpar, p.stats + 2)) break;
        const FactorSlot& F = S.slot[fs];
        const int n = F.n;
        if (n < 0) break;
        uint32_t todo = __ballot_sync(0xffffffffu, lane < n && ((F.mask[lane] >> warp) & 1u));
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            const float4 kx4 = *reinterpret_cast<const float4*>(&F.kx[b][kCPT * tc]);
            const float4 kd4 = *reinterpret_cast<const float4*>(&F.kd[b][kCPT * tc]);
            const float4 a0 = *reinterpret_cast<const float4*>(&F.ay[b][kRPT * tr]);
            const float4 a1 = *reinterpret_cast<const float4*>(&F.ay[b][kRPT * tr + 4]);
            const float4 c0 = *reinterpret_cast<const float4*>(&F.cy[b][kRPT * tr]);
            const float4 c1 = *reinterpret_cast<const float4*>(&F.cy[b][kRPT * tr + 4]);
            const float kxv[4] = {kx4.x, kx4.y, kx4.z, kx4.w};
            const float kdv[4] = {kd4.x, kd4.y, kd4.z, kd4.w};
            const float ayv[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float cyv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int r = 0; r < kRPT; ++r)
#pragma unroll
                for (int cc = 0; cc < kCPT; ++cc) {
                    h[r][cc] = fmaf(ayv[r], kxv[cc], h[r][cc]);
                    dx[r][cc] = fmaf(ayv[r], kdv[cc], dx[r][cc]);
                    dy[r][cc] = fmaf(cyv[r], kxv[cc], dy[r][cc]);
                }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[fs]);
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
            const float o[3][4] = {{h[r][0], h[r][1], h[r][2], h[r][3]},
                                   {dx[r][0], dx[r][1], dx[r][2], dx[r][3]},
                                   {dy[r][0], dy[r][1], dy[r][2], dy[r][3]}};
            store_row4(dst, plane, sp.W, iy, tx0 + kCPT * tc, o);
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kRPT; ++r) {
        const int iy = ty0 + kRPT * tr + r;
        if (iy >= sp.H) continue;
        float o[3][4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            const int ix = tx0 + kCPT * tc + cc;
            float bgv[3];
            const float w = blend_at(sp, ix, iy, bgv);
            o[0][cc] = w * h[r][cc] + (1.f - w) * bgv[0];
            o[1][cc] = w * dx[r][cc] + (1.f - w) * bgv[1];
            o[2][cc] = w * dy[r][cc] + (1.f - w) * bgv[2];
        }
        store_row4(p.out, plane, sp.W, iy, tx0 + kCPT * tc, o);
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

cudaError_t launch_blend_spans(const BlendSpan* spans, int n_spans, const PatchDev* pdevs, const SynthParams* sps,
                               cudaStream_t st) {
    const cudaError_t e = launch_pdl(k_blend_spans, n_spans, 256, 0, st, spans, pdevs, sps);
    count_launches(1);
    return e;
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
