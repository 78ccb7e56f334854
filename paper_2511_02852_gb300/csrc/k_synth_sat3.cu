// Summed-area synthesis, three-group variant: the same sums as k_synth_sat.cu
// (Sec. 4.2, kernel reading O11, analytic displacement O12; the identity and
// the exactness argument are stated there) with the nine S_ij planes taken
// as three groups of three, so that two 512-thread CTAs fit an SM.  Each
// candidate is turned into corner events once per group; the first 1984 of a
// bucket are staged in shared memory, the rest re-read from the records.  It
// wins where a (tile, bucket) has few candidates (per-texel work dominates,
// and the two CTAs of an SM hide each other's phase barriers); the
// persistent nine-plane kernel wins where candidates dominate.  The
// autotuner of api.cu times both on the live scene.  A bucket reaching more
// than 512 bin rows of a tile does not fit the row table; the host selects
// this variant only for patches whose buckets stay within it.
//
// One CTA per (tile, bucket group) item, 512 threads, two CTAs per SM.  The
// nine S components are processed in three groups of three (fixed p_i), so
// the difference array takes 48 KB of shared memory.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "blend_dev.cuh"
#include "internal.h"

namespace scwp {
namespace {

constexpr int kT = 64;                       // tile side in texels
constexpr int kSatThreads = 512;
constexpr int kSatWarps = kSatThreads / 32;
constexpr int kSegs = kSatThreads / kT;      // row segments of the column pass
constexpr int kSegRows = kT / kSegs;         // rows per segment
constexpr int kSatRowCap = 512;              // bin rows of the item's buckets held at once
constexpr int kSatStage = 1984;              // candidates of a bucket staged in shared memory
constexpr int32_t kQs = 65536, kHalfs = 32768;
static_assert(kSegs * kSegRows == kT && kSegs == 8, "column-pass mapping");

struct SatSmem {
    uint32_t E[3][kT * kT];               // difference array, then prefix sums (one component group)
    uint32_t seg[kSegs][3][kT];           // column sums of each row segment
    float2 ph[2 * kT];                    // the bucket's texel phases (cos, sin) a: rows, then columns
    float4 c4[kSatStage];                 // staged candidates: A, cos, sin (x), cos (y)
    float2 c2[kSatStage];                 //                    sin (y), support box (bits)
    int32_t rs[kSatRowCap];               // first record of each bin row (all buckets of a batch)
    int32_t cum[kSatRowCap];              // candidates of the bucket before the row
    BucketDev bk[kMaxBuckets];            // the item's buckets
    int32_t bx_lo[kMaxBuckets], bx_hi[kMaxBuckets], by_lo[kMaxBuckets], nrows[kMaxBuckets];
    int32_t rb[kMaxBuckets + 1];          // first row of each bucket of the batch
    int32_t ncand[kMaxBuckets];           // candidates of each bucket
    int32_t batch_end;                    // one past the last bucket of the batch
    alignas(16) unsigned char pd[sizeof(PatchDev)];
    alignas(16) unsigned char spd[sizeof(SynthParams)];
};

// element (row y, column x) of a 64 x 64 plane: columns XOR-swizzled by the
// row so that a warp walking a row (one row per lane) or a column (one
// column per lane) touches 32 different banks
__device__ __forceinline__ int sw(int y, int x) { return y * kT + (x ^ (y & 31)); }

__device__ __forceinline__ int clamp_t(int t) { return min(max(t, 0), kT); }

// the three components of one corner event
__device__ __forceinline__ void event3(SatSmem& S, int x, int y, uint32_t w0, uint32_t w1, uint32_t w2) {
    const int o = sw(y, x);
    atomicAdd(&S.E[0][o], w0);
    atomicAdd(&S.E[1][o], w1);
    atomicAdd(&S.E[2][o], w2);
}

// inclusive warp scan of v
__device__ __forceinline__ uint32_t warp_scan(uint32_t v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__global__ void __launch_bounds__(kSatThreads, 2) k_synth_sat3(const TcItem* items, const PatchDev* pdevs,
                                                            const SynthParams* sps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SatSmem& S = *reinterpret_cast<SatSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    pdl_enter();
    const TcItem it = items[blockIdx.x];
    {
        static_assert(sizeof(PatchDev) % 4 == 0 && sizeof(SynthParams) % 4 == 0, "descriptor copy");
        const uint32_t* a = reinterpret_cast<const uint32_t*>(pdevs + it.patch);
        const uint32_t* b = reinterpret_cast<const uint32_t*>(sps + it.patch);
        for (int k = tid; k < (int)(sizeof(PatchDev) / 4); k += kSatThreads) reinterpret_cast<uint32_t*>(S.pd)[k] = a[k];
        for (int k = tid; k < (int)(sizeof(SynthParams) / 4); k += kSatThreads)
            reinterpret_cast<uint32_t*>(S.spd)[k] = b[k];
    }
    __syncthreads();
    const PatchDev& p = *reinterpret_cast<const PatchDev*>(S.pd);
    const SynthParams& sp = *reinterpret_cast<const SynthParams*>(S.spd);
    const int G = item_groups(it), g = item_group(it), K = item_parts(it), part = item_part(it);
    const int ntx = (sp.W + kT - 1) / kT;
    const int tx0 = (it.tile % ntx) * kT, ty0 = (it.tile / ntx) * kT;
    const int b_begin = max((g * sp.nb) / G, sp.b_lo);
    const int b_end = min(((g + 1) * sp.nb) / G, sp.b_hi);
    const int nbk = max(0, b_end - b_begin);
    // Q16.16 centres of the tile's first and last texel columns and rows
    const int32_t X0 = tx0 * kQs + kHalfs, X1 = X0 + (kT - 1) * kQs;
    const int32_t Y0 = ty0 * kQs + kHalfs, Y1 = Y0 + (kT - 1) * kQs;
    const float lamq = 0.5f * sp.lam_half;   // lam / 4

    // ---- the item's buckets and the bin rows that reach the tile
    // (bins hold x_b + R in [bx C, (bx + 1) C))
    for (int t = tid; t < nbk; t += kSatThreads) {
        const BucketDev bk = p.bk[b_begin + t];
        S.bk[t] = bk;
        const int bx_lo = (int)((int64_t)X0 / bk.C);
        const int bx_hi = min((int)(((int64_t)X1 + 2 * (int64_t)bk.R - 1) / bk.C), bk.nbx - 1);
        const int by_lo = (int)((int64_t)Y0 / bk.C);
        const int by_hi = min((int)(((int64_t)Y1 + 2 * (int64_t)bk.R - 1) / bk.C), bk.nby - 1);
        S.bx_lo[t] = bx_lo;
        S.bx_hi[t] = bx_hi;
        S.by_lo[t] = by_lo;
        S.nrows[t] = (bx_lo > bx_hi || by_lo > by_hi) ? 0 : by_hi - by_lo + 1;
    }

    // column pass: this thread owns texel column cx of rows sg*8 .. sg*8 + 7
    const int cx = tid & (kT - 1), sg = tid / kT;
    float ah[kSegRows], adx[kSegRows], ady[kSegRows];
#pragma unroll
    for (int r = 0; r < kSegRows; ++r) ah[r] = adx[r] = ady[r] = 0.f;

    // buckets in batches whose bin rows fit the row tables
    for (int bb = 0; bb < nbk;) {
        __syncthreads();   // bucket geometry written; the previous batch is done with the tables
        if (tid == 0) {
            int n = 0, be = bb;
            while (be < nbk && (be == bb || n + S.nrows[be] <= kSatRowCap)) {
                S.rb[be - bb] = n;
                n += min(S.nrows[be], kSatRowCap);
                ++be;
            }
            S.rb[be - bb] = n;
            S.batch_end = be;
        }
        __syncthreads();
        const int be = S.batch_end;
        const int nq = S.rb[be - bb];
        // every row of the batch: record range from the bin offsets
        for (int q = tid; q < nq; q += kSatThreads) {
            int t = 0;
            while (S.rb[t + 1] <= q) ++t;
            const int bi = bb + t, r = q - S.rb[t];
            const BucketDev& bk = S.bk[bi];
            const int key0 = bk.base + (S.by_lo[bi] + r) * bk.nbx;
            const int s0 = (int)p.offsets[key0 + S.bx_lo[bi]];
            S.rs[q] = s0;
            S.cum[q] = (int)p.offsets[key0 + S.bx_hi[bi] + 1] - s0;   // row length for now
        }
        __syncthreads();
        // per bucket: exclusive prefix of the row lengths (warp w takes buckets w, w + 16, ...)
        for (int t = warp; t < be - bb; t += kSatWarps) {
            const int q0 = S.rb[t], q1 = S.rb[t + 1];
            uint32_t carry = 0u;
            for (int q = q0; q < q1; q += 32) {
                const uint32_t l = q + lane < q1 ? (uint32_t)S.cum[q + lane] : 0u;
                const uint32_t inc = warp_scan(l, lane);
                if (q + lane < q1) S.cum[q + lane] = (int32_t)(carry + inc - l);
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
            if (lane == 0) S.ncand[bb + t] = (int32_t)carry;
        }
        __syncthreads();

        for (int bi = bb; bi < be; ++bi) {
            const int t = bi - bb;
            const int ncand = S.ncand[bi];
            const float amax = p.amax[b_begin + bi];
            if (ncand == 0 || !(amax > 0.f)) continue;   // no bump of this bucket reaches the tile
            if (S.nrows[bi] > kSatRowCap) continue;   // not reached: the host selects this variant only
                                                      // where every bucket fits the row table
            const BucketDev bk = S.bk[bi];
            const int q0 = S.rb[t], q1 = S.rb[t + 1];
            for (int k = tid; k < 2 * kT; k += kSatThreads)
                S.ph[k] = p.phase[(size_t)(b_begin + bi) * p.phase_len + (k < kT ? ty0 + k : tx0 + (k - kT))];
            // stage the first kSatStage candidates: warp w takes rows w, w + 16, ...
            for (int q = q0 + warp; q < q1; q += kSatWarps) {
                const int f_row = S.cum[q];
                const int l = (q + 1 < q1 ? S.cum[q + 1] : ncand) - f_row;
                const int r0 = S.rs[q];
                for (int k = lane; k < l && f_row + k < kSatStage; k += 32) {
                    const float4* rp = reinterpret_cast<const float4*>(p.rec + r0 + k);
                    const float4 rx = rp[0];   // x, cos, sin, id
                    const float4 ry = rp[1];   // y, cos, sin, A
                    const int32_t xb = __float_as_int(rx.x), yb = __float_as_int(ry.x);
                    // texel t of the tile is inside iff x_b - R < X0 + t Q < x_b + R
                    const int a = clamp_t(((xb - bk.R - X0) >> 16) + 1);
                    const int b = clamp_t(-((X0 - xb - bk.R) >> 16));
                    const int c = clamp_t(((yb - bk.R - Y0) >> 16) + 1);
                    const int d = clamp_t(-((Y0 - yb - bk.R) >> 16));
                    const uint32_t box = (a < b && c < d) ? (uint32_t)a | ((uint32_t)b << 7) | ((uint32_t)c << 14) |
                                                                ((uint32_t)d << 21)
                                                          : 0u;
                    S.c4[f_row + k] = make_float4(ry.w, rx.y, rx.z, ry.y);
                    S.c2[f_row + k] = make_float2(ry.z, __uint_as_float(box));
                }
            }
            // passes of at most mch candidates, so that the integer rounding
            // of the corner weights stays within the bound set on the host
            const float nf = (float)ncand;
            const int kch = max(1, (int)ceilf(nf * sqrtf(nf) / bk.sat_c));
            const int mch = (ncand + kch - 1) / kch;
            for (int c0 = part * mch; c0 < ncand; c0 += K * mch) {   // this part's passes
            const int c1 = min(ncand, c0 + mch);
            if (tid == 0) atomicAdd(p.stats + 5 + p.nb, (unsigned long long)(c1 - c0));
            const float bound = 1.001f * (float)(c1 - c0) * amax;   // >= every |S_ij| of the pass
            const float scale = 1073741824.f / bound;              // 2^30 / bound
            const float inv = bound * (1.f / 1073741824.f);        // 1 / scale

            for (int i = 0; i < 3; ++i) {   // component group p_i: S_i0, S_i1, S_i2
                for (int k = tid; k < 3 * kT * kT / 4; k += kSatThreads)
                    reinterpret_cast<uint4*>(&S.E[0][0])[k] = make_uint4(0u, 0u, 0u, 0u);
                __syncthreads();
                // ---- corner events; candidate f of the bucket, all lanes of a
                // warp in the same trips.  The corner (0, 0) is shared by
                // every bump that covers the tile's first texel: its weights
                // are summed per thread here and per warp after the loop.
                uint32_t z0 = 0u, z1 = 0u, z2 = 0u;
                for (int f0 = c0 + warp * 32; f0 < c1; f0 += kSatThreads) {
                    const int f = f0 + lane;
                    float A = 0.f, pc = 0.f, ps = 0.f, qc = 0.f, qs = 0.f;
                    uint32_t box = 0u;   // empty box: no events
                    if (f < c1) {
                        if (f < kSatStage) {
                            const float4 c = S.c4[f];
                            const float2 e = S.c2[f];
                            A = c.x; pc = c.y; ps = c.z; qc = c.w; qs = e.x;
                            box = __float_as_uint(e.y);
                        } else {
                            // the row holding candidate f, and its record
                            int lo = q0, hi = q1 - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (S.cum[mid] <= f) lo = mid; else hi = mid - 1;
                            }
                            const float4* rp = reinterpret_cast<const float4*>(p.rec + S.rs[lo] + (f - S.cum[lo]));
                            const float4 rx = rp[0];   // x, cos, sin, id
                            const float4 ry = rp[1];   // y, cos, sin, A
                            const int32_t xb = __float_as_int(rx.x), yb = __float_as_int(ry.x);
                            // texel t of the tile is inside iff x_b - R < X0 + t Q < x_b + R
                            const int a = clamp_t(((xb - bk.R - X0) >> 16) + 1);
                            const int b = clamp_t(-((X0 - xb - bk.R) >> 16));
                            const int c = clamp_t(((yb - bk.R - Y0) >> 16) + 1);
                            const int d = clamp_t(-((Y0 - yb - bk.R) >> 16));
                            box = (a < b && c < d) ? (uint32_t)a | ((uint32_t)b << 7) | ((uint32_t)c << 14) |
                                                         ((uint32_t)d << 21)
                                                   : 0u;
                            A = ry.w; pc = rx.y; ps = rx.z; qc = ry.y; qs = ry.z;
                        }
                    }
                    const int a = box & 127, b = (box >> 7) & 127, c = (box >> 14) & 127, d = (box >> 21) & 127;
                    const bool ov = a < b;   // (an empty box has a = b = 0)
                    uint32_t w0 = 0u, w1 = 0u, w2 = 0u;
                    if (ov) {
                        const float pi = i == 0 ? 1.f : (i == 1 ? pc : ps);
                        const float m = A * pi * scale;
                        w0 = (uint32_t)__float2int_rn(m);
                        w1 = (uint32_t)__float2int_rn(m * qc);
                        w2 = (uint32_t)__float2int_rn(m * qs);
                    }
                    const bool z = ov && a == 0 && c == 0;
                    if (z) {
                        z0 += w0;
                        z1 += w1;
                        z2 += w2;
                    }
                    if (ov) {
                        if (!z) event3(S, a, c, w0, w1, w2);
                        if (b < kT) event3(S, b, c, 0u - w0, 0u - w1, 0u - w2);
                        if (d < kT) event3(S, a, d, 0u - w0, 0u - w1, 0u - w2);
                        if (b < kT && d < kT) event3(S, b, d, w0, w1, w2);
                    }
                }
                {
                    const uint32_t v0 = __reduce_add_sync(0xffffffffu, z0);
                    const uint32_t v1 = __reduce_add_sync(0xffffffffu, z1);
                    const uint32_t v2 = __reduce_add_sync(0xffffffffu, z2);
                    if (lane == 0 && (v0 | v1 | v2)) event3(S, 0, 0, v0, v1, v2);
                }
                __syncthreads();
                // ---- prefix along x: one row of one plane per thread, in
                // chunks of 4 with the next chunk loaded before this one is
                // stored (the loads need not wait for the stores)
                if (tid < 3 * kT) {
                    uint32_t* E = S.E[tid / kT];
                    const int y = tid % kT;
                    uint32_t cur[4], nxt[4], run = 0u;
#pragma unroll
                    for (int k = 0; k < 4; ++k) cur[k] = E[sw(y, k)];
#pragma unroll
                    for (int x0 = 0; x0 < kT; x0 += 4) {
                        if (x0 + 4 < kT) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) nxt[k] = E[sw(y, x0 + 4 + k)];
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            run += cur[k];
                            E[sw(y, x0 + k)] = run;
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
                    }
                }
                __syncthreads();
                // ---- prefix along y, in two steps: segment column sums ...
                {
                    uint32_t s0 = 0u, s1 = 0u, s2 = 0u;
#pragma unroll
                    for (int r = 0; r < kSegRows; ++r) {
                        const int o = sw(sg * kSegRows + r, cx);
                        s0 += S.E[0][o];
                        s1 += S.E[1][o];
                        s2 += S.E[2][o];
                    }
                    S.seg[sg][0][cx] = s0;
                    S.seg[sg][1][cx] = s1;
                    S.seg[sg][2][cx] = s2;
                }
                __syncthreads();
                // ... then this segment's rows from the sums of the segments above
                uint32_t run0 = 0u, run1 = 0u, run2 = 0u;
                for (int s = 0; s < sg; ++s) {
                    run0 += S.seg[s][0][cx];
                    run1 += S.seg[s][1][cx];
                    run2 += S.seg[s][2][cx];
                }
                // u_i(X), u'_i(X) with the constant factors and 1 / scale
                const float2 ux = S.ph[kT + cx];   // (cos a_X, sin a_X) of this column
                const float u = i == 0 ? 1.f : (i == 1 ? ux.x : -ux.y);
                const float up = i == 0 ? 0.f : (i == 1 ? ux.y : ux.x);
                const float ku = 0.25f * u * inv, kup = lamq * up * inv, kud = lamq * u * inv;
#pragma unroll
                for (int r = 0; r < kSegRows; ++r) {
                    const int y = sg * kSegRows + r;
                    const int o = sw(y, cx);
                    run0 += S.E[0][o];
                    run1 += S.E[1][o];
                    run2 += S.E[2][o];
                    const float2 vy = S.ph[y];   // (cos a_Y, sin a_Y)
                    const float f0 = (float)(int32_t)run0, f1 = (float)(int32_t)run1, f2 = (float)(int32_t)run2;
                    const float t = fmaf(-vy.y, f2, fmaf(vy.x, f1, f0));   // v . S_i.
                    const float tp = fmaf(vy.y, f1, vy.x * f2);            // v' . S_i.
                    ah[r] = fmaf(ku, t, ah[r]);
                    adx[r] = fmaf(kup, t, adx[r]);
                    ady[r] = fmaf(kud, tp, ady[r]);
                }
                __syncthreads();   // E and seg are rewritten by the next group
            }
            }   // passes
        }
        bb = be;
    }

    // ---- store: the group's partial planes, or (one group) the blended maps
    const int x = tx0 + cx;
    if (x >= sp.W) return;
    const size_t plane = (size_t)sp.W * sp.H;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        float* const dst =
            (G * K > 1 ? p.partial + ((size_t)(g * K + part) * 3 + f) * plane : p.out + (size_t)f * plane) + x;
#pragma unroll
        for (int r = 0; r < kSegRows; ++r) {
            const int y = ty0 + sg * kSegRows + r;
            const float v = f == 0 ? ah[r] : (f == 1 ? adx[r] : ady[r]);
            if (y < sp.H) dst[(size_t)y * sp.W] = G * K > 1 ? v : blend1(sp, x, y, f, v);
        }
    }
}

cudaError_t sat3_attributes() {
    static int attr[kMaxCachedDevices] = {};
    return cached_per_device(attr, [] {
               return cudaFuncSetAttribute(k_synth_sat3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(SatSmem)) == cudaSuccess ? 1 : -1;
           }) > 0
               ? cudaSuccess
               : cudaErrorInvalidValue;
}

}  // namespace

int synth_sat3_row_cap() { return kSatRowCap; }

// resident CTAs per SM from the SM's limits (shared memory, registers, threads)
static int synth_sat3_ctas_per_sm_query();
int synth_sat3_ctas_per_sm() {
    static int cache[kMaxCachedDevices] = {};
    return max(0, cached_per_device(cache, [] { return max(-1, synth_sat3_ctas_per_sm_query()); }));
}
static int synth_sat3_ctas_per_sm_query() {
    if (sat3_attributes() != cudaSuccess) return 0;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0;
    cudaFuncAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&a, k_synth_sat3) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 0;
    const int warps = kSatThreads / 32;
    const int regs_warp = ((a.numRegs * 32 + 255) / 256) * 256;
    int n = smem_sm / (int)(sizeof(SatSmem) + a.sharedSizeBytes + resv);
    n = min(n, regs_sm / (regs_warp * warps));
    n = min(n, thr_sm / kSatThreads);
    return n;
}

cudaError_t launch_synth_sat3(const TcItem* items, int n_items, const PatchDev* pdevs, const SynthParams* sps,
                              const BlendSpan* spans, int n_spans, cudaStream_t st) {
    cudaError_t e = sat3_attributes();
    if (e != cudaSuccess) return e;
    if (n_items > 0) {
        e = launch_pdl(k_synth_sat3, n_items, kSatThreads, sizeof(SatSmem), st, items, pdevs, sps);
        count_launches(1);
        if (e != cudaSuccess) return e;
    }
    if (n_spans > 0) return launch_blend_spans(spans, n_spans, pdevs, sps, st);
    return cudaGetLastError();
}

}  // namespace scwp
