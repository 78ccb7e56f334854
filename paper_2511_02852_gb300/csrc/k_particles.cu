// Wave-particle state kernels of the hybrid ocean (sm_103a):
//   advection + expiry + stable compaction  (Sec. 3.1 Lagrangian propagation,
//                                            Sec. 4.1 WP updates),
//   boundary injection and wake emission     (Sec. 3.3 Eqs. 15-17, Sec. 4.3),
//   per-bucket integer binning               (Sec. 4.2: the particles of a
//                                            bucket share radius and kernel).
// All particle state is integer (Q16.16 cell units); every decision is an
// integer test, so the state is bit-exact against any other implementation of
// the same rules.  No float atomics anywhere; integer atomics only for counts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "philox.h"

namespace scwp {
namespace {

constexpr int kTpb = 256;
constexpr int kItems = 4;                 // per thread in the compaction tiles
constexpr int kTileC = kTpb * kItems;     // 1024 particles per compaction block
constexpr int kSortItems = kSortTile / kTpb;
constexpr int kTileS = kSortTile;     // keys per sort block
constexpr int32_t kQi = 65536, kHalfi = 32768;

// Texel centres of [0, n) strictly inside (C - R, C + R) along one axis.
__device__ __forceinline__ int span_count(int32_t C, int32_t R, int n) {
    int64_t lo = (((int64_t)C - R - kHalfi) >> 16) + 1;
    int64_t hi = ((int64_t)C + R - kHalfi - 1) >> 16;
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
    return hi >= lo ? (int)(hi - lo + 1) : 0;
}

__device__ __forceinline__ int4 lookup_vq(const PatchDev& p, uint32_t bd) {
    const int b = (int)(bd >> 16), j = (int)(bd & 0xFFFFu);
    const int idx = j < p.nth ? b * p.nth + j : p.nb * p.nth + (j - p.nth);
    return p.vq[idx];
}

__device__ __forceinline__ float lookup_amp(const PatchDev& p, uint32_t bd) {
    const int b = (int)(bd >> 16), j = (int)(bd & 0xFFFFu);
    return j < p.nth ? p.amp[b * p.nth + j] : p.wake_amp;
}

// Block-wide exclusive scan of one value per thread (kTpb threads).
__device__ __forceinline__ uint32_t block_exscan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kTpb / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kTpb / 32) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[kTpb / 32 - 1];
    const uint32_t before = warp ? s_warp[warp - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

// ---- a3: advect, expire ------------------------------------------------------
__global__ void __launch_bounds__(kTpb) k_advect_flag(PatchDev p) {
    __shared__ uint32_t s_warp[kTpb / 32];
    pdl_enter();
    const int n = p.count[0];
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) p.count[2] = n;   // the pre-compaction count
        // this frame's statistics start from zero (evals, binned, live per
        // bucket, operand stages; the error flags stay)
        if (threadIdx.x < 2) p.stats[threadIdx.x] = 0ull;
        if (threadIdx.x <= p.nb) p.stats[3 + threadIdx.x] = 0ull;
        if (threadIdx.x == 0) p.stats[5 + p.nb] = 0ull;
    }
    const int base = blockIdx.x * kTileC;
    int32_t* X = p.x[p.cur];
    int32_t* Y = p.y[p.cur];
    const uint32_t* BD = p.bd[p.cur];
    uint32_t alive_cnt = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int i = base + threadIdx.x * kItems + k;
        if (i < n) {
            const uint32_t bd = BD[i];
            const int4 vq = lookup_vq(p, bd);
            const int32_t x = X[i] + vq.x, y = Y[i] + vq.y;
            X[i] = x;
            Y[i] = y;
            const int32_t R = p.bk[bd >> 16].R;
            const bool a = (span_count(x, R, p.W) > 0 && span_count(y, R, p.H) > 0) ||
                           (span_count(x - vq.z, R, p.W) > 0 && span_count(y - vq.w, R, p.H) > 0);
            p.flags[i] = a ? 1 : 0;
            alive_cnt += a ? 1u : 0u;
        }
    }
    uint32_t total;
    block_exscan(alive_cnt, s_warp, total);
    if (threadIdx.x == 0) p.blk[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kTpb) k_compact_scatter(PatchDev p) {
    __shared__ uint32_t s_warp[kTpb / 32];
    pdl_enter();
    const int base = blockIdx.x * kTileC;
    const int32_t* Xs = p.x[p.cur];
    const int32_t* Ys = p.y[p.cur];
    const uint32_t* Bs = p.bd[p.cur];
    int32_t* Xd = p.x[1 - p.cur];
    int32_t* Yd = p.y[1 - p.cur];
    uint32_t* Bd = p.bd[1 - p.cur];
    // only the pre-compaction live particles (count[2]) carry this frame's flags
    const int n = p.count[2];
    uint8_t f[kItems];
    int32_t xs[kItems], ys[kItems];
    uint32_t bs[kItems];
    uint32_t mine = 0;
    // every load first (one round trip): the earlier blocks' survivor
    // counts, this tile's flags and particles (dead ones too: few)
    uint32_t before = 0;
    for (int b = threadIdx.x; b < (int)blockIdx.x; b += kTpb) before += p.blk[b];
    const uint32_t blk_cnt = p.blk[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int i = base + threadIdx.x * kItems + k;
        f[k] = (i < n) ? p.flags[i] : 0;
        xs[k] = (i < n) ? Xs[i] : 0;
        ys[k] = (i < n) ? Ys[i] : 0;
        bs[k] = (i < n) ? Bs[i] : 0u;
        mine += f[k];
    }
    // survivors of the earlier blocks, summed by this block (integers: any
    // order); the last block also publishes the total as the new live count
    uint32_t blk_off;
    block_exscan(before, s_warp, blk_off);
    if (blockIdx.x + 1 == (unsigned)p.nblk_c && threadIdx.x == 0) {
        p.count[0] = (int32_t)(blk_off + blk_cnt);
        p.count[1] = (int32_t)(blk_off + blk_cnt);
    }
    if (blk_cnt == 0) return;
    uint32_t total;
    uint32_t off = block_exscan(mine, s_warp, total) + blk_off;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (f[k]) {
            Xd[off] = xs[k];
            Yd[off] = ys[k];
            Bd[off] = bs[k];
            ++off;
        }
    }
}

// ---- a4 + a5: injection and wake emission -------------------------------------
__device__ __forceinline__ void inject_body(const PatchDev& p, const InjectParams& ip) {
    const int base = p.count[1];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t want = (int64_t)base + ip.total;
        p.count[0] = (int32_t)(want > p.cap ? p.cap : want);
        if (want > p.cap) atomicOr(&p.stats[2], (unsigned long long)kErrCapacity);
    }
    int32_t* X = p.x[p.cur];
    int32_t* Y = p.y[p.cur];
    uint32_t* BD = p.bd[p.cur];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ip.total; e += gridDim.x * blockDim.x) {
        const int64_t idx = (int64_t)base + e;
        if (idx >= p.cap) break;
        int sidx = 0;
        while (sidx + 1 < ip.nseg && ip.seg[sidx + 1].first <= e) ++sidx;
        const Segment sg = ip.seg[sidx];
        const int le = e - sg.first;
        int32_t x, y;
        uint32_t bd;
        if (sg.s < 2) {
            const int g = le / sg.ndir, kk = le - g * sg.ndir;
            const int j = p.dirlist[(sg.bucket * 2 + sg.s) * p.nth + kk];
            const uint32_t ord = (uint32_t)(g * ip.nth + j);
            const U4 u = philox4x32_10(ip.frame, ip.patch, (uint32_t)sg.bucket | ((uint32_t)sg.s << 16),
                                       ord, ip.seed);
            const int4 vq = p.vq[sg.bucket * p.nth + j];
            const int32_t vn = sg.s == 0 ? vq.x : vq.y;
            const uint64_t avn = (uint64_t)(vn < 0 ? -(int64_t)vn : (int64_t)vn);
            const uint64_t len = (uint64_t)(sg.s == 0 ? ip.H : ip.W) * (uint64_t)kQi;
            const int32_t along = (int32_t)(((uint64_t)u.x * len) >> 32);
            const int32_t off = (int32_t)(((uint64_t)u.y * avn) >> 32);
            const int32_t far = (sg.s == 0 ? ip.W : ip.H) * kQi;
            const int32_t across = vn > 0 ? off : far - off;
            x = sg.s == 0 ? across : along;
            y = sg.s == 0 ? along : across;
            bd = ((uint32_t)sg.bucket << 16) | (uint32_t)j;
        } else {   // wake arms and ring ripples: positions placed on the host
            const int gi = sg.given + le;
            x = ip.gx[gi];
            y = ip.gy[gi];
            bd = ((uint32_t)sg.bucket << 16) | (uint32_t)(ip.nth + ip.ga[gi]);
        }
        X[idx] = x;
        Y[idx] = y;
        BD[idx] = bd;
    }
}

__global__ void __launch_bounds__(kTpb) k_inject(PatchDev p, InjectParams ip) { pdl_enter(); inject_body(p, ip); }

// the same with the frame's parameters in device memory (CUDA-graph replay)
__global__ void __launch_bounds__(kTpb) k_inject_dev(PatchDev p, const InjectParams* ip) { pdl_enter(); inject_body(p, *ip); }

// ---- a6: binning ---------------------------------------------------------------
// Block b takes the particles of sort tile b (kTileS / 2 particles, two
// bump keys each) and also produces the tile's histogram of the lowest key
// digit: the first radix pass needs no separate histogram launch.
__global__ void __launch_bounds__(kTpb) k_bin_keys(PatchDev p, uint32_t* keys, uint32_t* vals) {
    __shared__ unsigned long long s_ev[kTpb / 32];
    __shared__ unsigned int s_bin[kTpb / 32];
    __shared__ unsigned int s_live[kMaxBuckets];
    __shared__ uint32_t s_h[256];
    static_assert(kTpb == 256, "one digit counter per thread");
    pdl_enter();
    for (int i = threadIdx.x; i < p.nb; i += blockDim.x) s_live[i] = 0;
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int n = p.count[0];
    const int32_t* X = p.x[p.cur];
    const int32_t* Y = p.y[p.cur];
    const uint32_t* BD = p.bd[p.cur];
    unsigned long long ev = 0;
    unsigned int binned = 0;
    // the thread's kBinItems particles: every independent load first
    constexpr int kBinItems = (kTileS / 2) / kTpb;
    static_assert(kBinItems * kTpb == kTileS / 2, "whole particles per thread");
    const int i0 = blockIdx.x * (kTileS / 2) + threadIdx.x;
    uint32_t bd[kBinItems];
    int32_t px[kBinItems], py[kBinItems];
#pragma unroll
    for (int m = 0; m < kBinItems; ++m) {
        const int i = i0 + m * kTpb;
        bd[m] = i < n ? BD[i] : 0u;
        px[m] = i < n ? X[i] : 0;
        py[m] = i < n ? Y[i] : 0;
    }
#pragma unroll
    for (int m = 0; m < kBinItems; ++m) {
        const int i = i0 + m * kTpb;
        if (i >= n) continue;
        const int b = (int)(bd[m] >> 16);
        const int4 vq = lookup_vq(p, bd[m]);
        const BucketDev bk = p.bk[b];
        atomicAdd(&s_live[b], 1u);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int32_t cx = k ? px[m] - vq.z : px[m];
            const int32_t cy = k ? py[m] - vq.w : py[m];
            const int nx = span_count(cx, bk.R, p.W), ny = span_count(cy, bk.R, p.H);
            uint32_t key = (uint32_t)p.total_bins;
            if (nx > 0 && ny > 0) {
                const int bx = (int)(((int64_t)cx + bk.R) / bk.C);
                const int by = (int)(((int64_t)cy + bk.R) / bk.C);
                key = (uint32_t)(bk.base + by * bk.nbx + bx);
                ev += (unsigned long long)nx * (unsigned long long)ny;
                ++binned;
            }
            keys[2 * i + k] = key;
            vals[2 * i + k] = (uint32_t)(2 * i + k);
            atomicAdd(&s_h[key & 255u], 1u);
        }
    }
    // block reductions (integers: order-independent)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        ev += __shfl_down_sync(0xffffffffu, ev, o);
        binned += __shfl_down_sync(0xffffffffu, binned, o);
    }
    if (lane == 0) {
        s_ev[warp] = ev;
        s_bin[warp] = binned;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long e = 0;
        unsigned long long bb = 0;
        for (int w = 0; w < kTpb / 32; ++w) {
            e += s_ev[w];
            bb += s_bin[w];
        }
        if (e) {
            atomicAdd(&p.stats[0], e);
            atomicAdd(&p.stats[4 + p.nb], e);   // running total over frames
        }
        if (bb) atomicAdd(&p.stats[1], bb);
    }
    for (int i = threadIdx.x; i < p.nb; i += blockDim.x)
        if (s_live[i]) atomicAdd(&p.stats[3 + i], (unsigned long long)s_live[i]);
    p.hist[threadIdx.x * p.nblk_s + blockIdx.x] = s_h[threadIdx.x];   // (after the barrier above)
}

// LSD radix sort pass, 8-bit digit, stable.  Per-block digit histograms.
__global__ void __launch_bounds__(kTpb) k_radix_hist(const uint32_t* keys, const int32_t* count,
                                                     int shift, uint32_t* hist, int nblk) {
    __shared__ uint32_t s_h[256];
    pdl_enter();
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int n = 2 * count[0];
    const int base = blockIdx.x * kTileS;
    uint32_t key[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {   // all loads first: one round trip
        const int i = base + k * kTpb + threadIdx.x;
        key[k] = i < n ? keys[i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (base + k * kTpb + (int)threadIdx.x < n) atomicAdd(&s_h[(key[k] >> shift) & 255u], 1u);
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = s_h[threadIdx.x];
}

// exclusive scan of one digit's row of the digit-major histogram (block d
// scans hist[d * nblk .. + nblk)) and that digit's total into dtot[d]; each
// thread takes kScanItems consecutive entries per chunk, loaded together
constexpr int kScanItems = 4;

__global__ void __launch_bounds__(kTpb) k_scan_digits(uint32_t* hist, int nblk, uint32_t* dtot) {
    __shared__ uint32_t s_warp[kTpb / 32];
    pdl_enter();
    uint32_t* row = hist + (size_t)blockIdx.x * nblk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (int start = 0; start < nblk; start += kTpb * kScanItems) {
        const int i0 = start + threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            v[q] = i0 + q < nblk ? row[i0 + q] : 0u;
            sum += v[q];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t before = 0, all = 0;
#pragma unroll
        for (int w = 0; w < kTpb / 32; ++w) {
            const uint32_t t = s_warp[w];
            if (w < warp) before += t;
            all += t;
        }
        uint32_t run = carry + before + x - sum;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            if (i0 + q < nblk) row[i0 + q] = run;
            run += v[q];
        }
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

// stable scatter of one sort block's keys by digit: base of digit d = keys
// of smaller digits (exclusive scan of the 256 digit totals) + keys of
// digit d in earlier blocks (the scanned row)
__global__ void __launch_bounds__(kTpb) k_radix_scatter(const uint32_t* kin, const uint32_t* vin,
                                                        uint32_t* kout, uint32_t* vout,
                                                        const int32_t* count, int shift,
                                                        const uint32_t* hist, const uint32_t* dtot,
                                                        int nblk) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wc[kTpb / 32][256];
    __shared__ uint32_t s_dw[kTpb / 32];
    pdl_enter();
    const int n = 2 * count[0];
    const int base = blockIdx.x * kTileS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // every load of the block first (one round trip): the tile's keys and
    // ids, this digit's total and its count in the earlier tiles
    uint32_t kk[kSortItems], vv[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int i = base + k * kTpb + threadIdx.x;
        kk[k] = i < n ? kin[i] : 0u;
        vv[k] = i < n ? vin[i] : 0u;
    }
    const uint32_t h_before = hist[threadIdx.x * nblk + blockIdx.x];
    {
        // exclusive scan of the digit totals (one digit per thread)
        const uint32_t v = dtot[threadIdx.x];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_dw[warp] = x;
        __syncthreads();
        uint32_t before = 0;
#pragma unroll
        for (int w = 0; w < kTpb / 32; ++w)
            if (w < warp) before += s_dw[w];
        s_base[threadIdx.x] = before + x - v + h_before;
    }
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int i = base + k * kTpb + threadIdx.x;
        const bool act = i < n;
        const uint32_t key = kk[k], val = vv[k];
        const uint32_t d = act ? (key >> shift) & 255u : 0x100u + (uint32_t)warp;  // inactive sentinel
#pragma unroll
        for (int w = 0; w < kTpb / 32; ++w) s_wc[w][threadIdx.x] = 0;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (act && rank == 0) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        if (act) {
            uint32_t off = s_base[d] + rank;
            for (int w = 0; w < warp; ++w) off += s_wc[w][d];
            kout[off] = key;
            vout[off] = val;
        }
        __syncthreads();
        // (the next chunk reads s_base only after its first barrier)
        uint32_t add = 0;
#pragma unroll
        for (int w = 0; w < kTpb / 32; ++w) add += s_wc[w][threadIdx.x];
        s_base[threadIdx.x] += add;
    }
}

// One pass over the sorted (key, bump id) pairs:
//  * offsets[k] = first sorted position with key >= k (k = 0..total_bins):
//    position e is the answer for every k in (key[e-1], key[e]] (for e = 0
//    from 0, for e = n up to total_bins);
//  * the bump records in bin order (X, Y, signed amplitude, id and the
//    kernel phase pairs) of the entries with a bin (key < total_bins; the
//    others sort last).
__global__ void k_offsets_records(PatchDev p, const uint32_t* keys, const uint32_t* vals) {
    pdl_enter();
    const int n = 2 * p.count[0];
    const int32_t* X = p.x[p.cur];
    const int32_t* Y = p.y[p.cur];
    const uint32_t* BD = p.bd[p.cur];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= n; e += gridDim.x * blockDim.x) {
        const uint32_t key = e < n ? keys[e] : (uint32_t)p.total_bins;
        const int lo = e == 0 ? 0 : (int)keys[e - 1] + 1;
        const int hi = e == n ? p.total_bins : min((int)key, p.total_bins);
        for (int k = lo; k <= hi; ++k) p.offsets[k] = (uint32_t)e;
        if (e == n || key >= (uint32_t)p.total_bins) continue;
        const uint32_t id = vals[e];
        const int i = (int)(id >> 1);
        const bool trough = id & 1u;
        const uint32_t bd = BD[i];
        const int4 vq = lookup_vq(p, bd);
        const float A = lookup_amp(p, bd);
        const int32_t R = p.bk[bd >> 16].R;
        BumpRec r;
        r.x = trough ? X[i] - vq.z : X[i];
        r.y = trough ? Y[i] - vq.w : Y[i];
        r.amp = trough ? -A : A;
        r.id = id;
        // e^{-i pi (x mod 2R)/R}: exact integer reduction (2R < 2^31), then
        // sincospi of the FP32 quotient (within a few ulp of the exact one)
        const int32_t R2 = 2 * R;
        int32_t xm = r.x % R2, ym = r.y % R2;
        if (xm < 0) xm += R2;
        if (ym < 0) ym += R2;
        const float invR = p.bk[bd >> 16].invR;
        float sn, cs;
        sincospif((float)xm * invR, &sn, &cs);
        r.cx = cs;
        r.sx = -sn;
        sincospif((float)ym * invR, &sn, &cs);
        r.cy = cs;
        r.sy = -sn;
        p.rec[e] = r;
    }
}

}  // namespace

// ---- launchers -------------------------------------------------------------------
cudaError_t launch_advect_flag(const PatchDev& p, cudaStream_t st) {
    const cudaError_t e = launch_pdl(k_advect_flag, p.nblk_c, kTpb, 0, st, p);
    count_launches(1);
    return e;
}

cudaError_t launch_compact(const PatchDev& p, cudaStream_t st) {
    const cudaError_t e = launch_pdl(k_compact_scatter, p.nblk_c, kTpb, 0, st, p);
    count_launches(1);
    return e;
}

cudaError_t launch_inject(const PatchDev& p, const InjectParams& ip, cudaStream_t st) {
    int blocks = (ip.total + kTpb - 1) / kTpb;
    if (blocks < 1) blocks = 1;
    if (blocks > 1024) blocks = 1024;
    const cudaError_t e = launch_pdl(k_inject, blocks, kTpb, 0, st, p, ip);
    count_launches(1);
    return e;
}

cudaError_t launch_inject_dev(const PatchDev& p, const InjectParams* ip, cudaStream_t st) {
    const cudaError_t e = launch_pdl(k_inject_dev, 152 * 2, kTpb, 0, st, p, ip);
    count_launches(1);
    return e;
}

cudaError_t launch_bin(const PatchDev& p, cudaStream_t st) {
    // one block per sort tile: keys, vals and the first digit's histograms
    cudaError_t e = launch_pdl(k_bin_keys, p.nblk_s, kTpb, 0, st, p, p.keys[0], p.vals[0]);
    const int passes = (p.key_bits + 7) / 8;
    int src = 0;
    uint32_t* dtot = p.hist + (size_t)256 * p.nblk_s;
    for (int ps = 0; ps < passes && e == cudaSuccess; ++ps) {
        const int shift = 8 * ps;
        if (ps > 0)
            e = launch_pdl(k_radix_hist, p.nblk_s, kTpb, 0, st, (const uint32_t*)p.keys[src],
                           (const int32_t*)p.count, shift, p.hist, p.nblk_s);
        if (e == cudaSuccess) e = launch_pdl(k_scan_digits, 256, kTpb, 0, st, p.hist, p.nblk_s, dtot);
        if (e == cudaSuccess)
            e = launch_pdl(k_radix_scatter, p.nblk_s, kTpb, 0, st, (const uint32_t*)p.keys[src],
                           (const uint32_t*)p.vals[src], p.keys[1 - src], p.vals[1 - src],
                           (const int32_t*)p.count, shift, (const uint32_t*)p.hist, (const uint32_t*)dtot,
                           p.nblk_s);
        src = 1 - src;
    }
    int rb = (2 * p.cap + 1 + kTpb - 1) / kTpb;
    if (rb > 152 * 16) rb = 152 * 16;
    if (e == cudaSuccess)
        e = launch_pdl(k_offsets_records, rb, kTpb, 0, st, p, (const uint32_t*)p.keys[src],
                       (const uint32_t*)p.vals[src]);
    count_launches(1 + 3 * passes);
    return e;
}

int sorted_buffer_index(const PatchDev& p) { return ((p.key_bits + 7) / 8) & 1; }

}  // namespace scwp
