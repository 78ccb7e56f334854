// Wave-particle state kernels of the hybrid ocean (sm_103a):
//   advection + expiry + stable compaction  (Sec. 3.1 Lagrangian propagation,
//                                            Sec. 4.1 WP updates),
//   boundary injection and wake emission     (Sec. 3.3 Eqs. 15-17, Sec. 4.3),
//   per-bucket integer binning               (Sec. 4.2: the particles of a
//                                            bucket share radius and kernel):
//                                            a stable LSD radix sort of the bin
//                                            keys, one launch per 8-bit digit
//                                            (decoupled look-back for the
//                                            blocks' digit offsets).
// All particle state is integer (Q16.16 cell units); every decision is an
// integer test, so the state is bit-exact against any other implementation of
// the same rules.  No float atomics anywhere; integer atomics only for counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "internal.h"
#include "philox.h"

namespace scwp {
namespace {

constexpr int kTpb = 256;
constexpr int kItems = 4;                 // per thread in the compaction tiles
constexpr int kTileC = kTpb * kItems;     // 1024 particles per compaction block
constexpr int kTileS = kSortTile;     // keys per bin-key block
constexpr int32_t kQi = 65536, kHalfi = 32768;

// Texel centres of [0, n) strictly inside (C - R, C + R) along one axis.
__device__ __forceinline__ int span_count(int32_t C, int32_t R, int n) {
    int64_t lo = (((int64_t)C - R - kHalfi) >> 16) + 1;
    int64_t hi = ((int64_t)C + R - kHalfi - 1) >> 16;
    if (lo < 0) lo = 0;
    if (hi > n - 1) hi = n - 1;
    return hi >= lo ? (int)(hi - lo + 1) : 0;
}

// floor(x / d) and x - d floor(x / d) (in [0, d)) for d > 0: the quotient
// estimated in FP32 (relative error below 2^-21, so off by at most one where
// |x / d| < 2^19), then corrected in integers; exact integer division beyond
// that range.
__device__ __forceinline__ int32_t floor_divmod(int32_t x, int32_t d, int32_t& rem) {
    const float qf = floorf(__fdividef((float)x, (float)d));
    if (fabsf(qf) >= 524288.f) {   // 2^19: not in the estimate's range
        int32_t q = x / d, r = x % d;
        if (r < 0) {
            --q;
            r += d;
        }
        rem = r;
        return q;
    }
    int32_t q = (int32_t)qf;
    int64_t r = (int64_t)x - (int64_t)q * d;
    if (r < 0) {
        --q;
        r += d;
    } else if (r >= d) {
        ++q;
        r -= d;
    }
    rem = (int32_t)r;
    return q;
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
    // the thread's kItems consecutive particles: one 16-byte access per array
    // where all four are live (i0 is a multiple of 4)
    static_assert(kItems == 4, "16-byte accesses of four particles");
    const int i0 = base + threadIdx.x * kItems;
    const bool full = i0 + kItems <= n;
    int32_t xs[kItems], ys[kItems];
    uint32_t bs[kItems];
    if (full) {
        const int4 a = *reinterpret_cast<const int4*>(X + i0);
        const int4 b = *reinterpret_cast<const int4*>(Y + i0);
        const uint4 c = *reinterpret_cast<const uint4*>(BD + i0);
        xs[0] = a.x, xs[1] = a.y, xs[2] = a.z, xs[3] = a.w;
        ys[0] = b.x, ys[1] = b.y, ys[2] = b.z, ys[3] = b.w;
        bs[0] = c.x, bs[1] = c.y, bs[2] = c.z, bs[3] = c.w;
    } else {
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            xs[k] = i0 + k < n ? X[i0 + k] : 0;
            ys[k] = i0 + k < n ? Y[i0 + k] : 0;
            bs[k] = i0 + k < n ? BD[i0 + k] : 0u;
        }
    }
    uint32_t fl = 0u;   // the four alive flags, one byte each
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (i0 + k < n) {
            const uint32_t bd = bs[k];
            const int4 vq = lookup_vq(p, bd);
            const int32_t x = xs[k] + vq.x, y = ys[k] + vq.y;
            xs[k] = x;
            ys[k] = y;
            const int32_t R = p.bk[bd >> 16].R;
            const bool a = (span_count(x, R, p.W) > 0 && span_count(y, R, p.H) > 0) ||
                           (span_count(x - vq.z, R, p.W) > 0 && span_count(y - vq.w, R, p.H) > 0);
            fl |= (a ? 1u : 0u) << (8 * k);
            alive_cnt += a ? 1u : 0u;
            if (!full) {
                X[i0 + k] = x;
                Y[i0 + k] = y;
                p.flags[i0 + k] = a ? 1 : 0;
            }
        }
    }
    if (full) {
        *reinterpret_cast<int4*>(X + i0) = make_int4(xs[0], xs[1], xs[2], xs[3]);
        *reinterpret_cast<int4*>(Y + i0) = make_int4(ys[0], ys[1], ys[2], ys[3]);
        *reinterpret_cast<uint32_t*>(p.flags + i0) = fl;
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
    const int i0 = base + threadIdx.x * kItems;   // (a multiple of 4: 16-byte loads)
    if (i0 + kItems <= n) {
        const uint32_t fl = *reinterpret_cast<const uint32_t*>(p.flags + i0);
        const int4 a = *reinterpret_cast<const int4*>(Xs + i0);
        const int4 b = *reinterpret_cast<const int4*>(Ys + i0);
        const uint4 c = *reinterpret_cast<const uint4*>(Bs + i0);
        xs[0] = a.x, xs[1] = a.y, xs[2] = a.z, xs[3] = a.w;
        ys[0] = b.x, ys[1] = b.y, ys[2] = b.z, ys[3] = b.w;
        bs[0] = c.x, bs[1] = c.y, bs[2] = c.z, bs[3] = c.w;
#pragma unroll
        for (int k = 0; k < kItems; ++k) f[k] = (uint8_t)((fl >> (8 * k)) & 0xFFu);
    } else {
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int i = i0 + k;
            f[k] = (i < n) ? p.flags[i] : 0;
            xs[k] = (i < n) ? Xs[i] : 0;
            ys[k] = (i < n) ? Ys[i] : 0;
            bs[k] = (i < n) ? Bs[i] : 0u;
        }
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) mine += f[k];
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
// Block b takes the particles of key tile b (kTileS / 2 particles, two bump
// keys each) and adds the tile's counts of every sort pass's digit to the
// passes' digit totals, so the passes need no histogram launch; block b also
// clears the look-back words of sort-pass block b.
__global__ void __launch_bounds__(kTpb) k_bin_keys(PatchDev p, uint32_t* keys, uint32_t* vals, int passes) {
    __shared__ unsigned long long s_ev[kTpb / 32];
    __shared__ unsigned int s_bin[kTpb / 32];
    __shared__ unsigned int s_live[kMaxBuckets];
    __shared__ uint32_t s_h[kMaxSortPasses][256];
    static_assert(kTpb == 256, "one digit counter per thread");
    pdl_enter();
    for (int i = threadIdx.x; i < p.nb; i += blockDim.x) s_live[i] = 0;
#pragma unroll
    for (int ps = 0; ps < kMaxSortPasses; ++ps) s_h[ps][threadIdx.x] = 0;
    if ((int)blockIdx.x < p.nblk_o)
        for (int ps = 0; ps < passes; ++ps)
            p.sort_status[((size_t)ps * p.nblk_o + blockIdx.x) * 256 + threadIdx.x] = 0u;
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
    // the state packed per particle for the record pass (one 16-byte gather
    // per bump instead of three 4-byte ones)
#pragma unroll
    for (int m = 0; m < kBinItems; ++m) {
        const int i = i0 + m * kTpb;
        if (i < n) p.pk[i] = make_int4(px[m], py[m], (int)bd[m], 0);
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
                // (cx + R, cy + R > 0 here: the support reaches the patch)
                int32_t rx, ry;
                const int bx = floor_divmod(cx + bk.R, bk.C, rx);
                const int by = floor_divmod(cy + bk.R, bk.C, ry);
                key = (uint32_t)(bk.base + by * bk.nbx + bx);
                ev += (unsigned long long)nx * (unsigned long long)ny;
                ++binned;
            }
            keys[2 * i + k] = key;
            vals[2 * i + k] = (uint32_t)(2 * i + k);
            for (int ps = 0; ps < passes; ++ps) atomicAdd(&s_h[ps][(key >> (8 * ps)) & 255u], 1u);
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
    for (int ps = 0; ps < passes; ++ps)   // (after the barrier above)
        if (s_h[ps][threadIdx.x]) atomicAdd(&p.hist[ps * 256 + threadIdx.x], s_h[ps][threadIdx.x]);
}

// ---- one LSD radix-sort pass (8-bit digit, stable) -----------------------------
// Block-wide exclusive scan of one value per thread (kTpb threads); one
// barrier inside, s_warp free on entry.
__device__ __forceinline__ uint32_t block_exscan256(uint32_t v, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int w = 0; w < kTpb / 32; ++w)
        if (w < warp) before += s_warp[w];
    return before + x - v;
}

constexpr int kPassItems = kSortPassTile / kTpb;   // keys per thread
static_assert(kSortPassTile <= 65536, "tile ranks kept in 16 bits");
constexpr int kPassWarpKeys = 32 * kPassItems;     // keys per warp: a contiguous run of the tile
// look-back word: flag in the top two bits, a count below
constexpr uint32_t kLbAggregate = 1u << 30, kLbPrefix = 2u << 30, kLbCount = (1u << 30) - 1u;
constexpr long long kLbWaitCycles = 2000000000ll;  // the frame's limit: ~1 s at 2 GHz

constexpr int kLbBatch = 8;                        // look-back words read per round trip
// A look-back word carries its flag and count together, so plain relaxed
// accesses (atomic per word, no ordering against other data) suffice, and
// the loads of one batch overlap.
__device__ __forceinline__ void st_relaxed(uint32_t* a, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* a) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a));
    return v;
}

// One pass: a persistent grid whose blocks take tiles of kSortPassTile keys
// in ticket order.  A block ranks a tile's keys by digit (warp w holds the
// tile's keys [512 w, 512 w + 512) in order, so ranks follow the input
// order), publishes the tile's digit counts, and finds for each digit the
// keys of that digit in the earlier tiles by looking back over their
// published words (an inclusive prefix ends the walk) — the single-pass scan
// with decoupled look-back of Merrill and Garland.  Output position of a key:
// keys of smaller digits (the pass's digit totals, counted by the key kernel)
// + keys of its digit in earlier tiles + its rank in the tile.  The tile is
// reordered in shared memory first, so each digit's run leaves as
// consecutive stores.  A block only ever waits on tiles with earlier
// tickets, which running blocks hold or finished; every wait is bounded (the
// error flag records a timeout, after wait_cycles SM clocks).  The last block
// to finish clears the pass's digit totals and ticket for the next sort.
// Tickets start at tile first_tile: 0 in every frame; the failure-detection
// self-test starts at 1, so that tile 0's word is never published and the
// waits on it run out.  A block that gave up has summed a subset of the
// earlier tiles' counts, so its output positions stay below the true ones
// (in bounds, though the order is then wrong).
__global__ void __launch_bounds__(kTpb, 3) k_sort_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout,
                                                    uint32_t* vout, const int32_t* count, int shift,
                                                    uint32_t* dtot, uint32_t* status, uint32_t* ticket,
                                                    unsigned long long* err, long long wait_cycles,
                                                    int first_tile) {
    __shared__ uint32_t s_k[kSortPassTile];
    __shared__ uint32_t s_v[kSortPassTile];
    __shared__ uint32_t s_wh[kTpb / 32][256];   // per-warp digit counts, then the warp's offset in the digit
    __shared__ uint32_t s_ls[256];              // the digit's first position in the reordered tile
    __shared__ uint32_t s_gb[256];              // output position of reordered tile position 0 of the digit
    __shared__ uint32_t s_warp[kTpb / 32];
    __shared__ int s_bid;
    __shared__ bool s_last;
    pdl_enter();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = 2 * count[0];
    const uint32_t gd = block_exscan256(dtot[tid], s_warp);   // keys of smaller digits, all tiles
    const uint32_t lt = (1u << lane) - 1u;
    for (;;) {
        if (tid == 0) s_bid = (int)atomicAdd(ticket, 1u) + first_tile;
#pragma unroll
        for (int w = 0; w < kTpb / 32; ++w) s_wh[w][tid] = 0u;
        __syncthreads();   // (also: the previous tile's shared data is no longer read)
        const int bid = s_bid;
        const int base = bid * kSortPassTile;
        if (base >= n) break;   // (uniform)
        const int i0 = base + warp * kPassWarpKeys + lane;
        uint32_t kk[kPassItems], vv[kPassItems], rk[kPassItems / 2];   // ranks (< 4096): two per word
#pragma unroll
        for (int k = 0; k < kPassItems / 2; ++k) rk[k] = 0u;
#pragma unroll
        for (int k = 0; k < kPassItems; ++k) {   // every load first
            const int i = i0 + 32 * k;
            kk[k] = i < n ? kin[i] : 0u;
            vv[k] = i < n ? vin[i] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kPassItems; ++k) {
            const bool act = i0 + 32 * k < n;
            const uint32_t d = act ? (kk[k] >> shift) & 255u : 256u + (uint32_t)lane;   // inactive: alone
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t r = __popc(peers & lt);
            const uint32_t before = act ? s_wh[warp][d] : 0u;
            rk[k / 2] |= (before + r) << (16 * (k & 1));
            __syncwarp();
            if (act && r == 0) s_wh[warp][d] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // digit tid: each warp's offset within the tile's keys of the digit
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kTpb / 32; ++w) {
            const uint32_t x = s_wh[w][tid];
            s_wh[w][tid] = c;
            c += x;
        }
        // keys of digit tid in the earlier tiles: walk back over their words,
        // kLbBatch at a time, summing aggregates up to the nearest inclusive
        // prefix; an unpublished word ends the batch and is read again
        uint32_t excl = 0;
        uint32_t* mine = status + (size_t)bid * 256 + tid;
        if (bid == 0) {
            st_relaxed(mine, kLbPrefix | c);
        } else {
            st_relaxed(mine, kLbAggregate | c);
            const long long t0 = clock64();
            int j = bid - 1;   // the nearest word not yet summed
            for (;;) {
                uint32_t w[kLbBatch];
#pragma unroll
                for (int q = 0; q < kLbBatch; ++q)
                    w[q] = j - q >= 0 ? ld_relaxed(status + (size_t)(j - q) * 256 + tid) : kLbPrefix;
                bool done = false, stalled = false;
#pragma unroll
                for (int q = 0; q < kLbBatch; ++q) {
                    if (done || stalled) continue;
                    const uint32_t f = w[q] & ~kLbCount;
                    if (f == 0u) {
                        stalled = true;   // not yet published: read again from here
                    } else {
                        excl += w[q] & kLbCount;
                        --j;
                        done = f == kLbPrefix;
                    }
                }
                if (done) break;
                if (stalled && clock64() - t0 > wait_cycles) {
                    atomicOr(err, (unsigned long long)kErrTimeout);
                    break;
                }
            }
            st_relaxed(mine, kLbPrefix | (excl + c));
        }
        const uint32_t ls = block_exscan256(c, s_warp);   // (its barrier orders s_wh above)
        s_ls[tid] = ls;
        s_gb[tid] = gd + excl - ls;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPassItems; ++k) {
            if (i0 + 32 * k < n) {
                const uint32_t d = (kk[k] >> shift) & 255u;
                const uint32_t pos = s_ls[d] + s_wh[warp][d] + ((rk[k / 2] >> (16 * (k & 1))) & 0xFFFFu);
                s_k[pos] = kk[k];
                s_v[pos] = vv[k];
            }
        }
        __syncthreads();
        const int m = min(kSortPassTile, n - base);
        for (int i = tid; i < m; i += kTpb) {
            const uint32_t key = s_k[i];
            const uint32_t o = s_gb[(key >> shift) & 255u] + (uint32_t)i;
            kout[o] = key;
            vout[o] = s_v[i];
        }
    }
    // the last block out (every block has read the digit totals by then)
    // clears them and the ticket
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(ticket + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        dtot[tid] = 0u;
        if (tid == 0) {
            ticket[0] = 0u;
            ticket[1] = 0u;
        }
        __threadfence();
    }
}

int sort_pass_blocks_per_sm() {
    static int cache[kMaxCachedDevices];
    return cached_per_device(cache, [] {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sort_pass, kTpb, 0) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        return nb > 0 ? nb : -1;
    });
}

int sm_count() {
    static int cache[kMaxCachedDevices];
    return cached_per_device(cache, [] {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        return n > 0 ? n : -1;
    });
}

// One pass over the sorted (key, bump id) pairs:
//  * offsets[k] = first sorted position with key >= k (k = 0..total_bins):
//    position e is the answer for every k in (key[e-1], key[e]] (for e = 0
//    from 0, for e = n up to total_bins);
//  * the bump records in bin order (X, Y, signed amplitude, id and the
//    kernel phase pairs) of the entries with a bin (key < total_bins; the
//    others sort last).
constexpr int kRecItems = 4;   // sorted entries per thread and round, loads issued together

__global__ void __launch_bounds__(kTpb) k_offsets_records(PatchDev p, const uint32_t* keys, const uint32_t* vals) {
    // per warp: the 32 records of its 32 consecutive entries (1 KB), stored
    // out as 16-byte chunks of consecutive addresses (whole sectors)
    __shared__ uint4 s_rec[kTpb / 32][64];
    pdl_enter();
    const int n = 2 * p.count[0];
    const int4* PK = p.pk;
    const uint32_t tb = (uint32_t)p.total_bins;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int stride = gridDim.x * kTpb * kRecItems;
    // (the loop is uniform over a warp: its lanes take entries eb + lane)
    for (int eb = blockIdx.x * kTpb * kRecItems + (threadIdx.x & ~31); eb <= n; eb += stride) {
        const int e0 = eb + lane;
        uint32_t key[kRecItems], prev[kRecItems], id[kRecItems];
#pragma unroll
        for (int q = 0; q < kRecItems; ++q) {
            const int e = e0 + q * kTpb;
            key[q] = e < n ? keys[e] : tb;
            prev[q] = (e > 0 && e <= n) ? keys[e - 1] : 0u;
            id[q] = e < n ? vals[e] : 0u;
        }
        int4 st[kRecItems];
#pragma unroll
        for (int q = 0; q < kRecItems; ++q) {   // the particles' state: every gather first
            const int e = e0 + q * kTpb;
            const bool ok = e < n && key[q] < tb;
            st[q] = ok ? PK[id[q] >> 1] : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int q = 0; q < kRecItems; ++q) {
            const int e = e0 + q * kTpb;
            if (e <= n) {
                const int lo = e == 0 ? 0 : (int)prev[q] + 1;
                const int hi = e == n ? p.total_bins : min((int)key[q], p.total_bins);
                for (int k = lo; k <= hi; ++k) p.offsets[k] = (uint32_t)e;
            }
            const bool valid = e < n && key[q] < tb;
            uint4 r0 = make_uint4(0u, 0u, 0u, 0u), r1 = r0;
            if (valid) {
                const uint32_t bd = (uint32_t)st[q].z;
                const bool trough = id[q] & 1u;
                const int4 vq = lookup_vq(p, bd);
                const float A = lookup_amp(p, bd);
                const BucketDev& bk = p.bk[bd >> 16];
                const int32_t x = trough ? st[q].x - vq.z : st[q].x;
                const int32_t y = trough ? st[q].y - vq.w : st[q].y;
                // e^{-i pi (x mod 2R)/R}: exact integer reduction (2R < 2^31),
                // then sincospi of the FP32 quotient (within a few ulp of the
                // exact one)
                const int32_t R2 = 2 * bk.R;
                int32_t xm, ym;
                floor_divmod(x, R2, xm);
                floor_divmod(y, R2, ym);
                const float invR = bk.invR;
                float sx, cx, sy, cy;
                sincospif((float)xm * invR, &sx, &cx);
                sincospif((float)ym * invR, &sy, &cy);
                // BumpRec {x, cx, -sx, id, y, cy, -sy, amp}
                r0 = make_uint4((uint32_t)x, __float_as_uint(cx), __float_as_uint(-sx), id[q]);
                r1 = make_uint4((uint32_t)y, __float_as_uint(cy), __float_as_uint(-sy), __float_as_uint(trough ? -A : A));
            }
            s_rec[warp][2 * lane] = r0;
            s_rec[warp][2 * lane + 1] = r1;
            __syncwarp();
            // entries eb + q kTpb + r, r = 0 .. 31; chunk c (16 bytes) belongs
            // to entry r = c / 2 and leaves only if that entry has a record
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
            uint4* const dst = reinterpret_cast<uint4*>(p.rec + (eb + q * kTpb));
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                if ((vm >> (c >> 1)) & 1u) dst[c] = s_rec[warp][c];
            }
            __syncwarp();
        }
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
    // one block per key tile: keys, ids and every pass's digit totals
    const int passes = (p.key_bits + 7) / 8;
    // the sort passes: a persistent grid of the blocks that fit at once
    const int per_sm = sort_pass_blocks_per_sm(), sms = sm_count();
    const int grid = std::max(1, std::min(p.nblk_o, std::max(1, per_sm) * std::max(1, sms)));
    cudaError_t e = launch_pdl(k_bin_keys, p.nblk_s, kTpb, 0, st, p, p.keys[0], p.vals[0], passes);
    int src = 0;
    for (int ps = 0; ps < passes && e == cudaSuccess; ++ps) {
        e = launch_pdl(k_sort_pass, grid, kTpb, 0, st, (const uint32_t*)p.keys[src],
                       (const uint32_t*)p.vals[src], p.keys[1 - src], p.vals[1 - src], (const int32_t*)p.count,
                       8 * ps, p.hist + 256 * ps, p.sort_status + (size_t)ps * p.nblk_o * 256,
                       p.sort_ticket + 2 * ps, p.stats + 2, kLbWaitCycles, 0);
        src = 1 - src;
    }
    int rb = (2 * p.cap + 1 + kTpb * kRecItems - 1) / (kTpb * kRecItems);
    rb = std::max(1, std::min(rb, std::max(1, sm_count()) * 8));
    if (e == cudaSuccess)
        e = launch_pdl(k_offsets_records, rb, kTpb, 0, st, p, (const uint32_t*)p.keys[src],
                       (const uint32_t*)p.vals[src]);
    count_launches(2 + passes);
    return e;
}

int sorted_buffer_index(const PatchDev& p) { return ((p.key_bits + 7) / 8) & 1; }

cudaError_t launch_sort_stall(const PatchDev& p, long long wait_cycles, cudaStream_t st) {
    // the frame's keys and digit totals, then the first pass with tile 0
    // never taken: every block that looks back to it waits wait_cycles
    const int passes = (p.key_bits + 7) / 8;
    const int per_sm = sort_pass_blocks_per_sm(), sms = sm_count();
    const int grid = std::max(1, std::min(p.nblk_o, std::max(1, per_sm) * std::max(1, sms)));
    cudaError_t e = launch_pdl(k_bin_keys, p.nblk_s, kTpb, 0, st, p, p.keys[0], p.vals[0], passes);
    if (e == cudaSuccess)
        e = launch_pdl(k_sort_pass, grid, kTpb, 0, st, (const uint32_t*)p.keys[0], (const uint32_t*)p.vals[0],
                       p.keys[1], p.vals[1], (const int32_t*)p.count, 0, p.hist, p.sort_status, p.sort_ticket,
                       p.stats + 2, wait_cycles, 1);
    count_launches(2);
    return e;
}

}  // namespace scwp
