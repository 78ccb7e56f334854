// Summed-area synthesis of the wave-particle maps: the per-bucket kernel
// sums of Sec. 4.2 (kernel reading O11, analytic displacement O12) computed
// from the structure of the raised-cosine kernel instead of one evaluation
// per (bump, texel) pair.
//
// On its support |X - x_b| < R a bump's x factor is
//     1 + cos(pi (X - x_b)/R) = u(X) . p_b,   sin(pi (X - x_b)/R) = u'(X) . p_b,
// with u(X) = (1, cos a_X, -sin a_X), u'(X) = (0, sin a_X, cos a_X),
// a_X = pi (X mod 2R)/R and p_b = (1, c_b, s_b) = (1, e^{-i pi (x_b mod 2R)/R})
// (the bump record's phase pair); likewise v(Y), v'(Y), q_b for y.  Within a
// tile the support is a box [alpha_b, beta_b) x [gamma_b, delta_b) of texel
// indices, so
//     h(X, Y)  = 1/4     sum_ij u_i(X)  v_j(Y)  S_ij(X, Y),
//     Dx(X, Y) = lam/4   sum_ij u'_i(X) v_j(Y)  S_ij(X, Y),
//     Dy(X, Y) = lam/4   sum_ij u_i(X)  v'_j(Y) S_ij(X, Y),
//     S_ij(X, Y) = sum_b A_b p_i(b) q_j(b) [alpha_b <= X < beta_b][gamma_b <= Y < delta_b],
// and S_ij is the 2-D inclusive prefix sum of a difference array that holds
// +-A_b p_i q_j at the four corners of each box (corners at index 64 fall
// outside the tile and are dropped).  These are the same sums as the direct
// gather in another association.  Per (tile, bucket) the work is four corner
// events per bump, two prefix passes and a 3 x 3 contraction per texel: it
// no longer grows with the number of bumps covering a texel.
//
// Exactness of the prefix sums: the corner weights are rounded once to
// 32-bit integers with a per-pass scale 2^30 / (1.001 m A_max), m the
// candidate bumps of the pass and A_max the bucket's bound on |A| (its
// direction amplitudes, and the wake's).  Every S_ij then fits in 31 bits, the
// events accumulate exactly in any order (integer shared-memory atomics:
// deterministic results), and the prefix sums are exact modulo 2^32 (their
// intermediate values may wrap; the final ones do not).  The contraction is
// FP32.  The rounding error of a weight is at most 2^-31 m A_max; those of the
// n candidates covering a texel add up to about sqrt(n) m A_max 2^-31, so a
// (tile, bucket) whose n is large against the bound the host sets per bucket
// (BucketDev::sat_c) is split into passes of fewer candidates, each with its
// own scale, prefix sums and contraction (the FP32 accumulators carry over).
//
// Organisation: a persistent grid, one 1024-thread CTA per SM, pulls (tile,
// bucket group) items from a work queue (an atomic ticket over the plan's
// heaviest-first order; the last CTA to finish resets the queue for the next
// launch, so no CTA ever waits on another).  All nine S_ij planes of a
// bucket live in shared memory at once (144 KB), so each candidate bump
// enters exactly once per pass.  Per item, the buckets' bin geometry and the
// bin rows that reach the tile are read once into a row table (a bucket with
// more rows than the table spans several segments, each a pass of its own).
// Within a pass each thread takes the candidates c0 + tid, c0 + tid + 1024,
// ... on its own, with no barrier until the pass ends: it finds a
// candidate's bin row (a binary search of the row table) and copies the
// record with asynchronous 16-byte copies (cp.async) into its own slot of
// two, one candidate ahead, so the copy of its next candidate (of this pass,
// or the first of the next pass) overlaps the current one's events, and the
// next pass's first copies overlap the prefix passes.  As each thread reads
// only the slots it filled, no barrier guards them.  Each thread clips its
// candidate's support box to the tile and adds the nine weights at up to
// four corners; bumps whose box starts at the tile's first texel in both axes
// (every bump covering the whole tile among them) sum their (0, 0) corner in
// registers, added by one warp reduction per pass.  Then the x prefix (one
// row of one plane per thread), the y prefix (one column of one plane per
// thread, stored only at the first row of each 4-row segment of the
// contraction) and the contraction (one column of a segment per thread),
// which finishes the y prefix of the segment's other rows in registers and
// zeroes every difference-array element it reads, so no pass needs a
// clearing phase.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "blend_dev.cuh"
#include "internal.h"

namespace scwp {
namespace {

constexpr int kT = 64;                       // tile side in texels
constexpr int kSatThreads = 1024;
constexpr int kSegs = kSatThreads / kT;      // row segments of the contraction
constexpr int kSegRows = kT / kSegs;         // rows per segment
constexpr int kPlanes = 9;                   // S_ij, plane 3 i + j
constexpr int kScanThreads = kPlanes * kT;   // one row (or column) scan per thread
constexpr int kRowCap = 256;                 // bin rows held at once (all segments of a batch)
constexpr int kMaxSeg = 64;                  // segments per batch
constexpr int32_t kQs = 65536, kHalfs = 32768;
static_assert(kSegs * kSegRows == kT && kSegs == 16, "contraction mapping");
static_assert(kScanThreads % 32 == 0 && kScanThreads + 128 <= kSatThreads, "scan warps and helper warps");

struct SatSmem {
    uint32_t E[kPlanes][kT * kT];         // difference arrays, then prefix sums; zero between passes
    alignas(128) BumpRec raw[2][kSatThreads];   // two record slots per thread
    float2 ph[2][2 * kT];                 // texel phases (cos, sin) a of a segment's bucket: rows, then columns
    int32_t rs[kRowCap];                  // first record of each bin row of the batch
    int32_t cum[kRowCap];                 // candidates of the segment before the row
    // the item's buckets
    int32_t mR[kMaxBuckets], mC[kMaxBuckets], mnbx[kMaxBuckets], mbase[kMaxBuckets];
    int32_t mbx_lo[kMaxBuckets], mbx_hi[kMaxBuckets], mby_lo[kMaxBuckets], mnrows[kMaxBuckets];
    float mamax[kMaxBuckets], msatc[kMaxBuckets];
    // the batch's segments: bucket (item-relative), first row, first table
    // row, candidates, candidates per pass
    int32_t sgb[kMaxSeg], sgr0[kMaxSeg], sgrb[kMaxSeg + 1], sgnc[kMaxSeg], sgm[kMaxSeg];
    int32_t item, patch, nseg, bt_next, bt_r0, pad;
    alignas(16) unsigned char pd[sizeof(PatchDev)];
    alignas(16) unsigned char spd[sizeof(SynthParams)];
};
static_assert(sizeof(SatSmem) <= 227 * 1024, "shared memory of one CTA");
static_assert(sizeof(BumpRec) == 32, "32-byte records (two 16-byte copies)");

// element (row y, column x) of a 64 x 64 plane: columns XOR-swizzled by the
// row so that a warp walking a row (one row per lane) or a column (one
// column per lane) touches 32 different banks
__device__ __forceinline__ int sw(int y, int x) { return y * kT + (x ^ (y & 31)); }

__device__ __forceinline__ int clamp_t(int t) { return min(max(t, 0), kT); }

// the nine components of one corner event
__device__ __forceinline__ void event9(SatSmem& S, int x, int y, const uint32_t (&w)[kPlanes], bool neg) {
    const int o = sw(y, x);
#pragma unroll
    for (int k = 0; k < kPlanes; ++k) atomicAdd(&S.E[k][o], neg ? 0u - w[k] : w[k]);
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

// passes of segment candidates: a (tile, bucket) of n candidates goes in
// ceil(n^1.5 / sat_c) passes, so that the integer rounding of its corner
// weights stays within the bound the host set
__device__ __forceinline__ int pass_size(int ncand, float satc) {
    const float nf = (float)ncand;
    const int kch = max(1, (int)ceilf(nf * sqrtf(nf) / satc));
    return (ncand + kch - 1) / kch;
}

// ---- asynchronous 16-byte copies global -> shared (L2 only)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most one group of this thread's copies is still in flight
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Record slots are 32 bytes per thread.  Threads with bit 2 of their index
// set keep the two 16-byte halves of their record in swapped order, so that
// the eight threads of a quarter warp (whose 16-byte accesses one shared
// memory wavefront serves) touch eight different 16-byte bank groups: the
// copies into the slots and the reads from them are free of bank conflicts
// (with the halves in order, threads t and t + 4 met in the same banks).
__device__ __forceinline__ int half_swap(int tid) { return (tid >> 2) & 1; }

// A pass of this CTA's part: segment s, its candidates [c0, c1); s < 0: none.
struct Pass {
    int s, c0, c1;
};

__device__ __forceinline__ Pass make_pass(const SatSmem& S, int s, int c0) {
    return Pass{s, c0, min(S.sgnc[s], c0 + S.sgm[s])};
}

// The part's first pass of segments s0, s0 + 1, ... with candidates.
__device__ __forceinline__ Pass first_pass_from(const SatSmem& S, int s0, int nseg, int part) {
    for (int s = s0; s < nseg; ++s)
        if (part * S.sgm[s] < S.sgnc[s]) return make_pass(S, s, part * S.sgm[s]);
    return Pass{-1, 0, 0};
}

// The pass after P in this part's order: the part's next pass of the same
// segment (parts take every K-th pass), else the first of a later segment.
__device__ __forceinline__ Pass next_pass(const SatSmem& S, Pass P, int nseg, int K, int part) {
    const int c0 = P.c0 + K * S.sgm[P.s];
    if (c0 < S.sgnc[P.s]) return make_pass(S, P.s, c0);
    return first_pass_from(S, P.s + 1, nseg, part);
}

// This thread's copy of candidate j (of the segment whose table rows are
// [lo, hi]) into its slot `slot`; returns the candidate's row.  The row is
// the last one that starts at or before j (empty rows start where the next
// one does).
__device__ __forceinline__ int fetch_rows(SatSmem& S, const BumpRec* rec, int lo, int hi, int j, int slot, int tid) {
    if (lo < hi && S.cum[lo + 1] > j) hi = lo;   // still the row of the hint
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.cum[mid] <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    const unsigned char* src = reinterpret_cast<const unsigned char*>(rec + S.rs[lo] + (j - S.cum[lo]));
    unsigned char* dst = reinterpret_cast<unsigned char*>(&S.raw[slot][tid]);
    const int hs = half_swap(tid);
    cp_async16(dst + 16 * hs, src);
    cp_async16(dst + 16 * (hs ^ 1), src + 16);
    return lo;
}

// The record of this thread's slot (its two 16-byte halves in the order
// half_swap gives).
__device__ __forceinline__ BumpRec read_slot(const SatSmem& S, int slot, int tid) {
    const uint4* q = reinterpret_cast<const uint4*>(&S.raw[slot][tid]);
    const int hs = half_swap(tid);
    const uint4 a = q[hs], b = q[hs ^ 1];
    BumpRec r;
    r.x = (int32_t)a.x;
    r.cx = __uint_as_float(a.y);
    r.sx = __uint_as_float(a.z);
    r.id = a.w;
    r.y = (int32_t)b.x;
    r.cy = __uint_as_float(b.y);
    r.sy = __uint_as_float(b.z);
    r.amp = __uint_as_float(b.w);
    return r;
}

__global__ void __launch_bounds__(kSatThreads, 1) k_synth_sat(const TcItem* items, int n_items,
                                                            const PatchDev* pdevs, const SynthParams* sps,
                                                            unsigned int* queue) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SatSmem& S = *reinterpret_cast<SatSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // contraction: this thread owns texel column cx of rows sg*4 .. sg*4 + 3
    const int cx = tid & (kT - 1), sg = tid / kT;
    pdl_enter();
    // E starts zeroed, and every pass leaves it zeroed again
    {
        uint4* e4 = reinterpret_cast<uint4*>(&S.E[0][0]);
        for (int k = tid; k < kPlanes * kT * kT / 4; k += kSatThreads) e4[k] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        S.item = (int)atomicAdd(queue, 1u);
        S.patch = -1;
    }
    __syncthreads();
    for (;;) {
        const int ti = S.item;
        if (ti >= n_items) break;
        const TcItem it = items[ti];
        if (it.patch != S.patch) {   // (uniform) items of one patch share its descriptors
            static_assert(sizeof(PatchDev) % 4 == 0 && sizeof(SynthParams) % 4 == 0, "descriptor copy");
            const uint32_t* a = reinterpret_cast<const uint32_t*>(pdevs + it.patch);
            const uint32_t* b = reinterpret_cast<const uint32_t*>(sps + it.patch);
            for (int k = tid; k < (int)(sizeof(PatchDev) / 4); k += kSatThreads)
                reinterpret_cast<uint32_t*>(S.pd)[k] = a[k];
            for (int k = tid; k < (int)(sizeof(SynthParams) / 4); k += kSatThreads)
                reinterpret_cast<uint32_t*>(S.spd)[k] = b[k];
            __syncthreads();
            if (tid == 0) S.patch = it.patch;
        }
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
        // ---- the item's buckets, one thread each: bins hold x_b + R in
        // [bx C, (bx + 1) C); the bin rows and columns that reach the tile
        for (int t = tid; t < nbk; t += kSatThreads) {
            const BucketDev bk = p.bk[b_begin + t];
            const float amax = p.amax[b_begin + t];
            const int bx_lo = (int)((int64_t)X0 / bk.C);
            const int bx_hi = min((int)(((int64_t)X1 + 2 * (int64_t)bk.R - 1) / bk.C), bk.nbx - 1);
            const int by_lo = (int)((int64_t)Y0 / bk.C);
            const int by_hi = min((int)(((int64_t)Y1 + 2 * (int64_t)bk.R - 1) / bk.C), bk.nby - 1);
            S.mR[t] = bk.R;
            S.mC[t] = bk.C;
            S.mnbx[t] = bk.nbx;
            S.mbase[t] = bk.base;
            S.mbx_lo[t] = bx_lo;
            S.mbx_hi[t] = bx_hi;
            S.mby_lo[t] = by_lo;
            S.mnrows[t] = (bx_lo > bx_hi || by_lo > by_hi || !(amax > 0.f)) ? 0 : by_hi - by_lo + 1;
            S.mamax[t] = amax;
            S.msatc[t] = bk.sat_c;
        }
        float ah[kSegRows], adx[kSegRows], ady[kSegRows];
#pragma unroll
        for (int r = 0; r < kSegRows; ++r) ah[r] = adx[r] = ady[r] = 0.f;
        int t_next = 0, sub_r0 = 0;   // the first bucket (and its row) not yet batched
        for (;;) {
            __syncthreads();   // bucket table written; the previous batch is done with the row table
            // ---- a batch: segments (bucket, row range) whose bin rows fit the row table
            // (a bucket with more rows than the table spans several segments)
            if (tid == 0) {
                int n = 0, rows = 0, t = t_next, r0 = sub_r0;
                while (t < nbk && n < kMaxSeg) {
                    const int left = S.mnrows[t] - r0;
                    if (left <= 0) {
                        ++t;
                        r0 = 0;
                        continue;
                    }
                    const int take = min(left, kRowCap - rows);
                    if (take <= 0) break;
                    S.sgb[n] = t;
                    S.sgr0[n] = r0;
                    S.sgrb[n] = rows;
                    rows += take;
                    ++n;
                    r0 += take;
                    if (r0 >= S.mnrows[t]) {
                        ++t;
                        r0 = 0;
                    }
                }
                S.sgrb[n] = rows;
                S.nseg = n;
                S.bt_next = t;
                S.bt_r0 = r0;
            }
            __syncthreads();
            const int nseg = S.nseg;
            t_next = S.bt_next;
            sub_r0 = S.bt_r0;
            if (nseg == 0) break;
            // ---- the batch's row table: first record and length of every row
            const int nq = S.sgrb[nseg];
            for (int q = tid; q < nq; q += kSatThreads) {
                int s = 0;
                while (S.sgrb[s + 1] <= q) ++s;
                const int t = S.sgb[s];
                const int r = S.sgr0[s] + (q - S.sgrb[s]);
                const int key0 = S.mbase[t] + (S.mby_lo[t] + r) * S.mnbx[t];
                const int s0 = (int)p.offsets[key0 + S.mbx_lo[t]];
                S.rs[q] = s0;
                S.cum[q] = (int)p.offsets[key0 + S.mbx_hi[t] + 1] - s0;   // row length for now
            }
            __syncthreads();
            // exclusive prefix of the row lengths within each segment (warp w:
            // segments w, w + 32)
            for (int s = warp; s < nseg; s += kSatThreads / 32) {
                const int q0 = S.sgrb[s], q1 = S.sgrb[s + 1];
                uint32_t carry = 0u;
                for (int q = q0; q < q1; q += 32) {
                    const uint32_t l = q + lane < q1 ? (uint32_t)S.cum[q + lane] : 0u;
                    const uint32_t inc = warp_scan(l, lane);
                    if (q + lane < q1) S.cum[q + lane] = (int32_t)(carry + inc - l);
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
                if (lane == 0) {
                    S.sgnc[s] = (int32_t)carry;
                    S.sgm[s] = carry ? pass_size((int)carry, S.msatc[S.sgb[s]]) : 0;
                }
            }
            __syncthreads();

            // ---- the batch's passes of this part.  Invariant at a pass's
            // start: if this thread has a candidate in it (c0 + tid < c1),
            // its record is on the way into slot k (the last commit group).
            Pass P = first_pass_from(S, 0, nseg, part);
            int k = 0;
            if (P.s >= 0 && P.c0 + tid < P.c1) fetch_rows(S, p.rec, S.sgrb[P.s], S.sgrb[P.s + 1] - 1, P.c0 + tid, k, tid);
            cp_async_commit();
            while (P.s >= 0) {
                const int s = P.s;
                const int t = S.sgb[s];
                const int b = b_begin + t;
                const int R = S.mR[t];
                float2* const ph = S.ph[s & 1];
                const float bound = 1.001f * (float)(P.c1 - P.c0) * S.mamax[t];   // >= every |S_ij| of the pass
                const float scale = 1073741824.f / bound;                        // 2^30 / bound
                const float inv = bound * (1.f / 1073741824.f);                  // 1 / scale
                if (tid == 0) atomicAdd(p.stats + 5 + p.nb, (unsigned long long)(P.c1 - P.c0));
                const Pass Pn = next_pass(S, P, nseg, K, part);
                const bool pre = Pn.s >= 0 && Pn.c0 + tid < Pn.c1;   // a candidate in the next pass
                // the (0, 0) corner, shared by every bump whose box starts at
                // the tile's first texel in both axes: per-thread sums
                uint32_t z[kPlanes];
#pragma unroll
                for (int q = 0; q < kPlanes; ++q) z[q] = 0u;
                if (P.c0 + tid >= P.c1) {   // none here: the next pass's first copy
                    if (pre) fetch_rows(S, p.rec, S.sgrb[Pn.s], S.sgrb[Pn.s + 1] - 1, Pn.c0 + tid, k, tid);
                    cp_async_commit();
                }
                // the row of this thread's next candidate is at or after that of its current one
                int q = S.sgrb[s];
                const int qe = S.sgrb[s + 1] - 1;
                for (int j = P.c0 + tid; j < P.c1; j += kSatThreads) {
                    // the copy of this thread's next candidate starts now
                    if (j + kSatThreads < P.c1)
                        q = fetch_rows(S, p.rec, q, qe, j + kSatThreads, k ^ 1, tid);
                    else if (pre)
                        fetch_rows(S, p.rec, S.sgrb[Pn.s], S.sgrb[Pn.s + 1] - 1, Pn.c0 + tid, k ^ 1, tid);
                    cp_async_commit();
                    cp_async_wait_prev();   // this candidate's record has landed
                    const BumpRec rc = read_slot(S, k, tid);
                    k ^= 1;
                    // texel t of the tile is inside iff x_b - R < X0 + t Q < x_b + R
                    const int a = clamp_t(((rc.x - R - X0) >> 16) + 1);
                    const int bb = clamp_t(-((X0 - rc.x - R) >> 16));
                    const int c = clamp_t(((rc.y - R - Y0) >> 16) + 1);
                    const int d = clamp_t(-((Y0 - rc.y - R) >> 16));
                    if (a < bb && c < d) {
                        const float A = rc.amp;
                        const float m0 = A * scale, m1 = A * rc.cx * scale, m2 = A * rc.sx * scale;
                        uint32_t w[kPlanes];
                        w[0] = (uint32_t)__float2int_rn(m0);
                        w[1] = (uint32_t)__float2int_rn(m0 * rc.cy);
                        w[2] = (uint32_t)__float2int_rn(m0 * rc.sy);
                        w[3] = (uint32_t)__float2int_rn(m1);
                        w[4] = (uint32_t)__float2int_rn(m1 * rc.cy);
                        w[5] = (uint32_t)__float2int_rn(m1 * rc.sy);
                        w[6] = (uint32_t)__float2int_rn(m2);
                        w[7] = (uint32_t)__float2int_rn(m2 * rc.cy);
                        w[8] = (uint32_t)__float2int_rn(m2 * rc.sy);
                        if (a == 0 && c == 0) {
#pragma unroll
                            for (int q = 0; q < kPlanes; ++q) z[q] += w[q];
                        } else {
                            event9(S, a, c, w, false);
                        }
                        if (bb < kT) event9(S, bb, c, w, true);
                        if (d < kT) event9(S, a, d, w, true);
                        if (bb < kT && d < kT) event9(S, bb, d, w, false);
                    }
                }
                // (all threads converge here: one reduction per warp and pass)
#pragma unroll
                for (int q = 0; q < kPlanes; ++q) z[q] = __reduce_add_sync(0xffffffffu, z[q]);
                if (lane == 0) {
#pragma unroll
                    for (int q = 0; q < kPlanes; ++q)
                        if (z[q]) atomicAdd(&S.E[q][0], z[q]);
                }
                __syncthreads();   // E holds the pass's events
                if (tid < kScanThreads) {
                    // ---- prefix along x: one row of one plane per thread, in
                    // chunks of 4 with the next chunk loaded before this one
                    // is stored (the loads need not wait for the stores)
                    uint32_t* E = S.E[tid / kT];
                    const int y = tid % kT;
                    uint32_t cr[4], nx[4], run = 0u;
#pragma unroll
                    for (int k = 0; k < 4; ++k) cr[k] = E[sw(y, k)];
#pragma unroll
                    for (int x0 = 0; x0 < kT; x0 += 4) {
                        if (x0 + 4 < kT) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) nx[k] = E[sw(y, x0 + 4 + k)];
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            run += cr[k];
                            E[sw(y, x0 + k)] = run;
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) cr[k] = nx[k];
                    }
                } else if (tid < kScanThreads + 2 * kT) {
                    // ---- meanwhile spare warps fetch this bucket's texel phases
                    const int h = tid - kScanThreads;
                    ph[h] = p.phase[(size_t)b * p.phase_len + (h < kT ? ty0 + h : tx0 + (h - kT))];
                }
                __syncthreads();
                if (tid < kScanThreads) {
                    // ---- prefix along y: one column of one plane per thread.
                    // Only the first row of each contraction segment gets its
                    // prefix sum; the contraction adds the segment's other
                    // rows to it in registers
                    static_assert(kSegRows == 4, "one stored row per 4-row segment");
                    uint32_t* E = S.E[tid / kT];
                    const int x = tid % kT;
                    uint32_t cr[4], nx[4], run = 0u;
#pragma unroll
                    for (int k = 0; k < 4; ++k) cr[k] = E[sw(k, x)];
#pragma unroll
                    for (int y0 = 0; y0 < kT; y0 += 4) {
                        if (y0 + 4 < kT) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) nx[k] = E[sw(y0 + 4 + k, x)];
                        }
                        run += cr[0];
                        E[sw(y0, x)] = run;
                        run += cr[1] + cr[2] + cr[3];
#pragma unroll
                        for (int k = 0; k < 4; ++k) cr[k] = nx[k];
                    }
                }
                __syncthreads();
                // ---- this thread's texels contracted; each element of E is
                // zeroed once read (the next pass starts from a cleared array).
                // Row r > 0 of the segment: the prefix sum of row r - 1 plus
                // the x prefix of row r (exact modulo 2^32)
                const float2 ux = ph[kT + cx];   // (cos a_X, sin a_X) of this column
                const float kh = 0.25f * inv, kd = lamq * inv;
                uint32_t sy[kPlanes];
#pragma unroll
                for (int r = 0; r < kSegRows; ++r) {
                    const int y = sg * kSegRows + r;
                    const int o = sw(y, cx);
                    float f[kPlanes];
#pragma unroll
                    for (int k = 0; k < kPlanes; ++k) {
                        const uint32_t e = S.E[k][o];
                        sy[k] = r == 0 ? e : sy[k] + e;
                        f[k] = (float)(int32_t)sy[k];
                        S.E[k][o] = 0u;
                    }
                    const float2 vy = ph[y];   // (cos a_Y, sin a_Y)
                    float tt[3], tp[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        tt[i] = fmaf(-vy.y, f[3 * i + 2], fmaf(vy.x, f[3 * i + 1], f[3 * i]));   // v . S_i.
                        tp[i] = fmaf(vy.y, f[3 * i + 1], vy.x * f[3 * i + 2]);                 // v' . S_i.
                    }
                    ah[r] = fmaf(kh, fmaf(-ux.y, tt[2], fmaf(ux.x, tt[1], tt[0])), ah[r]);
                    adx[r] = fmaf(kd, fmaf(ux.y, tt[1], ux.x * tt[2]), adx[r]);
                    ady[r] = fmaf(kd, fmaf(-ux.y, tp[2], fmaf(ux.x, tp[1], tp[0])), ady[r]);
                }
                __syncthreads();   // E cleared; the phases may be rewritten
                P = Pn;
            }
        }

        // ---- store: the item's partial plane, or (one plane) the blended maps
        const int x = tx0 + cx;
        if (x < sp.W) {
            const size_t plane = (size_t)sp.W * sp.H;
            const int pl = g * K + part;
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                float* const dst =
                    (G * K > 1 ? p.partial + ((size_t)pl * 3 + f) * plane : p.out + (size_t)f * plane) + x;
#pragma unroll
                for (int r = 0; r < kSegRows; ++r) {
                    const int y = ty0 + sg * kSegRows + r;
                    const float v = f == 0 ? ah[r] : (f == 1 ? adx[r] : ady[r]);
                    if (y < sp.H) dst[(size_t)y * sp.W] = G * K > 1 ? v : blend1(sp, x, y, f, v);
                }
            }
        }
        if (tid == 0) S.item = (int)atomicAdd(queue, 1u);
        __syncthreads();   // the next item's ticket
    }
    // the last CTA out resets the queue for the next launch: every CTA takes
    // its last ticket before it counts itself out
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
            queue[0] = 0u;
            queue[1] = 0u;
            __threadfence();
        }
    }
}

cudaError_t sat_attributes() {
    static int attr[kMaxCachedDevices] = {};
    return cached_per_device(attr, [] {
               return cudaFuncSetAttribute(k_synth_sat, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(SatSmem)) == cudaSuccess ? 1 : -1;
           }) > 0
               ? cudaSuccess
               : cudaErrorInvalidValue;
}

}  // namespace

int synth_sat_tile() { return kT; }

// resident CTAs per SM from the SM's limits (shared memory, registers, threads)
static int synth_sat_ctas_per_sm_query();
int synth_sat_ctas_per_sm() {
    static int cache[kMaxCachedDevices] = {};
    return max(0, cached_per_device(cache, [] { return max(-1, synth_sat_ctas_per_sm_query()); }));
}
static int synth_sat_ctas_per_sm_query() {
    if (sat_attributes() != cudaSuccess) return 0;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0;
    cudaFuncAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&a, k_synth_sat) != cudaSuccess ||
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

cudaError_t launch_synth_sat(const TcItem* items, int n_items, const PatchDev* pdevs, const SynthParams* sps,
                             const BlendSpan* spans, int n_spans, unsigned int* queue, cudaStream_t st) {
    cudaError_t e = sat_attributes();
    if (e != cudaSuccess) return e;
    if (n_items > 0) {
        // persistent grid: one CTA per resident slot, no more than the items
        static int slots[kMaxCachedDevices] = {};
        const int n_slots = cached_per_device(slots, [] {
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return 152;
            return sms * max(1, synth_sat_ctas_per_sm());
        });
        const int grid = min(n_items, n_slots);
        e = launch_pdl(k_synth_sat, grid, kSatThreads, sizeof(SatSmem), st, items, n_items, pdevs, sps, queue);
        count_launches(1);
        if (e != cudaSuccess) return e;
    }
    if (n_spans > 0) return launch_blend_spans(spans, n_spans, pdevs, sps, st);
    return cudaGetLastError();
}

}  // namespace scwp
