// Tensor-core tile gather of the wave-particle synthesis (sm_103a tcgen05),
// Sec. 4.2.  Same sums as the CUDA-core kernel: for a tile of texel columns
// x and rows y and the bumps b that reach it,
//   h(x,y)  = sum_b k_b(u_x) A_b k_b(v_y)
//   Dx(x,y) = sum_b (lam/2) sin(pi u_x/R) A_b k_b(v_y)
//   Dy(x,y) = sum_b k_b(u_x) A_b (lam/2) sin(pi v_y/R)
// are one dense contraction over bumps,
//   D[m][n] = sum_b Aop[m][b] Bop[n][b],
//   Aop = [ 1 + cos(pi u_x/R) ; sin(pi u_x/R) ]              (128 x K: 64 columns x 2)
//   Bop = S [ A (1 + cos(pi v_y/R)) ; A sin(pi v_y/R) ]      (128 x K: 64 rows x 2)
// whose quadrants are 4 S h^T, (2 S/lam) Dx^T, (2 S/lam) Dy^T (the fourth is
// unused; the constant factors are applied when the sums are read out; S is
// a power of two that puts the largest |A| of the patch near 2^13), computed
// by tcgen05.mma (kind::f16, M = 128, K = 16) into FP32 accumulators in
// tensor memory.  Each operand is split as hi + lo in FP16: hi = x
// truncated to 10 mantissa bits (exact in FP16), lo = x - hi (exact in FP32,
// then rounded to FP16): 22 significant bits together, the precision of a
// TF32 pair at twice the tensor rate and half the shared-memory bytes.
// hi*hi accumulates in one accumulator and the small corrections
// hi*lo + lo*hi in a second one, so the large sum takes one rounding per step
// and the two are added in FP32 when read out.  Per K step: one N = 256 MMA
// of Ahi against the stacked [Bhi; Blo] (the two accumulators side by side
// in tensor memory, Ahi read from shared memory once) and one N = 128 MMA of
// Alo against Bhi.
//
// Warps 0-7 produce the operands of each 32-bump chunk into a 3-stage ring in
// shared memory (no-swizzle K-major canonical layout: 8-row x 16-byte core
// matrices, 128 B apart along K, 512 B apart along rows) from bump records
// that warp 9 stages in an eight-slot ring: it walks the bin ranges that
// reach the tile, bucket by bucket, and bulk-copies each chunk's records with
// the chunk's size and kernel radius beside them.  Each producer thread owns
// two tile rows or columns and a quarter of the chunk's bumps; the kernel phase
// pi (X_n - x_b)/R of its sample is the product of its own
// e^{i pi (X_n mod 2R)/R} (from the patch's float64 phase table, once per
// bucket) and the bump's
// e^{-i pi (x_b mod 2R)/R} (in the record, read as one 16-byte half per
// role), so a sample costs one complex multiply and an integer support test.
// Bumps whose support covers the whole tile on both axes (whole bins of
// them, by the bin geometry) skip the MMAs: for those the kernel factors are
// rank 3 in (texel, bump), so the loader sums their 3 x 3 moments
// M = sum_b A_b p_b q_b^T per bucket (p_b, q_b from the record's phase
// factors) and the read-out adds u^T M v per texel (u, v the texel's own
// phase factors) to the tensor-core sums: the same sums, a different
// rounding order.
// One thread of warp 8 issues the MMAs and commits each stage back to the
// producers; after the last stage the producer warps read the accumulator
// out of tensor memory (tcgen05.ld) and write the bucket group's partial
// sums, or the blended maps.  All waits are bounded in time; a timeout sets
// an error flag.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "internal.h"
#include "blend_dev.cuh"

namespace scwp {
namespace {

constexpr int kTX = 64;            // tile columns (x): the MMA's M = 2 * kTX
constexpr int kTY = 64;            // tile rows (y):    the MMA's N = 2 * kTY
constexpr int kKc = 32;            // bumps per stage (two K = 16 steps)
constexpr int kStages = 3;
constexpr int kRecSlots = 8;       // staged record chunks
constexpr int kProdThreads = 256;  // warps 0-7: two halves of each chunk
constexpr int kProdWarps = kProdThreads / 32;
constexpr int kMmaWarp = kProdWarps;        // warp 8: MMA issue
constexpr int kLoadWarp = kProdWarps + 1;   // warp 9: bin ranges and record copies
constexpr int kThreads = kProdThreads + 64;
constexpr int kBatchRows = 32;     // bin rows per range batch: one per loader lane
constexpr int kTmemCols = 256;     // main accumulator at column 0, corrections at 2 * kTY
constexpr uint32_t kCorrCol = 2 * kTY;
constexpr int32_t kQi = 65536, kHalfi = 32768;
constexpr long long kWaitCycles = 4000000000ll;
constexpr uint32_t kSBO = (kKc / 8) * 128;   // bytes between 8-row groups (16-bit elements)

struct __align__(1024) TcStage {   // FP16 operands
    uint16_t Ahi[2 * kTX * kKc];   // rows 0..63 1 + cos, 64..127 sin (tile columns)
    uint16_t Alo[2 * kTX * kKc];
    uint16_t Bhi[2 * kTY * kKc];   // rows 0..63 S A (1 + cos), 64..127 S A sin (tile rows)
    uint16_t Blo[2 * kTY * kKc];   // directly after Bhi: rows 128..255 of one N = 256 operand
};
static_assert(offsetof(TcStage, Blo) == offsetof(TcStage, Bhi) + sizeof(TcStage::Bhi),
              "Bhi and Blo form one 256-row operand");
static_assert(kCorrCol == 2 * kTY, "the corrections sit in the columns after the main sums");

// moments of one bucket's full-cover bumps over a tile: M[i][j] =
// sum_b A_b p_i(b) q_j(b), p = (1, cos, -sin)(pi (x_b mod 2R)/R), q likewise
// for y (the record's phase factors)
struct MomRec {
    int32_t b;      // bucket
    float m[9];
};

// what the loader tells the producers about a staged record chunk
struct ChunkMeta {
    int n;          // bumps in the chunk (the rest of the slot holds sentinels); -1 ends the stream
    int32_t R;      // kernel radius of the chunk's bucket (Q16.16)
    int32_t b;      // the chunk's bucket
    int32_t pad;
};

struct TcSmem {
    TcStage st[kStages];
    BumpRec rec[kRecSlots][kKc];
    ChunkMeta meta[kRecSlots];
    unsigned long long rbar[kRecSlots];  // loader -> producers: metadata and record copies (complete_tx)
    unsigned long long rfree[kRecSlots]; // producers done with a record chunk (one arrival per warp)
    unsigned long long full[kStages];    // producers -> MMA thread (one arrival per warp)
    unsigned long long empty[kStages];   // MMA commit -> producers (1 arrival)
    unsigned long long done;             // final MMA commit -> epilogue
    int stage_n[kStages];                // bumps in the stage; -1 ends the stream
    MomRec mom[kMaxBuckets];             // full-cover moments, one per bucket that has any
    int n_mom;
    uint32_t tmem;
    alignas(16) unsigned char pd[sizeof(PatchDev)];     // this item's patch
    alignas(16) unsigned char spd[sizeof(SynthParams)];
};
static_assert(sizeof(TcStage) % 1024 == 0, "stage alignment");
static_assert(offsetof(TcSmem, rec) % 16 == 0, "record staging alignment");
static_assert(offsetof(TcSmem, rbar) % 8 == 0, "mbarrier alignment");
static_assert(kKc <= 32 && kBatchRows == 32, "the loader warp covers a chunk's sentinels and a batch's rows");
static_assert(offsetof(TcSmem, meta) % 8 == 0, "chunk metadata alignment");

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("{\n\t.reg .b64 s;\n\tmbarrier.arrive.shared::cta.b64 s, [%0];\n\t}" ::"r"(sa(b)) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 s;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 s, [%0], %1;\n\t}" ::"r"(sa(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned long long* b, uint32_t par) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(par)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool bar_wait(unsigned long long* b, uint32_t par, unsigned long long* err) {
    if (bar_try(b, par)) return true;
    const long long t0 = clock64();
    while (!bar_try(b, par))
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(err, (unsigned long long)kErrTimeout);
            return false;
        }
    return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* b) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sa(dst)),
                 "l"(src), "r"(bytes), "r"(sa(b))
                 : "memory");
}

__device__ __forceinline__ void prod_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory"); }

// shared-memory matrix descriptor: no swizzle, K-major canonical layout
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((sa(p) & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// x truncated to 10 mantissa bits (exact in FP16 within its normal range);
// x - hi10(x) is exact in FP32 and smaller than 2^-10 |x|
__device__ __forceinline__ float hi10(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// two floats as FP16 (round to nearest), a in the low half (lower K index)
__device__ __forceinline__ uint32_t pack_f16(float a, float b) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// byte offset of element (row r, k) in a K-major canonical operand
__device__ __forceinline__ int canon(int r, int kq) { return kq * 128 + (r >> 3) * (int)kSBO + (r & 7) * 16; }

// one operand row, rounded to FP16 (no split), for 8 consecutive bumps
__device__ __forceinline__ void store_half8(uint16_t* hi, int off, const float (&f)[8]) {
    uint32_t h[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = pack_f16(f[2 * k], f[2 * k + 1]);
    *reinterpret_cast<uint4*>((char*)hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
}

// one operand row, hi and lo parts, for 8 consecutive bumps (one 16-byte
// core-matrix row each)
__device__ __forceinline__ void store_split8(uint16_t* hi, uint16_t* lo, int off, const float (&f)[8]) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float a = hi10(f[2 * k]), b = hi10(f[2 * k + 1]);
        h[k] = pack_f16(a, b);
        l[k] = pack_f16(f[2 * k] - a, f[2 * k + 1] - b);
    }
    *reinterpret_cast<uint4*>((char*)hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>((char*)lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Operand rows of one producer thread: bumps 8q .. 8q + 7 of a chunk (one
// 16-byte K chunk) for two tile rows or columns, idx and idx + 32.  ROW: the
// tile rows whose B rows are S A (1 + cos(pi v/R)) and S A sin(pi v/R)
// (`amul` = S); otherwise the tile columns whose A rows are 1 + cos(pi u/R)
// and sin(pi u/R) (`amul` = 1); zero outside the support |u| < R.  `rec`
// points at this role's 16-byte half of each 32-byte record: {x, cx, sx, id}
// or {y, cy, sy, amp}; (ct[e], st[e]) = e^{i pi (pos[e] mod 2R)/R}.
// SPLIT: hi + lo FP16 parts; otherwise one FP16 rounding (no lo part).
template <bool ROW, bool SPLIT>
__device__ __forceinline__ void gen_quarter(uint16_t* hi, uint16_t* lo, const float4* rec, int q, int idx,
                                            const int32_t (&pos)[2], int32_t R, const float (&ct)[2],
                                            const float (&st)[2], float amul) {
    const uint32_t span = (uint32_t)(2 * R - 1);
    float4 r[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        r[j] = rec[2 * (8 * q + j)];
        if (ROW) r[j].w *= amul;   // S A, shared by both rows
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        float f0[8], f1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int32_t u = pos[e] - __float_as_int(r[j].x);
            const bool in = (uint32_t)(u + R - 1) < span;              // -R < u < R
            const float cs = ct[e] * r[j].y - st[e] * r[j].z;          // cos pi u / R
            const float sn = st[e] * r[j].y + ct[e] * r[j].z;          // sin pi u / R
            const float m = in ? (ROW ? r[j].w : amul) : 0.f;          // S A, or 1; 0 outside the support
            f0[j] = fmaf(m, cs, m);
            f1[j] = m * sn;
        }
        const int ent = idx + 32 * e;
        if (SPLIT) {
            store_split8(hi, lo, canon(ent, q), f0);
            store_split8(hi, lo, canon(kTX + ent, q), f1);   // kTX == kTY: second half of either operand
        } else {
            store_half8(hi, canon(ent, q), f0);
            store_half8(hi, canon(kTX + ent, q), f1);
        }
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads, 2) k_synth_tc(const TcItem* items, const PatchDev* pdevs,
                                                          const SynthParams* sps) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    pdl_enter();
    // this CTA's (patch, tile, bucket group) item, in the host-planned order
    const TcItem it = items[blockIdx.x];
    {
        static_assert(sizeof(PatchDev) % 4 == 0 && sizeof(SynthParams) % 4 == 0, "descriptor copy");
        const uint32_t* a = reinterpret_cast<const uint32_t*>(pdevs + it.patch);
        const uint32_t* b = reinterpret_cast<const uint32_t*>(sps + it.patch);
        for (int k = tid; k < (int)(sizeof(PatchDev) / 4); k += kThreads) reinterpret_cast<uint32_t*>(S.pd)[k] = a[k];
        for (int k = tid; k < (int)(sizeof(SynthParams) / 4); k += kThreads)
            reinterpret_cast<uint32_t*>(S.spd)[k] = b[k];
    }
    const PatchDev& p = *reinterpret_cast<const PatchDev*>(S.pd);
    const SynthParams& sp = *reinterpret_cast<const SynthParams*>(S.spd);
    const int G = it.groups, g = it.group, tile = it.tile;
    // (read from global memory: the shared copies are read after the first barrier)
    const int ntx = (pdevs[it.patch].W + kTX - 1) / kTX, nb = sps[it.patch].nb;
    const int tx0 = (tile % ntx) * kTX, ty0 = (tile / ntx) * kTY;
    const int b_begin = max((g * nb) / G, sps[it.patch].b_lo);
    const int b_end = min(((g + 1) * nb) / G, sps[it.patch].b_hi);

    if (tid == 0) {
        for (int k = 0; k < kRecSlots; ++k) {
            bar_init(&S.rbar[k], 1);
            bar_init(&S.rfree[k], kProdWarps);
        }
        for (int k = 0; k < kStages; ++k) {
            bar_init(&S.full[k], kProdWarps);
            bar_init(&S.empty[k], 1);
        }
        bar_init(&S.done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&S.tmem)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem;
    // descriptor fields used inside the loops, read once from shared memory
    unsigned long long* const err = p.stats + 2;
    const float row_scale = sp.row_scale;

    if (warp == kMmaWarp) {
        // ======================= MMA issuer ==================================
        if (lane == 0) {
            // F32 += F16 x F16, M = 128; N = 128, or N = 256 for [Bhi; Blo]
            const uint32_t idesc =
                (1u << 4) | ((uint32_t)(2 * kTY >> 3) << 17) | ((uint32_t)(2 * kTX >> 4) << 24);
            const uint32_t idesc2 =
                (1u << 4) | ((uint32_t)(4 * kTY >> 3) << 17) | ((uint32_t)(2 * kTX >> 4) << 24);
            uint32_t acc = 0;
            int k = 0;   // stages consumed
            for (;; ++k) {
                const int fs = k % kStages;
                if (!bar_wait(&S.full[fs], (k / kStages) & 1u, err)) break;
                if (S.stage_n[fs] < 0) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const TcStage& T = S.st[fs];
#pragma unroll
                for (int s = 0; s < kKc / 16; ++s) {
                    const uint32_t off = (uint32_t)s * 256u;   // two 16-byte K chunks per step
                    const uint64_t ah = smem_desc((const char*)T.Ahi + off, 128, kSBO);
                    const uint64_t bh = smem_desc((const char*)T.Bhi + off, 128, kSBO);
                    if (SPLIT) {
                        // [main | corrections] (+)= Ahi [Bhi; Blo]^T in one N = 256 MMA
                        // (Ahi read once for both), then corrections += Alo Bhi^T
                        const uint64_t al = smem_desc((const char*)T.Alo + off, 128, kSBO);
                        mma_f16(tmem, ah, bh, idesc2, acc);
                        mma_f16(tmem + kCorrCol, al, bh, idesc, 1);
                    } else {
                        mma_f16(tmem, ah, bh, idesc, acc);
                    }
                    acc = 1;
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 sa(&S.empty[fs]))
                             : "memory");
            }
            // stages committed by this CTA (executed tensor work, for the roofline)
            if (k > 0) atomicAdd(p.stats + 3 + p.nb, (unsigned long long)k);
            // arrives once every MMA issued above has completed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             sa(&S.done))
                         : "memory");
        }
        __syncwarp();
    } else if (warp == kLoadWarp) {
        // ======================= record loader ===============================
        // Walks this CTA's buckets and, per batch of up to 32 bin rows (one
        // per lane), the bin ranges that reach the tile; cuts their
        // concatenation into chunks of kKc bumps and stages each chunk in the
        // next record slot: metadata by lane 0, one bulk copy per range piece
        // by the lane owning the range.
        const int32_t Xlo = tx0 * kQi + kHalfi, Xhi = (tx0 + kTX - 1) * kQi + kHalfi;
        const int32_t Ylo = ty0 * kQi + kHalfi, Yhi = (ty0 + kTY - 1) * kQi + kHalfi;
        int gc = 0;        // chunks published
        int n_mom = 0;     // buckets with full-cover moments
        bool ok = true;
        // slot of chunk gc once the producers are done with its previous chunk
        auto claim = [&]() -> int {
            const int slot = gc % kRecSlots;
            bool got = true;
            if (gc >= kRecSlots && lane == 0)
                got = bar_wait(&S.rfree[slot], (uint32_t)((gc / kRecSlots - 1) & 1), err);
            ok = ok && __shfl_sync(0xffffffffu, (int)got, 0) != 0;
            return slot;
        };
        for (int bi = b_begin; bi < b_end && ok; ++bi) {
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
            // Bins whose every bump covers the whole tile (every texel centre
            // strictly inside the support on both axes): bin bx holds
            // x_b + R in [bx C, (bx + 1) C), so it is full-cover in x iff
            // bx C > Xhi and (bx + 1) C <= Xlo + 2R.  Their bumps enter the
            // sums through the tile's 3 x 3 moments instead of the MMAs.
            const int fx_lo = max(bx_lo, (int)((int64_t)Xhi / bk.C) + 1);
            const int fx_hi = min(bx_hi, (int)(((int64_t)Xlo + 2 * (int64_t)bk.R) / bk.C) - 1);
            float mom[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) mom[q] = 0.f;
            bool any_full = false;
            for (int byb = by_lo; byb <= by_hi && ok; byb += kBatchRows) {
                const int nr = min(kBatchRows, by_hi - byb + 1);
                // this lane's bin row: dense record ranges [rs, rs + rl) and
                // [rs2, rs2 + rl2), full-cover range [fs, fs + fl)
                int rs = 0, rl = 0, rs2 = 0, rl2 = 0, fs = 0, fl = 0;
                if (lane < nr) {
                    const int by = byb + lane;
                    const int key0 = bk.base + by * bk.nbx;
                    const bool fy = (int64_t)by * bk.C > (int64_t)Yhi &&
                                    ((int64_t)by + 1) * bk.C <= (int64_t)Ylo + 2 * (int64_t)bk.R;
                    rs = (int)p.offsets[key0 + bx_lo];
                    const int e = (int)p.offsets[key0 + bx_hi + 1];
                    if (fy && fx_lo <= fx_hi) {
                        fs = (int)p.offsets[key0 + fx_lo];
                        const int f1 = (int)p.offsets[key0 + fx_hi + 1];
                        rl = fs - rs;
                        fl = f1 - fs;
                        rs2 = f1;
                        rl2 = e - f1;
                    } else {
                        rl = e - rs;
                    }
                }
                rl += rl2;      // dense length of this lane's row
                int inc = rl;   // inclusive prefix of the range lengths over the lanes
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, inc, d);
                    if (lane >= d) inc += t;
                }
                const int cum = inc - rl;
                const int total = __shfl_sync(0xffffffffu, inc, 31);
                for (int lo = 0; lo < total; lo += kKc) {
                    const int n = min(kKc, total - lo);
                    const int slot = claim();
                    if (!ok) break;
                    if (n < kKc) {   // sentinels: far outside every support
                        if (lane >= n && lane < kKc) {
                            BumpRec z;
                            z.x = z.y = 0x40000000;
                            z.cx = z.sx = z.cy = z.sy = z.amp = 0.f;
                            z.id = 0xFFFFFFFFu;
                            S.rec[slot][lane] = z;
                        }
                        // ordered before any later bulk copy into this slot
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    }
                    if (lane == 0) {
                        S.meta[slot].n = n;
                        S.meta[slot].R = bk.R;
                        S.meta[slot].b = bi;
                    }
                    __syncwarp();
                    if (lane == 0) bar_arrive_tx(&S.rbar[slot], (uint32_t)(n * sizeof(BumpRec)));
                    __syncwarp();
                    // this lane's row covers [cum, cum + rl) of the batch: its
                    // first dense range, then its second
                    const int l1 = rl - rl2;
                    int a = max(lo, cum), b = min(lo + n, cum + l1);
                    if (a < b)
                        bulk_g2s(&S.rec[slot][a - lo], p.rec + rs + (a - cum), (uint32_t)((b - a) * sizeof(BumpRec)),
                                 &S.rbar[slot]);
                    a = max(lo, cum + l1);
                    b = min(lo + n, cum + rl);
                    if (a < b)
                        bulk_g2s(&S.rec[slot][a - lo], p.rec + rs2 + (a - cum - l1),
                                 (uint32_t)((b - a) * sizeof(BumpRec)), &S.rbar[slot]);
                    ++gc;
                }
                // moments, after this batch's dense chunks are staged (the
                // producers work through them meanwhile): lane l takes records
                // l, l + 32, ... of each full-cover range, ranges in lane order
                // (a fixed order)
                if (__any_sync(0xffffffffu, fl > 0)) {
                    any_full = true;
                    for (int k = 0; k < nr; ++k) {
                        const int s0 = __shfl_sync(0xffffffffu, fs, k), l0 = __shfl_sync(0xffffffffu, fl, k);
                        // four records in flight per lane, summed in index order
                        for (int j0 = lane; j0 < l0; j0 += 128) {
                            float4 a4[4], b4[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int j = j0 + 32 * u;
                                a4[u] = b4[u] = make_float4(0.f, 0.f, 0.f, 0.f);   // A = 0 past the range
                                if (j < l0) {
                                    a4[u] = reinterpret_cast<const float4*>(p.rec + s0 + j)[0];   // x cx sx id
                                    b4[u] = reinterpret_cast<const float4*>(p.rec + s0 + j)[1];   // y cy sy A
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const float pv[3] = {b4[u].w, b4[u].w * a4[u].y, b4[u].w * a4[u].z};   // A p
                                const float qv[3] = {1.f, b4[u].y, b4[u].z};
#pragma unroll
                                for (int i2 = 0; i2 < 3; ++i2)
#pragma unroll
                                    for (int j2 = 0; j2 < 3; ++j2)
                                        mom[3 * i2 + j2] = fmaf(pv[i2], qv[j2], mom[3 * i2 + j2]);
                            }
                        }
                    }
                }
            }
            if (any_full) {   // this bucket's moments: a fixed reduction tree over the lanes
#pragma unroll
                for (int q = 0; q < 9; ++q)
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) mom[q] += __shfl_xor_sync(0xffffffffu, mom[q], d);
                if (lane == 0 && n_mom < kMaxBuckets) {
                    S.mom[n_mom].b = bi;
#pragma unroll
                    for (int q = 0; q < 9; ++q) S.mom[n_mom].m[q] = mom[q];
                }
                ++n_mom;
            }
        }
        if (lane == 0) S.n_mom = min(n_mom, kMaxBuckets);   // published by the end-of-stream arrival
        if (ok) {   // end of the stream
            const int slot = claim();
            if (ok) {
                if (lane == 0) {
                    S.meta[slot].n = -1;
                    S.meta[slot].R = 0;
                    S.meta[slot].b = -1;
                }
                __syncwarp();
                if (lane == 0) bar_arrive(&S.rbar[slot]);
                ++gc;
            }
        }
        // every copy issued above lands before this CTA's shared memory can
        // be reused (the last kRecSlots chunks hold the only ones that can
        // still be in flight)
        if (lane == 0)
            for (int g2 = max(0, gc - kRecSlots); g2 < gc; ++g2)
                bar_wait(&S.rbar[g2 % kRecSlots], (uint32_t)((g2 / kRecSlots) & 1), err);
        __syncwarp();
    } else {
        // ======================= producers ===================================
        const int32_t Xlo = tx0 * kQi + kHalfi, Ylo = ty0 * kQi + kHalfi;
        // producer warp w builds bumps 8 (w & 3) .. +7 of each chunk for tile
        // rows (w < 4) or columns (w >= 4); lane l for rows/columns l and l + 32
        static_assert(kTX == 64 && kTY == 64 && kKc == 32 && kProdWarps == 8, "producer mapping");
        const bool is_row = warp < 4;
        const int kq = warp & 3, idx = lane;
        const int32_t pos0 = (is_row ? Ylo : Xlo) + idx * kQi;   // this thread's texel centres
        const int32_t pos[2] = {pos0, pos0 + 32 * kQi};
        int produced = 0;      // stages filled
        int fs = 0;            // stage slot of the next stage, and its empty-barrier parity
        uint32_t fpar = 1u;
        int rs = 0;            // record slot of the next chunk, and its parity
        uint32_t rpar = 0u;
        int32_t R = 0;         // radius of the current bucket
        int32_t B = -1;        // the current bucket
        float st[2] = {0.f, 0.f}, ct[2] = {1.f, 1.f};
        for (;;) {
            bool ok = bar_wait(&S.rbar[rs], rpar, err);
            if (__any_sync(0xffffffffu, !ok)) break;   // this warp stops; the others time out in turn
            const ChunkMeta m = S.meta[rs];
            if (m.n < 0) break;
            if (m.b != B) {   // new bucket: this thread's phase factors e^{i pi (pos mod 2R) / R}
                B = m.b;
                R = m.R;
                // this thread's texels in the patch's phase table
                const float2* ph = p.phase + (size_t)B * p.phase_len + (is_row ? ty0 : tx0) + idx;
                const float2 a0 = ph[0], a1 = ph[32];
                ct[0] = a0.x;
                st[0] = a0.y;
                ct[1] = a1.x;
                st[1] = a1.y;
            }
            ok = bar_wait(&S.empty[fs], fpar, err);
            if (__any_sync(0xffffffffu, !ok)) break;
            TcStage& T = S.st[fs];
            // this thread's half of each record: {x, cx, sx, id} or {y, cy, sy, amp};
            // slots past n hold sentinel records outside every support
            const float4* rc = reinterpret_cast<const float4*>(S.rec[rs]) + (is_row ? 1 : 0);
            if (is_row)
                gen_quarter<true, SPLIT>(T.Bhi, T.Blo, rc, kq, idx, pos, R, ct, st, row_scale);
            else
                gen_quarter<false, SPLIT>(T.Ahi, T.Alo, rc, kq, idx, pos, R, ct, st, 1.f);
            if (tid == 0) S.stage_n[fs] = m.n;
            // every lane's operand stores visible to the tensor core, then
            // one arrival for the warp on each barrier
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                bar_arrive(&S.rfree[rs]);
                bar_arrive(&S.full[fs]);
            }
            ++produced;
            if (++fs == kStages) {
                fs = 0;
                fpar ^= 1u;
            }
            if (++rs == kRecSlots) {
                rs = 0;
                rpar ^= 1u;
            }
        }
        // end of the stream for the MMA thread
        {
            bar_wait(&S.empty[fs], fpar, err);
            if (tid == 0) S.stage_n[fs] = -1;
            __syncwarp();
            if (lane == 0) bar_arrive(&S.full[fs]);
        }
        // ======================= epilogue ====================================
        bar_wait(&S.done, 0u, err);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool any = produced > 0;   // otherwise no MMA ever wrote the accumulator
        // Full-cover moments: the operand stages are idle once every MMA has
        // completed, so they hold the tile's phase factors per moment bucket,
        // tab[b][e] = e^{i pi (X_e mod 2R_b)/R_b}, e < 64 the tile rows (y),
        // e >= 64 the tile columns (x).
        const int nm = S.n_mom;
        const float2* tab = reinterpret_cast<const float2*>(S.st);
        static_assert(sizeof(S.st) >= (size_t)kMaxBuckets * 128 * sizeof(float2), "phase tables fit the stages");
        if (nm > 0) {
            float2* wtab = reinterpret_cast<float2*>(S.st);
            for (int k = tid; k < nm * 128; k += kProdThreads) {
                const int b = k >> 7, e = k & 127;
                const int t = e < 64 ? ty0 + e : tx0 + (e - 64);   // texel row or column
                wtab[k] = p.phase[(size_t)S.mom[b].b * p.phase_len + t];
            }
            prod_sync();
        }
        // warp w reads TMEM lane quarter w & 3 (accumulator rows); the two
        // groups of four warps split the column blocks of those rows
        const int quarter = warp & 3, grp = warp >> 2;
        const int m = 32 * quarter + lane;        // accumulator row (TMEM lane)
        const int x = tx0 + (m & (kTX - 1));
        const bool lowm = m < kTX;                // h / Dy rows; else Dx rows
        const int nblk = lowm ? (2 * kTY) / 32 : kTY / 32;
        const int cb_lo = grp * (nblk / 2), cb_hi = cb_lo + nblk / 2;
        const size_t plane = (size_t)sp.W * sp.H;
        for (int cb = cb_lo; cb < cb_hi; ++cb) {
            uint32_t r[32], c[32];
            if (any) {
                const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(32 * cb);
                tmem_ld32(lane_base, r);
                if (SPLIT) {
                    tmem_ld32(lane_base + kCorrCol, c);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) c[j] = 0u;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = c[j] = 0u;
            }
            const int f = cb < kTY / 32 ? (lowm ? 0 : 1) : 2;
            const float scale = (f == 0 ? 0.25f : 0.5f * sp.lam_half) / row_scale;
            const int y0 = ty0 + 32 * (cb & (kTY / 32 - 1));
            // the tensor-core sums, then the full-cover terms: h = 1/4 u M v,
            // Dx = lam/4 u' M v, Dy = lam/4 u M v', u = (1, c, -s) and
            // u' = (0, s, c) of the column, v and v' of the row
            float val[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) val[j] = (__uint_as_float(r[j]) + __uint_as_float(c[j])) * scale;
            for (int b = 0; b < nm; ++b) {
                const float2 ux = tab[b * 128 + 64 + (m & (kTX - 1))];
                const float u0 = f == 1 ? 0.f : 1.f, u1 = f == 1 ? ux.y : ux.x, u2 = f == 1 ? ux.x : -ux.y;
                const float* M = S.mom[b].m;
                const float w0 = u0 * M[0] + u1 * M[3] + u2 * M[6];   // (u^T M)_j
                const float w1 = u0 * M[1] + u1 * M[4] + u2 * M[7];
                const float w2 = u0 * M[2] + u1 * M[5] + u2 * M[8];
                const float fs = f == 0 ? 0.25f : 0.5f * sp.lam_half;
                const int e0 = 32 * (cb & (kTY / 32 - 1));
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float2 vy = tab[b * 128 + e0 + j];
                    const float t = f == 2 ? fmaf(w1, vy.y, w2 * vy.x) : fmaf(w1, vy.x, fmaf(-w2, vy.y, w0));
                    val[j] = fmaf(fs, t, val[j]);
                }
            }
            // read once per block: the global stores below may alias shared
            // memory as far as the compiler knows
            const int Wd = sp.W, Hd = sp.H;
            if (x >= Wd) continue;
            // bucket groups: this group's partial plane; one group: the blended map
            float* const dst = (G > 1 ? p.partial + ((size_t)g * 3 + f) * plane : p.out + (size_t)f * plane) + x;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int y = y0 + j;
                if (y < Hd) dst[(size_t)y * Wd] = G > 1 ? val[j] : blend1(sp, x, y, f, val[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
}

}  // namespace

int synth_tc_tile() { return kTX; }
int synth_tc_stage_bumps() { return kKc; }

namespace {
// the largest shared-memory carveout, so that two CTAs fit on an SM
template <bool SPLIT>
cudaError_t tc_attributes_one() {
    cudaError_t e =
        cudaFuncSetAttribute(k_synth_tc<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_synth_tc<SPLIT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}
cudaError_t tc_attributes() {
    const cudaError_t e = tc_attributes_one<true>();
    return e != cudaSuccess ? e : tc_attributes_one<false>();
}
}  // namespace

// Resident CTAs per SM from the SM's limits: shared memory (with the
// per-block reservation), registers (allocated per warp in units of 256),
// threads, and tensor-memory columns (512 per SM).  The runtime occupancy
// query is not used: it reports one CTA for this 10-warp block although two
// fit every one of these limits.
int synth_tc_ctas_per_sm() {
    if (tc_attributes() != cudaSuccess) return 0;
    int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0;
    cudaFuncAttributes a;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaFuncGetAttributes(&a, k_synth_tc<true>) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return 0;
    const int warps = kThreads / 32;
    const int regs_warp = ((a.numRegs * 32 + 255) / 256) * 256;
    int n = smem_sm / (int)(sizeof(TcSmem) + a.sharedSizeBytes + resv);
    n = min(n, regs_sm / (regs_warp * warps));
    n = min(n, thr_sm / kThreads);
    n = min(n, 512 / kTmemCols);
    return n;
}

cudaError_t launch_synth_tc(const TcItem* items, int n_items, const PatchDev* pdevs, const SynthParams* sps,
                            const BlendSpan* spans, int n_spans, cudaStream_t st, bool split) {
    const size_t sm = sizeof(TcSmem);
    cudaError_t e = tc_attributes();
    if (e != cudaSuccess) return e;
    if (n_items > 0) {
        e = split ? launch_pdl(k_synth_tc<true>, n_items, kThreads, sm, st, items, pdevs, sps)
                  : launch_pdl(k_synth_tc<false>, n_items, kThreads, sm, st, items, pdevs, sps);
        count_launches(1);
        if (e != cudaSuccess) return e;
    }
    if (n_spans > 0) return launch_blend_spans(spans, n_spans, pdevs, sps, st);
    return cudaGetLastError();
}

}  // namespace scwp
