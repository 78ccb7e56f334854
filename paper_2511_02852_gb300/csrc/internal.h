// Internal interfaces between the C ABI layer (api.cu) and the sm_103a
// kernels of the hybrid ocean.  Nothing here crosses the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace scwp {

constexpr int kMaxBuckets = 64;
constexpr int kRotN = 128;          // per-bucket phase-rotation table length
constexpr int kSortTile = 1024;     // keys per block of the bin-key kernel
constexpr int kSortPassTile = 4096; // keys per block of a binning sort pass
constexpr int kMaxSortPasses = 4;   // 8-bit digits of keys up to 32 bits
constexpr int kMaxSegments = 2 * kMaxBuckets + 3;
constexpr int kMaxRing = 64;        // ring-ripple particles emitted per frame at most
constexpr int kMaxWakeRate = 64;    // wake particles per Kelvin arm per frame at most
constexpr int kMaxGiven = kMaxRing + 2 * kMaxWakeRate;   // host-placed particles per frame
constexpr uint32_t kErrCapacity = 1u;
constexpr uint32_t kErrTimeout = 2u;

// Per-bucket constants read by the binning and synthesis kernels.
struct BucketDev {
    int32_t R;      // kernel half-width, Q16.16 cells
    float invR;     // 1 / R (float)
    int32_t C;      // bin side, Q16.16 cells
    int32_t nbx, nby, base;  // bin grid and first key
    float sat_c;    // summed-area pass bound: a (tile, bucket) of n candidates goes in
                    // ceil(n^1.5 / sat_c) passes of at most as many candidates each
    int32_t pad1;
};

// A bump in bin order, as the synthesis kernels stage it (32 bytes).
// (cx, sx) = e^{-i pi (x mod 2R) / R}, (cy, sy) likewise for y: the bump's
// share of every kernel phase pi (X - x) / R, reduced exactly modulo 2R.
struct __align__(16) BumpRec {
    int32_t x;        // centre x, Q16.16 cells
    float cx, sx;
    uint32_t id;      // bump id 2 p + k
    int32_t y;        // centre y
    float cy, sy;
    float amp;        // signed amplitude (+A crest, -A trough)
};

// Device state of one patch.
struct PatchDev {
    int W = 0, H = 0, nb = 0, nth = 0, cap = 0;
    int emitter = 0;
    int total_bins = 0;
    float wake_amp = 0.f;
    int cur = 0;                          // which SoA buffer is live
    int32_t* x[2] = {nullptr, nullptr};
    int32_t* y[2] = {nullptr, nullptr};
    uint32_t* bd[2] = {nullptr, nullptr}; // bucket << 16 | direction
    int32_t* count = nullptr;             // [0] live, [1] live after compaction, [2] live before it
    uint8_t* flags = nullptr;             // [cap] alive flags
    uint32_t* blk = nullptr;              // [nblk_c + 1] compaction block sums
    int nblk_c = 0;
    int4* vq = nullptr;                   // [nb*nth (+4096)] (vx, vy, qx, qy)
    int16_t* dirlist = nullptr;           // [nb][2][nth] valid directions per edge pair
    float* amp = nullptr;                 // [nb*nth]
    BucketDev* bk = nullptr;              // [nb]
    float2* rot = nullptr;                // [nb][kRotN] (cos, sin)(pi n Q / R_i)
    float2* phase = nullptr;              // [nb][phase_len] (cos, sin)(pi (X_n mod 2 R_i) / R_i), X_n the
                                          // Q16.16 centre of texel n (float64 on the host, rounded)
    int phase_len = 0;                    // texels per bucket row of `phase` (whole tiles)
    float* amax = nullptr;                // [nb] bound on |A| of any bump of the bucket
    uint32_t* keys[2] = {nullptr, nullptr};  // [2 cap] bin keys (sort ping-pong)
    uint32_t* vals[2] = {nullptr, nullptr};  // [2 cap] bump ids
    // binning sort scratch (all zero between sorts: each pass's last block
    // clears its histogram and ticket, the key kernel clears the look-back
    // words before every sort)
    uint32_t* hist = nullptr;             // [kMaxSortPasses][256] digit totals of each pass
    uint32_t* sort_ticket = nullptr;      // [kMaxSortPasses][2] block ticket, blocks done
    uint32_t* sort_status = nullptr;      // [kMaxSortPasses][nblk_o][256] look-back words
    int nblk_s = 0;                       // key-kernel blocks (kSortTile keys each)
    int nblk_o = 0;                       // sort-pass blocks (kSortPassTile keys each)
    int key_bits = 16;
    uint32_t* offsets = nullptr;          // [total_bins + 1]
    int4* pk = nullptr;                   // [cap] (x, y, bd, 0) of the live particles, written by the key
                                          // kernel for the record pass's gathers
    BumpRec* rec = nullptr;               // [2 cap] bump records in bin order
    float* out = nullptr;                 // [3][H][W] blended maps
    float* partial = nullptr;             // [groups][3][H][W] per-bucket-group sums (groups > 1)
    int groups = 1;                       // bucket groups of the CUDA-core synthesis
    int groups_tc = 1;                    // bucket groups of the tensor-core synthesis
    int patch = 0;                        // index of the patch in its context
    unsigned long long* stats = nullptr;  // [0] evals, [1] binned, [2] flags, [3..3+nb) live per bucket,
                                          // [3+nb] operand stages of the last tensor-core synthesis,
                                          // [4+nb] evals summed over all frames,
                                          // [5+nb] candidates of the last summed-area synthesis
                                          // (summed over its (tile, bucket) pairs)
    float* layers = nullptr;              // layered variant scratch (lazy)
    size_t layers_bytes = 0;
};

// One work item of the tensor-core synthesis: bucket group `group` of
// `groups` over tile `tile` of patch `patch`.  The summed-area syntheses may
// also split each bucket's passes over K parts (tiles of very dense patches,
// whose buckets take many passes): group = g | part << 16, groups =
// G | K << 16 (K = 0 or 1: not split), and the item writes partial plane
// g K + part of G K.
struct TcItem {
    int32_t patch, tile, group, groups;
};
__host__ __device__ inline int item_groups(const TcItem& it) { return it.groups & 0xFFFF; }
__host__ __device__ inline int item_parts(const TcItem& it) { return (it.groups >> 16) > 1 ? (it.groups >> 16) : 1; }
__host__ __device__ inline int item_group(const TcItem& it) { return it.group & 0xFFFF; }
__host__ __device__ inline int item_part(const TcItem& it) { return it.group >> 16; }

// One span of the group-sum blend: quads [q0, q1) (4 texels of a row) of
// patch `patch`, whose synthesis used `groups` bucket groups.
struct BlendSpan {
    int32_t patch, q0, q1, groups;
};

// One spawn segment of a frame's injection (Sec. 3.3 Eqs. 15-17 / Sec. 4.3).
struct Segment {
    int32_t bucket;
    int32_t s;       // 0, 1: edge pairs; 2: wake arm; 3: ring ripples
    int32_t count;   // particles in the segment
    int32_t first;   // prefix of counts
    int32_t ndir;    // edge: number of valid directions; wake: rate
    int32_t arm;     // wake: arm index (0: +, 1: -)
    int32_t wake_a;  // wake: direction grid index
    int32_t given;   // wake and rings: first of the segment's host-placed positions
};

struct InjectParams {
    int nseg;
    int total;
    uint32_t frame;
    uint32_t patch;
    uint64_t seed;
    int W, H, nth;
    Segment seg[kMaxSegments];
    // wake (s = 2) and ring-ripple (s = 3) particles: Q16.16 positions and
    // wake-grid directions placed on the host in float64 (the operations that
    // decide these integers stay off the GPU)
    int32_t gx[kMaxGiven], gy[kMaxGiven], ga[kMaxGiven];
};

struct SynthParams {
    int W, H, nb;
    float lam_half;         // lambda_c / 2
    float band;             // blend band in cells
    float fx0, fy0, fsx;    // background coords: f = f0 + i * fs (grid units)
    int N;                  // background grid size
    const float* bg;        // [3][N][N]
    float row_scale;        // power of two putting the patch's largest |A| near 2^13
    int b_lo, b_hi;         // buckets synthesised: [b_lo, b_hi) (a diagnostic range; default all)
};

// Every launcher reports how many kernels it enqueued (a counter per host
// thread, read by the ABI layer around each call).
void count_launches(int n);

// Programmatic dependent launch.  A kernel launched by launch_pdl may be
// scheduled while its predecessor on the stream is still running; it calls
// pdl_enter() before touching global memory, which waits until the
// predecessor grid has completed (its writes visible) and then allows the
// successor grid to be scheduled.  Only the launch latency overlaps: no
// kernel reads or writes anything before its predecessor is done.  Launches
// recorded into a CUDA graph go without it: a replayed graph has no launch
// latency to hide, and with several patches' streams in one graph the early
// blocks only held SM slots (batched frames 1.6% slower with it).  Without
// the attribute pdl_enter() returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... K, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A&&... args) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return cudaGetLastError();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}
long long launches_total();

// A kernel's launch set-up (attributes, occupancy) done once per device:
// slot d of a function-local cache holds the result for device d, set on
// the first call with that device current.  Later calls skip the driver
// queries that would otherwise stall every eager launch on the host.
constexpr int kMaxCachedDevices = 64;
template <typename F>
inline int cached_per_device(int (&cache)[kMaxCachedDevices], F&& compute) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxCachedDevices) return compute();
    if (cache[dev] == 0) cache[dev] = compute();
    return cache[dev];
}

// ---- launchers (each enqueues on `st`) --------------------------------------
cudaError_t launch_advect_flag(const PatchDev& p, cudaStream_t st);
cudaError_t launch_compact(const PatchDev& p, cudaStream_t st);
cudaError_t launch_inject(const PatchDev& p, const InjectParams& ip, cudaStream_t st);
// injection with the frame's parameters read from device memory (a fixed
// grid, so that the launch can be replayed from a CUDA graph)
cudaError_t launch_inject_dev(const PatchDev& p, const InjectParams* ip, cudaStream_t st);
cudaError_t launch_bin(const PatchDev& p, cudaStream_t st);
// failure-detection self-test: the bin keys, then the first sort pass with
// its first tile never taken, so the look-back waits on it give up after
// wait_cycles SM clocks and set the timeout flag (outputs meaningless)
cudaError_t launch_sort_stall(const PatchDev& p, long long wait_cycles, cudaStream_t st);
cudaError_t launch_synth_gather(const PatchDev& p, const SynthParams& sp, cudaStream_t st);
// Tensor-core synthesis of `n_items` items (any patches) in one launch, then
// the group-sum blend of `n_spans` spans in one launch.  `pdevs` and `sps`
// are device arrays indexed by patch.
// split: FP16 hi/lo operands (3 MMAs per K step, the FP32 contract);
// otherwise single FP16 operands (1 MMA per K step, the FP16 contract).
cudaError_t launch_synth_tc(const TcItem* items, int n_items, const PatchDev* pdevs, const SynthParams* sps,
                            const BlendSpan* spans, int n_spans, cudaStream_t st, bool split = true);
// Summed-area synthesis (the same sums through 2-D difference arrays of the
// kernel's rank-3 factors) of `n_items` items in one persistent launch, then
// the group-sum blend, like launch_synth_tc.  `queue` is the launch's work
// queue, two zeroed device words that the kernel leaves zeroed again; the
// launches that share one must be ordered on a stream.
cudaError_t launch_synth_sat(const TcItem* items, int n_items, const PatchDev* pdevs, const SynthParams* sps,
                             const BlendSpan* spans, int n_spans, unsigned int* queue, cudaStream_t st);
int synth_sat_tile();
int synth_sat_ctas_per_sm();
// The three-group variant of the same synthesis (two 512-thread CTAs per SM,
// one CTA per item): faster where per-texel work dominates; every bucket of
// its patches must reach at most synth_sat3_row_cap() bin rows per tile.
cudaError_t launch_synth_sat3(const TcItem* items, int n_items, const PatchDev* pdevs, const SynthParams* sps,
                              const BlendSpan* spans, int n_spans, cudaStream_t st);
int synth_sat3_ctas_per_sm();
int synth_sat3_row_cap();
// tensor-core synthesis geometry: tile side (texels), bumps per operand stage,
// and resident CTAs per SM (0 on error)
int synth_tc_tile();
int synth_tc_stage_bumps();
int synth_tc_ctas_per_sm();
// unit normals [3][H][W] of the displaced surface of maps [3][H][W] (h, Dx, Dy)
cudaError_t launch_normals(const float* maps, int W, int H, float cell, float* dst, cudaStream_t st);

// group sums and blend of `n_spans` spans of any patches, one launch
cudaError_t launch_blend_spans(const BlendSpan* spans, int n_spans, const PatchDev* pdevs, const SynthParams* sps,
                               cudaStream_t st);
// sum `groups` partial [3][H][W] planes at src (in order), blend, store to p.out
cudaError_t launch_blend(const PatchDev& p, const SynthParams& sp, const float* src, int groups,
                         cudaStream_t st);
// layered variant: scratch (p.layers) must hold layered_scratch_bytes()
size_t layered_scratch_bytes(const PatchDev& p, const int32_t* R_host);
cudaError_t launch_layered(const PatchDev& p, const SynthParams& sp, const int32_t* R_host,
                           const int* base_host, const int* nbins_host, cudaStream_t st);

struct BgDev {
    int N = 0;
    const float2* h0 = nullptr;   // [N][N] FFT-natural order
    const float2* omega = nullptr;// [N][N] w(k) as a float pair (hi, lo), w = hi + lo
    const float2* tw = nullptr;   // twiddle tables of the stages (build_background_twiddles)
    float2* I = nullptr;          // [3][N/2 + 1][N] row-pass output (H1, Dx1, Dy1 of rows k_y <= N/2)
    float* out = nullptr;         // [3][N][N] h, Dx, Dy
    float lam = 1.f, dk = 0.f;
};
// t_dev: if not null, the time is read from device memory (graph replay) as
// a float pair (t_hi, t_lo), t = t_hi + t_lo, split on the host
cudaError_t launch_background(const BgDev& b, double t, cudaStream_t st, const float2* t_dev = nullptr);
// complex elements of the row-pass intermediate of an N x N background
size_t background_scratch_elems(int N);
// entries of the twiddle tables of a length-N transform (at most N / 3)
size_t background_twiddle_elems(int N);
// the twiddle tables of a length-N transform, built in float64 on the host:
// per stage after the first (span Ns = 16, 256, ..., radix R = min(16, N / Ns)),
// e^{2 pi i p k / (Ns R)} for p = 1, 2, 4, 8 (p < R) and k = 0 .. Ns - 1, as [p][k]
void build_background_twiddles(int N, float2* out);

}  // namespace scwp
