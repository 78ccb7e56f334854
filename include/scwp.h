/*
 * scwp.h — C ABI of the GB300 (sm_103a) hybrid wave-particle / FFT ocean
 * height-field synthesis of "Real-Time Interactive Hybrid Ocean:
 * Spectrum-Consistent Wave Particle-FFT Coupling" (arXiv 2511.02852).
 *
 * The calls follow the paper's statement of the problem:
 *   - a spectrum drives both a global FFT background and local wave-particle
 *     (WP) patches (Sec. 3.1 and Fig. "Pipeline overview", Sec. 4.1);
 *   - patches are rectangles placed around interactive objects inside which
 *     the WP field replaces the background (Sec. 3.1, local replacement);
 *   - every frame the background is evolved and inverse-transformed, the
 *     particles are injected at the patch boundaries with counts from
 *     Eqs. 15-17, advected, accumulated per frequency bucket and blended
 *     into the background (Sec. 4.1-4.2).
 *
 * Conventions shared by every call:
 *   - All pointers are plain host or device addresses; no C++ or framework
 *     types cross this boundary.  The caller owns every pointer it passes;
 *     the library copies what it keeps.
 *   - Every call returns an scwp_status.  No exception crosses the ABI.  A
 *     CUDA error is sticky: the context then answers SCWP_E_CUDA to every
 *     call and must be destroyed.  scwp_last_error() gives the message.
 *   - Calls on one context are not thread-safe; separate contexts are
 *     independent.  Device work is ordered on the stream given at create.
 *   - Device memory comes from the caller's allocator callback (if given),
 *     else cudaMalloc; it is freed by scwp_destroy.
 *   - Positions are Q16.16 fixed point in patch cell units relative to the
 *     patch origin; texel (ix, iy) has its centre at ((ix+1/2)Q, (iy+1/2)Q).
 *   - Maps are row-major float32 [height][width] (patch) or [N][N]
 *     (background), row index = y.
 */
#ifndef SCWP_H
#define SCWP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scwp_ctx scwp_ctx;

typedef enum {
    SCWP_OK = 0,
    SCWP_E_INVALID = 1,   /* bad argument; nothing was changed            */
    SCWP_E_NOMEM = 2,     /* the allocator failed                          */
    SCWP_E_CAPACITY = 3,  /* particle pool full: injection was truncated   */
    SCWP_E_CUDA = 4,      /* CUDA error (sticky)                           */
    SCWP_E_TIMEOUT = 5,   /* a bounded device wait gave up (sticky)        */
    SCWP_E_STATE = 6      /* call not valid in the current state           */
} scwp_status;

enum { SCWP_SPECTRUM_JONSWAP = 0, SCWP_SPECTRUM_PHILLIPS = 1 };
enum { SCWP_SPREAD_COS2S_MITSUYASU = 0, SCWP_SPREAD_COS2 = 1 };
enum { SCWP_AMP_NORMALIZED = 0, SCWP_AMP_LITERAL = 1 };
enum { SCWP_FIELD_H = 0, SCWP_FIELD_DX = 1, SCWP_FIELD_DY = 2 };
/* Synthesis modes (Sec. 4.2):
 *   SCWP_SYNTH_GATHER       tile gather on the tensor cores: tcgen05
 *                           FP16 MMAs with a hi/lo operand split, FP32
 *                           accumulation; the FP32 contract (1e-4 Hs);
 *   SCWP_SYNTH_LAYERED      the paper's layered-texture formulation;
 *   SCWP_SYNTH_GATHER_FP32  the same gather on the FP32 CUDA cores;
 *   SCWP_SYNTH_GATHER_FP16  the tensor-core gather with single FP16 operands
 *                           (one MMA per step instead of three), FP32
 *                           accumulation; the reduced-precision contract
 *                           (2e-3 Hs); positions and bins stay exact.
 *   SCWP_SYNTH_SAT          the same per-bucket sums (Sec. 4.2, kernel
 *                           reading O11/O12) through summed-area tables: on
 *                           its support a bump's raised-cosine factors are
 *                           rank 3 in (texel, bump), so per (tile, bucket)
 *                           the maps are a 3 x 3 contraction of 2-D prefix
 *                           sums of the bumps' support-box corners (integer
 *                           events, exact prefix sums, FP32 contraction);
 *                           the FP32 contract; the cost no longer grows with
 *                           the bumps that cover a texel.  The default. */
enum { SCWP_SYNTH_GATHER = 0, SCWP_SYNTH_LAYERED = 1, SCWP_SYNTH_GATHER_FP32 = 2, SCWP_SYNTH_GATHER_FP16 = 3,
       SCWP_SYNTH_SAT = 4 };

#define SCWP_MAX_BUCKETS 64
#define SCWP_MAX_THETA 256
#define SCWP_WAKE_DIRS 4096

/* Spectrum and background (Sec. 3.1 Eqs. 1-6; Sec. 3.3 Eq. 7 bucket range;
 * Sec. 5.2 scene parameters).  JONSWAP: alpha, omega_p from Eq. 4; gamma
 * from Eq. 4 unless gamma > 0.  Phillips (named in Sec. 2.1 / 3.1):
 * S = 0.0081 g^2 w^-5 exp(-(g/(U w))^4).  Spreading: cos-2s with Mitsuyasu's
 * s(w) (Eqs. 5-6), or one-sided (2/pi) cos^2.  Buckets: n_buckets
 * equal-energy buckets on [omega_lo_mul, omega_hi_mul] * omega_p (default
 * 0.5, 2.5; Sec. 3.3), or explicit ascending edges (n_buckets + 1 values,
 * copied).  Directions: N_theta on the grid theta_w - pi + (j+1/2) 2pi/N.
 * Background: fft_n x fft_n grid (power of two, 8..4096) over fft_L metres,
 * choppiness lambda_c for the horizontal displacement. */
typedef struct scwp_spectrum_desc {
    int32_t spectrum;          /* SCWP_SPECTRUM_*                          */
    int32_t spreading;         /* SCWP_SPREAD_*                            */
    double wind_speed;         /* U10, m/s (> 0)                           */
    double fetch;              /* m (> 0; JONSWAP)                         */
    double depth;              /* m; <= 0: deep water                      */
    double wind_dir;           /* rad                                      */
    double gamma;              /* <= 0: Eq. 4                              */
    int32_t n_buckets;         /* 1..SCWP_MAX_BUCKETS                      */
    int32_t n_theta;           /* 1..SCWP_MAX_THETA                        */
    const double* bucket_edges;/* n_buckets + 1 ascending, or NULL         */
    double omega_lo_mul;       /* <= 0: 0.5                                */
    double omega_hi_mul;       /* <= 0: 2.5                                */
    int32_t amp_mode;          /* SCWP_AMP_*                               */
    int32_t fft_n;             /* background grid size                     */
    double fft_L;              /* background side, m                       */
    double choppiness;         /* lambda_c                                 */
    uint64_t seed;             /* Philox4x32-10 key                        */
    /* device memory: alloc(bytes, user) -> device pointer or NULL;
     * free(ptr, user).  Both NULL: cudaMalloc / cudaFree. */
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* alloc_user;
    void* stream;              /* cudaStream_t; NULL: the legacy stream    */
} scwp_spectrum_desc;

/* A wave-particle patch (Sec. 3.1 local replacement; Sec. 3.3 injection;
 * Sec. 4.3 object emission).  Injection per frame and edge pair s follows
 * n = 4 L_s dt c_i / (pi r_i^2) * inject_scale (Eqs. 15-17) with a float64
 * carry; amplitudes scale by 1/sqrt(inject_scale).  `prefill` particles are
 * placed at creation, split over buckets in proportion to the injection's
 * steady state.  With `emitter`, an object of radius obj_radius moves on a
 * circle of radius obj_path_radius about the patch centre at obj_speed and
 * emits wake_rate particles per Kelvin arm per frame into the bucket whose
 * radius is closest to obj_radius, amplitude wake_amp.  The wake's and the
 * ring ripples' spawn points are placed on the host in float64 (they decide
 * integer positions); the GPU path itself uses no float64. */
typedef struct scwp_patch_desc {
    double origin_x, origin_y; /* world position of the patch corner, m    */
    double cell;               /* texel size, m                            */
    int32_t width, height;     /* texels (1..16384)                        */
    double band;               /* blend band, cells; <= 0: min(W,H)/8      */
    int32_t max_particles;     /* particle pool capacity (> 0)             */
    int32_t prefill;           /* particles placed at creation (>= 0)      */
    double inject_scale;       /* <= 0: 1                                  */
    int32_t bin_cells;         /* bin side in texels; <= 0: automatic      */
    int32_t emitter;           /* 0/1                                      */
    double obj_radius, obj_speed, obj_path_radius, wake_amp;
    int32_t wake_rate;         /* particles per arm per frame, 0..64       */
    int32_t n_buckets;         /* <= 0: the spectrum's                     */
    double heave_period;       /* s; > 0 (with emitter): the object heaves and emits
                                  ring ripples (Sec. 4.3, vertical motion)  */
    int32_t ring_rate;         /* ring particles per frame at full heave speed (>= 0) */
} scwp_patch_desc;

/* Per-patch statistics of the last completed frame (counts are exact). */
typedef struct scwp_stats {
    int64_t frame;             /* frames stepped                           */
    double time;               /* running sum of dt, s                     */
    int64_t live_particles;    /* after this frame's injection             */
    int64_t bumps_binned;      /* bumps with >= 1 texel centre in support  */
    int64_t eval_count;        /* sum over binned bumps of texels in support */
    int64_t injected_total;    /* particles injected since creation        */
    int32_t n_buckets;
    int32_t error_flags;       /* bit 0: particle pool full (injection truncated);
                                  bit 1: a bounded device wait timed out   */
    int64_t live_per_bucket[SCWP_MAX_BUCKETS];
    double injected_energy[SCWP_MAX_BUCKETS]; /* sum 1/8 A^2 pi r^2 (Eq. 12 / rho g) */
    int64_t mma_stages;        /* operand stages (6 MMAs of 128x128x16 each) the last
                                  tensor-core synthesis committed; 0 for the other modes */
    int64_t eval_total;        /* eval_count summed over every frame stepped */
    int64_t sat_candidates;    /* candidate bumps the last summed-area synthesis took, summed
                                  over its (tile, bucket) pairs (each candidate: 4 corner
                                  events of 9 components); 0 for the other modes */
} scwp_stats;

/* Scalar description of a patch's tables and bins. */
typedef struct scwp_patch_info {
    int32_t n_buckets, n_theta, n_dirs;   /* n_dirs = n_theta (+ 4096 with an emitter) */
    int32_t wake_bucket;
    int32_t width, height;
    int32_t total_bins;
    int32_t capacity;
    int32_t bin_cells[SCWP_MAX_BUCKETS];
    int32_t nbx[SCWP_MAX_BUCKETS], nby[SCWP_MAX_BUCKETS], bin_base[SCWP_MAX_BUCKETS];
    int32_t synth_groups;      /* bucket groups of the tensor-core synthesis (planned at creation) */
    int32_t synth_items;       /* its (tile, group) work items = CTAs per synthesis launch */
    int32_t synth_slots;       /* resident CTA slots of the device the plan assumed */
    int32_t sat_groups;        /* bucket groups of the summed-area synthesis */
    int32_t sat_items;         /* its (tile, group) work items */
    int32_t sat_slots;         /* resident CTA slots its plan assumed */
    int32_t frame_param_bytes; /* host-computed plan of one frame of this patch (injection
                                  counts, host-placed spawn points) copied to the device */
    int32_t sat_variant;       /* summed-area kernel of this patch: 0 the persistent
                                  nine-plane kernel, 1 the three-group kernel */
    int32_t sat_parts;         /* parts each bucket's passes are split over (1 but on
                                  very dense patches, whose buckets take many passes) */
} scwp_patch_info;

/* Table identifiers for scwp_get_table (element type, count). */
enum {
    SCWP_TAB_OMEGA = 0,   /* double[nb]  bucket representative frequency   */
    SCWP_TAB_K = 1,       /* double[nb]  wavenumber                        */
    SCWP_TAB_C = 2,       /* double[nb]  phase speed                       */
    SCWP_TAB_R = 3,       /* double[nb]  r = pi / k                        */
    SCWP_TAB_E = 4,       /* double[nb]  bucket energy int S dw            */
    SCWP_TAB_EDGES = 5,   /* double[nb+1]                                  */
    SCWP_TAB_AMP = 6,     /* double[nb*nth]                                */
    SCWP_TAB_RQ = 7,      /* int32[nb]   R_i = rint(r/dx Q)                */
    SCWP_TAB_VX = 8,      /* int32[nb*nth] rint(c dt cos/dx Q)             */
    SCWP_TAB_VY = 9,
    SCWP_TAB_QX = 10,     /* int32[nb*nth] rint(r cos/dx Q)                */
    SCWP_TAB_QY = 11,
    SCWP_TAB_WAKE_VX = 12,/* int32[4096] (emitter only)                    */
    SCWP_TAB_WAKE_VY = 13,
    SCWP_TAB_WAKE_QX = 14,
    SCWP_TAB_WAKE_QY = 15,
    SCWP_TAB_CARRY = 16   /* double[nb*2] injection carries                */
};

/* Create a context: validates the description, computes the spectrum
 * tables in float64 on the host, draws h0(k) (Philox4x32-10 + Box-Muller),
 * allocates the background's device state.  *out = NULL on failure. */
scwp_status scwp_create(const scwp_spectrum_desc* desc, scwp_ctx** out);

/* Add a patch: buckets, amplitudes and fixed-point tables (float64 host),
 * particle pool, bins and output maps; places `prefill` particles.
 * *patch_id = index in add order (0, 1, ...). */
scwp_status scwp_add_patch(scwp_ctx* ctx, const scwp_patch_desc* desc, int32_t* patch_id);

/* One frame of the hybrid ocean (Sec. 4.1): frame += 1, t += dt; the
 * background spectrum update and inverse FFT; per patch advection,
 * expiry, injection, wake emission, binning, synthesis and blend.
 * Asynchronous on the context's stream.  dt > 0; the fixed-point
 * velocity tables are rebuilt (float64, host) whenever dt changes. */
scwp_status scwp_step(scwp_ctx* ctx, double dt);

/* Copy one field of a finished map (Sec. 4.1-4.2: the frame's output is
 * the height field and the choppy horizontal displacement, the WP patch
 * blended into the FFT background across its boundary band):
 * patch_id >= 0 a patch's blended map (height x width), patch_id = -1 the
 * background (N x N); field SCWP_FIELD_H / DX / DY.  dst_elems must be at
 * least the map size.  dst_on_device = 1: device-to-device copy ordered on
 * the stream (asynchronous); 0: device-to-host copy, synchronises the
 * stream.  SCWP_E_INVALID for a bad field, patch_id or size. */
scwp_status scwp_height_map(scwp_ctx* ctx, int32_t patch_id, int32_t field,
                            float* dst, size_t dst_elems, int32_t dst_on_device);

/* All three fields of a finished map in one copy: dst receives [3][rows][cols]
 * (h, Dx, Dy planes, each as scwp_height_map gives it), dst_elems >= 3 x the
 * map size.  One device-to-host copy and one synchronisation for a host dst
 * (dst_on_device = 0); an asynchronous device-to-device copy otherwise. */
scwp_status scwp_height_maps(scwp_ctx* ctx, int32_t patch_id, float* dst, size_t dst_elems, int32_t dst_on_device);

/* Unit normals of a patch's last blended maps, [3][height][width] (nx, ny,
 * nz): the normal of the displaced surface p(i, j) = (i c + Dx, j c + Dy, h)
 * (c = the patch's cell size) by finite differences, central inside the
 * patch and one-sided at its edges, the normalised cross product of the
 * two tangents (Sec. 4.2 derives normals from the maps by finite
 * differences; the formula is this library's).  dst_elems >= 3 W H.
 * dst_on_device as in scwp_height_map. */
scwp_status scwp_normal_map(scwp_ctx* ctx, int32_t patch_id, float* dst, size_t dst_elems, int32_t dst_on_device);


/* Statistics of a patch after the last frame (synchronises the stream).
 * The statistics are filled in every case; the status reports the frame's
 * error flags: SCWP_E_TIMEOUT (sticky) for bit 1, SCWP_E_CAPACITY for bit 0,
 * SCWP_OK when none is set. */
scwp_status scwp_stats_get(scwp_ctx* ctx, int32_t patch_id, scwp_stats* out);

/* Table and bin geometry of a patch. */
scwp_status scwp_patch_info_get(scwp_ctx* ctx, int32_t patch_id, scwp_patch_info* out);

/* Copy one table (SCWP_TAB_*) of a patch into host memory; bytes must be at
 * least the table's size. */
scwp_status scwp_get_table(scwp_ctx* ctx, int32_t patch_id, int32_t table, void* dst, size_t bytes);

/* Copy the live particles (SoA, host memory): x, y Q16.16; bd = bucket << 16
 * | direction (direction >= n_theta: wake direction n_theta + a).  *n = live
 * count; at most cap are copied (synchronises). */
scwp_status scwp_get_particles(scwp_ctx* ctx, int32_t patch_id, int32_t* x, int32_t* y,
                               uint32_t* bd, int64_t cap, int64_t* n);

/* Replace the live particles of a patch (host SoA as above; n <= capacity).
 * Directions and buckets are checked. */
scwp_status scwp_set_particles(scwp_ctx* ctx, int32_t patch_id, const int32_t* x,
                               const int32_t* y, const uint32_t* bd, int64_t n);

/* Copy the last frame's bins of a patch (host memory): counts[total_bins],
 * offsets[total_bins + 1], entries[n_entries] (bump ids 2p + k, k = 0 crest,
 * 1 trough, stable in id order within a bin).  *n_entries = binned bumps. */
scwp_status scwp_get_bins(scwp_ctx* ctx, int32_t patch_id, uint32_t* counts, uint32_t* offsets,
                          uint32_t* entries, int64_t entries_cap, int64_t* n_entries);

/* Failure-detection self-test of the bounded device waits (the paper has no
 * counterpart: its binning is not described at this level).  Recomputes the
 * bin keys of the patch's live particles and runs the first pass of the
 * binning sort with the look-back word of its first key tile never
 * published, so that every wait on that word runs out after wait_seconds
 * (0 < wait_seconds <= 2) of SM clock; no kernel faults, traps or hangs.
 * Needs at least 2049 live particles in the patch (two sort tiles of 4096
 * bump keys), else SCWP_E_INVALID.  Returns SCWP_E_TIMEOUT when the kernel
 * reported the timeout, as a frame would; the context is then sticky
 * (every later call returns SCWP_E_TIMEOUT) and must be destroyed, while the
 * CUDA context and every other scwp context stay usable.  Synchronises. */
scwp_status scwp_debug_sort_timeout(scwp_ctx* ctx, int32_t patch_id, double wait_seconds);

/* Recompute the synthesis and blend of every patch from the current
 * particles and background without advancing the frame (the bins are
 * rebuilt).  mode: any SCWP_SYNTH_* (SCWP_SYNTH_SAT, the default path of
 * scwp_step; SCWP_SYNTH_GATHER, the tile gather on the tensor cores;
 * SCWP_SYNTH_GATHER_FP32, the same gather on the FP32 CUDA cores;
 * SCWP_SYNTH_GATHER_FP16; SCWP_SYNTH_LAYERED, per-bucket layer splat +
 * separable x / y passes + layer sum, Sec. 4.2). */
scwp_status scwp_resynthesize(scwp_ctx* ctx, int32_t mode);

/* Select the synthesis used by scwp_step (SCWP_SYNTH_*). */
scwp_status scwp_set_synth_mode(scwp_ctx* ctx, int32_t mode);

/* Diagnostic: the summed-area and tensor-core synthesis modes sum only the
 * buckets b_lo <= i < b_hi (clamped to each patch's count; default all), so
 * that the error against the FP64 oracle can be stated per bucket.  The
 * paper has no counterpart.  SCWP_E_INVALID if b_lo < 0 or b_hi <= b_lo.
 * The CUDA-core gather and the layered mode ignore the range. */
scwp_status scwp_set_bucket_range(scwp_ctx* ctx, int32_t b_lo, int32_t b_hi);

/* Batched frame step (on != 0): the synthesis of all patches of
 * the context runs as one launch over the (patch, tile, bucket group) items
 * of every patch, heaviest first by a work estimate, followed by one
 * group-sum blend launch; per-patch bucket-group counts are planned for the
 * whole frame instead of for each patch alone.  The results are the same
 * sums as the one-patch-per-launch path (with another grouping, the same
 * values up to FP32 rounding order).  Applies to SCWP_SYNTH_SAT,
 * SCWP_SYNTH_GATHER and SCWP_SYNTH_GATHER_FP16; the
 * paper has no counterpart (its frame is one scene on one GPU).  Returns
 * SCWP_E_INVALID for a null context; takes effect at the next synthesis. */
scwp_status scwp_set_batched(scwp_ctx* ctx, int32_t on);

/* Autotuner of the summed-area synthesis (SCWP_SYNTH_SAT), the frame's
 * dominant stage.  The paper has no counterpart (its synthesis is one
 * fixed-function pass).  Two kernel variants compute the same sums: the
 * persistent nine-plane kernel (one 1024-thread CTA per SM pulling (tile,
 * bucket group) items from a work queue) and the three-group kernel (two
 * 512-thread CTAs per SM, one per item; offered only where every bucket
 * reaches at most 512 bin rows of a tile).  For each variant and each
 * bucket-group multiplier of the host plan (1, 1/2, 2) the tuner
 * re-synthesises the last frame `reps` times on the context's stream (one
 * warm-up, then CUDA events), keeps the configuration of the smallest median
 * time, re-synthesises the last frame with it and caches it per device and
 * workload signature (every patch's size, buckets, prefill, capacity, bin
 * size, and the batching mode) for the life of the process; a later call
 * with the same signature applies the cached choice without timing unless
 * force != 0.  Needs at least one stepped frame; synchronises.  reps in
 * 1..100.  SCWP_E_STATE if the context's mode is not SCWP_SYNTH_SAT. */
#define SCWP_TUNE_MAX 8
typedef struct scwp_tune_result {
    int32_t n_configs;           /* configurations timed (1 with from_cache)      */
    int32_t chosen;              /* index of the one kept                           */
    int32_t from_cache;          /* 1: the cached choice was applied, nothing timed */
    int32_t pad;
    int32_t variant[SCWP_TUNE_MAX];   /* 0 nine-plane persistent, 1 three-group    */
    double gmul[SCWP_TUNE_MAX];       /* bucket-group multiplier of the plan       */
    double ms[SCWP_TUNE_MAX];         /* median synthesis + blend time, ms          */
} scwp_tune_result;
scwp_status scwp_autotune(scwp_ctx* ctx, int32_t reps, int32_t force, scwp_tune_result* out);

/* Set the autotuner's choice by hand: summed-area kernel variant (0 or 1, as
 * above) and bucket-group multiplier gmul (0.125..8) of the host plans.
 * SCWP_E_INVALID for variant 1 when a patch's buckets exceed the three-group
 * kernel's row table.  Synchronises; takes effect at the next synthesis. */
scwp_status scwp_set_sat_plan(scwp_ctx* ctx, int32_t variant, double gmul);

/* Stage timing with CUDA events on the context's stream: enable (1) or
 * disable (0).  scwp_timing_read sums, over the frames stepped since the
 * last read, the device time of [0] background FFT, [1] particle stages
 * (advect .. bin), [2] synthesis + blend, [3] whole frame, in ms, and the
 * number of frames; it synchronises and resets the sums.  With timing on,
 * frames launch one stage at a time and the background runs alone on the
 * context stream before the particle stages (instead of beside them on a
 * second stream), so that each sum times its stage by itself. */
scwp_status scwp_set_timing(scwp_ctx* ctx, int32_t enable);
scwp_status scwp_timing_read(scwp_ctx* ctx, double ms_sum[4], int64_t* frames);

/* Host-only: compute one table (SCWP_TAB_*, except SCWP_TAB_CARRY) of the
 * patch `pdesc` would get under `sdesc` at time step dt, without a context
 * or a GPU (the same float64 code scwp_add_patch runs).  bytes must be at
 * least the table's size; *count receives its element count. */
scwp_status scwp_host_table(const scwp_spectrum_desc* sdesc, const scwp_patch_desc* pdesc,
                            double dt, int32_t table, void* dst, size_t bytes, int64_t* count);

/* Background step without any device allocation, for callers that cannot
 * call cudaMalloc (code in host callbacks or real-time threads where an
 * allocation would synchronise the device, runtimes that only hand out
 * pre-registered buffers, plug-ins whose host owns every allocation).  The
 * paper has no counterpart: this is a deployment variant of the background
 * update of scwp_step (spectrum evolution + inverse 2-D FFT).
 *   h0     device, float32 complex interleaved [n][n] (FFT-natural order),
 *          8-byte aligned
 *   omega  device, float32 [n][n][2] dispersion w(k) as a float pair
 *          (hi, lo) with w = hi + lo (hi = (float)w, lo = (float)(w - hi)),
 *          8-byte aligned
 *   n      grid size: power of two, 8 <= n <= 512; larger grids are refused
 *          with SCWP_E_INVALID (the scratch is sized for 512 x 512)
 *   out    device, float32 [3][n][n]: h, Dx, Dy at x_j = j fft_L / n,
 *          4-byte aligned
 *   stream cudaStream_t (NULL: the legacy stream); asynchronous
 * The scratch (3 x 257 x 512 + 512 complex floats, about 3.0 MiB) is one
 * static __device__ array of the library:
 * every GPU that loads the library holds it until the process exits, and
 * every call shares it, so calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  The first call
 * on a device does a one-time set-up (looks up the array's address and
 * copies the twiddle table with a synchronous cudaMemcpy): make that first
 * call before any stream capture.  Returns SCWP_E_INVALID on bad arguments
 * (a null or misaligned pointer, a grid size out of range; nothing is
 * launched), SCWP_E_CUDA if the set-up or a launch fails. */
scwp_status scwp_background_noalloc(const float* h0, const float* omega, int32_t n, double fft_L,
                                    double choppiness, double t, float* out, void* stream);

/* Number of kernels this context has enqueued since creation (every
 * kernel of scwp_step / scwp_resynthesize counts once). */
scwp_status scwp_launch_count(scwp_ctx* ctx, int64_t* n);

/* Message of the last error on this context ("" if none). */
const char* scwp_last_error(const scwp_ctx* ctx);

/* Library version string. */
const char* scwp_version(void);

/* Free every device and host resource of the context (NULL is a no-op). */
void scwp_destroy(scwp_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Frame-step server: continuous batching of frame-step requests over many
 * device-resident scenes.  The paper has no counterpart (it runs one scene).
 *
 * Each scene is a context of its own (its spectrum, background and patches)
 * created by the server on the server's stream and allocator, in batched
 * mode.  scwp_server_tick takes every scene that has a pending request and
 * no frame in flight, enqueues each one's background and particle stages
 * (on eight internal streams) and runs the synthesis of all of them as ONE
 * launch over the union of their planned (patch, tile, bucket group) items,
 * heaviest first, followed by one group-sum blend launch (one such pair per
 * synthesis mode in use: a scene keeps its context's mode, by default
 * SCWP_SYNTH_SAT; SCWP_SYNTH_GATHER selects the tensor-core gather).
 * Per scene the arithmetic is that of a batched scwp_step, so each result
 * is the same whether the scene runs alone or in a mix.  At most
 * max_inflight ticks are outstanding; the next tick's particle stages
 * overlap the current tick's synthesis.  Requests of one scene run in
 * submission order, one frame per tick.
 * ------------------------------------------------------------------------- */
typedef struct scwp_server scwp_server;

typedef struct scwp_server_desc {
    void* stream;                /* cudaStream_t for the synthesis; NULL: legacy stream */
    int64_t hbm_budget_bytes;    /* device memory the scenes may hold; 0: no limit */
    int32_t max_inflight;        /* ticks outstanding at once, 1..16 */
    void* (*alloc)(size_t bytes, void* user);   /* as in scwp_spectrum_desc */
    void (*free)(void* ptr, void* user);
    void* alloc_user;
} scwp_server_desc;

typedef struct scwp_server_info {
    int32_t scenes;              /* admitted scenes                          */
    int32_t frames_in_flight;    /* scenes with a frame in an unfinished tick */
    int32_t ticks_in_flight;
    int32_t pad;
    int64_t pending_requests;    /* submitted, not yet in a tick             */
    int64_t device_bytes;        /* device memory held by admitted scenes    */
    int64_t budget_bytes;
    int64_t ticks_launched;
    int64_t requests_done;
} scwp_server_info;

/* SCWP_E_INVALID: bad descriptor; SCWP_E_CUDA: stream/event creation failed. */
scwp_status scwp_server_create(const scwp_server_desc* desc, scwp_server** out);

/* Admit a scene: creates its context (spec->stream and allocator are replaced
 * by the server's) with n_patches patches and plans its batched synthesis.
 * SCWP_E_NOMEM if its device memory would exceed the budget (the scene is
 * released again); any error of scwp_create / scwp_add_patch otherwise. */
scwp_status scwp_server_add_scene(scwp_server* sv, const scwp_spectrum_desc* spec, const scwp_patch_desc* patches,
                                  int32_t n_patches, int32_t* scene_id);

/* Release a scene and its device memory (SCWP_E_INVALID while it has a
 * frame in flight). */
scwp_status scwp_server_remove_scene(scwp_server* sv, int32_t scene_id);

/* Queue one frame step of dt seconds of a scene under a caller-chosen id. */
scwp_status scwp_server_submit(scwp_server* sv, int32_t scene_id, double dt, int64_t request_id);

/* Start one tick if a tick slot is free and any scene is ready; *started =
 * the number of requests it carries (0: nothing started). */
scwp_status scwp_server_tick(scwp_server* sv, int32_t* started);

/* Ids of completed requests, in completion order (at most max_ids; the rest
 * are reported by the next call).  Never blocks. */
scwp_status scwp_server_poll(scwp_server* sv, int64_t* done_ids, int32_t max_ids, int32_t* n_done);

/* The context of a scene, for scwp_height_map / scwp_stats_get of its last
 * completed frame (those calls run on the server stream). */
scwp_status scwp_server_scene(scwp_server* sv, int32_t scene_id, scwp_ctx** ctx);

scwp_status scwp_server_info_get(scwp_server* sv, scwp_server_info* out);
const char* scwp_server_last_error(scwp_server* sv);
void scwp_server_destroy(scwp_server* sv);

#ifdef __cplusplus
}
#endif
#endif /* SCWP_H */
