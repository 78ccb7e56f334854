// C ABI of the hybrid ocean (include/scwp.h): context and patch management,
// the per-frame orchestration of the sm_103a kernels (Sec. 4.1 pipeline), and
// the copy / inspection calls.  Host bookkeeping that decides integers (the
// injection carries, the wake's quantised angle) is float64 and lives in
// host_spectrum.cpp / here, compiled without floating-point contraction.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <algorithm>
#include <deque>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <queue>
#include <new>
#include <string>
#include <vector>

#include "../../include/scwp.h"
#include "host_spectrum.h"
#include "internal.h"
#include "philox.h"

using namespace scwp;

namespace scwp {
// Kernels enqueued by the calling thread.  A context call diffs this counter
// around its own work, which runs on the caller's thread, so launches made
// meanwhile by other threads (other contexts, the allocation-free
// background call) are never charged to it.
static thread_local long long t_launches = 0;
void count_launches(int n) { t_launches += n; }
long long launches_total() { return t_launches; }
}  // namespace scwp

namespace {

constexpr int kTimingRing = 4096;

struct PatchHost {
    scwp_patch_desc d{};
    int index = 0;
    PatchTablesHost T;
    PatchDev dev;
    std::vector<double> carry;        // [nb][2]
    std::vector<int32_t> nvalid;      // [nb][2]
    std::vector<int16_t> dirlist;     // [nb][2][nth]
    std::vector<BucketDev> bk;
    std::vector<int32_t> bin_cells;
    int64_t injected = 0;
    std::vector<double> energy;       // [nb]
    double band = 0;
    double ring_carry = 0.0;          // ring-ripple emission carry
    int64_t ring_total = 0;           // ring particles emitted so far
    std::vector<TcItem> tc_items;     // tensor-core synthesis items of this patch, launch order
    std::vector<BlendSpan> tc_spans;  // its group-sum blend spans (G > 1)
    TcItem* d_items = nullptr;
    BlendSpan* d_spans = nullptr;
    int partial_planes = 1;           // bucket-group partial planes allocated
    int tc_slots = 0;                 // resident CTA slots the plan assumed
    std::vector<TcItem> sat_items;    // summed-area synthesis items of this patch, launch order
    std::vector<BlendSpan> sat_spans;
    TcItem* d_sat_items = nullptr;
    BlendSpan* d_sat_spans = nullptr;
    int sat_groups = 1;
    int sat_slots = 0;
    int sat_item_cap = 0;             // capacity of d_sat_items (items of the largest G)
    int sat_parts = 1;                // parts each bucket's passes are split over (dense patches)
    bool sat3_ok = false;             // every bucket fits the three-group kernel's row table
};

// A frame (or a scene's part of a frame) captured as CUDA graphs, one per
// parity of the particle double buffers, with the pinned staging buffers
// and the device block through which each replay gets its parameters.
struct FrameGraph {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    bool valid[2] = {false, false};
    bool pending[2] = {false, false};
    uint64_t mask[2] = {0, 0};
    long long launches[2] = {0, 0};
    cudaEvent_t done[2] = {nullptr, nullptr};
    void* hstage[2] = {nullptr, nullptr};
    unsigned char* dparams = nullptr;
    size_t bytes = 0;
};

struct FrameEvents {
    cudaEvent_t e[6];                 // e0 start, e1 particles done, e2 synth start, e3 end, s0/s1 fft
};

}  // namespace

struct scwp_ctx {
    scwp_spectrum_desc d{};
    std::vector<double> edges;
    cudaStream_t st = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // particle-stage streams of a multi-patch context: patch i runs on
    // pst[i % pst.size()], all forked from and joined back into st
    std::vector<cudaStream_t> pst;
    std::vector<cudaEvent_t> pev;
    std::string err;
    scwp_status sticky = SCWP_OK;
    SpectrumModel sm;
    BgDev bg;
    float2* h0 = nullptr;
    float2* omega = nullptr;          // w(k) as float pairs (hi, lo)
    float2* tw = nullptr;
    float2* I = nullptr;              // row-pass intermediate of the background
    float* bgout = nullptr;
    int64_t frame = 0;
    double t = 0.0;
    double dt = -1.0;
    bool bg_valid = false;
    std::vector<PatchHost*> patches;
    std::vector<void*> allocs;
    int synth_mode = SCWP_SYNTH_SAT;
    bool timing = false;
    std::vector<FrameEvents> ring;
    int ring_n = 0;
    double ms_sum[4] = {0, 0, 0, 0};
    int64_t timed_frames = 0;
    int64_t launches = 0;             // kernels enqueued by this context
    // tensor-core synthesis: patch descriptors and parameters on the device,
    // and the batched plan (all patches in one launch)
    bool batched = false;
    bool synth_dirty = true;
    int b_lo = 0, b_hi = 1 << 30;     // buckets synthesised by the tensor-core modes
    int slots = 0;
    PatchDev* d_pdevs = nullptr;
    SynthParams* d_sps = nullptr;
    std::vector<TcItem> b_items;
    std::vector<BlendSpan> b_spans;
    TcItem* d_bitems = nullptr;
    BlendSpan* d_bspans = nullptr;
    // the batched plan of the summed-area synthesis
    int sat_slots = 0;
    int sat_variant = 0;              // 0: persistent nine-plane kernel, 1: three-group kernel
    double sat_gmul = 1.0;            // bucket-group multiplier of the plans (the autotuner's)
    std::vector<TcItem> s_items;
    std::vector<BlendSpan> s_spans;
    TcItem* d_sitems = nullptr;
    BlendSpan* d_sspans = nullptr;
    double s_makespan = 0.0;
    std::vector<double> s_work;
    double b_makespan = 0.0;
    // captured batched frames (one per parity of the particle buffers)
    FrameGraph gfull;                 // whole batched frames (scwp_step)
    FrameGraph gprep;                 // background + particle stages (the server's ticks)
    cudaStream_t gst = nullptr;       // capture origin (the caller's stream may be the legacy one)
    std::vector<InjectParams> ips;    // this frame's injection plans
    size_t alloc_bytes = 0;           // device memory held by the context
    unsigned int* queue = nullptr;    // work queue of the persistent summed-area synthesis (2 words)
    float* normal_scratch = nullptr;  // normals for host destinations
    size_t normal_bytes = 0;
    std::vector<double> b_work;       // estimated stages of each batched item
    std::vector<PatchDev> h_pdevs;    // host copies of the device descriptor arrays
    std::vector<SynthParams> h_sps;
};

namespace {

scwp_status fail(scwp_ctx* c, scwp_status s, const std::string& msg) {
    if (c) {
        c->err = msg;
        if (s == SCWP_E_CUDA || s == SCWP_E_TIMEOUT) c->sticky = s;
    }
    return s;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, SCWP_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void* dalloc(scwp_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (c->d.alloc) {
        p = c->d.alloc(bytes, c->d.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->allocs.push_back(p);
        c->alloc_bytes += bytes;
    }
    return p;
}

void dfree_all(scwp_ctx* c) {
    for (void* p : c->allocs) {
        if (c->d.free) c->d.free(p, c->d.alloc_user);
        else cudaFree(p);
    }
    c->allocs.clear();
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

scwp_status check_spectrum_desc(const scwp_spectrum_desc* d, std::string& why) {
    if (!d) { why = "null descriptor"; return SCWP_E_INVALID; }
    if (d->spectrum != SCWP_SPECTRUM_JONSWAP && d->spectrum != SCWP_SPECTRUM_PHILLIPS) { why = "spectrum"; return SCWP_E_INVALID; }
    if (d->spreading != SCWP_SPREAD_COS2S_MITSUYASU && d->spreading != SCWP_SPREAD_COS2) { why = "spreading"; return SCWP_E_INVALID; }
    if (!(d->wind_speed > 0)) { why = "wind_speed must be > 0"; return SCWP_E_INVALID; }
    if (d->spectrum == SCWP_SPECTRUM_JONSWAP && !(d->fetch > 0)) { why = "fetch must be > 0"; return SCWP_E_INVALID; }
    if (d->n_buckets < 1 || d->n_buckets > SCWP_MAX_BUCKETS) { why = "n_buckets out of range"; return SCWP_E_INVALID; }
    if (d->n_theta < 1 || d->n_theta > SCWP_MAX_THETA) { why = "n_theta out of range"; return SCWP_E_INVALID; }
    if (d->amp_mode != SCWP_AMP_NORMALIZED && d->amp_mode != SCWP_AMP_LITERAL) { why = "amp_mode"; return SCWP_E_INVALID; }
    if (!pow2(d->fft_n) || d->fft_n < 8 || d->fft_n > 4096) { why = "fft_n must be a power of two in [8, 4096]"; return SCWP_E_INVALID; }
    if (!(d->fft_L > 0)) { why = "fft_L must be > 0"; return SCWP_E_INVALID; }
    if (d->bucket_edges) {
        for (int i = 0; i < d->n_buckets; ++i)
            if (!(d->bucket_edges[i + 1] > d->bucket_edges[i]) || !(d->bucket_edges[i] > 0)) {
                why = "bucket_edges must be positive and ascending";
                return SCWP_E_INVALID;
            }
    }
    return SCWP_OK;
}

scwp_status check_patch_desc(const scwp_patch_desc* d, std::string& why) {
    if (!d) { why = "null descriptor"; return SCWP_E_INVALID; }
    if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384) { why = "patch size out of range"; return SCWP_E_INVALID; }
    if (!(d->cell > 0)) { why = "cell must be > 0"; return SCWP_E_INVALID; }
    if (d->max_particles < 1 || d->max_particles > (1 << 28)) { why = "max_particles out of range"; return SCWP_E_INVALID; }
    if (d->prefill < 0) { why = "prefill < 0"; return SCWP_E_INVALID; }
    if (d->n_buckets > SCWP_MAX_BUCKETS) { why = "n_buckets out of range"; return SCWP_E_INVALID; }
    if (d->emitter) {
        if (!(d->obj_path_radius > 0) || !(d->obj_radius > 0) || d->wake_rate < 0 || d->wake_rate > kMaxWakeRate ||
            d->ring_rate < 0 || d->ring_rate > 1 << 20 || d->heave_period < 0) {
            why = "emitter parameters";
            return SCWP_E_INVALID;
        }
    }
    return SCWP_OK;
}

void model_from_desc(const scwp_spectrum_desc& d, SpectrumModel& sm) {
    sm.init(d.spectrum, d.spreading, d.wind_speed, d.fetch, d.depth, d.wind_dir, d.gamma);
}

int patch_nb(const scwp_spectrum_desc& sd, const scwp_patch_desc& pd) {
    return pd.n_buckets > 0 ? pd.n_buckets : sd.n_buckets;
}

void build_tables(const scwp_spectrum_desc& sd, const std::vector<double>& edges,
                  const scwp_patch_desc& pd, const SpectrumModel& sm, PatchTablesHost& T) {
    const int nb = patch_nb(sd, pd);
    const double* e = (!edges.empty() && nb == sd.n_buckets) ? edges.data() : nullptr;
    const double lo = sd.omega_lo_mul > 0 ? sd.omega_lo_mul : 0.5;
    const double hi = sd.omega_hi_mul > 0 ? sd.omega_hi_mul : 2.5;
    T.build(sm, nb, e, lo, hi, sd.n_theta, sd.amp_mode, pd.width, pd.height, pd.cell,
            pd.inject_scale > 0 ? pd.inject_scale : 1.0, pd.obj_radius);
}

// bin side per bucket: 32 texels, doubled until the key space fits 16 bits
void bin_geometry(PatchHost& P) {
    const PatchTablesHost& T = P.T;
    int C = P.d.bin_cells > 0 ? P.d.bin_cells : 32;
    for (;;) {
        int64_t total = 0;
        for (int i = 0; i < T.nb; ++i) {
            const int64_t Cq = (int64_t)C * kQ;
            const int64_t nbx = ((int64_t)T.W * kQ + 2 * (int64_t)T.R[i]) / Cq + 1;
            const int64_t nby = ((int64_t)T.H * kQ + 2 * (int64_t)T.R[i]) / Cq + 1;
            total += nbx * nby;
        }
        if (total <= 65535 || P.d.bin_cells > 0 || C >= (1 << 14)) break;
        C *= 2;
    }
    P.bin_cells.assign(T.nb, C);
    P.bk.assign(T.nb, BucketDev{});
    int base = 0;
    for (int i = 0; i < T.nb; ++i) {
        BucketDev& b = P.bk[i];
        b.R = T.R[i];
        b.invR = (float)(1.0 / (double)T.R[i]);
        b.C = C * (int32_t)kQ;
        b.nbx = (int32_t)(((int64_t)T.W * kQ + 2 * (int64_t)T.R[i]) / b.C + 1);
        b.nby = (int32_t)(((int64_t)T.H * kQ + 2 * (int64_t)T.R[i]) / b.C + 1);
        b.base = base;
        base += b.nbx * b.nby;
    }
    P.dev.total_bins = base;
    int bits = 1;
    while ((1 << bits) < base + 1) ++bits;
    P.dev.key_bits = bits;
}

void valid_dirs(PatchHost& P) {
    const PatchTablesHost& T = P.T;
    P.nvalid.assign(T.nb * 2, 0);
    P.dirlist.assign((size_t)T.nb * 2 * T.nth, 0);
    for (int i = 0; i < T.nb; ++i)
        for (int s = 0; s < 2; ++s) {
            int n = 0;
            for (int j = 0; j < T.nth; ++j) {
                const int32_t vn = s == 0 ? T.vx[(size_t)i * T.nth + j] : T.vy[(size_t)i * T.nth + j];
                if (T.amp[(size_t)i * T.nth + j] > 0 && vn != 0)
                    P.dirlist[((size_t)i * 2 + s) * T.nth + n++] = (int16_t)j;
            }
            P.nvalid[i * 2 + s] = n;
        }
}

scwp_status upload_dt_tables(scwp_ctx* ctx, PatchHost& P) {
    const PatchTablesHost& T = P.T;
    const size_t ng = (size_t)T.nb * T.nth;
    std::vector<int4> vq(ng + (P.dev.emitter ? kWakeDirs : 0));
    for (size_t k = 0; k < ng; ++k) vq[k] = make_int4(T.vx[k], T.vy[k], T.qx[k], T.qy[k]);
    if (P.dev.emitter)
        for (int a = 0; a < kWakeDirs; ++a) vq[ng + a] = make_int4(T.wvx[a], T.wvy[a], T.wqx[a], T.wqy[a]);
    valid_dirs(P);
    CU(cudaMemcpyAsync(P.dev.vq, vq.data(), vq.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(P.dev.dirlist, P.dirlist.data(), P.dirlist.size() * sizeof(int16_t),
                       cudaMemcpyHostToDevice, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return SCWP_OK;
}

// Plans of the tensor-core synthesis.  Each (tile, bucket group) item's work
// is estimated in operand stages from the expected bump density of each
// bucket: steady-state shares proportional to (W Q + 2 R_i) / R_i^2 (the
// prefill rule), two bumps per particle, times the part of the tile's reach
// (the tile grown by R_i) that lies inside the particle domain (the patch
// grown by R_i).  Items run heaviest first, so in-order block dispatch
// approximates longest-processing-time scheduling.
constexpr double kItemStages = 2.0;   // set-up and read-out of one item, in stages
constexpr double kStageUs = 1.3;      // one stage on one CTA slot (two CTAs per SM)
constexpr double kHbmBytesPerUs = 6.8e6;

// expected operand stages of every (tile, bucket) of a patch, [tiles][nb]
std::vector<double> tile_bucket_stages(const PatchHost& P, int& tiles) {
    const PatchTablesHost& T = P.T;
    const int ts = synth_tc_tile(), kc = synth_tc_stage_bumps();
    const int ntx = (T.W + ts - 1) / ts, nty = (T.H + ts - 1) / ts;
    tiles = ntx * nty;
    // bumps: two per live particle (crest and trough)
    const double total = 2.0 * (P.d.prefill > 0 ? (double)P.d.prefill : 0.5 * (double)P.d.max_particles);
    std::vector<double> w(T.nb);
    double sw = 0.0;
    for (int i = 0; i < T.nb; ++i) {
        w[i] = ((double)T.W * kQ + 2.0 * T.R[i]) / ((double)T.R[i] * (double)T.R[i]);
        sw += w[i];
    }
    std::vector<double> est((size_t)tiles * T.nb);
    for (int i = 0; i < T.nb; ++i) {
        const double r = (double)T.R[i] / kQ;
        const double dens = total * w[i] / sw / ((T.W + 2 * r) * (T.H + 2 * r));
        for (int t = 0; t < tiles; ++t) {
            const double x0 = (t % ntx) * ts - r, x1 = (t % ntx + 1) * ts + r;
            const double y0 = (t / ntx) * ts - r, y1 = (t / ntx + 1) * ts + r;
            const double ax = std::max(0.0, std::min(x1, T.W + r) - std::max(x0, -r));
            const double ay = std::max(0.0, std::min(y1, T.H + r) - std::max(y0, -r));
            // bump centres that cover the whole tile go through the 3 x 3
            // moments, not the MMAs: the box (x_last - r, x_first + r),
            // shrunk by half a bin on each side for the bin rounding
            // (x0, x1 are the tile grown by r: the box is (x1 - 2r, x0 + 2r))
            const double hc = 0.5 * P.bin_cells[i];
            const double fx = std::max(0.0, std::min(x0 + 2 * r - hc, T.W + r) - std::max(x1 - 2 * r + hc, -r));
            const double fy = std::max(0.0, std::min(y0 + 2 * r - hc, T.H + r) - std::max(y1 - 2 * r + hc, -r));
            est[(size_t)t * T.nb + i] = std::ceil(dens * std::max(0.0, ax * ay - fx * fy) / kc);
        }
    }
    return est;
}

// Work of the summed-area synthesis per (tile, bucket), in the same stage
// units: a fixed part (three rounds of clearing, two prefix passes and the
// 3 x 3 contraction over the tile's texels) plus one part per candidate bump
// of the bins that reach the tile (its corner events).
constexpr double kSatBucketUs = 2.0;
constexpr double kSatBumpUs = 0.0008;

std::vector<double> tile_bucket_sat(const PatchHost& P, int& tiles, double* max_passes = nullptr) {
    const PatchTablesHost& T = P.T;
    const int ts = synth_sat_tile();
    const int ntx = (T.W + ts - 1) / ts, nty = (T.H + ts - 1) / ts;
    tiles = ntx * nty;
    const double total = 2.0 * (P.d.prefill > 0 ? (double)P.d.prefill : 0.5 * (double)P.d.max_particles);
    std::vector<double> w(T.nb);
    double sw = 0.0;
    for (int i = 0; i < T.nb; ++i) {
        w[i] = ((double)T.W * kQ + 2.0 * T.R[i]) / ((double)T.R[i] * (double)T.R[i]);
        sw += w[i];
    }
    std::vector<double> est((size_t)tiles * T.nb);
    for (int i = 0; i < T.nb; ++i) {
        const double r = (double)T.R[i] / kQ, c = (double)P.bin_cells[i];
        const double dens = total * w[i] / sw / ((T.W + 2 * r) * (T.H + 2 * r));
        for (int t = 0; t < tiles; ++t) {
            const double x0 = (t % ntx) * ts - r, x1 = (t % ntx + 1) * ts + r;
            const double y0 = (t / ntx) * ts - r, y1 = (t / ntx + 1) * ts + r;
            const double ax = std::max(0.0, std::min(x1 + c, T.W + r) - std::max(x0, -r));
            const double ay = std::max(0.0, std::min(y1 + c, T.H + r) - std::max(y0, -r));
            // dense pairs go in several passes, each with the fixed part
            const double n = dens * ax * ay;
            const double passes = std::max(1.0, std::ceil(n * std::sqrt(n) / (double)P.bk[i].sat_c));
            if (max_passes) *max_passes = std::max(*max_passes, passes);
            est[(size_t)t * T.nb + i] = (passes * kSatBucketUs + n * kSatBumpUs) / kStageUs;
        }
    }
    return est;
}

double item_work(const std::vector<double>& est, int nb, int t, int g, int G) {
    double s = kItemStages;
    for (int i = (g * nb) / G; i < ((g + 1) * nb) / G; ++i) s += est[(size_t)t * nb + i];
    return s;
}

// makespan of in-order dispatch of `work` (already in launch order) on `slots`
double makespan(const std::vector<double>& work, const std::vector<int>& order, int slots) {
    std::priority_queue<double, std::vector<double>, std::greater<double>> q;
    for (int k = 0; k < std::max(slots, 1); ++k) q.push(0.0);
    double m = 0.0;
    for (int it : order) {
        const double f = q.top() + work[it];
        q.pop();
        q.push(f);
        m = std::max(m, f);
    }
    return m;
}

std::vector<BlendSpan> blend_spans(const PatchHost& P, int G) {
    std::vector<BlendSpan> out;
    if (G <= 1) return out;
    const int nq = ((P.T.W + 3) / 4) * P.T.H;
    constexpr int kQuadsPerSpan = 256;   // one quad per thread of a 256-thread CTA
    for (int q0 = 0; q0 < nq; q0 += kQuadsPerSpan) out.push_back(BlendSpan{P.index, q0, std::min(nq, q0 + kQuadsPerSpan), G});
    return out;
}

// Parts K over which the summed-area items of a patch split each bucket's
// passes: the smallest K (up to kmax) that brings the patch's heaviest item
// to at most `cap` stages; a part item costs its set-up plus 1/K of the rest.
int sat_parts_for(double wmax, double cap, int kmax) {
    int K = 1;
    while (K < kmax && kItemStages + (wmax - kItemStages) / K > cap) ++K;
    return K;
}
double part_work(double w, int K) { return kItemStages + (w - kItemStages) / K; }

// Plan of one patch launched alone: G minimises the simulated makespan over
// the device's resident CTA slots plus the traffic of the group-sum blend.
// For the summed-area synthesis, gmul scales the chosen G (the autotuner's
// search axis), within [1, gcap].
void plan_patch(PatchHost& P, int slots, bool sat = false, double gmul = 1.0, int gcap = 16) {
    int tiles = 0;
    const std::vector<double> est = sat ? tile_bucket_sat(P, tiles) : tile_bucket_stages(P, tiles);
    const int nb = P.T.nb;
    double best_cost = 0.0;
    int& groups = sat ? P.sat_groups : P.dev.groups_tc;
    std::vector<TcItem>& plan = sat ? P.sat_items : P.tc_items;
    auto build = [&](int G) {   // the heaviest-first plan with G groups, and its modelled cost
        std::vector<double> work((size_t)tiles * G);
        for (int t = 0; t < tiles; ++t)
            for (int g = 0; g < G; ++g) work[(size_t)t * G + g] = item_work(est, nb, t, g, G);
        std::vector<int> order(work.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
        const double blend = G > 1 ? (G + 1) * 12.0 * P.T.W * P.T.H / kHbmBytesPerUs : 0.0;
        std::vector<TcItem> items;
        for (int k : order) items.push_back(TcItem{P.index, k / G, k % G, G});
        return std::make_pair(makespan(work, order, slots) * kStageUs + blend, items);
    };
    // the summed-area items cost about the same per bucket; the smallest G
    // that gives three waves over the slots, as far as the buckets allow
    const int gmax = std::max(1, std::min(std::min(nb, 16), gcap));
    int g_lo = 1;
    if (sat)
        while (g_lo < gmax && (double)tiles * g_lo < 3.0 * slots) ++g_lo;
    for (int G = g_lo; G <= gmax; ++G) {
        auto r = build(G);
        if (G == g_lo || r.first < best_cost) {
            best_cost = r.first;
            groups = G;
            plan.swap(r.second);
        }
    }
    if (sat && gmul != 1.0) {
        const int G = std::max(1, std::min(gmax, (int)std::lround(groups * gmul)));
        if (G != groups) {
            groups = G;
            plan = build(G).second;
        }
    }
    int K = 1;
    if (sat) {
        // dense patches: split each bucket's passes over K parts when the
        // heaviest item alone would outlast the balanced share of a slot
        // (the makespan's lower bound), with at most one wave of items
        double total = 0.0, wmax = 0.0;
        for (const TcItem& it : plan) {
            const double w = item_work(est, nb, it.tile, it.group, groups);
            total += w;
            wmax = std::max(wmax, w);
        }
        const int kwave = std::max(1, slots / std::max<int>(1, (int)plan.size()));
        K = sat_parts_for(wmax, total / std::max(slots, 1), std::max(1, std::min(std::min(8, kwave), gcap / groups)));
        if (K > 1) {
            std::vector<std::pair<double, TcItem>> parts;
            for (const TcItem& it : plan)
                for (int q = 0; q < K; ++q)
                    parts.push_back({part_work(item_work(est, nb, it.tile, it.group, groups), K),
                                     TcItem{it.patch, it.tile, it.group | (q << 16), groups | (K << 16)}});
            std::stable_sort(parts.begin(), parts.end(),
                             [](const std::pair<double, TcItem>& a, const std::pair<double, TcItem>& b) {
                                 return a.first > b.first;
                             });
            plan.clear();
            for (auto& pr : parts) plan.push_back(pr.second);
        }
        P.sat_parts = K;
    }
    (sat ? P.sat_spans : P.tc_spans) = blend_spans(P, groups * K);
}

// Resident CTA slots of a summed-area kernel variant on the current device
// (0: the persistent nine-plane kernel, 1: the three-group kernel).
int sat_slots_of(int variant) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = variant == 1 ? synth_sat3_ctas_per_sm() : synth_sat_ctas_per_sm();
    return sms * (per_sm > 0 ? per_sm : 1);
}

// Whether every bucket of the patch reaches at most the three-group kernel's
// row table of bin rows per tile: rows = floor((Y1 + 2R - 1) / C) -
// floor(Y0 / C) + 1 <= (63 Q + 2R - 1) / C + 2.
bool sat3_fits(const PatchHost& P) {
    const int cap = synth_sat3_row_cap();
    for (const BucketDev& b : P.bk)
        if ((63 * (int64_t)kQ + 2 * (int64_t)b.R - 1) / b.C + 2 > cap) return false;
    return true;
}

// Plan of all patches in one launch: each patch's G is the smallest that
// keeps its largest item under a quarter of the average per-slot load, and
// all items of all patches run heaviest first.
void plan_batched(scwp_ctx* ctx, int slots, std::vector<TcItem>& items, std::vector<BlendSpan>& spans,
                  double& model_makespan, std::vector<double>& item_work_out, bool sat = false) {
    items.clear();
    spans.clear();
    std::vector<std::vector<double>> est(ctx->patches.size());
    std::vector<int> tiles(ctx->patches.size());
    double total = 0.0;
    for (size_t k = 0; k < ctx->patches.size(); ++k) {
        est[k] = sat ? tile_bucket_sat(*ctx->patches[k], tiles[k]) : tile_bucket_stages(*ctx->patches[k], tiles[k]);
        for (double e : est[k]) total += e;
        total += kItemStages * tiles[k];
    }
    const double cap = 0.25 * total / std::max(slots, 1);
    std::vector<double> work;
    for (size_t k = 0; k < ctx->patches.size(); ++k) {
        const PatchHost& P = *ctx->patches[k];
        const int nb = P.T.nb, gmax = std::min(std::min(nb, 16), P.partial_planes);
        int G = 1;
        for (;; ++G) {
            double mx = 0.0;
            for (int t = 0; t < tiles[k]; ++t)
                for (int g = 0; g < G; ++g) mx = std::max(mx, item_work(est[k], nb, t, g, G));
            if (mx <= cap || G >= gmax) break;
        }
        // summed-area items: no more groups than the patch's own plan takes
        // (enough waves for the patch alone; more only adds blend traffic),
        // and each bucket's passes split over K parts where an item would
        // still outlast the balanced per-slot share of the frame (dense
        // patches whose buckets take many passes)
        int K = 1;
        if (sat) {
            G = std::max(1, std::min(G, P.sat_groups));
            double wmax = 0.0;
            for (int t = 0; t < tiles[k]; ++t)
                for (int g = 0; g < G; ++g) wmax = std::max(wmax, item_work(est[k], nb, t, g, G));
            K = sat_parts_for(wmax, 4.0 * cap, std::max(1, std::min(8, P.partial_planes / G)));
        }
        for (int t = 0; t < tiles[k]; ++t)
            for (int g = 0; g < G; ++g)
                for (int q = 0; q < K; ++q) {
                    items.push_back(K > 1 ? TcItem{P.index, t, g | (q << 16), G | (K << 16)} : TcItem{P.index, t, g, G});
                    work.push_back(part_work(item_work(est[k], nb, t, g, G), K));
                }
        const std::vector<BlendSpan> sp = blend_spans(P, G * K);
        spans.insert(spans.end(), sp.begin(), sp.end());
    }
    std::vector<int> order(items.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
    model_makespan = makespan(work, order, slots);
    std::vector<TcItem> sorted;
    item_work_out.clear();
    for (int k : order) {
        sorted.push_back(items[k]);
        item_work_out.push_back(work[k]);
    }
    items.swap(sorted);
}

scwp_status ready(scwp_ctx* ctx) {
    if (!ctx) return SCWP_E_INVALID;
    if (ctx->sticky != SCWP_OK) return ctx->sticky;
    return SCWP_OK;
}

SynthParams synth_params(scwp_ctx* ctx, const PatchHost& P) {
    SynthParams sp{};
    sp.W = P.T.W;
    sp.H = P.T.H;
    sp.nb = P.T.nb;
    sp.lam_half = (float)(0.5 * ctx->d.choppiness);
    sp.band = (float)P.band;
    const double N = ctx->d.fft_n, L = ctx->d.fft_L;
    double fx0 = (P.d.origin_x + 0.5 * P.d.cell) * N / L;
    double fy0 = (P.d.origin_y + 0.5 * P.d.cell) * N / L;
    fx0 -= N * std::floor(fx0 / N);
    fy0 -= N * std::floor(fy0 / N);
    sp.fx0 = (float)fx0;
    sp.fy0 = (float)fy0;
    sp.fsx = (float)(P.d.cell * N / L);
    sp.N = ctx->d.fft_n;
    sp.bg = ctx->bgout;
    // every record amplitude is a table entry or the wake amplitude
    double amax = std::fabs(P.d.wake_amp);
    for (double a : P.T.amp) amax = std::max(amax, std::fabs(a));
    int e = 0;
    if (amax > 0) {
        std::frexp(amax, &e);   // amax in [2^(e-1), 2^e)
        e = std::min(std::max(13 - e, -60), 60);
    }
    sp.row_scale = (float)std::ldexp(1.0, e);
    sp.b_lo = std::max(0, ctx->b_lo);
    sp.b_hi = std::min(P.T.nb, ctx->b_hi);
    return sp;
}

scwp_status reset_frame_stats(scwp_ctx* ctx, PatchHost& P, cudaStream_t st) {
    CU(cudaMemsetAsync(P.dev.stats, 0, 2 * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(P.dev.stats + 3, 0, ((size_t)P.T.nb + 1) * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(P.dev.stats + 5 + P.T.nb, 0, sizeof(unsigned long long), st));
    return SCWP_OK;
}

// drop the captured frames (after a change that the captures baked in)
void graph_reset(FrameGraph& G) {
    for (int k = 0; k < 2; ++k) {
        if (G.pending[k] && G.done[k]) cudaEventSynchronize(G.done[k]);
        G.pending[k] = false;
        if (G.exec[k]) cudaGraphExecDestroy(G.exec[k]);
        G.exec[k] = nullptr;
        G.valid[k] = false;
    }
    cudaGetLastError();
}

void graph_reset(scwp_ctx* ctx) {
    graph_reset(ctx->gfull);
    graph_reset(ctx->gprep);
}

// streams for the particle stages of up to kParticleStreams patches at once
constexpr int kParticleStreams = 8;
scwp_status particle_streams(scwp_ctx* ctx) {
    const size_t want = std::min<size_t>(ctx->patches.size(), kParticleStreams);
    while (ctx->pst.size() < want) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            if (s) cudaStreamDestroy(s);
            cudaGetLastError();
            return fail(ctx, SCWP_E_CUDA, "particle streams");
        }
        ctx->pst.push_back(s);
        ctx->pev.push_back(e);
    }
    return SCWP_OK;
}

// device copies of the patch descriptors and synthesis parameters (and the
// batched plan) after the set of patches or the batching mode changed
scwp_status sync_synth(scwp_ctx* ctx) {
    if (!ctx->synth_dirty) return SCWP_OK;
    const size_t n = ctx->patches.size();
    std::vector<PatchDev>& pd = ctx->h_pdevs;
    std::vector<SynthParams>& sp = ctx->h_sps;
    pd.resize(n);
    sp.resize(n);
    for (size_t k = 0; k < n; ++k) {
        pd[k] = ctx->patches[k]->dev;
        sp[k] = synth_params(ctx, *ctx->patches[k]);
    }
    ctx->d_pdevs = (PatchDev*)dalloc(ctx, std::max<size_t>(1, n) * sizeof(PatchDev));
    ctx->d_sps = (SynthParams*)dalloc(ctx, std::max<size_t>(1, n) * sizeof(SynthParams));
    if (!ctx->d_pdevs || !ctx->d_sps) return fail(ctx, SCWP_E_NOMEM, "synthesis descriptors");
    CU(cudaMemcpyAsync(ctx->d_pdevs, pd.data(), n * sizeof(PatchDev), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(ctx->d_sps, sp.data(), n * sizeof(SynthParams), cudaMemcpyHostToDevice, ctx->st));
    if (ctx->batched) {
        plan_batched(ctx, ctx->slots, ctx->b_items, ctx->b_spans, ctx->b_makespan, ctx->b_work);
        ctx->d_bitems = (TcItem*)dalloc(ctx, std::max<size_t>(1, ctx->b_items.size()) * sizeof(TcItem));
        ctx->d_bspans = (BlendSpan*)dalloc(ctx, std::max<size_t>(1, ctx->b_spans.size()) * sizeof(BlendSpan));
        if (!ctx->d_bitems || !ctx->d_bspans) return fail(ctx, SCWP_E_NOMEM, "batched plan");
        CU(cudaMemcpyAsync(ctx->d_bitems, ctx->b_items.data(), ctx->b_items.size() * sizeof(TcItem),
                           cudaMemcpyHostToDevice, ctx->st));
        if (!ctx->b_spans.empty())
            CU(cudaMemcpyAsync(ctx->d_bspans, ctx->b_spans.data(), ctx->b_spans.size() * sizeof(BlendSpan),
                               cudaMemcpyHostToDevice, ctx->st));
        plan_batched(ctx, ctx->sat_slots, ctx->s_items, ctx->s_spans, ctx->s_makespan, ctx->s_work, true);
        ctx->d_sitems = (TcItem*)dalloc(ctx, std::max<size_t>(1, ctx->s_items.size()) * sizeof(TcItem));
        ctx->d_sspans = (BlendSpan*)dalloc(ctx, std::max<size_t>(1, ctx->s_spans.size()) * sizeof(BlendSpan));
        if (!ctx->d_sitems || !ctx->d_sspans) return fail(ctx, SCWP_E_NOMEM, "batched plan");
        CU(cudaMemcpyAsync(ctx->d_sitems, ctx->s_items.data(), ctx->s_items.size() * sizeof(TcItem),
                           cudaMemcpyHostToDevice, ctx->st));
        if (!ctx->s_spans.empty())
            CU(cudaMemcpyAsync(ctx->d_sspans, ctx->s_spans.data(), ctx->s_spans.size() * sizeof(BlendSpan),
                               cudaMemcpyHostToDevice, ctx->st));
    }
    // the host vectors are copied before they go out of scope
    CU(cudaStreamSynchronize(ctx->st));
    ctx->synth_dirty = false;
    return SCWP_OK;
}

scwp_status synthesize(scwp_ctx* ctx, int mode) {
    const bool split = mode != SCWP_SYNTH_GATHER_FP16;
    if (mode == SCWP_SYNTH_SAT) {
        scwp_status s = sync_synth(ctx);
        if (s != SCWP_OK) return s;
        auto launch = [&](const TcItem* it, int n, const BlendSpan* sp, int ns) {
            return ctx->sat_variant == 1 ? launch_synth_sat3(it, n, ctx->d_pdevs, ctx->d_sps, sp, ns, ctx->st)
                                         : launch_synth_sat(it, n, ctx->d_pdevs, ctx->d_sps, sp, ns, ctx->queue, ctx->st);
        };
        if (ctx->batched) {
            CU(launch(ctx->d_sitems, (int)ctx->s_items.size(), ctx->d_sspans, (int)ctx->s_spans.size()));
        } else {
            for (PatchHost* P : ctx->patches)
                CU(launch(P->d_sat_items, (int)P->sat_items.size(), P->d_sat_spans, (int)P->sat_spans.size()));
        }
        return SCWP_OK;
    }
    if (mode == SCWP_SYNTH_GATHER || mode == SCWP_SYNTH_GATHER_FP16) {
        scwp_status s = sync_synth(ctx);
        if (s != SCWP_OK) return s;
        if (ctx->batched) {
            CU(launch_synth_tc(ctx->d_bitems, (int)ctx->b_items.size(), ctx->d_pdevs, ctx->d_sps, ctx->d_bspans,
                               (int)ctx->b_spans.size(), ctx->st, split));
            return SCWP_OK;
        }
    }
    for (PatchHost* P : ctx->patches) {
        const SynthParams sp = synth_params(ctx, *P);
        if (mode == SCWP_SYNTH_LAYERED) {
            PatchDev& D = P->dev;
            const size_t need = layered_scratch_bytes(D, P->T.R.data());
            if (D.layers_bytes < need) {
                // lazily sized on the first layered synthesis of this patch
                D.layers = (float*)dalloc(ctx, need);
                if (!D.layers) return fail(ctx, SCWP_E_NOMEM, "layered scratch");
                D.layers_bytes = need;
            }
            std::vector<int> base(P->T.nb), nbins(P->T.nb);
            for (int i = 0; i < P->T.nb; ++i) {
                base[i] = P->bk[i].base;
                nbins[i] = P->bk[i].nbx * P->bk[i].nby;
            }
            CU(launch_layered(D, sp, P->T.R.data(), base.data(), nbins.data(), ctx->st));
        } else if (mode == SCWP_SYNTH_GATHER_FP32) {
            CU(launch_synth_gather(P->dev, sp, ctx->st));
        } else {
            CU(launch_synth_tc(P->d_items, (int)P->tc_items.size(), ctx->d_pdevs, ctx->d_sps, P->d_spans,
                               (int)P->tc_spans.size(), ctx->st, split));
        }
    }
    return SCWP_OK;
}

}  // namespace

// =============================================================================
extern "C" {

const char* scwp_version(void) { return "scwp 0.1 (sm_103a)"; }

const char* scwp_last_error(const scwp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

scwp_status scwp_create(const scwp_spectrum_desc* desc, scwp_ctx** out) {
    if (!out) return SCWP_E_INVALID;
    *out = nullptr;
    std::string why;
    scwp_status s = check_spectrum_desc(desc, why);
    if (s != SCWP_OK) return s;
    scwp_ctx* ctx = new (std::nothrow) scwp_ctx();
    if (!ctx) return SCWP_E_NOMEM;
    ctx->d = *desc;
    if (desc->bucket_edges) ctx->edges.assign(desc->bucket_edges, desc->bucket_edges + desc->n_buckets + 1);
    ctx->d.bucket_edges = nullptr;
    ctx->st = (cudaStream_t)desc->stream;
    model_from_desc(ctx->d, ctx->sm);
    auto bail = [&](scwp_status st) {
        scwp_destroy(ctx);
        return st;
    };
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->gfull.done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->gfull.done[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->gprep.done[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->gprep.done[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bail(SCWP_E_CUDA);
    }
    const int N = desc->fft_n;
    std::vector<float> h0;
    std::vector<double> om;
    build_background(ctx->sm, N, desc->fft_L, desc->seed, h0, om);
    std::vector<float2> tw(N, make_float2(0.f, 0.f));   // the tables take at most N / 3 entries
    build_background_twiddles(N, tw.data());
    const size_t NN = (size_t)N * N;
    ctx->h0 = (float2*)dalloc(ctx, NN * sizeof(float2));
    ctx->omega = (float2*)dalloc(ctx, NN * sizeof(float2));
    ctx->tw = (float2*)dalloc(ctx, N * sizeof(float2));
    ctx->I = (float2*)dalloc(ctx, background_scratch_elems(N) * sizeof(float2));
    ctx->bgout = (float*)dalloc(ctx, 3 * NN * sizeof(float));
    ctx->queue = (unsigned int*)dalloc(ctx, 2 * sizeof(unsigned int));
    if (!ctx->h0 || !ctx->omega || !ctx->tw || !ctx->I || !ctx->bgout || !ctx->queue) return bail(SCWP_E_NOMEM);
    // w(k) split into float pairs on the host: hi = (float)w, lo = (float)(w - hi)
    std::vector<float2> omhl(NN);
    for (size_t k = 0; k < NN; ++k) {
        const float hi = (float)om[k];
        omhl[k] = make_float2(hi, (float)(om[k] - (double)hi));
    }
    if (cudaMemcpy(ctx->h0, h0.data(), NN * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->omega, omhl.data(), NN * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ctx->bgout, 0, 3 * NN * sizeof(float)) != cudaSuccess ||
        cudaMemset(ctx->queue, 0, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        return bail(SCWP_E_CUDA);
    }
    ctx->bg.N = N;
    ctx->bg.h0 = ctx->h0;
    ctx->bg.omega = ctx->omega;
    ctx->bg.tw = ctx->tw;
    ctx->bg.I = ctx->I;
    ctx->bg.out = ctx->bgout;
    ctx->bg.lam = (float)desc->choppiness;
    ctx->bg.dk = (float)(2.0 * M_PI / desc->fft_L);
    *out = ctx;
    return SCWP_OK;
}

scwp_status scwp_add_patch(scwp_ctx* ctx, const scwp_patch_desc* desc, int32_t* patch_id) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    std::string why;
    if ((s = check_patch_desc(desc, why)) != SCWP_OK) return fail(ctx, s, why);
    if (!ctx->edges.empty() && desc->n_buckets > 0 && desc->n_buckets != ctx->d.n_buckets) {
        // explicit edges belong to the spectrum's bucket count; another count
        // falls back to the equal-energy partition
    }
    PatchHost* P = new (std::nothrow) PatchHost();
    if (!P) return fail(ctx, SCWP_E_NOMEM, "host allocation");
    P->d = *desc;
    P->index = (int)ctx->patches.size();
    build_tables(ctx->d, ctx->edges, P->d, ctx->sm, P->T);
    P->band = desc->band > 0 ? desc->band : std::min(desc->width, desc->height) / 8.0;
    const PatchTablesHost& T = P->T;
    PatchDev& D = P->dev;
    D.W = T.W;
    D.H = T.H;
    D.nb = T.nb;
    D.nth = T.nth;
    D.cap = desc->max_particles;
    D.emitter = desc->emitter ? 1 : 0;
    D.wake_amp = (float)desc->wake_amp;
    bin_geometry(*P);
    // |A| bound per bucket: its directions' amplitudes and, with an emitter,
    // the wake amplitude (wake directions may sit in any bucket)
    std::vector<float> amax(T.nb, 0.f);
    for (int i = 0; i < T.nb; ++i) {
        for (int j = 0; j < T.nth; ++j) amax[i] = std::max(amax[i], std::fabs((float)T.amp[(size_t)i * T.nth + j]));
        if (D.emitter) amax[i] = std::max(amax[i], std::fabs(D.wake_amp));
    }
    // Summed-area passes.  The kernel rounds each corner weight once to an
    // integer unit of 2^-30 * 1.001 m A_max for a pass of m candidates; the
    // rounding errors of the n candidates that reach a texel add up to about
    // sqrt(n) m A_max 2^-31 per S_ij, of which 3/4 reach h (worst texel of a
    // tile: ~2 sigma).  A (tile, bucket) of n candidates therefore goes in
    // k = ceil(n^1.5 / c) passes of n / k candidates, c = eps Hs 2^31 /
    // (0.6 A_max), which keeps that error under eps = 2e-5 Hs / sqrt(nb) per
    // bucket, so that the nb buckets of a texel stay within about 2e-5 Hs
    // together (measured worst texel of the 32-patch batched workload before
    // this bound: 1.7e-4 Hs).  That is one pass for nearly every tile of the
    // realistic and mixed_large scenes and up to a few tens on patches holding
    // tens of particles per texel.
    {
        const double hs = 4.0 * std::sqrt(ctx->sm.m0());
        const double eps = 2e-5 * hs / std::sqrt((double)T.nb);
        for (int i = 0; i < T.nb; ++i)
            P->bk[i].sat_c = amax[i] > 0 ? (float)(eps * 2147483648.0 / (0.6 * (double)amax[i])) : 3.0e38f;
    }
    const size_t cap = (size_t)D.cap;
    D.nblk_c = (int)((cap + 1023) / 1024);
    D.nblk_s = (int)((2 * cap + kSortTile - 1) / kSortTile);
    D.nblk_o = (int)((2 * cap + kSortPassTile - 1) / kSortPassTile);
    bool ok = true;
    for (int k = 0; k < 2; ++k) {
        D.x[k] = (int32_t*)dalloc(ctx, cap * 4);
        D.y[k] = (int32_t*)dalloc(ctx, cap * 4);
        D.bd[k] = (uint32_t*)dalloc(ctx, cap * 4);
        D.keys[k] = (uint32_t*)dalloc(ctx, 2 * cap * 4);
        D.vals[k] = (uint32_t*)dalloc(ctx, 2 * cap * 4);
        ok = ok && D.x[k] && D.y[k] && D.bd[k] && D.keys[k] && D.vals[k];
    }
    D.count = (int32_t*)dalloc(ctx, 3 * sizeof(int32_t));
    D.flags = (uint8_t*)dalloc(ctx, cap);
    D.blk = (uint32_t*)dalloc(ctx, ((size_t)D.nblk_c + 1) * 4);
    const size_t ng = (size_t)T.nb * T.nth;
    D.vq = (int4*)dalloc(ctx, (ng + (D.emitter ? kWakeDirs : 0)) * sizeof(int4));
    D.dirlist = (int16_t*)dalloc(ctx, (size_t)T.nb * 2 * T.nth * sizeof(int16_t));
    D.amp = (float*)dalloc(ctx, ng * sizeof(float));
    D.bk = (BucketDev*)dalloc(ctx, T.nb * sizeof(BucketDev));
    D.rot = (float2*)dalloc(ctx, (size_t)T.nb * kRotN * sizeof(float2));
    {
        const int ts = synth_tc_tile();
        D.phase_len = std::max((T.W + ts - 1) / ts, (T.H + ts - 1) / ts) * ts;
        D.phase = (float2*)dalloc(ctx, (size_t)T.nb * D.phase_len * sizeof(float2));
        D.amax = (float*)dalloc(ctx, (size_t)T.nb * sizeof(float));
    }
    const size_t sort_words = (size_t)kMaxSortPasses * (256 + 2 + (size_t)256 * D.nblk_o);
    D.hist = (uint32_t*)dalloc(ctx, sort_words * 4);
    if (D.hist) {
        D.sort_ticket = D.hist + (size_t)kMaxSortPasses * 256;
        D.sort_status = D.sort_ticket + (size_t)kMaxSortPasses * 2;
    }
    D.offsets = (uint32_t*)dalloc(ctx, ((size_t)D.total_bins + 1) * 4);
    D.rec = (BumpRec*)dalloc(ctx, 2 * cap * sizeof(BumpRec));
    D.pk = (int4*)dalloc(ctx, cap * sizeof(int4));
    D.out = (float*)dalloc(ctx, (size_t)3 * T.W * T.H * sizeof(float));
    {
        // split the synthesis into bucket groups so that a frame has enough
        // CTAs to fill every SM several times over (about 4 waves of 3 CTAs
        // per SM on 152 SMs); each group writes its own partial sums
        auto groups_for = [&](int tiles, int ctas_per_sm) {
            int G = (4 * 152 * ctas_per_sm + tiles - 1) / tiles;
            if (G > T.nb) G = T.nb;
            return G < 1 ? 1 : G;
        };
        D.groups = groups_for(((T.W + 63) / 64) * ((T.H + 63) / 64), 2);       // CUDA-core tiles
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = synth_tc_ctas_per_sm();
        P->tc_slots = sms * (per_sm > 0 ? per_sm : 1);
        ctx->slots = P->tc_slots;
        D.patch = P->index;
        plan_patch(*P, P->tc_slots);
        P->sat3_ok = sat3_fits(*P);
        // partial planes for any plan the autotuner may choose: up to twice
        // the groups either summed-area variant plans on its own
        int gsat = 1;
        for (int v = 0; v < 2; ++v) {
            plan_patch(*P, sat_slots_of(v), true);
            gsat = std::max(gsat, P->sat_groups);
        }
        const int nbmax = std::min(T.nb, 16);
        // planes: room for twice the groups, and on dense patches (buckets
        // expected to take several passes) of up to 0.35M texels (at most
        // 256 MiB of planes) for 64 planes, so that their buckets' passes
        // can split into parts
        int gpart = std::min(nbmax, 2 * gsat);
        double max_passes = 0.0;
        int tiles_est = 0;
        tile_bucket_sat(*P, tiles_est, &max_passes);
        if (max_passes >= 2.0 && (size_t)64 * 12 * T.W * T.H <= ((size_t)256 << 20)) gpart = 64;
        P->partial_planes = std::max(std::max(D.groups, D.groups_tc), gpart);
        const int variant = (ctx->sat_variant == 1 && P->sat3_ok) ? 1 : 0;
        P->sat_slots = sat_slots_of(variant);
        ctx->sat_slots = P->sat_slots;
        plan_patch(*P, P->sat_slots, true, ctx->sat_gmul, P->partial_planes);
        P->d_items = (TcItem*)dalloc(ctx, P->tc_items.size() * sizeof(TcItem));
        P->d_spans = (BlendSpan*)dalloc(ctx, std::max<size_t>(1, P->tc_spans.size()) * sizeof(BlendSpan));
        int tiles_sat = 0;
        tile_bucket_sat(*P, tiles_sat);
        P->sat_item_cap = tiles_sat * P->partial_planes;   // G K <= the planes
        P->d_sat_items = (TcItem*)dalloc(ctx, (size_t)P->sat_item_cap * sizeof(TcItem));
        P->d_sat_spans = (BlendSpan*)dalloc(ctx, std::max<size_t>(1, blend_spans(*P, 2).size()) * sizeof(BlendSpan));
        ok = ok && P->d_items && P->d_spans && P->d_sat_items && P->d_sat_spans;
        const int G = P->partial_planes;
        if (G > 1) {
            D.partial = (float*)dalloc(ctx, (size_t)G * 3 * T.W * T.H * sizeof(float));
            ok = ok && D.partial;
        }
    }
    D.stats = (unsigned long long*)dalloc(ctx, (6 + (size_t)T.nb) * sizeof(unsigned long long));
    ok = ok && D.count && D.flags && D.blk && D.vq && D.dirlist && D.amp && D.bk && D.rot && D.phase && D.amax && D.hist &&
         D.offsets && D.rec && D.pk && D.out && D.stats;
    if (!ok) {
        delete P;
        return fail(ctx, SCWP_E_NOMEM, "device allocation failed");
    }
    std::vector<float> ampf(ng);
    for (size_t k = 0; k < ng; ++k) ampf[k] = (float)T.amp[k];
    // prefill (reading: bucket shares proportional to (W Q + 2 R_i) / R_i^2)
    std::vector<int32_t> px, py;
    std::vector<uint32_t> pbd;
    if (desc->prefill > 0) {
        const int64_t Wq = (int64_t)T.W * kQ, Hq = (int64_t)T.H * kQ;
        std::vector<double> w(T.nb);
        double sw = 0.0;
        for (int i = 0; i < T.nb; ++i) {
            w[i] = (double)(Wq + 2 * (int64_t)T.R[i]) / ((double)T.R[i] * (double)T.R[i]);
            sw += w[i];
        }
        for (int i = 0; i < T.nb; ++i) {
            const int64_t pop = (int64_t)std::floor((double)desc->prefill * w[i] / sw + 0.5);
            std::vector<int> valid;
            for (int j = 0; j < T.nth; ++j)
                if (T.amp[(size_t)i * T.nth + j] > 0) valid.push_back(j);
            if (pop <= 0 || valid.empty()) continue;
            const uint64_t R = (uint64_t)T.R[i];
            for (int64_t n = 0; n < pop; ++n) {
                const U4 u = philox4x32_10(0u, (uint32_t)P->index, (uint32_t)i | (3u << 16), (uint32_t)n,
                                           ctx->d.seed);
                const int32_t x = (int32_t)(-(int64_t)R + (int64_t)(((uint64_t)u.x * ((uint64_t)Wq + 2 * R)) >> 32));
                const int32_t y = (int32_t)(-(int64_t)R + (int64_t)(((uint64_t)u.y * ((uint64_t)Hq + 2 * R)) >> 32));
                px.push_back(x);
                py.push_back(y);
                pbd.push_back(((uint32_t)i << 16) | (uint32_t)valid[n % valid.size()]);
            }
        }
    }
    int32_t n0 = (int32_t)std::min<size_t>(px.size(), cap);
    uint64_t flags0 = px.size() > cap ? kErrCapacity : 0;
    int32_t counts[3] = {n0, n0, n0};
    CU(cudaMemcpyAsync(D.amp, ampf.data(), ng * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(D.bk, P->bk.data(), T.nb * sizeof(BucketDev), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(P->d_items, P->tc_items.data(), P->tc_items.size() * sizeof(TcItem), cudaMemcpyHostToDevice,
                       ctx->st));
    if (!P->tc_spans.empty())
        CU(cudaMemcpyAsync(P->d_spans, P->tc_spans.data(), P->tc_spans.size() * sizeof(BlendSpan),
                           cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(P->d_sat_items, P->sat_items.data(), P->sat_items.size() * sizeof(TcItem),
                       cudaMemcpyHostToDevice, ctx->st));
    if (!P->sat_spans.empty())
        CU(cudaMemcpyAsync(P->d_sat_spans, P->sat_spans.data(), P->sat_spans.size() * sizeof(BlendSpan),
                           cudaMemcpyHostToDevice, ctx->st));
    // per-bucket phase steps of n texels: e^{i pi n Q / R_i}, n < kRotN
    std::vector<float2> rot((size_t)T.nb * kRotN);
    for (int i = 0; i < T.nb; ++i)
        for (int n = 0; n < kRotN; ++n) {
            const double a = M_PI * (double)n * (double)kQ / (double)T.R[i];
            rot[(size_t)i * kRotN + n] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    CU(cudaMemcpyAsync(D.rot, rot.data(), rot.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->st));
    // per-bucket kernel phase of every texel centre X_n = n Q + Q/2: the
    // tensor-core synthesis reads its tile rows' and columns' factors here
    // (reduced exactly modulo 2 R_i in integers, the angle in float64)
    std::vector<float2> phase((size_t)T.nb * D.phase_len);
    for (int i = 0; i < T.nb; ++i) {
        const int64_t R2 = 2 * (int64_t)T.R[i];
        for (int n = 0; n < D.phase_len; ++n) {
            const int64_t pm = ((int64_t)n * kQ + kQ / 2) % R2;
            const double a = M_PI * ((double)pm / (double)T.R[i]);
            phase[(size_t)i * D.phase_len + n] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    }
    CU(cudaMemcpyAsync(D.phase, phase.data(), phase.size() * sizeof(float2), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemcpyAsync(D.amax, amax.data(), amax.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaMemsetAsync(D.flags, 0, cap, ctx->st));
    CU(cudaMemsetAsync(D.hist, 0, sort_words * 4, ctx->st));
    CU(cudaMemsetAsync(D.stats, 0, (6 + (size_t)T.nb) * sizeof(unsigned long long), ctx->st));
    CU(cudaMemsetAsync(D.offsets, 0, ((size_t)D.total_bins + 1) * 4, ctx->st));
    CU(cudaMemsetAsync(D.out, 0, (size_t)3 * T.W * T.H * sizeof(float), ctx->st));
    if (n0 > 0) {
        CU(cudaMemcpyAsync(D.x[0], px.data(), n0 * 4, cudaMemcpyHostToDevice, ctx->st));
        CU(cudaMemcpyAsync(D.y[0], py.data(), n0 * 4, cudaMemcpyHostToDevice, ctx->st));
        CU(cudaMemcpyAsync(D.bd[0], pbd.data(), n0 * 4, cudaMemcpyHostToDevice, ctx->st));
    }
    CU(cudaMemcpyAsync(D.count, counts, sizeof(counts), cudaMemcpyHostToDevice, ctx->st));
    if (flags0) CU(cudaMemcpyAsync(D.stats + 2, &flags0, sizeof(flags0), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    P->carry.assign((size_t)T.nb * 2, 0.0);
    P->energy.assign(T.nb, 0.0);
    graph_reset(ctx);
    ctx->patches.push_back(P);
    ctx->synth_dirty = true;
    if (patch_id) *patch_id = P->index;
    // velocity tables for the current dt (a provisional 1/60 s before the
    // first step, so the trough offsets are valid for scwp_resynthesize)
    P->T.set_dt(ctx->dt > 0 ? ctx->dt : 1.0 / 60.0);
    s = upload_dt_tables(ctx, *P);
    if (s != SCWP_OK) return s;
    return SCWP_OK;
}

static scwp_status record(scwp_ctx* ctx, cudaEvent_t e, cudaStream_t st) {
    CU(cudaEventRecord(e, st));
    return SCWP_OK;
}

static scwp_status drain_ring(scwp_ctx* ctx) {
    for (int i = 0; i < ctx->ring_n; ++i) {
        FrameEvents& f = ctx->ring[i];
        CU(cudaEventSynchronize(f.e[3]));
        float a = 0, b = 0, c = 0, d = 0;
        CU(cudaEventElapsedTime(&a, f.e[4], f.e[5]));
        CU(cudaEventElapsedTime(&b, f.e[0], f.e[1]));
        CU(cudaEventElapsedTime(&c, f.e[2], f.e[3]));
        CU(cudaEventElapsedTime(&d, f.e[0], f.e[3]));
        ctx->ms_sum[0] += a;
        ctx->ms_sum[1] += b;
        ctx->ms_sum[2] += c;
        ctx->ms_sum[3] += d;
        ctx->timed_frames += 1;
    }
    ctx->ring_n = 0;
    return SCWP_OK;
}

static scwp_status step_impl(scwp_ctx* ctx, double dt);

// Host side of one patch's frame: the injection plan (FP64 carries of
// Eqs. 15-17 per bucket and edge pair, Sec. 3.3) and the wake segments of
// the moving object (Sec. 4.3); updates the carries, injected counts and
// energies.
static void frame_injection(scwp_ctx* ctx, PatchHost* P, InjectParams& ip_out) {
    const PatchTablesHost& T = P->T;
    const PatchDev& D = P->dev;
    InjectParams& ip = ip_out;
    ip = InjectParams{};
    ip.frame = (uint32_t)ctx->frame;
    ip.patch = (uint32_t)P->index;
    ip.seed = ctx->d.seed;
    ip.W = T.W;
    ip.H = T.H;
    ip.nth = T.nth;
    int total = 0, nseg = 0;
    for (int i = 0; i < T.nb; ++i)
        for (int sp = 0; sp < 2; ++sp) {
            double& acc = P->carry[(size_t)i * 2 + sp];
            acc += T.injection_rate(i, sp);
            const double m = std::floor(acc);
            acc -= m;
            const int nv = P->nvalid[i * 2 + sp];
            if (m <= 0 || nv == 0) continue;
            const int mi = (int)m;
            Segment& g = ip.seg[nseg++];
            g.bucket = i;
            g.s = sp;
            g.count = mi * nv;
            g.first = total;
            g.ndir = nv;
            total += g.count;
            double e = 0.0;
            for (int k = 0; k < nv; ++k) {
                const int j = P->dirlist[((size_t)i * 2 + sp) * T.nth + k];
                const double A = T.amp[(size_t)i * T.nth + j];
                e += 0.125 * A * A * M_PI * T.r[i] * T.r[i];
            }
            P->energy[i] += mi * e;
        }
    int given = 0;
    if (D.emitter && P->d.wake_rate > 0) {
        // reading of Sec. 4.3: object on a circle about the patch centre
        const double dx = P->d.cell;
        const double Rp = P->d.obj_path_radius / dx;
        const double Om = P->d.obj_speed / P->d.obj_path_radius;
        const double phi = Om * ctx->t;
        const double Px = T.W * 0.5 + Rp * std::cos(phi);
        const double Py = T.H * 0.5 + Rp * std::sin(phi);
        const double psi = phi + M_PI / 2.0;
        const double rho = P->d.obj_radius / dx;
        const double kelvin = M_PI / 2.0 - std::asin(1.0 / 3.0);
        const double dpsi = 2.0 * M_PI / kWakeDirs;
        for (int arm = 0; arm < 2; ++arm) {
            const double sgn = arm == 0 ? 1.0 : -1.0;
            const double psa = psi + sgn * kelvin;
            int64_t a = (int64_t)std::floor(psa / dpsi + 0.5);
            a = ((a % kWakeDirs) + kWakeDirs) % kWakeDirs;
            const double ca = T.wake_cos[a], sa = T.wake_sin[a];
            Segment& g = ip.seg[nseg++];
            g.bucket = T.wake_bucket;
            g.s = 2;
            g.count = P->d.wake_rate;
            g.first = total;
            g.ndir = P->d.wake_rate;
            g.arm = arm;
            g.wake_a = (int)a;
            g.given = given;
            total += g.count;
            // spawn points on the object's rim, tangential offset tau uniform in
            // [-rho, rho) from Philox word u0 at counter (frame, patch,
            // bucket | 2 << 16, arm * rate + n):
            // rint((P + rho (ca, sa) + tau (-sa, ca)) Q), float64 in this order
            for (int n = 0; n < P->d.wake_rate; ++n) {
                const uint32_t ord = (uint32_t)(arm * P->d.wake_rate + n);
                const U4 u = philox4x32_10(ip.frame, ip.patch, (uint32_t)T.wake_bucket | (2u << 16), ord, ip.seed);
                const double tau = (((double)u.x * 0x1p-32) - 0.5) * 2.0 * rho;
                ip.gx[given] = (int32_t)std::nearbyint(((Px + rho * ca) - tau * sa) * (double)kQ);
                ip.gy[given] = (int32_t)std::nearbyint(((Py + rho * sa) + tau * ca) * (double)kQ);
                ip.ga[given] = (int32_t)a;
                ++given;
            }
            const double rw = T.r[T.wake_bucket];
            P->energy[T.wake_bucket] +=
                P->d.wake_rate * 0.125 * P->d.wake_amp * P->d.wake_amp * M_PI * rw * rw;
        }
    }
    if (D.emitter && P->d.ring_rate > 0 && P->d.heave_period > 0) {
        // reading of Sec. 4.3, vertical motion: the object heaves with
        // period T_h; each frame it emits ring_rate |cos(2 pi t / T_h)|
        // particles (its heave speed relative to the peak; an FP64 carry),
        // outward on its rim at successive directions of the wake grid
        // (stepping by 2531, odd, so every direction comes round), with the
        // wake's amplitude and bucket
        const double dx = P->d.cell;
        const double Rp = P->d.obj_path_radius / dx;
        const double Om = P->d.obj_speed / P->d.obj_path_radius;
        const double phi = Om * ctx->t;
        const double Px = T.W * 0.5 + Rp * std::cos(phi);
        const double Py = T.H * 0.5 + Rp * std::sin(phi);
        const double rho = P->d.obj_radius / dx;
        const double c = std::fabs(std::cos(2.0 * M_PI * ctx->t / P->d.heave_period));
        P->ring_carry += P->d.ring_rate * c;
        const double m = std::floor(P->ring_carry);
        P->ring_carry -= m;
        const int n = (int)std::min(m, (double)kMaxRing);
        P->ring_carry += m - n;
        if (n > 0) {
            Segment& g = ip.seg[nseg++];
            g.bucket = T.wake_bucket;
            g.s = 3;
            g.count = n;
            g.first = total;
            g.ndir = n;
            g.given = given;
            total += n;
            for (int k = 0; k < n; ++k) {
                const int a = (int)((P->ring_total * 2531) % kWakeDirs);
                P->ring_total += 1;
                ip.gx[given] = (int32_t)std::nearbyint((Px + rho * T.wake_cos[a]) * (double)kQ);
                ip.gy[given] = (int32_t)std::nearbyint((Py + rho * T.wake_sin[a]) * (double)kQ);
                ip.ga[given] = a;
                ++given;
            }
            const double rw = T.r[T.wake_bucket];
            P->energy[T.wake_bucket] += n * 0.125 * P->d.wake_amp * P->d.wake_amp * M_PI * rw * rw;
        }
    }
    ip.nseg = nseg;
    ip.total = total;
    P->injected += total;
}


scwp_status scwp_step(scwp_ctx* ctx, double dt) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    const long long before = launches_total();
    s = step_impl(ctx, dt);
    ctx->launches += launches_total() - before;
    return s;
}

// Enqueue one frame's kernels.  ips: the host plans (eager launches pass
// them by value); ip_dev / t_dev: their device copies (captured frames read
// the frame's parameters from device memory).
static scwp_status enqueue_frame(scwp_ctx* ctx, const std::vector<InjectParams>& ips, const InjectParams* ip_dev,
                          const float2* t_dev, FrameEvents* fe) {
    scwp_status s = SCWP_OK;
    // background on the side stream, concurrent with the particle stages;
    // with stage timing on, alone on the context stream ahead of them, so
    // that each stage's events time that stage by itself
    if (fe) {
        if ((s = record(ctx, fe->e[4], ctx->st)) != SCWP_OK) return s;
        CU(launch_background(ctx->bg, ctx->t, ctx->st, t_dev));
        if ((s = record(ctx, fe->e[5], ctx->st)) != SCWP_OK) return s;
        CU(cudaEventRecord(ctx->ev_fork, ctx->st));   // the particle streams start after it
        CU(cudaEventRecord(ctx->ev_join, ctx->st));
    } else {
        CU(cudaEventRecord(ctx->ev_fork, ctx->st));
        CU(cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
        CU(launch_background(ctx->bg, ctx->t, ctx->side, t_dev));
        CU(cudaEventRecord(ctx->ev_join, ctx->side));
    }
    ctx->bg_valid = true;

    // one patch: the context stream; several: up to kParticleStreams
    // streams, so that the small kernels of different patches overlap
    const bool multi = ctx->patches.size() > 1;
    if (multi) {
        if ((s = particle_streams(ctx)) != SCWP_OK) return s;
        for (cudaStream_t ps : ctx->pst) CU(cudaStreamWaitEvent(ps, ctx->ev_fork, 0));
    }
    for (size_t k = 0; k < ctx->patches.size(); ++k) {
        PatchHost* P = ctx->patches[k];
        PatchDev& D = P->dev;
        cudaStream_t pst = multi ? ctx->pst[P->index % ctx->pst.size()] : ctx->st;
        CU(launch_advect_flag(D, pst));
        CU(launch_compact(D, pst));
        D.cur ^= 1;
        if (ip_dev)
            CU(launch_inject_dev(D, ip_dev + k, pst));
        else if (ips[k].total > 0)
            CU(launch_inject(D, ips[k], pst));
        CU(launch_bin(D, pst));   // (the frame's statistics were zeroed by the advection)
    }
    if (multi)
        for (size_t k = 0; k < ctx->pst.size(); ++k) {
            CU(cudaEventRecord(ctx->pev[k], ctx->pst[k]));
            CU(cudaStreamWaitEvent(ctx->st, ctx->pev[k], 0));
        }
    if (fe && (s = record(ctx, fe->e[1], ctx->st)) != SCWP_OK) return s;
    CU(cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0));
    if (fe && (s = record(ctx, fe->e[2], ctx->st)) != SCWP_OK) return s;
    if ((s = synthesize(ctx, ctx->synth_mode)) != SCWP_OK) return s;
    if (fe && (s = record(ctx, fe->e[3], ctx->st)) != SCWP_OK) return s;
    CU(cudaGetLastError());
    return SCWP_OK;
}

// Background and particle stages of every patch of a scene, all on the
// context stream (the server's ticks).  ips / ip_dev / t_dev as in
// enqueue_frame.
static scwp_status enqueue_prepare(scwp_ctx* ctx, const std::vector<InjectParams>& ips, const InjectParams* ip_dev,
                                   const float2* t_dev) {
    scwp_status s = SCWP_OK;
    CU(launch_background(ctx->bg, ctx->t, ctx->st, t_dev));
    ctx->bg_valid = true;
    for (size_t k = 0; k < ctx->patches.size(); ++k) {
        PatchHost* P = ctx->patches[k];
        PatchDev& D = P->dev;
        CU(launch_advect_flag(D, ctx->st));
        CU(launch_compact(D, ctx->st));
        D.cur ^= 1;
        if (ip_dev)
            CU(launch_inject_dev(D, ip_dev + k, ctx->st));
        else if (ips[k].total > 0)
            CU(launch_inject(D, ips[k], ctx->st));
        CU(launch_bin(D, ctx->st));   // (the frame's statistics were zeroed by the advection)
    }
    CU(cudaGetLastError());
    return SCWP_OK;
}

// Replay (capturing first if needed) graph set G with this frame's
// parameters on `launch`.  A graph is captured once for each parity of the
// particle double buffers (every patch flips its live buffer each frame);
// the frame's varying inputs (time, injection plans) reach it through one
// copy from a pinned staging buffer per graph, rewritten only after that
// graph's previous replay completed.  full: the whole frame (enqueue_frame);
// otherwise the background and particle stages (enqueue_prepare).
static scwp_status run_graph(scwp_ctx* ctx, FrameGraph& G, const std::vector<InjectParams>& ips,
                             cudaStream_t launch, bool full) {
    scwp_status s = SCWP_OK;
    uint64_t mask = 0;
    for (size_t k = 0; k < ctx->patches.size(); ++k) mask |= (uint64_t)(ctx->patches[k]->dev.cur & 1) << k;
    int g = -1;
    for (int k = 0; k < 2; ++k)
        if (G.valid[k] && G.mask[k] == mask) g = k;
    if (g < 0) g = !G.valid[0] ? 0 : 1;
    const size_t bytes = 16 + ips.size() * sizeof(InjectParams);
    if (!G.dparams || G.bytes < bytes) {
        graph_reset(G);
        G.dparams = (unsigned char*)dalloc(ctx, bytes);
        if (!G.dparams) return fail(ctx, SCWP_E_NOMEM, "graph parameters");
        for (int k = 0; k < 2; ++k) {
            if (G.hstage[k]) cudaFreeHost(G.hstage[k]);
            if (cudaMallocHost(&G.hstage[k], bytes) != cudaSuccess) {
                G.hstage[k] = nullptr;
                cudaGetLastError();
                return fail(ctx, SCWP_E_NOMEM, "graph staging");
            }
        }
        G.bytes = bytes;
        g = 0;
    }
    if (G.pending[g]) CU(cudaEventSynchronize(G.done[g]));
    unsigned char* h = (unsigned char*)G.hstage[g];
    {
        // the frame's time as a float pair (t_hi, t_lo), split here in float64
        const float th = (float)ctx->t;
        const float2 tt = make_float2(th, (float)(ctx->t - (double)th));
        memcpy(h, &tt, sizeof(tt));
    }
    memcpy(h + 16, ips.data(), ips.size() * sizeof(InjectParams));
    if (!G.valid[g]) {
        // everything that synchronises or allocates happens before the capture
        if (full) {
            if ((s = sync_synth(ctx)) != SCWP_OK) return s;
            if (ctx->patches.size() > 1 && (s = particle_streams(ctx)) != SCWP_OK) return s;
        }
        if (!ctx->gst && cudaStreamCreateWithFlags(&ctx->gst, cudaStreamNonBlocking) != cudaSuccess) {
            ctx->gst = nullptr;
            return fail(ctx, SCWP_E_CUDA, "capture stream");
        }
        const long long before = launches_total();
        // the frame is recorded as if enqueued on the context stream
        cudaStream_t caller = ctx->st;
        ctx->st = ctx->gst;
        cudaError_t e = cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeRelaxed);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaSuccess;
        if (e == cudaSuccess) {
            e = cudaMemcpyAsync(G.dparams, h, bytes, cudaMemcpyHostToDevice, ctx->st);
            const InjectParams* ipd = reinterpret_cast<const InjectParams*>(G.dparams + 16);
            const float2* td = reinterpret_cast<const float2*>(G.dparams);
            if (e == cudaSuccess)
                s = full ? enqueue_frame(ctx, ips, ipd, td, nullptr) : enqueue_prepare(ctx, ips, ipd, td);
            e2 = cudaStreamEndCapture(ctx->st, &graph);
        }
        ctx->st = caller;
        if (e != cudaSuccess || s != SCWP_OK || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != SCWP_OK ? s : fail(ctx, SCWP_E_CUDA, "frame capture");
        }
        e = cudaGraphInstantiate(&G.exec[g], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            G.exec[g] = nullptr;
            return fail(ctx, SCWP_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        G.valid[g] = true;
        G.mask[g] = mask;
        G.launches[g] = launches_total() - before;
    } else {
        for (PatchHost* P : ctx->patches) P->dev.cur ^= 1;   // what the replay does on the device
        count_launches((int)G.launches[g]);
    }
    CU(cudaGraphLaunch(G.exec[g], launch));
    CU(cudaEventRecord(G.done[g], launch));
    G.pending[g] = true;
    return SCWP_OK;
}

// Host part of a frame: dt tables (on the context stream), frame counter
// and time, the injection plans.
static scwp_status frame_begin(scwp_ctx* ctx, double dt) {
    scwp_status s = SCWP_OK;
    if (!(dt > 0)) return fail(ctx, SCWP_E_INVALID, "dt must be > 0");
    if (dt != ctx->dt) {
        ctx->dt = dt;
        for (PatchHost* P : ctx->patches) {
            if (dt == P->T.dt) continue;
            P->T.set_dt(dt);
            if ((s = upload_dt_tables(ctx, *P)) != SCWP_OK) return s;
        }
    }
    ctx->frame += 1;
    ctx->t += dt;
    ctx->ips.resize(ctx->patches.size());
    for (size_t k = 0; k < ctx->patches.size(); ++k) frame_injection(ctx, ctx->patches[k], ctx->ips[k]);
    return SCWP_OK;
}

// A scene's frame up to the synthesis on `stream` (the server's ticks), as a
// replayed graph.
static scwp_status scene_prepare(scwp_ctx* ctx, double dt, cudaStream_t stream) {
    cudaStream_t caller = ctx->st;
    ctx->st = stream;
    scwp_status s = frame_begin(ctx, dt);
    ctx->st = caller;
    if (s != SCWP_OK) return s;
    return run_graph(ctx, ctx->gprep, ctx->ips, stream, false);
}

static scwp_status step_impl(scwp_ctx* ctx, double dt) {
    scwp_status s = frame_begin(ctx, dt);
    if (s != SCWP_OK) return s;
    // batched frames of several patches replay a captured graph unless
    // stage timing is on.  A one-patch frame (about 13 kernels) runs eagerly
    // instead: chained by programmatic dependent launch it measured faster
    // than the replay (0.308 against 0.317-0.322 ms on a 1024^2 patch with
    // 200k particles), whose staged-parameter copy heads the frame.
    if (ctx->batched && !ctx->timing && ctx->patches.size() > 1 && ctx->patches.size() <= 64 &&
        (ctx->synth_mode == SCWP_SYNTH_GATHER || ctx->synth_mode == SCWP_SYNTH_GATHER_FP16 ||
         ctx->synth_mode == SCWP_SYNTH_SAT))
        return run_graph(ctx, ctx->gfull, ctx->ips, ctx->st, true);
    FrameEvents* fe = nullptr;
    if (ctx->timing) {
        if (ctx->ring_n == kTimingRing && (s = drain_ring(ctx)) != SCWP_OK) return s;
        fe = &ctx->ring[ctx->ring_n++];
        if ((s = record(ctx, fe->e[0], ctx->st)) != SCWP_OK) return s;
    }
    return enqueue_frame(ctx, ctx->ips, nullptr, nullptr, fe);
}

scwp_status scwp_launch_count(scwp_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return SCWP_E_INVALID;
    *n = ctx->launches;
    return SCWP_OK;
}

scwp_status scwp_resynthesize(scwp_ctx* ctx, int32_t mode) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    const long long before = launches_total();
    if (mode != SCWP_SYNTH_GATHER && mode != SCWP_SYNTH_LAYERED && mode != SCWP_SYNTH_GATHER_FP32 &&
        mode != SCWP_SYNTH_GATHER_FP16 && mode != SCWP_SYNTH_SAT)
        return fail(ctx, SCWP_E_INVALID, "mode");
    if (!ctx->bg_valid) {
        CU(launch_background(ctx->bg, ctx->t, ctx->st));
        ctx->bg_valid = true;
    }
    for (PatchHost* P : ctx->patches) {
        if ((s = reset_frame_stats(ctx, *P, ctx->st)) != SCWP_OK) return s;
        CU(launch_bin(P->dev, ctx->st));
    }
    if ((s = synthesize(ctx, mode)) != SCWP_OK) return s;
    ctx->launches += launches_total() - before;
    CU(cudaStreamSynchronize(ctx->st));
    return SCWP_OK;
}

scwp_status scwp_set_batched(scwp_ctx* ctx, int32_t on) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    graph_reset(ctx);
    ctx->batched = on != 0;
    ctx->synth_dirty = true;
    return SCWP_OK;
}

scwp_status scwp_set_bucket_range(scwp_ctx* ctx, int32_t b_lo, int32_t b_hi) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (b_lo < 0 || b_hi <= b_lo) return fail(ctx, SCWP_E_INVALID, "bucket range");
    graph_reset(ctx);
    ctx->b_lo = b_lo;
    ctx->b_hi = b_hi;
    ctx->synth_dirty = true;
    return SCWP_OK;
}

scwp_status scwp_set_synth_mode(scwp_ctx* ctx, int32_t mode) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (mode != SCWP_SYNTH_GATHER && mode != SCWP_SYNTH_LAYERED && mode != SCWP_SYNTH_GATHER_FP32 &&
        mode != SCWP_SYNTH_GATHER_FP16 && mode != SCWP_SYNTH_SAT)
        return fail(ctx, SCWP_E_INVALID, "mode");
    graph_reset(ctx);
    ctx->synth_mode = mode;
    return SCWP_OK;
}

// Re-plan every patch's summed-area synthesis for the context's variant and
// bucket-group multiplier (the autotuner's choices) and upload the plans;
// the batched plan and the captured frames follow at the next synthesis.
static scwp_status replan_sat(scwp_ctx* ctx) {
    for (PatchHost* P : ctx->patches) {
        const int variant = (ctx->sat_variant == 1 && P->sat3_ok) ? 1 : 0;
        P->sat_slots = sat_slots_of(variant);
        plan_patch(*P, P->sat_slots, true, ctx->sat_gmul, P->partial_planes);
        if ((int)P->sat_items.size() > P->sat_item_cap) return fail(ctx, SCWP_E_STATE, "summed-area plan capacity");
        CU(cudaMemcpyAsync(P->d_sat_items, P->sat_items.data(), P->sat_items.size() * sizeof(TcItem),
                           cudaMemcpyHostToDevice, ctx->st));
        if (!P->sat_spans.empty())
            CU(cudaMemcpyAsync(P->d_sat_spans, P->sat_spans.data(), P->sat_spans.size() * sizeof(BlendSpan),
                               cudaMemcpyHostToDevice, ctx->st));
        ctx->sat_slots = P->sat_slots;
    }
    CU(cudaStreamSynchronize(ctx->st));
    graph_reset(ctx);
    ctx->synth_dirty = true;
    return SCWP_OK;
}

namespace {
// Choices of the autotuner per device and workload signature (process-wide).
std::mutex g_tune_mutex;
std::map<std::string, std::pair<int, double>> g_tune_cache;

// the workload signature the autotuner's choice is cached under: device,
// batching, and every patch's size, buckets, prefill, capacity and bin size
std::string tune_signature(const scwp_ctx* ctx) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::string s = "dev" + std::to_string(dev) + (ctx->batched ? "/b" : "/p");
    for (const PatchHost* P : ctx->patches) {
        s += "/" + std::to_string(P->T.W) + "x" + std::to_string(P->T.H) + ":" + std::to_string(P->T.nb) + ":" +
             std::to_string(P->d.prefill) + ":" + std::to_string(P->dev.cap) + ":" +
             std::to_string(P->bin_cells.empty() ? 0 : P->bin_cells[0]);
    }
    return s;
}
}  // namespace

scwp_status scwp_set_sat_plan(scwp_ctx* ctx, int32_t variant, double gmul) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if ((variant != 0 && variant != 1) || !(gmul >= 0.125 && gmul <= 8.0)) return fail(ctx, SCWP_E_INVALID, "plan");
    if (variant == 1)
        for (const PatchHost* P : ctx->patches)
            if (!P->sat3_ok) return fail(ctx, SCWP_E_INVALID, "a patch's buckets exceed the three-group row table");
    ctx->sat_variant = variant;
    ctx->sat_gmul = gmul;
    return replan_sat(ctx);
}

scwp_status scwp_autotune(scwp_ctx* ctx, int32_t reps, int32_t force, scwp_tune_result* out) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (!out || reps < 1 || reps > 100) return fail(ctx, SCWP_E_INVALID, "autotune arguments");
    if (ctx->synth_mode != SCWP_SYNTH_SAT) return fail(ctx, SCWP_E_STATE, "the autotuner tunes the summed-area synthesis");
    if (ctx->frame < 1 || ctx->patches.empty()) return fail(ctx, SCWP_E_STATE, "autotune needs a stepped frame");
    memset(out, 0, sizeof(*out));
    const long long before = launches_total();
    const std::string key = tune_signature(ctx);
    bool all3 = true;
    for (const PatchHost* P : ctx->patches) all3 = all3 && P->sat3_ok;
    if (!force) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            ctx->sat_variant = it->second.first;
            ctx->sat_gmul = it->second.second;
            out->n_configs = 1;
            out->chosen = 0;
            out->variant[0] = ctx->sat_variant;
            out->gmul[0] = ctx->sat_gmul;
            out->ms[0] = -1.0;
            out->from_cache = 1;
            return replan_sat(ctx);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return fail(ctx, SCWP_E_CUDA, "autotune events");
    }
    const double gmuls[3] = {1.0, 0.5, 2.0};
    int n = 0;
    for (int v = 0; v < 2 && s == SCWP_OK; ++v) {
        if (v == 1 && !all3) continue;
        for (double gm : gmuls) {
            if (n >= SCWP_TUNE_MAX) break;
            ctx->sat_variant = v;
            ctx->sat_gmul = gm;
            if ((s = replan_sat(ctx)) != SCWP_OK || (s = sync_synth(ctx)) != SCWP_OK) break;
            if ((s = synthesize(ctx, SCWP_SYNTH_SAT)) != SCWP_OK) break;   // warm-up
            std::vector<float> ms;
            for (int r = 0; r < reps && s == SCWP_OK; ++r) {
                float t = 0.f;
                if (cudaEventRecord(e0, ctx->st) != cudaSuccess) { s = fail(ctx, SCWP_E_CUDA, "autotune"); break; }
                if ((s = synthesize(ctx, SCWP_SYNTH_SAT)) != SCWP_OK) break;
                if (cudaEventRecord(e1, ctx->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                    s = fail(ctx, SCWP_E_CUDA, "autotune timing");
                    break;
                }
                ms.push_back(t);
            }
            if (s != SCWP_OK) break;
            std::sort(ms.begin(), ms.end());
            out->variant[n] = v;
            out->gmul[n] = gm;
            out->ms[n] = ms[ms.size() / 2];
            if (out->ms[n] < out->ms[out->chosen]) out->chosen = n;
            ++n;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->n_configs = n;
    if (s != SCWP_OK) return s;
    ctx->sat_variant = out->variant[out->chosen];
    ctx->sat_gmul = out->gmul[out->chosen];
    if ((s = replan_sat(ctx)) != SCWP_OK || (s = sync_synth(ctx)) != SCWP_OK) return s;
    // the maps of the last frame, synthesised with the chosen plan
    if ((s = synthesize(ctx, SCWP_SYNTH_SAT)) != SCWP_OK) return s;
    CU(cudaStreamSynchronize(ctx->st));
    ctx->launches += launches_total() - before;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = std::make_pair(ctx->sat_variant, ctx->sat_gmul);
    }
    return SCWP_OK;
}

scwp_status scwp_height_map(scwp_ctx* ctx, int32_t patch_id, int32_t field, float* dst, size_t dst_elems,
                            int32_t dst_on_device) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (!dst || field < 0 || field > 2) return fail(ctx, SCWP_E_INVALID, "field or dst");
    const float* src;
    size_t n;
    if (patch_id == -1) {
        n = (size_t)ctx->d.fft_n * ctx->d.fft_n;
        src = ctx->bgout + field * n;
    } else {
        if (patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "patch_id");
        const PatchHost* P = ctx->patches[patch_id];
        n = (size_t)P->T.W * P->T.H;
        src = P->dev.out + field * n;
    }
    if (dst_elems < n) return fail(ctx, SCWP_E_INVALID, "dst too small");
    if (dst_on_device) {
        CU(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    } else {
        CU(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
    }
    return SCWP_OK;
}

scwp_status scwp_height_maps(scwp_ctx* ctx, int32_t patch_id, float* dst, size_t dst_elems, int32_t dst_on_device) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (!dst) return fail(ctx, SCWP_E_INVALID, "dst");
    const float* src;
    size_t n;
    if (patch_id == -1) {
        n = (size_t)ctx->d.fft_n * ctx->d.fft_n;
        src = ctx->bgout;
    } else {
        if (patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "patch_id");
        const PatchHost* P = ctx->patches[patch_id];
        n = (size_t)P->T.W * P->T.H;
        src = P->dev.out;
    }
    if (dst_elems < 3 * n) return fail(ctx, SCWP_E_INVALID, "dst too small");
    if (dst_on_device) {
        CU(cudaMemcpyAsync(dst, src, 3 * n * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
    } else {
        CU(cudaMemcpyAsync(dst, src, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
    }
    return SCWP_OK;
}

scwp_status scwp_normal_map(scwp_ctx* ctx, int32_t patch_id, float* dst, size_t dst_elems, int32_t dst_on_device) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (!dst || patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "args");
    const PatchHost* P = ctx->patches[patch_id];
    const size_t n = (size_t)P->T.W * P->T.H;
    if (dst_elems < 3 * n) return fail(ctx, SCWP_E_INVALID, "dst too small");
    float* out = dst;
    if (!dst_on_device) {
        if (ctx->normal_bytes < 3 * n * sizeof(float)) {
            ctx->normal_scratch = (float*)dalloc(ctx, 3 * n * sizeof(float));
            if (!ctx->normal_scratch) return fail(ctx, SCWP_E_NOMEM, "normal scratch");
            ctx->normal_bytes = 3 * n * sizeof(float);
        }
        out = ctx->normal_scratch;
    }
    CU(launch_normals(P->dev.out, P->T.W, P->T.H, (float)P->d.cell, out, ctx->st));
    if (!dst_on_device) {
        CU(cudaMemcpyAsync(dst, out, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
    }
    return SCWP_OK;
}

scwp_status scwp_stats_get(scwp_ctx* ctx, int32_t patch_id, scwp_stats* out) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (!out || patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "args");
    PatchHost* P = ctx->patches[patch_id];
    std::vector<unsigned long long> st(6 + P->T.nb);
    int32_t cnt[2];
    CU(cudaMemcpyAsync(st.data(), P->dev.stats, st.size() * 8, cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaMemcpyAsync(cnt, P->dev.count, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    memset(out, 0, sizeof(*out));
    out->frame = ctx->frame;
    out->time = ctx->t;
    out->live_particles = cnt[0];
    out->eval_count = (int64_t)st[0];
    out->bumps_binned = (int64_t)st[1];
    out->error_flags = (int32_t)st[2];
    out->injected_total = P->injected;
    out->mma_stages = (int64_t)st[3 + P->T.nb];
    out->eval_total = (int64_t)st[4 + P->T.nb];
    out->sat_candidates = (int64_t)st[5 + P->T.nb];
    out->n_buckets = P->T.nb;
    for (int i = 0; i < P->T.nb; ++i) {
        out->live_per_bucket[i] = (int64_t)st[3 + i];
        out->injected_energy[i] = P->energy[i];
    }
    if (st[2] & kErrTimeout) return fail(ctx, SCWP_E_TIMEOUT, "a device wait timed out");
    if (st[2] & kErrCapacity) return fail(ctx, SCWP_E_CAPACITY, "particle pool full: injection was truncated");
    return SCWP_OK;
}

scwp_status scwp_patch_info_get(scwp_ctx* ctx, int32_t patch_id, scwp_patch_info* out) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (!out || patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "args");
    const PatchHost* P = ctx->patches[patch_id];
    memset(out, 0, sizeof(*out));
    out->n_buckets = P->T.nb;
    out->n_theta = P->T.nth;
    out->n_dirs = P->T.nth + (P->dev.emitter ? kWakeDirs : 0);
    out->wake_bucket = P->T.wake_bucket;
    out->width = P->T.W;
    out->height = P->T.H;
    out->total_bins = P->dev.total_bins;
    out->capacity = P->dev.cap;
    out->synth_groups = P->dev.groups_tc;
    out->synth_items = (int32_t)P->tc_items.size();
    out->synth_slots = P->tc_slots;
    out->sat_groups = P->sat_groups;
    out->sat_items = (int32_t)P->sat_items.size();
    out->sat_slots = P->sat_slots;
    out->sat_variant = (ctx->sat_variant == 1 && P->sat3_ok) ? 1 : 0;
    out->sat_parts = P->sat_parts;
    out->frame_param_bytes = (int32_t)sizeof(InjectParams);
    for (int i = 0; i < P->T.nb; ++i) {
        out->bin_cells[i] = P->bin_cells[i];
        out->nbx[i] = P->bk[i].nbx;
        out->nby[i] = P->bk[i].nby;
        out->bin_base[i] = P->bk[i].base;
    }
    return SCWP_OK;
}

}  // extern "C"

namespace {

scwp_status copy_table(const PatchTablesHost& T, const std::vector<double>* carry, int32_t table, void* dst,
                       size_t bytes, int64_t* count) {
    const void* src = nullptr;
    size_t n = 0, es = 0;
    switch (table) {
        case SCWP_TAB_OMEGA: src = T.omega.data(); n = T.omega.size(); es = 8; break;
        case SCWP_TAB_K: src = T.k.data(); n = T.k.size(); es = 8; break;
        case SCWP_TAB_C: src = T.c.data(); n = T.c.size(); es = 8; break;
        case SCWP_TAB_R: src = T.r.data(); n = T.r.size(); es = 8; break;
        case SCWP_TAB_E: src = T.E.data(); n = T.E.size(); es = 8; break;
        case SCWP_TAB_EDGES: src = T.edges.data(); n = T.edges.size(); es = 8; break;
        case SCWP_TAB_AMP: src = T.amp.data(); n = T.amp.size(); es = 8; break;
        case SCWP_TAB_RQ: src = T.R.data(); n = T.R.size(); es = 4; break;
        case SCWP_TAB_VX: src = T.vx.data(); n = T.vx.size(); es = 4; break;
        case SCWP_TAB_VY: src = T.vy.data(); n = T.vy.size(); es = 4; break;
        case SCWP_TAB_QX: src = T.qx.data(); n = T.qx.size(); es = 4; break;
        case SCWP_TAB_QY: src = T.qy.data(); n = T.qy.size(); es = 4; break;
        case SCWP_TAB_WAKE_VX: src = T.wvx.data(); n = T.wvx.size(); es = 4; break;
        case SCWP_TAB_WAKE_VY: src = T.wvy.data(); n = T.wvy.size(); es = 4; break;
        case SCWP_TAB_WAKE_QX: src = T.wqx.data(); n = T.wqx.size(); es = 4; break;
        case SCWP_TAB_WAKE_QY: src = T.wqy.data(); n = T.wqy.size(); es = 4; break;
        case SCWP_TAB_CARRY:
            if (!carry) return SCWP_E_INVALID;
            src = carry->data(); n = carry->size(); es = 8; break;
        default: return SCWP_E_INVALID;
    }
    if (count) *count = (int64_t)n;
    if (!dst) return SCWP_OK;
    if (bytes < n * es) return SCWP_E_INVALID;
    if (n) memcpy(dst, src, n * es);
    return SCWP_OK;
}

}  // namespace

extern "C" {

scwp_status scwp_get_table(scwp_ctx* ctx, int32_t patch_id, int32_t table, void* dst, size_t bytes) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "patch_id");
    const PatchHost* P = ctx->patches[patch_id];
    s = copy_table(P->T, &P->carry, table, dst, bytes, nullptr);
    if (s != SCWP_OK) return fail(ctx, s, "table id or size");
    return SCWP_OK;
}

scwp_status scwp_host_table(const scwp_spectrum_desc* sdesc, const scwp_patch_desc* pdesc, double dt,
                            int32_t table, void* dst, size_t bytes, int64_t* count) {
    std::string why;
    if (check_spectrum_desc(sdesc, why) != SCWP_OK || check_patch_desc(pdesc, why) != SCWP_OK)
        return SCWP_E_INVALID;
    if (!(dt > 0) || table == SCWP_TAB_CARRY) return SCWP_E_INVALID;
    SpectrumModel sm;
    model_from_desc(*sdesc, sm);
    std::vector<double> edges;
    if (sdesc->bucket_edges) edges.assign(sdesc->bucket_edges, sdesc->bucket_edges + sdesc->n_buckets + 1);
    PatchTablesHost T;
    build_tables(*sdesc, edges, *pdesc, sm, T);
    T.set_dt(dt);
    return copy_table(T, nullptr, table, dst, bytes, count);
}

scwp_status scwp_get_particles(scwp_ctx* ctx, int32_t patch_id, int32_t* x, int32_t* y, uint32_t* bd,
                               int64_t cap, int64_t* n) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (patch_id < 0 || patch_id >= (int)ctx->patches.size() || !n) return fail(ctx, SCWP_E_INVALID, "args");
    const PatchDev& D = ctx->patches[patch_id]->dev;
    int32_t cnt[2];
    CU(cudaMemcpyAsync(cnt, D.count, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    *n = cnt[0];
    const size_t m = (size_t)std::min<int64_t>(cap, cnt[0]);
    if (m && x) CU(cudaMemcpyAsync(x, D.x[D.cur], m * 4, cudaMemcpyDeviceToHost, ctx->st));
    if (m && y) CU(cudaMemcpyAsync(y, D.y[D.cur], m * 4, cudaMemcpyDeviceToHost, ctx->st));
    if (m && bd) CU(cudaMemcpyAsync(bd, D.bd[D.cur], m * 4, cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return SCWP_OK;
}

scwp_status scwp_set_particles(scwp_ctx* ctx, int32_t patch_id, const int32_t* x, const int32_t* y,
                               const uint32_t* bd, int64_t n) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (patch_id < 0 || patch_id >= (int)ctx->patches.size() || n < 0) return fail(ctx, SCWP_E_INVALID, "args");
    PatchHost* P = ctx->patches[patch_id];
    PatchDev& D = P->dev;
    if (n > D.cap) return fail(ctx, SCWP_E_INVALID, "n exceeds capacity");
    if (n > 0 && (!x || !y || !bd)) return fail(ctx, SCWP_E_INVALID, "null arrays");
    const int ndirs = P->T.nth + (D.emitter ? kWakeDirs : 0);
    for (int64_t i = 0; i < n; ++i)
        if ((int)(bd[i] >> 16) >= P->T.nb || (int)(bd[i] & 0xFFFFu) >= ndirs)
            return fail(ctx, SCWP_E_INVALID, "bucket or direction out of range");
    int32_t cnt[2] = {(int32_t)n, (int32_t)n};
    if (n) {
        CU(cudaMemcpyAsync(D.x[D.cur], x, n * 4, cudaMemcpyHostToDevice, ctx->st));
        CU(cudaMemcpyAsync(D.y[D.cur], y, n * 4, cudaMemcpyHostToDevice, ctx->st));
        CU(cudaMemcpyAsync(D.bd[D.cur], bd, n * 4, cudaMemcpyHostToDevice, ctx->st));
    }
    CU(cudaMemcpyAsync(D.count, cnt, sizeof(cnt), cudaMemcpyHostToDevice, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    return SCWP_OK;
}

scwp_status scwp_get_bins(scwp_ctx* ctx, int32_t patch_id, uint32_t* counts, uint32_t* offsets,
                          uint32_t* entries, int64_t entries_cap, int64_t* n_entries) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (patch_id < 0 || patch_id >= (int)ctx->patches.size()) return fail(ctx, SCWP_E_INVALID, "args");
    const PatchDev& D = ctx->patches[patch_id]->dev;
    std::vector<uint32_t> off((size_t)D.total_bins + 1);
    CU(cudaMemcpyAsync(off.data(), D.offsets, off.size() * 4, cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    const int64_t nv = off[D.total_bins];
    if (n_entries) *n_entries = nv;
    if (offsets) memcpy(offsets, off.data(), off.size() * 4);
    if (counts)
        for (int k = 0; k < D.total_bins; ++k) counts[k] = off[k + 1] - off[k];
    if (entries && nv > 0) {
        const int src = ((D.key_bits + 7) / 8) & 1;
        const size_t m = (size_t)std::min<int64_t>(nv, entries_cap);
        CU(cudaMemcpyAsync(entries, D.vals[src], m * 4, cudaMemcpyDeviceToHost, ctx->st));
        CU(cudaStreamSynchronize(ctx->st));
    }
    return SCWP_OK;
}

scwp_status scwp_debug_sort_timeout(scwp_ctx* ctx, int32_t patch_id, double wait_seconds) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (patch_id < 0 || patch_id >= (int)ctx->patches.size() || !(wait_seconds > 0.0) || wait_seconds > 2.0)
        return fail(ctx, SCWP_E_INVALID, "args");
    PatchHost* P = ctx->patches[patch_id];
    int32_t cnt = 0;
    CU(cudaMemcpyAsync(&cnt, P->dev.count, sizeof(cnt), cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    // at least two sort tiles of bump keys: tile 1 then looks back to tile 0
    if (2 * (int64_t)cnt <= kSortPassTile) return fail(ctx, SCWP_E_INVALID, "too few particles for two sort tiles");
    int dev = 0, khz = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const long long cycles = (long long)(wait_seconds * 1e3 * (double)(khz > 0 ? khz : 2070000));
    graph_reset(ctx);
    CU(launch_sort_stall(P->dev, cycles, ctx->st));
    unsigned long long flags = 0;
    CU(cudaMemcpyAsync(&flags, P->dev.stats + 2, sizeof(flags), cudaMemcpyDeviceToHost, ctx->st));
    CU(cudaStreamSynchronize(ctx->st));
    if (flags & kErrTimeout) return fail(ctx, SCWP_E_TIMEOUT, "a device wait timed out (sort look-back self-test)");
    return fail(ctx, SCWP_E_STATE, "the sort look-back self-test did not time out");
}

scwp_status scwp_set_timing(scwp_ctx* ctx, int32_t enable) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if (enable && ctx->ring.empty()) {
        ctx->ring.resize(kTimingRing);
        for (FrameEvents& f : ctx->ring)
            for (int k = 0; k < 6; ++k) CU(cudaEventCreate(&f.e[k]));
    }
    if (!enable && (s = drain_ring(ctx)) != SCWP_OK) return s;
    ctx->timing = enable != 0;
    return SCWP_OK;
}

scwp_status scwp_timing_read(scwp_ctx* ctx, double ms_sum[4], int64_t* frames) {
    scwp_status s = ready(ctx);
    if (s != SCWP_OK) return s;
    if ((s = drain_ring(ctx)) != SCWP_OK) return s;
    for (int k = 0; k < 4; ++k) {
        if (ms_sum) ms_sum[k] = ctx->ms_sum[k];
        ctx->ms_sum[k] = 0;
    }
    if (frames) *frames = ctx->timed_frames;
    ctx->timed_frames = 0;
    return SCWP_OK;
}

void scwp_destroy(scwp_ctx* ctx) {
    if (!ctx) return;
    if (ctx->st || ctx->side) {
        cudaStreamSynchronize(ctx->st);
        if (ctx->side) cudaStreamSynchronize(ctx->side);
    }
    for (cudaStream_t s : ctx->pst) cudaStreamSynchronize(s);
    graph_reset(ctx);
    for (FrameGraph* G : {&ctx->gfull, &ctx->gprep})
        for (int k = 0; k < 2; ++k) {
            if (G->hstage[k]) cudaFreeHost(G->hstage[k]);
            if (G->done[k]) cudaEventDestroy(G->done[k]);
        }
    if (ctx->gst) cudaStreamDestroy(ctx->gst);
    cudaGetLastError();
    for (FrameEvents& f : ctx->ring)
        for (int k = 0; k < 6; ++k)
            if (f.e[k]) cudaEventDestroy(f.e[k]);
    for (PatchHost* P : ctx->patches) delete P;
    dfree_all(ctx);
    for (cudaStream_t s : ctx->pst) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    for (cudaEvent_t e : ctx->pev) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    cudaGetLastError();
    delete ctx;
}


// =============================================================================
// Frame-step server: continuous batching of frame-step requests over many
// device-resident scenes (one context each).  A tick takes every idle scene
// with a pending request, enqueues each one's background and particle stages
// on one of eight streams, and runs the tensor-core synthesis of all of them
// as one launch over the union of their batched-plan items (heaviest first)
// on the server stream.  A scene has at most one frame in flight; at most
// `max_inflight` ticks are outstanding, so the next tick's particle stages
// overlap the current tick's synthesis.  Scenes are admitted while their
// device memory fits the budget.
// =============================================================================
}  // extern "C"

namespace {

struct ServerScene {
    scwp_ctx* ctx = nullptr;
    std::deque<std::pair<int64_t, double>> pending;   // request id, dt
    bool in_flight = false;
};

struct ServerTick {
    cudaEvent_t done = nullptr;
    int slot = 0;
    std::vector<std::pair<int, int64_t>> reqs;        // scene, request id
    size_t next = 0;                                  // first request not yet reported
};

}  // namespace

struct scwp_server {
    scwp_server_desc d{};
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> pst;
    std::vector<cudaEvent_t> pev;
    std::vector<ServerScene> scenes;
    std::deque<ServerTick> ticks;
    std::vector<cudaEvent_t> tick_events;             // one per staging slot
    std::vector<void*> hstage, dstage;
    std::vector<size_t> stage_cap;
    std::vector<bool> slot_busy;
    unsigned int* queue = nullptr;    // work queue of the summed-area synthesis launches (2 words)
    size_t used = 0;
    int rr = 0;
    int64_t ticks_launched = 0, requests_done = 0;
    std::string err;
};

namespace {

scwp_status sfail(scwp_server* sv, scwp_status s, const std::string& m) {
    if (sv) sv->err = m;
    return s;
}

#define SCU(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) return sfail(sv, SCWP_E_CUDA, std::string(#call) + ": " +  \
                                                             cudaGetErrorString(e_));     \
    } while (0)

void* sv_alloc(scwp_server* sv, size_t bytes) {
    void* p = nullptr;
    if (sv->d.alloc) return sv->d.alloc(bytes, sv->d.alloc_user);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void sv_free(scwp_server* sv, void* p) {
    if (!p) return;
    if (sv->d.free) sv->d.free(p, sv->d.alloc_user);
    else cudaFree(p);
}

size_t align16(size_t n) { return (n + 15) & ~(size_t)15; }

}  // namespace

extern "C" {

scwp_status scwp_server_create(const scwp_server_desc* desc, scwp_server** out) {
    if (!desc || !out || desc->max_inflight < 1 || desc->max_inflight > 16) return SCWP_E_INVALID;
    *out = nullptr;
    scwp_server* sv = new (std::nothrow) scwp_server();
    if (!sv) return SCWP_E_NOMEM;
    sv->d = *desc;
    sv->st = (cudaStream_t)desc->stream;
    const int slots = desc->max_inflight;
    sv->tick_events.assign(slots, nullptr);
    sv->hstage.assign(slots, nullptr);
    sv->dstage.assign(slots, nullptr);
    sv->stage_cap.assign(slots, 0);
    sv->slot_busy.assign(slots, false);
    bool ok = true;
    for (int k = 0; k < slots; ++k)
        ok = ok && cudaEventCreateWithFlags(&sv->tick_events[k], cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < kParticleStreams && ok; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (s) sv->pst.push_back(s);
        if (e) sv->pev.push_back(e);
    }
    if (ok) {
        sv->queue = (unsigned int*)sv_alloc(sv, 2 * sizeof(unsigned int));
        ok = sv->queue && cudaMemset(sv->queue, 0, 2 * sizeof(unsigned int)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        scwp_server_destroy(sv);
        return SCWP_E_CUDA;
    }
    *out = sv;
    return SCWP_OK;
}

scwp_status scwp_server_add_scene(scwp_server* sv, const scwp_spectrum_desc* spec, const scwp_patch_desc* patches,
                                  int32_t n_patches, int32_t* scene_id) {
    if (!sv || !spec || !scene_id || n_patches < 1 || !patches) return SCWP_E_INVALID;
    scwp_spectrum_desc d = *spec;
    d.stream = sv->st;
    d.alloc = sv->d.alloc;
    d.free = sv->d.free;
    d.alloc_user = sv->d.alloc_user;
    scwp_ctx* ctx = nullptr;
    scwp_status s = scwp_create(&d, &ctx);
    if (s != SCWP_OK) return sfail(sv, s, "scene: scwp_create failed");
    for (int32_t k = 0; k < n_patches && s == SCWP_OK; ++k) {
        int32_t pid = 0;
        s = scwp_add_patch(ctx, patches + k, &pid);
    }
    if (s == SCWP_OK) s = scwp_set_batched(ctx, 1);
    if (s == SCWP_OK) s = sync_synth(ctx);
    if (s != SCWP_OK) {
        sv->err = std::string("scene: ") + scwp_last_error(ctx);
        scwp_destroy(ctx);
        return s;
    }
    if (sv->d.hbm_budget_bytes > 0 && sv->used + ctx->alloc_bytes > (size_t)sv->d.hbm_budget_bytes) {
        scwp_destroy(ctx);
        return sfail(sv, SCWP_E_NOMEM, "scene refused: device memory budget");
    }
    sv->used += ctx->alloc_bytes;
    int id = -1;
    for (size_t k = 0; k < sv->scenes.size() && id < 0; ++k)
        if (!sv->scenes[k].ctx) id = (int)k;
    if (id < 0) {
        id = (int)sv->scenes.size();
        sv->scenes.emplace_back();
    }
    sv->scenes[id].ctx = ctx;
    sv->scenes[id].pending.clear();
    sv->scenes[id].in_flight = false;
    *scene_id = id;
    return SCWP_OK;
}

scwp_status scwp_server_remove_scene(scwp_server* sv, int32_t scene_id) {
    if (!sv || scene_id < 0 || scene_id >= (int)sv->scenes.size() || !sv->scenes[scene_id].ctx)
        return SCWP_E_INVALID;
    ServerScene& sc = sv->scenes[scene_id];
    if (sc.in_flight) return sfail(sv, SCWP_E_INVALID, "scene has a frame in flight");
    sv->used -= sc.ctx->alloc_bytes;
    scwp_destroy(sc.ctx);
    sc.ctx = nullptr;
    sc.pending.clear();
    return SCWP_OK;
}

scwp_status scwp_server_submit(scwp_server* sv, int32_t scene_id, double dt, int64_t request_id) {
    if (!sv || scene_id < 0 || scene_id >= (int)sv->scenes.size() || !sv->scenes[scene_id].ctx || !(dt > 0))
        return SCWP_E_INVALID;
    sv->scenes[scene_id].pending.emplace_back(request_id, dt);
    return SCWP_OK;
}

scwp_status scwp_server_tick(scwp_server* sv, int32_t* started) {
    if (!sv || !started) return SCWP_E_INVALID;
    *started = 0;
    int slot = -1;
    for (size_t k = 0; k < sv->slot_busy.size() && slot < 0; ++k)
        if (!sv->slot_busy[k]) slot = (int)k;
    if (slot < 0) return SCWP_OK;   // every tick slot is in flight
    const int ns = (int)sv->scenes.size();
    std::vector<int> take;
    for (int k = 0; k < ns; ++k) {
        const int i = (sv->rr + k) % ns;
        const ServerScene& sc = sv->scenes[i];
        if (sc.ctx && !sc.in_flight && !sc.pending.empty()) take.push_back(i);
    }
    if (take.empty()) return SCWP_OK;
    sv->rr = (sv->rr + 1) % ns;
    ServerTick tk;
    tk.slot = slot;
    tk.done = sv->tick_events[slot];
    // background and particle stages, one scene per stream in turn
    std::vector<bool> used(sv->pst.size(), false);
    for (size_t k = 0; k < take.size(); ++k) {
        ServerScene& sc = sv->scenes[take[k]];
        const size_t q = k % sv->pst.size();
        const std::pair<int64_t, double> rq = sc.pending.front();
        const scwp_status s = scene_prepare(sc.ctx, rq.second, sv->pst[q]);
        if (s != SCWP_OK) return sfail(sv, s, std::string("scene prepare: ") + sc.ctx->err);
        used[q] = true;
        sc.pending.pop_front();
        sc.in_flight = true;
        tk.reqs.emplace_back(take[k], rq.first);
    }
    for (size_t q = 0; q < sv->pst.size(); ++q)
        if (used[q]) {
            SCU(cudaEventRecord(sv->pev[q], sv->pst[q]));
            SCU(cudaStreamWaitEvent(sv->st, sv->pev[q], 0));
        }
    // the union of the scenes' synthesis plans, heaviest first: one list for
    // the scenes on the summed-area synthesis (the default), one for those on
    // the tensor-core gather
    std::vector<PatchDev> pd;
    std::vector<SynthParams> sp;
    std::vector<TcItem> items[2];
    std::vector<double> work[2];
    std::vector<BlendSpan> spans[2];
    for (int i : take) {
        scwp_ctx* c = sv->scenes[i].ctx;
        const int base = (int)pd.size();
        for (size_t p = 0; p < c->patches.size(); ++p) {
            pd.push_back(c->patches[p]->dev);
            sp.push_back(c->h_sps[p]);
        }
        const int m = c->synth_mode == SCWP_SYNTH_SAT ? 1 : 0;
        const std::vector<TcItem>& ci = m ? c->s_items : c->b_items;
        const std::vector<double>& cw = m ? c->s_work : c->b_work;
        for (size_t k = 0; k < ci.size(); ++k) {
            TcItem it = ci[k];
            it.patch += base;
            items[m].push_back(it);
            work[m].push_back(cw[k]);
        }
        for (BlendSpan b : (m ? c->s_spans : c->b_spans)) {
            b.patch += base;
            spans[m].push_back(b);
        }
    }
    std::vector<int> order[2];
    for (int m = 0; m < 2; ++m) {
        order[m].resize(items[m].size());
        for (size_t k = 0; k < order[m].size(); ++k) order[m][k] = (int)k;
        const std::vector<double>& w = work[m];
        std::stable_sort(order[m].begin(), order[m].end(), [&](int a, int b) { return w[a] > w[b]; });
    }
    const size_t o_sp = align16(pd.size() * sizeof(PatchDev));
    size_t o_it[2], o_bs[2];
    o_it[0] = o_sp + align16(sp.size() * sizeof(SynthParams));
    o_bs[0] = o_it[0] + align16(items[0].size() * sizeof(TcItem));
    o_it[1] = o_bs[0] + align16(spans[0].size() * sizeof(BlendSpan));
    o_bs[1] = o_it[1] + align16(items[1].size() * sizeof(TcItem));
    const size_t bytes = o_bs[1] + align16(std::max<size_t>(1, spans[1].size()) * sizeof(BlendSpan));
    if (sv->stage_cap[slot] < bytes) {
        if (sv->hstage[slot]) cudaFreeHost(sv->hstage[slot]);
        sv_free(sv, sv->dstage[slot]);
        sv->hstage[slot] = nullptr;
        sv->dstage[slot] = nullptr;
        sv->stage_cap[slot] = 0;
        const size_t cap = bytes * 2;
        if (cudaMallocHost(&sv->hstage[slot], cap) != cudaSuccess) {
            sv->hstage[slot] = nullptr;
            cudaGetLastError();
            return sfail(sv, SCWP_E_NOMEM, "tick staging");
        }
        sv->dstage[slot] = sv_alloc(sv, cap);
        if (!sv->dstage[slot]) return sfail(sv, SCWP_E_NOMEM, "tick staging");
        sv->stage_cap[slot] = cap;
    }
    unsigned char* h = (unsigned char*)sv->hstage[slot];
    memcpy(h, pd.data(), pd.size() * sizeof(PatchDev));
    memcpy(h + o_sp, sp.data(), sp.size() * sizeof(SynthParams));
    for (int m = 0; m < 2; ++m) {
        TcItem* hi = reinterpret_cast<TcItem*>(h + o_it[m]);
        for (size_t k = 0; k < order[m].size(); ++k) hi[k] = items[m][order[m][k]];
        if (!spans[m].empty()) memcpy(h + o_bs[m], spans[m].data(), spans[m].size() * sizeof(BlendSpan));
    }
    unsigned char* dv = (unsigned char*)sv->dstage[slot];
    SCU(cudaMemcpyAsync(dv, h, bytes, cudaMemcpyHostToDevice, sv->st));
    const PatchDev* dpd = reinterpret_cast<const PatchDev*>(dv);
    const SynthParams* dsp = reinterpret_cast<const SynthParams*>(dv + o_sp);
    if (!items[0].empty())
        SCU(launch_synth_tc(reinterpret_cast<const TcItem*>(dv + o_it[0]), (int)items[0].size(), dpd, dsp,
                            reinterpret_cast<const BlendSpan*>(dv + o_bs[0]), (int)spans[0].size(), sv->st));
    if (!items[1].empty())
        SCU(launch_synth_sat(reinterpret_cast<const TcItem*>(dv + o_it[1]), (int)items[1].size(), dpd, dsp,
                             reinterpret_cast<const BlendSpan*>(dv + o_bs[1]), (int)spans[1].size(), sv->queue,
                             sv->st));
    SCU(cudaEventRecord(tk.done, sv->st));
    sv->slot_busy[slot] = true;
    *started = (int32_t)tk.reqs.size();
    sv->ticks.push_back(std::move(tk));
    sv->ticks_launched += 1;
    return SCWP_OK;
}

scwp_status scwp_server_poll(scwp_server* sv, int64_t* done_ids, int32_t max_ids, int32_t* n_done) {
    if (!sv || !n_done || max_ids < 0 || (max_ids > 0 && !done_ids)) return SCWP_E_INVALID;
    *n_done = 0;
    while (!sv->ticks.empty()) {
        ServerTick& tk = sv->ticks.front();
        const cudaError_t q = cudaEventQuery(tk.done);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return sfail(sv, SCWP_E_CUDA, std::string("tick: ") + cudaGetErrorString(q));
        while (tk.next < tk.reqs.size() && *n_done < max_ids) {
            const std::pair<int, int64_t>& r = tk.reqs[tk.next++];
            sv->scenes[r.first].in_flight = false;
            done_ids[(*n_done)++] = r.second;
        }
        if (tk.next < tk.reqs.size()) break;   // the caller's array is full
        sv->slot_busy[tk.slot] = false;
        sv->requests_done += (int64_t)tk.reqs.size();
        sv->ticks.pop_front();
    }
    return SCWP_OK;
}

scwp_status scwp_server_scene(scwp_server* sv, int32_t scene_id, scwp_ctx** ctx) {
    if (!sv || !ctx || scene_id < 0 || scene_id >= (int)sv->scenes.size() || !sv->scenes[scene_id].ctx)
        return SCWP_E_INVALID;
    *ctx = sv->scenes[scene_id].ctx;
    return SCWP_OK;
}

scwp_status scwp_server_info_get(scwp_server* sv, scwp_server_info* out) {
    if (!sv || !out) return SCWP_E_INVALID;
    memset(out, 0, sizeof(*out));
    for (const ServerScene& sc : sv->scenes)
        if (sc.ctx) {
            out->scenes += 1;
            out->pending_requests += (int64_t)sc.pending.size();
            out->frames_in_flight += sc.in_flight ? 1 : 0;
        }
    out->device_bytes = (int64_t)sv->used;
    out->budget_bytes = (int64_t)sv->d.hbm_budget_bytes;
    out->ticks_in_flight = (int32_t)sv->ticks.size();
    out->ticks_launched = sv->ticks_launched;
    out->requests_done = sv->requests_done;
    return SCWP_OK;
}

const char* scwp_server_last_error(scwp_server* sv) { return sv ? sv->err.c_str() : "null server"; }

void scwp_server_destroy(scwp_server* sv) {
    if (!sv) return;
    if (sv->st) cudaStreamSynchronize(sv->st);
    for (cudaStream_t s : sv->pst) cudaStreamSynchronize(s);
    cudaGetLastError();
    for (ServerScene& sc : sv->scenes)
        if (sc.ctx) scwp_destroy(sc.ctx);
    for (size_t k = 0; k < sv->hstage.size(); ++k) {
        if (sv->hstage[k]) cudaFreeHost(sv->hstage[k]);
        sv_free(sv, sv->dstage[k]);
    }
    for (cudaEvent_t e : sv->tick_events)
        if (e) cudaEventDestroy(e);
    sv_free(sv, sv->queue);
    for (cudaStream_t s : sv->pst) cudaStreamDestroy(s);
    for (cudaEvent_t e : sv->pev) cudaEventDestroy(e);
    cudaGetLastError();
    delete sv;
}

}  // extern "C"
