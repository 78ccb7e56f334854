// FFT background of the hybrid ocean (sm_103a): the spectrum update fused
// with the row pass of the inverse 2-D FFT, then the column pass
// (Sec. 3.1 / Sec. 4.1: the conventional spectral evolution and inverse FFT).
//
//   h~(k,t) = h0(k) e^{i w t} + conj(h0(-k)) e^{-i w t}
//   D~(k,t) = -i lambda_c (k/|k|) h~(k,t)
//   h(x) = sum_k h~(k) e^{+i k.x},  Dx, Dy likewise     (real: h~(-k) = conj(h~(k)))
//
// Hermitian halves.  Every field is real, so the row pass (along x) runs
// only for the rows k_y = 0 .. N/2: H1(x, -k_y) = conj(H1(x, k_y)).  A row
// k_y reads h0 rows k_y and -k_y once each and w(k) (even in k) once, and
// transforms three rows: H~, D~x, D~y.  The column pass (along y) rebuilds
// the rows k_y > N/2 by conjugation and packs the real results two to a
// complex transform: Z = H1 + i Dx1 gives h + i Dx of a column; W = Dy1(x) +
// i Dy1(x + 1) gives Dy of two columns.  That is 1.5 complex transforms of
// length N per row and per column, and an intermediate of 3 x (N/2 + 1) x N
// complex values.
//
// Phase without float64: w(k) is stored as a float pair w_hi + w_lo and t
// comes as a float pair t_hi + t_lo (both split on the host); w t is formed
// as an unevaluated float pair (exact product by fma plus the cross terms)
// and reduced modulo 2 pi by Cody-Waite with 2 pi split in two floats (the
// residue p - n C1 is exact in float, the C2 term and the pair's low part
// each add one rounding), so the phase stays within 2.3e-7 rad of the float64
// value (checked on 20,000 random (w, t) with |w t| up to 4,000 rad; the
// workloads reach hundreds of radians after a minute), before a precise
// sincosf.
//
// The transforms: a radix-16 (last stage 8, 4 or 2) Stockham autosort in
// registers, 16 values per thread, each stage one shared-memory round trip
// (load, barrier, twiddle, 16-point transform, store, barrier) on one buffer
// per transform, padded by one element every 16 so that the strided stores
// of the first stage fall on distinct banks.  The inverse transform is
// unnormalised: f[j] = sum_m F[m] e^{+2 pi i m j / N}.
//
// Twiddles come from a float table built in float64 on the host, laid out by
// stage: for each stage after the first (span Ns = 16, 256, ..., radix
// R = min(16, N / Ns)) the powers e^{2 pi i p k / (Ns R)}, p = 1, 2, 4, 8
// (p < R), k = 0 .. Ns - 1, stored [p][k].  The threads of a warp take
// consecutive butterflies k, so each of their twiddle loads reads one run of
// consecutive entries (a table indexed by m = p k N / (Ns R) would scatter
// the loads of a warp over up to 32 sectors).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "internal.h"

namespace scwp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

template <int N>
__host__ __device__ constexpr int threads_per_transform() { return N >= 16 ? N / 16 : 1; }
template <int N>
__host__ __device__ constexpr int padded() { return N + N / 16; }
// columns per column-pass CTA for h + i Dx (twice as many for Dy, in pairs)
template <int N>
__host__ __device__ constexpr int col_group() { return N >= 2048 ? 4 : N >= 1024 ? 8 : N >= 32 ? 16 : N / 2; }
// stride of one transform in shared memory: the padded length, rounded to
// 16 / CZ mod 16 complex values (CZ = col_group).  The column pass's
// transposes put lane l of a warp at transform l mod CZ, row l / CZ; with
// that stride the 16 lanes of each half warp (the lanes one shared-memory
// wavefront of 8-byte accesses serves) meet 16 different two-word bank
// slots, so a warp's access takes two wavefronts, the least it can.
template <int N>
__host__ __device__ constexpr int tstride() {
    return padded<N>() + (((16 / col_group<N>()) % 16 - padded<N>() % 16 + 16) % 16);
}

// the stages' twiddle tables (see the header): radix of the stage of span
// Ns, and the offset of that stage's table
__host__ __device__ constexpr int log2c(int x) { return x <= 1 ? 0 : 1 + log2c(x / 2); }
__host__ __device__ constexpr int radix_at(int N, int Ns) { return N / Ns >= 16 ? 16 : N / Ns; }
__host__ __device__ constexpr int tw_base(int N, int Ns) {
    return Ns <= 16 ? 0 : tw_base(N, Ns / 16) + log2c(radix_at(N, Ns / 16)) * (Ns / 16);
}


// a e^{+2 pi i e / 16} for the exponents of the 16-point transform
constexpr float kC1 = 0.92387953251128674f;   // cos(pi / 8)
constexpr float kS1 = 0.38268343236508977f;   // sin(pi / 8)
constexpr float kH = 0.70710678118654752f;    // cos(pi / 4)
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }   // e = 4
__device__ __forceinline__ float2 mul_e2(float2 a) { return make_float2(kH * (a.x - a.y), kH * (a.x + a.y)); }
__device__ __forceinline__ float2 mul_e6(float2 a) { return make_float2(-kH * (a.x + a.y), kH * (a.x - a.y)); }
__device__ __forceinline__ float2 mul_cs(float2 a, float c, float s) {
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

// In-register inverse DFT of R points (R = 2, 4, 8, 16), natural order in
// and out: X[k] = sum_n v[n] e^{+2 pi i n k / R}.  R = 16 is a 4 x 4
// decomposition (n = 4 n1 + n2, k = k1 + 4 k2: four 4-point transforms over
// n1, the factors e^{2 pi i n2 k1 / 16}, four 4-point transforms over n2),
// R = 8 a 2 x 4 one; multiplications by 1 and i are moves, those by
// e^{i pi/4} and e^{3 i pi/4} two products each.
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = make_float2(d02.x - d13.y, d02.y + d13.x);   // d02 + i d13
    a3 = make_float2(d02.x + d13.y, d02.y - d13.x);   // d02 - i d13
}

template <int R>
__device__ __forceinline__ void dft_inv(float2 (&v)[R]) {
    if constexpr (R == 2) {
        const float2 a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    } else if constexpr (R == 4) {
        dft4(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        // even and odd halves, then X[k] = E[k] + e^{i pi k/4} O[k], X[k + 4] = E[k] - ...
        dft4(v[0], v[2], v[4], v[6]);
        dft4(v[1], v[3], v[5], v[7]);
        const float2 o1 = mul_e2(v[3]), o2 = mul_i(v[5]), o3 = mul_e6(v[7]);
        const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        v[0] = cadd(e0, v[1]);
        v[4] = csub(e0, v[1]);
        v[1] = cadd(e1, o1);
        v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2);
        v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3);
        v[7] = csub(e3, o3);
    } else {
        static_assert(R == 16, "radix 2, 4, 8 or 16");
        // y[n2][k1] in v[4 k1 + n2]... computed in place: the 4-point
        // transform over n1 of column n2 leaves k1 at v[n2 + 4 k1]
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
        // factors e^{2 pi i n2 k1 / 16} (n2, k1 >= 1)
        v[5] = mul_cs(v[5], kC1, kS1);     // 1
        v[6] = mul_e2(v[6]);               // 2
        v[7] = mul_cs(v[7], kS1, kC1);     // 3
        v[9] = mul_e2(v[9]);               // 2
        v[10] = mul_i(v[10]);              // 4
        v[11] = mul_e6(v[11]);             // 6
        v[13] = mul_cs(v[13], kS1, kC1);   // 3
        v[14] = mul_e6(v[14]);             // 6
        v[15] = mul_cs(v[15], -kC1, -kS1); // 9
        // 4-point transforms over n2 of row k1: X[k1 + 4 k2]
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
        // v[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4 x 4 block
        float2 t;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a + 1; b < 4; ++b) {
                t = v[4 * a + b];
                v[4 * a + b] = v[4 * b + a];
                v[4 * b + a] = t;
            }
    }
}

// Multiply v[r] by the twiddle e^{2 pi i r k / (Ns R)}, r = 1 .. R - 1, of
// butterfly k of a stage of span Ns: the powers r = 1, 2, 4, 8 come from
// the stage's table tws ([p][k], one load each), the others are products of
// two or three of them (at most three roundings, within 3e-7 of the exact
// values), so a radix-16 butterfly loads 4 twiddles instead of 15.
template <int R, int Ns>
__device__ __forceinline__ void apply_twiddles(float2 (&v)[R], int k, const float2* __restrict__ tws) {
    const float2 w1 = __ldg(&tws[k]);
    v[1] = cmul(v[1], w1);
    if constexpr (R >= 4) {
        const float2 w2 = __ldg(&tws[Ns + k]);
        const float2 w3 = cmul(w1, w2);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if constexpr (R >= 8) {
            const float2 w4 = __ldg(&tws[2 * Ns + k]);
            const float2 w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], w5);
            v[6] = cmul(v[6], w6);
            v[7] = cmul(v[7], w7);
            if constexpr (R >= 16) {
                const float2 w8 = __ldg(&tws[3 * Ns + k]);
                v[8] = cmul(v[8], w8);
                v[9] = cmul(v[9], cmul(w1, w8));
                v[10] = cmul(v[10], cmul(w2, w8));
                v[11] = cmul(v[11], cmul(w3, w8));
                v[12] = cmul(v[12], cmul(w4, w8));
                v[13] = cmul(v[13], cmul(w5, w8));
                v[14] = cmul(v[14], cmul(w6, w8));
                v[15] = cmul(v[15], cmul(w7, w8));
            }
        }
    }
}

// One Stockham stage of radix R over the transforms of a block: thread jt
// (0 <= jt < P = N / 16) of transform `buf` does the 16 / R butterflies
// j = jt + q P.  Butterfly j (span Ns): k = j mod Ns; inputs x[j + r N/R]
// times e^{2 pi i r k / (Ns R)}, an R-point transform, outputs at
// (j - k) R + k + s Ns.  All loads come before the barrier, all stores after.
// The first stage (Ns = 1) has no twiddles.
template <int N, int R, int Ns>
__device__ __forceinline__ void stage(float2* buf, int jt, const float2* __restrict__ tw) {
    constexpr int P = threads_per_transform<N>();
    constexpr int B = (N >= 16 ? 16 : N) / R;   // butterflies per thread
    float2 v[B][R];
#pragma unroll
    for (int q = 0; q < B; ++q)
#pragma unroll
        for (int r = 0; r < R; ++r) v[q][r] = buf[pad(jt + q * P + r * (N / R))];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = jt + q * P;
        const int k = j & (Ns - 1);
        if constexpr (Ns > 1) apply_twiddles<R, Ns>(v[q], k, tw + tw_base(N, Ns));
        dft_inv<R>(v[q]);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int s = 0; s < R; ++s) buf[pad(d + s * Ns)] = v[q][s];
    }
    __syncthreads();
}

// the stages of a length-N inverse transform: radix 16 while 16 divides the
// rest, then one stage of radix 8, 4 or 2
template <int N, int Ns>
__device__ __forceinline__ void stages_from(float2* buf, int jt, const float2* __restrict__ tw) {
    if constexpr (N / Ns >= 16) {
        stage<N, 16, Ns>(buf, jt, tw);
        stages_from<N, Ns * 16>(buf, jt, tw);
    } else if constexpr (N / Ns > 1) {
        stage<N, N / Ns, Ns>(buf, jt, tw);
    }
}

// Inverse FFT of length N of the transform in `buf` (padded layout) by the
// P = N / 16 threads jt of it (every thread of the block takes part in the
// barriers).
template <int N>
__device__ __forceinline__ void fft_inv(float2* buf, int jt, const float2* __restrict__ tw) {
    stages_from<N, 1>(buf, jt, tw);
}


// w t reduced into (-pi, pi] from float pairs (w_hi, w_lo), (t_hi, t_lo)
__device__ __forceinline__ float phase(float2 w, float th, float tl) {
    const float p = w.x * th;
    const float e = fmaf(w.x, th, -p);                  // w_hi t_hi - p, exactly
    const float c = fmaf(w.x, tl, w.y * th);            // the cross terms
    const float n = rintf(p * 0.15915493667125702f);    // p / (2 pi)
    float r = fmaf(-n, 6.2831854820251465f, p);         // p - n C1: exact in float
    r = fmaf(-n, -1.7484555314695172e-07f, r);          // 2 pi - C1
    return r + (e + c);
}

// Rows pass: spectrum update (a1) + inverse FFT along x of H~, D~x, D~y for
// row k_y = blockIdx.x in 0 .. N/2.  Block: 3 P threads; transform
// f = tid / P.  h0 is [N][N] (FFT-natural order), omega [N][N] float pairs
// (hi, lo); I is [3][N/2 + 1][N].
template <int N>
__global__ void __launch_bounds__(3 * threads_per_transform<N>(), N >= 4096 ? 1 : N >= 1024 ? 3 : 1)
    k_spectrum_rows(BgDev bg, float th, float tl, const float2* t_dev) {
    constexpr int P = threads_per_transform<N>(), Np = tstride<N>();
    constexpr int NT = 3 * P, E = (N + NT - 1) / NT;   // grid points per thread
    extern __shared__ float2 smem_rows[];
    float2 (*buf)[Np] = reinterpret_cast<float2 (*)[Np]>(smem_rows);   // [3][Np]
    pdl_enter();
    if (t_dev) {
        const float2 tt = *t_dev;
        th = tt.x;
        tl = tt.y;
    }
    const int my = blockIdx.x;
    const int mym = (N - my) & (N - 1);
    const int ny = my < N / 2 ? my : my - N;
    const float ky = bg.dk * (float)ny;
    // every load of the thread's grid points first
    float2 av[E], bv[E], wv[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int mx = threadIdx.x + i * NT;
        if (mx < N) {
            av[i] = bg.h0[(size_t)my * N + mx];
            bv[i] = bg.h0[(size_t)mym * N + ((N - mx) & (N - 1))];
            wv[i] = bg.omega[(size_t)my * N + mx];
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int mx = threadIdx.x + i * NT;
        if (mx >= N) continue;
        const int nx = mx < N / 2 ? mx : mx - N;
        const float2 a = av[i], b = bv[i];
        float s, c;
        sincosf(phase(wv[i], th, tl), &s, &c);
        // h~ = h0(k) e^{i w t} + conj(h0(-k) e^{i w t})
        const float2 q = make_float2(b.x * c - b.y * s, b.x * s + b.y * c);
        const float2 ht = make_float2(a.x * c - a.y * s + q.x, a.x * s + a.y * c - q.y);
        const float kx = bg.dk * (float)nx;
        const float k2 = kx * kx + ky * ky;
        float ux = 0.f, uy = 0.f;
        if (k2 > 0.f) {   // k / |k|
            const float rk = rsqrtf(k2);
            ux = kx * rk;
            uy = ky * rk;
        }
        // D~ = -i lam u h~ = lam u (h~.y, -h~.x)
        buf[0][pad(mx)] = ht;
        buf[1][pad(mx)] = make_float2(bg.lam * ux * ht.y, -bg.lam * ux * ht.x);
        buf[2][pad(mx)] = make_float2(bg.lam * uy * ht.y, -bg.lam * uy * ht.x);
    }
    __syncthreads();
    const int f = threadIdx.x / P, jt = threadIdx.x % P;
    fft_inv<N>(buf[f], jt, bg.tw);
    const size_t rows = (size_t)(N / 2 + 1) * N;
    for (int w = threadIdx.x; w < 3 * N; w += 3 * P) {
        const int g = w / N, x = w - g * N;
        bg.I[g * rows + (size_t)my * N + x] = buf[g][pad(x)];
    }
}

// Columns pass.  Blocks 0 .. N/CZ - 1: columns x0 .. x0 + CZ - 1 of h and Dx
// (one transform Z = H1 + i Dx1 per column); blocks N/CZ .. : columns
// x0 .. x0 + 2 CZ - 1 of Dy (one transform W = Dy1(x) + i Dy1(x + 1) per
// column pair).  The rows k_y > N/2 of H1, Dx1 and Dy1 are the conjugates of
// the rows N - k_y.  out is [3][N][N] (h, Dx, Dy), row-major.
template <int N>
__global__ void __launch_bounds__(col_group<N>() * threads_per_transform<N>(),
                                  col_group<N>() * threads_per_transform<N>() <= 512 ? 2 : 1) k_fft_cols(BgDev bg) {
    constexpr int P = threads_per_transform<N>(), Np = tstride<N>(), CZ = col_group<N>();
    constexpr int NT = CZ * P;
    extern __shared__ float2 smem_cols[];
    float2 (*buf)[Np] = reinterpret_cast<float2 (*)[Np]>(smem_cols);   // [CZ][Np]
    pdl_enter();
    const size_t rows = (size_t)(N / 2 + 1) * N;
    const bool dy = (int)blockIdx.x >= N / CZ;
    const int x0 = dy ? ((int)blockIdx.x - N / CZ) * 2 * CZ : (int)blockIdx.x * CZ;
    // load: element (k_y, c) with c fastest (CZ consecutive columns of a
    // row), every load of the thread issued before the first store
    constexpr int E = ((N / 2 + 1) * CZ + NT - 1) / NT;
    float4 ld[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int w = threadIdx.x + i * NT;
        if (w < (N / 2 + 1) * CZ) {
            const int m = w / CZ, c = w - m * CZ;
            if (!dy) {
                const float2 h = bg.I[(size_t)m * N + x0 + c], d = bg.I[rows + (size_t)m * N + x0 + c];
                ld[i] = make_float4(h.x, h.y, d.x, d.y);
            } else {
                ld[i] = *reinterpret_cast<const float4*>(&bg.I[2 * rows + (size_t)m * N + x0 + 2 * c]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int w = threadIdx.x + i * NT;
        if (w >= (N / 2 + 1) * CZ) continue;
        const int m = w / CZ, c = w - m * CZ;
        // (p, q) = (H1, Dx1) or (Dy1(x), Dy1(x + 1)): the transform's rows m
        // and N - m are p + i q and conj(p) + i conj(q)
        const float4 pq = ld[i];
        buf[c][pad(m)] = make_float2(pq.x - pq.w, pq.y + pq.z);
        if (m > 0 && m < N / 2) buf[c][pad(N - m)] = make_float2(pq.x + pq.w, pq.z - pq.y);
    }
    __syncthreads();
    const int t = threadIdx.x / P, jt = threadIdx.x % P;
    fft_inv<N>(buf[t], jt, bg.tw);
    const size_t plane = (size_t)N * N;
    if (!dy) {
        for (int w = threadIdx.x; w < N * CZ; w += NT) {
            const int y = w / CZ, c = w - y * CZ;
            const float2 v = buf[c][pad(y)];
            bg.out[(size_t)y * N + x0 + c] = v.x;
            bg.out[plane + (size_t)y * N + x0 + c] = v.y;
        }
    } else {
        for (int w = threadIdx.x; w < N * CZ; w += NT) {
            const int y = w / CZ, c = w - y * CZ;
            const float2 v = buf[c][pad(y)];
            *reinterpret_cast<float2*>(&bg.out[2 * plane + (size_t)y * N + x0 + 2 * c]) = v;
        }
    }
}

template <int N>
cudaError_t launch_n(const BgDev& bg, float th, float tl, cudaStream_t st, const float2* t_dev) {
    constexpr int P = threads_per_transform<N>(), CZ = col_group<N>();
    constexpr size_t smr = sizeof(float2) * 3 * tstride<N>(), smc = sizeof(float2) * CZ * tstride<N>();
    static_assert(smc <= 227 * 1024 && smr <= 227 * 1024, "shared memory of one CTA");
    static int attr[kMaxCachedDevices] = {};
    const int ok = cached_per_device(attr, [] {
        const cudaError_t e =
            cudaFuncSetAttribute(k_spectrum_rows<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
        return (e == cudaSuccess &&
                cudaFuncSetAttribute(k_fft_cols<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc) ==
                    cudaSuccess)
                   ? 1
                   : -1;
    });
    if (ok < 0) {
        cudaGetLastError();
        return cudaErrorInvalidValue;
    }
    cudaError_t e;
    e = launch_pdl(k_spectrum_rows<N>, N / 2 + 1, 3 * P, smr, st, bg, th, tl, t_dev);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_fft_cols<N>, N / CZ + N / (2 * CZ), CZ * P, smc, st, bg);
    count_launches(2);
    return e;
}

}  // namespace

cudaError_t launch_background(const BgDev& bg, double t, cudaStream_t st, const float2* t_dev) {
    // the time as a float pair (split on the host, in float64)
    const float th = (float)t;
    const float tl = (float)(t - (double)th);
    switch (bg.N) {
        case 8: return launch_n<8>(bg, th, tl, st, t_dev);
        case 16: return launch_n<16>(bg, th, tl, st, t_dev);
        case 32: return launch_n<32>(bg, th, tl, st, t_dev);
        case 64: return launch_n<64>(bg, th, tl, st, t_dev);
        case 128: return launch_n<128>(bg, th, tl, st, t_dev);
        case 256: return launch_n<256>(bg, th, tl, st, t_dev);
        case 512: return launch_n<512>(bg, th, tl, st, t_dev);
        case 1024: return launch_n<1024>(bg, th, tl, st, t_dev);
        case 2048: return launch_n<2048>(bg, th, tl, st, t_dev);
        case 4096: return launch_n<4096>(bg, th, tl, st, t_dev);
        default: return cudaErrorInvalidValue;
    }
}

size_t background_scratch_elems(int N) { return (size_t)3 * (N / 2 + 1) * N; }

size_t background_twiddle_elems(int N) {
    size_t n = 0;
    for (int Ns = 16; Ns < N; Ns *= 16) n += (size_t)log2c(radix_at(N, Ns)) * Ns;
    return n;
}

void build_background_twiddles(int N, float2* out) {
    size_t o = 0;
    for (int Ns = 16; Ns < N; Ns *= 16) {
        const int R = radix_at(N, Ns);
        for (int p = 1; p < R; p *= 2)
            for (int k = 0; k < Ns; ++k) {
                // e^{2 pi i p k / (Ns R)} = e^{2 pi i m / N}
                const long long m = (long long)p * k * (N / (Ns * R));
                const double a = 2.0 * M_PI * (double)m / (double)N;
                out[o++] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
    }
}

}  // namespace scwp
