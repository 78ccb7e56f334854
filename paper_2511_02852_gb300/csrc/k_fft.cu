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
// of the first stage fall on distinct banks.  Twiddles e^{2 pi i m / N} come
// from a float table built in float64 on the host.  The inverse transform is
// unnormalised: f[j] = sum_m F[m] e^{+2 pi i m j / N}.
#include <cuda_runtime.h>
#include <stdint.h>

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
// stride of one transform in shared memory: the padded length, rounded to
// 2 mod 16 complex values so that consecutive transforms start 4 banks apart
// (the column pass's loads and stores walk across transforms)
template <int N>
__host__ __device__ constexpr int tstride() { return padded<N>() + ((18 - padded<N>() % 16) % 16); }
// columns per column-pass CTA for h + i Dx (twice as many for Dy, in pairs)
template <int N>
__host__ __device__ constexpr int col_group() { return N >= 2048 ? 4 : N >= 1024 ? 8 : N >= 32 ? 16 : N / 2; }


// e^{+2 pi i k / 16}, k = 0 .. 7 (the roots the 16-point transform uses)
__device__ __forceinline__ float2 root16(int k) {
    constexpr float c1 = 0.9238795325f, c2 = 0.7071067812f, c3 = 0.3826834324f;
    switch (k & 7) {
        case 0: return make_float2(1.f, 0.f);
        case 1: return make_float2(c1, c3);
        case 2: return make_float2(c2, c2);
        case 3: return make_float2(c3, c1);
        case 4: return make_float2(0.f, 1.f);
        case 5: return make_float2(-c3, c1);
        case 6: return make_float2(-c2, c2);
        default: return make_float2(-c1, c3);
    }
}

// In-register inverse DFT of R points (R = 2, 4, 8, 16): radix-2
// decimation in time on bit-reversed input, result in natural order.
template <int R>
__device__ __forceinline__ void dft_inv(float2 (&v)[R]) {
    constexpr int L = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
    float2 u[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int r = 0;
#pragma unroll
        for (int b = 0; b < L; ++b) r |= ((i >> b) & 1) << (L - 1 - b);
        u[r] = v[i];
    }
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
        for (int i = 0; i < R; i += len) {
#pragma unroll
            for (int j = 0; j < len / 2; ++j) {
                const float2 w = root16(j * (16 / len));   // e^{2 pi i j / len}
                const float2 a = u[i + j];
                const float2 b = j == 0 ? u[i + j + len / 2] : cmul(w, u[i + j + len / 2]);
                u[i + j] = cadd(a, b);
                u[i + j + len / 2] = csub(a, b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = u[i];
}

// Multiply v[r] by the twiddle e^{2 pi i r m / N}, r = 1 .. R - 1, of one
// butterfly (m = k step): e^{2 pi i m / N} to the powers 1, 2, 4, 8 come
// from the table (one load each), the others are products of two or three
// of them (at most three roundings, within 3e-7 of the table values), so a
// radix-16 butterfly loads 4 twiddles instead of 15.
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 (&v)[R], int m, const float2* __restrict__ tw) {
    const float2 w1 = __ldg(&tw[m]);
    v[1] = cmul(v[1], w1);
    if constexpr (R >= 4) {
        const float2 w2 = __ldg(&tw[2 * m]);
        const float2 w3 = cmul(w1, w2);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if constexpr (R >= 8) {
            const float2 w4 = __ldg(&tw[4 * m]);
            const float2 w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], w5);
            v[6] = cmul(v[6], w6);
            v[7] = cmul(v[7], w7);
            if constexpr (R >= 16) {
                const float2 w8 = __ldg(&tw[8 * m]);
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
        if constexpr (Ns > 1) apply_twiddles<R>(v[q], k * (N / (Ns * R)), tw);
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
        const float kk = sqrtf(kx * kx + ky * ky);
        float ux = 0.f, uy = 0.f;
        if (kk > 0.f) {
            ux = kx / kk;
            uy = ky / kk;
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

}  // namespace scwp
