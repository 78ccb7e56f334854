/*
 * FP64 oracle loops for the wave-particle synthesis (Sec. 4.2) of the hybrid
 * ocean.  TEST INFRASTRUCTURE ONLY: called by the Python oracle through
 * ctypes; the CUDA library never links or calls this file.
 *
 * Bump kernel (reading of Fig. 1 and Sec. 4.2: a separable raised cosine,
 * the kernel that two separable passes along x and y implement):
 *   K(u, v) = k(u) k(v),  k(u) = 1/2 (1 + cos(pi u / R)) for |u| < R, else 0,
 * with u, v the texel-centre offsets from the bump centre in Q16.16 cells
 * and R the bucket's half-width (r = lambda / 2) in the same units.
 * Displacement (reading of "derived by finite differences", Sec. 4.2): the
 * analytic gradient, D = -(lambda_c / k) grad h per bump, k = pi / r, i.e.
 *   Dx += (lambda_c / 2) a sin(pi u / R) k(v),  Dy += (lambda_c / 2) a k(u) sin(pi v / R).
 *
 * Each texel sums its bumps in bump order; rows are independent, so the
 * result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>

#define Q 65536LL
#define HALF 32768LL

static int64_t floor_div_q(int64_t a) { return a >> 16; } /* arithmetic shift = floor(a / 2^16) */

void oracle_synth(int64_t W, int64_t H, int64_t nbump,
                  const int64_t* bx, const int64_t* by, const int64_t* br,
                  const double* ba, double lam_half,
                  double* h, double* dx, double* dy, int64_t* evals_per_row)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t iy = 0; iy < H; ++iy) {
        const int64_t yt = iy * Q + HALF;
        int64_t ev = 0;
        double* hr = h + iy * W;
        double* xr = dx + iy * W;
        double* yr = dy + iy * W;
        for (int64_t b = 0; b < nbump; ++b) {
            const int64_t R = br[b];
            const int64_t dyq = yt - by[b];
            if (dyq <= -R || dyq >= R) continue;
            const double ty = (double)dyq / (double)R;
            const double ky = 0.5 * (1.0 + cos(M_PI * ty));
            const double sy = sin(M_PI * ty);
            int64_t lo = floor_div_q(bx[b] - R - HALF) + 1;
            int64_t hi = floor_div_q(bx[b] + R - HALF - 1);
            if (lo < 0) lo = 0;
            if (hi > W - 1) hi = W - 1;
            const double a = ba[b];
            for (int64_t ix = lo; ix <= hi; ++ix) {
                const int64_t dxq = ix * Q + HALF - bx[b];
                const double tx = (double)dxq / (double)R;
                const double kx = 0.5 * (1.0 + cos(M_PI * tx));
                const double sx = sin(M_PI * tx);
                hr[ix] += a * kx * ky;
                xr[ix] += lam_half * a * sx * ky;
                yr[ix] += lam_half * a * kx * sy;
                ++ev;
            }
        }
        evals_per_row[iy] = ev;
    }
}

/* Point evaluation at a list of texels (ix, iy) over all bumps: the same sum
 * as oracle_synth, for sampled parity checks of large maps. */
void oracle_synth_points(int64_t npts, const int64_t* pix, const int64_t* piy,
                         int64_t nbump, const int64_t* bx, const int64_t* by,
                         const int64_t* br, const double* ba, double lam_half,
                         double* h, double* dx, double* dy)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t xt = pix[p] * Q + HALF, yt = piy[p] * Q + HALF;
        double sh = 0.0, sx = 0.0, sy = 0.0;
        for (int64_t b = 0; b < nbump; ++b) {
            const int64_t R = br[b];
            const int64_t du = xt - bx[b], dv = yt - by[b];
            if (du <= -R || du >= R || dv <= -R || dv >= R) continue;
            const double tu = (double)du / (double)R, tv = (double)dv / (double)R;
            const double ku = 0.5 * (1.0 + cos(M_PI * tu)), kv = 0.5 * (1.0 + cos(M_PI * tv));
            const double a = ba[b];
            sh += a * ku * kv;
            sx += lam_half * a * sin(M_PI * tu) * kv;
            sy += lam_half * a * ku * sin(M_PI * tv);
        }
        h[p] = sh;
        dx[p] = sx;
        dy[p] = sy;
    }
}
