// Float64 host construction of the spectrum, buckets and fixed-point tables
// of the hybrid ocean.  Sec. 3.1 (Eqs. 1-6), Sec. 3.2 (dispersion, Eq. A),
// Sec. 3.3 (Eqs. 7-17), Sec. 4.2-4.3.
//
// Every float64 value that decides an integer (table rint, carry floor,
// wake angle) is computed by one fixed sequence of IEEE operations with the
// C library's cos/sin; this file must be compiled with -ffp-contract=off so
// no multiply-add is fused behind our back.
#include "host_spectrum.h"

#include <algorithm>
#include <cmath>
#include <complex>

#include "philox.h"

namespace scwp {

// ---------------------------------------------------------------------------
// Gauss-Legendre rule of order 20, nodes by Newton on P_20 (Legendre
// recurrence), and an adaptive bisection driver on top of it.
namespace {
constexpr int kGL = 20;
struct GLRule {
    double x[kGL], w[kGL];
    GLRule() {
        const int n = kGL;
        for (int i = 0; i < n; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            double dp = 1.0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = z;
                for (int j = 2; j <= n; ++j) {
                    const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-17) break;
            }
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};
const GLRule& gl() {
    static GLRule rule;
    return rule;
}

template <class F>
double gl20(const F& f, double a, double b) {
    const GLRule& g = gl();
    const double m = 0.5 * (a + b), h = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < kGL; ++i) s += g.w[i] * f(m + h * g.x[i]);
    return s * h;
}

template <class F>
double adapt(const F& f, double a, double b, double whole, double scale, int depth) {
    const double m = 0.5 * (a + b);
    const double l = gl20(f, a, m), r = gl20(f, m, b);
    const double both = l + r;
    if (depth >= 48 || std::fabs(both - whole) <= 1e-15 * std::fabs(both) + 1e-18 * scale)
        return both;
    return adapt(f, a, m, l, scale, depth + 1) + adapt(f, m, b, r, scale, depth + 1);
}

template <class F>
double integrate(const F& f, double a, double b, double scale) {
    if (!(b > a)) return 0.0;
    return adapt(f, a, b, gl20(f, a, b), scale, 0);
}
}  // namespace

// ---------------------------------------------------------------------------
void SpectrumModel::init(int kind_, int spreading_, double U_, double F_, double depth_,
                         double theta_w_, double gamma_in) {
    kind = kind_;
    spreading = spreading_;
    U = U_;
    F = F_;
    depth = depth_;
    theta_w = theta_w_;
    if (kind == 0) {  // JONSWAP, Eq. 4
        alpha = 0.076 * std::pow(U * U / (F * kG), 0.22);
        wp = 22.0 * std::pow(kG * kG / (U * F), 1.0 / 3.0);
        gamma = gamma_in > 0 ? gamma_in : 7.0 * std::pow(kG * F / (U * U), -0.142);
    } else {          // Phillips reading: alpha_P = 0.0081, peak (4/5)^(1/4) g / U
        alpha = 0.0081;
        w0 = kG / U;
        wp = std::pow(4.0 / 5.0, 0.25) * w0;
        gamma = 1.0;
    }
}

double SpectrumModel::S1(double w) const {
    if (!(w > 0)) return 0.0;
    if (kind == 0) {
        const double sigma = w <= wp ? 0.07 : 0.09;
        const double d = w - wp;
        const double r = std::exp(-(d * d) / (2.0 * sigma * sigma * wp * wp));
        const double q = wp / w;
        return alpha * kG * kG * std::pow(w, -5.0) * std::exp(-1.25 * q * q * q * q) *
               std::pow(gamma, r);
    }
    const double q = w0 / w;
    return alpha * kG * kG * std::pow(w, -5.0) * std::exp(-(q * q * q * q));
}

double SpectrumModel::s_param(double w) const {
    const double mu = w <= wp ? 5.0 : -2.5;
    return 16.0 * std::pow(w / wp, mu);
}

double SpectrumModel::dir(double w, double dth) const {
    if (spreading == 0) {
        const double s = s_param(w);
        const double norm =
            std::exp(std::lgamma(s + 1.0) - std::lgamma(s + 0.5)) / (2.0 * std::sqrt(M_PI));
        return norm * std::pow(std::fabs(std::cos(0.5 * dth)), 2.0 * s);
    }
    if (std::fabs(dth) < 0.5 * M_PI) {
        const double c = std::cos(dth);
        return (2.0 / M_PI) * c * c;
    }
    return 0.0;
}

double SpectrumModel::k_of_omega(double w) const {
    double k = w * w / kG;
    if (depth <= 0) return k;
    // Newton on g k tanh(k d) - w^2, from the deep-water guess; the function
    // is increasing and concave in k, so the iteration is monotone.
    for (int it = 0; it < 200; ++it) {
        const double th = std::tanh(k * depth);
        const double f = kG * k * th - w * w;
        const double fp = kG * th + kG * k * depth * (1.0 - th * th);
        const double dk = f / fp;
        k -= dk;
        if (std::fabs(dk) <= 1e-16 * k) break;
    }
    return k;
}

double SpectrumModel::omega_of_k(double k) const {
    if (depth <= 0) return std::sqrt(kG * k);
    return std::sqrt(kG * k * std::tanh(k * depth));
}

double SpectrumModel::domega_dk(double k) const {
    const double w = omega_of_k(k);
    if (!(w > 0)) return 0.0;
    if (depth <= 0) return 0.5 * kG / w;
    const double th = std::tanh(k * depth);
    return (kG * th + kG * k * depth * (1.0 - th * th)) / (2.0 * w);
}

double SpectrumModel::energy(double a, double b) const {
    auto f = [this](double w) { return S1(w); };
    const double scale = std::max(1e-300, S1(wp) * wp);
    if (a < wp && wp < b) return integrate(f, a, wp, scale) + integrate(f, wp, b, scale);
    return integrate(f, a, b, scale);
}

double SpectrumModel::m0() const {
    auto f = [this](double w) { return S1(w); };
    const double scale = std::max(1e-300, S1(wp) * wp);
    const double lo = integrate(f, 0.0, wp, scale);
    // tail: w = wp / u, dw = wp / u^2 du, u in (0, 1]
    auto g = [this](double u) { return u > 0 ? S1(wp / u) * wp / (u * u) : 0.0; };
    return lo + integrate(g, 0.0, 1.0, scale);
}

// ---------------------------------------------------------------------------
namespace {
// smallest x in [a, b] with F(x) >= target for increasing F, by bisection
// down to adjacent doubles.
template <class F>
double bisect(const F& f, double a, double b, double target) {
    for (int it = 0; it < 400; ++it) {
        const double m = 0.5 * (a + b);
        if (m <= a || m >= b) break;
        if (f(m) < target) a = m; else b = m;
    }
    return 0.5 * (a + b);
}

int32_t rint32(double v) { return (int32_t)std::llrint(v); }
}  // namespace

void PatchTablesHost::build(const SpectrumModel& sm, int nb_, const double* edges_in,
                            double lo_mul, double hi_mul, int nth_, int amp_mode, int W_, int H_,
                            double dx_, double scale_, double obj_radius) {
    nb = nb_;
    nth = nth_;
    W = W_;
    H = H_;
    dx = dx_;
    scale = scale_ > 0 ? scale_ : 1.0;
    edges.assign(nb + 1, 0.0);
    if (edges_in) {
        for (int i = 0; i <= nb; ++i) edges[i] = edges_in[i];
    } else {
        const double lo = lo_mul * sm.wp, hi = hi_mul * sm.wp;
        const double total = sm.energy(lo, hi);
        edges[0] = lo;
        edges[nb] = hi;
        for (int i = 1; i < nb; ++i) {
            const double target = total * i / nb;
            edges[i] = bisect([&](double x) { return sm.energy(lo, x); }, lo, hi, target);
        }
    }
    E.assign(nb, 0.0);
    omega.assign(nb, 0.0);
    k.assign(nb, 0.0);
    c.assign(nb, 0.0);
    r.assign(nb, 0.0);
    for (int i = 0; i < nb; ++i) {
        const double a = edges[i], b = edges[i + 1];
        E[i] = sm.energy(a, b);
        const double half = 0.5 * E[i];
        omega[i] = bisect([&](double x) { return sm.energy(a, x); }, a, b, half);
        k[i] = sm.k_of_omega(omega[i]);
        r[i] = M_PI / k[i];
        c[i] = omega[i] / k[i];
    }
    // directions theta_j = theta_w - pi + (j + 1/2) dtheta
    const double dth = 2.0 * M_PI / nth;
    cos_j.assign(nth, 0.0);
    sin_j.assign(nth, 0.0);
    std::vector<double> rel(nth);
    for (int j = 0; j < nth; ++j) {
        const double th = (sm.theta_w - M_PI) + (j + 0.5) * dth;
        cos_j[j] = std::cos(th);
        sin_j[j] = std::sin(th);
        rel[j] = -M_PI + (j + 0.5) * dth;
    }
    amp.assign((size_t)nb * nth, 0.0);
    const double inv_sqrt_scale = 1.0 / std::sqrt(scale);
    for (int i = 0; i < nb; ++i) {
        double dsum = 0.0;
        std::vector<double> D(nth);
        for (int j = 0; j < nth; ++j) {
            D[j] = sm.dir(omega[i], rel[j]);
            dsum += D[j];
        }
        for (int j = 0; j < nth; ++j) {
            double A;
            if (amp_mode == 1)  // Eq. A
                A = std::sqrt(2.0 * sm.S1(omega[i]) * D[j] * (edges[i + 1] - edges[i]) * dth);
            else                // normalised: sum_j A^2 / 2 = E_i
                A = dsum > 0 ? std::sqrt(2.0 * E[i] * D[j] / dsum) : 0.0;
            amp[(size_t)i * nth + j] = A * inv_sqrt_scale;
        }
    }
    R.assign(nb, 0);
    qx.assign((size_t)nb * nth, 0);
    qy.assign((size_t)nb * nth, 0);
    for (int i = 0; i < nb; ++i) {
        R[i] = rint32(r[i] / dx * kQ);
        for (int j = 0; j < nth; ++j) {
            qx[(size_t)i * nth + j] = rint32(r[i] * cos_j[j] / dx * kQ);
            qy[(size_t)i * nth + j] = rint32(r[i] * sin_j[j] / dx * kQ);
        }
    }
    // wake bucket: radius closest to the object's (first on ties)
    wake_bucket = 0;
    double best = std::fabs(r[0] - obj_radius);
    for (int i = 1; i < nb; ++i) {
        const double d = std::fabs(r[i] - obj_radius);
        if (d < best) {
            best = d;
            wake_bucket = i;
        }
    }
    const double dpsi = 2.0 * M_PI / kWakeDirs;
    wake_cos.assign(kWakeDirs, 0.0);
    wake_sin.assign(kWakeDirs, 0.0);
    wqx.assign(kWakeDirs, 0);
    wqy.assign(kWakeDirs, 0);
    const double rw = r[wake_bucket];
    for (int a = 0; a < kWakeDirs; ++a) {
        wake_cos[a] = std::cos(a * dpsi);
        wake_sin[a] = std::sin(a * dpsi);
        wqx[a] = rint32(rw * wake_cos[a] / dx * kQ);
        wqy[a] = rint32(rw * wake_sin[a] / dx * kQ);
    }
    dt = -1;
}

void PatchTablesHost::set_dt(double dt_) {
    if (dt_ == dt) return;
    dt = dt_;
    vx.assign((size_t)nb * nth, 0);
    vy.assign((size_t)nb * nth, 0);
    for (int i = 0; i < nb; ++i)
        for (int j = 0; j < nth; ++j) {
            vx[(size_t)i * nth + j] = rint32(c[i] * dt * cos_j[j] / dx * kQ);
            vy[(size_t)i * nth + j] = rint32(c[i] * dt * sin_j[j] / dx * kQ);
        }
    wvx.assign(kWakeDirs, 0);
    wvy.assign(kWakeDirs, 0);
    const double cw = c[wake_bucket];
    for (int a = 0; a < kWakeDirs; ++a) {
        wvx[a] = rint32(cw * dt * wake_cos[a] / dx * kQ);
        wvy[a] = rint32(cw * dt * wake_sin[a] / dx * kQ);
    }
}

double PatchTablesHost::injection_rate(int i, int s) const {
    // general form of Eqs. 15-17: n_s = 4 L_s dt c / (pi r^2) (deep water:
    // 4 L_s dt w^3 / (pi^3 g)), L_s = height (s = 0, x-edges) or width.
    const double Ls = (double)(s == 0 ? H : W) * dx;
    const double ci = c[i], ri = r[i];
    return 4.0 * Ls * dt * ci / (M_PI * ri * ri) * scale;
}

// ---------------------------------------------------------------------------
void build_background(const SpectrumModel& sm, int N, double L, uint64_t seed,
                      std::vector<float>& h0, std::vector<double>& omega) {
    h0.assign((size_t)2 * N * N, 0.0f);
    omega.assign((size_t)N * N, 0.0);
    const double dk = 2.0 * M_PI / L;
    for (int my = 0; my < N; ++my) {
        const int ny = my < N / 2 ? my : my - N;
        for (int mx = 0; mx < N; ++mx) {
            const int nx = mx < N / 2 ? mx : mx - N;
            const double kx = dk * nx, ky = dk * ny;
            const double k = std::sqrt(kx * kx + ky * ky);
            const size_t idx = (size_t)my * N + mx;
            if (k <= 0) continue;
            omega[idx] = sm.omega_of_k(k);
            if (mx == N / 2 || my == N / 2) continue;
            // h0(k) carries waves travelling along -k (reading of the
            // evolution's sign convention): spectrum at angle theta_{-k}.
            double th = std::atan2(-ky, -kx) - sm.theta_w;
            th = std::remainder(th, 2.0 * M_PI);
            const double w = omega[idx];
            const double P = 0.5 * sm.S1(w) * sm.dir(w, th) * sm.domega_dk(k) / k * dk * dk;
            const U4 u = philox4x32_10((uint32_t)mx, (uint32_t)my, 0xFFFFFFFFu, 0u, seed);
            const double u1 = ((double)u.x + 1.0) * 0x1p-32;
            const double u2 = (double)u.y * 0x1p-32;
            const double rad = std::sqrt(-2.0 * std::log(u1));
            const double g1 = rad * std::cos(2.0 * M_PI * u2), g2 = rad * std::sin(2.0 * M_PI * u2);
            const double s = std::sqrt(P) / std::sqrt(2.0);
            h0[2 * idx] = (float)(g1 * s);
            h0[2 * idx + 1] = (float)(g2 * s);
        }
    }
}

}  // namespace scwp
