// Host-side float64 spectrum, bucket and fixed-point table construction of
// the hybrid ocean (Sec. 3.1-3.3 of the paper).  Runs at create / add_patch /
// dt change; the per-frame path only reads the tables it produces.
#pragma once
#include <stdint.h>

#include <vector>

namespace scwp {

constexpr double kG = 9.81;
constexpr int64_t kQ = 65536;
constexpr int64_t kHalf = 32768;
constexpr int kWakeDirs = 4096;

struct SpectrumModel {
    int kind = 0;        // 0 JONSWAP, 1 Phillips
    int spreading = 0;   // 0 cos-2s Mitsuyasu, 1 one-sided cos^2
    double U = 10, F = 1e5, depth = 0, theta_w = 0;
    double alpha = 0, wp = 1, gamma = 1, w0 = 1;

    void init(int kind, int spreading, double U, double F, double depth, double theta_w,
              double gamma_in);
    double S1(double w) const;                 // omnidirectional density
    double s_param(double w) const;            // Mitsuyasu s(w), Eq. 6
    double dir(double w, double dtheta) const; // spreading, relative angle
    double k_of_omega(double w) const;         // dispersion (deep / finite depth)
    double omega_of_k(double k) const;
    double domega_dk(double k) const;
    double energy(double a, double b) const;   // int_a^b S1
    double m0() const;                         // full-spectrum zeroth moment
};

struct PatchTablesHost {
    int nb = 0, nth = 0;
    std::vector<double> edges, E, omega, k, c, r;
    std::vector<double> amp;                   // [nb][nth] (already / sqrt(scale))
    std::vector<double> cos_j, sin_j;
    std::vector<int32_t> R;                    // [nb]
    std::vector<int32_t> vx, vy, qx, qy;       // [nb][nth]
    int wake_bucket = 0;
    std::vector<double> wake_cos, wake_sin;    // [4096]
    std::vector<int32_t> wvx, wvy, wqx, wqy;   // [4096]
    double dt = -1;
    double scale = 1;
    int W = 0, H = 0;
    double dx = 1;

    void build(const SpectrumModel& sm, int nb, const double* edges_or_null, double lo_mul,
               double hi_mul, int nth, int amp_mode, int W, int H, double dx, double scale,
               double obj_radius);
    void set_dt(double dt);                    // rebuilds vx, vy, wvx, wvy
    double injection_rate(int bucket, int s) const;  // groups per frame, edge pair s
};

// Box-Muller normals of the background's h0 draws and P(k); fills
// h0 (float2 interleaved, [N][N], FFT-natural order) and omega(k) (float64).
void build_background(const SpectrumModel& sm, int N, double L, uint64_t seed,
                      std::vector<float>& h0_interleaved, std::vector<double>& omega);

}  // namespace scwp
