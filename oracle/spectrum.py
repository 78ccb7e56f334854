"""Spectrum side of the oracle: JONSWAP / Phillips spectra, directional
spreading, dispersion, equal-energy frequency buckets and particle
amplitudes.  Float64 throughout; scipy's ``quad``, ``brentq`` and ``gammaln``
serve as library primitives.  TEST INFRASTRUCTURE ONLY (see package doc).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize, special

G = 9.81
JONSWAP, PHILLIPS = 0, 1
COS2S_MITSUYASU, COS2 = 0, 1
AMP_NORMALIZED, AMP_LITERAL = 0, 1
PHILLIPS_ALPHA = 0.0081

_QUAD = dict(epsabs=0.0, epsrel=2e-14, limit=400)


class Spectrum:
    """S(omega, theta) = S_1(omega) Dir(omega, theta) (Sec. 3.1, Eq. 1).

    JONSWAP (Eqs. 2-4):
        S_1 = alpha g^2 w^-5 exp(-5/4 (wp/w)^4) gamma^r,
        r = exp(-(w-wp)^2 / (2 sigma^2 wp^2)),
        alpha = 0.076 (U^2/(F g))^0.22, wp = 22 (g^2/(U F))^(1/3),
        gamma = 7.0 (g F / U^2)^-0.142 unless the description fixes gamma.
      reading: sigma = 0.07 for w <= wp, 0.09 above (the paper does not
      give sigma); F in metres.
    Phillips (named in Sec. 2.1 and 3.1, no formula given).
      reading: S_1 = alpha_P g^2 w^-5 exp(-(g/(U w))^4), alpha_P = 0.0081,
      i.e. the wavenumber form (alpha_P/2) k^-4 exp(-1/(k L_w)^2), L_w=U^2/g,
      through the deep-water Jacobian; its peak is wp = (4/5)^(1/4) g/U.
    Spreading:
      cos-2s (Eq. 5) with Mitsuyasu's s(w) = 16 (w/wp)^mu, mu = 5 for
      w <= wp, -2.5 above (Eq. 6);
      reading for "cos^2": one-sided (2/pi) cos^2(theta), |theta| < pi/2.
    """

    def __init__(self, cfg):
        self.kind = int(cfg["spectrum"])
        self.spreading = int(cfg["spreading"])
        self.U = float(cfg["wind_speed"])
        self.F = float(cfg["fetch"])
        self.depth = float(cfg["depth"])
        self.theta_w = float(cfg["wind_dir"])
        if self.kind == JONSWAP:
            U, F = self.U, self.F
            self.alpha = 0.076 * (U * U / (F * G)) ** 0.22
            self.wp = 22.0 * (G * G / (U * F)) ** (1.0 / 3.0)
            gam = float(cfg["gamma"])
            self.gamma = gam if gam > 0 else 7.0 * (G * F / (U * U)) ** (-0.142)
        elif self.kind == PHILLIPS:
            self.alpha = PHILLIPS_ALPHA
            self.w0 = G / self.U
            self.wp = (4.0 / 5.0) ** 0.25 * self.w0
            self.gamma = 1.0
        else:
            raise ValueError("unknown spectrum")

    # ---- 1-D spectrum ------------------------------------------------
    def S1(self, w):
        """Omnidirectional spectral density S_1(omega) [m^2 s]."""
        w = np.asarray(w, dtype=np.float64)
        out = np.zeros_like(w)
        pos = w > 0
        wv = w[pos]
        if self.kind == JONSWAP:
            sigma = np.where(wv <= self.wp, 0.07, 0.09)
            r = np.exp(-(wv - self.wp) ** 2 / (2.0 * sigma ** 2 * self.wp ** 2))
            out[pos] = (self.alpha * G * G * wv ** -5.0
                        * np.exp(-1.25 * (self.wp / wv) ** 4) * self.gamma ** r)
        else:
            out[pos] = (self.alpha * G * G * wv ** -5.0
                        * np.exp(-(self.w0 / wv) ** 4))
        return out

    def S1s(self, w):
        return float(self.S1(np.array([w]))[0])

    # ---- spreading -----------------------------------------------------
    def s_param(self, w):
        """Mitsuyasu spreading parameter, Eq. 6 (mu = 5 at w == wp)."""
        w = np.asarray(w, dtype=np.float64)
        mu = np.where(w <= self.wp, 5.0, -2.5)
        return 16.0 * (w / self.wp) ** mu

    def Dir(self, w, dth):
        """Directional spreading at relative angle dth in (-pi, pi]
        (w and dth broadcast)."""
        dth = np.asarray(dth, dtype=np.float64)
        if self.spreading == COS2S_MITSUYASU:
            s = self.s_param(w)
            norm = np.exp(special.gammaln(s + 1.0) - special.gammaln(s + 0.5)) \
                / (2.0 * math.sqrt(math.pi))
            c = np.abs(np.cos(dth / 2.0))
            return norm * c ** (2.0 * s)
        return np.where(np.abs(dth) < math.pi / 2.0,
                        (2.0 / math.pi) * np.cos(dth) ** 2, 0.0)

    def S2(self, w, dth):
        return self.S1s(w) * self.Dir(w, dth)

    # ---- integrals ---------------------------------------------------------
    def energy(self, a, b):
        """int_a^b S_1(w) dw (the spreading integrates to one)."""
        if b <= a:
            return 0.0
        if a < self.wp < b:
            return (integrate.quad(self.S1s, a, self.wp, **_QUAD)[0]
                    + integrate.quad(self.S1s, self.wp, b, **_QUAD)[0])
        return integrate.quad(self.S1s, a, b, **_QUAD)[0]

    def m0(self):
        """Zeroth moment over the full spectrum."""
        lo = integrate.quad(self.S1s, 0.0, self.wp, **_QUAD)[0]
        hi = integrate.quad(self.S1s, self.wp, np.inf, **_QUAD)[0]
        return lo + hi

    def Hs(self):
        return 4.0 * math.sqrt(self.m0())

    # ---- dispersion ---------------------------------------------------------
    def k_of_omega(self, w):
        """Wavenumber from omega.  Deep water: k = w^2/g (Sec. 3.2).
        reading (finite depth d > 0): w^2 = g k tanh(k d), Newton to 1e-15."""
        k = w * w / G
        if self.depth <= 0:
            return k
        d = self.depth
        k = k / math.sqrt(math.tanh(k * d))
        for _ in range(200):
            th = math.tanh(k * d)
            f = G * k * th - w * w
            fp = G * th + G * k * d * (1.0 - th * th)
            dk = f / fp
            k -= dk
            if abs(dk) <= 1e-16 * k:
                break
        return k

    def omega_of_k(self, k):
        k = np.asarray(k, dtype=np.float64)
        if self.depth <= 0:
            return np.sqrt(G * k)
        return np.sqrt(G * k * np.tanh(k * self.depth))

    def domega_dk(self, k):
        k = np.asarray(k, dtype=np.float64)
        w = self.omega_of_k(k)
        if self.depth <= 0:
            return np.where(k > 0, 0.5 * G / np.where(w > 0, w, 1.0), 0.0)
        d = self.depth
        th = np.tanh(k * d)
        return np.where(w > 0, (G * th + G * k * d * (1.0 - th * th))
                        / (2.0 * np.where(w > 0, w, 1.0)), 0.0)


class Buckets:
    """Frequency buckets of one patch (Sec. 3.3, Eqs. 7-8; Sec. 4.2).

    Edges: given, or an equal-energy partition of int S_1 over
    [lo*wp, hi*wp] (default [0.5, 2.5] wp) into n buckets by CDF inversion.
    reading: the representative frequency omega_i shared by a bucket is its
    energy median; E_i = int_bucket S_1 dw is the bucket's energy density.
    omega_i -> k_i by the dispersion relation, r_i = pi/k_i (half a
    wavelength; r = pi g / w^2 in deep water), c_i = omega_i / k_i.
    """

    def __init__(self, spec: Spectrum, n, edges=None, lo_mul=0.5, hi_mul=2.5):
        self.n = n
        if edges is not None:
            e = np.array(edges, dtype=np.float64)
            assert len(e) == n + 1
        else:
            lo, hi = lo_mul * spec.wp, hi_mul * spec.wp
            total = spec.energy(lo, hi)
            e = np.empty(n + 1)
            e[0], e[n] = lo, hi
            for i in range(1, n):
                target = total * i / n
                e[i] = optimize.brentq(lambda x: spec.energy(lo, x) - target,
                                       lo, hi, xtol=1e-15, rtol=1e-15,
                                       maxiter=400)
        self.edges = e
        self.E = np.array([spec.energy(e[i], e[i + 1]) for i in range(n)])
        om = np.empty(n)
        for i in range(n):
            half = 0.5 * self.E[i]
            a, b = e[i], e[i + 1]
            om[i] = optimize.brentq(lambda x: spec.energy(a, x) - half, a, b,
                                    xtol=1e-15, rtol=1e-15, maxiter=400)
        self.omega = om
        self.domega = np.diff(e)
        self.k = np.array([spec.k_of_omega(w) for w in om])
        self.r = math.pi / self.k
        self.c = om / self.k


def directions(theta_w, n_theta):
    """Direction grid (reading of Sec. 4.2 / Eq. 13): theta_j =
    theta_w - pi + (j + 1/2) dtheta, dtheta = 2 pi / N_theta.  Returns the
    absolute angles and the angles relative to the wind."""
    dth = 2.0 * math.pi / n_theta
    th = np.array([(theta_w - math.pi) + (j + 0.5) * dth for j in range(n_theta)])
    rel = np.array([-math.pi + (j + 0.5) * dth for j in range(n_theta)])
    return th, rel, dth


def amplitudes(spec: Spectrum, b: Buckets, n_theta, mode=AMP_NORMALIZED):
    """Particle amplitudes A_ij for bucket i, direction j.

    LITERAL: Eq. A, A = sqrt(2 S(w_i, theta_j) dw_i dtheta).
    NORMALIZED (default; reading): A_ij = sqrt(2 E_i Dir_ij / sum_j Dir_ij),
    so that sum_j A_ij^2 / 2 = E_i, the bucket integral of Eq. 8 taken exactly
    rather than by its midpoint rule S(w_i) dw_i.
    """
    _, rel, dth = directions(spec.theta_w, n_theta)
    A = np.zeros((b.n, n_theta))
    for i in range(b.n):
        D = spec.Dir(b.omega[i], rel)
        if mode == AMP_LITERAL:
            A[i] = np.sqrt(2.0 * spec.S1s(b.omega[i]) * D * b.domega[i] * dth)
        else:
            A[i] = np.sqrt(2.0 * b.E[i] * D / D.sum())
    return A
