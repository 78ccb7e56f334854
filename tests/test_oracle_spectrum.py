"""Pins of the oracle's spectrum side against closed forms and
normalisation conditions the paper fixes (Sec. 3.1 Eqs. 2-6, Sec. 3.2,
Sec. 3.3 Eqs. 7-17).  CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import spectrum as sp
from oracle.particles import PatchTables
from paper_2511_02852_gb300 import workloads as wl

G = 9.81
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_deep_dispersion_exact():
    spec = sp.Spectrum(wl.spectrum(depth=0.0))
    for w in [0.3, 0.88, 1.7, 3.1]:
        k = spec.k_of_omega(w)
        assert k == pytest.approx(w * w / G, rel=1e-15)
        r = math.pi / k
        assert r == pytest.approx(math.pi * G / (w * w), rel=1e-14)      # r = lambda/2
        assert w / k == pytest.approx(G / w, rel=1e-14)                  # c = g / w


def test_finite_depth_dispersion_residual_and_deep_limit():
    spec = sp.Spectrum(wl.spectrum(depth=50.0))
    for w in [0.2, 0.44, 0.88, 2.2, 4.0]:
        k = spec.k_of_omega(w)
        res = G * k * math.tanh(k * 50.0) - w * w
        assert abs(res) <= 1e-13 * w * w
    deep = sp.Spectrum(wl.spectrum(depth=1e5))
    for w in [0.5, 1.0, 2.0]:
        assert deep.k_of_omega(w) == pytest.approx(w * w / G, rel=1e-14)
    # omega(k) and its derivative invert k(omega)
    k = spec.k_of_omega(0.9)
    assert float(spec.omega_of_k(k)) == pytest.approx(0.9, rel=1e-14)
    h = 1e-6 * k
    fd = (float(spec.omega_of_k(k + h)) - float(spec.omega_of_k(k - h))) / (2 * h)
    assert float(spec.domega_dk(k)) == pytest.approx(fd, rel=1e-8)


@pytest.mark.parametrize("s_target,branch", [(0.1, 5), (0.5, 5), (1.0, 5), (4.0, -2.5),
                                             (16.0, 5), (0.3, -2.5)])
def test_cos2s_normalised(s_target, branch):
    """Eq. 5 integrates to one for s over Mitsuyasu's range (s <= 16)."""
    spec = sp.Spectrum(wl.spectrum())
    w = spec.wp * (s_target / 16.0) ** (1.0 / branch)
    assert float(spec.s_param(w)) == pytest.approx(s_target, rel=1e-12)
    val, _ = integrate.quad(lambda t: float(spec.Dir(w, t)), -math.pi, math.pi,
                            epsabs=0, epsrel=1e-13, limit=400)
    assert val == pytest.approx(1.0, abs=1e-11)


def test_cos2s_s1_closed_form():
    """s = 1: Gamma(2)/(2 sqrt(pi) Gamma(3/2)) cos^2(t/2) = (1 + cos t)/(2 pi)."""
    spec = sp.Spectrum(wl.spectrum())
    w = spec.wp * (1.0 / 16.0) ** (1 / 5.0)
    t = np.linspace(-3.1, 3.1, 41)
    assert np.allclose(spec.Dir(w, t), (1 + np.cos(t)) / (2 * math.pi), rtol=1e-13, atol=0)


def test_mitsuyasu_branch_at_peak():
    spec = sp.Spectrum(wl.spectrum())
    assert float(spec.s_param(spec.wp)) == pytest.approx(16.0, rel=1e-15)
    # mu = 5 below, -2.5 above (Eq. 6)
    assert float(spec.s_param(spec.wp * 0.5)) == pytest.approx(16 * 0.5 ** 5, rel=1e-13)
    assert float(spec.s_param(spec.wp * 2.0)) == pytest.approx(16 * 2.0 ** -2.5, rel=1e-13)


def test_cos2_one_sided_normalised():
    spec = sp.Spectrum(wl.spectrum(spreading=wl.COS2))
    val, _ = integrate.quad(lambda t: float(spec.Dir(1.0, t)), -math.pi, math.pi,
                            points=[-math.pi / 2, math.pi / 2], epsabs=0, epsrel=1e-13)
    assert val == pytest.approx(1.0, abs=1e-12)
    assert float(spec.Dir(1.0, 2.0)) == 0.0


def test_jonswap_gamma1_m0_closed_form():
    """gamma = 1: m0 = alpha g^2 / (5 wp^4) (substitution t = 5/4 (wp/w)^4)."""
    g = golden()["jonswap_gamma1"]
    spec = sp.Spectrum(wl.spectrum(wind_speed=g["U10"], fetch=g["fetch"], gamma=1.0))
    assert spec.wp == pytest.approx(g["omega_p"], rel=1e-12)
    assert spec.alpha == pytest.approx(g["alpha"], rel=1e-12)
    m0 = spec.alpha * G * G / (5 * spec.wp ** 4)
    assert spec.m0() == pytest.approx(m0, rel=1e-11)
    assert spec.m0() == pytest.approx(g["m0"], rel=1e-10)


def test_jonswap_gamma1_equal_energy_edges_closed_form():
    """gamma = 1: CDF(w) proportional to exp(-5/4 (wp/w)^4); equal-energy
    edges and energy medians in closed form (Sec. 3.3, Fig. 2b)."""
    spec = sp.Spectrum(wl.spectrum(wind_speed=12.0, fetch=40e3, gamma=1.0))
    n = 7
    b = sp.Buckets(spec, n)
    wp = spec.wp
    F = lambda w: math.exp(-1.25 * (wp / w) ** 4)
    Finv = lambda y: wp * (-0.8 * math.log(y)) ** -0.25
    lo, hi = 0.5 * wp, 2.5 * wp
    for i in range(n + 1):
        e = Finv(F(lo) + i / n * (F(hi) - F(lo)))
        assert b.edges[i] == pytest.approx(e, rel=1e-12)
    for i in range(n):
        m = Finv(0.5 * (F(b.edges[i]) + F(b.edges[i + 1])))
        assert b.omega[i] == pytest.approx(m, rel=1e-12)
    tot = spec.alpha * G * G / (5 * wp ** 4) * (F(hi) - F(lo))
    assert np.allclose(b.E, tot / n, rtol=1e-11)


def test_phillips_m0_closed_form():
    """Reading of the Phillips spectrum: m0 = alpha_P L_w^2 / 4, L_w = U^2/g."""
    g = golden()["phillips"]
    spec = sp.Spectrum(wl.spectrum(spectrum=wl.PHILLIPS, wind_speed=g["U10"]))
    Lw = g["U10"] ** 2 / G
    assert spec.m0() == pytest.approx(sp.PHILLIPS_ALPHA * Lw * Lw / 4, rel=1e-11)
    assert spec.Hs() == pytest.approx(g["Hs"], rel=1e-9)


def test_normalised_amplitudes_sum_to_bucket_energy():
    """sum_j A_ij^2 / 2 = E_i / inject_scale (Eq. A energy per component;
    Eq. 8 bucket energy taken as the exact bucket integral)."""
    sc = wl.small_jonswap()
    spec = sp.Spectrum(sc["spectrum"])
    T = PatchTables(spec, sc["spectrum"], sc["patches"][0], 1 / 60)
    lhs = (T.A ** 2).sum(axis=1) / 2
    assert np.allclose(lhs * T.scale, T.b.E, rtol=1e-13)


def test_literal_amplitude_is_eq_A():
    cfg = wl.spectrum(amp_mode=wl.AMP_LITERAL, n_buckets=5, n_theta=8)
    spec = sp.Spectrum(cfg)
    b = sp.Buckets(spec, 5)
    A = sp.amplitudes(spec, b, 8, sp.AMP_LITERAL)
    _, rel, dth = sp.directions(0.0, 8)
    for i in range(5):
        for j in range(8):
            S = spec.S1s(b.omega[i]) * float(spec.Dir(b.omega[i], rel[j]))
            assert A[i, j] == pytest.approx(math.sqrt(2 * S * b.domega[i] * dth), rel=1e-14)


def test_injection_count_reduces_to_eq15_17_in_deep_water():
    """n_s = 4 L_s dt c/(pi r^2) == 4 L_s dt w^3/(pi^3 g) (Eq. 17) in deep
    water; the two edge pairs of a square sum to Eq. 15."""
    sc = wl.tiny()
    spec = sp.Spectrum(sc["spectrum"])
    T = PatchTables(spec, sc["spectrum"], sc["patches"][0], 1 / 60)
    L = T.W * T.dx
    for i in range(T.nb):
        w = T.b.omega[i]
        eq17 = 4 * L * (1 / 60) * w ** 3 / (math.pi ** 3 * G)
        assert T.injection_rate(i, 0) == pytest.approx(eq17, rel=1e-13)
        eq15 = 8 * L * (1 / 60) * w ** 3 / (math.pi ** 3 * G)
        assert T.injection_rate(i, 0) + T.injection_rate(i, 1) == pytest.approx(eq15, rel=1e-13)


def test_group_energy_identity():
    """N_i E_group = E_square (Eqs. 11-15) with E_group = 1/8 pi r^2 sum_j A^2
    (Eq. 13, rho g dropped) and E_square = 2 L dt c E_i (Eq. 11)."""
    sc = wl.scaled(wl.small_jonswap(), width=160, height=160, inject_scale=1.0)
    spec = sp.Spectrum(sc["spectrum"])
    T = PatchTables(spec, sc["spectrum"], sc["patches"][0], 1 / 60)
    L = T.W * T.dx
    for i in range(T.nb):
        Ni = T.injection_rate(i, 0) + T.injection_rate(i, 1)
        Eg = 0.125 * math.pi * T.b.r[i] ** 2 * (T.A[i] ** 2).sum()
        Esq = 2 * L * (1 / 60) * T.b.c[i] * T.b.E[i]
        assert Ni * Eg == pytest.approx(Esq, rel=1e-12)


def test_wind_monotonicity_of_particle_rate():
    """Higher U10 -> lower wp -> fewer short-wave particles (Sec. 5.2)."""
    rates = []
    for U in [3.0, 5.0, 10.0, 15.0]:
        sc = wl.spectrum(wind_speed=U, fetch=10e3, n_buckets=16, n_theta=16)
        spec = sp.Spectrum(sc)
        T = PatchTables(spec, sc, wl.patch(width=400, height=400, cell=0.25), 1 / 60)
        rates.append(sum((T.injection_rate(i, 0) + T.injection_rate(i, 1)) * T.nth
                         for i in range(T.nb)))
    assert all(a > b for a, b in zip(rates, rates[1:]))


def test_paper_default_scene_constants():
    """Sec. 5.2 defaults U10 = 5, fetch 10000: Eq. 4 gives wp = 2.737 rad/s."""
    g = golden()["paper_default"]
    spec = sp.Spectrum(wl.spectrum(wind_speed=5.0, fetch=10000.0))
    assert spec.wp == pytest.approx(g["omega_p"], rel=1e-3)


def test_realistic_scene_peak_and_depth():
    """The realistic scene (U10 = 15 m/s, fetch 100 km, depth 50 m): Eq. 4's
    peak wp = 22 (g^2 / (U10 F))^(1/3) = 0.881 rad/s, where k d = 3.96 and
    tanh(k d) > 0.999 (depth changes the peak's phase speed by under 0.1%),
    while at the lowest bucket edge (0.5 wp) tanh(k d) = 0.83, so the
    finite-depth reading of O5 matters there."""
    cfg = wl.realistic()["spectrum"]
    spec = sp.Spectrum(cfg)
    wp = 22.0 * (G * G / (15.0 * 100e3)) ** (1.0 / 3.0)
    assert spec.wp == pytest.approx(wp, rel=1e-12)
    assert wp == pytest.approx(0.8807, abs=5e-4)
    kp = spec.k_of_omega(wp)
    assert kp * 50.0 == pytest.approx(3.96, abs=0.01)
    assert math.tanh(kp * 50.0) > 0.999
    deep_c = G / wp
    assert abs(wp / kp - deep_c) / deep_c < 1e-3
    k_lo = spec.k_of_omega(0.5 * wp)
    assert math.tanh(k_lo * 50.0) == pytest.approx(0.83, abs=0.005)


def test_literal_over_normalised_energy_is_the_midpoint_rule():
    """O8's two amplitude modes: LITERAL (Eq. A) carries S(w_i) dw_i per
    bucket (times the direction sum), NORMALIZED the exact bucket integral
    E_i.  Their per-bucket energy ratio is the midpoint rule's error on the
    bucket: on the interior buckets it shrinks as the buckets narrow (8, 16,
    64 equal-energy buckets), while on the lowest one, which spans the steep
    low-frequency flank from 0.5 wp, the value at the energy median
    overstates the integral more than twice at every count.  That is why
    NORMALIZED is the default.  Every bucket's deviation (the direction
    grid's sum taken out) stays within the bound Taylor's theorem gives about
    the representative frequency; the deviation is about half of it, and an
    E_i off by 2 % breaks it in most buckets at 16 and 64 buckets."""
    devs = []
    for n in (8, 16, 64):
        spec = sp.Spectrum(wl.spectrum(n_buckets=n, n_theta=16))
        b = sp.Buckets(spec, n)
        lit = sp.amplitudes(spec, b, 16, sp.AMP_LITERAL)
        nor = sp.amplitudes(spec, b, 16, sp.AMP_NORMALIZED)
        assert np.allclose((nor ** 2).sum(axis=1) / 2, b.E, rtol=1e-12)
        ratio = (lit ** 2).sum(axis=1) / (nor ** 2).sum(axis=1)
        print(f"[O8] {n} buckets: LITERAL/NORMALIZED energy {np.round(ratio, 4)}")
        assert ratio[0] > 2.0
        devs.append(np.abs(ratio[1:-1] - 1).max())
        # Bound from Taylor's theorem about the representative frequency
        # w_i (the bucket's energy median) on [a, b], mid = (a + b)/2:
        #   |S(w_i) dw - E_i| <= |S'(w_i)| dw |mid - w_i|
        #                        + 1/2 max|S''| ((b - w_i)^3 + (w_i - a)^3) / 3,
        # with S' and S'' by central differences of S on a fine grid of the
        # bucket.  The ratio is S(w_i) dw / E_i times the direction grid's
        # sum of Dir dtheta, taken out first.
        _, rel, dth = sp.directions(spec.theta_w, 16)
        for i in range(n):
            a, bb = b.edges[i], b.edges[i + 1]
            wi, dw = b.omega[i], b.domega[i]
            dsum = float((spec.Dir(wi, rel) * dth).sum())
            hd = 1e-4 * dw
            d1 = (spec.S1s(wi + hd) - spec.S1s(wi - hd)) / (2 * hd)
            g = np.linspace(a, bb, 201)
            d2 = max(abs((spec.S1s(x + hd) - 2 * spec.S1s(x) + spec.S1s(x - hd)) / (hd * hd)) for x in g)
            bound = abs(d1) * dw * abs(0.5 * (a + bb) - wi) + 0.5 * d2 * ((bb - wi) ** 3 + (wi - a) ** 3) / 3.0
            dev = abs(ratio[i] / dsum - 1.0)
            assert dev <= 1.05 * bound / b.E[i] + 1e-12, (n, i, dev, bound / b.E[i])
    assert devs[0] > devs[1] > devs[2]


# ---- Eq. 3: the JONSWAP peak enhancement gamma^r and its two sigma branches
def _gamma1_twin(cfg):
    """The same spectrum with gamma = 1: alpha and wp (Eqs. 2 and 4) do not
    depend on gamma, so the ratio S / S_{gamma=1} is the peak factor alone."""
    return sp.Spectrum(dict(cfg, gamma=1.0))


@pytest.mark.parametrize("gamma", [3.3, 0.0])   # given, and Eq. 4's (gamma <= 0)
def test_jonswap_peak_factor_sigma_branches(gamma):
    """Eq. 3: S(w) / S_{gamma=1}(w) = gamma^r, r = exp(-(w - wp)^2 / (2 sigma^2 wp^2)).
    At w = wp the ratio is gamma exactly; at w = wp (1 + d) it is
    gamma^exp(-d^2 / (2 sigma^2)) with sigma = 0.07 below the peak and 0.09
    above.  A swapped sigma, a dropped square or a wrong branch fails."""
    cfg = wl.spectrum(wind_speed=13.0, fetch=70e3, gamma=gamma)
    spec = sp.Spectrum(cfg)
    base = _gamma1_twin(cfg)
    assert spec.wp == base.wp and spec.alpha == base.alpha
    g = spec.gamma
    assert spec.S1s(spec.wp) / base.S1s(spec.wp) == pytest.approx(g, rel=1e-14)
    for d in (-0.3, -0.2, -0.1, -0.05, -0.01, 0.01, 0.05, 0.1, 0.2, 0.3):
        w = spec.wp * (1.0 + d)
        sigma = 0.07 if d < 0 else 0.09
        want = g ** math.exp(-d * d / (2.0 * sigma * sigma))
        assert spec.S1s(w) / base.S1s(w) == pytest.approx(want, rel=1e-13), d
    # the two flanks differ: the same |d| gives a larger factor above the peak
    lo = spec.S1s(spec.wp * 0.9) / base.S1s(spec.wp * 0.9)
    hi = spec.S1s(spec.wp * 1.1) / base.S1s(spec.wp * 1.1)
    assert hi > lo > 1.0


def test_jonswap_eq4_gamma_at_a_decade_of_dimensionless_fetch():
    """Eq. 4: gamma = 7.0 (g F / U^2)^-0.142.  With g F / U^2 = 10^4 that is
    7 * 10^-0.568 = 1.8927708548762 (30-digit decimal arithmetic); seen through the spectrum itself as the peak
    factor S(wp) / S_{gamma=1}(wp).  At 10^3 and 10^5 the factor follows the
    same power law (ratio 10^0.142 per decade)."""
    U = 10.0
    vals = []
    for dec in (3, 4, 5):
        F = 10.0 ** dec * U * U / G
        cfg = wl.spectrum(wind_speed=U, fetch=F, gamma=0.0)
        spec = sp.Spectrum(cfg)
        vals.append(spec.S1s(spec.wp) / _gamma1_twin(cfg).S1s(spec.wp))
    assert vals[1] == pytest.approx(1.8927708548762, rel=1e-12)
    assert vals[0] / vals[1] == pytest.approx(10.0 ** 0.142, rel=1e-12)
    assert vals[1] / vals[2] == pytest.approx(10.0 ** 0.142, rel=1e-12)


def test_literal_ratio_per_bucket_against_independent_quadrature():
    """Eq. A's per-bucket energy S(w_i) dw_i sum_j Dir_ij dtheta over the exact
    bucket integral E_i, checked bucket by bucket: E_i against a composite
    Simpson rule of its own (4000 panels per bucket, independent of the
    oracle's adaptive quadrature) and the LITERAL/NORMALIZED ratio against
    S_1(w_i) dw_i sum_j Dir_ij dtheta / E_i built from that Simpson value."""
    n = 64
    spec = sp.Spectrum(wl.spectrum(n_buckets=n, n_theta=16))
    b = sp.Buckets(spec, n)
    lit = sp.amplitudes(spec, b, 16, sp.AMP_LITERAL)
    nor = sp.amplitudes(spec, b, 16, sp.AMP_NORMALIZED)
    ratio = (lit ** 2).sum(axis=1) / (nor ** 2).sum(axis=1)
    dth = 2 * math.pi / 16
    _, rel, _ = sp.directions(spec.theta_w, 16)
    for i in range(n):
        a, c = b.edges[i], b.edges[i + 1]
        x = np.linspace(a, c, 4001)
        y = spec.S1(x)
        simpson = (c - a) / 12000.0 * (y[0] + y[-1] + 4 * y[1:-1:2].sum() + 2 * y[2:-1:2].sum())
        assert b.E[i] == pytest.approx(simpson, rel=1e-10)
        dsum = float(np.sum(spec.Dir(b.omega[i], rel))) * dth
        want = spec.S1s(b.omega[i]) * (c - a) * dsum / simpson
        assert ratio[i] == pytest.approx(want, rel=1e-9), i
