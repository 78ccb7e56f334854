"""Pins of the oracle's FFT background (Sec. 4.1 "conventional spectral
evolution and inverse FFT"): brute-force DFTs, Hermitian symmetry, a single
plane wave, the spectrum's variance.  CPU only."""
import math

import numpy as np
import pytest

from oracle import background as bg
from oracle import spectrum as sp
from oracle.philox import philox4x32_10, philox_scalar
from paper_2511_02852_gb300 import workloads as wl


@pytest.mark.parametrize("N", [8, 16])
def test_inverse_dft_matches_brute_force(N):
    rng = np.random.default_rng(N)
    X = rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N))
    a = bg.inverse_dft2(X)
    b = bg.inverse_dft2_brute(X)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


def test_inverse_dft_rectangular_brute_and_transposed_index():
    """A single mode (mx, my) = (1, 0) varies along x only: catches a
    transposed index."""
    N = 8
    X = np.zeros((N, N), complex)
    X[0, 1] = 1.0
    f = bg.inverse_dft2(X)
    jx = np.arange(N)
    assert np.allclose(f, np.exp(2j * math.pi * jx / N)[None, :].repeat(N, 0), atol=1e-13)


def test_hermitian_background_is_real():
    sc = wl.small_jonswap()
    spec = sp.Spectrum(sc["spectrum"])
    N, L = 64, 300.0
    h0 = bg.h0_grid(spec, N, L, 11)
    for t in [0.0, 0.37, 12.5]:
        ht, dxt, dyt = bg.evolve(spec, h0, L, t, 0.8)
        neg = (-np.arange(N)) % N
        for X in (ht, dxt, dyt):
            assert np.allclose(X[neg][:, neg], np.conj(X), atol=1e-15)
        h, dx, dy, im = bg.background(spec, h0, L, t, 0.8)
        assert im <= 1e-12 * spec.Hs()


def test_nyquist_and_dc_are_zero():
    spec = sp.Spectrum(wl.spectrum())
    N = 16
    h0 = bg.h0_grid(spec, N, 200.0, 0)
    assert h0[0, 0] == 0 and np.all(h0[N // 2, :] == 0) and np.all(h0[:, N // 2] == 0)


def test_single_plane_wave_closed_form_and_phase_speed():
    """h0 = a e^{i phi} at one k, zero elsewhere: h = 2a cos(k.x + w t + phi),
    D = 2a lam k_hat sin(k.x + w t + phi); the crest moves along -k at
    w/|k| (the direction reading for h0).  With n = -k_hat the direction of
    travel and psi = -(k.x + w t + phi): h = 2a cos psi, D = 2a lam n sin psi,
    the same relation as a particle train (D = lam n A sin for h = A cos)."""
    spec = sp.Spectrum(wl.spectrum(depth=40.0))
    N, L, lam = 32, 160.0, 0.9
    h0 = np.zeros((N, N), complex)
    mx, my = 3, 2
    a, phi = 0.37, 0.6
    h0[my, mx] = a * np.exp(1j * phi)
    kx, ky = 2 * math.pi * mx / L, 2 * math.pi * my / L
    k = math.hypot(kx, ky)
    w = float(spec.omega_of_k(k))
    xs = np.arange(N) * L / N
    X, Y = np.meshgrid(xs, xs)
    for t in [0.0, 1.3, 7.7]:
        h, dx, dy, _ = bg.background(spec, h0, L, t, lam)
        arg = kx * X + ky * Y + w * t + phi
        assert np.allclose(h, 2 * a * np.cos(arg), atol=1e-12)
        assert np.allclose(dx, 2 * a * lam * (kx / k) * np.sin(arg), atol=1e-12)
        assert np.allclose(dy, 2 * a * lam * (ky / k) * np.sin(arg), atol=1e-12)
    # the crest (arg = 0 mod 2 pi) moves along -k_hat by (w/|k|) t
    t1 = 2.0
    x0 = np.array([10.0, 20.0])
    kv = np.array([kx, ky])
    x1 = x0 - (kv / k) * (w / k) * t1
    assert kv @ x0 + 0.0 == pytest.approx(kv @ x1 + w * t1, abs=1e-12)


def test_power_jacobian_variance():
    """2 sum_k P(k) approximates m0 (sum over the grid of the wavenumber
    spectrum; the full spectrum of a 1 km, 512^2 grid)."""
    sc = wl.realistic()
    spec = sp.Spectrum(sc["spectrum"])
    P = bg.power(spec, 512, 1000.0)
    assert 2 * P.sum() == pytest.approx(spec.m0(), rel=0.03)


def test_spectrum_direction_reading_downwind():
    """Energy of h0(k) sits where -k points downwind (theta_w = 0 -> k_x < 0)."""
    spec = sp.Spectrum(wl.spectrum(wind_speed=10.0, fetch=100e3))
    P = bg.power(spec, 64, 400.0)
    n = bg.signed_index(64)
    upwind_k = P[:, n < 0].sum()
    downwind_k = P[:, n > 0].sum()
    assert upwind_k > 10 * downwind_k


def test_philox_vectorised_equals_scalar_and_uniform():
    rng = np.random.default_rng(1)
    c = rng.integers(0, 2 ** 32, size=(4, 16), dtype=np.uint64)
    key = 0x0123456789ABCDEF
    v = philox4x32_10(c[0], c[1], c[2], c[3], key)
    for i in range(16):
        s = philox_scalar(int(c[0, i]), int(c[1, i]), int(c[2, i]), int(c[3, i]), key)
        assert tuple(int(x[i]) for x in v) == s
    n = np.arange(200000, dtype=np.uint64)
    out = philox4x32_10(n, 7, 3, 0, 5)
    for w in out:
        u = w.astype(np.float64) * 2.0 ** -32
        assert abs(u.mean() - 0.5) < 3e-3
        assert abs(u.var() - 1 / 12) < 2e-3


def test_philox_matches_triton_reference_implementation():
    """Cross-check against an independent Philox4x32-10 (Triton's
    tl.philox, run by its CPU interpreter)."""
    import os
    import subprocess
    import sys
    pytest.importorskip("triton")
    code = r'''
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import torch, triton, triton.language as tl
@triton.jit
def k(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
    offs = tl.arange(0, BLOCK)
    m = offs < n
    c0 = tl.load(c_ptr + offs * 4 + 0, mask=m).to(tl.uint32)
    c1 = tl.load(c_ptr + offs * 4 + 1, mask=m).to(tl.uint32)
    c2 = tl.load(c_ptr + offs * 4 + 2, mask=m).to(tl.uint32)
    c3 = tl.load(c_ptr + offs * 4 + 3, mask=m).to(tl.uint32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + offs * 4 + 0, a.to(tl.int64) & 0xffffffff, mask=m)
    tl.store(out_ptr + offs * 4 + 1, b.to(tl.int64) & 0xffffffff, mask=m)
    tl.store(out_ptr + offs * 4 + 2, c.to(tl.int64) & 0xffffffff, mask=m)
    tl.store(out_ptr + offs * 4 + 3, d.to(tl.int64) & 0xffffffff, mask=m)
ctr = json.loads(sys.argv[1]); seed = int(sys.argv[2])
c = torch.tensor(ctr, dtype=torch.int64).to(torch.int32)
out = torch.zeros(len(ctr) * 4, dtype=torch.int64)
k[(1,)](out, c.view(-1), seed, len(ctr), BLOCK=16)
print(json.dumps(out.view(-1, 4).tolist()))
'''
    import json
    ctrs = [[0, 0, 0, 0], [1, 2, 3, 4], [7, 0, 0xFFFFFFFF, 0], [600, 3, 15 | (1 << 16), 1234],
            [2 ** 31 - 1, 2 ** 31 - 5, 12345, 2 ** 31 - 3]]
    seed = 0x1234ABCD5678
    env = dict(os.environ, TRITON_INTERPRET="1")
    try:
        out = subprocess.run([sys.executable, "-c", code, json.dumps(ctrs), str(seed)],
                             capture_output=True, text=True, timeout=240, env=env)
    except subprocess.TimeoutExpired:
        pytest.skip("triton interpreter timed out")
    if out.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + out.stderr[-200:])
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for c, r in zip(ctrs, ref):
        got = philox_scalar(c[0] & 0xFFFFFFFF, c[1] & 0xFFFFFFFF, c[2] & 0xFFFFFFFF,
                            c[3] & 0xFFFFFFFF, seed)
        assert list(got) == [x & 0xFFFFFFFF for x in r]


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the published known-answer vectors of the
    Random123 distribution (Salmon et al., SC'11): counter, key -> output.
    This needs nothing but the oracle, so it cannot skip."""
    kat = [
        ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
         (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
        ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
         (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
        ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
         (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
    ]
    for ctr, (k0, k1), want in kat:
        key = k0 | (k1 << 32)                  # the oracle's key: k0 low word, k1 high word
        assert philox_scalar(*ctr, key) == want
        got = philox4x32_10(*[np.array([c], dtype=np.uint64) for c in ctr], key)
        assert tuple(int(x[0]) for x in got) == want


def test_h0_gaussian_draw_is_unit_complex_normal():
    """xi = (g1 + i g2)/sqrt 2 with g1, g2 standard normal (Box-Muller): over
    the 512^2 draws mean |xi|^2 = 1, mean Re^2 = mean Im^2 = 1/2, Re and Im
    uncorrelated, all within 5 standard errors; sqrt 2 Re and sqrt 2 Im pass
    a Kolmogorov-Smirnov test against N(0, 1) and |xi|^2 against Exp(1).  A
    missing 1/sqrt 2, a Box-Muller radius without its factor 2, or cos used
    for both parts each fail."""
    from scipy import stats
    N = 512
    xi = bg.gaussian_pairs(N, 0x5EED).ravel()
    n = xi.size
    a = np.abs(xi) ** 2
    assert abs(a.mean() - 1.0) < 5.0 / math.sqrt(n)           # var |xi|^2 = 1
    for part in (xi.real, xi.imag):
        assert abs((part ** 2).mean() - 0.5) < 5.0 * math.sqrt(0.5) / math.sqrt(n)   # var = 1/2
        assert abs(part.mean()) < 5.0 * math.sqrt(0.5 / n)
        assert stats.kstest(part * math.sqrt(2.0), "norm").pvalue > 1e-4
    assert abs(np.corrcoef(xi.real, xi.imag)[0, 1]) < 5.0 / math.sqrt(n)
    assert stats.kstest(a, "expon").pvalue > 1e-4


def test_h0_and_evolved_energy_against_the_power_spectrum():
    """sum |h0|^2 / sum P = 1 within 5 standard errors (the error of a sum of
    P-weighted Exp(1) draws is sqrt(sum P^2) / sum P); the evolved spectrum
    carries sum |h~(k, t)|^2 = 2 sum P in expectation (h~ holds the +k and -k
    draws), checked at three times on the realistic 512^2 grid; and the
    background's mean square equals sum |h~|^2 (Parseval for the
    unnormalised inverse)."""
    cfg = wl.realistic()["spectrum"]
    spec = sp.Spectrum(cfg)
    N, L = 512, 1000.0
    P = bg.power(spec, N, L)
    h0 = bg.h0_grid(spec, N, L, int(cfg["seed"]))
    se = math.sqrt((P ** 2).sum()) / P.sum()
    assert abs((np.abs(h0) ** 2).sum() / P.sum() - 1.0) < 5.0 * se
    for t in (0.0, 3.7, 41.0):
        ht, _, _ = bg.evolve(spec, h0, L, t, 1.0)
        e = (np.abs(ht) ** 2).sum()
        assert abs(e / (2.0 * P.sum()) - 1.0) < 5.0 * math.sqrt(2.0) * se
        h, _, _, _ = bg.background(spec, h0, L, t, 1.0)
        assert (h ** 2).mean() == pytest.approx(e, rel=1e-10)
