"""FFT background of the oracle (Sec. 3.1 / Sec. 4.1: the conventional
spectral evolution plus inverse FFT of Tessendorf, the paper's ref. for the
"well-established" FFT update).  Float64.  TEST INFRASTRUCTURE ONLY.

Grid: N x N, side L; wavenumbers k_n = 2 pi n / L, n in [-N/2, N/2), stored
in FFT-natural order (index m = n mod N), arrays indexed [m_y, m_x].
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x32_10
from .spectrum import Spectrum

H0_STREAM = 0xFFFFFFFF   # counter word c2 of the h0 draws


def signed_index(N):
    m = np.arange(N)
    return np.where(m < N // 2, m, m - N)


def wavevectors(N, L):
    n = signed_index(N)
    kx = 2.0 * math.pi * n[None, :] / L * np.ones((N, 1))
    ky = 2.0 * math.pi * n[:, None] / L * np.ones((1, N))
    return kx, ky


def wrap_angle(a):
    return np.mod(a + math.pi, 2.0 * math.pi) - math.pi


def gaussian_pairs(N, seed):
    """xi = (g1 + i g2)/sqrt(2) per grid point.  reading: g1, g2 by
    Box-Muller from Philox4x32-10 words x0, x1 at counter (m_x, m_y,
    0xFFFFFFFF, 0), key = seed; U1 = (x0+1) 2^-32 in (0,1], U2 = x1 2^-32."""
    my, mx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    x0, x1, _, _ = philox4x32_10(mx, my, H0_STREAM, 0, seed)
    u1 = (x0.astype(np.float64) + 1.0) * 2.0 ** -32
    u2 = x1.astype(np.float64) * 2.0 ** -32
    rad = np.sqrt(-2.0 * np.log(u1))
    g1 = rad * np.cos(2.0 * math.pi * u2)
    g2 = rad * np.sin(2.0 * math.pi * u2)
    return (g1 + 1j * g2) / math.sqrt(2.0)


def power(spec: Spectrum, N, L):
    """P(k) = 1/2 Psi(-k) (2 pi / L)^2 with the wavenumber spectrum
    Psi(k) = S(omega(k), theta_k - theta_w) omega'(k) / k (change of
    variables from (omega, theta) to (k_x, k_y)).
    reading (direction): with h~(k,t) = h0(k) e^{iwt} + conj(h0(-k)) e^{-iwt}
    and the inverse transform sum_k h~ e^{ik.x}, the component h0(k) moves
    along -k; h0(k) therefore carries the spectral density of waves
    travelling along -k, so that the background and the particles (which
    move along theta_j) propagate the same way.
    reading: P = 0 at k = 0 and on the Nyquist row and column, so the
    inverse transforms are real."""
    kx, ky = wavevectors(N, L)
    k = np.hypot(kx, ky)
    P = np.zeros((N, N))
    w = spec.omega_of_k(k)
    dw = spec.domega_dk(k)
    th = wrap_angle(np.arctan2(-ky, -kx) - spec.theta_w)
    pos = k > 0
    wp_ = w[pos]
    D = spec.Dir(wp_, th[pos])
    P[pos] = 0.5 * spec.S1(wp_) * D * dw[pos] / k[pos] * (2.0 * math.pi / L) ** 2
    P[N // 2, :] = 0.0
    P[:, N // 2] = 0.0
    return P


def h0_grid(spec: Spectrum, N, L, seed):
    """h0(k) = xi sqrt(P(k))."""
    return gaussian_pairs(N, seed) * np.sqrt(power(spec, N, L))


def evolve(spec: Spectrum, h0, L, t, lam):
    """h~(k,t) = h0(k) e^{i w t} + conj(h0(-k)) e^{-i w t};
    D~ = -i lam (k/|k|) h~ (choppy displacement)."""
    N = h0.shape[0]
    kx, ky = wavevectors(N, L)
    k = np.hypot(kx, ky)
    w = spec.omega_of_k(k)
    neg = (-np.arange(N)) % N
    h0m = h0[neg][:, neg]
    ht = h0 * np.exp(1j * w * t) + np.conj(h0m) * np.exp(-1j * w * t)
    ks = np.where(k > 0, k, 1.0)
    dxt = -1j * lam * (kx / ks) * ht
    dyt = -1j * lam * (ky / ks) * ht
    dxt[k == 0] = 0.0
    dyt[k == 0] = 0.0
    return ht, dxt, dyt


def inverse_dft2(X):
    """Unnormalised inverse 2-D DFT, f[jy, jx] = sum_m X[my, mx]
    e^{2 pi i (mx jx + my jy)/N} (numpy's ifft2 as the library primitive)."""
    N = X.shape[0]
    return np.fft.ifft2(X) * (N * N)


def inverse_dft2_brute(X):
    """Brute-force O(N^4) inverse 2-D DFT (pins ``inverse_dft2``)."""
    N0, N1 = X.shape
    out = np.zeros((N0, N1), dtype=np.complex128)
    for jy in range(N0):
        for jx in range(N1):
            acc = 0j
            for my in range(N0):
                for mx in range(N1):
                    acc += X[my, mx] * np.exp(2j * math.pi * (mx * jx / N1 + my * jy / N0))
            out[jy, jx] = acc
    return out


def background(spec: Spectrum, h0, L, t, lam):
    """Real background maps (h, Dx, Dy) at x_j = j L / N, indexed [jy, jx].
    Returns the imaginary residues too (zero up to rounding by Hermitian
    symmetry)."""
    ht, dxt, dyt = evolve(spec, h0, L, t, lam)
    h = inverse_dft2(ht)
    dx = inverse_dft2(dxt)
    dy = inverse_dft2(dyt)
    im = max(np.abs(h.imag).max(), np.abs(dx.imag).max(), np.abs(dy.imag).max())
    return h.real.copy(), dx.real.copy(), dy.real.copy(), im
