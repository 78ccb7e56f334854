"""Writes closed_forms.json: closed-form values (no oracle, no CUDA path)
used as pins of the oracle, each with its derivation and the paper passage
it rests on.  Run: python tests/golden/make_closed_forms.py"""
import json
import math
import os

G = 9.81


def main():
    out = {}
    # JONSWAP with gamma = 1 (Eqs. 2-4 with gamma^r -> 1):
    # m0 = alpha g^2/(5 wp^4) by the substitution t = 5/4 (wp/w)^4.
    U, F = 10.0, 100e3
    alpha = 0.076 * (U * U / (F * G)) ** 0.22
    wp = 22.0 * (G * G / (U * F)) ** (1.0 / 3.0)
    out["jonswap_gamma1"] = dict(
        cite="Sec. 3.1 Eqs. 2-4 (gamma = 1)", U10=U, fetch=F, alpha=alpha,
        omega_p=wp, m0=alpha * G * G / (5 * wp ** 4),
        derivation="m0 = int alpha g^2 w^-5 exp(-5/4 (wp/w)^4) dw = alpha g^2 / (5 wp^4)")
    # Phillips reading: S = alpha_P g^2 w^-5 exp(-(g/(U w))^4):
    # m0 = alpha_P U^4 / (4 g^2) = alpha_P L_w^2 / 4.
    U = 10.0
    Lw = U * U / G
    m0 = 0.0081 * Lw * Lw / 4
    out["phillips"] = dict(
        cite="Sec. 2.1 / 3.1 (Phillips named, no formula; reading alpha_P = 0.0081)",
        U10=U, m0=m0, Hs=4 * math.sqrt(m0),
        derivation="t = (g/(U w))^4 -> m0 = alpha_P g^2 / (4 (g/U)^4)")
    # Paper's default scene (Sec. 5.2): U10 = 5, FetchSize = 10000 -> Eq. 4.
    U, F = 5.0, 10000.0
    out["paper_default"] = dict(
        cite="Sec. 5.2 defaults (U10 = 5, FetchSize = 10000, N_omega = N_theta = 16, "
             "Res = 512^2, OceanSize_FFT = 500, OceanSize_WP = 100) with Eq. 4",
        U10=U, fetch=F, omega_p=22.0 * (G * G / (U * F)) ** (1.0 / 3.0),
        n_omega=16, n_theta=16, res=512, ocean_fft_m=500.0, ocean_wp_m=100.0)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
