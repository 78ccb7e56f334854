"""The summed-area form of the per-bucket kernel sums of Sec. 4.2 (the
default synthesis), restated in numpy and checked against the oracle's
direct sums.  CPU only.  This pins the identity that the GPU kernel is
built on, not the kernel itself (its parity is in test_gpu_sat.py).

With a = pi X / R, b = pi Y / R and a bump at (x, y):

    1 + cos(pi (X - x) / R) = u(X) . p(x),   u = (1, cos a, -sin a),
                                             p = (1, cos(pi x / R), -sin(pi x / R)),
    sin(pi (X - x) / R)     = u'(X) . p(x),  u' = (0, sin a, cos a),

and v, v', q likewise in y.  On a tile, with [box_b] the indicator of the
texel centres strictly inside bump b's square support,

    h  = 1/4     sum_ij u_i(X)  v_j(Y)  S_ij(X, Y)
    Dx = lam/4   sum_ij u'_i(X) v_j(Y)  S_ij(X, Y)
    Dy = lam/4   sum_ij u_i(X)  v'_j(Y) S_ij(X, Y)
    S_ij(X, Y) = sum_b A_b p_i(x_b) q_j(y_b) [box_b](X, Y),

and each S_ij is the 2-D prefix sum of a difference array that holds
+-A p_i q_j at the four corners of every box (corners past the tile's last
row or column are dropped).  With the corner weights quantised to
integers, prefix sums taken modulo 2^32 are exact whenever the final sums
fit in int32, so the result then carries only the quantisation error."""
import math

import numpy as np

from oracle.particles import HALF, Q
from oracle.synth import synth_maps_numpy

T = 64


def support_span(c, R):
    """Texel indices [lo, hi] whose centres lie strictly inside (c - R, c + R)
    (Q16.16 integers; empty when hi < lo)."""
    lo = (c - R - HALF) // Q + 1
    hi = (c + R - HALF - 1) // Q
    return lo, hi


def factors(t, R):
    """(u, u') of texel indices t for half-width R: shape [3, len(t)] each."""
    a = math.pi * (np.asarray(t, dtype=np.int64) * Q + HALF) / R
    u = np.stack([np.ones_like(a), np.cos(a), -np.sin(a)])
    du = np.stack([np.zeros_like(a), np.sin(a), np.cos(a)])
    return u, du


def corner_planes(bumps, tx0, ty0, W, H, scale=None):
    """The nine difference arrays of one tile [9, T, T] (float64 weights,
    or int64 weights quantised by `scale`), and the bumps that reached it."""
    E = np.zeros((3, 3, T, T), dtype=np.float64 if scale is None else np.int64)
    used = 0
    for X, Y, R, A in zip(bumps["X"], bumps["Y"], bumps["R"], bumps["amp"]):
        X, Y, R = int(X), int(Y), int(R)
        xl, xh = support_span(X, R)
        yl, yh = support_span(Y, R)
        # the box inside the patch, then inside the tile ([lo, hi) in tile coordinates)
        xl, xh = max(xl, 0, tx0), min(xh, W - 1, tx0 + T - 1)
        yl, yh = max(yl, 0, ty0), min(yh, H - 1, ty0 + T - 1)
        if xh < xl or yh < yl:
            continue
        used += 1
        al, ah = xl - tx0, xh + 1 - tx0
        gl, gh = yl - ty0, yh + 1 - ty0
        px = (1.0, math.cos(math.pi * X / R), -math.sin(math.pi * X / R))
        py = (1.0, math.cos(math.pi * Y / R), -math.sin(math.pi * Y / R))
        for i in range(3):
            for j in range(3):
                w = A * px[i] * py[j]
                if scale is not None:
                    w = int(round(w * scale))
                E[i, j, gl, al] += w
                if ah < T:
                    E[i, j, gl, ah] -= w
                if gh < T:
                    E[i, j, gh, al] -= w
                if ah < T and gh < T:
                    E[i, j, gh, ah] += w
    return E, used


def contract(S, tx0, ty0, R, lam):
    """h, Dx, Dy of one tile from its nine summed-area planes [3, 3, T, T]."""
    u, du = factors(np.arange(tx0, tx0 + T), R)
    v, dv = factors(np.arange(ty0, ty0 + T), R)
    h = 0.25 * np.einsum("ix,jy,ijyx->yx", u, v, S)
    dx = 0.25 * lam * np.einsum("ix,jy,ijyx->yx", du, v, S)
    dy = 0.25 * lam * np.einsum("ix,jy,ijyx->yx", u, dv, S)
    return h, dx, dy


def bucket_bumps(rng, n, R_cells, W, H, amp=1.0):
    """n bumps of one half-width, centres spread over the patch grown by the
    support (so that boxes are clipped by the patch and by the tiles)."""
    R = int(round(R_cells * Q))
    X = rng.integers(-R, W * Q + R, n)
    Y = rng.integers(-R, H * Q + R, n)
    A = amp * rng.uniform(-1.0, 1.0, n)
    return {"X": X, "Y": Y, "R": np.full(n, R), "amp": A}


def test_summed_area_form_equals_direct_sums():
    """FP64: the 3 x 3 contraction of the prefix-summed corner planes equals
    the oracle's bump-by-bump sums on every texel of ragged 64 x 64 tiles,
    for small radii (boxes inside a tile), large ones (boxes covering and
    clipped by tiles) and a fractional radius."""
    rng = np.random.default_rng(11)
    W, H, lam = 150, 131, 0.8
    for R_cells, n in ((2.6, 120), (9.25, 60), (41.0, 25), (97.5, 10)):
        bumps = bucket_bumps(rng, n, R_cells, W, H)
        ref = synth_maps_numpy(W, H, bumps, lam)
        R = int(bumps["R"][0])
        scale_ref = float(np.abs(bumps["amp"]).sum())
        for ty0 in range(0, H, T):
            for tx0 in range(0, W, T):
                E, _ = corner_planes(bumps, tx0, ty0, W, H)
                S = E.cumsum(axis=2).cumsum(axis=3)
                got = contract(S, tx0, ty0, R, lam)
                ys, xs = slice(ty0, min(ty0 + T, H)), slice(tx0, min(tx0 + T, W))
                ny, nx = ys.stop - ys.start, xs.stop - xs.start
                for g, r in zip(got, ref):
                    err = np.abs(g[:ny, :nx] - r[ys, xs]).max()
                    assert err <= 1e-11 * scale_ref, (R_cells, tx0, ty0, err)


def test_one_bump_box_matches_its_support_exactly():
    """A single bump: S_00 is the indicator of its support box times A, so
    the planes vanish outside the support and the h plane is the product
    kernel inside it."""
    W = H = 64
    R = int(5.5 * Q)
    bumps = {"X": np.array([20 * Q + 7000]), "Y": np.array([33 * Q - 900]), "R": np.array([R]),
             "amp": np.array([0.75])}
    E, used = corner_planes(bumps, 0, 0, W, H)
    assert used == 1
    S = E.cumsum(axis=2).cumsum(axis=3)
    xl, xh = support_span(int(bumps["X"][0]), R)
    yl, yh = support_span(int(bumps["Y"][0]), R)
    box = np.zeros((H, W), dtype=bool)
    box[yl:yh + 1, xl:xh + 1] = True
    assert np.array_equal(S[0, 0] != 0, box)
    assert np.allclose(S[0, 0][box], 0.75)
    h, _, _ = contract(S, 0, 0, R, 1.0)
    ref, _, _ = synth_maps_numpy(W, H, bumps, 1.0)
    assert np.abs(h - ref).max() < 1e-14


def test_integer_corner_events_wrap_exactly_and_bound_the_error():
    """Quantised corner weights (scale = 2^30 / (1.001 n amax), so that no
    final sum leaves int32): prefix sums taken modulo 2^32 equal the exact
    integer prefix sums, and the maps differ from the direct sums by at
    most the quantisation bound (n half-steps per plane entry)."""
    rng = np.random.default_rng(5)
    W, H, lam = 128, 128, 1.0
    bumps = bucket_bumps(rng, 400, 23.0, W, H, amp=0.3)
    amax = float(np.abs(bumps["amp"]).max())
    R = int(bumps["R"][0])
    ref = synth_maps_numpy(W, H, bumps, lam)
    for ty0 in (0, 64):
        for tx0 in (0, 64):
            n = corner_planes(bumps, tx0, ty0, W, H)[1]
            scale = 2.0 ** 30 / (1.001 * n * amax)
            Ei, _ = corner_planes(bumps, tx0, ty0, W, H, scale)
            exact = Ei.cumsum(axis=2).cumsum(axis=3)
            assert np.abs(exact).max() < 2 ** 31
            # the same sums in uint32 arithmetic (wrap-around), read as int32
            wrapped = (Ei.astype(np.uint32).cumsum(axis=2, dtype=np.uint32)
                       .cumsum(axis=3, dtype=np.uint32)).view(np.int32)
            assert np.array_equal(wrapped.astype(np.int64), exact)
            got = contract(wrapped.astype(np.float64) / scale, tx0, ty0, R, lam)
            # each plane entry sums at most n weights, each off by <= 1/2 step;
            # |u_i|, |v_j| <= 1 and |u'_i|, |v'_j| <= 1 over the 3 x 3 terms
            bound_h = 0.25 * 9 * n * 0.5 / scale
            for g, r, b in zip(got, ref, (bound_h, lam * bound_h, lam * bound_h)):
                err = np.abs(g - r[ty0:ty0 + T, tx0:tx0 + T]).max()
                assert err <= b, (tx0, ty0, err, b)
