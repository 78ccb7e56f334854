"""Pins of the oracle's wave-particle side: the integer support test, the
pair kernel's closed forms (Fig. 1), the crest train, binning, the
injected energy per bucket (Eqs. 8-15), N_theta invariance (Sec. 3.3 last
paragraph / Sec. 5.2), the blend limits and the layered variant.  CPU only."""
import math

import numpy as np
import pytest

from oracle import spectrum as sp
from oracle.particles import HALF, Q, PatchState, PatchTables, texel_span
from oracle.scene import OracleScene
from oracle.synth import (blend, blend_weight, layered_maps, sample_background,
                          synth_maps, synth_maps_numpy, synth_points)
from paper_2511_02852_gb300 import workloads as wl


def test_texel_span_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        n = int(rng.integers(1, 40))
        R = int(rng.integers(1, 20 * Q))
        C = int(rng.integers(-30 * Q, (n + 30) * Q))
        lo, hi, cnt = texel_span(C, R, n)
        brute = [ix for ix in range(n) if abs(ix * Q + HALF - C) < R]
        assert int(cnt) == len(brute)
        if brute:
            assert int(lo) == brute[0] and int(hi) == brute[-1]


def test_texel_span_boundary_is_strict():
    # a texel centre exactly R away is outside
    lo, hi, cnt = texel_span(HALF + 3 * Q, 3 * Q, 10)
    assert (int(lo), int(hi), int(cnt)) == (1, 5, 5)


def _bumps(X, Y, R, A):
    X = np.asarray(X, dtype=np.int64)
    return dict(X=X, Y=np.asarray(Y, dtype=np.int64), R=np.asarray(R, dtype=np.int64),
                amp=np.asarray(A, dtype=np.float64), ec=np.ones(len(X), dtype=np.int64))


def test_single_pair_closed_form():
    """Positive-negative pair (Fig. 1): crest +A at p, trough -A at p - r;
    on the crest-to-trough segment h = A cos(pi s / r) and
    Dx = lambda A sin(pi s / r) exactly (s = x - p)."""
    W, H = 200, 5
    R = 37 * Q + 12345
    X = 120 * Q + 777
    Y = 2 * Q + HALF          # on the centre line of row 2
    A, lam = 0.7, 0.9
    bm = _bumps([X, X - R], [Y, Y], [R, R], [A, -A])
    h, dx, dy, _ = synth_maps(W, H, bm, lam)
    for ix in range(W):
        s = ix * Q + HALF - X
        if -R < s < 0:
            assert h[2, ix] == pytest.approx(A * math.cos(math.pi * s / R), abs=1e-14)
            assert dx[2, ix] == pytest.approx(lam * A * math.sin(math.pi * s / R), abs=1e-14)
            assert dy[2, ix] == pytest.approx(0.0, abs=1e-15)


def test_crest_train_reproduces_cosine():
    """A train of pairs spaced lambda = 2r reproduces A cos(pi (x - p)/r) in
    its interior (Fig. 1b)."""
    W, H = 600, 3
    R = 21 * Q + 999
    A, lam = 0.4, 1.0
    p0 = 500 * Q + 3
    X, Y, Rs, As = [], [], [], []
    for n in range(14):
        c = p0 - 2 * n * R
        X += [c, c - R]
        Y += [Q + HALF] * 2
        Rs += [R, R]
        As += [A, -A]
    h, dx, dy, _ = synth_maps(W, H, _bumps(X, Y, Rs, As), lam)
    for ix in range(100, 450):
        s = ix * Q + HALF - p0
        assert h[1, ix] == pytest.approx(A * math.cos(math.pi * s / R), abs=1e-13)
        assert dx[1, ix] == pytest.approx(lam * A * math.sin(math.pi * s / R), abs=1e-13)


def test_c_synthesis_matches_numpy_restatement():
    rng = np.random.default_rng(4)
    W, H = 37, 29
    n = 60
    R = rng.integers(2 * Q, 15 * Q, n)
    X = rng.integers(-10 * Q, (W + 10) * Q, n)
    Y = rng.integers(-10 * Q, (H + 10) * Q, n)
    A = rng.normal(size=n)
    bm = _bumps(X, Y, R, A)
    a = synth_maps(W, H, bm, 0.7)
    b = synth_maps_numpy(W, H, bm, 0.7)
    for u, v in zip(a[:3], b):
        assert np.abs(u - v).max() < 1e-12
    # eval count = brute-force count of (bump, texel) pairs inside the support
    xt = np.arange(W) * Q + HALF
    yt = np.arange(H) * Q + HALF
    cnt = sum(int(((np.abs(xt - x) < r).sum()) * ((np.abs(yt - y) < r).sum()))
              for x, y, r in zip(X, Y, R))
    assert a[3] == cnt
    pts = rng.integers(0, [W, H], size=(20, 2))
    ph, px, py = synth_points(pts[:, 0], pts[:, 1], bm, 0.7)
    assert np.allclose(ph, a[0][pts[:, 1], pts[:, 0]], atol=1e-13)
    assert np.allclose(px, a[1][pts[:, 1], pts[:, 0]], atol=1e-13)


def test_bump_integral():
    """int bump = A r^2 (continuous); the texel sum of a wide bump matches to
    O((Q/R)^2)."""
    R = 200 * Q
    W = H = 420
    h, _, _, _ = synth_maps(W, H, _bumps([210 * Q], [210 * Q], [R], [1.0]), 0.0)
    assert h.sum() == pytest.approx((R / Q) ** 2, rel=1e-4)


def _tiny_scene(**over):
    sc = wl.tiny()
    sc["patches"][0].update(over)
    return sc


def test_bins_are_stable_and_complete():
    sc = OracleScene(wl.small_jonswap())
    for _ in range(3):
        sc.step(1 / 60)
    ps = sc.patches[0]
    C = [16, 32, 32, 64, 8, 16]
    b = ps.bins(C)
    bm = b["bumps"]
    valid = bm["ec"] > 0
    assert b["counts"].sum() == valid.sum()
    assert b["offsets"][-1] == valid.sum()
    # each entry's bin recomputed independently
    T = ps.T
    for key in np.nonzero(b["counts"])[0][:200]:
        ents = b["entries"][b["offsets"][key]:b["offsets"][key + 1]]
        assert np.all(np.diff(ents) > 0)            # stable: ids ascending
        for e in ents:
            i = int(bm["B"][e])
            Cq = C[i] * Q
            bx = (int(bm["X"][e]) + int(T.R[i])) // Cq
            by = (int(bm["Y"][e]) + int(T.R[i])) // Cq
            assert key == b["base"][i] + by * b["nbx"][i] + bx
    assert b["eval_count"] == int(bm["ec"].sum())


def test_injected_energy_per_bucket_matches_spectrum_integral():
    """Over F frames the injected 1/8 A^2 pi r^2 per bucket equals
    F sum_s L_s dt c_i E_i (Eq. 11 for each edge pair, with the exact bucket
    integral E_i of Eq. 8) up to one group per edge pair (the carry)."""
    sc = wl.scaled(wl.small_jonswap(), prefill=0, emitter=0, inject_scale=1.0,
                   max_particles=10 ** 6)
    o = OracleScene(sc)
    F = 40
    for _ in range(F):
        o.step(1 / 60)
    ps = o.patches[0]
    T = ps.T
    for i in range(T.nb):
        expect = F * (T.H + T.W) * T.dx * (1 / 60) * T.b.c[i] * T.b.E[i]
        group = 0.25 * math.pi * T.b.r[i] ** 2 * T.b.E[i]
        assert abs(ps.energy[i] - expect) <= 2 * group + 1e-12 * expect


def test_energy_invariant_under_n_theta():
    """Raising N_theta raises particle numbers but lowers amplitudes; the
    injected energy per bucket is unchanged (Sec. 3.3, Sec. 5.2)."""
    energies = []
    counts = []
    for nth in (8, 16, 32):
        sc = wl.scaled(wl.small_jonswap(), prefill=0, emitter=0, inject_scale=1.0,
                       max_particles=10 ** 6)
        sc["spectrum"]["n_theta"] = nth
        o = OracleScene(sc)
        for _ in range(30):
            o.step(1 / 60)
        energies.append(o.patches[0].energy.copy())
        counts.append(o.patches[0].injected)
    T = o.patches[0].T
    for i in range(T.nb):
        group = 0.25 * math.pi * T.b.r[i] ** 2 * T.b.E[i]
        assert max(e[i] for e in energies) - min(e[i] for e in energies) <= 4 * group + 1e-9
    assert counts[0] < counts[1] < counts[2]


def test_advection_speed_matches_dispersion():
    """A particle moves c_i dt per frame (to the fixed-point rounding), the
    same phase speed the FFT background gives the same k (Sec. 5.2: long
    waves travel at matching speeds)."""
    sc = wl.small_jonswap()
    spec = sp.Spectrum(sc["spectrum"])
    T = PatchTables(spec, sc["spectrum"], sc["patches"][0], 1 / 60)
    for i in range(T.nb):
        for j in range(T.nth):
            d = math.hypot(T.vx[i, j], T.vy[i, j]) / Q * T.dx / (1 / 60)
            assert d == pytest.approx(T.b.c[i], abs=1.0 / Q * T.dx * 60 * 1.5)
        assert float(spec.omega_of_k(T.b.k[i])) / T.b.k[i] == pytest.approx(T.b.c[i], rel=1e-13)


def test_particles_flow_inward_and_expire_outside():
    o = OracleScene(wl.scaled(wl.small_jonswap(), prefill=0, emitter=0))
    for _ in range(5):
        o.step(1 / 60)
    ps = o.patches[0]
    T = ps.T
    vx, vy, _, _, _ = T.lookup(ps.B, ps.J)
    # every injected particle started on the edge its direction enters through
    assert np.all((ps.X >= -abs(vx) * 6) & (ps.X <= T.W * Q + abs(vx) * 6))
    assert len(ps.X) > 0
    n0 = len(ps.X)
    # far outside: put one particle 2r beyond the right edge moving right
    far = int(T.W * Q + 3 * T.R[0])
    ps.X = np.append(ps.X, far)
    ps.Y = np.append(ps.Y, T.H * Q // 2)
    ps.B = np.append(ps.B, 0)
    ps.J = np.append(ps.J, int(np.argmax(T.vx[0])))
    o.step(1 / 60)
    assert far + int(np.max(T.vx[0])) not in set(ps.X.tolist())
    assert len(ps.X) >= n0 - 50


def test_wake_arms_symmetric_about_heading():
    sc = wl.scaled(wl.small_jonswap(), prefill=0, wake_rate=64, inject_scale=1e-9)
    o = OracleScene(sc)
    o.step(1 / 60)
    ps = o.patches[0]
    T = ps.T
    wake = ps.J >= T.nth
    assert wake.sum() == 128
    ang = (ps.J[wake] - T.nth) * 2 * math.pi / 4096
    t = o.t
    heading = T.obj_speed / T.obj_path_radius * t + math.pi / 2
    d = np.angle(np.exp(1j * (ang - heading)))
    arm = math.pi / 2 - math.asin(1 / 3)
    assert np.allclose(np.sort(np.unique(np.round(d, 2))), [-round(arm, 2), round(arm, 2)], atol=0.01)
    assert np.all(ps.B[wake] == T.bw)


def test_scene_is_deterministic():
    a = OracleScene(wl.small_jonswap())
    b = OracleScene(wl.small_jonswap())
    for _ in range(4):
        a.step(1 / 60)
        b.step(1 / 60)
    pa, pb = a.patches[0], b.patches[0]
    assert np.array_equal(pa.X, pb.X) and np.array_equal(pa.J, pb.J)


def test_blend_limits_and_monotone():
    W, H, band = 40, 30, 6.0
    w = blend_weight(W, H, band)
    assert np.all(w[6:-6, 6:-6] == 1.0)         # interior: WP exactly
    assert np.all(w > 0) and np.all(w <= 1)
    row = w[H // 2, : W // 2]
    assert np.all(np.diff(row) >= 0)
    pcfg = wl.patch(width=W, height=H, band=band, cell=0.5, origin_x=3.0, origin_y=-2.0)
    rng = np.random.default_rng(2)
    wp = [rng.normal(size=(H, W)) for _ in range(3)]
    bgm = [rng.normal(size=(32, 32)) for _ in range(3)]
    out = blend(pcfg, wp, bgm, 64.0)
    for o, m in zip(out, wp):
        assert np.array_equal(o[6:-6, 6:-6], m[6:-6, 6:-6])


def test_bilinear_background_exact_on_grid_and_linear_between():
    N, L = 16, 32.0
    rng = np.random.default_rng(3)
    g = rng.normal(size=(N, N))
    xs = np.arange(N) * L / N
    assert np.allclose(sample_background(g, L, xs[None, :].repeat(N, 0),
                                         xs[:, None].repeat(N, 1)), g, atol=1e-14)
    # midpoint of two x neighbours, and periodic wrap
    v = sample_background(g, L, np.array([L / N * 2.5]), np.array([L / N * 3]))
    assert v[0] == pytest.approx(0.5 * (g[3, 2] + g[3, 3]))
    v = sample_background(g, L, np.array([-L / N * 0.5]), np.array([0.0]))
    assert v[0] == pytest.approx(0.5 * (g[0, N - 1] + g[0, 0]))


def test_layered_variant_equals_gather_at_texel_centres():
    """Bumps exactly at texel centres: layer splat + separable x/y passes
    (Sec. 4.2) reproduce the gather exactly."""
    rng = np.random.default_rng(7)
    W, H = 48, 40
    Rb = np.array([9 * Q + 1234, 4 * Q + 77])
    n = 30
    B = rng.integers(0, 2, n)
    X = rng.integers(-5, W + 5, n) * Q + HALF
    Y = rng.integers(-5, H + 5, n) * Q + HALF
    A = rng.normal(size=n)
    bm = dict(X=X.astype(np.int64), Y=Y.astype(np.int64), R=Rb[B], amp=A, B=B)
    _, _, cx = texel_span(bm["X"], bm["R"], W)
    _, _, cy = texel_span(bm["Y"], bm["R"], H)
    bm["ec"] = cx * cy
    g = synth_maps(W, H, bm, 0.8)
    lay = layered_maps(W, H, bm, 0.8, 2, Rb)
    for a, b in zip(g[:3], lay):
        assert np.abs(a - b).max() < 1e-12


def test_layered_variant_close_to_gather_off_centre():
    """Off texel centres the bilinear splat is a second-order approximation."""
    o = OracleScene(_tiny_scene())
    o.step(1 / 60)
    ps = o.patches[0]
    bm = ps.bumps()
    g = synth_maps(ps.T.W, ps.T.H, bm, 1.0)
    lay = layered_maps(ps.T.W, ps.T.H, bm, 1.0, ps.T.nb, ps.T.R)
    rel = np.linalg.norm(g[0] - lay[0]) / np.linalg.norm(g[0])
    assert rel < 0.02


def _ring_scene(frames_per_period=60, periods=4, rate=5):
    from paper_2511_02852_gb300 import workloads as wl
    cfg = wl.small_jonswap()
    p = cfg["patches"][0]
    p.update(emitter=1, wake_rate=0, heave_period=frames_per_period * cfg["dt"], ring_rate=rate,
             obj_radius=3.0, obj_speed=2.0, obj_path_radius=6.0, max_particles=200000)
    return cfg, frames_per_period * periods


def test_ring_ripples_follow_the_heave_speed_and_start_on_the_rim():
    """Ring ripples (vertical motion, Sec. 4.3): over whole heave periods the
    particle count approaches rate x frames x 2/pi (the mean of |cos|);
    every ring particle starts on the object's rim, moving outward."""
    import math
    from oracle.particles import Q, WAKE_DIRS
    from oracle.scene import OracleScene
    cfg, frames = _ring_scene()
    orc = OracleScene(cfg)
    ps = orc.patches[0]
    T = ps.T
    counts = []
    for _ in range(frames):
        n0 = len(ps.X)
        before = set(zip(ps.X.tolist(), ps.Y.tolist()))
        orc.step(cfg["dt"])
        ring = ps.J >= T.nth
        t = ps.t
        Rp, Om, rho = T.obj_path_radius / T.dx, T.obj_speed / T.obj_path_radius, T.obj_radius / T.dx
        Px, Py = T.W * 0.5 + Rp * math.cos(Om * t), T.H * 0.5 + Rp * math.sin(Om * t)
        new = [k for k in np.nonzero(ring)[0] if (int(ps.X[k]), int(ps.Y[k])) not in before]
        fresh = [k for k in new if abs(math.hypot(ps.X[k] / Q - Px, ps.Y[k] / Q - Py) - rho) < 1e-3]
        counts.append(len(fresh))
        for k in fresh:   # outward: the direction points away from the object centre
            a = int(ps.J[k] - T.nth)
            ux, uy = math.cos(2 * math.pi * a / WAKE_DIRS), math.sin(2 * math.pi * a / WAKE_DIRS)
            assert (ps.X[k] / Q - Px) * ux + (ps.Y[k] / Q - Py) * uy > 0.99 * rho
    total = sum(counts)
    expect = T.ring_rate * frames * 2.0 / math.pi
    assert abs(total - expect) <= 0.03 * expect + 2, (total, expect)
    assert total == ps.ring_total


def test_ring_directions_visit_the_whole_grid():
    """Stepping the wake grid by 2531 (odd, coprime with 4096): 4096
    successive ring particles take 4096 distinct directions."""
    from oracle.particles import WAKE_DIRS
    assert len({(k * 2531) % WAKE_DIRS for k in range(WAKE_DIRS)}) == WAKE_DIRS


@pytest.mark.parametrize("n_theta", [8, 12, 16, 32])
def test_direction_grid_half_offset_never_parallel_to_an_edge(n_theta):
    """The fixed grid theta_j = theta_w - pi + (j + 1/2) dtheta (reading of
    Sec. 4.2 / Eq. 13): with the wind along +x no direction is parallel to
    a patch edge, so every direction flows in through exactly one edge of
    each pair; the grid is symmetric about the wind and covers the circle
    evenly."""
    th, rel, dth = sp.directions(0.0, n_theta)
    assert dth == pytest.approx(2 * math.pi / n_theta)
    assert np.all(np.abs(np.cos(th)) > 1e-3) and np.all(np.abs(np.sin(th)) > 1e-3)
    assert np.allclose(np.sort(rel), np.sort(-rel), atol=1e-12)      # symmetric about the wind
    assert np.allclose(np.diff(th), dth, atol=1e-12)
    assert rel[0] == pytest.approx(-math.pi + dth / 2) and rel[-1] == pytest.approx(math.pi - dth / 2)


def test_injection_carry_sums_to_floor_of_total_rate():
    """The FP64 carry of the fractional group counts (reading of Eqs. 15-17):
    with dyadic rates (every sum exact in FP64) the groups injected over F
    frames through each (bucket, edge pair) are exactly floor(F n), the
    carry left is frac(F n), and each group adds one particle per direction
    with A_ij > 0 that flows in through that pair."""
    cfg = wl.small_jonswap()
    ps = PatchState(sp.Spectrum(cfg["spectrum"]), cfg["spectrum"], dict(cfg["patches"][0], prefill=0),
                    0, 3, cfg["dt"])
    T = ps.T
    rng = np.random.default_rng(2)
    rates = rng.integers(1, 400, size=(T.nb, 2)) / 128.0          # dyadic: k / 2^7
    T.injection_rate = lambda i, s: float(rates[i, s])
    F = 97
    for f in range(F):
        ps.inject(f)
    expect = 0
    for i in range(T.nb):
        for s in (0, 1):
            total = F * rates[i, s]
            assert ps.carry[i, s] == total - math.floor(total)
            vn = T.vx[i] if s == 0 else T.vy[i]
            ndir = int(((T.A[i] > 0) & (vn != 0)).sum())
            expect += math.floor(total) * ndir
    assert len(ps.X) == expect
