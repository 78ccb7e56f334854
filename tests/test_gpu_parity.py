"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI, with
the synthesis on the tensor-core gather (the summed-area synthesis has its
own file, test_gpu_sat.py).

Contract: integer particle state, bins and eval counts bit-exact; float32
maps within max |d| <= 1e-4 Hs and relative L2 <= 1e-5 of the FP64 oracle
(per field: h, Dx, Dy)."""
import math

import numpy as np
import pytest

from oracle.scene import OracleScene
from oracle.synth import synth_points, blend_weight, patch_world_coords, sample_background
from paper_2511_02852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ABS = 1e-4     # times Hs
REL_L2 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02852_gb300 import scwp
    scwp.lib()
    yield
    torch.cuda.synchronize()


def make(cfg, mode=None):
    """A scene on the tensor-core gather (this file's path) unless `mode`
    names another synthesis."""
    from paper_2511_02852_gb300 import scwp
    sc = scwp.Scene(cfg, device=0)
    sc.set_synth_mode(scwp.SYNTH_GATHER if mode is None else mode)
    return sc


def compare_state(sc, orc, p):
    x, y, bd = sc.particles(p)
    ps = orc.patches[p]
    assert len(x) == len(ps.X), (len(x), len(ps.X))
    assert np.array_equal(x, ps.X)
    assert np.array_equal(y, ps.Y)
    assert np.array_equal((bd >> 16).astype(np.int64), ps.B)
    assert np.array_equal((bd & 0xFFFF).astype(np.int64), ps.J)


def compare_bins(sc, orc, p):
    info = sc.info(p)
    C = [info.bin_cells[i] for i in range(info.n_buckets)]
    ob = orc.patches[p].bins(C)
    counts, offsets, entries = sc.bins(p)
    assert info.total_bins == len(ob["counts"])
    assert np.array_equal(counts.astype(np.int64), ob["counts"])
    assert np.array_equal(offsets.astype(np.int64), ob["offsets"])
    assert np.array_equal(entries.astype(np.int64), ob["entries"])
    st = sc.stats(p)
    assert st.eval_count == ob["eval_count"]
    assert st.bumps_binned == int((ob["bumps"]["ec"] > 0).sum())
    assert st.live_particles == len(orc.patches[p].X)
    lpb = orc.patches[p].live_per_bucket()
    assert [st.live_per_bucket[i] for i in range(info.n_buckets)] == lpb.tolist()


def compare_maps(got, ref, hs, tag=""):
    errs = []
    for g, r, name in zip(got, ref, ("h", "Dx", "Dy")):
        g = g.astype(np.float64)
        mx = np.abs(g - r).max()
        rel = np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)
        errs.append((name, mx / hs, rel))
    print(f"[parity] {tag}: " + ", ".join(f"{n} max {m:.2e} Hs rel {r:.2e}" for n, m, r in errs))
    for name, mx, rel in errs:
        assert mx <= MAX_ABS, f"{tag} {name}: max|d| = {mx:.2e} Hs  (all: {errs})"
        assert rel <= REL_L2, f"{tag} {name}: rel L2 = {rel:.3e}  (all: {errs})"
    return errs


@pytest.mark.parametrize("N", [8, 64, 128, 512])
def test_background_fft_matches_oracle(N):
    cfg = wl.scene("bg", wl.spectrum(wind_speed=12.0, fetch=80e3, depth=40.0, fft_n=N,
                                     fft_L=N * 2.0, choppiness=0.9, seed=N),
                   [wl.patch(width=8, height=8, max_particles=64)], frames=3)
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(3):
        sc.step(1 / 60)
        orc.step(1 / 60)
    got = sc.maps(-1)
    ref = orc.background()
    compare_maps(got, ref, orc.spec.Hs(), f"bg N={N}")
    sc.close()


@pytest.mark.parametrize("make_cfg,frames,checks", [
    (wl.tiny, 60, (1, 2, 17, 60)),
    (wl.small_jonswap, 12, (1, 5, 12)),
    (wl.small_two_patches, 8, (1, 8)),
])
def test_scene_parity(make_cfg, frames, checks):
    cfg = make_cfg()
    sc = make(cfg)
    orc = OracleScene(cfg)
    hs = orc.spec.Hs()
    for f in range(1, frames + 1):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
        if f in checks:
            bg = orc.background()
            for p in range(len(cfg["patches"])):
                compare_state(sc, orc, p)
                compare_bins(sc, orc, p)
                ref, ev = orc.patch_maps(p, bg)
                assert sc.stats(p).eval_count == ev
                compare_maps(sc.maps(p), ref, hs, f"{cfg['name']} frame {f} patch {p}")
    sc.close()


def test_injected_energy_and_counts_match_oracle():
    cfg = wl.scaled(wl.small_jonswap(), prefill=0)
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(20):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    st = sc.stats(0)
    ps = orc.patches[0]
    assert st.injected_total == ps.injected
    e = np.array([st.injected_energy[i] for i in range(st.n_buckets)])
    assert np.allclose(e, ps.energy, rtol=1e-12, atol=0)
    compare_state(sc, orc, 0)
    sc.close()


def test_realistic_full_size_state_bins_and_sampled_maps():
    """The bench workload at full size (1024^2 patch, 16 buckets, ~200k
    particles, wake): bit-exact state/bins/evals after 3 frames, and the
    maps at sampled texels (corners, edges, blend band, interior, ragged
    tile borders) against the oracle's point sums."""
    cfg = wl.realistic()
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(3):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    compare_state(sc, orc, 0)
    compare_bins(sc, orc, 0)
    h, dx, dy = sc.maps(0)
    ps = orc.patches[0]
    W, H = ps.T.W, ps.T.H
    rng = np.random.default_rng(0)
    pts = [(0, 0), (W - 1, H - 1), (W - 1, 0), (0, H - 1), (63, 64), (64, 63), (511, 512),
           (W // 2, H // 2), (127, 900), (5, 700)]
    pts += [tuple(v) for v in rng.integers(0, [W, H], size=(150, 2))]
    ix = np.array([p[0] for p in pts])
    iy = np.array([p[1] for p in pts])
    oh, odx, ody = synth_points(ix, iy, ps.bumps(), orc.lam)
    w = blend_weight(W, H, float(cfg["patches"][0]["band"]))[iy, ix]
    xw, yw = patch_world_coords(cfg["patches"][0])
    bg = orc.background()
    ref = [w * o + (1 - w) * sample_background(b, orc.L, xw[iy, ix], yw[iy, ix])
           for o, b in zip((oh, odx, ody), bg)]
    got = [h[iy, ix], dx[iy, ix], dy[iy, ix]]
    compare_maps(got, ref, orc.spec.Hs(), "realistic sampled")
    sc.close()


def test_bins_exact_with_sort_tiles_past_one_scan_chunk():
    """600k particles in a 700k-particle patch: 1.2M bump keys fill more
    than 1024 sort tiles, so the scan of each digit's per-tile counts runs
    in several chunks (4 entries per thread per chunk).  Particle state and
    bins (counts, offsets, entries) bit-exact after two frames."""
    cfg = wl.scaled(wl.realistic(), max_particles=700000, prefill=600000)
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    assert 2 * sc.stats(0).live_particles > 1024 * 1024
    compare_state(sc, orc, 0)
    compare_bins(sc, orc, 0)
    sc.close()


@pytest.mark.parametrize("mode_name", ["SYNTH_GATHER", "SYNTH_SAT"])
def test_single_particle_closed_form_on_gpu(mode_name):
    """One particle moving along +x: on the crest-to-trough segment the GPU map
    is A cos(pi s / R) (Fig. 1 pair), away from the blend band; a 300 x 40
    patch, so the tiles are ragged in both directions."""
    cfg = wl.scene("one", wl.spectrum(n_buckets=3, n_theta=16, wind_dir=math.pi / 16,
                                      fft_n=16, fft_L=64.0, seed=1),
                   [wl.patch(width=300, height=40, cell=0.5, band=1.0, max_particles=16,
                             inject_scale=1e-12)], frames=1)
    sc = make(cfg)
    info = sc.info(0)
    from paper_2511_02852_gb300 import scwp
    R = sc.table(0, scwp.TAB_RQ)
    A = sc.table(0, scwp.TAB_AMP).reshape(info.n_buckets, info.n_theta)
    j = 7                       # theta_j = 0 for wind_dir = pi/16
    b = 1
    X = 200 * 65536 + 4321
    Y = 20 * 65536 + 32768
    sc.set_particles(0, [X], [Y], [(b << 16) | j])
    sc.resynthesize(getattr(scwp, mode_name))
    h, dx, dy = sc.maps(0)
    Rb = int(R[b])
    for ix in range(2, 298):
        s = ix * 65536 + 32768 - X
        if -Rb < s < 0:
            assert abs(h[20, ix] - A[b, j] * math.cos(math.pi * s / Rb)) < 2e-6 * A[b, j] + 1e-7
    sc.close()


def test_empty_patch_is_blended_background():
    cfg = wl.scene("empty", wl.spectrum(fft_n=64, fft_L=200.0, seed=9),
                   [wl.patch(width=75, height=51, cell=0.5, max_particles=4096, prefill=0,
                             inject_scale=1e-9, origin_x=10.3, origin_y=-7.7)], frames=2)
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    assert sc.stats(0).live_particles == 0
    ref, ev = orc.patch_maps(0)
    assert ev == 0
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), "empty")
    sc.close()


def test_capacity_overflow_truncates_like_oracle():
    cfg = wl.scaled(wl.small_jonswap(), max_particles=2900)
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(6):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    assert orc.patches[0].overflow
    assert sc.stats(0).error_flags & 1
    compare_state(sc, orc, 0)
    sc.close()


def test_dt_change_rebuilds_tables():
    cfg = wl.small_jonswap()
    sc = make(cfg)
    orc = OracleScene(cfg)
    for dt in (1 / 60, 1 / 60, 1 / 30, 1 / 45, 1 / 30):
        sc.step(dt)
        orc.step(dt)
    compare_state(sc, orc, 0)
    compare_bins(sc, orc, 0)
    sc.close()


def test_rerun_is_deterministic():
    cfg = wl.small_two_patches()
    a = make(cfg)
    b = make(cfg)
    for _ in range(4):
        a.step()
        b.step()
    for p in range(2):
        for u, v in zip(a.maps(p), b.maps(p)):
            assert np.array_equal(u, v)
    a.close()
    b.close()


@pytest.mark.parametrize("make_cfg", [wl.tiny, wl.small_jonswap, wl.small_two_patches])
def test_layered_variant_matches_oracle(make_cfg):
    """Layer splat + separable x/y passes + layer sum (Sec. 4.2) against the
    oracle's layered restatement, after a few frames."""
    from paper_2511_02852_gb300 import scwp
    from oracle.synth import blend, layered_maps
    cfg = make_cfg()
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(3):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    sc.resynthesize(scwp.SYNTH_LAYERED)
    bg = orc.background()
    for p in range(len(cfg["patches"])):
        ps = orc.patches[p]
        bm = ps.bumps()
        wp = layered_maps(ps.T.W, ps.T.H, bm, orc.lam, ps.T.nb, ps.T.R)
        ref = blend(cfg["patches"][p], wp, bg, orc.L)
        compare_maps(sc.maps(p), ref, orc.spec.Hs(), f"layered {cfg['name']} patch {p}")
    # and the default path still reproduces the gather afterwards
    sc.resynthesize(scwp.SYNTH_GATHER)
    ref, _ = orc.patch_maps(0, bg)
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), "gather after layered")
    sc.close()



@pytest.mark.parametrize("mode_name", ["SYNTH_GATHER", "SYNTH_GATHER_FP32"])
def test_both_gather_kernels_match_oracle(mode_name):
    """The tensor-core gather (default) and the CUDA-core gather give the
    oracle's maps within the contract on the same frames."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.small_jonswap()
    sc = make(cfg)
    sc.set_synth_mode(getattr(scwp, mode_name))
    orc = OracleScene(cfg)
    for _ in range(4):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    ref, _ = orc.patch_maps(0)
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), mode_name)
    sc.close()


def test_batched_frame_matches_plain_and_oracle():
    """One synthesis launch over all patches (scwp_set_batched): bit-exact
    state and bins, maps within the contract of the oracle, and within
    FP32 rounding of the one-patch-per-launch path, on a frame of five
    uneven patches."""
    cfg = wl.small_batch()
    a = make(cfg)
    b = make(cfg)
    b.set_batched(True)          # captured frame graphs, replayed from frame 3
    c = make(cfg)
    c.set_batched(True)
    c.set_timing(True)           # the same frames launched one kernel at a time
    orc = OracleScene(cfg)
    hs = orc.spec.Hs()
    for f in range(1, 7):
        a.step(cfg["dt"])
        b.step(cfg["dt"])
        c.step(cfg["dt"])
        orc.step(cfg["dt"])
        if f in (2, 6):
            bg = orc.background()
            for p in range(len(cfg["patches"])):
                compare_state(b, orc, p)
                compare_bins(b, orc, p)
                ref, ev = orc.patch_maps(p, bg)
                assert b.stats(p).eval_count == ev
                mb, ma = b.maps(p), a.maps(p)
                compare_maps(mb, ref, hs, f"batched frame {f} patch {p}")
                for x, y in zip(mb, ma):
                    assert np.abs(x.astype(np.float64) - y).max() <= 1e-5 * hs
                for x, y in zip(mb, c.maps(p)):
                    assert np.array_equal(x, y)     # graph replay == eager launches
                assert b.stats(p).injected_total == c.stats(p).injected_total
    # the captured frame launches the injection kernel even when a patch
    # injects nothing this frame (the eager path skips it)
    n_inj = len(cfg["patches"]) * 6
    assert c.launch_count() <= b.launch_count() <= c.launch_count() + n_inj
    a.close()
    b.close()
    c.close()


FP16_MAX_ABS = 2e-3    # times Hs: the contract of reduced-precision synthesis


@pytest.mark.parametrize("make_cfg", [wl.small_jonswap, wl.small_batch])
def test_fp16_synthesis_within_2e3_hs_per_bucket_and_patch(make_cfg):
    """Single-FP16 tensor-core operands (SCWP_SYNTH_GATHER_FP16): state and
    bins unchanged (bit-exact), and every patch's maps, and every bucket's
    share of them, within 2e-3 Hs of the FP64 oracle.  The errors are
    printed per patch and bucket."""
    from paper_2511_02852_gb300 import scwp
    cfg = make_cfg()
    sc = make(cfg)
    sc.set_batched(True)
    sc.set_synth_mode(scwp.SYNTH_GATHER_FP16)
    orc = OracleScene(cfg)
    hs = orc.spec.Hs()
    for _ in range(3):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    bg = orc.background()
    worst = 0.0
    for p in range(len(cfg["patches"])):
        compare_state(sc, orc, p)
        compare_bins(sc, orc, p)
        ref, _ = orc.patch_maps(p, bg)
        err = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(sc.maps(p), ref)) / hs
        print(f"[fp16] {cfg['name']} patch {p}: max|d| = {err:.2e} Hs")
        assert err <= FP16_MAX_ABS
        worst = max(worst, err)
    nbs = [sc.info(p).n_buckets for p in range(len(cfg["patches"]))]
    for i in range(max(nbs)):
        sc.set_bucket_range(i, i + 1)
        sc.resynthesize(scwp.SYNTH_GATHER_FP16)
        for p in range(len(cfg["patches"])):
            if i >= nbs[p]:
                continue
            ref, _ = orc.patch_maps(p, bg, buckets=(i, i + 1))
            err = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(sc.maps(p), ref)) / hs
            print(f"[fp16] {cfg['name']} patch {p} bucket {i}: max|d| = {err:.2e} Hs")
            assert err <= FP16_MAX_ABS
    sc.close()


def test_normal_map_matches_oracle_formula():
    """scwp_normal_map: the GPU normals of the GPU maps equal the oracle's
    finite-difference normals of the same maps (1e-5), and stay within the
    slope error the map contract allows of the normals of the oracle's own
    maps (a one-sided difference of two texels each off by at most
    max|d map|: |d slope| <= 2 max|d map| / cell)."""
    from oracle.synth import normal_map
    cfg = wl.small_jonswap()
    sc = make(cfg)
    orc = OracleScene(cfg)
    for _ in range(3):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    hs = orc.spec.Hs()
    cell = float(cfg["patches"][0]["cell"])
    got = sc.normals(0)
    maps = sc.maps(0)
    mine = normal_map(*maps, cell)
    assert np.abs(got - mine).max() <= 1e-5
    ref, _ = orc.patch_maps(0)
    theirs = normal_map(*ref, cell)
    d_map = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(maps, ref))
    err = np.abs(got - theirs).max()
    print(f"[normals] max|d n| = {err:.2e} (map error {d_map / hs:.2e} Hs, bound {2 * d_map / cell:.2e})")
    assert err <= 2 * d_map / cell + 1e-6
    assert np.allclose(np.sum(got.astype(np.float64) ** 2, axis=0), 1.0, atol=1e-5)
    sc.close()


@pytest.mark.parametrize("mode_name", ["SYNTH_GATHER", "SYNTH_SAT"])
def test_ring_ripples_state_bins_and_maps_match_oracle(mode_name):
    """A heaving object (ring ripples, Sec. 4.3 vertical motion) on top of
    its Kelvin wake: particle state and bins bit-exact, injected energy and
    counts equal, maps within the contract (both syntheses: the wake
    amplitude enters the summed-area bound)."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.small_jonswap()
    cfg["patches"][0].update(emitter=1, wake_rate=1, heave_period=20 * cfg["dt"], ring_rate=6,
                             obj_radius=3.0, obj_speed=2.0, obj_path_radius=6.0)
    sc = make(cfg, getattr(scwp, mode_name))
    orc = OracleScene(cfg)
    for f in range(1, 31):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
        if f in (5, 17, 30):
            compare_state(sc, orc, 0)
            compare_bins(sc, orc, 0)
    ps = orc.patches[0]
    assert ps.ring_total > 0
    st = sc.stats(0)
    assert st.injected_total == ps.injected
    assert np.allclose([st.injected_energy[i] for i in range(st.n_buckets)], ps.energy, rtol=1e-12, atol=0)
    ref, _ = orc.patch_maps(0)
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), f"ring ripples {mode_name}")
    sc.close()
