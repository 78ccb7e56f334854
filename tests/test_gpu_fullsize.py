"""GPU parity at the full sizes of the benchmark workloads, on the default
summed-area synthesis (SCWP_SYNTH_SAT), through the C ABI.

* batched: 1024^2 FFT, 32 patches of 64^2..1024^2 texels with 8-32 buckets
  and 4M particles in all, stepped in batched mode (one synthesis launch
  over every patch, frames replayed as captured graphs);
* mixed_large: 2048^2 FFT over 4 km, 8 patches of 1024^2 texels with 2M
  particles and 32 buckets each;
* realistic: one 1024^2 patch with 16 buckets, ~200k particles and a wake,
  over its whole 600-frame run (checked at frames 100, 300 and 600);
* the background FFT at 1024^2 and 2048^2, at t = 0.05 s and t = 60 s (the
  phase w t reduced without float64 on the GPU).

Integer state, bins and eval counts bit-exact; maps at sampled texels
(corners, edges, tile borders, blend band and seeded random texels, each
computed by the oracle's point sums) within max |d| <= 1e-4 Hs and relative
L2 <= 1e-5.  Each test prints the largest candidate count of a (tile,
bucket) pair of the summed-area kernel, whose corner-weight quantum grows
with it, beside the worst error."""
import numpy as np
import pytest

from oracle.scene import OracleScene
from oracle.synth import synth_points, blend_weight, patch_world_coords, sample_background
from paper_2511_02852_gb300 import workloads as wl

from test_gpu_parity import MAX_ABS, REL_L2, compare_bins, compare_maps, compare_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TILE = 64
Q = 65536


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02852_gb300 import scwp
    scwp.lib()
    yield
    torch.cuda.synchronize()


def sample_points(W, H, n_random, seed):
    """Corners, edges, tile borders, the blend band and random texels."""
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (W - 1, H - 1), (W - 1, 0), (0, H - 1), (W // 2, H // 2)]
    for t in range(TILE, max(W, H), TILE):
        if t < W and t < H:
            pts += [(t - 1, t), (t, t - 1), (min(W - 1, t + 5), t)]
    pts += [(3, H // 3), (W - 4, (2 * H) // 3), (W // 3, 2), (W // 5, H - 3)]
    pts += [tuple(v) for v in rng.integers(0, [W, H], size=(n_random, 2))]
    ix = np.array([min(max(p[0], 0), W - 1) for p in pts])
    iy = np.array([min(max(p[1], 0), H - 1) for p in pts])
    return ix, iy


def sampled_reference(orc, cfg, p, ix, iy, bg, buckets=None):
    ps = orc.patches[p]
    bm = ps.bumps()
    if buckets is not None:
        sel = (bm["B"] >= buckets[0]) & (bm["B"] < buckets[1])
        bm = {k: (v[sel] if isinstance(v, np.ndarray) and len(v) == len(sel) else v) for k, v in bm.items()}
    oh, odx, ody = synth_points(ix, iy, bm, orc.lam)
    pc = cfg["patches"][p]
    w = blend_weight(ps.T.W, ps.T.H, float(pc["band"]))[iy, ix]
    xw, yw = patch_world_coords(pc)
    return [w * o + (1 - w) * sample_background(b, orc.L, xw[iy, ix], yw[iy, ix])
            for o, b in zip((oh, odx, ody), bg)]


def max_tile_candidates(orc, sc, p):
    """The largest number of binned bumps in the bins that reach one (64 x 64
    tile, bucket) pair, with the kernel's own bin-range rule: bins hold
    x + R in [bx C, (bx + 1) C); a tile reaches bins floor(X0 / C) ..
    floor((X1 + 2R - 1) / C) per axis (X0, X1 its first and last texel
    centres)."""
    info = sc.info(p)
    ps = orc.patches[p]
    C = [info.bin_cells[i] for i in range(info.n_buckets)]
    ob = ps.bins(C)
    W, H = ps.T.W, ps.T.H
    best = 0
    for i in range(info.n_buckets):
        nbx, nby, base = int(ob["nbx"][i]), int(ob["nby"][i]), int(ob["base"][i])
        cnt = ob["counts"][base:base + nbx * nby].reshape(nby, nbx)
        S = np.zeros((nby + 1, nbx + 1), dtype=np.int64)
        S[1:, 1:] = cnt.cumsum(0).cumsum(1)
        R = int(ps.T.R[i])
        Cq = C[i] * Q
        for ty in range(0, H, TILE):
            Y0 = ty * Q + Q // 2
            Y1 = Y0 + (TILE - 1) * Q
            by0, by1 = Y0 // Cq, min((Y1 + 2 * R - 1) // Cq, nby - 1)
            for tx in range(0, W, TILE):
                X0 = tx * Q + Q // 2
                X1 = X0 + (TILE - 1) * Q
                bx0, bx1 = X0 // Cq, min((X1 + 2 * R - 1) // Cq, nbx - 1)
                if bx0 > bx1 or by0 > by1:
                    continue
                n = S[by1 + 1, bx1 + 1] - S[by0, bx1 + 1] - S[by1 + 1, bx0] + S[by0, bx0]
                best = max(best, int(n))
    return best


def run_scene(cfg, frames, batched):
    from paper_2511_02852_gb300 import scwp
    sc = scwp.Scene(cfg, device=0)
    sc.set_synth_mode(scwp.SYNTH_SAT)
    sc.set_batched(batched)
    orc = OracleScene(cfg)
    for _ in range(frames):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    torch.cuda.synchronize()
    return sc, orc


def check_patches(sc, orc, cfg, n_random, tag):
    hs = orc.spec.Hs()
    bg = orc.background()
    worst, n_max = 0.0, 0
    for p in range(len(cfg["patches"])):
        compare_state(sc, orc, p)
        compare_bins(sc, orc, p)
        ps = orc.patches[p]
        ix, iy = sample_points(ps.T.W, ps.T.H, n_random, 100 + p)
        ref = sampled_reference(orc, cfg, p, ix, iy, bg)
        got = sc.maps(p)
        errs = compare_maps([g[iy, ix] for g in got], ref, hs, f"{tag} patch {p}")
        worst = max(worst, max(e[1] for e in errs))
        n_max = max(n_max, max_tile_candidates(orc, sc, p))
    print(f"[fullsize] {tag}: largest (tile, bucket) candidate count {n_max}, worst |d| {worst:.2e} Hs")
    return worst, n_max


def test_batched_32_patches_full_size():
    """The 32-patch batched workload after 2 frames in batched mode."""
    cfg = wl.batched()
    sc, orc = run_scene(cfg, 2, batched=True)
    check_patches(sc, orc, cfg, 150, "batched 32 patches")
    sc.close()


def test_mixed_large_full_size():
    """mixed_large (8 x 1024^2, 2M particles and 32 buckets per patch) after
    2 frames: the largest candidate counts per (tile, bucket) of any
    workload, where the summed-area kernel's corner-weight quantum is
    largest."""
    cfg = wl.mixed_large()
    sc, orc = run_scene(cfg, 2, batched=True)
    worst, n_max = check_patches(sc, orc, cfg, 150, "mixed_large")
    assert n_max > 5000          # the regime the quantum bound is about
    sc.close()


def test_realistic_600_frames_full_size():
    """The realistic workload over its whole 600-frame run (1024^2 patch,
    16 buckets, ~200k particles, wake; 10 s of simulated time): state, bins
    and eval counts bit-exact and the sampled maps within the contract at
    frames 100, 300 and 600, so neither the integer particle state nor the
    background's phase drifts from the oracle over the run."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.realistic()
    sc = scwp.Scene(cfg, device=0)
    sc.set_synth_mode(scwp.SYNTH_SAT)
    orc = OracleScene(cfg)
    for f in range(1, 601):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
        if f in (100, 300, 600):
            torch.cuda.synchronize()
            assert sc.stats(0).live_particles > 150000
            check_patches(sc, orc, cfg, 150, f"realistic frame {f}")
    sc.close()


@pytest.mark.parametrize("N,dt", [(1024, 1 / 40), (2048, 1 / 40), (2048, 30.0)])
def test_background_fft_full_size(N, dt):
    """The background at the batched (1024^2) and mixed_large (2048^2) grid
    sizes after two steps: t = 0.05 s, and t = 60 s (the longest run of the
    workloads, where the phase w t reaches hundreds of radians)."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.scene("bg", wl.spectrum(wind_speed=15.0, fetch=100e3, depth=50.0, fft_n=N,
                                     fft_L=N * 2.0, choppiness=1.0, seed=N + 3),
                   [wl.patch(width=8, height=8, max_particles=64, inject_scale=1e-9)], frames=2)
    sc = scwp.Scene(cfg, device=0)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc.step(dt)
        orc.step(dt)
    compare_maps(sc.maps(-1), orc.background(), orc.spec.Hs(), f"bg N={N} t={2 * dt:g}")
    sc.close()


@pytest.mark.parametrize("mode_name,bar", [("SYNTH_SAT", MAX_ABS), ("SYNTH_GATHER_FP16", 2e-3)])
def test_mixed_large_error_per_patch_and_bucket(mode_name, bar):
    """The precision row's error statement on mixed_large after 2 frames: the
    blended maps of every patch, and every bucket's share of them
    (scwp_set_bucket_range, against the oracle's sum over that bucket's bumps
    alone), at sampled texels against the FP64 oracle.  Bars: 1e-4 Hs for the
    FP32 summed-area path, 2e-3 Hs for the single-FP16-operand gather; the
    worst error of each patch and bucket is printed."""
    from paper_2511_02852_gb300 import scwp
    mode = getattr(scwp, mode_name)
    cfg = wl.mixed_large()
    sc, orc = run_scene(cfg, 2, batched=True)
    hs = orc.spec.Hs()
    bg = orc.background()
    npatch = len(cfg["patches"])
    pts = [sample_points(orc.patches[p].T.W, orc.patches[p].T.H, 48, 300 + p) for p in range(npatch)]
    sc.resynthesize(mode)
    per_patch = []
    for p in range(npatch):
        ix, iy = pts[p]
        ref = sampled_reference(orc, cfg, p, ix, iy, bg)
        got = sc.maps(p)
        per_patch.append(max(np.abs(g[iy, ix].astype(np.float64) - r).max() for g, r in zip(got, ref)) / hs)
    nb = sc.info(0).n_buckets
    per_bucket = []
    for i in range(nb):
        sc.set_bucket_range(i, i + 1)
        sc.resynthesize(mode)
        worst = 0.0
        for p in range(npatch):
            ix, iy = pts[p]
            ref = sampled_reference(orc, cfg, p, ix, iy, bg, buckets=(i, i + 1))
            got = sc.maps(p)
            worst = max(worst, max(np.abs(g[iy, ix].astype(np.float64) - r).max()
                                   for g, r in zip(got, ref)) / hs)
        per_bucket.append(worst)
    sc.set_bucket_range(0, 1 << 30)
    print(f"[precision] mixed_large {mode_name}: per patch max|d|/Hs "
          + " ".join(f"{e:.1e}" for e in per_patch))
    print(f"[precision] mixed_large {mode_name}: per bucket max|d|/Hs "
          + " ".join(f"{e:.1e}" for e in per_bucket))
    assert max(per_patch) <= bar and max(per_bucket) <= bar
    sc.close()
