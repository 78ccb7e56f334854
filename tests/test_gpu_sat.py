"""GPU parity of the summed-area synthesis (SCWP_SYNTH_SAT) against the FP64
oracle, through the C ABI.

The mode computes the per-bucket kernel sums of Sec. 4.2 through 2-D
prefix sums of the bumps' support-box corners instead of per-pair kernel
evaluations.  Same contract as the gather: state, bins and eval counts
bit-exact (the particle stages are shared); maps within max |d| <= 1e-4 Hs
and relative L2 <= 1e-5 of the oracle's direct sums."""
import numpy as np
import pytest

from oracle.scene import OracleScene
from oracle.synth import synth_points, blend_weight, patch_world_coords, sample_background
from paper_2511_02852_gb300 import workloads as wl

from test_gpu_parity import MAX_ABS, compare_bins, compare_maps, compare_state, make

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02852_gb300 import scwp
    scwp.lib()
    yield
    torch.cuda.synchronize()


def sat_scene(cfg, batched=False):
    from paper_2511_02852_gb300 import scwp
    sc = make(cfg)
    sc.set_synth_mode(scwp.SYNTH_SAT)
    if batched:
        sc.set_batched(True)
    return sc


@pytest.mark.parametrize("make_cfg,frames,checks", [
    (wl.tiny, 60, (1, 17, 60)),
    (wl.small_jonswap, 12, (1, 12)),
    (wl.small_two_patches, 8, (1, 8)),
    (wl.small_batch, 4, (4,)),
])
def test_sat_scene_parity(make_cfg, frames, checks):
    """Every patch's blended maps against the oracle over a run of frames
    (small buckets whose support fits inside a tile in `tiny`, ragged
    patch sizes and several patches in the others)."""
    cfg = make_cfg()
    sc = sat_scene(cfg)
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
                compare_maps(sc.maps(p), ref, hs, f"sat {cfg['name']} frame {f} patch {p}")
    sc.close()


def test_sat_realistic_full_size_sampled_maps():
    """The bench workload at full size (1024^2 patch, 16 buckets, ~200k
    particles, wake): maps at sampled texels against the oracle's point
    sums, and the whole map against the tensor-core gather."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.realistic()
    sc = sat_scene(cfg)
    orc = OracleScene(cfg)
    for _ in range(3):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    compare_state(sc, orc, 0)
    h, dx, dy = sc.maps(0)
    ps = orc.patches[0]
    W, H = ps.T.W, ps.T.H
    rng = np.random.default_rng(1)
    pts = [(0, 0), (W - 1, H - 1), (W - 1, 0), (0, H - 1), (63, 64), (64, 63), (511, 512),
           (W // 2, H // 2), (127, 900), (5, 700), (960, 1023), (1023, 960)]
    pts += [tuple(v) for v in rng.integers(0, [W, H], size=(150, 2))]
    ix = np.array([p[0] for p in pts])
    iy = np.array([p[1] for p in pts])
    oh, odx, ody = synth_points(ix, iy, ps.bumps(), orc.lam)
    w = blend_weight(W, H, float(cfg["patches"][0]["band"]))[iy, ix]
    xw, yw = patch_world_coords(cfg["patches"][0])
    bg = orc.background()
    ref = [w * o + (1 - w) * sample_background(b, orc.L, xw[iy, ix], yw[iy, ix])
           for o, b in zip((oh, odx, ody), bg)]
    compare_maps([h[iy, ix], dx[iy, ix], dy[iy, ix]], ref, orc.spec.Hs(), "sat realistic sampled")
    sc.resynthesize(scwp.SYNTH_GATHER)
    hs = orc.spec.Hs()
    for a, b in zip((h, dx, dy), sc.maps(0)):
        assert np.abs(a.astype(np.float64) - b).max() <= 2 * MAX_ABS * hs
    sc.close()


def test_sat_per_bucket_shares_match_oracle():
    """Each bucket's share of the maps (scwp_set_bucket_range) against the
    oracle's sum over that bucket's bumps alone."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.small_jonswap()
    sc = sat_scene(cfg)
    orc = OracleScene(cfg)
    hs = orc.spec.Hs()
    for _ in range(3):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    bg = orc.background()
    for i in range(sc.info(0).n_buckets):
        sc.set_bucket_range(i, i + 1)
        sc.resynthesize(scwp.SYNTH_SAT)
        ref, _ = orc.patch_maps(0, bg, buckets=(i, i + 1))
        err = max(np.abs(g.astype(np.float64) - r).max() for g, r in zip(sc.maps(0), ref)) / hs
        print(f"[sat] bucket {i}: max|d| = {err:.2e} Hs")
        assert err <= MAX_ABS
    sc.close()


def test_sat_batched_graph_eager_and_plain():
    """The batched summed-area frame (one launch over all patches, captured
    graphs) equals the same frames launched one kernel at a time bit for
    bit, and the one-patch-per-launch path within FP32 rounding."""
    cfg = wl.small_batch()
    a = sat_scene(cfg)
    b = sat_scene(cfg, batched=True)
    c = sat_scene(cfg, batched=True)
    c.set_timing(True)
    orc = OracleScene(cfg)
    hs = orc.spec.Hs()
    for f in range(1, 6):
        for s in (a, b, c):
            s.step(cfg["dt"])
        orc.step(cfg["dt"])
    bg = orc.background()
    for p in range(len(cfg["patches"])):
        ref, _ = orc.patch_maps(p, bg)
        mb = b.maps(p)
        compare_maps(mb, ref, hs, f"sat batched patch {p}")
        for x, y in zip(mb, c.maps(p)):
            assert np.array_equal(x, y)
        for x, y in zip(mb, a.maps(p)):
            assert np.abs(x.astype(np.float64) - y).max() <= 1e-5 * hs
    for s in (a, b, c):
        s.close()


def test_sat_rerun_is_deterministic():
    """Integer corner events make the sums independent of the order in
    which threads add them: two runs give identical maps."""
    cfg = wl.small_two_patches()
    a = sat_scene(cfg)
    b = sat_scene(cfg)
    for _ in range(4):
        a.step()
        b.step()
    for p in range(2):
        for u, v in zip(a.maps(p), b.maps(p)):
            assert np.array_equal(u, v)
    a.close()
    b.close()


def test_sat_empty_patch_is_background():
    """No particles: the summed-area path writes the blended background."""
    cfg = wl.scene("empty", wl.spectrum(fft_n=64, fft_L=200.0, seed=9),
                   [wl.patch(width=75, height=51, cell=0.5, max_particles=4096, prefill=0,
                             inject_scale=1e-9, origin_x=10.3, origin_y=-7.7)], frames=2)
    sc = sat_scene(cfg)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    assert sc.stats(0).live_particles == 0
    ref, ev = orc.patch_maps(0)
    assert ev == 0
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), "sat empty")
    sc.close()


def test_sat_fine_bins_many_rows_and_three_radix_passes():
    """One-cell bins: 64 + 2R bin rows per bucket and tile (more than the
    kernel's 512-row table over the item's buckets, so the buckets go in
    batches), 20-bit bin keys (three radix passes); bins bit-exact and maps
    within the contract."""
    cfg = wl.scaled(wl.small_jonswap(), bin_cells=1)
    sc = sat_scene(cfg)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    info = sc.info(0)
    assert info.bin_cells[0] == 1 and info.total_bins > 1 << 16
    compare_state(sc, orc, 0)
    compare_bins(sc, orc, 0)
    ref, _ = orc.patch_maps(0)
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), "sat one-cell bins")
    assert sc.stats(0).error_flags == 0
    sc.close()


def test_sat_bucket_rows_beyond_the_row_table():
    """One-cell bins on a 0.1 m patch whose longest bucket has R = 290
    cells: 64 + 2R = 645 bin rows of that bucket reach a tile, more than the
    summed-area kernel's 512-row table, so the kernel takes the bucket in two
    row chunks.  Bins bit-exact, maps within the contract, no error flag."""
    cfg = wl.scaled(wl.small_jonswap(), bin_cells=1, cell=0.1)
    sc = sat_scene(cfg)
    orc = OracleScene(cfg)
    sc.step(cfg["dt"])
    orc.step(cfg["dt"])
    info = sc.info(0)
    R = orc.patches[0].T.R
    assert 64 + 2 * int(R.max()) // 65536 > 512 and info.bin_cells[0] == 1
    compare_state(sc, orc, 0)
    compare_bins(sc, orc, 0)
    ref, _ = orc.patch_maps(0)
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), "sat rows beyond the table")
    assert sc.stats(0).error_flags == 0
    sc.close()


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("gmul", [0.5, 1.0, 2.0])
def test_sat_variants_and_group_plans_match_oracle(variant, gmul):
    """Both summed-area kernels (0: persistent nine-plane, 1: three-group)
    under each bucket-group multiplier the autotuner searches, in batched
    mode on the five-patch scene: maps within the contract of the oracle."""
    cfg = wl.small_batch()
    sc = sat_scene(cfg, batched=True)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc.step(cfg["dt"])
        orc.step(cfg["dt"])
    sc.set_sat_plan(variant, gmul)
    sc.step(cfg["dt"])
    orc.step(cfg["dt"])
    bg = orc.background()
    for p in range(len(cfg["patches"])):
        assert sc.info(p).sat_variant == variant
        ref, ev = orc.patch_maps(p, bg)
        assert sc.stats(p).eval_count == ev
        compare_maps(sc.maps(p), ref, orc.spec.Hs(), f"sat variant {variant} gmul {gmul} patch {p}")
    sc.close()


def test_autotune_chooses_caches_and_keeps_parity():
    """scwp_autotune times the variants and multipliers, keeps one, and a
    second context with the same workload signature takes the cached choice
    without timing; the maps stay within the contract of the oracle."""
    from paper_2511_02852_gb300 import scwp
    cfg = wl.small_batch()
    a = sat_scene(cfg, batched=True)
    orc = OracleScene(cfg)
    a.step(cfg["dt"])
    orc.step(cfg["dt"])
    rows, chosen, cached = a.autotune(reps=2, force=True)
    assert not cached and len(rows) == 6 and 0 <= chosen < len(rows)
    assert rows[chosen][2] == min(r[2] for r in rows)
    print("[autotune] small_batch: " + ", ".join(f"v{v} x{g:g}: {m:.4f} ms" for v, g, m in rows))
    a.step(cfg["dt"])
    orc.step(cfg["dt"])
    bg = orc.background()
    for p in range(len(cfg["patches"])):
        assert a.info(p).sat_variant == rows[chosen][0]
        ref, _ = orc.patch_maps(p, bg)
        compare_maps(a.maps(p), ref, orc.spec.Hs(), f"tuned patch {p}")
    b = sat_scene(cfg, batched=True)
    b.step(cfg["dt"])
    rows_b, _, cached_b = b.autotune(reps=2)
    assert cached_b and rows_b[0][:2] == rows[chosen][:2]
    a.close()
    b.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_sat_dense_patch_passes_split_into_parts(variant):
    """The densest patch of the 32-patch batched workload alone (69 x 69
    texels, 262k particles, 24 buckets: tens of bumps per texel and bucket,
    so its buckets take many passes): the plan splits each bucket's passes
    over several parts (items writing their own partial planes), and the
    maps stay within the contract of the oracle on both kernels."""
    cfg = wl.batched()
    cfg["patches"] = [cfg["patches"][9]]
    sc = sat_scene(cfg)
    sc.set_sat_plan(variant, 1.0)
    orc = OracleScene(cfg)
    sc.step(cfg["dt"])
    orc.step(cfg["dt"])
    assert sc.info(0).sat_parts > 1
    compare_state(sc, orc, 0)
    ref, ev = orc.patch_maps(0)
    assert sc.stats(0).eval_count == ev
    compare_maps(sc.maps(0), ref, orc.spec.Hs(), f"dense patch, parts {sc.info(0).sat_parts}")
    sc.close()
