"""The frame-step server (scwp_server_*) through the C ABI: each scene's
result is the same alone and in a mix of scenes, admission follows the
device-memory budget, and a scene's requests complete in order."""
import numpy as np
import pytest

from paper_2511_02852_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    torch.cuda.synchronize()


def _mix():
    return [wl.small_jonswap(), wl.small_two_patches(), wl.small_batch(), wl.tiny()]


def _drain(sv, want):
    done = []
    for _ in range(100000):
        sv.tick()
        done += sv.poll()
        if len(done) >= want:
            return done
    raise AssertionError(f"only {len(done)} of {want} requests completed")


@pytest.mark.parametrize("modes", ["sat", "gather", "mixed"])
def test_each_scene_same_alone_and_in_the_mix(modes):
    """Scenes on the summed-area synthesis (the default), on the tensor-core
    gather, or both in the same ticks (two synthesis launches a tick)."""
    from paper_2511_02852_gb300 import scwp
    cfgs = _mix()
    frames = [3, 2, 4, 5]
    mode = [scwp.SYNTH_SAT if modes == "sat" or (modes == "mixed" and k % 2 == 0) else scwp.SYNTH_GATHER
            for k in range(len(cfgs))]
    sv = scwp.Server(max_inflight=3)
    ids = [sv.add_scene(c) for c in cfgs]
    assert all(i is not None for i in ids)
    for s, m in zip(ids, mode):
        sv.scene(s).set_synth_mode(m)
    rid = 0
    order = {}
    # interleaved submissions: the scenes share ticks
    for f in range(max(frames)):
        for s, c in zip(ids, cfgs):
            if f < frames[ids.index(s)]:
                sv.submit(s, c["dt"], rid)
                order.setdefault(s, []).append(rid)
                rid += 1
    done = _drain(sv, rid)
    assert sorted(done) == list(range(rid))
    for s in ids:   # a scene's requests complete in submission order
        pos = [done.index(r) for r in order[s]]
        assert pos == sorted(pos)
    info = sv.info()
    assert info.requests_done == rid and info.ticks_launched >= max(frames)
    torch.cuda.synchronize()
    for s, c, n, m in zip(ids, cfgs, frames, mode):
        alone = scwp.Scene(c)
        alone.set_batched(True)
        alone.set_synth_mode(m)
        for _ in range(n):
            alone.step(c["dt"])
        view = sv.scene(s)
        for p in range(len(c["patches"])):
            xa, ya, ba = alone.particles(p)
            xm, ym, bm = view.particles(p)
            assert np.array_equal(xa, xm) and np.array_equal(ya, ym) and np.array_equal(ba, bm)
            for a, m in zip(alone.maps(p), view.maps(p)):
                assert np.array_equal(a, m), f"scene {s} patch {p}"
            assert alone.stats(p).eval_count == view.stats(p).eval_count
        alone.close()
    sv.close()


@pytest.mark.parametrize("mode_name", ["SYNTH_SAT", "SYNTH_GATHER"])
def test_scenes_served_in_a_mix_match_the_oracle(mode_name):
    """Every scene of a mix served in shared ticks against the FP64 oracle
    stepped alone: particle state and bins bit-exact, maps within the
    contract (max |d| <= 1e-4 Hs, relative L2 <= 1e-5)."""
    from oracle.scene import OracleScene
    from paper_2511_02852_gb300 import scwp
    from test_gpu_parity import compare_bins, compare_maps, compare_state
    cfgs = _mix()
    frames = [4, 3, 2, 5]
    sv = scwp.Server(max_inflight=3)
    ids = [sv.add_scene(c) for c in cfgs]
    assert all(i is not None for i in ids)
    for s in ids:
        sv.scene(s).set_synth_mode(getattr(scwp, mode_name))
    rid = 0
    for f in range(max(frames)):
        for k, (s, c) in enumerate(zip(ids, cfgs)):
            if f < frames[k]:
                sv.submit(s, c["dt"], rid)
                rid += 1
    _drain(sv, rid)
    torch.cuda.synchronize()
    for s, c, n in zip(ids, cfgs, frames):
        orc = OracleScene(c)
        for _ in range(n):
            orc.step(c["dt"])
        view = sv.scene(s)
        bg = orc.background()
        for p in range(len(c["patches"])):
            compare_state(view, orc, p)
            compare_bins(view, orc, p)
            ref, ev = orc.patch_maps(p, bg)
            assert view.stats(p).eval_count == ev
            compare_maps(view.maps(p), ref, orc.spec.Hs(), f"served {c['name']} patch {p}")
    sv.close()


def test_admission_follows_the_memory_budget():
    from paper_2511_02852_gb300 import scwp
    a, b = wl.small_jonswap(), wl.small_two_patches()
    probe = scwp.Server()
    ia = probe.add_scene(a)
    need_a = probe.info().device_bytes
    ib = probe.add_scene(b)
    need_b = probe.info().device_bytes - need_a
    probe.close()
    assert ia is not None and ib is not None and need_a > 0 and need_b > 0
    sv = scwp.Server(hbm_budget_bytes=need_a + need_b // 2)
    s0 = sv.add_scene(a)
    assert s0 is not None
    assert sv.add_scene(b) is None             # would exceed the budget
    assert sv.info().scenes == 1 and sv.info().device_bytes <= need_a + need_b // 2
    sv.submit(s0, a["dt"], 7)
    assert _drain(sv, 1) == [7]
    sv.remove_scene(s0)                         # memory frees up: the other scene fits
    s1 = sv.add_scene(b)
    assert s1 is not None and sv.info().scenes == 1
    sv.submit(s1, b["dt"], 8)
    assert _drain(sv, 1) == [8]
    sv.close()
