"""Failure detection on the GPU without a GPU fault.

Every device wait of the library is bounded: the binning sort's look-back
(decoupled look-back over the key tiles' published digit counts) gives up
after a limit, sets the frame's timeout flag, and the host reports
SCWP_E_TIMEOUT.  scwp_debug_sort_timeout runs the real sort pass with the
word of its first key tile never published (a flag that nothing sets), with
a short limit, so the wait runs out; nothing faults, traps or hangs.  The
test checks the status, that the wait took its limit, that the scene's
context is then sticky, and that the CUDA context is intact: a fresh scene
afterwards matches the FP64 oracle bit for bit in its particle state and
bins."""
import time

import pytest

from oracle.scene import OracleScene
from paper_2511_02852_gb300 import workloads as wl

from test_gpu_parity import compare_bins, compare_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_INVALID, E_TIMEOUT = 1, 5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    torch.cuda.synchronize()


def test_sort_lookback_wait_runs_out_and_reports_timeout():
    from paper_2511_02852_gb300 import scwp
    L = scwp.lib()
    cfg = wl.small_jonswap()          # 3,000 particles: 6,000 bump keys, two sort tiles
    sc = scwp.Scene(cfg, device=0)
    sc.step(cfg["dt"])
    assert 2 * sc.stats(0).live_particles > 4096
    # arguments are checked before anything is launched
    assert L.scwp_debug_sort_timeout(sc.ctx, 0, 0.0) == E_INVALID
    assert L.scwp_debug_sort_timeout(sc.ctx, 7, 0.05) == E_INVALID
    wait = 0.05
    t0 = time.perf_counter()
    rc = L.scwp_debug_sort_timeout(sc.ctx, 0, wait)
    took = time.perf_counter() - t0
    assert rc == E_TIMEOUT, scwp.STATUS.get(rc, rc)
    assert took >= 0.8 * wait, f"the wait gave up after {took:.3f} s, limit {wait} s"
    assert b"timed out" in L.scwp_last_error(sc.ctx)
    # the context is sticky: no further frame runs on it
    assert L.scwp_step(sc.ctx, cfg["dt"]) == E_TIMEOUT
    sc.close()
    # the CUDA context is intact
    one = torch.ones(1024, device="cuda")
    assert float(one.sum().item()) == 1024.0
    sc2 = scwp.Scene(cfg, device=0)
    orc = OracleScene(cfg)
    for _ in range(2):
        sc2.step(cfg["dt"])
        orc.step(cfg["dt"])
    torch.cuda.synchronize()
    st = sc2.stats(0)
    assert st.error_flags == 0
    compare_state(sc2, orc, 0)
    compare_bins(sc2, orc, 0)
    sc2.close()
