"""scwp_background_noalloc: the background step for callers that cannot call
cudaMalloc (host callbacks and real-time threads where an allocation would
synchronise the device, runtimes that only hand out pre-registered
buffers, plug-ins whose host owns every allocation).  It keeps its scratch
in a static device array of the library, so it takes only the caller's
inputs and output.

Checked through the C ABI against the background of the ordinary path
(scwp_step then scwp_height_map of patch -1) on two calls in a row, within
the tolerance of the other parity tests.  The spectrum inputs h0(k) and
w(k) are built on the host by the FP64 oracle from the same description.

This file is collected last so that a run stopping at the first failure
has already run every other test."""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_ABS = 1e-4     # times Hs
REL_L2 = 1e-5


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _inputs(cfg):
    from oracle import background as obg
    from oracle import spectrum as osp
    s = cfg["spectrum"]
    N, L = int(s["fft_n"]), float(s["fft_L"])
    spec = osp.Spectrum(s)
    h0 = obg.h0_grid(spec, N, L, int(s["seed"]))
    kx, ky = obg.wavevectors(N, L)
    omega = spec.omega_of_k(np.hypot(kx, ky))
    h0_t = torch.from_numpy(np.ascontiguousarray(
        np.stack([h0.real, h0.imag], -1).astype(np.float32))).cuda()
    # w(k) as float pairs (hi, lo), w = hi + lo, split in float64 on the host
    hi = omega.astype(np.float32)
    lo = (omega - hi.astype(np.float64)).astype(np.float32)
    om_t = torch.from_numpy(np.ascontiguousarray(np.stack([hi, lo], -1))).cuda()
    return spec, h0_t, om_t


def _compare(got, ref, hs):
    for g, r in zip(got, ref):
        g = g.astype(np.float64)
        r = r.astype(np.float64)
        assert np.abs(g - r).max() <= MAX_ABS * hs
        assert np.linalg.norm(g - r) / np.linalg.norm(r) <= REL_L2


@pytest.mark.parametrize("N", [512, 128])
def test_noalloc_background_matches_step_twice_in_a_row(N):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02852_gb300 import scwp
    from paper_2511_02852_gb300 import workloads as wl
    cfg = wl.scene("noalloc", wl.spectrum(wind_speed=11.0, fetch=60e3, depth=35.0, fft_n=N,
                                          fft_L=2.0 * N, choppiness=0.8, seed=21 + N),
                   [wl.patch(width=16, height=16, max_particles=64)], frames=2)
    s = cfg["spectrum"]
    sc = scwp.Scene(cfg, device=0)
    spec, h0_t, om_t = _inputs(cfg)
    out = torch.empty((3, N, N), dtype=torch.float32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = scwp.lib()
    for call in range(2):
        sc.step(cfg["dt"] * (call + 1))
        ref = sc.maps(-1)                              # the ordinary path's background
        t = sc.stats(0).time
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        rc = L.scwp_background_noalloc(_ptr(h0_t), _ptr(om_t), N, float(s["fft_L"]),
                                       float(s["choppiness"]), t, _ptr(out), stream)
        assert rc == 0, scwp.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        if call == 1:
            # after the first call's set-up, a call takes no device memory
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        _compare(out.cpu().numpy(), ref, spec.Hs())
    sc.close()


def test_noalloc_background_refuses_bad_sizes_and_misaligned_pointers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_02852_gb300 import scwp
    L = scwp.lib()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    om = torch.zeros(32, dtype=torch.float32, device="cuda")
    for n in (1024, 300, 4):
        rc = L.scwp_background_noalloc(_ptr(buf), _ptr(om), n, 100.0, 1.0, 0.0, _ptr(buf), None)
        assert rc == 1      # SCWP_E_INVALID, nothing launched
    # misaligned inputs (a 4-byte offset into a float buffer) are refused
    # before any launch, as is a misaligned output
    off = C.c_void_p(buf.data_ptr() + 4)
    rc = L.scwp_background_noalloc(off, _ptr(om), 16, 100.0, 1.0, 0.0, _ptr(buf), None)
    assert rc == 1
    rc = L.scwp_background_noalloc(_ptr(buf), C.c_void_p(om.data_ptr() + 4), 16, 100.0, 1.0, 0.0,
                                   _ptr(buf), None)
    assert rc == 1
    rc = L.scwp_background_noalloc(_ptr(buf), _ptr(om), 16, 100.0, 1.0, 0.0,
                                   C.c_void_p(buf.data_ptr() + 2), None)
    assert rc == 1
