"""CPU checks of the C-ABI library: it loads, exports every symbol the
header declares, and its float64 host tables (the same code scwp_add_patch
runs) match the oracle's: integer tables bit-exact, float tables to 1e-12.
No GPU calls."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import spectrum as sp
from oracle.particles import PatchTables
from paper_2511_02852_gb300 import scwp
from paper_2511_02852_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "scwp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(scwp_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = scwp.lib()
    names = header_functions()
    assert "scwp_create" in names and "scwp_step" in names
    for n in names:
        assert hasattr(L, n), n
        assert n in scwp.EXPORTS, f"binding lacks {n}"


def test_version_and_null_context_errors():
    L = scwp.lib()
    assert L.scwp_version().startswith(b"scwp")
    assert L.scwp_step(None, 1 / 60) == 1            # SCWP_E_INVALID
    L.scwp_destroy(None)


def test_invalid_descriptors_rejected_without_gpu():
    cfg = wl.tiny()
    bad = dict(cfg["spectrum"], fft_n=100)
    with pytest.raises(scwp.ScwpError):
        scwp.scwp_host_table(bad, cfg["patches"][0], 1 / 60, scwp.TAB_OMEGA)
    badp = dict(cfg["patches"][0], width=0)
    with pytest.raises(scwp.ScwpError):
        scwp.scwp_host_table(cfg["spectrum"], badp, 1 / 60, scwp.TAB_OMEGA)


SCENES = [wl.tiny, wl.realistic, wl.small_jonswap, wl.small_two_patches]


@pytest.mark.parametrize("make", SCENES, ids=lambda f: f.__name__)
@pytest.mark.parametrize("dt", [1 / 60, 1 / 30])
def test_host_tables_match_oracle(make, dt):
    cfg = make()
    spec = sp.Spectrum(cfg["spectrum"])
    for pc in cfg["patches"]:
        T = PatchTables(spec, cfg["spectrum"], pc, dt)
        get = lambda t: scwp.scwp_host_table(cfg["spectrum"], pc, dt, t)
        for tab, ref in [(scwp.TAB_OMEGA, T.b.omega), (scwp.TAB_K, T.b.k), (scwp.TAB_C, T.b.c),
                         (scwp.TAB_R, T.b.r), (scwp.TAB_E, T.b.E), (scwp.TAB_EDGES, T.b.edges),
                         (scwp.TAB_AMP, T.A.ravel())]:
            got = get(tab)
            assert np.allclose(got, ref, rtol=1e-12, atol=0), (tab, np.abs(got / ref - 1).max())
        for tab, ref in [(scwp.TAB_RQ, T.R), (scwp.TAB_VX, T.vx.ravel()), (scwp.TAB_VY, T.vy.ravel()),
                         (scwp.TAB_QX, T.qx.ravel()), (scwp.TAB_QY, T.qy.ravel()),
                         (scwp.TAB_WAKE_VX, T.wvx), (scwp.TAB_WAKE_VY, T.wvy),
                         (scwp.TAB_WAKE_QX, T.wqx), (scwp.TAB_WAKE_QY, T.wqy)]:
            got = get(tab)
            assert np.array_equal(got, ref.astype(np.int32)), tab


def test_host_tables_batched_scene_bucket_counts():
    cfg = wl.batched(n_patches=4, total_particles=40000)
    spec = sp.Spectrum(cfg["spectrum"])
    for pc in cfg["patches"]:
        T = PatchTables(spec, cfg["spectrum"], pc, 1 / 60)
        got = scwp.scwp_host_table(cfg["spectrum"], pc, 1 / 60, scwp.TAB_RQ)
        assert len(got) == pc["n_buckets"]
        assert np.array_equal(got, T.R.astype(np.int32))
