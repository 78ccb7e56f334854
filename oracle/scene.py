"""A whole hybrid-ocean scene stepped by the oracle (Sec. 4.1 pipeline:
FFT background update, WP inject/advect/accumulate, blend).  Float64.
TEST INFRASTRUCTURE ONLY."""
from __future__ import annotations

import numpy as np

from . import background as bgm
from .particles import PatchState
from .spectrum import Spectrum
from .synth import blend, layered_maps, synth_maps


class OracleScene:
    def __init__(self, scene_cfg, dt=None):
        self.cfg = scene_cfg
        sc = scene_cfg["spectrum"]
        self.scfg = sc
        self.spec = Spectrum(sc)
        self.N = int(sc["fft_n"])
        self.L = float(sc["fft_L"])
        self.lam = float(sc["choppiness"])
        self.seed = int(sc["seed"])
        self._h0 = None
        dt = scene_cfg.get("dt", 1.0 / 60.0) if dt is None else dt
        self.patches = [PatchState(self.spec, sc, p, i, self.seed, dt)
                        for i, p in enumerate(scene_cfg["patches"])]
        self.frame = 0
        self.t = 0.0

    @property
    def h0(self):
        if self._h0 is None:
            self._h0 = bgm.h0_grid(self.spec, self.N, self.L, self.seed)
        return self._h0

    def step(self, dt):
        """reading: t is the running float64 sum of the dt sequence."""
        self.frame += 1
        self.t += dt
        for ps in self.patches:
            ps.step(dt, self.t)

    def background(self):
        h, dx, dy, _ = bgm.background(self.spec, self.h0, self.L, self.t, self.lam)
        return h, dx, dy

    def wp_maps(self, p):
        ps = self.patches[p]
        bm = ps.bumps()
        return synth_maps(ps.T.W, ps.T.H, bm, self.lam)

    def patch_maps(self, p, bg=None, layered=False, buckets=None):
        """Blended (h, Dx, Dy) of patch p and its eval count.  buckets =
        (lo, hi): only the bumps of buckets lo <= i < hi enter the WP sum (a
        selection for per-bucket error statements; the sums are unchanged)."""
        ps = self.patches[p]
        bm = ps.bumps()
        if buckets is not None:
            sel = (bm["B"] >= buckets[0]) & (bm["B"] < buckets[1])
            bm = {k: (v[sel] if isinstance(v, np.ndarray) and len(v) == len(sel) else v) for k, v in bm.items()}
        if layered:
            wp = layered_maps(ps.T.W, ps.T.H, bm, self.lam, ps.T.nb, ps.T.R)
            ev = int(bm["ec"].sum())
        else:
            h, dx, dy, ev = synth_maps(ps.T.W, ps.T.H, bm, self.lam)
            wp = (h, dx, dy)
        if bg is None:
            bg = self.background()
        return blend(self.cfg["patches"][p], wp, bg, self.L), ev
