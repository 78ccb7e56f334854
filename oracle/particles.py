"""Wave-particle side of the oracle: fixed-point tables, boundary injection,
advection, expiry, wake emission and per-bucket binning.  Integer state is
int64 numpy (exact); table values are float64.  TEST INFRASTRUCTURE ONLY.

Positions are Q16.16 cell units relative to the patch origin: texel (ix, iy)
has its centre at (ix*Q + Q/2, iy*Q + Q/2), Q = 2^16.

Every float64 value that decides an integer (a rint, a floor) is computed by
a fixed sequence of IEEE operations, scalar by scalar, with the C library's
cos/sin (Python's ``math``), so that the same decision is reachable by any
other implementation that performs the same operations.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import philox4x32_10
from .spectrum import Buckets, Spectrum, amplitudes, directions

Q = 65536
HALF = 32768
S_EDGE_X, S_EDGE_Y, S_WAKE, S_PREFILL = 0, 1, 2, 3
WAKE_DIRS = 4096
DPSI = 2.0 * math.pi / WAKE_DIRS
KELVIN_ARM = math.pi / 2.0 - math.asin(1.0 / 3.0)   # 90 deg - 19.47 deg


def rint(x):
    """Round half to even (IEEE rint)."""
    return int(np.rint(x))


def texel_span(C, R, n):
    """Texels ix in [0, n) whose centre lies strictly inside (C - R, C + R)
    (integer test in Q16.16).  Returns lo, hi, count (count 0 when empty)."""
    C = np.asarray(C, dtype=np.int64)
    R = np.asarray(R, dtype=np.int64)
    lo = ((C - R - HALF) >> 16) + 1
    hi = (C + R - HALF - 1) >> 16
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, n - 1)
    return lo, hi, np.maximum(hi - lo + 1, 0)


class PatchTables:
    """Per-patch bucket and fixed-point tables (Sec. 3.2-3.3, Sec. 4.2).

    R_i   = rint(r_i / dx * Q)             kernel half-width (r = lambda/2)
    v_ij  = rint(c_i dt d_j / dx * Q)      per-frame step (phase speed c)
    q_ij  = rint(r_i d_j / dx * Q)         crest-to-trough offset
    A_ij  amplitude (Eq. A or its normalised reading) / sqrt(inject_scale)
    Wake directions (reading of Sec. 4.3): a grid of 4096 angles a*2pi/4096
    for the bucket whose radius is closest to the object's radius.
    """

    def __init__(self, spec: Spectrum, scfg, pcfg, dt):
        nb = int(pcfg.get("n_buckets", 0)) or int(scfg["n_buckets"])
        edges = scfg.get("bucket_edges")
        if edges is not None and nb != int(scfg["n_buckets"]):
            edges = None
        self.b = Buckets(spec, nb, edges, scfg["omega_lo_mul"], scfg["omega_hi_mul"])
        self.nb = nb
        self.nth = int(scfg["n_theta"])
        self.W, self.H = int(pcfg["width"]), int(pcfg["height"])
        self.dx = float(pcfg["cell"])
        scale = float(pcfg["inject_scale"])
        self.scale = scale if scale > 0 else 1.0
        self.A = amplitudes(spec, self.b, self.nth, int(scfg["amp_mode"])) \
            / math.sqrt(self.scale)
        self.theta, _, _ = directions(spec.theta_w, self.nth)
        self.cos_j = [math.cos(t) for t in self.theta]
        self.sin_j = [math.sin(t) for t in self.theta]
        dx = self.dx
        self.R = np.array([rint(self.b.r[i] / dx * Q) for i in range(nb)], dtype=np.int64)
        self.qx = np.array([[rint(self.b.r[i] * self.cos_j[j] / dx * Q)
                             for j in range(self.nth)] for i in range(nb)], dtype=np.int64)
        self.qy = np.array([[rint(self.b.r[i] * self.sin_j[j] / dx * Q)
                             for j in range(self.nth)] for i in range(nb)], dtype=np.int64)
        self.emitter = int(pcfg["emitter"])
        self.obj_radius = float(pcfg["obj_radius"])
        self.bw = int(np.argmin(np.abs(self.b.r - self.obj_radius)))
        self.wake_amp = float(pcfg["wake_amp"])
        self.wake_rate = int(pcfg["wake_rate"])
        self.obj_speed = float(pcfg["obj_speed"])
        self.obj_path_radius = float(pcfg["obj_path_radius"])
        self.heave_period = float(pcfg.get("heave_period", 0.0))
        self.ring_rate = int(pcfg.get("ring_rate", 0))
        ca = [math.cos(a * DPSI) for a in range(WAKE_DIRS)]
        sa = [math.sin(a * DPSI) for a in range(WAKE_DIRS)]
        rw = self.b.r[self.bw]
        self.wqx = np.array([rint(rw * c / dx * Q) for c in ca], dtype=np.int64)
        self.wqy = np.array([rint(rw * s / dx * Q) for s in sa], dtype=np.int64)
        self._wca, self._wsa = ca, sa
        self.dt = None
        self.set_dt(dt)

    def set_dt(self, dt):
        if dt == self.dt:
            return
        self.dt = dt
        dx, nb, nth = self.dx, self.nb, self.nth
        c = self.b.c
        self.vx = np.array([[rint(c[i] * dt * self.cos_j[j] / dx * Q) for j in range(nth)]
                            for i in range(nb)], dtype=np.int64)
        self.vy = np.array([[rint(c[i] * dt * self.sin_j[j] / dx * Q) for j in range(nth)]
                            for i in range(nb)], dtype=np.int64)
        cw = c[self.bw]
        self.wvx = np.array([rint(cw * dt * v / dx * Q) for v in self._wca], dtype=np.int64)
        self.wvy = np.array([rint(cw * dt * v / dx * Q) for v in self._wsa], dtype=np.int64)

    # per-particle lookups (direction j >= N_theta is a wake direction)
    def lookup(self, B, J):
        B = np.asarray(B, dtype=np.int64)
        J = np.asarray(J, dtype=np.int64)
        wake = J >= self.nth
        jg = np.where(wake, 0, J)
        jw = np.where(wake, J - self.nth, 0)
        vx = np.where(wake, self.wvx[jw], self.vx[B, jg])
        vy = np.where(wake, self.wvy[jw], self.vy[B, jg])
        qx = np.where(wake, self.wqx[jw], self.qx[B, jg])
        qy = np.where(wake, self.wqy[jw], self.qy[B, jg])
        A = np.where(wake, self.wake_amp, self.A[B, jg])
        return vx, vy, qx, qy, A

    def injection_rate(self, i, s):
        """Groups per frame through edge pair s of bucket i: the general form
        n = 4 L_s dt c_i / (pi r_i^2) of Eqs. 15-17 (deep water:
        4 L_s dt w^3 / (pi^3 g)); L_s = patch height (s=0, x-edges) or width
        (s=1, y-edges) in metres; times inject_scale."""
        Ls = (self.H if s == 0 else self.W) * self.dx
        c, r = self.b.c[i], self.b.r[i]
        return 4.0 * Ls * self.dt * c / (math.pi * r * r) * self.scale


class PatchState:
    """Particle pool of one patch, stepped frame by frame (Sec. 4.1 WP
    updates: inject, advect, accumulate)."""

    def __init__(self, spec: Spectrum, scfg, pcfg, patch_index, seed, dt=1.0 / 60.0):
        self.T = PatchTables(spec, scfg, pcfg, dt)
        self.p = int(patch_index)
        self.seed = int(seed)
        self.cap = int(pcfg["max_particles"])
        self.frame = 0
        self.t = 0.0
        self.carry = np.zeros((self.T.nb, 2))
        self.X = np.zeros(0, dtype=np.int64)
        self.Y = np.zeros(0, dtype=np.int64)
        self.B = np.zeros(0, dtype=np.int64)
        self.J = np.zeros(0, dtype=np.int64)
        self.injected = 0
        self.energy = np.zeros(self.T.nb)
        self.ring_carry = 0.0
        self.ring_total = 0
        self.overflow = False
        self.prefill(int(pcfg["prefill"]))

    # -- prefill (reading: the workload's particle total, distributed over the
    #    buckets in proportion to the steady state (W + 2 r_i) / r_i^2 of
    #    Eq. 15's injection over a crossing time; uniform positions over the
    #    patch grown by r_i; directions cycling over the valid grid ones).
    def prefill(self, total):
        if total <= 0:
            return
        T = self.T
        Wq, Hq = T.W * Q, T.H * Q
        w = [float(Wq + 2 * int(T.R[i])) / (float(T.R[i]) * float(T.R[i])) for i in range(T.nb)]
        sw = 0.0
        for v in w:
            sw += v
        Xs, Ys, Bs, Js = [], [], [], []
        for i in range(T.nb):
            pop = int(math.floor(float(total) * w[i] / sw + 0.5))
            valid = [j for j in range(T.nth) if T.A[i, j] > 0]
            if pop <= 0 or not valid:
                continue
            n = np.arange(pop, dtype=np.int64)
            u0, u1, _, _ = philox4x32_10(0, self.p, i | (S_PREFILL << 16), n, self.seed)
            R = int(T.R[i])
            X = -R + ((u0 * np.uint64(Wq + 2 * R)) >> np.uint64(32)).astype(np.int64)
            Y = -R + ((u1 * np.uint64(Hq + 2 * R)) >> np.uint64(32)).astype(np.int64)
            Xs.append(X)
            Ys.append(Y)
            Bs.append(np.full(pop, i, dtype=np.int64))
            Js.append(np.array(valid, dtype=np.int64)[n % len(valid)])
        self._append(np.concatenate(Xs), np.concatenate(Ys), np.concatenate(Bs),
                     np.concatenate(Js), count_injected=False)

    def _append(self, X, Y, B, J, count_injected=True):
        room = self.cap - len(self.X)
        if len(X) > room:
            self.overflow = True
            X, Y, B, J = X[:room], Y[:room], B[:room], J[:room]
        self.X = np.concatenate([self.X, X])
        self.Y = np.concatenate([self.Y, Y])
        self.B = np.concatenate([self.B, B])
        self.J = np.concatenate([self.J, J])
        if count_injected:
            self.injected += len(X)
            _, _, _, _, A = self.T.lookup(B, J)
            r = self.T.b.r[B]
            np.add.at(self.energy, B, 0.125 * A * A * math.pi * r * r)

    def bump_counts(self, X, Y, B):
        T = self.T
        R = T.R[B]
        _, _, nx = texel_span(X, R, T.W)
        _, _, ny = texel_span(Y, R, T.H)
        return nx * ny

    # -- one frame -----------------------------------------------------------
    def step(self, dt, t):
        """Frame order (reading; Sec. 4.1 names inject and advect without an
        order): (1) advect survivors by v; (2) expire particles none of whose
        two bumps has a texel centre strictly inside its support; (3) inject
        at the edges; (4) wake emission.  ``t`` is the running sum of dt."""
        T = self.T
        T.set_dt(dt)
        self.frame += 1
        self.t = t
        f = self.frame
        vx, vy, qx, qy, _ = T.lookup(self.B, self.J)
        self.X = self.X + vx
        self.Y = self.Y + vy
        alive = (self.bump_counts(self.X, self.Y, self.B) > 0) | \
            (self.bump_counts(self.X - qx, self.Y - qy, self.B) > 0)
        self.X, self.Y = self.X[alive], self.Y[alive]
        self.B, self.J = self.B[alive], self.J[alive]
        self.inject(f)
        if T.emitter:
            self.wake(f, t)
            self.ring(t)

    def inject(self, f):
        """Boundary injection (Sec. 3.3 Eqs. 15-17, Sec. 4.2).
        reading: a deterministic float64 carry per (bucket, edge pair) turns
        the fractional group count into whole groups; each group holds one
        particle per grid direction with A_ij > 0, placed on the edge of the
        pair through which that direction flows in (v_n > 0 on the inward
        normal; v_n == 0 is skipped); uniform along the edge (u0) and across
        the strip swept this frame (u1 in [0, |v_n|)); Philox counter
        (frame, patch, bucket | s<<16, group*N_theta + j)."""
        T = self.T
        Xs, Ys, Bs, Js = [], [], [], []
        for i in range(T.nb):
            for s in (S_EDGE_X, S_EDGE_Y):
                self.carry[i, s] += T.injection_rate(i, s)
                m = int(math.floor(self.carry[i, s]))
                self.carry[i, s] -= m
                if m <= 0:
                    continue
                g = np.repeat(np.arange(m, dtype=np.int64), T.nth)
                j = np.tile(np.arange(T.nth, dtype=np.int64), m)
                vn = (T.vx[i] if s == 0 else T.vy[i])[j]
                keep = (T.A[i, j] > 0) & (vn != 0)
                g, j, vn = g[keep], j[keep], vn[keep]
                if len(g) == 0:
                    continue
                u0, u1, _, _ = philox4x32_10(f, self.p, i | (s << 16), g * T.nth + j, self.seed)
                length = (T.H if s == 0 else T.W) * Q
                along = ((u0 * np.uint64(length)) >> np.uint64(32)).astype(np.int64)
                off = ((u1 * np.abs(vn).astype(np.uint64)) >> np.uint64(32)).astype(np.int64)
                far = (T.W if s == 0 else T.H) * Q
                across = np.where(vn > 0, off, far - off)
                if s == 0:
                    X, Y = across, along
                else:
                    X, Y = along, across
                Xs.append(X)
                Ys.append(Y)
                Bs.append(np.full(len(X), i, dtype=np.int64))
                Js.append(j)
        if Xs:
            self._append(np.concatenate(Xs), np.concatenate(Ys),
                         np.concatenate(Bs), np.concatenate(Js))

    def wake(self, f, t):
        """Minimal wake emitter (reading of Sec. 4.3): the object moves on a
        circle of radius R_o about the patch centre at speed V (phase
        Omega t, Omega = V / R_o, heading phase + pi/2); each frame it emits
        ``wake_rate`` particles per Kelvin arm, propagating at heading
        +/- (90 deg - 19.47 deg) (angle snapped to the 4096-direction grid),
        spawned on the object's rim in that direction with a tangential
        offset uniform in [-rho, rho); amplitude ``wake_amp``; bucket = the
        one whose radius is closest to the object's radius; Philox counter
        (frame, patch, bucket | 2<<16, arm*rate + n)."""
        T = self.T
        dx = T.dx
        Rp = T.obj_path_radius / dx
        Om = T.obj_speed / T.obj_path_radius
        phi = Om * t
        Px = T.W * 0.5 + Rp * math.cos(phi)
        Py = T.H * 0.5 + Rp * math.sin(phi)
        psi = phi + math.pi / 2.0
        rho = T.obj_radius / dx
        rate = T.wake_rate
        Xs, Ys, Js = [], [], []
        for arm, sgn in ((0, 1.0), (1, -1.0)):
            psa = psi + sgn * KELVIN_ARM
            a = int(math.floor(psa / DPSI + 0.5)) % WAKE_DIRS
            ca, sa = T._wca[a], T._wsa[a]
            ords = np.arange(rate, dtype=np.int64) + arm * rate
            u0, _, _, _ = philox4x32_10(f, self.p, T.bw | (S_WAKE << 16), ords, self.seed)
            for n in range(rate):
                tau = (float(int(u0[n])) * 2.0 ** -32 - 0.5) * 2.0 * rho
                Xs.append(rint((Px + rho * ca - tau * sa) * Q))
                Ys.append(rint((Py + rho * sa + tau * ca) * Q))
                Js.append(T.nth + a)
        n = len(Xs)
        if n:
            self._append(np.array(Xs, dtype=np.int64), np.array(Ys, dtype=np.int64),
                         np.full(n, T.bw, dtype=np.int64), np.array(Js, dtype=np.int64))

    def ring(self, t):
        """Ring ripples of the heaving object (reading of Sec. 4.3, vertical
        motion): with heave period T_h the object emits, each frame,
        ring_rate |cos(2 pi t / T_h)| particles (its heave speed relative to
        the peak), through a float64 carry capped at 64 a frame (the excess
        stays in the carry); the k-th ring particle since creation goes out
        along wake-grid direction (2531 k) mod 4096 from the rim point in that
        direction; amplitude wake_amp, the wake's bucket."""
        T = self.T
        if T.ring_rate <= 0 or T.heave_period <= 0:
            return
        dx = T.dx
        Rp = T.obj_path_radius / dx
        Om = T.obj_speed / T.obj_path_radius
        phi = Om * t
        Px = T.W * 0.5 + Rp * math.cos(phi)
        Py = T.H * 0.5 + Rp * math.sin(phi)
        rho = T.obj_radius / dx
        c = abs(math.cos(2.0 * math.pi * t / T.heave_period))
        self.ring_carry += T.ring_rate * c
        m = math.floor(self.ring_carry)
        self.ring_carry -= m
        n = int(min(m, 64.0))
        self.ring_carry += m - n
        Xs, Ys, Js = [], [], []
        for _ in range(n):
            a = (self.ring_total * 2531) % WAKE_DIRS
            self.ring_total += 1
            Xs.append(rint((Px + rho * T._wca[a]) * Q))
            Ys.append(rint((Py + rho * T._wsa[a]) * Q))
            Js.append(T.nth + a)
        if n:
            self._append(np.array(Xs, dtype=np.int64), np.array(Ys, dtype=np.int64),
                         np.full(n, T.bw, dtype=np.int64), np.array(Js, dtype=np.int64))

    # -- bumps and bins ------------------------------------------------------
    def bumps(self):
        """All bumps in id order (id = 2 p + k; k = 0 crest at p with +A,
        k = 1 trough at p - q with -A: the positive-negative pair of
        Fig. 1), with their in-patch texel counts."""
        T = self.T
        _, _, qx, qy, A = T.lookup(self.B, self.J)
        n = len(self.X)
        X = np.empty(2 * n, dtype=np.int64)
        Y = np.empty(2 * n, dtype=np.int64)
        X[0::2], X[1::2] = self.X, self.X - qx
        Y[0::2], Y[1::2] = self.Y, self.Y - qy
        B = np.repeat(self.B, 2)
        amp = np.empty(2 * n)
        amp[0::2], amp[1::2] = A, -A
        ec = self.bump_counts(X, Y, B)
        return dict(X=X, Y=Y, B=B, amp=amp, R=T.R[B], ec=ec,
                    id=np.arange(2 * n, dtype=np.int64))

    def bins(self, bin_cells):
        """Per-bucket integer bins (counts, exclusive offsets, entries).
        A bump with at least one texel in its support goes to bin
        (floor((X + R_i) / C_i), floor((Y + R_i) / C_i)), C_i = bin_cells_i*Q,
        of a grid of nbx_i x nby_i bins, nbx_i = floor((W Q + 2 R_i)/C_i) + 1;
        key = base_i + by*nbx_i + bx; entries are bump ids, stable in id
        order."""
        T = self.T
        bm = self.bumps()
        valid = bm["ec"] > 0
        C = np.asarray(bin_cells, dtype=np.int64) * Q
        nbx = (T.W * Q + 2 * T.R) // C + 1
        nby = (T.H * Q + 2 * T.R) // C + 1
        base = np.concatenate([[0], np.cumsum(nbx * nby)]).astype(np.int64)
        B = bm["B"][valid]
        bx = (bm["X"][valid] + T.R[B]) // C[B]
        by = (bm["Y"][valid] + T.R[B]) // C[B]
        key = base[B] + by * nbx[B] + bx
        order = np.argsort(key, kind="stable")
        counts = np.bincount(key, minlength=int(base[-1])).astype(np.int64)
        offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        return dict(counts=counts, offsets=offsets, entries=bm["id"][valid][order],
                    nbx=nbx, nby=nby, base=base, eval_count=int(bm["ec"].sum()),
                    bumps=bm, valid=valid)

    def live_per_bucket(self):
        return np.bincount(self.B, minlength=self.T.nb)
