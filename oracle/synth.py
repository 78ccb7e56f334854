"""Synthesis, displacement and blend of the oracle (Sec. 4.2) plus the
layered-texture variant.  Float64.  TEST INFRASTRUCTURE ONLY.

The heavy loops live in ``csynth.c`` (plain C, float64), compiled on demand
with gcc into ``oracle/_lib`` and called through ctypes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from .particles import HALF, Q

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_lib(force=False):
    """Compile csynth.c (gcc, -O2, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "csynth.c")
    if (not force and os.path.exists(_LIBPATH)
            and os.path.getmtime(_LIBPATH) >= os.path.getmtime(src)):
        return _LIBPATH
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIBPATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp",
                           "-ffp-contract=off", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build_lib())
            P = ctypes.c_void_p
            I = ctypes.c_int64
            D = ctypes.c_double
            _lib.oracle_synth.argtypes = [I, I, I, P, P, P, P, D, P, P, P, P]
            _lib.oracle_synth.restype = None
            _lib.oracle_synth_points.argtypes = [I, P, P, I, P, P, P, P, D, P, P, P]
            _lib.oracle_synth_points.restype = None
        return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def synth_maps(W, H, bumps, lam, only_valid=True):
    """WP maps (h, Dx, Dy), float64 [H, W], and the integer eval count: the
    sum over bumps of +-A k(u) k(v) (Sec. 4.2 accumulation; kernel reading
    in csynth.c)."""
    sel = bumps["ec"] > 0 if only_valid else np.ones(len(bumps["X"]), bool)
    X = np.ascontiguousarray(bumps["X"][sel], dtype=np.int64)
    Y = np.ascontiguousarray(bumps["Y"][sel], dtype=np.int64)
    R = np.ascontiguousarray(bumps["R"][sel], dtype=np.int64)
    A = np.ascontiguousarray(bumps["amp"][sel], dtype=np.float64)
    h = np.zeros((H, W))
    dx = np.zeros((H, W))
    dy = np.zeros((H, W))
    ev = np.zeros(H, dtype=np.int64)
    lib().oracle_synth(W, H, len(X), _p(X), _p(Y), _p(R), _p(A), 0.5 * lam,
                       _p(h), _p(dx), _p(dy), _p(ev))
    return h, dx, dy, int(ev.sum())


def synth_points(ix, iy, bumps, lam):
    """The same sums at selected texels only."""
    ix = np.ascontiguousarray(ix, dtype=np.int64)
    iy = np.ascontiguousarray(iy, dtype=np.int64)
    sel = bumps["ec"] > 0
    X = np.ascontiguousarray(bumps["X"][sel], dtype=np.int64)
    Y = np.ascontiguousarray(bumps["Y"][sel], dtype=np.int64)
    R = np.ascontiguousarray(bumps["R"][sel], dtype=np.int64)
    A = np.ascontiguousarray(bumps["amp"][sel], dtype=np.float64)
    n = len(ix)
    h, dx, dy = np.zeros(n), np.zeros(n), np.zeros(n)
    lib().oracle_synth_points(n, _p(ix), _p(iy), len(X), _p(X), _p(Y), _p(R), _p(A),
                              0.5 * lam, _p(h), _p(dx), _p(dy))
    return h, dx, dy


def synth_maps_numpy(W, H, bumps, lam):
    """Pure-numpy restatement of ``synth_maps`` for small cases (pins the C
    loops): every bump against every texel, support test |u|,|v| < R."""
    xt = np.arange(W, dtype=np.int64) * Q + HALF
    yt = np.arange(H, dtype=np.int64) * Q + HALF
    h = np.zeros((H, W))
    dx = np.zeros((H, W))
    dy = np.zeros((H, W))
    for X, Y, R, a in zip(bumps["X"], bumps["Y"], bumps["R"], bumps["amp"]):
        u = xt - X
        v = yt - Y
        mu = np.abs(u) < R
        mv = np.abs(v) < R
        ku = np.where(mu, 0.5 * (1 + np.cos(math.pi * u / R)), 0.0)
        kv = np.where(mv, 0.5 * (1 + np.cos(math.pi * v / R)), 0.0)
        su = np.where(mu, np.sin(math.pi * u / R), 0.0)
        sv = np.where(mv, np.sin(math.pi * v / R), 0.0)
        h += a * np.outer(kv, ku)
        dx += 0.5 * lam * a * np.outer(kv, su)
        dy += 0.5 * lam * a * np.outer(sv, ku)
    return h, dx, dy


# ---- blend (Sec. 4.2 last sentence; Sec. 3.1 local replacement) -------------
def blend_weight(W, H, band):
    """reading: w = smoothstep(0, b, d) = 3t^2 - 2t^3, t = clamp(d/b, 0, 1),
    d = distance in cells from the texel centre to the nearest patch edge;
    b = band (cells), default min(W, H)/8."""
    b = band if band > 0 else min(W, H) / 8.0
    ix = np.arange(W) + 0.5
    iy = np.arange(H) + 0.5
    dxe = np.minimum(ix, W - ix)
    dye = np.minimum(iy, H - iy)
    d = np.minimum(dye[:, None], dxe[None, :])
    t = np.clip(d / b, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def sample_background(bg, L, xw, yw):
    """reading: bilinear, periodic interpolation of the N x N background
    (grid point j at x = j L / N)."""
    N = bg.shape[0]
    fx = np.asarray(xw) * N / L
    fy = np.asarray(yw) * N / L
    x0 = np.floor(fx)
    y0 = np.floor(fy)
    a = fx - x0
    b = fy - y0
    x0 = x0.astype(np.int64) % N
    y0 = y0.astype(np.int64) % N
    x1 = (x0 + 1) % N
    y1 = (y0 + 1) % N
    return ((1 - a) * (1 - b) * bg[y0, x0] + a * (1 - b) * bg[y0, x1]
            + (1 - a) * b * bg[y1, x0] + a * b * bg[y1, x1])


def patch_world_coords(pcfg):
    W, H = int(pcfg["width"]), int(pcfg["height"])
    dx = float(pcfg["cell"])
    xw = pcfg["origin_x"] + (np.arange(W) + 0.5) * dx
    yw = pcfg["origin_y"] + (np.arange(H) + 0.5) * dx
    return np.broadcast_to(xw[None, :], (H, W)), np.broadcast_to(yw[:, None], (H, W))


def blend(pcfg, wp_maps, bg_maps, L):
    """out = w WP + (1 - w) bg for h, Dx, Dy (smooth distance-based weights,
    Sec. 4.2; the patch replaces the background inside, Sec. 3.1)."""
    W, H = int(pcfg["width"]), int(pcfg["height"])
    w = blend_weight(W, H, float(pcfg["band"]))
    xw, yw = patch_world_coords(pcfg)
    return [w * m + (1.0 - w) * sample_background(b, L, xw, yw)
            for m, b in zip(wp_maps, bg_maps)]


# ---- layered variant (Sec. 4.2: one layer per bucket, two separable passes
#      along x and y, layers summed) ----------------------------------------
def layer_taps(R):
    """Integer-offset taps of the bucket kernel: k(n) and sin(pi n Q / R) for
    |n Q| < R."""
    M = int((R - 1) // Q)
    n = np.arange(-M, M + 1, dtype=np.int64)
    t = (n * Q) / float(R)
    return n, 0.5 * (1.0 + np.cos(math.pi * t)), np.sin(math.pi * t)


def layered_maps(W, H, bumps, lam, nb, Rb):
    """reading of the layered textures: each bump's signed amplitude is
    splatted bilinearly onto its bucket's layer at texel-centre resolution
    (position (X - Q/2)/Q in texel units), each layer is filtered by the
    bucket kernel along x, then along y (h = k*k, Dx = s*k, Dy = k*s scaled
    by lambda_c / 2), and the layers are summed.  The splatted bumps are the
    binned ones (at least one texel centre inside the support), the set the
    gather sums.  Bumps exactly at texel centres give exactly the gather
    result."""
    h = np.zeros((H, W))
    dxm = np.zeros((H, W))
    dym = np.zeros((H, W))
    for i in range(nb):
        R = int(Rb[i])
        n, k, s = layer_taps(R)
        M = int(n.max()) + 2
        sel = (bumps["B"] == i) & (bumps["ec"] > 0)
        px = (bumps["X"][sel] - HALF) / Q
        py = (bumps["Y"][sel] - HALF) / Q
        amp = bumps["amp"][sel]
        x0 = np.floor(px).astype(np.int64)
        y0 = np.floor(py).astype(np.int64)
        fx = px - x0
        fy = py - y0
        Lw, Lh = W + 2 * M, H + 2 * M
        layer = np.zeros((Lh, Lw))
        for ox, oy, wgt in ((0, 0, (1 - fx) * (1 - fy)), (1, 0, fx * (1 - fy)),
                            (0, 1, (1 - fx) * fy), (1, 1, fx * fy)):
            gx = x0 + ox + M
            gy = y0 + oy + M
            ok = (gx >= 0) & (gx < Lw) & (gy >= 0) & (gy < Lh)
            np.add.at(layer, (gy[ok], gx[ok]), (amp * wgt)[ok])
        # x pass: columns 0..W-1 of the patch, all layer rows
        lx = np.zeros((Lh, W))
        lxs = np.zeros((Lh, W))
        for nn, kk, ss in zip(n, k, s):
            src = layer[:, M - nn: M - nn + W]
            lx += kk * src
            lxs += ss * src
        # y pass: rows 0..H-1
        for nn, kk, ss in zip(n, k, s):
            a = lx[M - nn: M - nn + H, :]
            b = lxs[M - nn: M - nn + H, :]
            h += kk * a
            dxm += 0.5 * lam * kk * b
            dym += 0.5 * lam * ss * a
    return h, dxm, dym


def normal_map(h, dx, dy, cell):
    """Unit normals (nx, ny, nz), float64 [3, H, W], of the displaced surface
    p(i, j) = (i c + Dx, j c + Dy, h) by finite differences (the paper
    derives normals from the height maps by finite differences, Sec. 4.2;
    the formula is this reading's): tangents by central differences inside,
    one-sided at the edges, normal = their normalised cross product."""
    h = np.asarray(h, dtype=np.float64)
    dx = np.asarray(dx, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    H, W = h.shape
    i = np.arange(W)
    il, ir = np.maximum(i - 1, 0), np.minimum(i + 1, W - 1)
    j = np.arange(H)
    jl, jr = np.maximum(j - 1, 0), np.minimum(j + 1, H - 1)
    sx = ((ir - il) * cell)[None, :] * np.ones((H, 1))
    sy = ((jr - jl) * cell)[:, None] * np.ones((1, W))
    tx = np.stack([sx + dx[:, ir] - dx[:, il], dy[:, ir] - dy[:, il], h[:, ir] - h[:, il]])
    ty = np.stack([dx[jr, :] - dx[jl, :], sy + dy[jr, :] - dy[jl, :], h[jr, :] - h[jl, :]])
    if W == 1:
        tx = np.stack([np.full((H, W), cell), np.zeros((H, W)), np.zeros((H, W))])
    if H == 1:
        ty = np.stack([np.zeros((H, W)), np.full((H, W), cell), np.zeros((H, W))])
    n = np.cross(tx, ty, axis=0)
    return n / np.linalg.norm(n, axis=0, keepdims=True)
