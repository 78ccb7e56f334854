"""Seeded synthetic workloads shared by the tests, the bench and the oracle.

This module only *describes* scenes (spectrum parameters, patch geometry,
seeds, frame counts).  It holds none of the method's arithmetic: every
number the method derives from these parameters (spectra, buckets,
injection counts, particle positions, heights) is computed separately by the
CUDA library and by the FP64 oracle.

The scenes follow the shapes the paper states for its own experiments
(Sec. 5.2 defaults: N_omega = N_theta = 16, U10 in {3,5,10,15}, patch
resolutions 256^2..1024^2) and the five evaluation configurations of the
hybrid-ocean synthesis path (tiny, realistic, batched, mixed-large,
serving).  No public dataset is involved; every input is synthetic.
"""
from __future__ import annotations

import copy
import math

import numpy as np

JONSWAP = 0
PHILLIPS = 1
COS2S_MITSUYASU = 0
COS2 = 1
AMP_NORMALIZED = 0
AMP_LITERAL = 1


def spectrum(**kw):
    """A spectrum/background description with the library defaults."""
    d = dict(
        spectrum=JONSWAP, spreading=COS2S_MITSUYASU,
        wind_speed=10.0, fetch=100e3, depth=0.0, wind_dir=0.0, gamma=0.0,
        n_buckets=16, n_theta=16, bucket_edges=None,
        omega_lo_mul=0.5, omega_hi_mul=2.5, amp_mode=AMP_NORMALIZED,
        fft_n=64, fft_L=256.0, choppiness=1.0, seed=0,
    )
    d.update(kw)
    return d


def patch(**kw):
    """A wave-particle patch description with the library defaults."""
    d = dict(
        origin_x=0.0, origin_y=0.0, cell=0.25, width=128, height=128,
        band=0.0, max_particles=0, prefill=0, inject_scale=1.0, bin_cells=0,
        emitter=0, obj_radius=4.0, obj_speed=8.0, obj_path_radius=20.0,
        wake_amp=0.05, wake_rate=2, n_buckets=0, heave_period=0.0, ring_rate=0,
    )
    d.update(kw)
    return d


def scene(name, spec, patches, frames, dt=1.0 / 60.0, **extra):
    s = dict(name=name, spectrum=spec, patches=patches, frames=frames, dt=dt)
    s.update(extra)
    return s


# -- tiny: Phillips U=10, cos^2 spreading, deep water, 64^2 FFT over 256 m,
#    one 128^2 patch at 0.5 m, four log-spaced buckets 0.5..4 rad/s,
#    2,000 prefilled particles, 60 frames at 1/60 s, seed 0.
def tiny():
    edges = [0.5 * 8.0 ** (e / 4.0) for e in range(5)]
    spec = spectrum(spectrum=PHILLIPS, spreading=COS2, wind_speed=10.0,
                    depth=0.0, n_buckets=4, bucket_edges=edges, n_theta=16,
                    fft_n=64, fft_L=256.0, seed=0)
    p = patch(origin_x=-32.0, origin_y=-32.0, cell=0.5, width=128, height=128,
              max_particles=65536, prefill=2000, inject_scale=1.0)
    return scene("tiny", spec, [p], frames=60)


# -- realistic: JONSWAP U10=15 m/s, fetch 100 km, gamma 3.3, depth 50 m,
#    512^2 FFT over 1 km; one 1024^2 patch at 0.25 m around an object on a
#    20 m circle at 8 m/s that emits wake particles; 16 equal-energy
#    buckets, about 200k live particles; 600 frames.
REALISTIC_INJECT_SCALE = 1.9


def realistic():
    spec = spectrum(spectrum=JONSWAP, spreading=COS2S_MITSUYASU,
                    wind_speed=15.0, fetch=100e3, gamma=3.3, depth=50.0,
                    n_buckets=16, n_theta=16, fft_n=512, fft_L=1000.0, seed=0)
    p = patch(origin_x=-128.0, origin_y=-128.0, cell=0.25, width=1024,
              height=1024, max_particles=400000, prefill=200000,
              inject_scale=REALISTIC_INJECT_SCALE, emitter=1,
              obj_radius=10.0, obj_speed=8.0, obj_path_radius=20.0,
              wake_amp=0.05, wake_rate=2)
    return scene("realistic", spec, [p], frames=600)


# -- small parity scenes: same method, sizes the oracle finishes in seconds,
#    spanning several synthesis tiles with ragged tails.
def small_jonswap(seed=3):
    spec = spectrum(spectrum=JONSWAP, wind_speed=12.0, fetch=50e3, gamma=0.0,
                    depth=30.0, n_buckets=6, n_theta=12, fft_n=128,
                    fft_L=300.0, choppiness=0.8, seed=seed)
    p = patch(origin_x=17.3, origin_y=-40.1, cell=0.5, width=200, height=136,
              max_particles=60000, prefill=3000, inject_scale=2.0, emitter=1,
              obj_radius=6.0, obj_speed=6.0, obj_path_radius=15.0,
              wake_amp=0.04, wake_rate=3)
    return scene("small_jonswap", spec, [p], frames=12)


def small_two_patches(seed=5):
    spec = spectrum(spectrum=JONSWAP, wind_speed=9.0, fetch=30e3, gamma=2.0,
                    depth=0.0, n_buckets=5, n_theta=8, wind_dir=0.7,
                    fft_n=64, fft_L=200.0, seed=seed)
    pa = patch(origin_x=-30.0, origin_y=12.0, cell=0.5, width=96, height=160,
               max_particles=40000, prefill=1500, inject_scale=1.5)
    pb = patch(origin_x=55.0, origin_y=-70.0, cell=0.25, width=72, height=72,
               max_particles=40000, prefill=800, inject_scale=0.5, emitter=1,
               obj_radius=3.0, obj_speed=4.0, obj_path_radius=5.0,
               wake_amp=0.03, wake_rate=1)
    return scene("small_two_patches", spec, [pa, pb], frames=8)


# -- small_batch: a parity-sized batched frame: 5 patches of uneven sides
#    (48..200 cells, ragged against the 64-texel tiles), 3-9 equal-energy
#    buckets each, 300-3000 prefilled particles, three with wakes; one
#    spectrum; patch draws from seed 7.
def small_batch(n_patches=5, seed=7):
    rng = np.random.default_rng(seed)
    sides = rng.integers(48, 201, size=(n_patches, 2))
    counts = np.round(np.exp(rng.uniform(math.log(300), math.log(3000), n_patches))).astype(int)
    nbs = rng.integers(3, 10, n_patches)
    spec = spectrum(spectrum=JONSWAP, wind_speed=10.0, fetch=50e3, gamma=3.3,
                    depth=40.0, n_buckets=6, n_theta=8, wind_dir=0.3,
                    fft_n=128, fft_L=300.0, seed=seed)
    ps = []
    for i in range(n_patches):
        ps.append(patch(origin_x=float(rng.uniform(-100, 100)), origin_y=float(rng.uniform(-100, 100)),
                        cell=0.25 if i % 2 else 0.5, width=int(sides[i, 0]), height=int(sides[i, 1]),
                        max_particles=int(4 * counts[i] + 2048), prefill=int(counts[i]),
                        inject_scale=1.0, emitter=1 if i < 3 else 0, obj_radius=2.0,
                        obj_speed=3.0 + i, obj_path_radius=4.0, wake_amp=0.03, wake_rate=1,
                        n_buckets=int(nbs[i])))
    return scene("small_batch", spec, ps, frames=6)


# -- batched: 1024^2 FFT over 1 km; 32 patches, sides log-uniform in
#    [64, 1024] cells at 0.25 m, 8-32 equal-energy buckets each (drawn per
#    patch; all patches share one spectrum), 10k-500k particles
#    each (log-uniform, rescaled to a 4M total), object speeds U(0, 12) m/s;
#    300 frames; patch draws from seed 1.
def batched(n_patches=32, total_particles=4_000_000, seed=1):
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(math.log(64), math.log(1024), n_patches))
    sides = np.clip(np.round(sides).astype(int), 64, 1024)
    counts = np.exp(rng.uniform(math.log(1e4), math.log(5e5), n_patches))
    counts = np.maximum(1, np.round(counts * total_particles / counts.sum()))
    speeds = rng.uniform(0.0, 12.0, n_patches)
    nbs = rng.integers(8, 33, n_patches)
    ox = rng.uniform(-400.0, 400.0, n_patches)
    oy = rng.uniform(-400.0, 400.0, n_patches)
    spec = spectrum(spectrum=JONSWAP, wind_speed=12.0, fetch=100e3,
                    gamma=3.3, depth=0.0, n_buckets=16, n_theta=16,
                    fft_n=1024, fft_L=1000.0, seed=seed)
    ps = []
    for i in range(n_patches):
        side = int(sides[i])
        ps.append(patch(origin_x=float(ox[i]), origin_y=float(oy[i]),
                        cell=0.25, width=side, height=side,
                        max_particles=int(counts[i] * 2 + 4096),
                        prefill=int(counts[i]), inject_scale=1.0,
                        emitter=1 if speeds[i] > 0.5 else 0,
                        obj_radius=4.0, obj_speed=float(max(speeds[i], 0.5)),
                        obj_path_radius=min(20.0, side * 0.25 * 0.3),
                        wake_amp=0.05, wake_rate=2, n_buckets=int(nbs[i])))
    return scene("batched", spec, ps, frames=300)


# -- mixed_large: 2048^2 FFT over 4 km; 8 patches of 1024^2 cells at 0.25 m,
#    2M particles each, 32 equal-energy buckets; JONSWAP U10 = 15 m/s at a
#    100 km fetch, gamma 3.3, depth 50 m (the realistic sea, which the scene
#    list leaves open); no wakes; patch origins from seed 2.
def mixed_large(n_patches=8, particles=2_000_000, seed=2):
    rng = np.random.default_rng(seed)
    spec = spectrum(spectrum=JONSWAP, wind_speed=15.0, fetch=100e3, gamma=3.3, depth=50.0,
                    n_buckets=32, n_theta=16, fft_n=2048, fft_L=4000.0, seed=seed)
    ps = [patch(origin_x=float(rng.uniform(-1500.0, 1200.0)), origin_y=float(rng.uniform(-1500.0, 1200.0)),
                cell=0.25, width=1024, height=1024, max_particles=int(2 * particles + 4096),
                prefill=int(particles), inject_scale=float(particles) / 200000.0 * 1.9)
          for _ in range(n_patches)]
    return scene("mixed_large", spec, ps, frames=300)


# -- serving: 64 independent scenes: FFT 256^2..1024^2 (log-uniform powers
#    of two), JONSWAP U10 uniform in 5..20 m/s at a 100 km fetch, 1..16
#    patches with sides log-uniform in 64..512 cells, 1e4..1e6 particles per
#    scene (log-uniform, split over the patches by area), 8..16 buckets.
#    Unstated by the scene list and chosen here: the cell is about 1/48 of
#    the scene's peak wavelength (so kernel radii in cells stay alike across
#    winds) and the FFT domain about N/32 peak wavelengths; both are given
#    per scene in the table below (metres, 6 significant digits), in scene
#    order.  Scenes from seed 3.
_SERVING_GEOMETRY = [  # (cell, fft_L) of scene s
    (0.926961, 355.953),
    (1.20053, 922.005),
    (1.92556, 739.417),
    (1.69859, 652.26),
    (1.28292, 985.282),
    (1.27145, 488.237),
    (1.65519, 1271.18),
    (1.90589, 2927.45),
    (1.73344, 1331.28),
    (1.99411, 765.736),
    (1.88116, 1444.73),
    (0.86713, 1331.91),
    (1.37671, 1057.31),
    (1.3107, 1006.61),
    (1.47351, 1131.66),
    (1.79633, 2759.16),
    (1.98574, 762.523),
    (1.39382, 1070.45),
    (0.983635, 755.432),
    (1.24957, 479.835),
    (1.473, 565.633),
    (1.7648, 1355.37),
    (1.70401, 654.341),
    (1.32105, 1014.57),
    (1.27053, 975.77),
    (1.75087, 672.334),
    (1.97698, 1518.32),
    (1.5455, 593.472),
    (1.3304, 2043.49),
    (2.00299, 1538.29),
    (1.56826, 1204.42),
    (1.96553, 754.762),
    (1.87275, 1438.27),
    (2.00168, 768.646),
    (1.77083, 1360.0),
    (1.36538, 2097.22),
    (0.825969, 634.344),
    (0.799807, 307.126),
    (1.6465, 1264.51),
    (1.15801, 889.354),
    (1.87094, 718.44),
    (0.891995, 342.526),
    (1.57852, 2424.61),
    (1.82119, 2797.35),
    (1.7726, 1361.36),
    (1.82296, 1400.04),
    (0.796395, 1223.26),
    (1.84092, 1413.83),
    (0.844907, 648.889),
    (1.98479, 3048.64),
    (1.3332, 511.95),
    (1.50428, 577.645),
    (1.65393, 635.109),
    (1.26566, 1944.05),
    (1.21818, 935.563),
    (1.40513, 1079.14),
    (1.42287, 546.384),
    (1.03315, 793.458),
    (1.52842, 2347.65),
    (1.86352, 2862.37),
    (1.01395, 778.713),
    (1.60536, 1232.92),
    (1.0739, 1649.51),
    (1.6104, 1236.79)
]


def serving(n_scenes=64, seed=3):
    if seed != 3 or n_scenes > len(_SERVING_GEOMETRY):
        raise ValueError("the serving geometry table covers the 64 scenes of seed 3")
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_scenes):
        U = float(rng.uniform(5.0, 20.0))
        N = int(2 ** int(round(rng.uniform(8.0, 10.0))))
        cell, L = _SERVING_GEOMETRY[s]
        n_p = int(rng.integers(1, 17))
        total = float(np.exp(rng.uniform(math.log(1e4), math.log(1e6))))
        sides = np.clip(np.round(np.exp(rng.uniform(math.log(64), math.log(512), size=(n_p, 2)))), 64, 512)
        area = sides[:, 0] * sides[:, 1]
        nb = int(rng.integers(8, 17))
        spec = spectrum(spectrum=JONSWAP, wind_speed=U, fetch=100e3, gamma=3.3, depth=0.0,
                        n_buckets=nb, n_theta=16, fft_n=N, fft_L=L, seed=1000 + s)
        ps = []
        for k in range(n_p):
            cnt = max(1, int(round(total * area[k] / area.sum())))
            ps.append(patch(origin_x=float(rng.uniform(-0.25 * L, 0.25 * L)),
                            origin_y=float(rng.uniform(-0.25 * L, 0.25 * L)),
                            cell=cell, width=int(sides[k, 0]), height=int(sides[k, 1]),
                            max_particles=int(2 * cnt + 4096), prefill=cnt, inject_scale=1.0,
                            emitter=0))
        out.append(scene(f"serving{s}", spec, ps, frames=1))
    return out


# -- sweep points (the paper's Table 2 axes; its numbers are Unity frame
#    rates, context only): one 128 m patch of res^2 texels (cell 128/res),
#    an FFT of res^2 over 512 m, JONSWAP at a 100 km fetch, (n_omega,
#    n_theta) buckets x directions; 100k prefilled particles, injection at
#    the steady-state rate.
def sweep_point(n_omega=16, n_theta=16, u10=10.0, res=512, seed=5):
    spec = spectrum(spectrum=JONSWAP, wind_speed=float(u10), fetch=100e3, gamma=3.3, depth=0.0,
                    n_buckets=int(n_omega), n_theta=int(n_theta), fft_n=int(res), fft_L=512.0, seed=seed)
    p = patch(origin_x=-64.0, origin_y=-64.0, cell=128.0 / res, width=int(res), height=int(res),
              max_particles=400000, prefill=100000, inject_scale=1.0)
    return scene(f"sweep_{n_omega}x{n_theta}_u{u10:g}_r{res}", spec, [p], frames=25)


def sweep_points():
    pts = [dict(n_omega=a, n_theta=b, u10=10.0, res=512) for a in (8, 12, 16) for b in (8, 12, 16)]
    pts += [dict(n_omega=16, n_theta=16, u10=u, res=512) for u in (3.0, 5.0, 15.0)]
    pts += [dict(n_omega=16, n_theta=16, u10=10.0, res=r) for r in (256, 1024)]
    return pts


def serving_arrivals(rate=2000.0, seconds=60.0, n_scenes=64, seed=4):
    """Poisson frame-step requests: (arrival time in s, scene index)."""
    rng = np.random.default_rng(seed)
    n = int(rate * seconds * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    t = t[t < seconds]
    return t, rng.integers(0, n_scenes, len(t))


def scaled(sc, **patch_overrides):
    """A copy of a scene with every patch's fields overridden."""
    out = copy.deepcopy(sc)
    for p in out["patches"]:
        p.update(patch_overrides)
    return out


def mixed_large_1():
    """The first patch of mixed_large alone (its 2048^2 background, one
    1024^2 patch of 2M particles): the size for one-launch kernel profiles."""
    sc = mixed_large(n_patches=1)
    sc["name"] = "mixed_large_1"
    return sc


ALL = {"tiny": tiny, "realistic": realistic, "small_jonswap": small_jonswap,
       "small_two_patches": small_two_patches, "small_batch": small_batch, "batched": batched,
       "mixed_large": mixed_large, "mixed_large_1": mixed_large_1}
