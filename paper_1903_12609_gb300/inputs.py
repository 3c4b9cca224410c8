"""Seeded synthetic inputs for the filament-suspension workloads.

This module draws random numbers and lays out plain geometry only. It holds
none of the method's arithmetic (no RPY tensor, no quaternion, no residual),
so both the CUDA path and the oracle can take their inputs from it without
sharing any computation.

Workloads (shapes follow the paper's experiments; no dataset is involved):

* ``mobility_inputs`` -- mobility apply alone: M filaments of N segments, each
  centreline a random walk with a fixed bond length (2.2a), filament centroids
  uniform in a cube sized for a given volume fraction, forces and torques
  i.i.d. N(0, 1) per component.
* ``cloud_frames`` -- isotropic cloud of straight filaments (App. A.5): uniform
  base points in a cube, uniformly random orientations, overlapping filaments
  redrawn. Orientations are returned as an orthonormal pair (tangent t,
  normal mu) per filament, drawn uniformly on SO(3); each side builds the
  quaternion from the pair itself (App. A.1).
* ``single_filament`` -- one straight filament tilted 45 degrees from the
  vertical with a seeded small Lie-algebra perturbation per segment.

``workload_params`` turns the dimensionless settings of a workload (number of
segments, elasto-gravitational number B, time step as a fraction of the
settling time T = eta L / W) into the physical parameters.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def box_side(n_segments: int, volume_fraction: float, a: float = 1.0) -> float:
    """Cube side for n spheres of radius a at the given volume fraction."""
    return (n_segments * (4.0 / 3.0) * math.pi * a ** 3 / volume_fraction) ** (1.0 / 3.0)


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def mobility_inputs(n_fil: int = 100, n_seg: int = 32, bond: float = 2.2,
                    volume_fraction: float = 0.05, a: float = 1.0, seed: int = 0):
    """Random-walk filaments and N(0,1) forces/torques.

    Returns (Y, FT): Y is (S, 3) float64 centres, FT is (S, 6) float64 with
    the force in columns 0-2 and the torque in columns 3-5, S = n_fil*n_seg.
    """
    rng = np.random.default_rng(seed)
    S = n_fil * n_seg
    side = box_side(S, volume_fraction, a)
    Y = np.empty((S, 3))
    for i in range(n_fil):
        steps = _unit_vectors(rng, n_seg - 1) * bond
        walk = np.zeros((n_seg, 3))
        if n_seg > 1:
            walk[1:] = np.cumsum(steps, axis=0)
        centre = rng.uniform(0.0, side, size=3)
        Y[i * n_seg:(i + 1) * n_seg] = walk - walk.mean(axis=0) + centre
    FT = rng.standard_normal((S, 6))
    return Y, FT


def random_frames(rng: np.random.Generator, n: int):
    """n orthonormal (t, mu) pairs, uniformly distributed on SO(3)."""
    t = _unit_vectors(rng, n)
    g = rng.standard_normal((n, 3))
    g -= np.sum(g * t, axis=1, keepdims=True) * t
    mu = g / np.linalg.norm(g, axis=1, keepdims=True)
    return t, mu


def cloud_frames(n_fil: int, n_seg, dL: float = 2.2, volume_fraction: float = 0.02,
                 a: float = 1.0, seed: int = 0, max_tries: int = 1000, rng=None):
    """Isotropic cloud of straight filaments with no overlapping segments.

    n_seg: segments per filament (an int, or a list of n_fil counts). Returns
    (base, t, mu, side): base (M, 3) positions of the s = 0 ends, t and mu
    (M, 3) tangent and normal of each filament, and the cube side. Segment n of
    filament i sits at base[i] + n*dL*t[i] (n = 0..N_i-1); a filament whose
    segments come closer than 2a to an accepted filament is redrawn.
    """
    rng = np.random.default_rng(seed) if rng is None else rng
    segs = [int(n_seg)] * n_fil if np.isscalar(n_seg) else [int(n) for n in n_seg]
    side = box_side(sum(segs), volume_fraction, a)
    cell = 2.0 * a
    grid: dict = {}
    base = np.empty((n_fil, 3))
    tt = np.empty((n_fil, 3))
    mm = np.empty((n_fil, 3))
    for i in range(n_fil):
        offs = np.arange(segs[i])[:, None] * dL
        for _ in range(max_tries):
            b = rng.uniform(0.0, side, size=3)
            t, mu = random_frames(rng, 1)
            pts = b[None, :] + offs * t
            keys = np.floor(pts / cell).astype(np.int64)
            clash = False
            for p, k in zip(pts, keys):
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            for q in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                                if np.sum((p - q) ** 2) < (2.0 * a) ** 2:
                                    clash = True
                                    break
                            if clash:
                                break
                        if clash:
                            break
                    if clash:
                        break
                if clash:
                    break
            if not clash:
                break
        else:
            raise RuntimeError("cloud_frames: could not place filament %d" % i)
        for p, k in zip(pts, keys):
            grid.setdefault((int(k[0]), int(k[1]), int(k[2])), []).append(p)
        base[i], tt[i], mm[i] = b, t[0], mu[0]
    return base, tt, mm, side


def single_filament(n_seg: int = 20, tilt_deg: float = 45.0, perturbation: float = 1e-3,
                    seed: int = 0):
    """One straight filament tilted from the vertical, plus a seeded perturbation.

    Returns (base, t, mu, xi): base (1, 3), tangent and normal (1, 3) and the
    per-segment Lie-algebra perturbation xi (N, 3) ~ perturbation * N(0, 1).
    """
    rng = np.random.default_rng(seed)
    th = math.radians(tilt_deg)
    t = np.array([[math.sin(th), 0.0, math.cos(th)]])
    mu = np.array([[0.0, 1.0, 0.0]])
    xi = perturbation * rng.standard_normal((n_seg, 3))
    return np.zeros((1, 3)), t, mu, xi


@dataclass
class Workload:
    """Physical parameters of a filament workload (a = 1 units)."""
    n_fil: int
    seg_per_fil: list
    a: float = 1.0
    eta: float = 1.0
    dL: float = 2.2
    KB: float = 1.0
    KT: float = 1.0
    W: float = 1.0
    dt: float = 0.01
    tol: float = 1e-4
    max_iter: int = 50
    extra: dict = field(default_factory=dict)


def workload_params(n_fil: int, n_seg: int, B: float = 1000.0, dt_over_T: float = 0.01,
                    tol: float = 1e-4, a: float = 1.0, eta: float = 1.0, dL: float = 2.2,
                    W: float = 1.0, KT_over_KB: float = 1.0, max_iter: int = 50) -> Workload:
    """Elasto-gravitational number B = L^3 W / K_B, settling time T = eta L / W."""
    L = n_seg * dL
    KB = L ** 3 * W / B
    T = eta * L / W
    return Workload(n_fil=n_fil, seg_per_fil=[n_seg] * n_fil, a=a, eta=eta, dL=dL, KB=KB,
                    KT=KT_over_KB * KB, W=W, dt=dt_over_T * T, tol=tol, max_iter=max_iter,
                    extra={"L": L, "T": T, "B": B})


def suspension(n_fil: int = 1000, n_seg: int = 32, seed: int = 0, volume_fraction: float = 0.02):
    """The suspension workload: n_fil straight filaments of n_seg segments in a
    cube at the given volume fraction (cloud_frames), half sedimenting passive
    filaments (gravity -W dL per segment, B = 1000) and half active filaments
    driven by a compressive tip follower force f with f L^2 / K_B = 100 (no
    weight); BDF2 with dt = T/200, Broyden tolerance 1e-4.
    Returns (Workload, base, t, mu, Fext [S x 3], follower [n_fil])."""
    wl = workload_params(n_fil, n_seg, B=1000.0, dt_over_T=1.0 / 200.0, tol=1e-4, max_iter=60)
    base, t, mu, _ = cloud_frames(n_fil, n_seg, dL=wl.dL, volume_fraction=volume_fraction,
                                  seed=seed)
    S = n_fil * n_seg
    passive = np.arange(n_fil) < n_fil // 2
    Fext = np.zeros((S, 3))
    Fext[np.repeat(passive, n_seg), 2] = -wl.W * wl.dL
    L = wl.extra["L"]
    follower = np.where(passive, 0.0, 100.0 * wl.KB / L ** 2)
    return wl, base, t, mu, Fext, follower


def ensemble(n_sys: int = 256, seed: int = 0, fil_range=(1, 64), seg_range=(16, 48),
             volume_fraction: float = 0.02):
    """Batch of independent suspensions with the physics of `suspension`:
    system k has U[fil_range] filaments of U[seg_range] segments each
    (inclusive, seeded), placed as an isotropic cloud at the given volume
    fraction; in every system the first half of the filaments sediment and the
    rest carry a tip follower force f_i = 100 K_B / L_i^2 (L_i = N_i dL). K_B,
    K_T and dt are those of the 32-segment suspension (B = 1000 for N = 32,
    dt = T/200), tolerance 1e-4.
    Returns (Workload, fil_per_sys, seg_per_fil, base, t, mu, Fext, follower)."""
    rng = np.random.default_rng(seed)
    wl = workload_params(1, 32, B=1000.0, dt_over_T=1.0 / 200.0, tol=1e-4, max_iter=60)
    fil_per_sys = rng.integers(fil_range[0], fil_range[1] + 1, size=n_sys)
    segs_all, bases, ts, mus, Fs, fols = [], [], [], [], [], []
    for k in range(n_sys):
        m = int(fil_per_sys[k])
        segs = [int(x) for x in rng.integers(seg_range[0], seg_range[1] + 1, size=m)]
        base, t, mu, _ = cloud_frames(m, segs, dL=wl.dL, volume_fraction=volume_fraction,
                                      rng=rng)
        passive = np.arange(m) < m // 2
        for i in range(m):
            F = np.zeros((segs[i], 3))
            if passive[i]:
                F[:, 2] = -wl.W * wl.dL
            Fs.append(F)
            fols.append(0.0 if passive[i] else 100.0 * wl.KB / (segs[i] * wl.dL) ** 2)
        segs_all += segs
        bases.append(base)
        ts.append(t)
        mus.append(mu)
    wl.n_fil = len(segs_all)
    wl.seg_per_fil = segs_all
    return (wl, [int(x) for x in fil_per_sys], segs_all, np.concatenate(bases), np.concatenate(ts),
            np.concatenate(mus), np.concatenate(Fs), np.array(fols))
