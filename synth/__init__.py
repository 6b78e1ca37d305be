"""Seeded synthetic point clouds with oriented normals.

This module is shared by the tests, the oracle checks and the benchmark.  It
produces *inputs only*: point positions x_i and unit normals n_i of a known
surface (the data of Section II.A.1 of the paper, "point cloud X with surface
normals").  It contains none of the reconstruction arithmetic (no off-surface
points, no kernel, no solve): those live on each side of the parity boundary
separately.

All randomness comes from numpy's PCG64 generator (O'Neill, "PCG: A family of
simple fast space-efficient statistically good algorithms for random number
generation", 2014) seeded explicitly, so every cloud is reproducible bit for
bit from (shape, size, seed).  Arrays are float32, shape (N, 3), C-contiguous.

Shapes (the paper's workloads are laser scans of closed surfaces; these stand
in for them, see Section IV):
  * ``sphere``    - uniform on the unit sphere (normalised Gaussian triples),
                    normal = position.  The synthetic test of Section IV.A.
  * ``torus``     - uniform by area on a ring torus (rejection on the tube
                    angle), analytic normals, optional Gaussian position noise
                    added after the normal is taken.
  * ``ellipsoid`` - uniform by area on an axis-aligned ellipsoid (rejection on
                    the area element), analytic normals.
  * ``metaball``  - iso-surface of a sum of Gaussian blobs, points by
                    rejection-sampled cells of a level-set grid plus Newton
                    projection, normals = normalised gradient, optional height
                    dependent density.
  * ``batch``     - many ellipsoids/tori of log-uniform sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "sphere", "torus", "ellipsoid", "metaball", "batch", "halton",
    "Cloud", "lattice", "mean_nn_spacing", "mlp_init", "MLP_SIZES",
]

# layer sizes of the learned block preconditioner (inputs, hidden, hidden, outputs)
MLP_SIZES = (256, 256, 256, 64)


@dataclass
class Cloud:
    """A point cloud with normals and the generator parameters that made it."""
    points: np.ndarray          # (N, 3) float32
    normals: np.ndarray         # (N, 3) float32, unit length
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.points.shape[0])


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def sphere(n: int, seed: int = 0, radius: float = 1.0) -> Cloud:
    """``n`` points uniform on the sphere of ``radius`` about the origin."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, 3))
    u = g / np.linalg.norm(g, axis=1, keepdims=True)
    return Cloud(_f32(radius * u), _f32(u),
                 dict(shape="sphere", n=n, seed=seed, radius=radius))


def torus(n: int, R: float = 1.0, r: float = 0.35, noise: float = 0.0,
          seed: int = 0, center=(0.0, 0.0, 0.0), theta_max: float = 2 * math.pi) -> Cloud:
    """``n`` points uniform by area on the ring torus (major ``R``, minor ``r``).

    The area element is r (R + r cos(phi)) dtheta dphi, so phi is accepted with
    probability (R + r cos phi) / (R + r).  The normal is the analytic one at the
    clean point; isotropic Gaussian noise of std ``noise`` is then added to the
    position only.  ``theta_max`` < 2 pi keeps the sector 0 <= theta < theta_max
    (a patch with the density of n * 2 pi / theta_max points on the whole torus).
    """
    rng = np.random.default_rng(seed)
    th_out, ph_out, got = [], [], 0
    while got < n:
        m = max(1024, int(1.3 * (n - got)) + 16)
        th = rng.uniform(0.0, theta_max, m)
        ph = rng.uniform(0.0, 2 * math.pi, m)
        keep = rng.uniform(0.0, 1.0, m) < (R + r * np.cos(ph)) / (R + r)
        th_out.append(th[keep]); ph_out.append(ph[keep]); got += int(keep.sum())
    th = np.concatenate(th_out)[:n]
    ph = np.concatenate(ph_out)[:n]
    ring = R + r * np.cos(ph)
    p = np.stack([ring * np.cos(th), ring * np.sin(th), r * np.sin(ph)], axis=1)
    nrm = np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], axis=1)
    if noise > 0:
        p = p + rng.normal(0.0, noise, size=p.shape)
    p = p + np.asarray(center, dtype=np.float64)
    return Cloud(_f32(p), _f32(nrm),
                 dict(shape="torus", n=n, R=R, r=r, noise=noise, seed=seed,
                      center=list(map(float, center)), theta_max=theta_max))


def ellipsoid(n: int, axes=(1.0, 1.0, 1.0), seed: int = 0,
              center=(0.0, 0.0, 0.0)) -> Cloud:
    """``n`` points uniform by area on the ellipsoid with semi-axes ``axes``.

    A direction u uniform on S^2 maps to p = a*u; the area element of that map is
    proportional to |(u_x/a, u_y/b, u_z/c)|, so u is accepted with probability
    |(u/a)| / max|(u/a)|.  The normal is grad(sum (x_k/a_k)^2) normalised.
    """
    a = np.asarray(axes, dtype=np.float64)
    rng = np.random.default_rng(seed)
    wmax = float(np.max(1.0 / a))
    out, got = [], 0
    while got < n:
        m = max(1024, int(2.0 * (n - got)) + 16)
        g = rng.standard_normal((m, 3))
        u = g / np.linalg.norm(g, axis=1, keepdims=True)
        w = np.linalg.norm(u / a, axis=1)
        keep = rng.uniform(0.0, 1.0, m) < w / wmax
        out.append(u[keep]); got += int(keep.sum())
    u = np.concatenate(out)[:n]
    p = u * a
    nrm = p / (a * a)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    p = p + np.asarray(center, dtype=np.float64)
    return Cloud(_f32(p), _f32(nrm),
                 dict(shape="ellipsoid", n=n, axes=list(map(float, a)), seed=seed,
                      center=list(map(float, center))))


def _blob_field(x: np.ndarray, c: np.ndarray, w: np.ndarray):
    """F(x) = sum_k exp(-|x - c_k|^2 / w_k^2) and its gradient."""
    F = np.zeros(len(x))
    G = np.zeros_like(x)
    for ck, wk in zip(c, w):
        d = x - ck
        e = np.exp(-(d * d).sum(1) / (wk * wk))
        F += e
        G += (-2.0 / (wk * wk)) * e[:, None] * d
    return F, G


def metaball(n: int, nblobs: int = 8, seed: int = 0, density_power: float = 3.0,
             density_gain: float = 9.0, grid: int = 96) -> Cloud:
    """``n`` points on the iso-surface F = T of ``nblobs`` seeded Gaussian blobs.

    Blob centres are U[-0.5, 0.5]^3 and widths U[0.15, 0.3].  The iso level T is
    the largest of a few candidate levels for which the inside set is a single
    connected component on the ``grid``^3 sample lattice.  Points are produced by
    (1) choosing lattice cells whose corners straddle T uniformly at random,
    (2) a uniform point in that cell, (3) Newton projection onto F = T along grad F.
    Each accepted point is kept with probability (1 + g*u^p)/(1 + g), u the
    normalised height (z - zmin)/(zmax - zmin): the surface density is then
    proportional to 1 + g*u^p.  Normals are -grad F / |grad F| (outward).
    """
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.5, 0.5, (nblobs, 3))
    w = rng.uniform(0.15, 0.3, nblobs)
    lo = c.min(0) - 2.5 * w.max()
    hi = c.max(0) + 2.5 * w.max()
    ax = [np.linspace(lo[k], hi[k], grid) for k in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    F, _ = _blob_field(P, c, w)
    F = F.reshape(grid, grid, grid)
    T = None
    for cand in (0.5, 0.4, 0.3, 0.25, 0.2, 0.15, 0.1):
        if _single_component(F > cand):
            T = cand
            break
    if T is None:
        T = 0.1
    s = F - T
    straddle = np.zeros((grid - 1,) * 3, dtype=bool)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                sub = s[dx:grid - 1 + dx, dy:grid - 1 + dy, dz:grid - 1 + dz]
                straddle |= sub > 0
    allneg = np.ones((grid - 1,) * 3, dtype=bool)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                allneg &= s[dx:grid - 1 + dx, dy:grid - 1 + dy, dz:grid - 1 + dz] <= 0
    cells = np.argwhere(straddle & ~allneg)
    h = (hi - lo) / (grid - 1)
    out, got = [], 0
    zmin = lo[2] + cells[:, 2].min() * h[2]
    zmax = lo[2] + (cells[:, 2].max() + 1) * h[2]
    while got < n:
        m = max(4096, int(1.6 * (n - got) * (1 + density_gain) / (1 + 0.4 * density_gain)) + 64)
        pick = cells[rng.integers(0, len(cells), m)]
        x = lo + (pick + rng.uniform(0.0, 1.0, (m, 3))) * h
        for _ in range(6):
            Fx, Gx = _blob_field(x, c, w)
            g2 = np.maximum((Gx * Gx).sum(1), 1e-30)
            x = x - ((Fx - T) / g2)[:, None] * Gx
        Fx, Gx = _blob_field(x, c, w)
        ok = np.abs(Fx - T) < 1e-6
        u = np.clip((x[:, 2] - zmin) / (zmax - zmin), 0.0, 1.0)
        keep = ok & (rng.uniform(0.0, 1.0, m) < (1.0 + density_gain * u ** density_power) / (1.0 + density_gain))
        xs = x[keep]
        gs = Gx[keep]
        out.append((xs, -gs / np.linalg.norm(gs, axis=1, keepdims=True)))
        got += len(xs)
    p = np.concatenate([o[0] for o in out])[:n]
    nr = np.concatenate([o[1] for o in out])[:n]
    return Cloud(_f32(p), _f32(nr),
                 dict(shape="metaball", n=n, nblobs=nblobs, seed=seed, iso=T,
                      blob_centres=c.tolist(), blob_widths=w.tolist(),
                      density=f"1+{density_gain}*u^{density_power}"))


def _single_component(mask: np.ndarray) -> bool:
    from scipy import ndimage
    lab, k = ndimage.label(mask)
    return k == 1


def mean_nn_spacing(points: np.ndarray) -> float:
    """Mean distance from each point to its nearest other point (k-d tree)."""
    from scipy.spatial import cKDTree
    d, _ = cKDTree(points.astype(np.float64)).query(points.astype(np.float64), k=2)
    return float(d[:, 1].mean())


def batch(nclouds: int = 512, nmin: int = 500, nmax: int = 20000, seed: int = 0,
          sigma_factor: float = 3.0) -> list:
    """``nclouds`` clouds with log-uniform sizes in [nmin, nmax].

    Even-indexed clouds are ellipsoids with semi-axes U[0.5, 1.5]; odd-indexed
    clouds are tori with R ~ U[0.5, 1.5], r = R * U[0.2, 0.4].  Each cloud
    carries ``params['sigma'] = sigma_factor * mean nearest-neighbour spacing``.
    """
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nclouds)).astype(np.int64)
    clouds = []
    for b in range(nclouds):
        s = int(rng.integers(0, 2**31 - 1))
        if b % 2 == 0:
            cl = ellipsoid(int(sizes[b]), axes=tuple(rng.uniform(0.5, 1.5, 3)), seed=s)
        else:
            R = float(rng.uniform(0.5, 1.5))
            cl = torus(int(sizes[b]), R=R, r=R * float(rng.uniform(0.2, 0.4)), seed=s)
        cl.params["sigma"] = sigma_factor * mean_nn_spacing(cl.points)
        clouds.append(cl)
    return clouds


def fibonacci_sphere(n: int, radius: float = 1.0) -> Cloud:
    """``n`` quasi-uniform points on the sphere: the golden-angle spiral, point i at
    height z_i = 1 - (2 i + 1)/n and longitude i pi (3 - sqrt 5).  Normals are the
    positions.  A scan-like cloud whose gaps are all about the spacing (unlike
    random samples, whose largest gaps set the fill distance)."""
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    lon = math.pi * (3.0 - math.sqrt(5.0)) * i
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    u = np.stack([r * np.cos(lon), r * np.sin(lon), z], 1)
    return Cloud(_f32(radius * u), _f32(u), {"kind": "fibonacci_sphere", "n": n, "radius": radius})


def lattice(m: int, h: float, origin=(0.0, 0.0, 0.0)) -> np.ndarray:
    """The m^3 regular lattice of spacing ``h`` (float64, x fastest)."""
    i = np.arange(m, dtype=np.float64) * h
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + np.asarray(origin, dtype=np.float64)


def halton(n: int, bases=(2, 3), start: int = 1) -> np.ndarray:
    """First ``n`` points of the Halton sequence (radical inverse in ``bases``)."""
    out = np.zeros((n, len(bases)))
    for d, b in enumerate(bases):
        for i in range(n):
            k, f, r = i + start, 1.0, 0.0
            while k > 0:
                f /= b
                r += f * (k % b)
                k //= b
            out[i, d] = r
    return out


def mlp_init(seed: int = 0, sizes=MLP_SIZES, last_scale: float = 0.1) -> np.ndarray:
    """Seeded initial weights, He-normal (std sqrt(2 / fan_in)) with zero biases,
    the output layer scaled by ``last_scale`` (the network starts near its skip
    connection), packed layer by layer as W[out][in] row-major followed by b[out];
    float32."""
    rng = np.random.default_rng(seed)
    parts = []
    nl = len(sizes) - 1
    for li, (fin, fout) in enumerate(zip(sizes[:-1], sizes[1:])):
        sc = math.sqrt(2.0 / fin) * (last_scale if li == nl - 1 else 1.0)
        parts.append((rng.standard_normal((fout, fin)) * sc).ravel())
        parts.append(np.zeros(fout))
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)
