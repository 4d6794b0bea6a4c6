"""Seeded synthetic rectangle collections (MBRs) for the spatial-join filter step.

This module only draws random numbers and lays them out; it holds none of the
join's arithmetic.  It is the one module both the CPU oracle's tests and the
CUDA path's tests / benchmark use to build inputs.

Layout of every collection: ``float32[n, 4]`` with columns ``(xl, yl, xu, yu)``
(the ``sj_rect`` struct of the C-ABI), coordinates in the normalised space
``[0, 1]^2`` of Sec. 4.1 (centres may spill slightly past the border, extents
never are negative).  Corners are computed in float64 as ``c -/+ w/2`` and then
rounded to float32, which keeps ``xl <= xu`` exactly.

Random streams: ``numpy.random.Generator(PCG64(SeedSequence(seed)))``; a seed's
``SeedSequence`` is split with ``spawn(3)`` into (world, R, S).  The "world"
stream draws what R and S share (mixture components, Zipf rank->cell maps);
each side draws its own rectangles in the order (cx, cy, w, h).

Workloads (stand-ins for the Tiger 2015 / OSM layers of Table 1, which are not
available here):

* ``uniform_pair``  -- plain join: uniform centres, uniform extents.
* ``gis_pair``      -- layers shaped like large GIS layers: 64-component Gaussian
  mixture (sigma ~ U[0.01, 0.1], truncated to the unit square) plus 20%
  uniform background, log-normal extents (median 2e-5, sigma 1, clipped at
  1e-2).
* ``zipf_pair``     -- extent / skew stress: Zipf(s=1.2) ranks onto a 1024^2
  lattice with uniform jitter inside the cell; S uses R's rank->cell map with
  probability ``rho`` and an independent map otherwise.
* ``batch_pairs``   -- many independent joins of uneven size.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_pair",
    "gis_pair",
    "zipf_pair",
    "batch_pairs",
    "degenerate_pair",
    "rects_from_centres",
]


def _streams(seed: int):
    ss = np.random.SeedSequence(seed)
    w, r, s = ss.spawn(3)
    mk = lambda q: np.random.Generator(np.random.PCG64(q))  # noqa: E731
    return mk(w), mk(r), mk(s)


def rects_from_centres(cx, cy, w, h) -> np.ndarray:
    """float64 centres / extents -> float32 [n,4] (xl, yl, xu, yu)."""
    cx = np.asarray(cx, np.float64)
    cy = np.asarray(cy, np.float64)
    hw = 0.5 * np.asarray(w, np.float64)
    hh = 0.5 * np.asarray(h, np.float64)
    out = np.empty((cx.shape[0], 4), np.float32)
    out[:, 0] = cx - hw
    out[:, 1] = cy - hh
    out[:, 2] = cx + hw
    out[:, 3] = cy + hh
    return out


def uniform_pair(n_r: int = 10_000, n_s: int = 10_000, max_extent: float = 2e-3,
                 seed: int = 1):
    """Plain join: centres U[0,1]^2, width and height each U[0, max_extent].

    Defaults: |R| = |S| = 10^4, extents in [0, 2e-3], seed 1 (joined on a
    64 x 64 grid)."""
    _, gr, gs = _streams(seed)
    out = []
    for g, n in ((gr, n_r), (gs, n_s)):
        cx = g.random(n)
        cy = g.random(n)
        w = g.uniform(0.0, max_extent, n)
        h = g.uniform(0.0, max_extent, n)
        out.append(rects_from_centres(cx, cy, w, h))
    return out[0], out[1]


def _mixture_world(world, n_comp: int = 64):
    mu = world.random((n_comp, 2))
    sigma = world.uniform(0.01, 0.1, n_comp)
    return mu, sigma


def _mixture_centres(g, n, mu, sigma, background: float, with_comp: bool = False):
    """cx, cy from an equal-weight isotropic Gaussian mixture plus a uniform
    background fraction, truncated to [0,1]^2: a component draw that falls
    outside is redrawn from the same component (clipping instead would pile
    thousands of centres onto the border lines).  With ``with_comp`` also the
    component of every centre (-1 for the background)."""
    comp = g.integers(0, mu.shape[0], n)
    is_bg = g.random(n) < background
    z = g.standard_normal((n, 2))
    u = g.random((n, 2))
    c = mu[comp] + sigma[comp, None] * z
    out = ~is_bg & ((c < 0.0) | (c > 1.0)).any(axis=1)
    while out.any():
        idx = np.nonzero(out)[0]
        c[idx] = mu[comp[idx]] + sigma[comp[idx], None] * g.standard_normal((len(idx), 2))
        out[idx] = ((c[idx] < 0.0) | (c[idx] > 1.0)).any(axis=1)
    c = np.where(is_bg[:, None], u, c)
    if with_comp:
        return c[:, 0], c[:, 1], np.where(is_bg, -1, comp)
    return c[:, 0], c[:, 1]


def gis_pair(n_r: int = 10_000_000, n_s: int = 20_000_000, seed: int = 2,
             median_extent: float = 2e-5, log_sigma: float = 1.0,
             max_extent: float = 1e-2, background: float = 0.2):
    """Plain join shaped like large GIS layers.

    Defaults: |R| = 10M, |S| = 20M; centres from a 64-component Gaussian
    mixture (sigma U[0.01,0.1], means U[0,1]^2, equal weights, shared by R and
    S, truncated to [0,1]^2) plus 20% uniform background; width and height
    independently log-normal with median 2e-5 and sigma 1.0, clipped to 1e-2.
    Smaller n give the same spatial distribution at lower density."""
    world, gr, gs = _streams(seed)
    mu, sigma = _mixture_world(world)
    out = []
    for g, n in ((gr, n_r), (gs, n_s)):
        cx, cy = _mixture_centres(g, n, mu, sigma, background)
        w = np.minimum(np.exp(g.normal(np.log(median_extent), log_sigma, n)), max_extent)
        h = np.minimum(np.exp(g.normal(np.log(median_extent), log_sigma, n)), max_extent)
        out.append(rects_from_centres(cx, cy, w, h))
    return out[0], out[1]


def aniso_pair(n_r: int = 10_000_000, n_s: int = 20_000_000, seed: int = 5,
               ratio: float = 10.0, median_extent: float = 2e-5, log_sigma: float = 1.0,
               max_extent: float = 1e-2, background: float = 0.2):
    """GIS-shaped layers of elongated objects (roads, rivers): the centres of
    ``gis_pair`` (64-component Gaussian mixture shared by R and S, plus 20%
    uniform background), and every rectangle ``ratio`` times longer along one
    axis than along the other.  Each mixture component has one orientation
    (wide or tall, drawn once per component from the world stream, shared by R
    and S); background rectangles draw theirs at random.  The geometric mean
    of width and height is log-normal with median ``median_extent`` and sigma
    ``log_sigma``; both are clipped to ``max_extent``."""
    world, gr, gs = _streams(seed)
    mu, sigma = _mixture_world(world)
    wide = world.random(mu.shape[0]) < 0.5
    out = []
    k = np.sqrt(ratio)
    for g, n in ((gr, n_r), (gs, n_s)):
        cx, cy, comp = _mixture_centres(g, n, mu, sigma, background, with_comp=True)
        e = np.exp(g.normal(np.log(median_extent), log_sigma, n))
        bg_wide = g.random(n) < 0.5
        is_wide = np.where(comp >= 0, wide[np.maximum(comp, 0)], bg_wide)
        w = np.minimum(np.where(is_wide, e * k, e / k), max_extent)
        h = np.minimum(np.where(is_wide, e / k, e * k), max_extent)
        out.append(rects_from_centres(cx, cy, w, h))
    return out[0], out[1]


def gis_points(n_p: int = 10_000_000, n_q: int = 20_000_000, seed: int = 2,
               background: float = 0.2):
    """Point sets for the eps-distance join, with the spatial distribution of
    the GIS-shaped layers: centres from the same 64-component Gaussian
    mixture (shared by P and Q, truncated to [0,1]^2) plus 20% uniform
    background.  Returns float32 [n, 2] (x, y) arrays."""
    world, gp, gq = _streams(seed)
    mu, sigma = _mixture_world(world)
    out = []
    for g, n in ((gp, n_p), (gq, n_q)):
        cx, cy = _mixture_centres(g, n, mu, sigma, background)
        out.append(np.stack([cx, cy], 1).astype(np.float32))
    return out[0], out[1]


def lattice_points(n: int, pitch: float, x0: float, y0: float) -> np.ndarray:
    """n x n points (x0 + i * pitch, y0 + j * pitch), index i * n + j, as
    float32 [n*n, 2] (exact when pitch and the offsets are binary fractions)."""
    i = np.arange(n)
    gx, gy = np.meshgrid(i, i, indexing="ij")
    return np.stack([x0 + gx.ravel() * pitch, y0 + gy.ravel() * pitch], 1).astype(np.float32)


def zipf_pair(n_r: int = 20_000_000, n_s: int = 20_000_000, seed: int = 3,
              rho: float = 0.0, zipf_s: float = 1.2, lattice: int = 1024,
              r_max_extent: float = 1e-4, s_max_extent: float = 1e-3):
    """Extent and skew stress.

    Centres: Zipf(s) rank over lattice^2 cells (truncated at lattice^2 ranks),
    mapped to a cell by a seeded random permutation, then jittered uniformly
    inside the 1/lattice-wide cell.  R uses map A.  Each S rectangle uses map A
    with probability ``rho`` and an independent map B otherwise (rho = 1 is
    the literal "same skew" reading, rho = 0 independent hot spots).
    Extents: R w,h ~ U[0, 1e-4]; S w,h ~ U[0, 1e-3]."""
    world, gr, gs = _streams(seed)
    ncell = lattice * lattice
    ranks = np.arange(1, ncell + 1, dtype=np.float64)
    p = ranks ** (-zipf_s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    map_a = world.permutation(ncell)
    map_b = world.permutation(ncell)
    out = []
    for side, (g, n, emax) in enumerate(((gr, n_r, r_max_extent), (gs, n_s, s_max_extent))):
        rank = np.searchsorted(cdf, g.random(n), side="right")
        np.minimum(rank, ncell - 1, out=rank)
        if side == 0:
            cell = map_a[rank]
        else:
            use_a = g.random(n) < rho
            cell = np.where(use_a, map_a[rank], map_b[rank])
        jx = g.random(n)
        jy = g.random(n)
        cx = ((cell % lattice) + jx) / lattice
        cy = ((cell // lattice) + jy) / lattice
        w = g.uniform(0.0, emax, n)
        h = g.uniform(0.0, emax, n)
        out.append(rects_from_centres(cx, cy, w, h))
    return out[0], out[1]


def batch_pairs(n_joins: int = 256, seed0: int = 4000, n_min: float = 1e3,
                n_max: float = 2e6, median_extent: float = 1e-4,
                log_sigma: float = 1.0, max_extent: float = 1e-2):
    """Many independent joins of uneven size.

    Join j uses seed ``seed0 + j``; per-side sizes log-uniform in
    [n_min, n_max]; even j: uniform centres, odd j: 64-component mixture
    (+20% background); extents log-normal (median 1e-4, sigma 1, clip 1e-2).
    Returns a list of (R, S)."""
    joins = []
    for j in range(n_joins):
        world, gr, gs = _streams(seed0 + j)
        mu, sigma = _mixture_world(world)
        pair = []
        for g in (gr, gs):
            n = int(np.exp(g.uniform(np.log(n_min), np.log(n_max))))
            if j % 2 == 0:
                cx = g.random(n)
                cy = g.random(n)
            else:
                cx, cy = _mixture_centres(g, n, mu, sigma, 0.2)
            w = np.minimum(np.exp(g.normal(np.log(median_extent), log_sigma, n)), max_extent)
            h = np.minimum(np.exp(g.normal(np.log(median_extent), log_sigma, n)), max_extent)
            pair.append(rects_from_centres(cx, cy, w, h))
        joins.append((pair[0], pair[1]))
    return joins


def degenerate_pair(n_r: int = 600, n_s: int = 500, seed: int = 11, lattice: int = 16):
    """Edge-case mix for parity tests: coordinates snapped to a coarse binary
    lattice (so many rectangles share edges, corners and x_l values exactly),
    zero-width / zero-height / point rectangles, exact duplicates, negative
    zero, rectangles spanning the whole space and centres outside [0,1]."""
    _, gr, gs = _streams(seed)
    out = []
    for g, n in ((gr, n_r), (gs, n_s)):
        a = g.integers(-2, lattice + 3, (n, 2)).astype(np.float64) / lattice
        ext = g.integers(0, 4, (n, 2)).astype(np.float64) / lattice
        kind = g.integers(0, 10, n)
        ext[kind == 0, 0] = 0.0                      # zero width
        ext[kind == 1, 1] = 0.0                      # zero height
        ext[kind == 2] = 0.0                         # points
        big = kind == 3
        a[big] = -0.25
        ext[big] = 1.5                               # spans everything
        r = np.empty((n, 4), np.float32)
        r[:, 0] = a[:, 0]
        r[:, 1] = a[:, 1]
        r[:, 2] = a[:, 0] + ext[:, 0]
        r[:, 3] = a[:, 1] + ext[:, 1]
        dup = g.integers(0, n, n // 10)
        r[dup[1:]] = r[dup[:-1]]                     # exact duplicates
        negz = (r == 0.0) & (g.random((n, 4)) < 0.5)
        r[negz] = -0.0                               # negative zero
        out.append(r)
    return out[0], out[1]
