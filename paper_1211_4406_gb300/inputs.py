"""Seeded synthetic particle boxes for the short-range TreePM path.

This module only draws random inputs; it holds none of the force, tree or
list arithmetic, so both the CPU oracle and the CUDA path can consume it.

The paper's workload (Sec. III-A) is a 10240^3 cosmological box at redshift
~31 whose initial conditions are not available.  The generators below stand
in for it with the regime the paper describes (Sec. II): a periodic unit box,
mostly clustered matter with density contrasts of 10^2..10^7 around uniform
background, and r_cut = 3 / N_PM^(1/3) (Sec. III-A).

Recipes
-------
uniform   : x ~ U[0,1)^3, m = 1/N.
clustered : n_h halo masses M ~ p(M) propto M^-1.9 on [1, 1000] (inverse CDF);
            round(0.7 N) particles split between halos proportionally to M by
            largest remainder, the rest uniform background; halo centres
            U[0,1)^3; NFW profile with concentration 10 truncated at r_200
            (mean density 1, overdensity 200); radii by bisection on the
            enclosed-mass fraction; isotropic directions; wrapped mod 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 14406          # config k uses SEED_BASE + k (k = 1..5)
SEED_BATCH = 14406000      # batched box b uses SEED_BATCH + b


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_box(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """n particles uniform in [0,1)^3; FP64 positions [n,3], masses 1/n."""
    rng = _rng(seed)
    pos = rng.random((n, 3), dtype=np.float64)
    mass = np.full(n, 1.0 / max(n, 1), dtype=np.float64)
    return pos, mass


def _nfw_mu(s: np.ndarray) -> np.ndarray:
    return np.log1p(s) - s / (1.0 + s)


def _bisect_mu(uu: np.ndarray, conc: float) -> np.ndarray:
    lo = np.zeros_like(uu)
    hi = np.full_like(uu, conc)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = _nfw_mu(mid) < uu
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def _nfw_radius(uu: np.ndarray, conc: float) -> np.ndarray:
    """s in [0, conc] with mu(s) = uu by 60 bisection steps (element by
    element, so large inputs are split into chunks that run on several host
    threads with the same result)."""
    chunk = 1 << 22
    if uu.size <= 2 * chunk:
        return _bisect_mu(uu, conc)
    import concurrent.futures as cf
    import os
    parts = [uu[i:i + chunk] for i in range(0, uu.size, chunk)]
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
        return np.concatenate(list(ex.map(lambda p: _bisect_mu(p, conc), parts)))


def clustered_box(n: int, n_halo: int, seed: int, frac: float = 0.7,
                  m_lo: float = 1.0, m_hi: float = 1000.0, slope: float = 1.9,
                  conc: float = 10.0) -> tuple[np.ndarray, np.ndarray]:
    """NFW-clustered box (recipe in the module docstring)."""
    rng = _rng(seed)
    n_halo = max(1, int(n_halo))
    # halo masses: inverse CDF of M^-slope on [m_lo, m_hi]
    a = 1.0 - slope
    u = rng.random(n_halo)
    mh = (m_lo ** a + u * (m_hi ** a - m_lo ** a)) ** (1.0 / a)
    # particles per halo: largest remainder of round(frac*n) proportional to mh
    n_in = int(round(frac * n))
    share = mh / mh.sum() * n_in
    cnt = np.floor(share).astype(np.int64)
    rem = n_in - int(cnt.sum())
    if rem > 0:
        order = np.argsort(-(share - cnt), kind="stable")
        cnt[order[:rem]] += 1
    n_bg = n - int(cnt.sum())
    centres = rng.random((n_halo, 3))
    # NFW radii per particle
    halo_of = np.repeat(np.arange(n_halo), cnt)
    m_frac = cnt.astype(np.float64) / n                   # halo mass, total 1
    r200 = (3.0 * m_frac / (800.0 * math.pi)) ** (1.0 / 3.0)
    rs = r200 / conc
    uu = rng.random(halo_of.size) * _nfw_mu(np.array(conc))
    s = _nfw_radius(uu, conc)
    rad = s * rs[halo_of]
    dirs = rng.standard_normal((halo_of.size, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    halo_pos = centres[halo_of] + rad[:, None] * dirs
    bg = rng.random((n_bg, 3))
    pos = np.concatenate([halo_pos, bg], axis=0)
    pos -= np.floor(pos)
    pos[pos >= 1.0] = 0.0
    # shuffle so that the input order carries no spatial structure
    perm = rng.permutation(n)
    pos = np.ascontiguousarray(pos[perm])
    mass = np.full(n, 1.0 / n, dtype=np.float64)
    return pos, mass


def cotangent(n: int, seed: int) -> np.ndarray:
    """w ~ N(0,1)^3 in FP32: the cotangent dL/da of L = sum_i w_i . a_i."""
    return _rng(seed).standard_normal((n, 3)).astype(np.float32)


@dataclass
class Box:
    """One periodic unit box and the short-range parameters used on it."""
    name: str
    pos: np.ndarray
    mass: np.ndarray
    G: float
    eps: float
    r_cut: float
    theta: float
    n_crit: int = 64
    n_leaf: int = 8
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def config_box(k: int, n_override: int | None = None) -> Box:
    """Boxes of the five workloads (k = 1..5); n_override shrinks the particle
    count for quick checks while keeping the recipe (r_cut, eps follow N)."""
    seed = SEED_BASE + k
    if k == 1:
        n = n_override or 32 ** 3
        side = round(n ** (1.0 / 3.0))
        pos, mass = uniform_box(n, seed)
        return Box("uniform-32k", pos, mass, 1.0, 1.0 / (50 * side), 3.0 / side,
                   0.5, seed=seed)
    if k == 2:
        n = n_override or 128 ** 3
        side = n ** (1.0 / 3.0)
        pos, mass = clustered_box(n, max(1, round(2000 * n / 128 ** 3)), seed)
        return Box("clustered-2M", pos, mass, 1.0, 1.0 / (50 * side), 3.0 / side,
                   0.5, seed=seed)
    if k == 4:
        n = n_override or 64 ** 3
        side = n ** (1.0 / 3.0)
        pos, mass = clustered_box(n, max(1, round(250 * n / 64 ** 3)), seed)
        return Box("clustered-262k", pos, mass, 1.0, 1.0 / (50 * side), 3.0 / side,
                   0.5, seed=seed)
    if k == 5:
        n = n_override or 512 ** 3
        side = n ** (1.0 / 3.0)
        pos, mass = clustered_box(n, max(1, round(100000 * n / 512 ** 3)), seed)
        return Box("clustered-134M", pos, mass, 1.0, 1.0 / (50 * side), 3.0 / side,
                   0.5, seed=seed)
    raise ValueError(f"no single-box workload {k}")


def batched_sizes(nbox: int = 64, lo: int = 16 ** 3, hi: int = 96 ** 3,
                  seed: int = SEED_BASE + 3) -> np.ndarray:
    """Per-box particle counts, log-uniform in [lo, hi]."""
    u = _rng(seed).random(nbox)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def batched_boxes(nbox: int = 64, scale: float = 1.0) -> list[Box]:
    """The batched workload: even boxes uniform, odd boxes NFW-clustered with
    halo count scaled as 2000 * N / 128^3; r_cut = 3/N^(1/3),
    eps = 1/(50 N^(1/3)).  `scale` shrinks every box for quick checks."""
    out = []
    for b, nb in enumerate(batched_sizes(nbox)):
        nb = max(2, int(round(int(nb) * scale)))
        seed = SEED_BATCH + b
        side = nb ** (1.0 / 3.0)
        if b % 2 == 0:
            pos, mass = uniform_box(nb, seed)
            kind = "uniform"
        else:
            pos, mass = clustered_box(nb, max(1, round(2000 * nb / 128 ** 3)), seed)
            kind = "clustered"
        out.append(Box(f"batch{b}-{kind}", pos, mass, 1.0, 1.0 / (50 * side),
                       3.0 / side, 0.5, seed=seed))
    return out


def lattice_box(side: int, offset: float = 0.5) -> tuple[np.ndarray, np.ndarray]:
    """Perfect cubic lattice of side^3 equal-mass particles (a symmetry case)."""
    g = (np.arange(side, dtype=np.float64) + offset) / side
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    n = pos.shape[0]
    return np.ascontiguousarray(pos), np.full(n, 1.0 / n)
