"""Spatial decomposition of one periodic box over several GPUs (Sec. II).

The paper cuts its box into rectangular domains by a 3-D multi-section
decomposition, one domain per process, and sets the cuts with the sampling
method: each process samples its particles at a rate proportional to its
measured force-calculation time, the samples are gathered, and the cuts are
placed so that every domain holds the same number of samples; to damp the
jumps that sampling noise causes, each boundary is a linearly weighted moving
average over the last five steps.  The short-range force vanishes beyond
r_cut, so besides its own particles a process needs only the particles within
r_cut of its domain (ghosts).

This module holds the host logic of that scheme (the cuts, their moving
average, the sample counts, the variable all-to-all exchange) and the per-rank
step on the GPU (`DomainShortRange`): particle exchange to the owners, ghost
exchange, the tree over own particles followed by ghosts, the forces and the
adjoint in one pass, and the return of the ghosts' share of the adjoint to
their owners.  Selection, packing and unpacking run in the library's kernels
(tp_halo_select, tp_gather_rows, tp_scatter_add_rows); the collectives are
torch.distributed (NCCL between GPUs, gloo for the CPU tests of the exchange).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch
import torch.distributed as dist

from . import _lib

AVERAGE_STEPS = 5       # boundaries: linearly weighted moving average over the last five steps


# ---------------------------------------------------------------------------
# geometry (host logic)
# ---------------------------------------------------------------------------
@dataclass
class Geometry:
    """Cuts of an nx x ny x nz multi-section decomposition of the unit box:
    xc [nx+1]; yc [nx, ny+1] (per slab); zc [nx, ny, nz+1] (per column).
    Domain d = (i ny + j) nz + k is [xc[i], xc[i+1]) x [yc[i,j], yc[i,j+1]) x
    [zc[i,j,k], zc[i,j,k+1])."""
    xc: np.ndarray
    yc: np.ndarray
    zc: np.ndarray

    @property
    def shape(self):
        return self.xc.size - 1, self.yc.shape[1] - 1, self.zc.shape[2] - 1

    @property
    def ndom(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz

    def box(self, d: int):
        nx, ny, nz = self.shape
        i, j, k = d // (ny * nz), (d // nz) % ny, d % nz
        lo = np.array([self.xc[i], self.yc[i, j], self.zc[i, j, k]])
        hi = np.array([self.xc[i + 1], self.yc[i, j + 1], self.zc[i, j, k + 1]])
        return lo, hi

    def volume(self, d: int) -> float:
        lo, hi = self.box(d)
        return float(np.prod(hi - lo))


def uniform_geometry(nx: int, ny: int, nz: int) -> Geometry:
    xc = np.linspace(0.0, 1.0, nx + 1)
    yc = np.tile(np.linspace(0.0, 1.0, ny + 1), (nx, 1))
    zc = np.tile(np.linspace(0.0, 1.0, nz + 1), (nx, ny, 1))
    return Geometry(xc, yc, zc)


def factor_domains(n: int):
    """(nx, ny, nz) with nx ny nz = n, as close to a cube as possible
    (nx >= ny >= nz)."""
    best = None
    for nx in range(1, n + 1):
        if n % nx:
            continue
        for ny in range(1, n // nx + 1):
            if (n // nx) % ny:
                continue
            nz = n // nx // ny
            shape = tuple(sorted((nx, ny, nz), reverse=True))
            score = max(shape) / min(shape)
            if best is None or score < best[0]:
                best = (score, shape)
    return best[1]


def _cuts(values: np.ndarray, m: int, lo: float, hi: float) -> np.ndarray:
    """m + 1 cuts of [lo, hi] that put the same number of the sorted values
    (within +-1) between consecutive cuts: each inner cut halfway between the
    two values it separates; without values, evenly spaced."""
    out = np.empty(m + 1)
    out[0], out[m] = lo, hi
    v = np.sort(values)
    for q in range(1, m):
        if v.size == 0:
            out[q] = lo + (hi - lo) * q / m
            continue
        t = int(round(q * v.size / m))
        a = v[t - 1] if t >= 1 else lo
        b = v[t] if t < v.size else hi
        out[q] = 0.5 * (a + b)
    return np.maximum.accumulate(np.clip(out, lo, hi))


def multisection(samples: np.ndarray, nx: int, ny: int, nz: int) -> Geometry:
    """The 3-D multi-section decomposition with equal sample counts per
    domain: x cuts on all samples, y cuts per slab on that slab's samples,
    z cuts per column on that column's samples."""
    s = np.mod(np.asarray(samples, dtype=np.float64).reshape(-1, 3), 1.0)
    xc = _cuts(s[:, 0], nx, 0.0, 1.0)
    yc = np.zeros((nx, ny + 1))
    zc = np.zeros((nx, ny, nz + 1))
    ix = np.clip(np.searchsorted(xc, s[:, 0], side="right") - 1, 0, nx - 1)
    for i in range(nx):
        si = s[ix == i]
        yc[i] = _cuts(si[:, 1], ny, 0.0, 1.0)
        iy = np.clip(np.searchsorted(yc[i], si[:, 1], side="right") - 1, 0, ny - 1)
        for j in range(ny):
            zc[i, j] = _cuts(si[iy == j, 2], nz, 0.0, 1.0)
    return Geometry(xc, yc, zc)


def moving_average(history: list[Geometry]) -> Geometry:
    """Cut by cut, the linearly weighted average of the last AVERAGE_STEPS
    geometries (oldest first; weights 1, 2, ... up to the newest).  The
    average of non-decreasing cut lists that start at 0 and end at 1 is one
    too."""
    h = history[-AVERAGE_STEPS:]
    w = np.arange(1, len(h) + 1, dtype=np.float64)
    w /= w.sum()
    xc = sum(wi * g.xc for wi, g in zip(w, h))
    yc = sum(wi * g.yc for wi, g in zip(w, h))
    zc = sum(wi * g.zc for wi, g in zip(w, h))
    fix = lambda c: np.maximum.accumulate(np.clip(c, 0.0, 1.0), axis=-1)
    xc, yc, zc = fix(xc), fix(yc), fix(zc)
    xc[0] = 0.0; xc[-1] = 1.0
    yc[..., 0] = 0.0; yc[..., -1] = 1.0
    zc[..., 0] = 0.0; zc[..., -1] = 1.0
    return Geometry(xc, yc, zc)


def sample_counts(costs, total_samples: int) -> list[int]:
    """Samples per rank in proportion to each rank's measured cost (the
    sampling method with rates proportional to calculation time); at least
    one per rank with a positive cost."""
    c = np.maximum(np.asarray(costs, dtype=np.float64), 0.0)
    if c.sum() <= 0:
        c = np.ones_like(c)
    n = np.floor(total_samples * c / c.sum()).astype(np.int64)
    n[(n == 0) & (c > 0)] = 1
    return [int(v) for v in n]


def partition_boxes(costs, world: int) -> list[list[int]]:
    """Independent boxes shared among `world` ranks by the longest-processing-
    time rule: boxes in decreasing cost (ties by index), each to the rank with
    the least total so far (ties by rank).  Deterministic, so every rank
    computes the same split from the same costs.  Returns each rank's box
    indices in increasing order."""
    order = sorted(range(len(costs)), key=lambda b: (-float(costs[b]), b))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(b)
        load[r] += float(costs[b])
    return [sorted(v) for v in out]


# ---------------------------------------------------------------------------
# collectives
# ---------------------------------------------------------------------------
def _world(group=None):
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def alltoallv(send: torch.Tensor, counts, group=None):
    """Variable all-to-all of rows: send holds the rows for rank 0, then rank
    1, ... (counts[r] rows each).  Returns the received rows (from rank 0
    first) and the count from each rank.  Without a process group (one rank)
    the rows come back unchanged."""
    rank, world = _world(group)
    counts = [int(c) for c in counts]
    if len(counts) != world or sum(counts) != send.shape[0]:
        raise ValueError("counts must give one row count per rank, summing to the rows sent")
    if world == 1:
        return send, counts
    cdev = send.device if send.is_cuda else torch.device("cpu")
    sc = torch.tensor(counts, dtype=torch.int64, device=cdev)
    rc = torch.empty_like(sc)
    dist.all_to_all_single(rc, sc, group=group)
    rcounts = [int(v) for v in rc.tolist()]
    out = torch.empty((sum(rcounts),) + tuple(send.shape[1:]), dtype=send.dtype, device=send.device)
    dist.all_to_all_single(out, send.contiguous(), rcounts, counts, group=group)
    return out, rcounts


def gather_samples(samples: torch.Tensor, group=None) -> np.ndarray:
    """Every rank's samples [m_r, 3] (FP64), concatenated in rank order, on
    every rank."""
    rank, world = _world(group)
    if world == 1:
        return samples.detach().cpu().numpy().reshape(-1, 3)
    dev = samples.device
    m = torch.tensor([samples.shape[0]], dtype=torch.int64, device=dev)
    ms = [torch.empty_like(m) for _ in range(world)]
    dist.all_gather(ms, m, group=group)
    mmax = max(int(v.item()) for v in ms)
    pad = torch.zeros((mmax, 3), dtype=torch.float64, device=dev)
    pad[:samples.shape[0]] = samples
    outs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(outs, pad, group=group)
    return np.concatenate([o[:int(k.item())].cpu().numpy() for o, k in zip(outs, ms)], axis=0)


# ---------------------------------------------------------------------------
# the library's selection, packing and unpacking
# ---------------------------------------------------------------------------
class Halo:
    """tp_halo: a geometry on the device and the selections it makes."""

    def __init__(self, nx: int, ny: int, nz: int):
        h = C.c_void_p()
        _lib.check(_lib.load().tp_halo_create(int(nx), int(ny), int(nz), C.byref(h)), "tp_halo_create")
        self._h = h
        self.shape = (nx, ny, nz)
        self.ndom = nx * ny * nz

    def set_geometry(self, g: Geometry) -> None:
        if g.shape != self.shape:
            raise ValueError(f"geometry {g.shape} does not match the halo's {self.shape}")
        xc = np.ascontiguousarray(g.xc, dtype=np.float64)
        yc = np.ascontiguousarray(g.yc, dtype=np.float64)
        zc = np.ascontiguousarray(g.zc, dtype=np.float64)
        _lib.check(_lib.load().tp_halo_set_cuts(self._h, xc.ctypes.data_as(C.c_void_p), yc.ctypes.data_as(C.c_void_p),
                                                zc.ctypes.data_as(C.c_void_p)), "tp_halo_set_cuts")

    def select(self, pos: torch.Tensor, mode: str, self_domain: int = 0, r_cut: float = 0.0, stream=None):
        """(indices [total] int32 grouped by destination, counts per destination)."""
        if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dtype == torch.float64 and pos.dim() == 2
                and pos.shape[1] == 3):
            raise ValueError("pos must be a float64 CUDA tensor [n, 3]")
        pos = pos.contiguous()
        m = {"owner": 0, "ghosts": 1}[mode]
        counts = np.zeros(self.ndom, dtype=np.int64)
        s = C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        lib = _lib.load()
        cap = max(1, pos.shape[0] if m == 0 else 2 * pos.shape[0])
        for _ in range(2):
            idx = torch.empty(cap, dtype=torch.int32, device=pos.device)
            code = lib.tp_halo_select(self._h, C.c_void_p(pos.data_ptr()), pos.shape[0], m, int(self_domain),
                                      float(r_cut), C.c_void_p(idx.data_ptr()), cap,
                                      counts.ctypes.data_as(C.c_void_p), s)
            if code == -4 and int(counts.sum()) > cap:        # too many ghosts for the first guess
                cap = int(counts.sum())
                continue
            _lib.check(code, "tp_halo_select")
            return idx[:int(counts.sum())], [int(c) for c in counts]
        raise RuntimeError("tp_halo_select: ghost count changed between calls")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.load().tp_halo_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gather_rows(src: torch.Tensor, idx: torch.Tensor, stream=None) -> torch.Tensor:
    """src[idx] by the library's row gather (rows of any 4-byte-multiple width)."""
    src = src.contiguous()
    m = int(idx.shape[0])
    out = torch.empty((m,) + tuple(src.shape[1:]), dtype=src.dtype, device=src.device)
    row_bytes = src.element_size() * (int(np.prod(src.shape[1:])) if src.dim() > 1 else 1)
    if row_bytes % 4:
        raise ValueError("rows must be a multiple of 4 bytes")
    if m:
        s = C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
        _lib.check(_lib.load().tp_gather_rows(C.c_void_p(src.data_ptr()), row_bytes // 4, C.c_void_p(idx.data_ptr()),
                                              m, C.c_void_p(out.data_ptr()), s), "tp_gather_rows")
    return out


def scatter_add_rows(dst: torch.Tensor, idx: torch.Tensor, src: torch.Tensor, stream=None) -> None:
    """dst[idx] += src by the library (FP64 rows; repeated indices add up)."""
    if dst.dtype != torch.float64 or src.dtype != torch.float64 or not dst.is_contiguous():
        raise ValueError("scatter_add_rows takes contiguous float64 tensors")
    m = int(idx.shape[0])
    if m == 0:
        return
    width = int(np.prod(dst.shape[1:])) if dst.dim() > 1 else 1
    s = C.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _lib.check(_lib.load().tp_scatter_add_rows(C.c_void_p(dst.data_ptr()), width, C.c_void_p(idx.data_ptr()),
                                               C.c_void_p(src.contiguous().data_ptr()), m, s), "tp_scatter_add_rows")


# ---------------------------------------------------------------------------
# the per-rank step
# ---------------------------------------------------------------------------
@dataclass
class Exchanged:
    """The ghost exchange of one step: what was sent (for the way back) and
    what arrived."""
    send_idx: torch.Tensor
    send_counts: list
    recv_counts: list
    ghost_pos: torch.Tensor
    ghost_mass: torch.Tensor


@dataclass
class DomainShortRange:
    """One rank's share of the short-range force and adjoint of one box.

    Each rank owns the particles of one domain of an nx x ny x nz
    multi-section decomposition (nx ny nz = world size).  update_geometry()
    re-cuts the domains from cost-weighted samples (moving average over the
    last five steps); exchange() moves particles to their owners; step()
    computes the accelerations and dL/dx of the own particles for a cotangent
    dL/da, through a tree over own particles followed by ghosts."""
    params: object
    group: object = None
    samples_total: int = 65536
    seed: int = 1211
    history: list = field(default_factory=list)

    def __post_init__(self):
        self.rank, self.world = _world(self.group)
        self.shape = factor_domains(self.world)
        self.halo = Halo(*self.shape)
        self.geometry = uniform_geometry(*self.shape)
        self.halo.set_geometry(self.geometry)
        self._step = 0

    # -- domain decomposition --------------------------------------------------
    def update_geometry(self, pos: torch.Tensor, cost: float) -> Geometry:
        """New cuts from samples of every rank's particles, each rank sampling
        in proportion to its measured cost; averaged with the previous ones."""
        rank, world = self.rank, self.world
        dev = pos.device
        costs = torch.tensor([float(cost)], dtype=torch.float64, device=dev)
        if world > 1:
            allc = [torch.empty_like(costs) for _ in range(world)]
            dist.all_gather(allc, costs, group=self.group)
            costs_all = [float(c.item()) for c in allc]
        else:
            costs_all = [float(cost)]
        m = min(sample_counts(costs_all, self.samples_total)[rank], int(pos.shape[0]))
        g = torch.Generator(device=dev)
        g.manual_seed(self.seed * 1000003 + self._step * 131 + rank)
        pick = torch.randperm(int(pos.shape[0]), generator=g, device=dev)[:m]
        samples = gather_samples(pos.index_select(0, pick), self.group)
        new = multisection(samples, *self.shape)
        self.history = (self.history + [new])[-AVERAGE_STEPS:]
        self.geometry = moving_average(self.history)
        self.halo.set_geometry(self.geometry)
        self._step += 1
        return self.geometry

    def exchange(self, pos: torch.Tensor, mass: torch.Tensor, ids: torch.Tensor):
        """Send every particle to the rank whose domain holds it; returns the
        rank's own particles (positions, masses, global ids)."""
        idx, counts = self.halo.select(pos, "owner")
        p, _ = alltoallv(gather_rows(pos, idx), counts, self.group)
        m, _ = alltoallv(gather_rows(mass, idx), counts, self.group)
        i, _ = alltoallv(gather_rows(ids, idx), counts, self.group)
        return p, m, i

    def ghosts(self, pos: torch.Tensor, mass: torch.Tensor) -> Exchanged:
        """Send the own particles within r_cut of other domains to those
        domains; receive this domain's ghosts."""
        idx, counts = self.halo.select(pos, "ghosts", self.rank, self.params.r_cut)
        gp, rcounts = alltoallv(gather_rows(pos, idx), counts, self.group)
        gm, _ = alltoallv(gather_rows(mass, idx), counts, self.group)
        return Exchanged(idx, counts, rcounts, gp, gm)

    def step(self, pos: torch.Tensor, mass: torch.Tensor, cot: torch.Tensor):
        """(acc [n, 3] float32, grad [n, 3] float64) of the own particles for
        the cotangent cot = dL/da of the own accelerations."""
        from .api import ShortRangeTree
        n = int(pos.shape[0])
        ex = self.ghosts(pos, mass)
        allp = torch.cat([pos, ex.ghost_pos])
        allm = torch.cat([mass, ex.ghost_mass])
        allc = torch.cat([cot.to(torch.float32), torch.zeros_like(ex.ghost_pos, dtype=torch.float32)])
        tree = ShortRangeTree(allp, allm, self.params)
        try:
            acc, grad = tree.force_vjp(allc)
        finally:
            tree.close()
        back, _ = alltoallv(grad[n:], ex.recv_counts, self.group)
        out = grad[:n].contiguous()
        scatter_add_rows(out, ex.send_idx, back)
        return acc[:n], out
