"""Python front end of the short-range TreePM library.

Thin marshalling over the C-ABI: torch tensors on the GPU supply device
pointers, torch's current stream supplies the CUDA stream, and every step of
the path runs in libtreepm_sr.so.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _order(stream, *tensors) -> None:
    """Make a call on `stream` safe for tensors prepared on torch's current
    stream.  The conversions and allocations of the binding (contiguous
    copies, dtype casts, outputs) run on the current stream; when the library
    is given another stream, that stream first waits for the current one, and
    each tensor is recorded on it, so that the caching allocator does not hand
    its memory to someone else while the library still reads or writes it."""
    if stream is None:
        return
    cur = torch.cuda.current_stream(stream.device)
    if stream == cur:
        return
    stream.wait_stream(cur)
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def _dev_f64(x: torch.Tensor, shape_last=None) -> torch.Tensor:
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if x.dtype != torch.float64:
        raise TypeError("positions and masses must be float64")
    x = x.contiguous()
    if shape_last is not None and (x.dim() != 2 or x.shape[1] != shape_last):
        raise ValueError(f"expected shape [n, {shape_last}]")
    return x


def _dev_mass(mass, n: int):
    """Masses as a float64 CUDA tensor [n], or None (every mass 1/n).  The
    library reads n values, so the length is checked here."""
    if mass is None:
        return None
    mass = _dev_f64(mass)
    if mass.dim() != 1 or mass.shape[0] != n:
        raise ValueError(f"mass must be a float64 CUDA tensor [n] with n = {n}")
    return mass


def _dev_vec3(x, n: int, dtype, name: str) -> torch.Tensor:
    """A contiguous CUDA buffer [n, 3] of `dtype` that the library reads or
    writes in full."""
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != dtype or not x.is_contiguous() \
            or tuple(x.shape) != (n, 3):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor [n, 3] with n = {n}")
    return x


def _dev_cot(cot, n: int, dtype) -> torch.Tensor:
    """A cotangent dL/da [n, 3] (any float dtype, converted to `dtype`)."""
    if not isinstance(cot, torch.Tensor) or not cot.is_cuda or not cot.is_floating_point() \
            or tuple(cot.shape) != (n, 3):
        raise ValueError(f"cot must be a floating-point CUDA tensor [n, 3] with n = {n}")
    return cot.to(dtype).contiguous()


@dataclass
class Params:
    """Short-range parameters of one periodic unit box (Sec. II, III-A)."""
    G: float = 1.0
    eps: float = 0.0
    r_cut: float = 0.1
    theta: float = 0.5
    n_crit: int = 64
    n_leaf: int = 8
    precision: str = "fp32"
    chunked: bool = False     # force the bounded-list-memory mode (TP_FLAG_CHUNKED)
    xi: str = "plain"         # cutoff argument of Eq. 3: "plain" r or "softened" sqrt(r^2+eps^2)
    rsqrt: str = "hardware"   # 1/s: the "hardware" MUFU root or the paper's "refined" estimate

    def c(self) -> _lib.TPParams:
        if self.xi not in ("plain", "softened"):
            raise ValueError(f"xi must be 'plain' or 'softened', not {self.xi!r}")
        if self.rsqrt not in ("hardware", "refined"):
            raise ValueError(f"rsqrt must be 'hardware' or 'refined', not {self.rsqrt!r}")
        p = _lib.params(self.G, self.eps, self.r_cut, self.theta, self.n_crit, self.n_leaf,
                        self.precision)
        p.flags = ((_lib.TP_FLAG_CHUNKED if self.chunked else 0) |
                   (_lib.TP_FLAG_XI_SOFTENED if self.xi == "softened" else 0) |
                   (_lib.TP_FLAG_RSQRT_REFINED if self.rsqrt == "refined" else 0))
        return p


class ShortRangeTree:
    """A built tree (keys, octree, monopoles, groups, interaction lists) over
    one box or a batch of independent boxes, owned by the library."""

    def __init__(self, pos: torch.Tensor, mass: torch.Tensor | None, params,
                 box_offsets=None, stream=None):
        lib = _lib.load()
        pos = _dev_f64(pos, 3)
        self.n = int(pos.shape[0])
        mass = _dev_mass(mass, self.n)
        if isinstance(params, Params):
            params = [params]
        params = list(params)
        if box_offsets is None:
            box_offsets = [0, self.n]
        box_offsets = [int(v) for v in box_offsets]
        if len(box_offsets) != len(params) + 1 or box_offsets[-1] != self.n:
            raise ValueError("box_offsets must have len(params)+1 entries ending at n")
        self.params = params
        self.box_offsets = box_offsets
        self.precision = params[0].precision
        self.acc_dtype = torch.float32 if self.precision == "fp32" else torch.float64
        self._pos, self._mass = pos, mass          # keep alive until the build completes
        _order(stream, pos, mass)
        arr = (C.c_int64 * len(box_offsets))(*box_offsets)
        prm = (_lib.TPParams * len(params))(*[p.c() for p in params])
        h = C.c_void_p()
        code = lib.tp_build_tree_batched(C.c_void_p(pos.data_ptr()),
                                         C.c_void_p(mass.data_ptr()) if mass is not None else None,
                                         arr, len(params), prm, _stream(stream), C.byref(h))
        _lib.check(code, "tp_build_tree_batched")
        self._h = h

    # -- lifetime -----------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.load().tp_tree_free(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise RuntimeError("tree has been freed")
        return self._h

    # -- path ---------------------------------------------------------------
    def rebuild(self, pos: torch.Tensor, mass: torch.Tensor | None = None, stream=None) -> None:
        pos = _dev_f64(pos, 3)
        if pos.shape[0] != self.n:
            raise ValueError("rebuild needs the same particle count")
        mass = _dev_mass(mass, self.n)
        self._pos, self._mass = pos, mass
        _order(stream, pos, mass)
        code = _lib.load().tp_rebuild_tree(self.handle, C.c_void_p(pos.data_ptr()),
                                           C.c_void_p(mass.data_ptr()) if mass is not None else None,
                                           _stream(stream))
        _lib.check(code, "tp_rebuild_tree")

    def refit(self, pos: torch.Tensor, mass: torch.Tensor | None = None, stream=None) -> None:
        """Keep structure, groups and lists; refresh images, monopoles and
        entry records from new positions (same particles, small moves)."""
        pos = _dev_f64(pos, 3)
        if pos.shape[0] != self.n:
            raise ValueError("refit needs the same particle count")
        mass = _dev_mass(mass, self.n)
        self._pos, self._mass = pos, mass
        _order(stream, pos, mass)
        code = _lib.load().tp_refit_tree(self.handle, C.c_void_p(pos.data_ptr()),
                                         C.c_void_p(mass.data_ptr()) if mass is not None else None,
                                         _stream(stream))
        _lib.check(code, "tp_refit_tree")

    def force(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Short-range accelerations (Eq. 2), [n, 3] in input order."""
        if out is None:
            out = torch.empty((self.n, 3), dtype=self.acc_dtype, device=self._pos.device)
        _dev_vec3(out, self.n, self.acc_dtype, "out (the tree's precision)")
        _order(stream, out)
        code = _lib.load().tp_short_range_force(self.handle, C.c_void_p(out.data_ptr()), _stream(stream))
        _lib.check(code, "tp_short_range_force")
        return out

    def vjp(self, cot: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """dL/dx (float64 [n,3]) for the cotangent dL/da of the force."""
        cot = _dev_cot(cot, self.n, self.acc_dtype)
        if out is None:
            out = torch.empty((self.n, 3), dtype=torch.float64, device=self._pos.device)
        _dev_vec3(out, self.n, torch.float64, "out")
        _order(stream, cot, out)
        code = _lib.load().tp_short_range_vjp(self.handle, C.c_void_p(cot.data_ptr()),
                                              C.c_void_p(out.data_ptr()), _stream(stream))
        _lib.check(code, "tp_short_range_vjp")
        return out

    def force_vjp(self, cot: torch.Tensor, acc: torch.Tensor | None = None, grad: torch.Tensor | None = None,
                  stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """(forces, dL/dx) in one pass over the lists, for a cotangent known in advance."""
        cot = _dev_cot(cot, self.n, self.acc_dtype)
        dev = self._pos.device
        if acc is None:
            acc = torch.empty((self.n, 3), dtype=self.acc_dtype, device=dev)
        if grad is None:
            grad = torch.empty((self.n, 3), dtype=torch.float64, device=dev)
        _dev_vec3(acc, self.n, self.acc_dtype, "acc (the tree's precision)")
        _dev_vec3(grad, self.n, torch.float64, "grad")
        _order(stream, cot, acc, grad)
        code = _lib.load().tp_short_range_force_vjp(self.handle, C.c_void_p(acc.data_ptr()),
                                                    C.c_void_p(cot.data_ptr()), C.c_void_p(grad.data_ptr()),
                                                    _stream(stream))
        _lib.check(code, "tp_short_range_force_vjp")
        return acc, grad

    def status(self) -> int:
        return int(_lib.load().tp_tree_status(self.handle))

    # -- tuning and kernel timing ----------------------------------------------
    def set_tile(self, fwd_particles: int = 2, adj_entries: int = 4) -> None:
        """Particles per thread of the forward pair kernel (1, 2, 4) and list
        entries per thread of the adjoint kernel (2, 4; or 8, held as four
        pairs of entries in the one-pass kernel, 4 for the adjoint alone)."""
        _lib.check(_lib.load().tp_tree_set_tile(self.handle, int(fwd_particles), int(adj_entries)),
                   "tp_tree_set_tile")
        self.tile = (int(fwd_particles), int(adj_entries))

    def set_walk_budget(self, budget: int = 0) -> None:
        """Failure injection: cap the node visits of every walk of later builds
        (0 restores the default); a walk that runs out latches TP_ERR_TIMEOUT."""
        _lib.check(_lib.load().tp_tree_set_walk_budget(self.handle, int(budget)), "tp_tree_set_walk_budget")

    def set_kernel_timing(self, enable: bool = True) -> None:
        _lib.check(_lib.load().tp_tree_set_kernel_timing(self.handle, 1 if enable else 0),
                   "tp_tree_set_kernel_timing")

    def kernel_ms(self) -> tuple[float, float]:
        """(force, vjp) launch durations in ms of the last timed calls (-1: none)."""
        f, v = C.c_double(), C.c_double()
        _lib.check(_lib.load().tp_tree_kernel_ms(self.handle, C.byref(f), C.byref(v)), "tp_tree_kernel_ms")
        return f.value, v.value

    # -- statistics and parity exports ----------------------------------------
    def stats(self) -> dict:
        st = _lib.TPStats()
        _lib.check(_lib.load().tp_tree_stats(self.handle, C.byref(st)), "tp_tree_stats")
        return {f: getattr(st, f) for f, _ in _lib.TPStats._fields_}

    def export_keys(self):
        n = self.n
        keys = np.zeros(n, dtype=np.uint64)
        perm = np.zeros(n, dtype=np.int64)
        _lib.check(_lib.load().tp_export_keys(self.handle, keys.ctypes.data_as(C.c_void_p),
                                              perm.ctypes.data_as(C.c_void_p)), "tp_export_keys")
        return keys, perm

    def export_nodes(self):
        nn = self.stats()["n_nodes"]
        ints = np.zeros((max(nn, 1), 7), dtype=np.int64)
        dbl = np.zeros((max(nn, 1), 16))
        _lib.check(_lib.load().tp_export_nodes(self.handle, ints.ctypes.data_as(C.c_void_p),
                                               dbl.ctypes.data_as(C.c_void_p)), "tp_export_nodes")
        return ints[:nn], dbl[:nn]

    def export_groups(self):
        ng = self.stats()["n_groups"]
        ints = np.zeros((max(ng, 1), 3), dtype=np.int64)
        dbl = np.zeros((max(ng, 1), 6))
        _lib.check(_lib.load().tp_export_groups(self.handle, ints.ctypes.data_as(C.c_void_p),
                                                dbl.ctypes.data_as(C.c_void_p)), "tp_export_groups")
        return ints[:ng], dbl[:ng]

    def export_lists(self):
        st = self.stats()
        off = np.zeros(st["n_groups"] + 1, dtype=np.int64)
        ent = np.zeros(max(st["n_entries"], 1), dtype=np.int32)
        _lib.check(_lib.load().tp_export_lists(self.handle, off.ctypes.data_as(C.c_void_p),
                                               ent.ctypes.data_as(C.c_void_p)), "tp_export_lists")
        return off, ent[:st["n_entries"]]


class PMSolver:
    """The long-range (PM) half (Sec. II): an n_mesh^3 periodic mesh with its
    Green's function and FFT plans, owned by the library.  force() runs the PM
    cycle (TSC assignment, FFT, Green's function, four-point difference, TSC
    interpolation); with the same r_cut and G it completes ShortRangeTree's
    short-range force to the whole TreePM acceleration."""

    def __init__(self, n_mesh: int, r_cut: float, G: float = 1.0, stream=None):
        h = C.c_void_p()
        _lib.check(_lib.load().tp_pm_create(int(n_mesh), float(r_cut), float(G), _stream(stream), C.byref(h)),
                   "tp_pm_create")
        self._h = h
        self.n_mesh, self.r_cut, self.G = int(n_mesh), float(r_cut), float(G)

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.load().tp_pm_free(h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def force(self, pos: torch.Tensor, mass: torch.Tensor | None = None, out: torch.Tensor | None = None,
              accumulate: bool = False, stream=None) -> torch.Tensor:
        """Long-range accelerations [n, 3] (FP32, input order); added to `out`
        when accumulate is set (e.g. onto the short-range force)."""
        if self._h is None:
            raise RuntimeError("PM solver has been freed")
        pos = _dev_f64(pos, 3)
        n = int(pos.shape[0])
        mass = _dev_mass(mass, n)
        if out is None:
            if accumulate:
                raise ValueError("accumulate needs out")
            out = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        _dev_vec3(out, n, torch.float32, "out")
        _order(stream, pos, mass, out)
        code = _lib.load().tp_pm_force(self._h, C.c_void_p(pos.data_ptr()),
                                       C.c_void_p(mass.data_ptr()) if mass is not None else None, n,
                                       C.c_void_p(out.data_ptr()), int(bool(accumulate)), _stream(stream))
        _lib.check(code, "tp_pm_force")
        return out

    def vjp(self, pos: torch.Tensor, mass: torch.Tensor | None, cot: torch.Tensor, out: torch.Tensor | None = None,
            accumulate: bool = False, stream=None) -> torch.Tensor:
        """dL/dx (float64 [n, 3]) of L = sum_i cot_i . a_i over the PM cycle;
        added to `out` when accumulate is set (e.g. onto the short-range VJP)."""
        pos, mass, cot, out = self._adjoint_args(pos, mass, cot, out, accumulate)
        _order(stream, pos, mass, cot, out)
        code = _lib.load().tp_pm_vjp(self._h, C.c_void_p(pos.data_ptr()),
                                     C.c_void_p(mass.data_ptr()) if mass is not None else None, int(pos.shape[0]),
                                     C.c_void_p(cot.data_ptr()), C.c_void_p(out.data_ptr()), int(bool(accumulate)),
                                     _stream(stream))
        _lib.check(code, "tp_pm_vjp")
        return out

    def force_vjp(self, pos: torch.Tensor, mass: torch.Tensor | None, cot: torch.Tensor,
                  acc: torch.Tensor | None = None, grad: torch.Tensor | None = None, accumulate: bool = False,
                  stream=None):
        """force() and vjp() with one mesh-force computation; returns (acc, grad)."""
        pos, mass, cot, grad = self._adjoint_args(pos, mass, cot, grad, accumulate)
        n = int(pos.shape[0])
        if acc is None:
            if accumulate:
                raise ValueError("accumulate needs acc")
            acc = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        _dev_vec3(acc, n, torch.float32, "acc")
        _order(stream, pos, mass, cot, acc, grad)
        code = _lib.load().tp_pm_force_vjp(self._h, C.c_void_p(pos.data_ptr()),
                                           C.c_void_p(mass.data_ptr()) if mass is not None else None, n,
                                           C.c_void_p(acc.data_ptr()), C.c_void_p(cot.data_ptr()),
                                           C.c_void_p(grad.data_ptr()), int(bool(accumulate)), _stream(stream))
        _lib.check(code, "tp_pm_force_vjp")
        return acc, grad

    def _adjoint_args(self, pos, mass, cot, out, accumulate):
        if self._h is None:
            raise RuntimeError("PM solver has been freed")
        pos = _dev_f64(pos, 3)
        n = int(pos.shape[0])
        mass = _dev_mass(mass, n)
        if not isinstance(cot, torch.Tensor) or not cot.is_cuda or cot.dtype != torch.float32 \
                or tuple(cot.shape) != (n, 3):
            raise ValueError("cot must be a float32 CUDA tensor [n,3]")
        cot = cot.contiguous()
        if out is None:
            if accumulate:
                raise ValueError("accumulate needs out")
            out = torch.empty((n, 3), dtype=torch.float64, device=pos.device)
        _dev_vec3(out, n, torch.float64, "out")
        return pos, mass, cot, out

    def export_mesh(self, which: str = "potential") -> np.ndarray:
        """The potential [N,N,N] or the mesh acceleration [N,N,N,3] of the last
        force() call (synchronous copy)."""
        N = self.n_mesh
        idx = {"potential": 0, "acceleration": 1}[which]
        out = np.zeros((N, N, N) if idx == 0 else (N, N, N, 3), dtype=np.float32)
        _lib.check(_lib.load().tp_pm_export_mesh(self._h, idx, out.ctypes.data_as(C.c_void_p)),
                   "tp_pm_export_mesh")
        return out


def short_range_force(pos: torch.Tensor, mass: torch.Tensor | None, params: Params,
                      stream=None) -> torch.Tensor:
    """Build and evaluate in one call (the tree is freed afterwards)."""
    t = ShortRangeTree(pos, mass, params, stream=stream)
    try:
        return t.force(stream=stream)
    finally:
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        t.close()


def axpy(y: torch.Tensor, x: torch.Tensor, a: float, stream=None) -> None:
    """y += a * x in the library (y float64; x float32 or float64, as many
    elements as y; both contiguous CUDA tensors)."""
    if not (isinstance(y, torch.Tensor) and isinstance(x, torch.Tensor) and y.is_cuda and x.is_cuda):
        raise TypeError("x and y must be CUDA tensors")
    if y.dtype != torch.float64 or not y.is_contiguous() or not x.is_contiguous():
        raise TypeError("y must be contiguous float64, x contiguous")
    if x.dtype not in (torch.float32, torch.float64) or x.numel() != y.numel():
        raise ValueError("x must be float32 or float64 with as many elements as y")
    code = _lib.load().tp_axpy(C.c_void_p(y.data_ptr()), C.c_void_p(x.data_ptr()),
                               1 if x.dtype == torch.float32 else 0, float(a), y.numel(), _stream(stream))
    _lib.check(code, "tp_axpy")


def scale(out: torch.Tensor, x: torch.Tensor, a: float, stream=None) -> None:
    """out = a * x in the library (x float64; out float32 or float64, as many
    elements as x; both contiguous CUDA tensors)."""
    if not (isinstance(out, torch.Tensor) and isinstance(x, torch.Tensor) and out.is_cuda and x.is_cuda):
        raise TypeError("out and x must be CUDA tensors")
    if x.dtype != torch.float64 or not x.is_contiguous() or not out.is_contiguous():
        raise TypeError("x must be contiguous float64, out contiguous")
    if out.dtype not in (torch.float32, torch.float64) or out.numel() != x.numel():
        raise ValueError("out must be float32 or float64 with as many elements as x")
    code = _lib.load().tp_scale(C.c_void_p(out.data_ptr()), 1 if out.dtype == torch.float32 else 0,
                                C.c_void_p(x.data_ptr()), float(a), x.numel(), _stream(stream))
    _lib.check(code, "tp_scale")


def measure_peak(kind: str, stream=None) -> float:
    """FLOP/s of a dependency-free FMA loop: 'fp32', 'fp32x2' or 'fp64'."""
    k = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    v = C.c_double()
    _lib.check(_lib.load().tp_measure_peak(k, C.byref(v), _stream(stream)), "tp_measure_peak")
    return v.value


def launch_count() -> int:
    return int(_lib.load().tp_launch_count())


class CapturedStep:
    """One whole hot-path step -- rebuild, then the forces and their adjoint
    for the fixed cotangent `cot` in one pass -- captured once in a CUDA graph
    and replayed with a single launch.  With a PMSolver `pm` (same r_cut and
    G) the long-range force and adjoint are added onto both outputs in the
    same graph: the whole TreePM step.  `pos` (and `mass`,
    `cot`) are read in place at every replay; `acc` and `grad` are written.
    The tree keeps the capacities of its allocating build: check
    tree.status() after replays whose particles moved far."""

    def __init__(self, tree: ShortRangeTree, pos: torch.Tensor, mass, cot: torch.Tensor,
                 acc: torch.Tensor, grad: torch.Tensor, with_vjp: bool = True, pm: "PMSolver | None" = None):
        if tree.stats()["n_windows"] > 1:
            raise ValueError("a tree in chunked mode (bounded list memory) plans its windows with a host "
                             "synchronisation and cannot be captured in a CUDA graph")
        self.tree, self.pos, self.mass, self.cot, self.acc, self.grad = tree, pos, mass, cot, acc, grad
        self.with_vjp, self.pm = with_vjp, pm
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self._body()                       # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="relaxed"):
            self._body()

    def _body(self):
        self.tree.rebuild(self.pos, self.mass)
        if self.with_vjp:                    # the cotangent is fixed: forces and adjoint in one pass
            self.tree.force_vjp(self.cot, self.acc, self.grad)
            if self.pm is not None:          # the long-range half added onto both
                self.pm.force_vjp(self.pos, self.mass, self.cot, acc=self.acc, grad=self.grad, accumulate=True)
        else:
            self.tree.force(self.acc)
            if self.pm is not None:
                self.pm.force(self.pos, self.mass, out=self.acc, accumulate=True)

    def replay(self):
        self.graph.replay()
