"""CPU FP64 oracle of the short-range TreePM path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  The product path
(the CUDA library and its Python binding) never imports it and shares no code
with it; the two meet only in the seeded input generators.

The arithmetic lives in ``treepm_oracle.c`` (plain C, FP64, no FMA
contraction); this module compiles it with gcc and exposes it through ctypes.
Every function follows the paper (Ishiyama, Nitadori & Makino, SC12):
Eq. 2 (pair sum), Eq. 3 (cutoff g_P3M), the tree algorithm of Sec. I and
Barnes' grouped traversal of Sec. II; the readings where the paper is silent
are listed at the top of the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "treepm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_U64 = C.POINTER(C.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2 -ffp-contract=off -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                               "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    lib.or_g.restype = C.c_double
    lib.or_g.argtypes = [C.c_double]
    lib.or_gpx.restype = C.c_double
    lib.or_gpx.argtypes = [C.c_double]
    for name in ("or_rsqrt_seed", "or_rsqrt_refined"):
        getattr(lib, name).restype = C.c_double
        getattr(lib, name).argtypes = [C.c_double]
    lib.or_rsqrt_third_order.restype = C.c_double
    lib.or_rsqrt_third_order.argtypes = [C.c_double, C.c_double]
    lib.or_pair.argtypes = [_D, C.c_double, C.c_double, C.c_double, C.c_double, _D, C.c_int]
    lib.or_pair_jw.argtypes = [_D, C.c_double, _D, C.c_double, C.c_double, C.c_double, _D, C.c_int]
    lib.or_brute_force.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double, C.c_double, _D, C.c_int]
    lib.or_brute_force_sample.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double, C.c_double,
                                          C.c_int64, _I64, _D, C.c_int]
    lib.or_brute_vjp.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double, C.c_double, _D, _D,
                                 C.c_int]
    lib.or_brute_vjp_sample.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double, C.c_double, _D,
                                        C.c_int64, _I64, _D, C.c_int]
    lib.or_morton.restype = C.c_uint64
    lib.or_morton.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
    lib.or_key_of.restype = C.c_uint64
    lib.or_key_of.argtypes = [C.c_double, C.c_double, C.c_double]
    lib.or_build.restype = C.c_void_p
    lib.or_build.argtypes = [C.c_int64, _D, _D, C.c_int32, C.c_int32]
    lib.or_lists.restype = C.c_int64
    lib.or_lists.argtypes = [C.c_void_p, C.c_double, C.c_double]
    lib.or_list_forces.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _D, C.c_int]
    lib.or_list_vjp.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _D, _D, C.c_int]
    lib.or_list_forces_range.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                         C.c_double, _D, C.c_int]
    lib.or_list_vjp_range.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                      C.c_double, _D, _D, C.c_int]
    lib.or_list_loss_groups.restype = C.c_double
    lib.or_list_loss_groups.argtypes = [C.c_void_p, _I64, C.c_int64, C.c_double, C.c_double, C.c_double, _D,
                                        C.c_int]
    lib.or_count_useful.restype = C.c_int64
    lib.or_count_useful.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int]
    lib.or_refresh_moments.argtypes = [C.c_void_p, _D]
    lib.or_sizes.argtypes = [C.c_void_p, _I64]
    lib.or_export_keys.argtypes = [C.c_void_p, _U64, _I64]
    lib.or_export_nodes.argtypes = [C.c_void_p, _I64, _D]
    lib.or_export_groups.argtypes = [C.c_void_p, _I64, _D]
    lib.or_export_lists.argtypes = [C.c_void_p, _I64, _I64]
    lib.or_free.argtypes = [C.c_void_p]
    lib.or_num_threads.restype = C.c_int
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _variant(xi_softened=False, rsqrt_refined=False) -> int:
    """The variant bitmask of the C functions: 1 = softened cutoff argument,
    2 = the paper's refined inverse square root for 1/s^3."""
    return int(bool(xi_softened)) | (2 if rsqrt_refined else 0)


def rsqrt_seed(x: float) -> float:
    """The estimate of 1/sqrt(x) that the refinement starts from."""
    return float(_load().or_rsqrt_seed(float(x)))


def rsqrt_third_order(x: float, y0: float) -> float:
    """The paper's third-order step from an estimate y0 of 1/sqrt(x)."""
    return float(_load().or_rsqrt_third_order(float(x), float(y0)))


def rsqrt_refined(x: float) -> float:
    """1/sqrt(x) by the paper's refinement of rsqrt_seed(x)."""
    return float(_load().or_rsqrt_refined(float(x)))


def num_threads() -> int:
    return int(_load().or_num_threads())


def g(xi) -> np.ndarray | float:
    """Cutoff function g_P3M of Eq. 3."""
    lib = _load()
    if np.isscalar(xi):
        return lib.or_g(float(xi))
    return np.array([lib.or_g(float(v)) for v in np.ravel(xi)]).reshape(np.shape(xi))


def gpx(xi) -> np.ndarray | float:
    """g'(xi)/xi, Eq. 3 differentiated."""
    lib = _load()
    if np.isscalar(xi):
        return lib.or_gpx(float(xi))
    return np.array([lib.or_gpx(float(v)) for v in np.ravel(xi)]).reshape(np.shape(xi))


def pair(d, mj, G, eps, rcut, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
    """One term of Eq. 2: acceleration from mass mj at offset d = x_j - x_i.
    xi_softened: take the cutoff argument of Eq. 3 from the softened distance
    sqrt(r^2 + eps^2) (the paper's kernel form) instead of r; every force and
    adjoint function below takes the same switch."""
    d = _f64(d)
    out = np.zeros(3)
    _load().or_pair(_dp(d), float(mj), float(G), float(eps), float(rcut), _dp(out), _variant(xi_softened, rsqrt_refined))
    return out


def pair_jw(d, mj, w, G, eps, rcut, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
    """G mj J(d) w for the Jacobian J of one Eq. 2 term."""
    d, w = _f64(d), _f64(w)
    out = np.zeros(3)
    _load().or_pair_jw(_dp(d), float(mj), _dp(w), float(G), float(eps), float(rcut), _dp(out),
                       _variant(xi_softened, rsqrt_refined))
    return out


def brute_force(pos, mass, G, eps, rcut, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
    """Eq. 2 summed over all pairs (O(N^2), periodic minimum image)."""
    pos, mass = _f64(pos), _f64(mass)
    n = pos.shape[0]
    acc = np.zeros((n, 3))
    _load().or_brute_force(n, _dp(pos), _dp(mass), G, eps, rcut, _dp(acc), _variant(xi_softened, rsqrt_refined))
    return acc


def brute_force_sample(pos, mass, G, eps, rcut, idx, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
    pos, mass = _f64(pos), _f64(mass)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    acc = np.zeros((idx.size, 3))
    _load().or_brute_force_sample(pos.shape[0], _dp(pos), _dp(mass), G, eps, rcut, idx.size,
                                  idx.ctypes.data_as(_I64), _dp(acc), _variant(xi_softened, rsqrt_refined))
    return acc


def brute_vjp(pos, mass, G, eps, rcut, w, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
    """dL/dx of L = sum_i w_i . a_i for the direct sum."""
    pos, mass, w = _f64(pos), _f64(mass), _f64(w)
    grad = np.zeros_like(pos)
    _load().or_brute_vjp(pos.shape[0], _dp(pos), _dp(mass), G, eps, rcut, _dp(w), _dp(grad),
                         _variant(xi_softened, rsqrt_refined))
    return grad


def brute_vjp_sample(pos, mass, G, eps, rcut, w, idx, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
    """Rows idx of brute_vjp (each O(N)), for boxes too large for the full sum."""
    pos, mass, w = _f64(pos), _f64(mass), _f64(w)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    grad = np.zeros((idx.size, 3))
    _load().or_brute_vjp_sample(pos.shape[0], _dp(pos), _dp(mass), G, eps, rcut, _dp(w), idx.size,
                                idx.ctypes.data_as(_I64), _dp(grad), _variant(xi_softened, rsqrt_refined))
    return grad


def morton(qx: int, qy: int, qz: int) -> int:
    return int(_load().or_morton(qx, qy, qz))


def key_of(x: float, y: float, z: float) -> int:
    return int(_load().or_key_of(x, y, z))


@dataclass
class Tree:
    """Snapshot of an oracle tree (all arrays in key order unless noted)."""
    n: int
    keys: np.ndarray           # uint64 [n]
    perm: np.ndarray           # int64  [n]  sorted -> input index
    level: np.ndarray          # per node
    first: np.ndarray
    count: np.ndarray
    child: np.ndarray
    nchild: np.ndarray
    parent: np.ndarray
    M: np.ndarray
    com: np.ndarray            # [nodes,3]
    lo: np.ndarray
    hi: np.ndarray
    cen: np.ndarray
    half: np.ndarray
    gfirst: np.ndarray
    gcount: np.ndarray
    gcen: np.ndarray
    ghalf: np.ndarray
    loff: np.ndarray | None = None
    ent: np.ndarray | None = None


class OracleTree:
    """Owns one oracle tree built from (pos, mass)."""

    def __init__(self, pos, mass=None, n_leaf: int = 8, n_crit: int = 64):
        lib = _load()
        self.pos = _f64(pos)
        self.mass = None if mass is None else _f64(mass)
        self.n = self.pos.shape[0]
        h = lib.or_build(self.n, _dp(self.pos), _dp(self.mass) if self.mass is not None else None,
                         n_leaf, n_crit)
        if not h:
            raise ValueError("oracle rejected the tree parameters")
        self._h = h
        self.has_lists = False

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().or_free(h)
            self._h = None

    def sizes(self):
        s = np.zeros(4, dtype=np.int64)
        _load().or_sizes(self._h, s.ctypes.data_as(_I64))
        return [int(v) for v in s]

    def lists(self, rcut: float, theta: float) -> int:
        n_ent = int(_load().or_lists(self._h, rcut, theta))
        self.has_lists = True
        return n_ent

    def list_forces(self, G, eps, rcut, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
        assert self.has_lists
        acc = np.zeros((self.n, 3))
        _load().or_list_forces(self._h, G, eps, rcut, _dp(acc), _variant(xi_softened, rsqrt_refined))
        return acc

    def list_vjp(self, G, eps, rcut, w, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
        assert self.has_lists
        w = _f64(w)
        grad = np.zeros((self.n, 3))
        _load().or_list_vjp(self._h, G, eps, rcut, _dp(w), _dp(grad), _variant(xi_softened, rsqrt_refined))
        return grad

    def list_forces_range(self, g0, g1, G, eps, rcut, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
        """Forces of groups [g0, g1) only (other rows stay zero)."""
        assert self.has_lists
        acc = np.zeros((self.n, 3))
        _load().or_list_forces_range(self._h, int(g0), int(g1), G, eps, rcut, _dp(acc),
                                     _variant(xi_softened, rsqrt_refined))
        return acc

    def list_vjp_range(self, g0, g1, G, eps, rcut, w, xi_softened=False, rsqrt_refined=False) -> np.ndarray:
        """Gradient of sum over groups [g0, g1) of w_i . a_i."""
        assert self.has_lists
        w = _f64(w)
        grad = np.zeros((self.n, 3))
        _load().or_list_vjp_range(self._h, int(g0), int(g1), G, eps, rcut, _dp(w), _dp(grad),
                                  _variant(xi_softened, rsqrt_refined))
        return grad

    def list_loss_groups(self, groups, G, eps, rcut, w, xi_softened=False, rsqrt_refined=False) -> float:
        """sum over the given groups' particles i of w_i . a_i (list forces)."""
        assert self.has_lists
        g = np.ascontiguousarray(groups, dtype=np.int64)
        w = _f64(w)
        return float(_load().or_list_loss_groups(self._h, g.ctypes.data_as(_I64), g.size, G, eps, rcut, _dp(w),
                                                 _variant(xi_softened, rsqrt_refined)))

    def count_useful(self, eps, rcut, xi_softened=False) -> int:
        """Pairs (group particle, list entry other than itself) at a positive
        distance whose cutoff distance (r, or sqrt(r^2 + eps^2) with
        xi_softened) is below r_cut: the evaluated pairs whose Eq. 2 term is not
        identically zero."""
        assert self.has_lists
        return int(_load().or_count_useful(self._h, eps, rcut, int(bool(xi_softened))))

    def refresh(self, pos) -> None:
        """Re-take monopoles from new positions with the structure frozen."""
        pos = _f64(pos)
        _load().or_refresh_moments(self._h, _dp(pos))

    def export(self) -> Tree:
        lib = _load()
        n, nn, ng, ne = self.sizes()
        keys = np.zeros(n, dtype=np.uint64)
        perm = np.zeros(n, dtype=np.int64)
        lib.or_export_keys(self._h, keys.ctypes.data_as(_U64), perm.ctypes.data_as(_I64))
        ints = np.zeros((nn, 6), dtype=np.int64)
        dbl = np.zeros((nn, 16))
        lib.or_export_nodes(self._h, ints.ctypes.data_as(_I64), _dp(dbl))
        gi = np.zeros((ng, 2), dtype=np.int64)
        gd = np.zeros((ng, 6))
        lib.or_export_groups(self._h, gi.ctypes.data_as(_I64), _dp(gd))
        loff = ent = None
        if self.has_lists:
            loff = np.zeros(ng + 1, dtype=np.int64)
            ent = np.zeros(max(ne, 1), dtype=np.int64)
            lib.or_export_lists(self._h, loff.ctypes.data_as(_I64), ent.ctypes.data_as(_I64))
            ent = ent[:ne]
        return Tree(n=n, keys=keys, perm=perm, level=ints[:, 0], first=ints[:, 1],
                    count=ints[:, 2], child=ints[:, 3], nchild=ints[:, 4], parent=ints[:, 5],
                    M=dbl[:, 0], com=dbl[:, 1:4], lo=dbl[:, 4:7], hi=dbl[:, 7:10],
                    cen=dbl[:, 10:13], half=dbl[:, 13:16], gfirst=gi[:, 0], gcount=gi[:, 1],
                    gcen=gd[:, 0:3], ghalf=gd[:, 3:6], loff=loff, ent=ent)


def tree_forces(pos, mass, G, eps, rcut, theta, n_leaf=8, n_crit=64, xi_softened=False, rsqrt_refined=False):
    """Build, list and sum: the oracle's whole short-range force path."""
    t = OracleTree(pos, mass, n_leaf, n_crit)
    t.lists(rcut, theta)
    return t.list_forces(G, eps, rcut, xi_softened), t


def leapfrog(pos0, vel0, mass, G, eps, rcut, theta, dt, steps, n_leaf=8, n_crit=64,
             keep_trees=False):
    """Kick-drift-kick leapfrog with the short-range force only, rebuilding the
    tree every force evaluation.  Returns (x_T, v_T, a_T, trees); `trees` holds
    the oracle tree of each evaluation when keep_trees is set (for frozen-
    structure finite differences and the adjoint)."""
    x = _f64(pos0).copy()
    v = _f64(vel0).copy()
    trees = []
    a, t = tree_forces(x, mass, G, eps, rcut, theta, n_leaf, n_crit)
    if keep_trees:
        trees.append(t)
    for _ in range(steps):
        v = v + a * (0.5 * dt)
        x = x + v * dt
        a, t = tree_forces(x, mass, G, eps, rcut, theta, n_leaf, n_crit)
        if keep_trees:
            trees.append(t)
        v = v + a * (0.5 * dt)
    return x, v, a, trees


def leapfrog_frozen(pos0, vel0, trees, G, eps, rcut, dt, steps):
    """The same integration with every force evaluation's structure frozen to
    the given trees (monopoles re-taken from the current positions).
    Returns (x_T, v_T, a_T)."""
    x = _f64(pos0).copy()
    v = _f64(vel0).copy()

    def force(t):
        t.refresh(x)
        return t.list_forces(G, eps, rcut)

    a = force(trees[0])
    for s in range(steps):
        v = v + a * (0.5 * dt)
        x = x + v * dt
        a = force(trees[s + 1])
        v = v + a * (0.5 * dt)
    return x, v, a


def leapfrog_adjoint(pos0, vel0, trees, G, eps, rcut, dt, steps, g_xT, g_vT, g_aT):
    """Reverse-mode derivative of leapfrog_frozen: given dL/dx_T, dL/dv_T and
    dL/da_T returns (dL/dx_0, dL/dv_0).  Each step v_h = v + a dt/2,
    x1 = x + v_h dt, a1 = F(x1), v1 = v_h + a1 dt/2 is reversed as
    g_a1 += (dt/2) g_v1; g_x1 += VJP_F(x1)[g_a1]; g_vh = g_v1 + dt g_x1;
    g_a = (dt/2) g_vh, with VJP_F the list adjoint of each frozen tree."""
    xs = [_f64(pos0).copy()]
    x = xs[0]
    v = _f64(vel0).copy()
    trees[0].refresh(x)
    a = trees[0].list_forces(G, eps, rcut)
    for s in range(steps):
        v = v + a * (0.5 * dt)
        x = x + v * dt
        xs.append(x)
        trees[s + 1].refresh(x)
        a = trees[s + 1].list_forces(G, eps, rcut)
        v = v + a * (0.5 * dt)
    gx, gv, ga = _f64(g_xT).copy(), _f64(g_vT).copy(), _f64(g_aT).copy()
    for s in range(steps, 0, -1):
        ga = ga + 0.5 * dt * gv
        trees[s].refresh(xs[s])
        gx = gx + trees[s].list_vjp(G, eps, rcut, ga)
        gvh = gv + dt * gx
        ga = 0.5 * dt * gvh
        gv = gvh
    trees[0].refresh(xs[0])
    gx = gx + trees[0].list_vjp(G, eps, rcut, ga)
    return gx, gv
