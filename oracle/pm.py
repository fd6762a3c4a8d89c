"""CPU FP64 oracle of the long-range (PM) half of TreePM -- TEST INFRASTRUCTURE
ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this module; the CUDA library shares no code with
it.

It follows the PM cycle of Sec. II-B (Ishiyama, Nitadori & Makino, SC12) step by
step, in plain numpy over an N^3 periodic mesh of the unit box (spacing
h = 1/N, mesh point (i, j, k) at (i h, j h, k h)):

  1. assign      mass density by the triangular-shaped cloud (TSC): each
                 particle reaches the 3 x 3 x 3 mesh points around its nearest
                 one (27 points)
  2. potential   FFT of the density, product with the Green's function of the
                 long-range force, inverse FFT
  3. gradient    four-point finite difference of the potential on the mesh
  4. interpolate the mesh force back to each particle with the same TSC weights

The long-range force is what the PP cutoff g_P3M of Eq. 3 leaves out: the
force between two S2 clouds of radius r_cut/2 (the density of Eq. 1), whose
Fourier transform is S(k)^2 times Newton's.  Readings where the paper is
silent (each is listed in the design notes):
  - Green's function: -4 pi G S(k)^2 / k^2, divided by the square of the TSC
    window W(k) = prod_axes sinc(k_a h / 2)^3 (once for the assignment, once
    for the interpolation); zero for k = 0 (the mean density is removed, as in
    a periodic Ewald sum).
  - the four-point difference is (8 (P[i+1] - P[i-1]) - (P[i+2] - P[i-2])) / 12h.
  - the softening eps does not enter the PM part (eps << r_cut).
"""
from __future__ import annotations

import numpy as np


def s2_transform(x):
    """Fourier transform of the unit-mass S2 density of Eq. 1 at x = k r_cut/2:
    12 (2 - 2 cos x - x sin x) / x^4.  Below x = 0.3 the bracket (about
    x^4 / 12) cancels in the closed form, so the Taylor series to x^8 is used
    there (its first omitted term is below 1e-14)."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(all="ignore"):
        closed = 12.0 * (2.0 - 2.0 * np.cos(x) - x * np.sin(x)) / x ** 4
    x2 = x * x
    series = 1.0 + x2 * (-1.0 / 15.0 + x2 * (1.0 / 560.0 + x2 * (-1.0 / 37800.0 + x2 / 3991680.0)))
    return np.where(np.abs(x) < 0.3, series, closed)


def tsc_weights(d):
    """TSC weights of the mesh points at offsets -1, 0, +1 from the nearest
    one, for a particle d (in mesh units, |d| <= 1/2) away from it."""
    d = np.asarray(d, dtype=np.float64)
    return np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2])


def _stencil(pos, n_mesh):
    """Nearest mesh point (integer, per axis) and the TSC weights [3 axes][3 offsets][n]."""
    u = (np.asarray(pos, dtype=np.float64) % 1.0) * n_mesh
    i0 = np.rint(u).astype(np.int64)
    d = u - i0
    return i0, [tsc_weights(d[:, a]) for a in range(3)]


def assign(pos, mass, n_mesh):
    """Step 1: mass density on the mesh (mass per cell / h^3)."""
    i0, w = _stencil(pos, n_mesh)
    mass = np.asarray(mass, dtype=np.float64)
    rho = np.zeros((n_mesh,) * 3)
    h3 = (1.0 / n_mesh) ** 3
    for a in range(3):
        for b in range(3):
            for c in range(3):
                idx = ((i0[:, 0] + a - 1) % n_mesh, (i0[:, 1] + b - 1) % n_mesh,
                       (i0[:, 2] + c - 1) % n_mesh)
                np.add.at(rho, idx, mass * w[0][a] * w[1][b] * w[2][c] / h3)
    return rho


def green(n_mesh, r_cut, G):
    """Step 2's Green's function on the FFT grid (numpy fftn frequency order)."""
    h = 1.0 / n_mesh
    k1 = 2.0 * np.pi * np.fft.fftfreq(n_mesh, d=h)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    s = s2_transform(np.sqrt(k2) * (0.5 * r_cut))

    def sinc(t):
        with np.errstate(all="ignore"):
            return np.where(t == 0.0, 1.0, np.sin(t) / np.where(t == 0.0, 1.0, t))

    window = (sinc(0.5 * h * kx) * sinc(0.5 * h * ky) * sinc(0.5 * h * kz)) ** 3
    with np.errstate(all="ignore"):
        gk = np.where(k2 > 0.0, -4.0 * np.pi * G * s * s / (k2 * window * window), 0.0)
    return gk


def potential(rho, gk):
    """Step 2: the long-range potential on the mesh."""
    return np.real(np.fft.ifftn(gk * np.fft.fftn(rho)))


def gradient(phi):
    """Step 3: the mesh acceleration -grad(phi) by the four-point difference."""
    n_mesh = phi.shape[0]
    h = 1.0 / n_mesh
    out = []
    for a in range(3):
        d = (8.0 * (np.roll(phi, -1, a) - np.roll(phi, 1, a))
             - (np.roll(phi, -2, a) - np.roll(phi, 2, a))) / (12.0 * h)
        out.append(-d)
    return out


def interpolate(pos, amesh):
    """Step 4: the mesh acceleration at each particle, TSC weights."""
    n_mesh = amesh[0].shape[0]
    i0, w = _stencil(pos, n_mesh)
    acc = np.zeros((i0.shape[0], 3))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                idx = ((i0[:, 0] + a - 1) % n_mesh, (i0[:, 1] + b - 1) % n_mesh,
                       (i0[:, 2] + c - 1) % n_mesh)
                wt = w[0][a] * w[1][b] * w[2][c]
                for q in range(3):
                    acc[:, q] += wt * amesh[q][idx]
    return acc


def pm_forces(pos, mass, n_mesh, r_cut, G):
    """The whole PM cycle: long-range accelerations of every particle."""
    rho = assign(pos, mass, n_mesh)
    phi = potential(rho, green(n_mesh, r_cut, G))
    return interpolate(pos, gradient(phi))


def tsc_weight_derivatives(d):
    """d/dd of tsc_weights (offsets -1, 0, +1); they sum to zero."""
    d = np.asarray(d, dtype=np.float64)
    return np.stack([-(0.5 - d), -2.0 * d, 0.5 + d])


def divergence(field):
    """Sum over axes of the four-point difference of field[a] along axis a
    (the transpose of gradient() up to sign)."""
    n_mesh = field[0].shape[0]
    h = 1.0 / n_mesh
    out = np.zeros_like(field[0])
    for a in range(3):
        f = field[a]
        out += (8.0 * (np.roll(f, -1, a) - np.roll(f, 1, a))
                - (np.roll(f, -2, a) - np.roll(f, 2, a))) / (12.0 * h)
    return out


def pm_vjp(pos, mass, n_mesh, r_cut, G, w):
    """dL/dx of L = sum_i w_i . a_i over the PM cycle (the adjoint of
    pm_forces).  With U_a = the TSC assignment of the cotangent component
    w_a, A = -grad(phi) the mesh force and B = K div(U), K the potential
    solve of step 2 (symmetric) and div the four-point divergence
    (the four-point difference is antisymmetric):
        dL/dx_k = sum_c grad W_k(c) [w_k . A(c) + (m_k / h^3) B(c)],
    grad W_k the derivative of particle k's TSC weight at mesh point c."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    h3 = (1.0 / n_mesh) ** 3
    gk = green(n_mesh, r_cut, G)
    amesh = gradient(potential(assign(pos, mass, n_mesh), gk))
    # U: each cotangent component assigned like a mass (assign() divides by h^3)
    umesh = [assign(pos, w[:, a], n_mesh) * h3 for a in range(3)]
    bmesh = potential(divergence(umesh), gk)
    u = (pos % 1.0) * n_mesh
    i0 = np.rint(u).astype(np.int64)
    d = u - i0
    W = [tsc_weights(d[:, a]) for a in range(3)]
    dW = [tsc_weight_derivatives(d[:, a]) * n_mesh for a in range(3)]
    grad = np.zeros_like(pos)
    for a in range(3):
        for b in range(3):
            for c in range(3):
                idx = ((i0[:, 0] + a - 1) % n_mesh, (i0[:, 1] + b - 1) % n_mesh,
                       (i0[:, 2] + c - 1) % n_mesh)
                s = (w[:, 0] * amesh[0][idx] + w[:, 1] * amesh[1][idx] + w[:, 2] * amesh[2][idx]
                     + mass / h3 * bmesh[idx])
                grad[:, 0] += dW[0][a] * W[1][b] * W[2][c] * s
                grad[:, 1] += W[0][a] * dW[1][b] * W[2][c] * s
                grad[:, 2] += W[0][a] * W[1][b] * dW[2][c] * s
    return grad


# ---------------------------------------------------------------------------
# TreePM time integration with multiple step sizes (the paper's Sec. III-A
# schedule: one PM cycle and two PP cycles per step).  The slow PM force
# kicks at the step's ends; the short-range force is integrated with two
# kick-drift-kick sub-steps of dt/2 in between:
#     v += a_PM(x) dt/2
#     twice:  v += a_PP dt/4;  x += v dt/2;  a_PP = PP(x);  v += a_PP dt/4
#     a_PM = PM(x);  v += a_PM dt/2
# ---------------------------------------------------------------------------
def treepm_leapfrog(pos0, vel0, mass, G, eps, r_cut, theta, n_mesh, dt, steps, n_leaf=8, n_crit=64,
                    refit=False):
    """Integrate `steps` TreePM steps; returns (x_T, v_T, a_PP(x_T),
    a_PM(x_T), evals) with evals = [(tree, x)] for every PP evaluation in
    order (the initial one and two per step).  With refit the second PP
    sub-step of each step keeps the first sub-step's tree structure and only
    re-takes its monopoles from the new positions (OracleTree.refresh)."""
    from . import OracleTree
    mass = np.asarray(mass, dtype=np.float64)
    x = np.asarray(pos0, dtype=np.float64).copy()
    v = np.asarray(vel0, dtype=np.float64).copy()

    def build(xx):
        t = OracleTree(xx, mass, n_leaf, n_crit)
        t.lists(r_cut, theta)
        return t

    t = build(x)
    a_pp = t.list_forces(G, eps, r_cut)
    evals = [(t, x.copy())]
    a_pm = pm_forces(x, mass, n_mesh, r_cut, G)
    h = 0.5 * dt
    for _ in range(steps):
        v = v + a_pm * (0.5 * dt)
        for sub in range(2):
            v = v + a_pp * (0.5 * h)
            x = x + v * h
            if sub == 1 and refit:
                t.refresh(x)
            else:
                t = build(x)
            a_pp = t.list_forces(G, eps, r_cut)
            evals.append((t, x.copy()))
            v = v + a_pp * (0.5 * h)
        a_pm = pm_forces(x, mass, n_mesh, r_cut, G)
        v = v + a_pm * (0.5 * dt)
    return x, v, a_pp, a_pm, evals


def treepm_leapfrog_frozen(pos0, vel0, mass, evals, G, eps, r_cut, n_mesh, dt, steps):
    """treepm_leapfrog with every PP evaluation's tree structure frozen to
    `evals` (monopoles re-taken from the current positions): the function
    whose derivative treepm_leapfrog_adjoint computes.  Returns (x_T, v_T,
    a_PP, a_PM, xs) with xs the positions of every PP evaluation."""
    mass = np.asarray(mass, dtype=np.float64)
    x = np.asarray(pos0, dtype=np.float64).copy()
    v = np.asarray(vel0, dtype=np.float64).copy()

    def pp(k, xx):
        t = evals[k][0]
        t.refresh(xx)
        return t.list_forces(G, eps, r_cut)

    xs = [x.copy()]
    a_pp = pp(0, x)
    a_pm = pm_forces(x, mass, n_mesh, r_cut, G)
    h = 0.5 * dt
    k = 1
    for _ in range(steps):
        v = v + a_pm * (0.5 * dt)
        for _sub in range(2):
            v = v + a_pp * (0.5 * h)
            x = x + v * h
            xs.append(x.copy())
            a_pp = pp(k, x)
            k += 1
            v = v + a_pp * (0.5 * h)
        a_pm = pm_forces(x, mass, n_mesh, r_cut, G)
        v = v + a_pm * (0.5 * dt)
    return x, v, a_pp, a_pm, xs


def treepm_leapfrog_adjoint(pos0, vel0, mass, evals, G, eps, r_cut, n_mesh, dt, steps,
                            g_x, g_v, g_app, g_apm):
    """Reverse-mode derivative of treepm_leapfrog_frozen: given dL/dx_T,
    dL/dv_T, dL/da_PP(x_T) and dL/da_PM(x_T), returns (dL/dx_0, dL/dv_0).
    Each operation of the step is reversed in turn; a force a = F(x) sends
    its cotangent g_a to g_x += VJP_F(x)[g_a] (the list adjoint of the frozen
    tree for PP, pm_vjp for PM)."""
    mass = np.asarray(mass, dtype=np.float64)
    *_, xs = treepm_leapfrog_frozen(pos0, vel0, mass, evals, G, eps, r_cut, n_mesh, dt, steps)

    def pp_vjp(k, ga):
        t = evals[k][0]
        t.refresh(xs[k])
        return t.list_vjp(G, eps, r_cut, ga)

    h = 0.5 * dt
    gx, gv = np.asarray(g_x, dtype=np.float64).copy(), np.asarray(g_v, dtype=np.float64).copy()
    g_pp, g_pm = np.asarray(g_app, dtype=np.float64).copy(), np.asarray(g_apm, dtype=np.float64).copy()
    for s in range(steps, 0, -1):
        x_end = xs[2 * s]
        # v += a_PM(x_end) dt/2 ;  a_PM = PM(x_end)
        g_pm = g_pm + gv * (0.5 * dt)
        gx = gx + pm_vjp(x_end, mass, n_mesh, r_cut, G, g_pm)
        g_pm = np.zeros_like(g_pm)
        for k in (2 * s, 2 * s - 1):
            # v += a_PP dt/4 ; a_PP = PP(x_k)
            g_pp = g_pp + gv * (0.5 * h)
            gx = gx + pp_vjp(k, g_pp)
            # x += v h
            gv = gv + gx * h
            # v += a_PP(previous) dt/4
            g_pp = gv * (0.5 * h)
        # v += a_PM(x_start) dt/2
        g_pm = gv * (0.5 * dt)
    gx = gx + pp_vjp(0, g_pp) + pm_vjp(xs[0], mass, n_mesh, r_cut, G, g_pm)
    return gx, gv
