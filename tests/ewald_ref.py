"""Periodic Ewald summation of point masses in the unit box: a textbook
reference for the tests of the long-range half (not part of the method)."""
import numpy as np
from scipy.special import erfc


def ewald(pos, mass, G, alpha=5.0, n_real=3, k_max=12):
    """Periodic Newtonian accelerations in the unit box, mean density removed."""
    n = pos.shape[0]
    r1 = np.arange(-n_real, n_real + 1)
    shifts = np.array(np.meshgrid(r1, r1, r1, indexing="ij")).reshape(3, -1).T.astype(float)
    k1 = np.arange(-k_max, k_max + 1)
    kv = np.array(np.meshgrid(k1, k1, k1, indexing="ij")).reshape(3, -1).T.astype(float)
    kv = kv[np.any(kv != 0, axis=1)] * (2 * np.pi)
    k2 = np.sum(kv * kv, axis=1)
    kfac = 4 * np.pi * np.exp(-k2 / (4 * alpha ** 2)) / k2
    acc = np.zeros((n, 3))
    for i in range(n):
        d = pos - pos[i]
        for j in range(n):
            dd = d[j] + shifts
            r = np.linalg.norm(dd, axis=1)
            keep = r > 0
            dd, r = dd[keep], r[keep]
            f = (erfc(alpha * r) + 2 * alpha * r / np.sqrt(np.pi) * np.exp(-(alpha * r) ** 2)) / r ** 3
            acc[i] += G * mass[j] * (f[:, None] * dd).sum(0)
            acc[i] += G * mass[j] * ((kfac * np.sin(kv @ d[j]))[:, None] * kv).sum(0)
    return acc
