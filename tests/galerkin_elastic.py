"""Independent check of the elasticity oracle: dense Galerkin solves in a displacement basis.

The compatible strains of trigonometric order N are the symmetric gradients of Y-periodic
trigonometric displacements u = e_i cos(2 pi k.x), e_i sin(2 pi k.x) for the non-zero k in Z_N
(one k of each pair +-k) and i = 1..d. Their strains sym(e_i (x) grad phi) have closed-form
derivatives; sampled at the nodes (Mandel components) they span the conforming space of the
GaNi strain problem without any DFT or projection, so its minimiser is one dense linear solve.
"""
import math

import numpy as np

from tests.galerkin_basis import half_frequencies
from microstructure import node_coords

SQ2 = math.sqrt(2.0)


def pairs(d):
    return [(0, 0), (1, 1), (0, 1)] if d == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def strain_basis(N):
    """Columns: Mandel strains of the displacement basis, sampled at the nodes of N."""
    d = len(N)
    xs = node_coords(N)
    cols = []
    for k in half_frequencies(N):
        phase = np.broadcast_to(sum(2 * np.pi * k[a] * xs[a] for a in range(d)), tuple(N))
        s, c = np.sin(phase), np.cos(phase)
        for grad_scalar in (-s, c):          # d/dx_a of cos = -2 pi k_a sin, of sin = 2 pi k_a cos
            g = [2 * np.pi * k[a] * grad_scalar for a in range(d)]
            for i in range(d):               # displacement direction e_i
                comps = []
                for a, b in pairs(d):
                    # sym(e_i (x) g)_ab = (delta_ia g_b + delta_ib g_a) / 2
                    t = 0.5 * ((g[b] if i == a else 0.0) + (g[a] if i == b else 0.0))
                    t = np.broadcast_to(t, tuple(N))
                    comps.append(t if a == b else SQ2 * t)
                cols.append(np.stack(comps).ravel())
    return np.array(cols).T


def apply_stiffness(C, v):
    return np.einsum("ab...,b...->a...", C, v)


def dense_minimiser(C, E, N):
    """min over the displacement basis of the nodal mean of (E + e) : C : (E + e); returns
    (e field in Mandel form, energy)."""
    d = len(N)
    nc = d * (d + 1) // 2
    B = strain_basis(N)
    shp = (nc,) + tuple(N)
    Ef = np.broadcast_to(np.asarray(E, float).reshape((nc,) + (1,) * d), shp)
    CB = np.stack([apply_stiffness(C, B[:, j].reshape(shp)).ravel() for j in range(B.shape[1])], 1)
    K = B.T @ CB
    f = -B.T @ apply_stiffness(C, Ef).ravel()
    c = np.linalg.lstsq(K, f, rcond=None)[0]
    e = (B @ c).reshape(shp)
    v = Ef + e
    return e, float(np.mean(np.sum(apply_stiffness(C, v) * v, axis=0)))
