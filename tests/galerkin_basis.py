"""Independent check of the oracle: dense Galerkin solves in a real trigonometric basis.

The conforming space E_N of zero-mean curl-free trigonometric polynomials (Section 2.2) is
spanned by the gradients of cos(2 pi k.x) and sin(2 pi k.x) for the non-zero k in Z_N, one k of
each pair +-k. Sampling those gradients (closed-form derivatives) at the nodes of a grid gives a
basis of I_N[E_N] (or, on a double grid M, of I_M[E_N]) without any DFT or projection, so the
minimisers of eqs. (Ga)/(GaNi) follow from one dense linear solve.
"""
import numpy as np

from microstructure import node_coords, signed_index


def half_frequencies(N):
    ks = np.stack(np.meshgrid(*[signed_index(n) for n in N], indexing="ij"), -1).reshape(-1, len(N))
    keep = []
    for k in ks:
        nz = np.nonzero(k)[0]
        if len(nz) and k[nz[0]] > 0:
            keep.append(k)
    return np.array(keep)


def basis(N, grid):
    """Columns: gradients of cos/sin(2 pi k.x), k in half of Z_N \\ {0}, sampled on `grid`."""
    d = len(N)
    xs = node_coords(grid)
    cols = []
    for k in half_frequencies(N):
        phase = sum(2 * np.pi * k[a] * xs[a] for a in range(d))
        phase = np.broadcast_to(phase, tuple(grid))
        s, c = np.sin(phase), np.cos(phase)
        cols.append(np.stack([-2 * np.pi * k[a] * s for a in range(d)]).ravel())
        cols.append(np.stack([2 * np.pi * k[a] * c for a in range(d)]).ravel())
    return np.array(cols).T


def apply_coeff(A, v, d):
    if A.ndim == d:
        return A[None] * v
    return np.einsum("ab...,b...->a...", A, v)


def dense_minimiser(A, E, N, grid):
    """min_c (A(E + B c), E + B c) on `grid` (nodal mean); returns (e field, energy)."""
    d = len(N)
    B = basis(N, grid)
    shp = (d,) + tuple(grid)
    Ef = np.broadcast_to(np.asarray(E, float).reshape((d,) + (1,) * d), shp)
    AB = np.stack([apply_coeff(A, B[:, j].reshape(shp), d).ravel() for j in range(B.shape[1])], 1)
    K = B.T @ AB
    f = -B.T @ apply_coeff(A, Ef, d).ravel()
    c = np.linalg.solve(K, f)
    e = (B @ c).reshape(shp)
    v = Ef + e
    en = float(np.mean(np.sum(apply_coeff(A, v, d) * v, axis=0)))
    return e, en, c
