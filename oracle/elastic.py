"""Plain FP64 NumPy oracle of the linear-elasticity form of the method (test infrastructure only).

Section 1 (Limitations) names "more involved applications" as the next step for the
Fourier-Galerkin solvers; linear elasticity is the standard one. The homogenized stiffness is
defined as in Section 2 with vectors replaced by symmetric strain tensors:

    (C_H E) : E = min over compatible e of  mean over Y of (E + e) : C(x) : (E + e),

"compatible" meaning e = sym(grad u) for a Y-periodic displacement u, the analogue of the
curl-free fields of eq. (homog_form). Everything of Sections 2-3 carries over with
  * fields with nc = d (d + 1) / 2 components (symmetric d x d tensors),
  * the projection Gamma^(k) onto compatible strains replacing eq. (proj),
  * the stiffness C(x), SPD on symmetric tensors, replacing A(x) (bounds c_A, C_A of eq. (A)
    are its extreme eigenvalues),
and Algorithms 1-4 unchanged (they only use matvecs, inner products and c_A, C_A).

Storage (Mandel notation, so that the Frobenius product e : t of symmetric tensors is the
Euclidean product of the stored vectors): component order
    d = 2: (e_11, e_22, sqrt2 e_12)
    d = 3: (e_11, e_22, e_33, sqrt2 e_23, sqrt2 e_13, sqrt2 e_12),
a strain field is an array (nc, N_1, ..., N_d), a stiffness field an array (nc, nc, N...) of
symmetric Mandel matrices, grids and frequencies as in hom.py (FFT-natural order).

Projection: for k != 0 the compatible strains at frequency k are the tensors sym(k (x) u),
u in C^d. The orthogonal projection (Frobenius product) of a symmetric e onto them follows
from the normal equations (e - sym(k (x) u)) k = 0, i.e. u |k|^2 + k (k.u) = 2 e k, so
k.u = (k.e.k)/|k|^2 and
    Gamma^(k) e = (k (x) q + q (x) k) / |k|^2 - (k.e.k) k (x) k / |k|^4,   q = e k,
and Gamma^(0) = 0 (the mean strain is E, eq. (proj) analogue).
"""
from __future__ import annotations

import math

import numpy as np

from .hom import dft, energy, frequencies, idft, apply_A

__all__ = ["mandel_pairs", "to_tensor", "to_mandel", "gamma_sym_apply", "project_strain",
           "isotropic_stiffness", "expand_stiffness", "GaNiElastic", "ncomp"]

SQ2 = math.sqrt(2.0)


def ncomp(d: int) -> int:
    """Components of a symmetric d x d tensor."""
    return d * (d + 1) // 2


def mandel_pairs(d: int) -> list[tuple[int, int]]:
    """Tensor index (i, j) of every Mandel component, in storage order."""
    if d == 2:
        return [(0, 0), (1, 1), (0, 1)]
    if d == 3:
        return [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    raise ValueError("d must be 2 or 3")


def to_tensor(v: np.ndarray, d: int) -> np.ndarray:
    """Mandel vector field (nc, ...) -> symmetric tensor field (d, d, ...)."""
    t = np.zeros((d, d) + v.shape[1:], dtype=v.dtype)
    for m, (i, j) in enumerate(mandel_pairs(d)):
        if i == j:
            t[i, i] = v[m]
        else:
            t[i, j] = v[m] / SQ2
            t[j, i] = v[m] / SQ2
    return t


def to_mandel(t: np.ndarray, d: int) -> np.ndarray:
    """Symmetric tensor field (d, d, ...) -> Mandel vector field (nc, ...)."""
    out = []
    for i, j in mandel_pairs(d):
        out.append(t[i, i] if i == j else SQ2 * t[i, j])
    return np.stack(out)


def gamma_sym_apply(vh: np.ndarray, d: int) -> np.ndarray:
    """Gamma^(k) of the module docstring applied to the Fourier coefficients vh (nc, grid) of a
    Mandel strain field; zero at k = 0."""
    grid = vh.shape[1:]
    ks = frequencies(grid)
    kk = sum(k * k for k in ks)
    safe = np.where(kk > 0, kk, 1.0)
    e = to_tensor(vh, d)
    q = [sum(e[i, j] * ks[j] for j in range(d)) for i in range(d)]      # q = e k
    kek = sum(ks[i] * q[i] for i in range(d))                              # k . e . k
    out = np.zeros_like(e)
    for i in range(d):
        for j in range(d):
            out[i, j] = (ks[i] * q[j] + q[i] * ks[j]) / safe - kek * ks[i] * ks[j] / (safe * safe)
    out = np.where(kk > 0, out, 0.0)
    return to_mandel(out, d)


def project_strain(v: np.ndarray, d: int) -> np.ndarray:
    """G v = F^{-1} Gamma^ F v on the grid of v (the strain form of eq. (discrete_proj))."""
    return idft(gamma_sym_apply(dft(v, d), d), d).real


def isotropic_stiffness(lam: float, mu: float, d: int) -> np.ndarray:
    """Mandel matrix of C e = lam tr(e) I + 2 mu e."""
    nc = ncomp(d)
    C = np.zeros((nc, nc))
    for a in range(d):
        for b in range(d):
            C[a, b] = lam + (2.0 * mu if a == b else 0.0)
    for m in range(d, nc):
        C[m, m] = 2.0 * mu
    return C


def expand_stiffness(phase: np.ndarray, table: np.ndarray) -> np.ndarray:
    """Stiffness field (nc, nc, N...) from a phase image and a (nphase, nc, nc) table."""
    t = np.asarray(table, dtype=np.float64)
    a = t[np.asarray(phase, dtype=np.int64)]
    return np.moveaxis(np.moveaxis(a, -1, 0), -1, 0)


class GaNiElastic:
    """GaNi system of the strain problem: C x = G C~_N x, b = -G C~_N E (eq. (GaNi_ls) with the
    stiffness sampled at the nodes and the strain projection)."""

    def __init__(self, C: np.ndarray, d: int):
        self.A = C
        self.d = d
        self.nc = ncomp(d)

    @property
    def grid(self):
        return self.A.shape[-self.d:]

    def matvec(self, x):
        return project_strain(apply_A(self.A, x), self.d)

    def rhs(self, E):
        return -self.matvec(self.const(E))

    def const(self, E):
        E = np.asarray(E, dtype=np.float64).reshape((self.nc,) + (1,) * self.d)
        return np.broadcast_to(E, (self.nc,) + tuple(self.grid)).copy()

    def energy(self, E, x):
        """(C(E + x), E + x) with the 1/|N|-weighted inner product."""
        return energy(self.A, self.const(E) + x)

    def em_project(self, v):
        """F^{-1}(I - 2 Gamma^)F v (Algorithm 4 with the strain projection)."""
        vh = dft(v, self.d)
        return idft(vh - 2.0 * gamma_sym_apply(vh, self.d), self.d).real
