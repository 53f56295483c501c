"""Plain FP64 NumPy oracle of the method (test infrastructure only; see the package docstring).

Array conventions: a vector field on a grid of order N is an array of shape (d, N_1, ..., N_d)
in FFT-natural order along every axis (index j holds the signed index j or j - N_a); component
a pairs with spatial axis a. A coefficient field is either a scalar array (N_1, ..., N_d)
(isotropic) or a tensor array (d, d, N_1, ..., N_d).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "signed_index", "dft_matrix", "dft", "idft", "frequencies", "gamma_apply", "project",
    "apply_A", "expand_phase", "GaNi", "Ga", "prolongate", "energy", "richardson", "cg",
    "chebyshev", "eyre_milton", "SolveResult", "spectral_bounds", "double_grid",
    "ga_coefficients", "voxel_fourier_coefficients", "restrict",
]


# ----------------------------------------------------------------------------------------
# Section 2.1: index sets, the DFT and its inverse
# ----------------------------------------------------------------------------------------

def signed_index(n: int) -> np.ndarray:
    """Signed index of every storage position: Z_N = {k : |k| < N/2} for odd N (eq. (grid))."""
    if n <= 0 or n % 2 == 0:
        raise ValueError(f"N must be odd, got {n}")
    j = np.arange(n)
    return np.where(j <= (n - 1) // 2, j, j - n)


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """One-axis factor of eq. (DFT): F_N = (1/N) (omega^{-mk}), F_N^{-1} = (omega^{mk}),
    omega^{mk} = exp(2 pi i m k / N), with m, k in Z_N (storage order of signed_index).
    The angle is reduced exactly (m k mod N) before the trigonometric evaluation."""
    m = signed_index(n)
    mk = np.mod(np.outer(m, m), n).astype(np.float64)
    ang = 2.0 * np.pi * mk / n
    w = np.cos(ang) + 1j * np.sin(ang)
    if inverse:
        return w
    return np.conj(w) / n


def _apply_axis(mat: np.ndarray, v: np.ndarray, axis: int) -> np.ndarray:
    return np.moveaxis(np.tensordot(mat, v, axes=([1], [axis])), 0, axis)


def dft(v: np.ndarray, nspatial: int) -> np.ndarray:
    """F_N applied to the trailing `nspatial` axes of v (eq. (DFT), with the 1/|N| factor)."""
    out = v.astype(np.complex128)
    for ax in range(v.ndim - nspatial, v.ndim):
        out = _apply_axis(dft_matrix(v.shape[ax]), out, ax)
    return out


def idft(vh: np.ndarray, nspatial: int) -> np.ndarray:
    """F_N^{-1} applied to the trailing `nspatial` axes (eq. (DFT), no scaling)."""
    out = vh.astype(np.complex128)
    for ax in range(vh.ndim - nspatial, vh.ndim):
        out = _apply_axis(dft_matrix(vh.shape[ax], inverse=True), out, ax)
    return out


def frequencies(shape) -> list[np.ndarray]:
    """Broadcastable signed integer frequencies k_a on a grid of the given shape."""
    d = len(shape)
    ks = []
    for a, n in enumerate(shape):
        s = [1] * d
        s[a] = n
        ks.append(signed_index(n).reshape(s).astype(np.float64))
    return ks


# ----------------------------------------------------------------------------------------
# Section 2, eq. (proj) and Section 2.3, eq. (discrete_proj): the projection
# ----------------------------------------------------------------------------------------

def gamma_apply(vh: np.ndarray, support=None) -> np.ndarray:
    """Block-diagonal Fourier projection: Gamma^(k) v^(k) = k (k . v^(k)) / (k . k), zero at
    k = 0 (eq. (proj)); with `support` = N on a grid M, additionally zero for k outside Z_N
    (eq. (discrete_proj))."""
    d = vh.shape[0]
    grid = vh.shape[1:]
    ks = frequencies(grid)
    kk = sum(k * k for k in ks)
    kv = sum(ks[a] * vh[a] for a in range(d))
    safe = np.where(kk > 0, kk, 1.0)
    coef = np.where(kk > 0, kv / safe, 0.0)
    if support is not None:
        inside = np.ones(grid, dtype=bool)
        for a in range(d):
            inside = inside & (np.abs(ks[a]) < support[a] / 2.0)
        coef = np.where(inside, coef, 0.0)
    return np.stack([ks[a] * coef for a in range(d)])


def project(v: np.ndarray, support=None) -> np.ndarray:
    """G_{N,M} v = F_M^{-1} G^_{N,M} F_M v (eq. (discrete_proj)); G_N when support is None."""
    d = v.shape[0]
    return idft(gamma_apply(dft(v, d), support), d).real


# ----------------------------------------------------------------------------------------
# Coefficients: eq. (A), the sampled matrix of GaNi (Section 2.2), eq. (Ga_exact_integration)
# ----------------------------------------------------------------------------------------

def expand_phase(phase: np.ndarray, table: np.ndarray) -> np.ndarray:
    """Coefficient tensor field A(x^k) from a phase image and a (nphase, d, d) table."""
    t = np.asarray(table, dtype=np.float64)
    a = t[np.asarray(phase, dtype=np.int64)]          # (N..., d, d)
    return np.moveaxis(np.moveaxis(a, -1, 0), -1, 0)   # (d, d, N...)


def apply_A(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Block-diagonal coefficient product (A v)^k = A^k v^k; A scalar or (d, d, N...)."""
    d = v.shape[0]
    if A.ndim == v.ndim - 1:
        return A[None] * v
    return np.stack([sum(A[a, b] * v[b] for b in range(d)) for a in range(d)])


def double_grid(N) -> tuple:
    """Double grid 2N - 1 of exact integration (Section 2.2, eq. (Ga_eval))."""
    return tuple(2 * int(n) - 1 for n in N)


def ga_coefficients(Ahat: np.ndarray, nspatial: int) -> np.ndarray:
    """A_M^k = sum_{n in Z_M} omega_M^{kn} A^(n) (eq. (Ga_exact_integration)) from the Fourier
    coefficients A^(n) given on Z_M; scalar (M...) or tensor (d, d, M...). Real part kept (the
    coefficients of a real field are Hermitian)."""
    return idft(Ahat, nspatial).real


def voxel_fourier_coefficients(a: np.ndarray, M) -> np.ndarray:
    """Fourier coefficients A^(n), n in Z_M (FFT-natural order), of the voxel-wise constant
    scalar coefficient that takes the value a[k] on the cell of side 1/N_a centred at the node
    x = k/N (the pixel/voxel images for which Section 2.2 assembles eq. (Ga_exact_integration)
    by FFT). Integrating exp(-2 pi i n.x) (eq. (FT_def)) over one cell gives
    prod_a sinc(pi n_a / N_a) exp(-2 pi i n.k/N) / |N|, so
    A^(n) = prod_a sinc(pi n_a / N_a) (F_N a)(n mod N), with F_N the DFT of eq. (DFT) and
    sinc(t) = sin(t)/t. Parity pinned by brute-force quadrature and by the analytic box
    coefficients of an inclusion made of whole voxels (tests/test_oracle_transforms.py)."""
    N = a.shape
    d = len(N)
    ah = dft(np.asarray(a, dtype=np.float64), d)
    pos, sinc = [], []
    for ax in range(d):
        n = signed_index(int(M[ax]))
        if M[ax] < N[ax]:
            raise ValueError("the coefficient grid must contain Z_N")
        pos.append(np.mod(n, N[ax]))                    # storage position of n mod N
        s = [1] * d
        s[ax] = int(M[ax])
        sinc.append(np.sinc(n / N[ax]).reshape(s))       # numpy sinc(u) = sin(pi u)/(pi u)
    out = ah[np.ix_(*pos)]
    for f in sinc:
        out = out * f
    return out


def spectral_bounds(A: np.ndarray, d: int) -> tuple[float, float]:
    """c_A, C_A of eq. (A): extreme eigenvalues of the coefficient over the grid (A scalar
    field with d spatial axes, or a (d, d, N...) tensor field)."""
    if A.ndim == d:
        return float(A.min()), float(A.max())
    nc = A.shape[0]  # d, or d (d + 1) / 2 for a stiffness in Mandel form (oracle/elastic.py)
    mats = np.moveaxis(np.moveaxis(A, 0, -1), 0, -1).reshape(-1, nc, nc)
    ev = np.linalg.eigvalsh(mats)
    return float(ev.min()), float(ev.max())


# ----------------------------------------------------------------------------------------
# Section 2.3, eq. (linsys): the two linear systems C x = b
# ----------------------------------------------------------------------------------------

@dataclass
class GaNi:
    """GaNi system: C = G_N A~_N, b = -G_N A~_N E (eq. (GaNi_ls)); A sampled at the nodes."""
    A: np.ndarray
    d: int

    @property
    def grid(self):
        return self.A.shape[-self.d:]

    def matvec(self, x):
        return project(apply_A(self.A, x))

    def rhs(self, E):
        return -self.matvec(self.const(E))

    def const(self, E):
        return np.broadcast_to(np.asarray(E, dtype=np.float64).reshape((self.d,) + (1,) * self.d),
                               (self.d,) + tuple(self.grid)).copy()

    def energy(self, E, x):
        """(A(E + x), E + x) with the weighted inner product (eq. (GaNi), Section 2.2)."""
        return energy(self.A, self.const(E) + x)

    def em_project(self, v):
        """F^{-1}(I - 2 G^)F v (Algorithm 4)."""
        d = self.d
        vh = dft(v, d)
        return idft(vh - 2.0 * gamma_apply(vh), d).real


@dataclass
class Ga:
    """Ga system on the double grid M: C = G_{N,M} A_M, b = -G_{N,M} A_M E (eq. (Ga_ls))."""
    A_M: np.ndarray
    N: tuple
    d: int

    @property
    def grid(self):
        return self.A_M.shape[-self.d:]

    def matvec(self, x):
        return project(apply_A(self.A_M, x), support=self.N)

    def rhs(self, E):
        return -self.matvec(self.const(E))

    def const(self, E):
        return np.broadcast_to(np.asarray(E, dtype=np.float64).reshape((self.d,) + (1,) * self.d),
                               (self.d,) + tuple(self.grid)).copy()

    def energy(self, E, x):
        """Eq. (ev_bounds_Ga): (A_M(E + x), E + x) on the double grid."""
        return energy(self.A_M, self.const(E) + x)


def energy(A: np.ndarray, v: np.ndarray) -> float:
    """Weighted inner product (A v, v) = (1/|N|) sum_k (A^k v^k, v^k) (Notation section)."""
    return float(np.mean(np.sum(apply_A(A, v) * v, axis=0)))


def prolongate(v: np.ndarray, M) -> np.ndarray:
    """R_{N,M} = I_M o I_N^{-1} (eq. (ev_bounds)): the trigonometric polynomial with nodal values
    v on grid N, sampled on grid M: F_N, place coefficients of Z_N into Z_M, F_M^{-1}."""
    d = v.shape[0]
    N = v.shape[1:]
    vh = dft(v, d)
    out = np.zeros((d,) + tuple(M), dtype=np.complex128)
    idx = []
    for a in range(d):
        idx.append(np.mod(signed_index(N[a]), M[a]))
    out[(slice(None),) + np.ix_(*idx)] = vh
    return idft(out, d).real


def restrict(v: np.ndarray, N) -> np.ndarray:
    """Samples on the grid N of the trigonometric polynomial of order N given by its nodal values
    v on a grid M >= N (every Ga iterate is one, Section 2.3): F_M, the coefficients of Z_N
    (eq. (DFT); a polynomial of order N has no others), F_N^{-1}. The inverse of prolongate on
    such fields."""
    d = v.shape[0]
    M = v.shape[1:]
    vh = dft(v, d)
    idx = [np.mod(signed_index(int(N[a])), M[a]) for a in range(d)]
    return idft(vh[(slice(None),) + np.ix_(*idx)], d).real


# ----------------------------------------------------------------------------------------
# Section 3: Algorithms 1-4
# ----------------------------------------------------------------------------------------

def _norm(v):
    """||v||_2 with the 1/|N| weight (Notation section)."""
    return math.sqrt(float(np.mean(np.sum(v * v, axis=0))))


def _dot(u, v):
    return float(np.mean(np.sum(u * v, axis=0)))


@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    converged: bool
    history: list = field(default_factory=list)   # per-iteration stopping quantity
    iterates: list = field(default_factory=list)  # optional copies of x_m


def richardson(sys, E, cA, CA, tol=1e-6, maxit=100000, stop="increment", fixed_iters=None,
               omega=None, keep_iterates=False) -> SolveResult:
    """Algorithm 1: x_m = x_{m-1} - omega (C x_{m-1} - b), x_0 = 0, omega = 2/(c_A + C_A).

    stop="increment": ||x_m - x_{m-1}|| <= eps ||E|| (as printed); stop="residual":
    ||C x_m - b|| <= eps ||b||, tested on the residual formed at the start of the next step.
    fixed_iters runs exactly that many updates with no stopping test."""
    if omega is None:
        omega = 2.0 / (cA + CA)
    b = sys.rhs(E)
    x = np.zeros_like(b)
    nE = float(np.linalg.norm(E))
    nb = _norm(b)
    hist, its = [], []
    nmax = fixed_iters if fixed_iters is not None else maxit
    for m in range(1, nmax + 1):
        r = sys.matvec(x) - b
        if fixed_iters is None and stop == "residual":
            rn = _norm(r)
            hist.append(rn)
            if rn <= tol * nb:
                return SolveResult(x, m - 1, True, hist, its)
        x_new = x - omega * r
        dx = _norm(x_new - x)
        x = x_new
        if keep_iterates:
            its.append(x.copy())
        if fixed_iters is None and stop == "increment":
            hist.append(dx)
            if dx <= tol * nE:
                return SolveResult(x, m, True, hist, its)
    return SolveResult(x, nmax, fixed_iters is not None, hist, its)


def cg(sys, E, tol=1e-6, maxit=100000, fixed_iters=None, keep_iterates=False) -> SolveResult:
    """Algorithm 2 (conjugate gradients), x_0 = 0, stop on ||r_m|| <= eps ||b||."""
    b = sys.rhs(E)
    x = np.zeros_like(b)
    r = b - sys.matvec(x)
    p = r.copy()
    rr = _dot(r, r)
    nb = _norm(b)
    hist, its = [], []
    nmax = fixed_iters if fixed_iters is not None else maxit
    for m in range(1, nmax + 1):
        Cp = sys.matvec(p)
        alpha = rr / _dot(Cp, p)
        x = x + alpha * p
        r = r - alpha * Cp
        rr_new = _dot(r, r)
        if keep_iterates:
            its.append(x.copy())
        hist.append(math.sqrt(rr_new))
        if fixed_iters is None and math.sqrt(rr_new) <= tol * nb:
            return SolveResult(x, m, True, hist, its)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
    return SolveResult(x, nmax, fixed_iters is not None, hist, its)


def chebyshev(sys, E, cA, CA, tol=1e-6, maxit=100000, fixed_iters=None,
              keep_iterates=False) -> SolveResult:
    """Algorithm 3 (Chebyshev semi-iteration, two-term recurrence), taken literally:
    c = (C_A - c_A)/2, d = (c_A + C_A)/2, alpha = 1/d, beta = -(c/d)^2 / 2; for m > 1
    alpha = 1/(d + beta/alpha), beta = -(c alpha / 2)^2; r -= alpha C p; x += alpha p;
    p = r - beta p; stop on ||r_m|| <= eps ||b||."""
    b = sys.rhs(E)
    x = np.zeros_like(b)
    r = b - sys.matvec(x)
    c = 0.5 * (CA - cA)
    dd = 0.5 * (cA + CA)
    alpha = 1.0 / dd
    beta = -0.5 * (c / dd) ** 2
    p = r.copy()
    nb = _norm(b)
    hist, its = [], []
    nmax = fixed_iters if fixed_iters is not None else maxit
    for m in range(1, nmax + 1):
        if m > 1:
            alpha = 1.0 / (dd + beta / alpha)
            beta = -((c * alpha / 2.0) ** 2)
        r = r - alpha * sys.matvec(p)
        x = x + alpha * p
        p = r - beta * p
        rn = _norm(r)
        hist.append(rn)
        if keep_iterates:
            its.append(x.copy())
        if fixed_iters is None and rn <= tol * nb:
            return SolveResult(x, m, True, hist, its)
    return SolveResult(x, nmax, fixed_iters is not None, hist, its)


def eyre_milton(sys: GaNi, E, cA, CA, tol=1e-6, maxit=100000, fixed_iters=None,
                literal_sign=False, keep_iterates=False) -> SolveResult:
    """Algorithm 4 (Eyre-Milton), GaNi only: x_0 = E, omega = sqrt(c_A C_A),
    x_m = (A + omega)^{-1} F^{-1}(I - 2 G^)F (A - omega) x_{m-1} + q,
    stop on ||x_m - x_{m-1}|| <= eps ||E||.

    As printed, q = -2 omega (A + omega)^{-1} x_0, whose fixed point is -(E + e~) (multiply the
    fixed-point equation by (A + omega) and apply G). The default reading takes
    q = +2 omega (A + omega)^{-1} E, whose fixed point is E + e~; literal_sign=True keeps the
    printed sign. The returned x approximates E + e~ (not e~)."""
    if not (isinstance(sys, GaNi) or hasattr(sys, "nc")):
        raise ValueError("Eyre-Milton is defined for the GaNi system only (Section 3.4)")
    omega = math.sqrt(cA * CA)
    d = sys.d
    nc = getattr(sys, "nc", d)  # components: d, or d (d + 1) / 2 for strains
    A = sys.A
    Econst = sys.const(E)
    if A.ndim == d:
        inv = lambda v: v / (A[None] + omega)  # noqa: E731
    else:
        Ap = A + omega * np.eye(nc).reshape((nc, nc) + (1,) * d)
        Am = np.moveaxis(np.moveaxis(Ap, 0, -1), 0, -1)
        Ainv = np.linalg.inv(Am)
        Ainv = np.moveaxis(np.moveaxis(Ainv, -1, 0), -1, 0)
        inv = lambda v: apply_A(Ainv, v)  # noqa: E731
    sgn = -1.0 if literal_sign else 1.0
    q = sgn * 2.0 * omega * inv(Econst)
    x = Econst.copy()
    nE = float(np.linalg.norm(E))
    hist, its = [], []
    nmax = fixed_iters if fixed_iters is not None else maxit
    for m in range(1, nmax + 1):
        y = apply_A(A, x) - omega * x
        x_new = inv(sys.em_project(y)) + q
        dx = _norm(x_new - x)
        x = x_new
        hist.append(dx)
        if keep_iterates:
            its.append(x.copy())
        if fixed_iters is None and dx <= tol * nE:
            return SolveResult(x, m, True, hist, its)
    return SolveResult(x, nmax, fixed_iters is not None, hist, its)
