"""Seeded synthetic periodic microstructures: the inputs shared by the GPU path and the oracle.

This module describes *problems*, it computes nothing of the solution method: phase images
sampled at the grid nodes, per-phase coefficient tables, the Fourier coefficients of a box
inclusion (the microstructure written in Fourier space), random macroscopic fields and random
trial vectors. Both the CUDA path (through its tests and the benchmark) and the CPU oracle
read their inputs from here; neither side's arithmetic lives here.

Conventions (shared by every field in this project):
  * The unit cell is Y = (-1/2, 1/2)^d (Section 2).
  * A grid of odd order N = (N_1, ..., N_d) has nodes x^m = (m_a / N_a)_a for m in Z_N
    (Section 2.1, eq. (grid)); array index j along an axis stores the signed index
    m = j for j <= (N-1)/2 and m = j - N otherwise ("FFT-natural order"), so index 0 is x = 0.
  * Scalar images have shape (N_1, ..., N_d) in C order (axis d contiguous); vector fields
    have shape (d, N_1, ..., N_d), component a belongs to spatial axis a.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "signed_index", "node_coords", "box_phase", "laminate_phase", "rsa_spheres",
    "box_fourier_coefficients", "isotropic_table", "random_spd_table", "random_unit_vector",
    "random_field", "inclusion_side_for_fraction",
]


def signed_index(n: int) -> np.ndarray:
    """Signed node/frequency index of each storage position along one axis of odd length n."""
    if n <= 0 or n % 2 == 0:
        raise ValueError(f"grid order must be odd and positive, got {n}")
    j = np.arange(n)
    return np.where(j <= (n - 1) // 2, j, j - n)


def node_coords(N) -> list[np.ndarray]:
    """Broadcastable node coordinates x_a = m_a / N_a of a grid of order N."""
    N = tuple(int(n) for n in N)
    d = len(N)
    out = []
    for a, n in enumerate(N):
        shape = [1] * d
        shape[a] = n
        out.append((signed_index(n) / n).reshape(shape))
    return out


def box_phase(N, h) -> np.ndarray:
    """Centred box inclusion of side h (a scalar or one side per axis): phase 1 at every node
    with |x_a| < h_a/2 for all a, phase 0 elsewhere (point sampling at the nodes)."""
    N = tuple(int(n) for n in N)
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (len(N),))
    inside = np.ones(N, dtype=bool)
    for a, x in enumerate(node_coords(N)):
        inside = inside & (np.abs(x) < hs[a] / 2)
    return inside.astype(np.uint8)


def laminate_phase(N, h, axis: int = 0) -> np.ndarray:
    """Layer |x_axis| < h/2 (phase 1) in a matrix (phase 0): a laminate varying along `axis`."""
    N = tuple(int(n) for n in N)
    x = node_coords(N)[axis]
    return np.broadcast_to(np.abs(x) < h / 2, N).astype(np.uint8).copy()


def inclusion_side_for_fraction(vf: float, d: int) -> float:
    """Side of a centred box inclusion whose continuous volume fraction is vf."""
    return float(vf) ** (1.0 / d)


def rsa_spheres(N, seed: int, rmin: float = 0.02, rmax: float = 0.06, vf: float = 0.3,
                max_tries: int = 200000):
    """Random sequential addition of non-overlapping periodic spheres (minimum image).

    Radii are uniform in [rmin, rmax] (fractions of the cell), centres uniform in the cell.
    Spheres are added until the node-sampled volume fraction reaches vf. Returns
    (phase, centres, radii): phase is uint16, 0 for the matrix and s+1 inside sphere s.
    Each sphere is rasterised only over its periodic bounding box of nodes.
    """
    N = tuple(int(n) for n in N)
    d = len(N)
    rng = np.random.default_rng(seed)
    phase = np.zeros(N, dtype=np.uint16)
    centres = np.zeros((0, d))
    radii = np.zeros(0)
    covered = 0
    total = int(np.prod(N))
    tries = 0
    while covered < vf * total and tries < max_tries and len(radii) < 65534:
        tries += 1
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(-0.5, 0.5, size=d)
        if len(radii):
            dv = centres - c[None, :]
            dv -= np.round(dv)
            if np.any(np.sum(dv * dv, axis=1) < (radii + r) ** 2):
                continue
        # nodes m/N_a within the periodic bounding box of the sphere
        idx, offs = [], []
        for a, n in enumerate(N):
            lo = int(np.floor((c[a] - r) * n)) - 1
            hi = int(np.ceil((c[a] + r) * n)) + 1
            m = np.arange(lo, hi + 1)
            idx.append(np.mod(m, n))
            offs.append(m / n - c[a])
        dist2 = np.zeros([len(o) for o in offs])
        for a in range(d):
            shape = [1] * d
            shape[a] = len(offs[a])
            dist2 = dist2 + (offs[a] ** 2).reshape(shape)
        inside = dist2 < r * r
        sub = phase[np.ix_(*idx)]
        newly = inside & (sub == 0)
        sub[newly] = len(radii) + 1
        phase[np.ix_(*idx)] = sub
        covered += int(newly.sum())
        centres = np.vstack([centres, c[None, :]])
        radii = np.append(radii, r)
    return phase, centres, radii


def box_fourier_coefficients(M, h, a_matrix: float, a_incl: float) -> np.ndarray:
    """Fourier coefficients A^(n), n in Z_M (FFT-natural order), of the isotropic scalar
    coefficient a_matrix + (a_incl - a_matrix) * chi_box for a centred box of side h.

    The characteristic function of the box |x_a| < h_a/2 has the coefficients
    prod_a h_a sinc(pi n_a h_a) with sinc(t) = sin(t)/t, sinc(0) = 1 (eq. (FT_def) integrated
    over the box). The result is real because the box is centred at the origin.
    """
    M = tuple(int(m) for m in M)
    d = len(M)
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (d,))
    coef = np.ones(M)
    for a, m in enumerate(M):
        n = signed_index(m).astype(np.float64)
        f = hs[a] * np.sinc(n * hs[a])  # numpy sinc(t) = sin(pi t)/(pi t)
        shape = [1] * d
        shape[a] = m
        coef = coef * f.reshape(shape)
    coef = (a_incl - a_matrix) * coef
    coef[(0,) * d] += a_matrix
    return coef


def isotropic_table(values, d: int) -> np.ndarray:
    """Per-phase coefficient table (nphase, d, d) of isotropic phases a_p * I."""
    v = np.asarray(values, dtype=np.float64)
    return v[:, None, None] * np.eye(d)[None, :, :]


def random_spd_table(nphase: int, d: int, seed: int, scales, aniso=(1.0, 3.0)) -> np.ndarray:
    """Anisotropic SPD phase tensors R diag(lambda) R^T with Haar-random rotations R
    (QR of a Gaussian matrix, signs fixed) and lambda_i = scale_p * logU[aniso]."""
    rng = np.random.default_rng(seed)
    out = np.empty((nphase, d, d))
    scales = np.broadcast_to(np.asarray(scales, dtype=np.float64), (nphase,))
    lo, hi = np.log(aniso[0]), np.log(aniso[1])
    for p in range(nphase):
        q, r = np.linalg.qr(rng.standard_normal((d, d)))
        q = q * np.sign(np.diag(r))[None, :]
        lam = scales[p] * np.exp(rng.uniform(lo, hi, size=d))
        t = (q * lam[None, :]) @ q.T
        out[p] = 0.5 * (t + t.T)
    return out


def random_unit_vector(d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(d)
    return v / np.linalg.norm(v)


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded standard-normal trial field (used as an operator argument in parity tests)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=tuple(shape)).astype(dtype)
