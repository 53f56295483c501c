"""Pins of the linear-elasticity oracle (oracle/elastic.py) against facts it does not compute
itself: closed-form symmetric gradients and equilibrated stresses, Saint-Venant compatibility
evaluated with NumPy's FFT, the laminate (Backus) closed form, the reduction of antiplane shear
to the scalar conductivity problem, dense Galerkin solves in a displacement basis, the spectrum
of the assembled operator, and the Voigt/Reuss bounds."""
import math

import numpy as np
import pytest

import microstructure as ms
import oracle as O
from tests.galerkin_elastic import dense_minimiser

EL = O.elastic
SQ2 = math.sqrt(2.0)


def trig_displacement(N, seed, nmodes=5):
    """A random trigonometric displacement field of order N: its Mandel strain sym(grad u) at
    the nodes, by closed-form derivatives."""
    rng = np.random.default_rng(seed)
    d = len(N)
    xs = ms.node_coords(N)
    grad = np.zeros((d, d) + tuple(N))  # grad[i, a] = d u_i / d x_a
    for _ in range(nmodes):
        k = np.array([rng.integers(-(n - 1) // 2, (n - 1) // 2 + 1) for n in N])
        amp = rng.standard_normal((d, 2))
        t = np.broadcast_to(sum(2 * np.pi * k[a] * xs[a] for a in range(d)), tuple(N))
        for i in range(d):
            for a in range(d):
                grad[i, a] += 2 * np.pi * k[a] * (-amp[i, 0] * np.sin(t) + amp[i, 1] * np.cos(t))
    sym = 0.5 * (grad + np.swapaxes(grad, 0, 1))
    return EL.to_mandel(sym, d)


def random_stiffness_table(nphase, d, seed, scale=(1.0, 10.0)):
    """SPD Mandel matrices: Q diag(lambda) Q^T with random orthogonal Q."""
    rng = np.random.default_rng(seed)
    nc = EL.ncomp(d)
    out = []
    for p in range(nphase):
        q, r = np.linalg.qr(rng.standard_normal((nc, nc)))
        q = q * np.sign(np.diag(r))
        lam = scale[p % len(scale)] * np.exp(rng.uniform(0, np.log(3.0), nc))
        out.append(q @ np.diag(lam) @ q.T)
    return np.array(out)


def test_mandel_storage_makes_the_frobenius_product_euclidean():
    rng = np.random.default_rng(1)
    for d in (2, 3):
        a = rng.standard_normal((d, d, 4))
        b = rng.standard_normal((d, d, 4))
        a = a + np.swapaxes(a, 0, 1)
        b = b + np.swapaxes(b, 0, 1)
        frob = np.einsum("ij...,ij...->...", a, b)
        np.testing.assert_allclose(np.sum(EL.to_mandel(a, d) * EL.to_mandel(b, d), axis=0), frob)
        np.testing.assert_allclose(EL.to_tensor(EL.to_mandel(a, d), d), a)


@pytest.mark.parametrize("N", [(9, 7), (5, 7, 9)])
def test_projection_fixes_symmetric_gradients_and_kills_constants(N):
    d = len(N)
    e = trig_displacement(N, 3)
    np.testing.assert_allclose(EL.project_strain(e, d), e, atol=1e-11)
    const = np.ones((EL.ncomp(d),) + N) * np.arange(1, EL.ncomp(d) + 1).reshape((-1,) + (1,) * d)
    np.testing.assert_allclose(EL.project_strain(const, d), 0.0, atol=1e-12)


def test_projection_kills_equilibrated_stresses_2d():
    # Airy stress function phi: s11 = phi_,22, s22 = phi_,11, s12 = -phi_,12 (div s = 0)
    N = (9, 11)
    rng = np.random.default_rng(5)
    xs = ms.node_coords(N)
    s = np.zeros((2, 2) + N)
    for _ in range(4):
        k = np.array([rng.integers(-4, 5), rng.integers(-5, 6)])
        a, b = rng.standard_normal(2)
        t = np.broadcast_to(2 * np.pi * (k[0] * xs[0] + k[1] * xs[1]), N)
        f = -(2 * np.pi) ** 2 * (a * np.cos(t) + b * np.sin(t))  # second derivative factor
        s[0, 0] += k[1] * k[1] * f
        s[1, 1] += k[0] * k[0] * f
        s[0, 1] += -k[0] * k[1] * f
        s[1, 0] += -k[0] * k[1] * f
    np.testing.assert_allclose(EL.project_strain(EL.to_mandel(s, 2), 2), 0.0, atol=1e-9)


def test_projection_kills_equilibrated_stresses_3d():
    # fields of two coordinates: an Airy block in the (x_p, x_q) plane, an out-of-plane normal
    # stress of (x_p, x_q) and an antiplane pair s_pr = psi_,q, s_qr = -psi_,p; div s = 0
    N = (7, 5, 9)
    rng = np.random.default_rng(6)
    xs = ms.node_coords(N)
    for p, q, r in [(0, 1, 2), (0, 2, 1), (1, 2, 0)]:
        s = np.zeros((3, 3) + N)
        for _ in range(3):
            k = np.zeros(3, int)
            k[p] = rng.integers(-(N[p] - 1) // 2, (N[p] - 1) // 2 + 1)
            k[q] = rng.integers(-(N[q] - 1) // 2, (N[q] - 1) // 2 + 1)
            a, b, c = rng.standard_normal(3)
            t = np.broadcast_to(2 * np.pi * sum(k[i] * xs[i] for i in range(3)), N)
            f2 = -(2 * np.pi) ** 2 * (a * np.cos(t) + b * np.sin(t))
            s[p, p] += k[q] * k[q] * f2
            s[q, q] += k[p] * k[p] * f2
            s[p, q] += -k[p] * k[q] * f2
            s[q, p] += -k[p] * k[q] * f2
            s[r, r] += c * np.cos(t)  # depends on x_p, x_q only: d/dx_r of it is zero
            f1 = 2 * np.pi * c * np.cos(t)  # psi = c sin(t)
            s[p, r] += k[q] * f1
            s[r, p] += k[q] * f1
            s[q, r] += -k[p] * f1
            s[r, q] += -k[p] * f1
        s -= s.mean(axis=(2, 3, 4), keepdims=True)
        np.testing.assert_allclose(EL.project_strain(EL.to_mandel(s, 3), 3), 0.0, atol=1e-9)


def _fft_k(N):
    return np.meshgrid(*[np.fft.fftfreq(n, 1.0 / n) for n in N], indexing="ij")


def test_projection_output_is_compatible_saint_venant():
    # 2-D: k2^2 e11 + k1^2 e22 - 2 k1 k2 e12 = 0; 3-D: inc(e)_ij = eps_ikl eps_jmn k_k k_m e_ln = 0
    rng = np.random.default_rng(8)
    N = (9, 7)
    y = EL.to_tensor(EL.project_strain(rng.standard_normal((3,) + N), 2), 2)
    yh = np.fft.fftn(y, axes=(2, 3))
    k1, k2 = _fft_k(N)
    inc = k2 * k2 * yh[0, 0] + k1 * k1 * yh[1, 1] - 2 * k1 * k2 * yh[0, 1]
    assert np.max(np.abs(inc)) < 1e-9 * np.max(np.abs(yh))
    N3 = (5, 7, 3)
    y = EL.to_tensor(EL.project_strain(rng.standard_normal((6,) + N3), 3), 3)
    yh = np.fft.fftn(y, axes=(2, 3, 4))
    k = _fft_k(N3)
    eps = np.zeros((3, 3, 3))
    for i, j, l in [(0, 1, 2), (1, 2, 0), (2, 0, 1)]:
        eps[i, j, l], eps[j, i, l] = 1.0, -1.0
    inc = np.einsum("ikl,jmn,k...,m...,ln...->ij...", eps, eps, np.array(k), np.array(k), yh)
    assert np.max(np.abs(inc)) < 1e-9 * np.max(np.abs(yh))


@pytest.mark.parametrize("d", [2, 3])
def test_projection_is_an_orthogonal_projection(d):
    rng = np.random.default_rng(9)
    N = (7, 9) if d == 2 else (5, 3, 7)
    nc = EL.ncomp(d)
    u = rng.standard_normal((nc,) + N)
    v = rng.standard_normal((nc,) + N)
    Gu = EL.project_strain(u, d)
    np.testing.assert_allclose(EL.project_strain(Gu, d), Gu, atol=1e-12)
    assert abs(np.sum(Gu * v) - np.sum(u * EL.project_strain(v, d))) < 1e-10 * np.sum(np.abs(u * v))


def backus_energy(phase, lam, mu, E, d):
    """Closed-form laminate (layers normal to x_1, isotropic phases): traction continuity
    s_11, s_12, s_13 constant; e_22, e_33, e_23 equal to E; means of e_11, e_12, e_13 equal to
    E's. Returns the nodal mean of e : C : e of that strain field."""
    lam = np.asarray(lam)[phase]
    mu = np.asarray(mu)[phase]
    T = EL.to_tensor(np.asarray(E, float).reshape(-1, 1), d)[..., 0]
    M = lam + 2 * mu
    tr_t = sum(T[a, a] for a in range(1, d))
    s1 = (T[0, 0] + tr_t * np.mean(lam / M)) / np.mean(1.0 / M)
    e = np.broadcast_to(T.reshape((d, d) + (1,) * phase.ndim), (d, d) + phase.shape).copy()
    e[0, 0] = (s1 - lam * tr_t) / M
    for b in range(1, d):
        sb = T[0, b] / np.mean(1.0 / (2 * mu))
        e[0, b] = e[b, 0] = sb / (2 * mu)
    tr = sum(e[a, a] for a in range(d))
    w = lam * tr * tr + 2 * mu * np.einsum("ij...,ij...->...", e, e)
    return float(np.mean(w))


@pytest.mark.parametrize("N", [(15, 5), (21, 3), (9, 5, 3), (15, 3, 5)])
def test_laminate_closed_form(N):
    d = len(N)
    ph = ms.laminate_phase(N, 0.4, axis=0)
    lam, mu = [1.0, 30.0], [0.8, 12.0]
    table = np.array([EL.isotropic_stiffness(lam[p], mu[p], d) for p in range(2)])
    sysn = EL.GaNiElastic(EL.expand_stiffness(ph, table), d)
    rng = np.random.default_rng(11)
    for E in list(np.eye(EL.ncomp(d))) + [rng.standard_normal(EL.ncomp(d))]:
        x = O.cg(sysn, E, tol=1e-13).x
        ref = backus_energy(ph, lam, mu, E, d)
        assert abs(sysn.energy(E, x) - ref) < 1e-10 * ref


def test_antiplane_shear_reduces_to_scalar_conduction():
    # 3-D fields constant along x_3, E with only e_13, e_23: the elastic energy equals the
    # scalar energy with conductivity mu and macroscopic gradient F = 2 (E_13, E_23)
    N2 = (9, 7)
    ph2 = ms.box_phase(N2, 0.6)
    lam, mu = [2.0, 40.0], [1.0, 15.0]
    ph3 = np.repeat(ph2[:, :, None], 3, axis=2)
    table = np.array([EL.isotropic_stiffness(lam[p], mu[p], 3) for p in range(2)])
    sys3 = EL.GaNiElastic(EL.expand_stiffness(ph3, table), 3)
    e13, e23 = 0.3, -0.7
    E = np.zeros(6)
    E[3], E[4] = SQ2 * e23, SQ2 * e13
    en3 = sys3.energy(E, O.cg(sys3, E, tol=1e-13).x)
    a = np.asarray(mu)[ph2]
    sys2 = O.GaNi(a, 2)
    F = np.array([2 * e13, 2 * e23])
    en2 = sys2.energy(F, O.cg(sys2, F, tol=1e-13).x)
    assert abs(en3 - en2) < 1e-10 * en2


@pytest.mark.parametrize("N", [(5, 7), (7, 5), (3, 5, 3), (5, 3, 3)])
def test_dense_displacement_galerkin(N):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = random_stiffness_table(2, d, seed=2, scale=(1.0, 20.0))
    C = EL.expand_stiffness(ph, table)
    sysn = EL.GaNiElastic(C, d)
    E = np.random.default_rng(3).standard_normal(EL.ncomp(d))
    e_ref, en_ref = dense_minimiser(C, E, N)
    x = O.cg(sysn, E, tol=1e-14, maxit=5000).x
    np.testing.assert_allclose(x, e_ref, atol=1e-9 * np.max(np.abs(e_ref)))
    assert abs(sysn.energy(E, x) - en_ref) < 1e-11 * en_ref


def test_operator_spectrum_lies_in_the_stiffness_bounds():
    # the non-zero eigenvalues of G C (assembled column by column) lie in [c_A, C_A]; the
    # nullity is that of G: |N| nc - d (|N| - 1)
    N = (5, 3)
    d = 2
    nc = 3
    ph = ms.box_phase(N, 0.6)
    table = random_stiffness_table(2, d, seed=4, scale=(1.0, 8.0))
    C = EL.expand_stiffness(ph, table)
    sysn = EL.GaNiElastic(C, d)
    n = nc * int(np.prod(N))
    K = np.stack([sysn.matvec(np.eye(n)[j].reshape((nc,) + N)).ravel() for j in range(n)], 1)
    ev = np.sort(np.linalg.eigvals(K).real)
    cA, CA = O.spectral_bounds(C, d)
    nz = ev[np.abs(ev) > 1e-9]
    assert len(nz) == d * (int(np.prod(N)) - 1)
    assert nz.min() >= cA * (1 - 1e-10) and nz.max() <= CA * (1 + 1e-10)


def test_voigt_reuss_and_isotropic_homogeneous():
    N = (7, 5, 9)
    d = 3
    ph, _, radii = ms.rsa_spheres(N, 3, rmin=0.15, rmax=0.25, vf=0.3)
    table = np.array([EL.isotropic_stiffness(1.0, 1.0, 3)] +
                     [EL.isotropic_stiffness(20.0, 8.0, 3)] * len(radii))
    C = EL.expand_stiffness(ph, table)
    sysn = EL.GaNiElastic(C, d)
    rng = np.random.default_rng(12)
    Cm = np.moveaxis(np.moveaxis(C, 0, -1), 0, -1)
    voigt = Cm.mean(axis=(0, 1, 2))
    reuss = np.linalg.inv(np.linalg.inv(Cm).mean(axis=(0, 1, 2)))
    for _ in range(3):
        E = rng.standard_normal(6)
        en = sysn.energy(E, O.cg(sysn, E, tol=1e-12).x)
        assert E @ reuss @ E < en < E @ voigt @ E
    hom = EL.GaNiElastic(EL.expand_stiffness(np.zeros(N, np.uint8),
                                             EL.isotropic_stiffness(3.0, 2.0, 3)[None]), 3)
    E = rng.standard_normal(6)
    x = O.cg(hom, E, tol=1e-12).x
    assert np.max(np.abs(x)) < 1e-13
    assert abs(hom.energy(E, x) - E @ EL.isotropic_stiffness(3.0, 2.0, 3) @ E) < 1e-12


def test_all_four_solvers_reach_the_same_stiffness():
    N = (9, 7)
    d = 2
    ph = ms.box_phase(N, 0.6)
    table = np.array([EL.isotropic_stiffness(1.0, 1.0, 2), EL.isotropic_stiffness(10.0, 5.0, 2)])
    C = EL.expand_stiffness(ph, table)
    sysn = EL.GaNiElastic(C, d)
    cA, CA = O.spectral_bounds(C, d)
    E = np.array([1.0, 0.2, 0.3])
    ref = sysn.energy(E, O.cg(sysn, E, tol=1e-12).x)
    r = O.richardson(sysn, E, cA, CA, tol=1e-11, stop="residual")
    c = O.chebyshev(sysn, E, cA, CA, tol=1e-11)
    em = O.eyre_milton(sysn, E, cA, CA, tol=1e-12)
    assert r.converged and c.converged and em.converged
    for x in (r.x, c.x):
        assert abs(sysn.energy(E, x) - ref) < 1e-9 * ref
    # Eyre-Milton's iterate approximates E + e; its conforming part G x_m is the corrector
    e_em = EL.project_strain(em.x, d)
    assert abs(sysn.energy(E, e_em) - ref) < 1e-8 * ref
