"""Pins of the oracle's linear systems (eq. (linsys)), solvers (Algorithms 1-4), energies and
bounds (eqs. (bounds), (ev_bounds)) against closed forms and dense Galerkin solves in a real
trigonometric basis that uses no DFT (tests/galerkin_basis.py)."""
import math

import numpy as np
import pytest

import microstructure as ms
import oracle as O
from tests.galerkin_basis import dense_minimiser


def _square(N, h, lo, hi):
    d = len(N)
    ph = ms.box_phase(N, h)
    return O.expand_phase(ph, ms.isotropic_table([lo, hi], d))[0, 0]


def _solve(name, sys, E, cA, CA, **kw):
    if name == "richardson":
        r = O.richardson(sys, E, cA, CA, **kw)
        return r, r.x
    if name == "cg":
        r = O.cg(sys, E, **kw)
        return r, r.x
    if name == "chebyshev":
        r = O.chebyshev(sys, E, cA, CA, **kw)
        return r, r.x
    r = O.eyre_milton(sys, E, cA, CA, **kw)
    return r, O.project(r.x)  # e = G_N x for the non-conforming iterate


SOLVERS = ["richardson", "cg", "chebyshev", "eyre_milton"]


@pytest.mark.parametrize("N,axis", [((15, 13), 0), ((9, 7, 5), 1)])
def test_laminate_closed_form(N, axis):
    # A laminate a(x_axis): the GaNi minimiser has a constant flux across the layers, so
    # A_H = harmonic mean of the nodal values across and arithmetic mean along the layers.
    d = len(N)
    ph = ms.laminate_phase(N, 0.4, axis)
    a = np.where(ph == 1, 10.0, 1.0).astype(float)
    sysn = O.GaNi(a, d)
    across = np.zeros(d)
    across[axis] = 1.0
    along = np.zeros(d)
    along[(axis + 1) % d] = 1.0
    harm = 1.0 / np.mean(1.0 / a)
    arit = np.mean(a)
    r = O.cg(sysn, across, tol=1e-12)
    assert abs(sysn.energy(across, r.x) - harm) < 1e-11 * harm
    r = O.cg(sysn, along, tol=1e-12)
    assert abs(sysn.energy(along, r.x) - arit) < 1e-11 * arit


@pytest.mark.parametrize("N", [(9, 9), (7, 5), (5, 5, 5)])
@pytest.mark.parametrize("solver", SOLVERS)
def test_solvers_match_dense_galerkin_gani(N, solver):
    d = len(N)
    a = _square(N, 0.6, 1.0, 10.0)
    E = ms.random_unit_vector(d, 3)
    e_ref, en_ref, _ = dense_minimiser(a, E, N, N)
    sysn = O.GaNi(a, d)
    r, e = _solve(solver, sysn, E, 1.0, 10.0, tol=1e-11)
    assert r.converged
    assert abs(sysn.energy(E, e) - en_ref) < 1e-9 * en_ref
    assert np.abs(e - e_ref).max() < 1e-8


def test_anisotropic_tensor_gani_matches_dense():
    N = (7, 9)
    d = 2
    ph = ms.box_phase(N, 0.5)
    table = ms.random_spd_table(2, d, seed=5, scales=[1.0, 20.0])
    A = O.expand_phase(ph, table)
    cA, CA = O.spectral_bounds(A, d)
    E = ms.random_unit_vector(d, 8)
    _, en_ref, _ = dense_minimiser(A, E, N, N)
    sysn = O.GaNi(A, d)
    for solver in SOLVERS:
        r, e = _solve(solver, sysn, E, cA, CA, tol=1e-11)
        assert abs(sysn.energy(E, e) - en_ref) < 1e-9 * en_ref, solver


@pytest.mark.parametrize("N", [(7, 7), (5, 5, 5)])
@pytest.mark.parametrize("solver", ["richardson", "cg", "chebyshev"])
def test_ga_solvers_match_dense_galerkin(N, solver):
    # eq. (Ga): minimise the exact bilinear form; the basis is sampled on the double grid.
    d = len(N)
    M = O.double_grid(N)
    A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 10.0), d)
    E = np.eye(d)[0]
    e_ref, en_ref, _ = dense_minimiser(A_M, E, N, M)
    sysg = O.Ga(A_M, N, d)
    r, e = _solve(solver, sysg, E, 1.0, 10.0, tol=1e-11)
    assert abs(sysg.energy(E, e) - en_ref) < 1e-9 * en_ref
    assert np.abs(e - e_ref).max() < 1e-7


def test_gani_bound_via_independent_prolongation():
    # eq. (ev_bounds_GaNi): U_E(R[E + e~]). The GaNi minimiser's basis coefficients, re-sampled
    # on the double grid by the closed-form basis, give the same bound as the oracle's
    # prolongation.
    N = (9, 9)
    d = 2
    M = O.double_grid(N)
    a = _square(N, 0.6, 1.0, 10.0)
    A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 10.0), d)
    E = np.array([1.0, 0.0])
    from tests.galerkin_basis import basis
    _, _, c = dense_minimiser(a, E, N, N)
    eM = (basis(N, M) @ c).reshape((d,) + M)
    bound_ref = O.energy(A_M, O.Ga(A_M, N, d).const(E) + eM)
    sysn = O.GaNi(a, d)
    r = O.cg(sysn, E, tol=1e-12)
    xb = O.prolongate(sysn.const(E) + r.x, M)
    assert abs(O.energy(A_M, xb) - bound_ref) < 1e-10 * bound_ref


def test_voigt_reuss_and_initial_energy():
    # e = 0 is admissible: U_E(0) = Voigt (Section 4.3); Reuss <= A~_H <= Voigt.
    N = (11, 11)
    a = _square(N, 0.6, 1.0, 50.0)
    sysn = O.GaNi(a, 2)
    E = np.array([1.0, 0.0])
    voigt = a.mean()
    reuss = 1.0 / np.mean(1.0 / a)
    assert abs(sysn.energy(E, np.zeros((2,) + N)) - voigt) < 1e-12
    r = O.cg(sysn, E, tol=1e-10)
    ah = sysn.energy(E, r.x)
    assert reuss < ah < voigt


def test_hashin_shtrikman_and_bound_ordering():
    # eq. (bounds): A_H <= A_{H,N} (Ga) <= GaNi bound; the isotropic two-phase lower HS bound
    # stays below the true A_H, hence below Ga.
    N = (15, 15)
    d = 2
    M = O.double_grid(N)
    a = _square(N, 0.6, 1.0, 10.0)
    A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 10.0), d)
    E = np.array([1.0, 0.0])
    sysn = O.GaNi(a, d)
    x = O.cg(sysn, E, tol=1e-12).x
    bound = O.energy(A_M, O.prolongate(sysn.const(E) + x, M))
    sysg = O.Ga(A_M, N, d)
    ga = sysg.energy(E, O.cg(sysg, E, tol=1e-12).x)
    f2 = 0.36
    f1 = 1 - f2
    hs = 1.0 + f2 / (1.0 / (10.0 - 1.0) + f1 / (d * 1.0))
    assert hs < ga < bound


def test_ga_exact_for_any_odd_double_grid():
    # Products of order-N polynomials have frequencies |k| <= N - 1, so any odd M >= 2N - 1
    # integrates them exactly: A_{H,N} is the same on M = 2N - 1 and M = 2N + 1.
    N = (7, 7)
    vals = []
    for M in [O.double_grid(N), (15, 15)]:
        A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 10.0), 2)
        sysg = O.Ga(A_M, N, 2)
        vals.append(sysg.energy(np.array([1.0, 0.0]), O.cg(sysg, np.array([1.0, 0.0]), tol=1e-13).x))
    assert abs(vals[0] - vals[1]) < 1e-11


def test_moulinec_suquet_is_richardson():
    # Footnote of Section 3.1: x_m = x_{m-1} - (G/c0) A (E + x_{m-1}) with c0 = (c_A + C_A)/2.
    N = (9, 9)
    a = _square(N, 0.6, 1.0, 10.0)
    sysn = O.GaNi(a, 2)
    E = np.array([1.0, 0.0])
    x = np.zeros((2,) + N)
    c0 = 0.5 * (1.0 + 10.0)
    for _ in range(15):
        x = x - O.project(a[None] * (sysn.const(E) + x)) / c0
    r = O.richardson(sysn, E, 1.0, 10.0, fixed_iters=15)
    np.testing.assert_allclose(r.x, x, atol=1e-13)


def test_eyre_milton_printed_sign_gives_negated_solution():
    N = (11, 11)
    a = _square(N, 0.6, 1.0, 10.0)
    sysn = O.GaNi(a, 2)
    E = np.array([1.0, 0.0])
    rp = O.eyre_milton(sysn, E, 1.0, 10.0, tol=1e-12)
    rl = O.eyre_milton(sysn, E, 1.0, 10.0, tol=1e-12, literal_sign=True)
    np.testing.assert_allclose(rl.x, -rp.x, atol=1e-10)
    # the corrected iterate converges to E + e~ with e~ the CG minimiser
    xc = O.cg(sysn, E, tol=1e-13).x
    np.testing.assert_allclose(rp.x, sysn.const(E) + xc, atol=1e-9)
    assert abs(O.energy(a, rl.x) - O.energy(a, rp.x)) < 1e-12


def test_error_estimates_hold():
    # eqs. (Richard_estimate), (CG_estimate) (also valid for Chebyshev, Section 3.3).
    N = (15, 15)
    a = _square(N, 0.6, 1.0, 10.0)
    sysn = O.GaNi(a, 2)
    E = np.array([1.0, 0.0])
    kappa = 10.0
    xs = O.cg(sysn, E, tol=1e-14).x
    nrm = lambda v: math.sqrt(np.mean(np.sum(v * v, 0)))  # noqa: E731
    cnrm = lambda v: math.sqrt(np.mean(np.sum(sysn.matvec(v) * v, 0)))  # noqa: E731
    q = (kappa - 1) / (kappa + 1)
    rr = O.richardson(sysn, E, 1.0, 10.0, fixed_iters=30, keep_iterates=True)
    for m, xm in enumerate(rr.iterates, start=1):
        assert nrm(xm - xs) <= q ** m * nrm(xs) * (1 + 1e-9) + 1e-13
    qc = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    for fn in (lambda: O.cg(sysn, E, fixed_iters=20, keep_iterates=True),
               lambda: O.chebyshev(sysn, E, 1.0, 10.0, fixed_iters=20, keep_iterates=True)):
        res = fn()
        for m, xm in enumerate(res.iterates, start=1):
            assert cnrm(xm - xs) <= 2 * qc ** m * cnrm(xs) * (1 + 1e-9) + 1e-12


def test_conformity_of_iterates():
    # Section 4.4: R/CG/Chebyshev iterates stay in E (||G x - x|| at round-off); EM iterates
    # do not (||G x + E - x|| > 0 but -> 0).
    N = (15, 15)
    a = _square(N, 0.6, 1.0, 100.0)
    sysn = O.GaNi(a, 2)
    E = np.array([1.0, 0.0])
    nrm = lambda v: math.sqrt(np.mean(np.sum(v * v, 0)))  # noqa: E731
    for res in (O.richardson(sysn, E, 1.0, 100.0, fixed_iters=25),
                O.cg(sysn, E, fixed_iters=25),
                O.chebyshev(sysn, E, 1.0, 100.0, fixed_iters=25)):
        assert nrm(O.project(res.x) - res.x) < 1e-12
    em = O.eyre_milton(sysn, E, 1.0, 100.0, fixed_iters=3)
    assert nrm(O.project(em.x) + sysn.const(E) - em.x) > 1e-4
    em = O.eyre_milton(sysn, E, 1.0, 100.0, tol=1e-10)
    assert nrm(O.project(em.x) + sysn.const(E) - em.x) < 1e-8


def test_ga_upper_bound_monotone_for_richardson_and_cg():
    # Section 4.3 / Table 1: on Ga the bound U_E(x_m) decreases monotonically for Richardson
    # and CG.
    N = (15, 15)
    d = 2
    M = O.double_grid(N)
    A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 100.0), d)
    sysg = O.Ga(A_M, N, d)
    E = np.array([1.0, 0.0])
    for res in (O.richardson(sysg, E, 1.0, 100.0, fixed_iters=40, keep_iterates=True),
                O.cg(sysg, E, fixed_iters=40, keep_iterates=True)):
        u = [sysg.energy(E, xm) for xm in res.iterates]
        assert all(u[i + 1] <= u[i] + 1e-12 for i in range(len(u) - 1))


def test_iteration_scaling_with_contrast():
    # Section 4.6: Richardson needs O(kappa) iterations, CG/Chebyshev/EM O(sqrt(kappa)).
    N = (15, 15)
    E = np.array([1.0, 0.0])
    its = {}
    for kappa in (10.0, 1000.0):
        a = _square(N, 0.6, 1.0, kappa)
        sysn = O.GaNi(a, 2)
        its[kappa] = {
            "richardson": O.richardson(sysn, E, 1.0, kappa, tol=1e-6, stop="residual").iterations,
            "cg": O.cg(sysn, E, tol=1e-6).iterations,
            "chebyshev": O.chebyshev(sysn, E, 1.0, kappa, tol=1e-6).iterations,
        }
    ratio = {k: its[1000.0][k] / its[10.0][k] for k in its[10.0]}
    assert ratio["richardson"] > 30          # ~ kappa ratio 100
    assert ratio["chebyshev"] < 15           # ~ sqrt(kappa) ratio 10
    assert ratio["cg"] < 15


def test_eyre_milton_rejects_ga():
    N = (5, 5)
    M = O.double_grid(N)
    A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 10.0), 2)
    with pytest.raises(ValueError):
        O.eyre_milton(O.Ga(A_M, N, 2), np.array([1.0, 0.0]), 1.0, 10.0)


def _gnorm(v):
    return float(np.sqrt(np.mean(np.sum(v * v, axis=0))))


def test_nonconformity_of_iterates_section_4_4():
    # Section 4.4 on the square inclusion (15^2, contrast 100): the Eyre-Milton iterate's
    # distance ||G x_m + E - x_m|| is largest at the first iteration and then falls, not
    # monotonically; it splits into orthogonal parts (squared norms add: Helmholtz
    # decomposition, the paper prints the split without the squares); the conforming solvers'
    # ||G x_m - x_m|| is round-off that grows with m
    N = (15, 15)
    a = _square(N, 0.6, 1.0, 100.0)
    sysn = O.GaNi(a, 2)
    E = np.array([1.0, 0.0])
    Ec = sysn.const(E)
    r = O.eyre_milton(sysn, E, 1.0, 100.0, fixed_iters=30, keep_iterates=True)
    nc = [_gnorm(O.project(x) + Ec - x) for x in r.iterates]
    assert int(np.argmax(nc)) == 0
    assert nc[-1] < 0.2 * nc[0]
    assert any(nc[m + 1] > nc[m] for m in range(len(nc) - 1))
    for x in r.iterates[:5]:
        mean = x.reshape(2, -1).mean(axis=1).reshape(2, 1, 1) * np.ones_like(x)
        lhs = _gnorm(O.project(x) + Ec - x) ** 2
        rhs = _gnorm(Ec - mean) ** 2 + _gnorm(O.project(x) - x + mean) ** 2
        assert abs(lhs - rhs) < 1e-12 * lhs
    for res in (O.cg(sysn, E, fixed_iters=30, keep_iterates=True),
                O.richardson(sysn, E, 1.0, 100.0, fixed_iters=30, keep_iterates=True)):
        rel = [_gnorm(O.project(x) - x) / _gnorm(x) for x in res.iterates]
        assert max(rel) < 1e-12
