"""Per-iteration diagnostics through the C ABI: the history of each solver's stopping quantity
(Algorithms 1-4) and the iterate of every step, with its energy and guaranteed upper bound
(eq. (guar_upper_bound_m), Section 4.3), against the FP64 oracle's own histories and iterates.
"""
import numpy as np
import pytest

import microstructure as ms
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402

# both sides run the same recurrences in FP64 with a different rounding order: the histories
# agree to round-off amplified by the iteration, far below the stopping tolerances
HIST_RTOL = 1e-7


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gnorm(v):
    # ||v|| with the 1/|N| weight of Section 1: sum over components, mean over the grid
    return float(np.sqrt(np.mean(np.sum(v * v, axis=0))))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def square(N, h, lo, hi):
    d = len(N)
    ph = ms.box_phase(N, h)
    table = ms.isotropic_table([lo, hi], d)
    return ph, table, O.expand_phase(ph, table)[0, 0]


CASES = [("richardson", "increment"), ("richardson", "residual"), ("cg", None),
         ("chebyshev", None), ("eyre_milton", None)]


@pytest.mark.parametrize("N", [(15, 15), (9, 7, 11)])
@pytest.mark.parametrize("solver,stop", CASES)
def test_history_matches_oracle(N, solver, stop):
    d = len(N)
    lo, hi = 1.0, 10.0
    ph, table, A = square(N, 0.6, lo, hi)
    P = H.Problem(d, N, H.phase_material(ph, table))
    E = np.eye(d)[0]
    tol = 1e-8
    hstop = {None: H.HOM_STOP_DEFAULT, "increment": H.HOM_STOP_INCREMENT,
             "residual": H.HOM_STOP_RESIDUAL}[stop]
    _, _, stats, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], tol, H.make_opts(stop=hstop))
    hist = H.hom_solve_history(P.h)
    sysn = O.GaNi(A, d)
    kw = {"stop": stop} if solver == "richardson" else {}
    if solver == "richardson":
        r = O.richardson(sysn, E, lo, hi, tol=tol, **kw)
    elif solver == "cg":
        r = O.cg(sysn, E, tol=tol)
    elif solver == "chebyshev":
        r = O.chebyshev(sysn, E, lo, hi, tol=tol)
    else:
        r = O.eyre_milton(sysn, E, lo, hi, tol=tol)
    ref = np.array(r.history)
    assert len(ref) > 3
    # one entry an iteration (Richardson on the residual: one more, the converged residual)
    extra = 1 if stop == "residual" else 0
    assert len(hist) == stats["iterations"] + extra
    assert abs(len(hist) - len(ref)) <= 1
    m = min(len(hist), len(ref))
    err = np.abs(hist[:m] - ref[:m]) / ref[:m]
    assert err.max() < HIST_RTOL, (err.max(), int(err.argmax()))
    # the last entry met the stopping test, the one before did not
    thresh = tol * (np.linalg.norm(E) if stop == "increment" or solver == "eyre_milton"
                    else gnorm(sysn.rhs(E)))
    assert hist[-1] <= thresh * (1 + 1e-9) and hist[-2] > thresh * (1 - 1e-9)
    P.close()


@pytest.mark.parametrize("solver", ["cg", "chebyshev", "richardson", "eyre_milton"])
def test_every_iterate_and_its_bound(solver):
    # e_m after each single step, its energy and the guaranteed bound U_E(R_{N,M}[E + e_m])
    N = (15, 15)
    d = 2
    lo, hi = 1.0, 100.0
    ph, table, A = square(N, 0.6, lo, hi)
    Pn = H.Problem(d, N, H.phase_material(ph, table))
    M = O.double_grid(N)
    Ahat = ms.box_fourier_coefficients(M, 0.6, lo, hi)
    Pg = H.Problem(d, N, H.fourier_material(Ahat.astype(np.complex128), lo, hi, M), H.HOM_EXACT)
    A_M = O.ga_coefficients(Ahat, d)
    E = np.array([1.0, 0.0])
    steps = 8
    H.hom_solve_begin(Pn.h, E, H.SOLVERS[solver], 0.0, H.make_opts(fixed_iters=steps))
    sysn = O.GaNi(A, d)
    if solver == "cg":
        r = O.cg(sysn, E, fixed_iters=steps, keep_iterates=True)
    elif solver == "chebyshev":
        r = O.chebyshev(sysn, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    elif solver == "richardson":
        r = O.richardson(sysn, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    else:
        r = O.eyre_milton(sysn, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    x = Pn.field()
    bounds = []
    for m in range(1, steps + 1):
        H.hom_solve_iterate(Pn.h, 1)
        H.hom_solve_current(Pn.h, x)
        xr = r.iterates[m - 1]
        if solver == "eyre_milton":
            xr = O.project(xr)  # the conforming part G x_m (Section 4.4)
        assert rel(x.cpu().numpy(), xr) < 1e-10, m
        en, _ = H.hom_energy(Pn.h, E, x)
        assert abs(en - sysn.energy(E, xr)) < 1e-10 * abs(en)
        ub = H.hom_bound(Pn.h, Pg.h, E, x)
        ub_ref = O.energy(A_M, O.prolongate(sysn.const(E) + xr, M))
        assert abs(ub - ub_ref) < 1e-10 * ub_ref, m
        bounds.append(ub)
    AH, _, stats, _ = H.hom_solve_end(Pn.h, d, x)
    assert stats["iterations"] == steps
    # after the session the history stays readable (one entry a step); the last bound is that
    # of the returned iterate
    assert len(H.hom_solve_history(Pn.h)) == steps
    assert abs(H.hom_bound(Pn.h, Pg.h, E, x) - bounds[-1]) < 1e-13 * bounds[-1]
    with pytest.raises(H.HomError):
        H.hom_solve_current(Pn.h, x)  # no active session
    Pn.close()
    Pg.close()


def test_refined_history_is_the_outer_residual():
    N = (21, 23, 19)
    d = 3
    ph, table, A = square(N, 0.6, 1.0, 100.0)
    P = H.Problem(d, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    E = np.eye(d)[0]
    tol = 1e-9
    _, _, stats, _ = H.hom_solve(P.h, E, H.HOM_CG, tol, H.make_opts(inner_tol=1e-4))
    hist = H.hom_solve_history(P.h)
    assert len(hist) == stats["iterations"] >= 2
    assert np.all(np.diff(hist) < 0)
    nb = gnorm(O.GaNi(A, d).rhs(E))
    assert abs(hist[-1] / nb - stats["residual"]) < 1e-6 * stats["residual"]
    assert hist[-1] <= tol * nb and hist[-2] > tol * nb
    P.close()


def ga_square(N, h, lo, hi):
    d = len(N)
    M = O.double_grid(N)
    Ahat = ms.box_fourier_coefficients(M, h, lo, hi)
    P = H.Problem(d, N, H.fourier_material(Ahat.astype(np.complex128), lo, hi, M), H.HOM_EXACT)
    return P, O.Ga(O.ga_coefficients(Ahat, d), N, d)


@pytest.mark.parametrize("solver,monotone", [("cg", True), ("richardson", True),
                                             ("chebyshev", False)])
def test_ga_upper_bound_monotonicity(solver, monotone):
    # Table of Section 5: on Ga the bound U_E(x_m) decreases monotonically for Richardson and
    # CG and not for Chebyshev (23^2 square on 45^2, contrast 100), on both sides, iterate by
    # iterate
    N = (23, 23)
    lo, hi = 1.0, 100.0
    P, sysg = ga_square(N, 0.6, lo, hi)
    E = np.array([1.0, 0.0])
    steps = 25
    H.hom_solve_begin(P.h, E, H.SOLVERS[solver], 0.0, H.make_opts(fixed_iters=steps))
    if solver == "cg":
        r = O.cg(sysg, E, fixed_iters=steps, keep_iterates=True)
    elif solver == "richardson":
        r = O.richardson(sysg, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    else:
        r = O.chebyshev(sysg, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    x = P.field()
    u, u_ref = [], []
    for m in range(steps):
        H.hom_solve_iterate(P.h, 1)
        H.hom_solve_current(P.h, x)
        u.append(H.hom_energy(P.h, E, x)[0])
        u_ref.append(sysg.energy(E, r.iterates[m]))
    H.hom_solve_end(P.h, 2)
    u, u_ref = np.array(u), np.array(u_ref)
    assert np.max(np.abs(u - u_ref) / u_ref) < 1e-10
    rise = np.max(np.diff(u)) / u[0]
    if monotone:
        assert rise <= 1e-13
    else:
        assert rise > 1e-3 and np.max(np.diff(u_ref)) / u_ref[0] > 1e-3
    P.close()


def test_iterations_against_contrast_match_oracle():
    # Section 4.6 on the square inclusion: iterations to the relative residual 1e-6 (Eyre-Milton
    # on its increment) for contrast 10 and 1000, GaNi and Ga, against the oracle's counts; and
    # the O(kappa) / O(sqrt(kappa)) growth
    N = (15, 15)
    E = np.array([1.0, 0.0])
    tol = 1e-6
    its = {}
    for kappa in (10.0, 1000.0):
        ph, table, A = square(N, 0.6, 1.0, kappa)
        Pn = H.Problem(2, N, H.phase_material(ph, table))
        Pg, sysg = ga_square(N, 0.6, 1.0, kappa)
        sysn = O.GaNi(A, 2)
        for disc, P, sy in (("gani", Pn, sysn), ("ga", Pg, sysg)):
            for s in ("richardson", "cg", "chebyshev", "eyre_milton"):
                if disc == "ga" and s == "eyre_milton":
                    continue
                stop = H.HOM_STOP_INCREMENT if s == "eyre_milton" else H.HOM_STOP_RESIDUAL
                _, _, st, _ = H.hom_solve(P.h, E, H.SOLVERS[s], tol, H.make_opts(stop=stop))
                if s == "richardson":
                    ref = O.richardson(sy, E, 1.0, kappa, tol=tol, stop="residual").iterations
                elif s == "cg":
                    ref = O.cg(sy, E, tol=tol).iterations
                elif s == "chebyshev":
                    ref = O.chebyshev(sy, E, 1.0, kappa, tol=tol).iterations
                else:
                    ref = O.eyre_milton(sy, E, 1.0, kappa, tol=tol).iterations
                assert abs(st["iterations"] - ref) <= 1, (disc, s, kappa, st["iterations"], ref)
                its[(disc, s, kappa)] = st["iterations"]
        Pn.close()
        Pg.close()
    growth = {k[:2]: its[k[:2] + (1000.0,)] / its[k[:2] + (10.0,)] for k in its if k[2] == 10.0}
    assert growth[("gani", "richardson")] > 30 and growth[("ga", "richardson")] > 30
    for k, g in growth.items():
        if k[1] != "richardson":
            assert g < 15, (k, g)


@pytest.mark.parametrize("solver", ["eyre_milton", "cg", "richardson"])
def test_nonconformity_every_iterate(solver):
    # Section 4.4: ||G x_m + E - x_m|| (Eyre-Milton) and ||G x_m - x_m|| (conforming solvers,
    # round-off) after each of 10 single steps, against the oracle's iterates
    N = (15, 15)
    lo, hi = 1.0, 100.0
    ph, table, A = square(N, 0.6, lo, hi)
    P = H.Problem(2, N, H.phase_material(ph, table))
    E = np.array([1.0, 0.0])
    steps = 10
    H.hom_solve_begin(P.h, E, H.SOLVERS[solver], 0.0, H.make_opts(fixed_iters=steps))
    sysn = O.GaNi(A, 2)
    if solver == "eyre_milton":
        r = O.eyre_milton(sysn, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    elif solver == "cg":
        r = O.cg(sysn, E, fixed_iters=steps, keep_iterates=True)
    else:
        r = O.richardson(sysn, E, lo, hi, fixed_iters=steps, keep_iterates=True)
    Ec = sysn.const(E)
    got = []
    for m in range(steps):
        H.hom_solve_iterate(P.h, 1)
        got.append(H.hom_solve_nonconformity(P.h))
        x = r.iterates[m]
        if solver == "eyre_milton":
            ref = gnorm(O.project(x) + Ec - x)
            assert abs(got[-1] - ref) < 1e-9 * ref, m
        else:
            assert got[-1] < 1e-12 * gnorm(x), m
    if solver == "eyre_milton":
        assert int(np.argmax(got)) == 0  # largest at the first iteration (Section 4.4)
    H.hom_solve_end(P.h, 2)
    with pytest.raises(H.HomError):
        H.hom_solve_nonconformity(P.h)
    P.close()
