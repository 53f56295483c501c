"""CUDA path vs the FP64 oracle, through the C ABI (libhom.so).

Per operator application the bar is 1e-12 relative (norm-wise); per solve 1e-10 on
A_H. Iterates are compared at fixed iteration counts first (Section 3 algorithms taken step by
step), then at tolerance.
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

OP_TOL = 1e-12
AH_TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def square(N, h, lo, hi, seed=None, tensor=False, idx16=False):
    d = len(N)
    ph = ms.box_phase(N, h)
    if tensor:
        table = ms.random_spd_table(2, d, seed=seed or 1, scales=[lo, hi])
    else:
        table = ms.isotropic_table([lo, hi], d)
    if idx16:
        ph = ph.astype(np.uint16)
    A = O.expand_phase(ph, table)
    if not tensor:
        A = A[0, 0]
    return ph, table, A


GRIDS = [(3, 3), (9, 7), (15, 15), (63, 63), (85, 85), (5, 7, 9), (15, 15, 15), (27, 25, 21),
         (45, 45, 45)]


@pytest.mark.parametrize("N", [(135, 135, 135), (81, 81, 81), (161, 7, 9)])
def test_operator_parity_larger_grids(N):
    # tile geometry of the served grid sizes (135 = 27*5 / 15*9, 81, 161 = 7*23)
    d = len(N)
    ph, table, A = square(N, 0.6, 1.0, 10.0)
    P = H.Problem(d, N, H.phase_material(ph, table))
    x = ms.random_field((d,) + N, 9)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    assert rel(y.cpu().numpy(), O.GaNi(A, d).matvec(x)) < OP_TOL
    P.close()


@pytest.mark.parametrize("N", GRIDS)
@pytest.mark.parametrize("op", ["affine", "linear", "project", "em"])
def test_operator_parity(N, op):
    d = len(N)
    ph, table, A = square(N, 0.6, 1.0, 10.0)
    P = H.Problem(d, N, H.phase_material(ph, table))
    x = ms.random_field((d,) + N, 7)
    E = ms.random_unit_vector(d, 2)
    y = P.field()
    opc = {"affine": H.HOM_OP_AFFINE, "linear": H.HOM_OP_LINEAR, "project": H.HOM_OP_PROJECT,
           "em": H.HOM_OP_EM}[op]
    H.hom_apply(P.h, opc, E, to_dev(x), y)
    torch.cuda.synchronize()
    sysn = O.GaNi(A, d)
    if op == "affine":
        ref = sysn.matvec(sysn.const(E) + x)
    elif op == "linear":
        ref = sysn.matvec(x)
    elif op == "project":
        ref = O.project(x)
    else:
        ref = sysn.em_project(O.apply_A(A, x) - np.sqrt(10.0) * x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()


@pytest.mark.parametrize("N", [(9, 11), (7, 5, 9)])
def test_operator_parity_anisotropic_uint16(N):
    d = len(N)
    ph, table, A = square(N, 0.5, 1.0, 30.0, seed=4, tensor=True, idx16=True)
    P = H.Problem(d, N, H.phase_material(ph, table))
    x = ms.random_field((d,) + N, 3)
    E = ms.random_unit_vector(d, 5)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_AFFINE, E, to_dev(x), y)
    sysn = O.GaNi(A, d)
    assert rel(y.cpu().numpy(), sysn.matvec(sysn.const(E) + x)) < OP_TOL
    cA, CA = O.spectral_bounds(A, d)
    H.hom_apply(P.h, H.HOM_OP_EM, None, to_dev(x), y)
    ref = sysn.em_project(O.apply_A(A, x) - np.sqrt(cA * CA) * x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()


def test_operator_parity_scalar_field():
    N = (21, 15, 9)
    d = 3
    a = 1.0 + 9.0 * np.random.default_rng(3).random(N)
    P = H.Problem(d, N, H.scalar_material(a))
    x = ms.random_field((d,) + N, 8)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    assert rel(y.cpu().numpy(), O.GaNi(a, d).matvec(x)) < OP_TOL
    P.close()


def ga_problem(N, h, lo, hi, M=None):
    d = len(N)
    Mg = tuple(M) if M is not None else O.double_grid(N)
    Ahat = ms.box_fourier_coefficients(Mg, h, lo, hi)
    P = H.Problem(d, N, H.fourier_material(Ahat.astype(np.complex128), lo, hi, M), H.HOM_EXACT)
    A_M = O.ga_coefficients(Ahat, d)
    return P, A_M, Mg


@pytest.mark.parametrize("N", [(5, 5), (15, 15), (7, 9, 5), (9, 9, 9)])
def test_ga_operator_parity(N):
    d = len(N)
    P, A_M, M = ga_problem(N, 0.6, 1.0, 10.0)
    assert P.grid == M
    x = ms.random_field((d,) + M, 9)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    ref = O.Ga(A_M, N, d).matvec(x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    # energy on the double grid: the exact Voigt value at x = 0 and a random field
    E = np.eye(d)[0]
    en, _ = H.hom_energy(P.h, E)
    assert abs(en - O.energy(A_M, O.Ga(A_M, N, d).const(E))) < 1e-12 * abs(en)
    en, _ = H.hom_energy(P.h, E, to_dev(x))
    assert abs(en - O.Ga(A_M, N, d).energy(E, x)) < 1e-12 * abs(en)
    P.close()


SOLVER_NAMES = ["richardson", "cg", "chebyshev", "eyre_milton"]


def oracle_solve(name, sysn, E, cA, CA, **kw):
    if name == "richardson":
        r = O.richardson(sysn, E, cA, CA, **kw)
        return r, r.x
    if name == "cg":
        r = O.cg(sysn, E, **kw)
        return r, r.x
    if name == "chebyshev":
        r = O.chebyshev(sysn, E, cA, CA, **kw)
        return r, r.x
    r = O.eyre_milton(sysn, E, cA, CA, **kw)
    return r, O.project(r.x)


@pytest.mark.parametrize("N", [(15, 15), (9, 7, 11)])
@pytest.mark.parametrize("solver", SOLVER_NAMES)
def test_solver_fixed_iterations(N, solver):
    d = len(N)
    ph, table, A = square(N, 0.6, 1.0, 100.0)
    P = H.Problem(d, N, H.phase_material(ph, table))
    E = np.eye(d)[0]
    x = P.field()
    its = 20
    AH, flux, stats, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 0.0, H.make_opts(fixed_iters=its), x)
    assert stats["iterations"] == its
    sysn = O.GaNi(A, d)
    _, xr = oracle_solve(solver, sysn, E, 1.0, 100.0, fixed_iters=its)
    assert rel(x.cpu().numpy(), xr) < 1e-10
    assert abs(AH - sysn.energy(E, xr)) < AH_TOL * abs(AH)
    P.close()


@pytest.mark.parametrize("N", [(63, 63), (85, 85), (15, 17, 13)])
@pytest.mark.parametrize("solver", SOLVER_NAMES)
def test_solver_tolerance(N, solver):
    d = len(N)
    ph, table, A = square(N, 0.6, 1.0, 10.0)
    P = H.Problem(d, N, H.phase_material(ph, table))
    E = np.eye(d)[0]
    tol = 1e-8
    x = P.field()
    AH, flux, stats, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], tol, None, x)
    sysn = O.GaNi(A, d)
    stop = {} if solver in ("eyre_milton",) else ({"stop": "residual"} if solver == "richardson" else {})
    r, xr = oracle_solve(solver, sysn, E, 1.0, 10.0, tol=tol, **stop)
    assert abs(stats["iterations"] - r.iterations) <= 1
    ref = sysn.energy(E, xr)
    assert abs(AH - ref) < AH_TOL * ref
    P.close()


def test_ga_cg_and_bound_square_85():
    # Section 4.3 values (2.793 GaNi bound, 2.241 Ga) through the library
    N = (85, 85)
    d = 2
    ph, table, A = square(N, 0.6, 1.0, 100.0)
    Pn = H.Problem(d, N, H.phase_material(ph, table))
    Pg, A_M, M = ga_problem(N, 0.6, 1.0, 100.0)
    E = np.array([1.0, 0.0])
    xn = Pn.field()
    H.hom_solve(Pn.h, E, H.HOM_CG, 1e-10, None, xn)
    ub = H.hom_bound(Pn.h, Pg.h, E, xn)
    xg = Pg.field()
    AHg, _, _, _ = H.hom_solve(Pg.h, E, H.HOM_CG, 1e-10, None, xg)
    sysn = O.GaNi(A, d)
    xr = O.cg(sysn, E, tol=1e-10).x
    ub_ref = O.energy(A_M, O.prolongate(sysn.const(E) + xr, M))
    sysg = O.Ga(A_M, N, d)
    ga_ref = sysg.energy(E, O.cg(sysg, E, tol=1e-10).x)
    assert abs(ub - ub_ref) < 1e-9 * ub_ref
    assert abs(AHg - ga_ref) < 1e-9 * ga_ref
    assert abs(ub - 2.793) < 5e-4 and abs(AHg - 2.241) < 5e-4
    Pn.close()
    Pg.close()


@pytest.mark.parametrize("N,M", [((5, 7), (9, 13)), ((7, 5, 9), (13, 11, 17))])
def test_prolongation_parity(N, M):
    d = len(N)
    ph, table, A = square(N, 0.6, 1.0, 10.0)
    Pn = H.Problem(d, N, H.phase_material(ph, table))
    Pm, _, _ = ga_problem(N, 0.6, 1.0, 10.0, M=M)
    x = ms.random_field((d,) + N, 12)
    y = Pm.field()
    H.hom_prolongate(Pn.h, Pm.h, to_dev(x), y)
    assert rel(y.cpu().numpy(), O.prolongate(x, M)) < OP_TOL
    Pn.close()
    Pm.close()


def test_error_paths():
    N = (9, 9)
    Pg, _, _ = ga_problem(N, 0.6, 1.0, 10.0)
    with pytest.raises(H.HomError) as ei:
        H.hom_solve(Pg.h, np.array([1.0, 0.0]), H.HOM_EYRE_MILTON, 1e-6)
    assert ei.value.status == H.HOM_ERR_UNSUPPORTED
    ph, table, _ = square(N, 0.6, 1.0, 100.0)
    P = H.Problem(2, N, H.phase_material(ph, table))
    AH, _, stats, st = H.hom_solve(P.h, np.array([1.0, 0.0]), H.HOM_RICHARDSON, 1e-12,
                                   H.make_opts(maxit=5), allow_not_converged=True)
    assert st == H.HOM_ERR_NOT_CONVERGED and stats["iterations"] == 5
    Pg.close()
    P.close()


def test_autotune_keeps_parity():
    N = (45, 45, 45)
    d = 3
    ph, table, A = square(N, 0.6, 1.0, 10.0)
    P = H.Problem(d, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    rep = H.hom_autotune(P.h, reps=2)
    assert rep["rmax64"] in (9, 15) and rep["rmax32"] in (9, 15, 27)
    assert rep["smem_kb64"] in (56, 80, 96, 110, 150, 200) and rep["ms64"] > 0 and rep["ms32"] > 0
    assert rep["smem_kb32"] in (56, 80, 96, 110, 150, 200)
    x = ms.random_field((d,) + N, 6)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    ref = O.GaNi(A, d).matvec(x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, to_dev(x), y)
    assert rel(y.cpu().numpy(), ref) < 2e-6
    # a later problem of the same grid starts from the tuned plan and solves correctly
    Q = H.Problem(d, N, H.phase_material(ph, table))
    AH, _, _, _ = H.hom_solve(Q.h, np.eye(d)[0], H.HOM_CG, 1e-10)
    sysn = O.GaNi(A, d)
    assert abs(AH - sysn.energy(np.eye(d)[0], O.cg(sysn, np.eye(d)[0], tol=1e-10).x)) < 1e-10 * AH
    P.close()
    Q.close()
