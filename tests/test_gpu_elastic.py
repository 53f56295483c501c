"""Linear elasticity on the GPU (HOM_A_STIFFNESS) against the elasticity oracle.

Strain fields of nc = d (d + 1) / 2 Mandel components run through the same FFT passes as the
conductivity fields, with the compatibility projection onto symmetric gradients in the axis-0
pass (oracle/elastic.py states it). Operator applications are compared at 1e-12 relative,
iterates at fixed iteration counts at 1e-10, (A_H E, E) at 1e-10, iteration counts to
tolerance within one; the laminate closed form checks the whole GPU pipeline directly.
"""
import numpy as np
import pytest

import microstructure as ms
import oracle as O
from tests.test_oracle_elastic import backus_energy, random_stiffness_table

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402

EL = O.elastic
OP_TOL = 1e-12
IT_TOL = 1e-10
AH_TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def problem(N, aniso=False, idx16=False, h=0.6, seed=2):
    d = len(N)
    ph = ms.box_phase(N, h)
    if idx16:
        ph = ph.astype(np.uint16)
    if aniso:
        table = random_stiffness_table(2, d, seed=seed, scale=(1.0, 15.0))
    else:
        table = np.array([EL.isotropic_stiffness(1.0, 1.0, d), EL.isotropic_stiffness(12.0, 6.0, d)])
    C = EL.expand_stiffness(ph, table)
    return H.Problem(d, N, H.stiffness_material(ph, table)), EL.GaNiElastic(C, d), C


GRIDS = [(9, 7), (15, 15), (63, 45), (5, 7, 9), (15, 15, 15), (27, 25, 21), (45, 45, 45),
         (243, 5, 3), (3, 175, 5), (7, 5, 189)]


@pytest.mark.parametrize("N", GRIDS)
@pytest.mark.parametrize("op", ["affine", "linear", "project", "em"])
def test_elastic_operator_parity(N, op):
    d = len(N)
    P, sysn, C = problem(N, aniso=(op in ("linear", "em")))
    nc = EL.ncomp(d)
    x = ms.random_field((nc,) + N, 7)
    E = ms.random_field((nc,), 2)
    y = P.field()
    opc = {"affine": H.HOM_OP_AFFINE, "linear": H.HOM_OP_LINEAR, "project": H.HOM_OP_PROJECT,
           "em": H.HOM_OP_EM}[op]
    H.hom_apply(P.h, opc, E, to_dev(x), y)
    torch.cuda.synchronize()
    if op == "affine":
        ref = sysn.matvec(sysn.const(E) + x)
    elif op == "linear":
        ref = sysn.matvec(x)
    elif op == "project":
        ref = EL.project_strain(x, d)
    else:
        cA, CA = O.spectral_bounds(C, d)
        ref = sysn.em_project(O.apply_A(C, x) - np.sqrt(cA * CA) * x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()


@pytest.mark.parametrize("N", [(15, 13), (9, 7, 11)])
@pytest.mark.parametrize("solver", ["richardson", "cg", "chebyshev", "eyre_milton"])
def test_elastic_solvers_fixed_iterations(N, solver):
    d = len(N)
    P, sysn, C = problem(N, aniso=True, idx16=True)
    cA, CA = O.spectral_bounds(C, d)
    E = ms.random_field((EL.ncomp(d),), 3)
    k = 20
    x = P.field()
    stop = H.HOM_STOP_INCREMENT if solver in ("eyre_milton",) else H.HOM_STOP_RESIDUAL
    AH, _, st, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-6,
                               H.make_opts(fixed_iters=k, stop=stop), x)
    if solver == "richardson":
        ref = O.richardson(sysn, E, cA, CA, fixed_iters=k).x
    elif solver == "cg":
        ref = O.cg(sysn, E, fixed_iters=k).x
    elif solver == "chebyshev":
        ref = O.chebyshev(sysn, E, cA, CA, fixed_iters=k).x
    else:
        ref = EL.project_strain(O.eyre_milton(sysn, E, cA, CA, fixed_iters=k).x, d)
    assert rel(x.cpu().numpy(), ref) < IT_TOL
    assert abs(AH - sysn.energy(E, ref)) < AH_TOL * abs(AH)
    P.close()


@pytest.mark.parametrize("solver", ["richardson", "cg", "chebyshev", "eyre_milton"])
def test_elastic_solvers_to_tolerance(solver):
    N = (21, 19, 17)
    d = 3
    P, sysn, C = problem(N)
    cA, CA = O.spectral_bounds(C, d)
    E = np.array([0.3, -0.2, 0.5, 0.1, 0.4, -0.3])
    AH, flux, st, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-8)
    assert st["converged"]
    if solver == "richardson":
        r = O.richardson(sysn, E, cA, CA, tol=1e-8, stop="residual")
        x = r.x
    elif solver == "cg":
        r = O.cg(sysn, E, tol=1e-8)
        x = r.x
    elif solver == "chebyshev":
        r = O.chebyshev(sysn, E, cA, CA, tol=1e-8)
        x = r.x
    else:
        r = O.eyre_milton(sysn, E, cA, CA, tol=1e-8)
        x = EL.project_strain(r.x, d)
    assert abs(st["iterations"] - r.iterations) <= 1
    ref = sysn.energy(E, x)
    assert abs(AH - ref) < 1e-7 * ref
    # flux <C (E + e)> against the oracle's
    v = sysn.const(E) + x
    fl = np.mean(O.apply_A(C, v).reshape(6, -1), axis=1)
    np.testing.assert_allclose(flux, fl, rtol=1e-6, atol=1e-8)
    P.close()


@pytest.mark.parametrize("N", [(45, 7), (81, 5, 7)])
def test_elastic_laminate_closed_form(N):
    d = len(N)
    ph = ms.laminate_phase(N, 0.4, axis=0)
    lam, mu = [1.0, 30.0], [0.8, 12.0]
    table = np.array([EL.isotropic_stiffness(lam[p], mu[p], d) for p in range(2)])
    P = H.Problem(d, N, H.stiffness_material(ph, table))
    rng = np.random.default_rng(11)
    for E in list(np.eye(EL.ncomp(d))) + [rng.standard_normal(EL.ncomp(d))]:
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-12)
        ref = backus_energy(ph, lam, mu, E, d)
        assert abs(AH - ref) < AH_TOL * ref
    P.close()


def test_elastic_cube_81_cg_matches_oracle():
    N = (81, 81, 81)
    P, sysn, C = problem(N, h=ms.inclusion_side_for_fraction(0.2, 3))
    E = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    x = P.field()
    AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-6, H.make_opts(fixed_iters=6), x)
    ref = O.cg(sysn, E, fixed_iters=6).x
    assert rel(x.cpu().numpy(), ref) < IT_TOL
    assert abs(AH - sysn.energy(E, ref)) < AH_TOL * AH
    # Voigt at x = 0
    en0, _ = H.hom_energy(P.h, E, None)
    assert abs(en0 - sysn.energy(E, np.zeros_like(ref))) < 1e-13 * en0
    P.close()


def test_elastic_unsupported_combinations():
    N = (9, 9)
    ph = ms.box_phase(N, 0.6)
    table = np.array([EL.isotropic_stiffness(1.0, 1.0, 2), EL.isotropic_stiffness(5.0, 2.0, 2)])
    mat = H.stiffness_material(ph, table)
    for integ, prec in [(H.HOM_EXACT, H.HOM_FP64), (H.HOM_EXACT, H.HOM_FP32_REFINED)]:
        with pytest.raises(H.HomError) as ei:
            H.hom_create(2, N, mat, integ, prec)
        assert ei.value.status == H.HOM_ERR_UNSUPPORTED
    # prolongation and the GaNi bound take vector fields only
    Pe = H.Problem(2, N, mat)
    Pf = H.Problem(2, (17, 17), H.stiffness_material(ms.box_phase((17, 17), 0.6), table))
    y = Pf.field()
    with pytest.raises(H.HomError) as ei:
        H.hom_prolongate(Pe.h, Pf.h, Pe.field(), y)
    assert ei.value.status == H.HOM_ERR_UNSUPPORTED
    Pe.close()
    Pf.close()
    bad = table.copy()
    bad[1, 0, 1] += 1.0  # not symmetric
    with pytest.raises(H.HomError) as ei:
        H.hom_create(2, N, H.stiffness_material(ph, bad))
    assert ei.value.status == H.HOM_ERR_INVALID


def refined_problem(N, seed=2):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = random_stiffness_table(2, d, seed=seed, scale=(1.0, 15.0))
    C = EL.expand_stiffness(ph, table)
    P = H.Problem(d, N, H.stiffness_material(ph, table), precision=H.HOM_FP32_REFINED)
    return P, EL.GaNiElastic(C, d), C


@pytest.mark.parametrize("N", [(15, 13), (21, 19, 17), (45, 45, 45), (81, 27, 45)])
def test_elastic_fp32_operator(N):
    # the FP32 twin of the strain operator (runtime and specialised plans) against the oracle
    d = len(N)
    P, sysn, C = refined_problem(N)
    x = ms.random_field((EL.ncomp(d),) + N, 7)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, to_dev(x), y)
    torch.cuda.synchronize()
    assert rel(y.cpu().numpy(), sysn.matvec(x)) < 2e-6
    P.close()


@pytest.mark.parametrize("N", [(21, 19, 17), (45, 45, 45)])
@pytest.mark.parametrize("solver", ["cg", "chebyshev"])
def test_elastic_refined_solve_matches_fp64_oracle(N, solver):
    # FP32 inner solves (field form, six components) in FP64 refinement reach the FP64 oracle
    d = len(N)
    P, sysn, C = refined_problem(N, seed=5)
    E = np.array([0.3, -0.2, 0.5, 0.1, 0.4, -0.3])
    xr = O.cg(sysn, E, tol=1e-12).x
    ref = sysn.energy(E, xr)
    x = P.field()
    AH, _, st, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-10, None, x)
    assert st["converged"] and st["true_residual"] <= 1e-10
    assert abs(AH - ref) < 1e-8 * ref
    assert rel(x.cpu().numpy(), xr) < 1e-8
    P.close()


def test_elastic_batch_equals_solo():
    # two same-shape strain problems advanced by one launch per pass (hom_batch) end exactly
    # where their solo solves end
    N = (15, 13, 11)
    Es = [np.array([1.0, 0, 0, 0, 0, 0]), np.array([0.2, -0.1, 0.4, 0.3, 0.0, -0.5])]
    solo = []
    for E in Es:
        P, _, _ = problem(N, aniso=True)
        solo.append(H.hom_solve(P.h, E, H.HOM_CG, 1e-9)[0])
        P.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        probs = [problem(N, aniso=True)[0] for _ in Es]
        for P, E in zip(probs, Es):
            H.hom_solve_begin(P.h, E, H.HOM_CG, 1e-9, None)
        B = H.hom_batch_create([P.h for P in probs])
        for _ in range(500):
            if H.hom_batch_iterate(B, 8, use_graph=True, poll=True):
                break
        for P, ref in zip(probs, solo):
            AH, _, st, _ = H.hom_solve_end(P.h, 6)
            assert st["converged"] and AH == ref
        H.hom_batch_destroy(B)
        for P in probs:
            P.close()


@pytest.mark.parametrize("solver", ["cg", "chebyshev"])
def test_elastic_refined_batch_equals_solo(solver):
    # FP32-refined strain problems of one shape advanced together (hom_batch, graph replays)
    # end exactly where their solo solves end
    N = (45, 45, 45)
    Es = [np.array([1.0, 0, 0, 0, 0, 0]), np.array([0.2, -0.1, 0.4, 0.3, 0.0, -0.5])]
    solo = []
    for k, E in enumerate(Es):
        P, _, _ = refined_problem(N, seed=7 + k)
        solo.append(H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-9)[:3])
        P.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        probs = [refined_problem(N, seed=7 + k)[0] for k in range(len(Es))]
        for P, E in zip(probs, Es):
            H.hom_solve_begin(P.h, E, H.SOLVERS[solver], 1e-9, None)
        B = H.hom_batch_create([P.h for P in probs])
        for _ in range(1000):
            if H.hom_batch_iterate(B, 8, use_graph=True, poll=True):
                break
        for P, (AH, _, st) in zip(probs, solo):
            AHb, _, stb, _ = H.hom_solve_end(P.h, 6)
            assert stb["converged"] and AHb == AH
            assert stb["inner_iterations"] == st["inner_iterations"]
        H.hom_batch_destroy(B)
        for P in probs:
            P.close()


def test_server_serves_strain_problems_with_vector_ones():
    # stiffness requests (FP64 CG and Chebyshev, FP32-refined CG) in flight with a conductivity
    # request: each result equals its solo solve; E and the flux carry six entries
    N = (21, 19, 17)
    plan = []
    for k, (solver, prec) in enumerate([("cg", H.HOM_FP64), ("chebyshev", H.HOM_FP64),
                                         ("cg", H.HOM_FP32_REFINED), ("cg", H.HOM_FP64)]):
        ph = ms.box_phase(N, 0.6)
        table = random_stiffness_table(2, 3, seed=30 + k, scale=(1.0, 12.0))
        E = ms.random_field((6,), 40 + k)
        plan.append((H.stiffness_material(ph, table), E, solver, prec))
    phc = ms.box_phase(N, 0.5)
    conductivity = (H.phase_material(phc, ms.isotropic_table([1.0, 20.0], 3)),
                    np.array([1.0, 0.0, 0.0]), "cg", H.HOM_FP64)
    S = H.hom_server_create(1 << 30, max_batch=2)
    ids = {}
    for i, (mat, E, solver, prec) in enumerate(plan + [conductivity]):
        req = H.make_request(3, N, mat, E, H.SOLVERS[solver], 1e-9, precision=prec)
        ids[H.hom_server_submit(S, req)] = i
    results = {}
    for _ in range(20000):
        H.hom_server_step(S, 4)
        for r in H.hom_server_poll(S):
            results[r["id"]] = r
        if len(results) == len(ids):
            break
    H.hom_server_destroy(S)
    assert len(results) == len(ids)
    for rid, r in results.items():
        mat, E, solver, prec = (plan + [conductivity])[ids[rid]]
        assert r["status"] == H.HOM_OK
        P = H.Problem(3, N, mat, precision=prec)
        AH, flux, st, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-9)
        P.close()
        assert r["stats"]["iterations"] == st["iterations"]
        assert abs(r["AH_EE"] - AH) <= 1e-14 * abs(AH)
        nc = len(E)
        np.testing.assert_allclose(r["flux"][:nc], flux[:nc], rtol=1e-13, atol=1e-14)
