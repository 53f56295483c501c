"""The FP32 inner CG of the refinement in potential coordinates (pcg_pot.cuh) against the FP64
oracle and against the field form.

Algorithm 2 on C = G A (field form) and CG on K = D* A D preconditioned by the Laplacian
(potential form, x = D u) produce the same iterates in exact arithmetic, so both inner forms
must bring the refined solve to the FP64 oracle's A_H (1e-8) and corrector (1e-8), with inner
iteration totals that differ only by FP32 rounding; batched refined CG must equal the solo
solve bit for bit in the potential form too.
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

AH_TOL_MIXED = 1e-8


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def spheres(N, seed, vf=0.25):
    ph, _, radii = ms.rsa_spheres(N, seed, rmin=0.08, rmax=0.15, vf=vf)
    rng = np.random.default_rng(seed)
    table = ms.isotropic_table(np.concatenate([[1.0], np.exp(rng.uniform(np.log(10), np.log(500), len(radii)))]), 3)
    return ph, table


@pytest.mark.parametrize("N", [(45, 45, 45), (81, 63, 45), (63, 45, 81)])
def test_potential_inner_cg_reaches_the_fp64_oracle(N):
    ph, table = spheres(N, 3)
    E = np.array([0.3, 1.0, -0.2])
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], 3)
    xr = O.cg(sysn, E, tol=1e-12).x
    ref = sysn.energy(E, xr)
    res = {}
    for form in (0, 1):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
        x = P.field()
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-10, H.make_opts(inner_form=form), x)
        assert st["converged"] and st["true_residual"] <= 1e-10
        assert abs(AH - ref) < AH_TOL_MIXED * ref
        assert rel(x.cpu().numpy(), xr) < 1e-8
        res[form] = st
        P.close()
    # the same iteration in exact arithmetic: the inner totals agree up to FP32 rounding
    a, b = res[0]["inner_iterations"], res[1]["inner_iterations"]
    assert abs(a - b) <= max(3, 0.1 * b), (a, b)


@pytest.mark.parametrize("N", [(45, 45, 45), (81, 63, 45)])
def test_potential_inner_chebyshev_reaches_the_fp64_oracle(N):
    # Algorithm 3 on M^{-1} K with the bounds [c_A, C_A] of A: the field-form iteration on G A
    # in exact arithmetic, so both inner forms reach the oracle, in about as many inner steps
    ph, table = spheres(N, 4)
    E = np.array([0.5, -0.4, 0.7])
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], 3)
    xr = O.cg(sysn, E, tol=1e-12).x
    ref = sysn.energy(E, xr)
    res = {}
    for form in (0, 1):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
        x = P.field()
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CHEBYSHEV, 1e-10, H.make_opts(inner_form=form), x)
        assert st["converged"] and st["true_residual"] <= 1e-10
        assert abs(AH - ref) < AH_TOL_MIXED * ref
        assert rel(x.cpu().numpy(), xr) < 1e-8
        res[form] = st["inner_iterations"]
        P.close()
    assert abs(res[0] - res[1]) <= max(3, 0.1 * res[1]), res


@pytest.mark.parametrize("solver", [H.HOM_CG, H.HOM_CHEBYSHEV])
def test_potential_batch_of_both_solvers_equals_solo(solver):
    N = (45, 63, 81)
    mats = [spheres(N, s) for s in (8, 9, 10)]
    Es = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.6, 0.8]), np.array([0.3, 0.3, -0.9])]
    solo = []
    for (ph, table), E in zip(mats, Es):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
        solo.append(H.hom_solve(P.h, E, solver, 1e-9)[:3])
        P.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        probs = [H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
                 for ph, table in mats]
        for P, E in zip(probs, Es):
            H.hom_solve_begin(P.h, E, solver, 1e-9, None)
        B = H.hom_batch_create([P.h for P in probs])
        for _ in range(1000):
            if H.hom_batch_iterate(B, 8, use_graph=True, poll=True):
                break
        for P, (AH, _, st) in zip(probs, solo):
            AHb, _, stb, _ = H.hom_solve_end(P.h, 3)
            assert stb["converged"] and AHb == AH
            assert stb["inner_iterations"] == st["inner_iterations"]
        H.hom_batch_destroy(B)
        for P in probs:
            P.close()


@pytest.mark.parametrize("solver", ["cg", "chebyshev"])
@pytest.mark.parametrize("form", [0, 1])
def test_fp32_inner_iterates_follow_the_algorithms(solver, form):
    # one inner solve of exactly k FP32 steps from zero (fixed_iters) is Algorithm 2 or 3 run
    # k steps on C x = b: the iterate of the FP64 oracle at k steps, up to FP32 rounding
    N = (45, 63, 81)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 30.0], 3)
    E = np.array([0.2, 0.9, -0.4])
    A = O.expand_phase(ph, table)[0, 0]
    sysn = O.GaNi(A, 3)
    cA, CA = O.spectral_bounds(A, 3)
    for k in (1, 4, 12):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
        x = P.field()
        AH, _, st, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 0.0,
                                   H.make_opts(fixed_iters=k, inner_form=form), x)
        assert st["iterations"] == 1 and st["inner_iterations"] == k
        if solver == "cg":
            ref = O.cg(sysn, E, fixed_iters=k).x
        else:
            ref = O.chebyshev(sysn, E, cA, CA, fixed_iters=k).x
        assert rel(x.cpu().numpy(), ref) < 2e-5, (k, rel(x.cpu().numpy(), ref))
        P.close()


@pytest.mark.parametrize("N", [(161, 45, 63), (175, 63, 45), (189, 45, 81), (135, 81, 45),
                               (405, 45, 45), (45, 45, 243), (45, 45, 405), (45, 63, 175),
                               (63, 45, 189), (45, 45, 161), (45, 81, 135)])
def test_potential_inner_iterates_on_every_specialised_plan(N):
    # the nine two-stage FP32 plans (27x9, 27x15, 27x3, 15x9, 15x3, 23x7, 21x3, 21x9, 25x7) on
    # axis 0 and on the contiguous axis, and the plans of 45, 63 and 81 on axis 1: four inner
    # CG steps in potential coordinates against the oracle's Algorithm 2 after four steps
    ph, table = spheres(N, 12, vf=0.2)
    E = np.array([0.6, -0.3, 0.74])
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], 3)
    P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    x = P.field()
    H.hom_solve(P.h, E, H.HOM_CG, 0.0, H.make_opts(fixed_iters=4), x)
    ref = O.cg(sysn, E, fixed_iters=4).x
    assert rel(x.cpu().numpy(), ref) < 2e-5
    P.close()


@pytest.mark.parametrize("N", [(23, 23, 23), (41, 23, 23)])
def test_potential_inner_cg_exact_integration(N):
    # Ga on the double grid 2N - 1 (45, 81: specialised plans on every axis): the preconditioner
    # keeps the directions inside Z_N, and the refined solve reaches the FP64 Ga oracle
    M = O.double_grid(N)
    Ahat = ms.box_fourier_coefficients(M, 0.6, 1.0, 50.0)
    sysg = O.Ga(O.ga_coefficients(Ahat, 3), N, 3)
    E = np.array([0.2, 1.0, -0.4])
    xr = O.cg(sysg, E, tol=1e-12).x
    ref = sysg.energy(E, xr)
    for form in (0, 1):
        P = H.Problem(3, N, H.fourier_material(Ahat.astype(np.complex128), 1.0, 50.0), H.HOM_EXACT,
                      precision=H.HOM_FP32_REFINED)
        assert P.grid == M
        x = P.field()
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-10, H.make_opts(inner_form=form), x)
        assert st["converged"]
        assert abs(AH - ref) < AH_TOL_MIXED * ref
        assert rel(x.cpu().numpy(), xr) < 1e-8
        P.close()


def test_potential_form_needs_specialised_plans_everywhere():
    # (33, 35, 31): no specialised FP32 plan on the contiguous axis, so the field form runs
    # (the results stay those of the FP64 oracle either way)
    N = (33, 35, 31)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 100.0], 3)
    P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    E = np.array([1.0, 0.0, 0.0])
    a = H.hom_solve(P.h, E, H.HOM_CG, 1e-10, H.make_opts(inner_form=0))
    b = H.hom_solve(P.h, E, H.HOM_CG, 1e-10, H.make_opts(inner_form=1))
    assert a[0] == b[0] and a[2]["inner_iterations"] == b[2]["inner_iterations"]
    P.close()


def test_potential_batch_equals_solo():
    N = (45, 45, 45)
    mats = [spheres(N, s) for s in (5, 6)]
    Es = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.6, 0.8])]
    solo = []
    for (ph, table), E in zip(mats, Es):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
        solo.append(H.hom_solve(P.h, E, H.HOM_CG, 1e-9)[:3])
        P.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        probs = [H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
                 for ph, table in mats]
        for P, E in zip(probs, Es):
            H.hom_solve_begin(P.h, E, H.HOM_CG, 1e-9, None)
        B = H.hom_batch_create([P.h for P in probs])
        for _ in range(500):
            if H.hom_batch_iterate(B, 8, use_graph=True, poll=True):
                break
        for P, (AH, _, st) in zip(probs, solo):
            AHb, _, stb, _ = H.hom_solve_end(P.h, 3)
            assert stb["converged"] and AHb == AH
            assert stb["inner_iterations"] == st["inner_iterations"]
        H.hom_batch_destroy(B)
        for P in probs:
            P.close()
