"""FP32 operator inside FP64 iterative refinement (HOM_FP32_REFINED) vs the FP64 oracle.

The FP32 operator is compared at FP32 accuracy; the refined solves must reach A_H within the
mixed-precision bar (1e-8 relative) because the outer residual is formed in FP64.
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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def spheres(N, seed, contrast=(10.0, 1000.0)):
    d = len(N)
    ph, c, r = ms.rsa_spheres(N, seed, vf=0.3)
    rng = np.random.default_rng(seed + 100)
    vals = np.concatenate([[1.0], np.exp(rng.uniform(np.log(contrast[0]), np.log(contrast[1]), len(r)))])
    return ph, ms.isotropic_table(vals, d)


@pytest.mark.parametrize("N", [(63, 63), (27, 25, 21), (45, 45, 45)])
def test_fp32_operator_parity(N):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    P = H.Problem(d, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    x = ms.random_field((d,) + N, 4)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, torch.from_numpy(x).cuda(), y)
    ref = O.GaNi(O.expand_phase(ph, table)[0, 0], d).matvec(x)
    err = rel(y.cpu().numpy(), ref)
    assert err < 2e-6, err  # FP32 arithmetic, ~log2(N) stages of rounding
    P.close()


# axis lengths whose FP32 column passes run the compile-time two-stage kernels: each appears
# along axis 0 (projection pass) and along axis 1 (strided pass), with ragged column tiles
TWO_STAGE_GRIDS = [(243, 7, 5), (5, 243, 3), (405, 3, 3), (3, 405, 5), (81, 9, 5), (7, 81, 9),
                   (135, 5, 3), (3, 135, 7), (45, 11, 3), (161, 3, 5), (3, 161, 3), (63, 5, 3),
                   (3, 63, 7), (189, 3, 3), (5, 189, 3), (175, 3, 5), (3, 175, 3), (243, 7),
                   # both column axes specialised: the scalar projection's two-line chain
                   (63, 45, 5), (45, 243, 3), (243, 45, 3), (135, 81, 7), (175, 161, 3)]


@pytest.mark.parametrize("N", TWO_STAGE_GRIDS)
@pytest.mark.parametrize("op", ["linear", "em", "project"])
def test_fp32_two_stage_plans(N, op):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    A = O.expand_phase(ph, table)[0, 0]
    P = H.Problem(d, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    x = ms.random_field((d,) + N, 5)
    y = P.field()
    opc = {"linear": H.HOM_OP_LINEAR, "em": H.HOM_OP_EM, "project": H.HOM_OP_PROJECT}[op]
    H.hom_apply(P.h, opc | H.HOM_OP_FP32, None, torch.from_numpy(x).cuda(), y)
    sysn = O.GaNi(A, d)
    if op == "linear":
        ref = sysn.matvec(x)
    elif op == "em":
        ref = sysn.em_project(O.apply_A(A, x) - np.sqrt(10.0) * x)
    else:
        ref = O.project(x)
    err = rel(y.cpu().numpy(), ref)
    assert err < 2e-6, err
    P.close()


@pytest.mark.parametrize("N", [(81, 5, 3), (3, 81, 5), (81, 81, 3)])
def test_fp32_two_stage_plans_exact_integration(N):
    # double grid 2N - 1 = 161: the truncation to Z_N runs inside the specialised projection
    d = len(N)
    M = O.double_grid(N)
    Ahat = ms.box_fourier_coefficients(M, 0.6, 1.0, 10.0)
    P = H.Problem(d, N, H.fourier_material(Ahat.astype(np.complex128), 1.0, 10.0), H.HOM_EXACT,
                  precision=H.HOM_FP32_REFINED)
    assert P.grid == M
    A_M = O.ga_coefficients(Ahat, d)
    x = ms.random_field((d,) + M, 6)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, torch.from_numpy(x).cuda(), y)
    err = rel(y.cpu().numpy(), O.Ga(A_M, N, d).matvec(x))
    assert err < 2e-6, err
    P.close()


@pytest.mark.parametrize("solver", ["cg", "chebyshev"])
@pytest.mark.parametrize("N", [(85, 85), (33, 35, 31)])
def test_refined_solve_matches_fp64_oracle(N, solver):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 100.0], d)
    P = H.Problem(d, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    E = np.eye(d)[0]
    x = P.field()
    AH, flux, stats, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-10, None, x)
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], d)
    xr = O.cg(sysn, E, tol=1e-12).x
    ref = sysn.energy(E, xr)
    assert stats["converged"] and stats["true_residual"] <= 1e-10
    assert abs(AH - ref) < AH_TOL_MIXED * ref
    assert rel(x.cpu().numpy(), xr) < 1e-8
    assert stats["iterations"] <= 6  # outer FP64 residuals: FP32 inner solves to 1e-4 each
    P.close()


def test_refined_spheres_anisotropic_contrast():
    # the 405^3 workload's microstructure at 45^3: RSA spheres, log-uniform conductivities
    N = (45, 45, 45)
    ph, table = spheres(N, 7)
    P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    E = np.array([1.0, 0.0, 0.0])
    AH, _, stats, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-8, None, None)
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], 3)
    ref = sysn.energy(E, O.cg(sysn, E, tol=1e-11).x)
    assert abs(AH - ref) < AH_TOL_MIXED * ref
    P.close()


def test_refined_rejects_other_solvers():
    N = (9, 9)
    P = H.Problem(2, N, H.phase_material(ms.box_phase(N, 0.6), ms.isotropic_table([1.0, 10.0], 2)),
                  precision=H.HOM_FP32_REFINED)
    with pytest.raises(H.HomError) as ei:
        H.hom_solve(P.h, np.array([1.0, 0.0]), H.HOM_RICHARDSON, 1e-6)
    assert ei.value.status == H.HOM_ERR_UNSUPPORTED
    P.close()


@pytest.mark.parametrize("kind", ["iso8_vector", "iso8_many", "iso16", "tensor", "field"])
def test_fp32_line_pass_material_branches(kind):
    # the specialised FP32 line pass streams 16-byte vectors for isotropic one-byte phase images
    # with at most 64 phases and takes the node-by-node pre-operator otherwise: every branch
    # against the oracle, on a grid whose contiguous axis has a compile-time plan (81 = 27 x 3)
    N = (9, 11, 81)
    d = 3
    rng = np.random.default_rng(17)
    nph = {"iso8_vector": 40, "iso8_many": 100, "iso16": 300, "tensor": 5, "field": 0}[kind]
    if kind == "field":
        a = rng.uniform(1.0, 30.0, N)
        mat, A = H.scalar_material(a), a
    else:
        ph = rng.integers(0, nph, size=N).astype(np.uint16 if kind == "iso16" else np.uint8)
        if kind == "tensor":
            table = ms.random_spd_table(nph, d, seed=3, scales=np.linspace(1.0, 20.0, nph))
            A = O.expand_phase(ph, table)
        else:
            table = ms.isotropic_table(rng.uniform(1.0, 30.0, nph), d)
            A = O.expand_phase(ph, table)[0, 0]
        mat = H.phase_material(ph, table)
    P = H.Problem(d, N, mat, precision=H.HOM_FP32_REFINED)
    x = ms.random_field((d,) + N, 8)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, torch.from_numpy(x).cuda(), y)
    err = rel(y.cpu().numpy(), O.GaNi(A, d).matvec(x))
    assert err < 2e-6, err
    # the fused CG step of the refined solve on the same material reaches the FP64 A_H
    E = np.array([0.0, 0.0, 1.0])
    AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-10)
    sysn = O.GaNi(A, d)
    ref = sysn.energy(E, O.cg(sysn, E, tol=1e-11).x)
    assert st["converged"] and abs(AH - ref) < AH_TOL_MIXED * ref
    P.close()
