"""FP64 operator and solver parity on axes whose FP64 radix plan has three Stockham stages.

FP64 plans group the prime factors of an axis into register radices of at most 15, so the
axis lengths 243 = [9, 9, 3], 405 = [15, 9, 3], 189 = [9, 7, 3] and 175 = [7, 5, 5] run a
first stage, a twiddled shared-memory-to-shared-memory middle stage and a last stage. Each
length is placed on every axis (contiguous axis: line passes; middle axis: strided pass;
axis 0: projection pass), in 2-D and 3-D, and compared with the oracle at the operator
tolerance of eq. (linsys) parity (1e-12 relative per application). The 243^3 cube of volume
fraction 0.2 and contrast 1e3 is the benchmarked workload: one full application and three
fixed CG iterations (Algorithm 2) are compared at full size. Plans with radices up to 27
(set with hom_set_plan) are compared on axes 27, 81, 243 and 729.
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

OP_TOL = 1e-12   # one operator application, relative 2-norm
IT_TOL = 1e-10   # iterates after a fixed number of iterations
AH_TOL = 1e-10   # (A_H E, E)

THREE_STAGE = [(243, 7, 5), (5, 243, 3), (3, 5, 243), (405, 3, 3), (3, 405, 5), (5, 3, 405),
               (189, 3, 5), (7, 189, 3), (3, 5, 189), (175, 5, 3), (3, 175, 5), (5, 3, 175),
               (243, 5), (7, 243), (405, 3), (3, 175)]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


OPS = {"affine": H.HOM_OP_AFFINE, "linear": H.HOM_OP_LINEAR, "project": H.HOM_OP_PROJECT,
       "em": H.HOM_OP_EM}


@pytest.mark.parametrize("N", THREE_STAGE)
@pytest.mark.parametrize("op", list(OPS))
def test_three_stage_operator_parity(N, op):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    A = O.expand_phase(ph, table)[0, 0]
    P = H.Problem(d, N, H.phase_material(ph, table))
    x = ms.random_field((d,) + N, 11)
    E = ms.random_unit_vector(d, 4)
    y = P.field()
    H.hom_apply(P.h, OPS[op], E, to_dev(x), y)
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


@pytest.mark.parametrize("N", [(243, 5, 3), (3, 7, 405), (5, 175, 3)])
def test_three_stage_anisotropic_parity(N):
    # tensor-valued phases (random rotations of diagonal SPD tensors), uint16 indices
    d = len(N)
    ph = ms.box_phase(N, 0.5).astype(np.uint16)
    table = ms.random_spd_table(2, d, seed=6, scales=[1.0, 40.0])
    A = O.expand_phase(ph, table)
    P = H.Problem(d, N, H.phase_material(ph, table))
    x = ms.random_field((d,) + N, 12)
    E = ms.random_unit_vector(d, 8)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_AFFINE, E, to_dev(x), y)
    sysn = O.GaNi(A, d)
    assert rel(y.cpu().numpy(), sysn.matvec(sysn.const(E) + x)) < OP_TOL
    cA, CA = O.spectral_bounds(A, d)
    H.hom_apply(P.h, H.HOM_OP_EM, None, to_dev(x), y)
    ref = sysn.em_project(O.apply_A(A, x) - np.sqrt(cA * CA) * x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()


@pytest.mark.parametrize("N,M", [((81, 81, 81), (175, 175, 175)), ((81, 3, 3), (175, 5, 5)),
                                 ((3, 81, 3), (5, 175, 5)), ((3, 3, 81), (7, 5, 175))])
def test_ga_operator_parity_on_175(N, M):
    # exact integration on the double grid M = 175 = 7 * 5 * 5 (three FP64 stages), any odd
    # M >= 2N - 1 being exact (eq. (Ga_exact_integration))
    d = len(N)
    h = ms.inclusion_side_for_fraction(0.3, 3)
    Ahat = ms.box_fourier_coefficients(M, h, 1.0, 100.0)
    P = H.Problem(d, N, H.fourier_material(Ahat.astype(np.complex128), 1.0, 100.0, M),
                  H.HOM_EXACT)
    assert P.grid == tuple(M)
    x = ms.random_field((d,) + tuple(M), 13)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    ref = O.Ga(O.ga_coefficients(Ahat, d), N, d).matvec(x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()


def bench_workload():
    """243^3, centred cube of volume fraction 0.2 (143^3 nodes), contrast 1e3, E = e_1."""
    N = (243, 243, 243)
    h = ms.inclusion_side_for_fraction(0.2, 3)
    ph = ms.box_phase(N, h)
    table = ms.isotropic_table([1.0, 1000.0], 3)
    return N, ph, table


def test_full_243_cubed_application():
    N, ph, table = bench_workload()
    A = O.expand_phase(ph, table)[0, 0]
    P = H.Problem(3, N, H.phase_material(ph, table))
    x = ms.random_field((3,) + N, 21)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    ref = O.GaNi(A, 3).matvec(x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()


def test_cg_three_fixed_iterations_243_cubed():
    # the benchmarked CG step (fused vector update, FP64 partials) against Algorithm 2 as
    # printed, iterate by iterate
    N, ph, table = bench_workload()
    A = O.expand_phase(ph, table)[0, 0]
    E = np.array([1.0, 0.0, 0.0])
    P = H.Problem(3, N, H.phase_material(ph, table))
    x = P.field()
    AH, _, stats, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-6, H.make_opts(fixed_iters=3), x)
    assert stats["iterations"] == 3
    sysn = O.GaNi(A, 3)
    ref = O.cg(sysn, E, fixed_iters=3)
    assert rel(x.cpu().numpy(), ref.x) < IT_TOL
    hist = H.hom_solve_history(P.h)
    assert np.allclose(hist, ref.history, rtol=1e-9, atol=0)
    assert abs(AH - sysn.energy(E, ref.x)) < AH_TOL * abs(AH)
    P.close()


PLAN27 = {"rmax64": 27, "smem_kb64": 110, "threads64": 256, "rmax32": 27, "smem_kb32": 110,
          "threads32": 256, "two_line32": 1}


@pytest.mark.parametrize("N", [(81, 5, 3), (3, 243, 5), (5, 3, 27), (27, 81), (3, 729)])
@pytest.mark.parametrize("op", ["linear", "em"])
def test_radix27_fp64_plans(N, op):
    # FP64 plans with register radices up to 27 (81 = [27, 3], 243 = [27, 9], 27 = [27],
    # 729 = [27, 27]): the untwiddled 27-point DFT split 3 x 9 with its internal twiddles
    # factored into the 9-point rows, and behind it twiddled radices 3, 9 and 27
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    A = O.expand_phase(ph, table)[0, 0]
    P = H.Problem(d, N, H.phase_material(ph, table))
    H.hom_set_plan(P.h, PLAN27)
    x = ms.random_field((d,) + N, 13)
    y = P.field()
    H.hom_apply(P.h, OPS[op], None, to_dev(x), y)
    sysn = O.GaNi(A, d)
    if op == "linear":
        ref = sysn.matvec(x)
    else:
        ref = sysn.em_project(O.apply_A(A, x) - np.sqrt(10.0) * x)
    assert rel(y.cpu().numpy(), ref) < OP_TOL
    P.close()
