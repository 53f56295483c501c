"""Exact integration (Ga) of voxel images through the C ABI: the coefficients
A^(n) = prod sinc(pi n_a / N_a) (F_N a)(n mod N) assembled on the device against the oracle's
voxel_fourier_coefficients, the operator and the solves, the analytic box as a special case,
and the bound ordering of Section 2.2 on a random-sphere image."""
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


def random_image(N, nphase, seed):
    rng = np.random.default_rng(seed)
    ph = rng.integers(0, nphase, size=N).astype(np.uint8)
    values = np.exp(rng.uniform(0.0, np.log(50.0), nphase))
    return ph, values


@pytest.mark.parametrize("N,M", [((9, 7), None), ((7, 9, 5), None), ((5, 7), (11, 15)),
                                 ((9, 9, 9), None)])
def test_voxel_operator_parity(N, M):
    d = len(N)
    ph, values = random_image(N, 4, 7)
    Mg = tuple(M) if M is not None else O.double_grid(N)
    P = H.Problem(d, N, H.phase_material(ph, ms.isotropic_table(values, d), M=M), H.HOM_EXACT)
    assert P.grid == Mg
    A_M = O.ga_coefficients(O.voxel_fourier_coefficients(values[ph], Mg), d)
    x = ms.random_field((d,) + Mg, 11)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, to_dev(x), y)
    assert rel(y.cpu().numpy(), O.Ga(A_M, N, d).matvec(x)) < OP_TOL
    # the double-grid mean of A_M is the exact integral of the image: its voxel mean
    E = np.eye(d)[0]
    en, _ = H.hom_energy(P.h, E)
    assert abs(en - values[ph].mean()) < 1e-12 * en
    P.close()


@pytest.mark.parametrize("N", [(15, 13), (9, 7, 11)])
def test_voxel_solve_parity_phase_and_scalar(N):
    d = len(N)
    ph, values = random_image(N, 3, 5)
    a = values[ph]
    M = O.double_grid(N)
    sysg = O.Ga(O.ga_coefficients(O.voxel_fourier_coefficients(a, M), d), N, d)
    E = np.eye(d)[0]
    ref = sysg.energy(E, O.cg(sysg, E, tol=1e-10).x)
    for mat in (H.phase_material(ph, ms.isotropic_table(values, d)), H.scalar_material(a)):
        P = H.Problem(d, N, mat, H.HOM_EXACT)
        assert H.hom_bounds(P.h) == (a.min(), a.max())
        AH, _, _, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-10)
        assert abs(AH - ref) < AH_TOL * ref
        P.close()


def test_whole_voxel_box_equals_analytic_coefficients():
    # 15^2 with h = 0.6: the box is 9 x 9 voxels, so the image and the analytic box define the
    # same coefficient and the two Ga problems the same A_H
    N = (15, 15)
    M = O.double_grid(N)
    Pv = H.Problem(2, N, H.phase_material(ms.box_phase(N, 0.6), ms.isotropic_table([1.0, 100.0], 2)),
                   H.HOM_EXACT)
    Pa = H.Problem(2, N, H.fourier_material(ms.box_fourier_coefficients(M, 0.6, 1.0, 100.0)
                                            .astype(np.complex128), 1.0, 100.0, M), H.HOM_EXACT)
    E = np.array([1.0, 0.0])
    AHv, _, _, _ = H.hom_solve(Pv.h, E, H.HOM_CG, 1e-10)
    AHa, _, _, _ = H.hom_solve(Pa.h, E, H.HOM_CG, 1e-10)
    assert abs(AHv - AHa) < 1e-10 * AHa
    Pv.close()
    Pa.close()


def test_random_spheres_bound_ordering():
    # Section 2.2: the Ga value of an image lies below the guaranteed bound of the GaNi solution
    # prolonged to the double grid, and above the Reuss (harmonic mean) value; 3-D RSA spheres
    N = (23, 23, 23)
    ph, _, radii = ms.rsa_spheres(N, 3, rmin=0.1, rmax=0.2, vf=0.25)
    values = np.concatenate([[1.0], np.full(len(radii), 100.0)])
    table = ms.isotropic_table(values, 3)
    Pn = H.Problem(3, N, H.phase_material(ph, table))
    Pg = H.Problem(3, N, H.phase_material(ph, table), H.HOM_EXACT)
    E = np.array([1.0, 0.0, 0.0])
    xn = Pn.field()
    AHn, _, _, _ = H.hom_solve(Pn.h, E, H.HOM_CG, 1e-10, None, xn)
    ub = H.hom_bound(Pn.h, Pg.h, E, xn)
    AHg, _, _, _ = H.hom_solve(Pg.h, E, H.HOM_CG, 1e-10)
    a = values[ph.astype(np.int64)]
    reuss = 1.0 / np.mean(1.0 / a)
    assert reuss < AHg < ub
    assert AHg < a.mean()  # Voigt
    # the bound agrees with the oracle's: GaNi iterate prolonged, energy with the voxel A_M
    M = O.double_grid(N)
    A_M = O.ga_coefficients(O.voxel_fourier_coefficients(a, M), 3)
    sysn = O.GaNi(a, 3)
    ub_ref = O.energy(A_M, O.prolongate(sysn.const(E) + xn.cpu().numpy(), M))
    assert abs(ub - ub_ref) < 1e-10 * ub_ref
    Pn.close()
    Pg.close()


def test_voxel_ga_refined_matches_fp64():
    # the FP32 operator of an exactly integrated image inside FP64 refinement reaches the FP64
    # A_H (1e-8, the mixed-precision bar)
    N = (15, 13, 11)
    ph, values = random_image(N, 3, 9)
    table = ms.isotropic_table(values, 3)
    E = np.array([0.0, 1.0, 0.0])
    P64 = H.Problem(3, N, H.phase_material(ph, table), H.HOM_EXACT)
    P32 = H.Problem(3, N, H.phase_material(ph, table), H.HOM_EXACT, precision=H.HOM_FP32_REFINED)
    AH64, _, _, _ = H.hom_solve(P64.h, E, H.HOM_CG, 1e-11)
    AH32, _, st, _ = H.hom_solve(P32.h, E, H.HOM_CG, 1e-11)
    assert st["converged"]
    assert abs(AH32 - AH64) < 1e-8 * AH64
    P64.close()
    P32.close()
