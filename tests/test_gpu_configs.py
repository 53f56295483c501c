"""The exact-integration workload at 3-D size: trigonometric order 81^3 on the double grid
161^3 = 7 * 23 (radix-23 stage), cubic inclusion of volume fraction 0.3, contrast 100."""
import numpy as np
import pytest

import microstructure as ms
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402


def ga(N, h, lo, hi, M=None):
    Mg = tuple(M) if M is not None else O.double_grid(N)
    Ahat = ms.box_fourier_coefficients(Mg, h, lo, hi)
    return H.Problem(3, N, H.fourier_material(Ahat.astype(np.complex128), lo, hi, M), H.HOM_EXACT), Ahat, Mg


def test_ga_operator_parity_161():
    N = (81, 81, 81)
    h = ms.inclusion_side_for_fraction(0.3, 3)
    P, Ahat, M = ga(N, h, 1.0, 100.0)
    assert P.grid == (161, 161, 161)
    x = ms.random_field((3,) + M, 5)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR, None, torch.from_numpy(x).cuda(), y)
    ref = O.Ga(O.ga_coefficients(Ahat, 3), N, 3).matvec(x)
    err = float(np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref))
    assert err < 1e-12
    P.close()


def test_exact_integration_bound_ordering_81():
    # eq. (bounds): A_H <= A_{H,N} (Ga) <= GaNi guaranteed bound; Hashin-Shtrikman lower bound
    # of the two-phase isotropic composite below the true A_H
    N = (81, 81, 81)
    vf = 0.3
    h = ms.inclusion_side_for_fraction(vf, 3)
    E = np.array([1.0, 0.0, 0.0])
    ph = ms.box_phase(N, h)
    Pn = H.Problem(3, N, H.phase_material(ph, ms.isotropic_table([1.0, 100.0], 3)))
    xn = Pn.field()
    AH_gani, _, st_n, _ = H.hom_solve(Pn.h, E, H.HOM_CG, 1e-8, None, xn)
    Pg, _, _ = ga(N, h, 1.0, 100.0)
    bound = H.hom_bound(Pn.h, Pg.h, E, xn)
    AH_ga, _, st_g, _ = H.hom_solve(Pg.h, E, H.HOM_CG, 1e-8, None, None)
    Pg2, _, _ = ga(N, h, 1.0, 100.0, M=(175, 175, 175))  # any odd M >= 2N - 1 is exact
    AH_ga175, _, _, _ = H.hom_solve(Pg2.h, E, H.HOM_CG, 1e-8, None, None)
    a1, a2, f2 = 1.0, 100.0, vf
    hs = a1 + f2 / (1.0 / (a2 - a1) + (1 - f2) / (3 * a1))
    assert st_n["converged"] and st_g["converged"]
    assert hs < AH_ga < bound
    assert abs(AH_ga - AH_ga175) < 1e-7 * AH_ga
    for P in (Pn, Pg, Pg2):
        P.close()
