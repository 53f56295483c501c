"""Launch plans change rounding order at most: hom_set_plan with other register-radix limits,
tile budgets and thread counts gives the same FP64 operator to rounding, and the FP32 two- and
three-line chains of the 3-D scalar projection the same refined solve; invalid plans are
refused."""
import numpy as np
import pytest

import microstructure as ms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402

BASE = {"rmax64": 15, "smem_kb64": 110, "threads64": 256, "rmax32": 27, "smem_kb32": 110,
        "threads32": 256, "two_line32": 1}


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("N", [(45, 45, 45), (81, 63, 135)])
def test_plans_agree(N):
    ph = ms.box_phase(N, 0.6)
    P = H.Problem(3, N, H.phase_material(ph, ms.isotropic_table([1.0, 30.0], 3)),
                  precision=H.HOM_FP32_REFINED)
    x = torch.from_numpy(ms.random_field((3,) + N, 4)).cuda()
    E = np.array([0.0, 0.0, 1.0])
    ref_y, ref_AH = None, None
    for plan in (BASE, dict(BASE, rmax64=9, smem_kb64=56, threads64=128, two_line32=0),
                 dict(BASE, smem_kb64=200, rmax32=15, smem_kb32=150, threads32=128)):
        H.hom_set_plan(P.h, plan)
        y = P.field()
        H.hom_apply(P.h, H.HOM_OP_LINEAR, None, x, y)
        AH = H.hom_solve(P.h, E, H.HOM_CG, 1e-10)[0]
        if ref_y is None:
            ref_y, ref_AH = y, AH
        assert rel(y, ref_y) < 1e-13
        assert abs(AH - ref_AH) < 1e-9 * ref_AH
    P.close()


def test_invalid_plans_are_refused():
    N = (15, 15, 15)
    P = H.Problem(3, N, H.phase_material(ms.box_phase(N, 0.6), ms.isotropic_table([1.0, 3.0], 3)))
    for bad in ({"rmax64": 1}, {"smem_kb64": 0}, {"threads64": 100}, {"smem_kb64": 100000}):
        with pytest.raises(H.HomError) as ei:
            H.hom_set_plan(P.h, dict(BASE, **bad))
        assert ei.value.status == H.HOM_ERR_INVALID
    H.hom_set_plan(P.h, dict(BASE, rmax64=9))
    AH, _, st, _ = H.hom_solve(P.h, np.array([1.0, 0.0, 0.0]), H.HOM_CG, 1e-9)
    assert st["converged"]
    P.close()
