"""Snapshot and restore of an FP64 solve session: a solve preempted after some iterations and
restored into a problem created the same way continues bit for bit (iterate, A_H and the
per-iteration history equal those of the uninterrupted solve), for each of the four solvers of
Algorithms 1-4; restoring into a session of another solver, or snapshotting an FP32-refined
session, is refused."""
import numpy as np
import pytest

import microstructure as ms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402

N = (27, 27, 27)
E = np.array([0.3, -0.5, 0.8])
ITERS = 20    # fixed iterations of each solve
CUT = 8       # the snapshot is taken after this many


def problem():
    ph = ms.box_phase(N, 0.6)
    return H.Problem(3, N, H.phase_material(ph, ms.isotropic_table([1.0, 50.0], 3)))


def finish(P):
    x = P.field()
    H.hom_solve_iterate(P.h, ITERS + 2)
    AH, _, st, _ = H.hom_solve_end(P.h, 3, x)
    return x, AH, st, H.hom_solve_history(P.h)


@pytest.mark.parametrize("solver", list(H.SOLVERS))
def test_restored_session_continues_bit_for_bit(solver):
    opts = H.make_opts(fixed_iters=ITERS)
    A = problem()
    H.hom_solve_begin(A.h, E, H.SOLVERS[solver], 0.0, opts)
    H.hom_solve_iterate(A.h, CUT)
    snap = H.hom_solve_snapshot(A.h)
    x_a, AH_a, st_a, hist_a = finish(A)
    A.close()

    B = problem()
    H.hom_solve_begin(B.h, E, H.SOLVERS[solver], 0.0, opts)
    H.hom_solve_restore(B.h, snap)
    x_b, AH_b, st_b, hist_b = finish(B)
    B.close()

    assert torch.equal(x_a, x_b)
    assert AH_a == AH_b
    assert st_a["iterations"] == st_b["iterations"] == ITERS
    assert np.array_equal(hist_a, hist_b)


def test_restore_refuses_another_session():
    opts = H.make_opts(fixed_iters=ITERS)
    A = problem()
    H.hom_solve_begin(A.h, E, H.HOM_CG, 0.0, opts)
    H.hom_solve_iterate(A.h, CUT)
    snap = H.hom_solve_snapshot(A.h)
    H.hom_solve_end(A.h, 3, allow_not_converged=True)
    # another solver, another macroscopic field, a truncated buffer
    for solver, E2, buf in ((H.HOM_CHEBYSHEV, E, snap), (H.HOM_CG, -E, snap),
                            (H.HOM_CG, E, snap[:100])):
        H.hom_solve_begin(A.h, E2, solver, 0.0, opts)
        with pytest.raises(H.HomError) as ei:
            H.hom_solve_restore(A.h, buf)
        assert ei.value.status == H.HOM_ERR_INVALID
        H.hom_solve_end(A.h, 3, allow_not_converged=True)
    A.close()
    # an FP32-refined session has no snapshot
    ph = ms.box_phase(N, 0.6)
    R = H.Problem(3, N, H.phase_material(ph, ms.isotropic_table([1.0, 50.0], 3)),
                  precision=H.HOM_FP32_REFINED)
    H.hom_solve_begin(R.h, E, H.HOM_CG, 1e-8)
    with pytest.raises(H.HomError) as ei:
        H.hom_solve_snapshot(R.h)
    assert ei.value.status == H.HOM_ERR_UNSUPPORTED
    H.hom_solve_end(R.h, 3, allow_not_converged=True)
    R.close()
