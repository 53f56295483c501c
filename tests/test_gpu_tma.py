"""The FP32 strided pass on tiles staged by the TMA unit (k_pair_strided_tma) against the oracle
and against the register-load kernel it replaces.

The TMA kernel runs when a problem's spectrum rows start on 16-byte boundaries (the half axis
(n_last + 1) / 2 even) and the axis has a compile-time two-stage plan of at most 256 points.
Each persistent CTA (three a SM) walks its column tiles with two buffers, so grids with more
than three tiles a CTA (135 x 45 x 243: 1080 tiles on axis 1) take every buffer and barrier
phase at least twice. The FP32 operator must match the FP64 oracle at FP32 accuracy, and the
register-load kernel (HOM_PAIR_TMA=0, in a child process) must give the same bits: both
kernels run the same butterflies on the same values in the same order.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import microstructure as ms
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EL = O.elastic


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def fp32_apply(N, seed=5):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    P = H.Problem(d, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    x = ms.random_field((d,) + N, seed)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    P.close()
    return ph, table, x, out


# (axis-1 plan, half axis): (15x9, 122) with 1080 tiles, (27x9, 32), (21x3, 14 ragged),
# (15x3, 32) with the two-line chain of the scalar projection on both column axes
@pytest.mark.parametrize("N", [(135, 45, 243), (45, 243, 63), (63, 63, 27), (45, 45, 63)])
def test_tma_strided_fp32_operator_matches_oracle(N):
    ph, table, x, y = fp32_apply(N)
    ref = O.GaNi(O.expand_phase(ph, table)[0, 0], 3).matvec(x)
    err = rel(y, ref)
    assert err < 2e-6, err


def test_tma_strided_elastic_axis0_pass():
    # six strain components: the axis-0 column passes around the strain projection run the plain
    # strided pass over 45 x 32 columns a plane (540 tiles of six components)
    N = (63, 45, 63)
    ph = ms.box_phase(N, 0.6)
    table = np.array([EL.isotropic_stiffness(1.0, 1.0, 3), EL.isotropic_stiffness(12.0, 6.0, 3)])
    P = H.Problem(3, N, H.stiffness_material(ph, table), precision=H.HOM_FP32_REFINED)
    x = ms.random_field((6,) + N, 7)
    y = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    ref = EL.GaNiElastic(EL.expand_stiffness(ph, table), 3).matvec(x)
    assert rel(y.cpu().numpy(), ref) < 2e-6
    P.close()


CHILD = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
from tests.test_gpu_tma import fp32_apply
np.save({out!r}, fp32_apply({N!r})[3])
"""


def test_tma_and_register_load_kernels_give_the_same_bits(tmp_path):
    N = (135, 45, 243)
    y_tma = fp32_apply(N)[3]
    out = str(tmp_path / "y_reg.npy")
    env = dict(os.environ, HOM_PAIR_TMA="0")
    subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, out=out, N=N)], env=env,
                   cwd=ROOT, check=True, timeout=600)
    y_reg = np.load(out)
    assert np.array_equal(y_tma, y_reg), float(np.max(np.abs(y_tma - y_reg)))


def test_tma_refined_solve_reaches_the_fp64_oracle():
    N = (45, 45, 63)
    ph, _, radii = ms.rsa_spheres(N, 3, rmin=0.08, rmax=0.15, vf=0.25)
    rng = np.random.default_rng(3)
    table = ms.isotropic_table(np.concatenate([[1.0], np.exp(rng.uniform(np.log(10), np.log(500), len(radii)))]), 3)
    E = np.array([0.3, 1.0, -0.2])
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], 3)
    xr = O.cg(sysn, E, tol=1e-12).x
    ref = sysn.energy(E, xr)
    for form in (0, 1):
        P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
        x = P.field()
        AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-10, H.make_opts(inner_form=form), x)
        assert st["converged"] and st["true_residual"] <= 1e-10
        assert abs(AH - ref) < 1e-8 * ref
        assert rel(x.cpu().numpy(), xr) < 1e-8
        P.close()


def test_tma_wait_that_runs_out_returns_timeout():
    # hom_debug_tma_stall announces 16 bytes more than each tile copy delivers: no barrier phase
    # completes, each wait gives up after ~1 s, the solve reports HOM_ERR_TIMEOUT, and the
    # context stays usable for the next solve (no fault, no hang)
    N = (45, 45, 63)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], 3)
    E = np.array([1.0, 0.0, 0.0])
    P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    H.hom_debug_tma_stall(1)
    try:
        with pytest.raises(H.HomError) as e:
            H.hom_solve(P.h, E, H.HOM_CG, 1e-6, H.make_opts(fixed_iters=1), P.field())
        assert e.value.status == H.HOM_ERR_TIMEOUT
    finally:
        H.hom_debug_tma_stall(0)
    P.close()
    ref = O.GaNi(O.expand_phase(ph, table)[0, 0], 3)
    xr = O.cg(ref, E, tol=1e-12).x
    P = H.Problem(3, N, H.phase_material(ph, table), precision=H.HOM_FP32_REFINED)
    x = P.field()
    AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-10, None, x)
    assert st["converged"] and abs(AH - ref.energy(E, xr)) < 1e-8 * abs(AH)
    P.close()
