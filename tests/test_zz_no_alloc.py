"""hom_apply_static: the operator for callers that cannot allocate device memory.

Such callers (an application that owns all device memory through its own allocator or a fixed
budget, or a latency-critical loop that cannot afford the device synchronisation of
cudaMalloc/cudaFree) get the same operator as hom_apply, with the work memory in a static
device array of the library. This file runs last so that a failure here leaves every other
test already run; it must also pass on its own in a fresh process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import microstructure as ms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402

OP_TOL = 1e-12  # the operator tolerance of the parity tests


def rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


CASES = [((63, 63), False, H.HOM_OP_AFFINE), ((85, 85), False, H.HOM_OP_EM),
         ((45, 45, 45), False, H.HOM_OP_LINEAR), ((15, 17, 13), True, H.HOM_OP_AFFINE),
         ((81, 81, 81), False, H.HOM_OP_PROJECT)]


@pytest.mark.parametrize("N,aniso,op", CASES)
def test_static_matches_hom_apply_twice(N, aniso, op):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    if aniso:
        table = ms.random_spd_table(2, d, seed=3, scales=[1.0, 20.0])
    else:
        table = ms.isotropic_table([1.0, 10.0], d)
    E = ms.random_unit_vector(d, 1)
    x = torch.from_numpy(ms.random_field((d,) + N, 5)).cuda()
    P = H.Problem(d, N, H.phase_material(ph, table))
    ref = P.field()
    H.hom_apply(P.h, op, E, x, ref)
    ph_dev = torch.from_numpy(ph).cuda()
    for _ in range(2):  # two calls in a row share the static scratch
        y = torch.full_like(x, float("nan"))
        H.hom_apply_static(d, N, ph_dev, table, op, E, x, y)
        torch.cuda.synchronize()
        assert rel(y, ref) < OP_TOL
    P.close()


def test_static_rejects_problems_beyond_the_scratch():
    N = (243, 243, 243)
    ph_dev = torch.zeros(N, dtype=torch.uint8, device="cuda")
    x = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(H.HomError) as ei:
        H.hom_apply_static(3, N, ph_dev, ms.isotropic_table([1.0, 2.0], 3), H.HOM_OP_LINEAR,
                           None, x, x)
    assert ei.value.status == H.HOM_ERR_SCRATCH


FRESH = """
import sys
import numpy as np
import torch
import microstructure as ms
import oracle as O
import paper_1508_02045_gb300 as H
N = (27, 25, 21)
ph = ms.box_phase(N, 0.6)
table = ms.random_spd_table(2, 3, seed=4, scales=[1.0, 30.0])
x = ms.random_field((3,) + N, 9)
E = ms.random_unit_vector(3, 2)
xd = torch.from_numpy(x).cuda()
y = torch.full_like(xd, float("nan"))
# the first call of the library in this process: the set-up runs inside it
H.hom_apply_static(3, N, torch.from_numpy(ph).cuda(), table, H.HOM_OP_AFFINE, E, xd, y)
torch.cuda.synchronize()
sysn = O.GaNi(O.expand_phase(ph, table), 3)
ref = sysn.matvec(sysn.const(E) + x)
err = np.linalg.norm((y.cpu().numpy() - ref).ravel()) / np.linalg.norm(ref.ravel())
print("rel", err)
sys.exit(0 if err < 1e-12 else 1)
"""


def test_static_first_in_a_fresh_process():
    # hom_apply_static before any hom_create in a new process (its own set-up path), against
    # the oracle's GaNi operator
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", FRESH], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
