"""Pass kernels on a created stream are launched with a programmatic dependency on the kernel
before them (each waits for it before touching memory); on the legacy default stream they are
plain launches. Both must give the same results bit for bit: the operator in FP64 and FP32,
and solves of every solver."""
import numpy as np
import pytest

import microstructure as ms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402


def run(N, prec, stream, solver):
    with torch.cuda.stream(stream):
        ph = ms.box_phase(N, 0.6)
        P = H.Problem(len(N), N, H.phase_material(ph, ms.isotropic_table([1.0, 20.0], len(N))),
                      precision=prec)
        x = torch.from_numpy(ms.random_field((len(N),) + N, 2)).cuda()
        y = P.field()
        op = H.HOM_OP_LINEAR | (H.HOM_OP_FP32 if prec == H.HOM_FP32_REFINED else 0)
        H.hom_apply(P.h, op, None, x, y)
        stream.synchronize()
        E = np.eye(len(N))[0]
        xs = P.field()
        AH, _, st, _ = H.hom_solve(P.h, E, H.SOLVERS[solver], 1e-9, None, xs)
        P.close()
    return y.cpu(), xs.cpu(), AH, st["iterations"]


@pytest.mark.parametrize("N,prec,solver", [((45, 45, 45), H.HOM_FP64, "cg"),
                                           ((27, 25, 21), H.HOM_FP64, "chebyshev"),
                                           ((27, 25, 21), H.HOM_FP64, "eyre_milton"),
                                           ((63, 63), H.HOM_FP64, "richardson"),
                                           ((81, 81, 81), H.HOM_FP32_REFINED, "cg"),
                                           ((45, 45, 45), H.HOM_FP32_REFINED, "chebyshev")])
def test_side_stream_equals_default_stream(N, prec, solver):
    a = run(N, prec, torch.cuda.default_stream(), solver)
    b = run(N, prec, torch.cuda.Stream(), solver)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]
