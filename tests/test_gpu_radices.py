"""Every supported prime factor and the longest axis, against the oracle.

Axis lengths are odd with prime factors up to 31 (the register DFTs of fft_reg.cuh), at most
1023. The other parity tests use lengths built from 3, 5, 7 and 23; here every remaining
prime radix (11, 13, 17, 19, 29, 31) appears as a prime axis and inside composite ones, on
each of the three axes (contiguous axis: line passes; middle axis: strided pass; axis 0:
projection pass), and the longest axis 1023 = 3 * 11 * 31 runs on each axis too, in FP64 at
the operator tolerance 1e-12 and through the FP32 operator at 2e-6.
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

GRIDS = [(11, 13, 17), (19, 29, 31), (31, 5, 3), (3, 29, 5), (5, 3, 19), (77, 65), (51, 57),
         (1023, 3, 3), (3, 1023, 3), (3, 3, 1023), (1023, 5), (5, 1023), (143, 7, 9), (9, 7, 187)]


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.mark.parametrize("N", GRIDS)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_radix_and_the_longest_axis(N, precision):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    prec = H.HOM_FP64 if precision == "fp64" else H.HOM_FP32_REFINED
    P = H.Problem(d, N, H.phase_material(ph, table), precision=prec)
    x = ms.random_field((d,) + N, 17)
    E = ms.random_unit_vector(d, 3)
    y = P.field()
    op = H.HOM_OP_AFFINE | (H.HOM_OP_FP32 if precision == "fp32" else 0)
    H.hom_apply(P.h, op, E, torch.from_numpy(x).cuda(), y)
    sysn = O.GaNi(O.expand_phase(ph, table)[0, 0], d)
    ref = sysn.matvec(sysn.const(E) + x)
    err = rel(y.cpu().numpy(), ref)
    assert err < (1e-12 if precision == "fp64" else 2e-6), err
    P.close()
