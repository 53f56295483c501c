"""The C-ABI boundary beyond device pointers: host-memory inputs and outputs flagged per field,
the Ga corrector returned as N-grid samples, and host-side failure injection.

Host fields: page-locked memory is read and written by the pass kernels through its device
mapping, other host memory is staged; both must give the device-pointer result bit for bit.
Ga output: the iterate of exact integration is a trigonometric polynomial of order N (Section
2.3); its N-grid samples are compared with the oracle's iterate restricted to the N grid.
Failures: the allocation-failure hook makes one device allocation fail as a full device would;
the call returns HOM_ERR_OOM, frees what it had, and the context stays usable.
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

OP_TOL = 1e-12
IT_TOL = 1e-10


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def square_problem(N, precision=H.HOM_FP64):
    d = len(N)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], d)
    return H.Problem(d, N, H.phase_material(ph, table), precision=precision), ph, table


@pytest.mark.parametrize("N", [(45, 45, 45), (63, 63), (243, 7, 5)])
@pytest.mark.parametrize("kind", ["pinned", "pageable", "numpy"])
def test_apply_with_host_fields_matches_device_fields(N, kind):
    d = len(N)
    P, _, _ = square_problem(N)
    x = torch.from_numpy(ms.random_field((d,) + N, 3))
    E = ms.random_unit_vector(d, 1)
    ref = P.field()
    H.hom_apply(P.h, H.HOM_OP_AFFINE, E, x.cuda(), ref)
    torch.cuda.synchronize()
    if kind == "pinned":
        xh, yh = x.pin_memory(), torch.full(x.shape, np.nan, dtype=torch.float64).pin_memory()
    elif kind == "pageable":
        xh, yh = x.clone(), torch.full(x.shape, np.nan, dtype=torch.float64)
    else:
        xh, yh = x.numpy().copy(), np.full(x.shape, np.nan)
    for _ in range(2):
        H.hom_apply(P.h, H.HOM_OP_AFFINE, E, xh, yh)  # returns with y written
        got = yh if isinstance(yh, np.ndarray) else yh.numpy()
        assert np.array_equal(got, ref.cpu().numpy())
    # mixed: host input, device output and the other way round
    yd = P.field()
    H.hom_apply(P.h, H.HOM_OP_AFFINE, E, xh, yd)
    torch.cuda.synchronize()
    assert torch.equal(yd, ref)
    H.hom_apply(P.h, H.HOM_OP_AFFINE, E, x.cuda(), yh)
    got = yh if isinstance(yh, np.ndarray) else yh.numpy()
    assert np.array_equal(got, ref.cpu().numpy())
    P.close()


def test_fp32_operator_with_host_fields():
    N = (45, 45, 45)
    P, _, _ = square_problem(N, H.HOM_FP32_REFINED)
    x = torch.from_numpy(ms.random_field((3,) + N, 5))
    ref = P.field()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, x.cuda(), ref)
    yh = torch.empty(x.shape, dtype=torch.float64).pin_memory()
    H.hom_apply(P.h, H.HOM_OP_LINEAR | H.HOM_OP_FP32, None, x.pin_memory(), yh)
    assert np.array_equal(yh.numpy(), ref.cpu().numpy())
    P.close()


def test_solve_writes_the_corrector_to_host_memory():
    N = (27, 25, 21)
    P, _, _ = square_problem(N)
    E = np.array([0.0, 1.0, 0.0])
    xd = P.field()
    AH_d, _, _, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-9, None, xd)
    xh = np.full((3,) + N, np.nan)
    AH_h, _, _, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-9, None, xh)
    assert AH_h == AH_d
    assert np.array_equal(xh, xd.cpu().numpy())
    P.close()


def ga_box(N, M=None):
    d = len(N)
    Mg = tuple(M) if M is not None else O.double_grid(N)
    h = 0.6
    Ahat = ms.box_fourier_coefficients(Mg, h, 1.0, 10.0)
    P = H.Problem(d, N, H.fourier_material(Ahat.astype(np.complex128), 1.0, 10.0, M), H.HOM_EXACT)
    return P, O.Ga(O.ga_coefficients(Ahat, d), tuple(N), d)


@pytest.mark.parametrize("N,M", [((9, 7), None), ((7, 9, 5), None), ((9, 9, 9), (19, 21, 17))])
def test_ga_corrector_on_the_N_grid(N, M):
    d = len(N)
    P, sysg = ga_box(N, M)
    E = ms.random_unit_vector(d, 6)
    ref = O.cg(sysg, E, fixed_iters=12).x          # the oracle's Ga iterate on the grid M
    opts = H.make_opts(fixed_iters=12, out_flags=H.HOM_OUT_NGRID)
    xN = torch.zeros((d,) + tuple(N), dtype=torch.float64, device="cuda")
    AH, _, _, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-9, opts, xN)
    assert rel(xN.cpu().numpy(), O.restrict(ref, N)) < IT_TOL
    # the same on the host, and the solve-grid field beside it
    opts = H.make_opts(fixed_iters=12, out_flags=H.HOM_OUT_NGRID | H.HOM_OUT_HOST)
    xNh = np.zeros((d,) + tuple(N))
    H.hom_solve(P.h, E, H.HOM_CG, 1e-9, opts, xNh)
    assert np.array_equal(xNh, xN.cpu().numpy())
    xM = P.field()
    AH2, _, _, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-9, H.make_opts(fixed_iters=12), xM)
    assert AH2 == AH
    assert rel(xM.cpu().numpy(), ref) < IT_TOL
    # hom_restrict is the same map on its own, and prolongation returns the solve-grid field
    yN = torch.zeros_like(xN)
    H.hom_restrict(P.h, xM, yN)
    torch.cuda.synchronize()
    assert torch.equal(yN, xN)
    assert rel(O.prolongate(xN.cpu().numpy(), P.grid), xM.cpu().numpy()) < 1e-12
    P.close()


def test_injected_allocation_failures_return_oom_and_leak_nothing():
    N = (45, 45, 45)
    ph = ms.box_phase(N, 0.6)
    table = ms.isotropic_table([1.0, 10.0], 3)
    mat = H.phase_material(ph, table)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    created = False
    failures = 0
    for n in range(64):
        H.hom_debug_fail_alloc(n)
        try:
            h = H.hom_create(3, N, mat, H.HOM_APPROX, H.HOM_FP32_REFINED)
        except H.HomError as e:
            assert e.status == H.HOM_ERR_OOM
            failures += 1
            continue
        H.hom_debug_fail_alloc(-1)
        created = True
        # the context is intact: the problem solves normally after the earlier failures
        AH, _, st, _ = H.hom_solve(h, np.array([1.0, 0.0, 0.0]), H.HOM_CG, 1e-8)
        assert st["converged"] and AH > 1.0
        H.hom_destroy(h)
        break
    H.hom_debug_fail_alloc(-1)
    assert created and failures >= 10
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)


def test_injected_failure_in_solve_begin_and_server_admission():
    N = (15, 15, 15)
    P, ph, table = square_problem(N)
    E = np.array([1.0, 0.0, 0.0])
    H.hom_debug_fail_alloc(0)  # the first solve allocates its iteration history
    with pytest.raises(H.HomError) as ei:
        H.hom_solve(P.h, E, H.HOM_CG, 1e-8)
    assert ei.value.status == H.HOM_ERR_OOM
    H.hom_debug_fail_alloc(-1)
    AH, _, st, _ = H.hom_solve(P.h, E, H.HOM_CG, 1e-8)
    assert st["converged"]
    P.close()
    S = H.hom_server_create(1 << 30, max_batch=2)
    mat = H.phase_material(ph, table)
    ids = [H.hom_server_submit(S, H.make_request(3, N, mat, E, H.HOM_CG, 1e-8)) for _ in range(2)]
    H.hom_debug_fail_alloc(0)  # the first admission's hom_create fails
    results = {}
    for _ in range(200):
        H.hom_server_step(S, 4)
        for r in H.hom_server_poll(S):
            results[r["id"]] = r
        if len(results) == 2:
            break
    H.hom_debug_fail_alloc(-1)
    H.hom_server_destroy(S)
    assert results[ids[0]]["status"] == H.HOM_ERR_OOM
    assert results[ids[1]]["status"] == H.HOM_OK
    assert abs(results[ids[1]]["AH_EE"] - AH) < 1e-10 * AH


def test_fp64_throughput_probe():
    ms_fma, flops = H.hom_measure_fp64(0, 400)
    ms_add, adds = H.hom_measure_fp64(1, 400)
    assert ms_fma > 0 and ms_add > 0
    tf = flops / ms_fma / 1e9
    assert 0.1 < tf < 10.0  # TFLOP/s: a GB300 runs FP64 FMAs near 1.2 T


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second CUDA device")
def test_problem_on_a_second_device():
    # the kernels' per-device set-up (DFT constants, shared-memory limits) runs for each device
    N = (27, 25, 21)
    E = np.array([1.0, 0.0, 0.0])
    res = []
    for dev in (0, 1):
        with torch.cuda.device(dev):
            P, _, _ = square_problem(N)
            res.append(H.hom_solve(P.h, E, H.HOM_CG, 1e-10)[0])
            P.close()
    assert res[0] == res[1]
