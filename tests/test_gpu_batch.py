"""Batched iterations (hom_batch) and the continuous-batching server (hom_server).

Every request runs the same solver steps as a solo solve with its own buffers, scalars and
fixed-order reductions, so its result must be the same alone and in the mix: bit-identical
for the batched iterations, and within 1e-14 for the server (checked against solo solves).
"""
import numpy as np
import pytest

import microstructure as ms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1508_02045_gb300 as H  # noqa: E402


def material(N, seed, contrast):
    d = len(N)
    ph, c, r = ms.rsa_spheres(N, seed, rmin=0.08, rmax=0.15, vf=0.25)
    rng = np.random.default_rng(seed + 7)
    vals = np.concatenate([[1.0], np.exp(rng.uniform(0.0, np.log(contrast), len(r)))])
    return H.phase_material(ph, ms.isotropic_table(vals, d))


def solo(N, mat, E, solver, precision, opts, tol):
    P = H.Problem(len(N), N, mat, precision=precision)
    x = P.field()
    AH, _, stats, _ = H.hom_solve(P.h, E, solver, tol, opts, x, allow_not_converged=True)
    P.close()
    return AH, x, stats


@pytest.mark.parametrize("solver", ["richardson", "cg", "chebyshev", "eyre_milton"])
def test_batch_matches_solo_bitwise(solver):
    N = (27, 25, 21)
    mats = [material(N, s, 100.0) for s in (1, 2, 3)]
    Es = [ms.random_unit_vector(3, s) for s in (4, 5, 6)]
    its = 12
    opts = H.make_opts(fixed_iters=its)
    ref = [solo(N, m, E, H.SOLVERS[solver], H.HOM_FP64, opts, 0.0) for m, E in zip(mats, Es)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        probs = [H.Problem(3, N, m) for m in mats]
        for P, E in zip(probs, Es):
            H.hom_solve_begin(P.h, E, H.SOLVERS[solver], 0.0, opts)
        B = H.hom_batch_create([P.h for P in probs])
        H.hom_batch_iterate(B, its, use_graph=True)
        for P, E, (AH_ref, x_ref, _) in zip(probs, Es, ref):
            x = P.field()
            AH, _, stats, _ = H.hom_solve_end(P.h, 3, x)
            assert stats["iterations"] == its
            assert AH == AH_ref
            assert torch.equal(x, x_ref)
        H.hom_batch_destroy(B)
        for P in probs:
            P.close()


@pytest.mark.parametrize("N", [(21, 23, 19), (45, 45, 21)])
def test_batch_refined_matches_solo(N):
    mats = [material(N, s, 1000.0) for s in (11, 12)]
    Es = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.6, 0.8])]
    ref = [solo(N, m, E, H.HOM_CG, H.HOM_FP32_REFINED, None, 1e-9) for m, E in zip(mats, Es)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        probs = [H.Problem(3, N, m, precision=H.HOM_FP32_REFINED) for m in mats]
        for P, E in zip(probs, Es):
            H.hom_solve_begin(P.h, E, H.HOM_CG, 1e-9, None)
        B = H.hom_batch_create([P.h for P in probs])
        for _ in range(200):
            if H.hom_batch_iterate(B, 8, use_graph=True, poll=True):
                break
        for P, (AH_ref, _, st_ref) in zip(probs, ref):
            AH, _, stats, _ = H.hom_solve_end(P.h, 3)
            assert stats["converged"]
            assert abs(AH - AH_ref) <= 1e-14 * abs(AH_ref)
        H.hom_batch_destroy(B)
        for P in probs:
            P.close()


def test_server_results_equal_solo_solves():
    shapes = [(15, 13, 11), (21, 21, 21)]
    plan = []
    seed = 20
    for N in shapes:
        for solver, prec in [("cg", H.HOM_FP64), ("chebyshev", H.HOM_FP64),
                             ("eyre_milton", H.HOM_FP64), ("cg", H.HOM_FP32_REFINED),
                             ("richardson", H.HOM_FP64)]:
            seed += 1
            plan.append((N, material(N, seed, 50.0), ms.random_unit_vector(3, seed), solver, prec))
    S = H.hom_server_create(64 << 20, max_batch=4)  # a small budget forces queueing
    ids = {}
    for i, (N, mat, E, solver, prec) in enumerate(plan):
        req = H.make_request(3, N, mat, E, H.SOLVERS[solver], 1e-8, precision=prec)
        ids[H.hom_server_submit(S, req)] = i
    results = {}
    for _ in range(20000):
        H.hom_server_step(S, 4)
        for r in H.hom_server_poll(S):
            results[r["id"]] = r
        if len(results) == len(plan):
            break
    active, queued, used = H.hom_server_status(S)
    H.hom_server_destroy(S)
    assert len(results) == len(plan) and active == 0 and queued == 0 and used == 0
    for rid, r in results.items():
        N, mat, E, solver, prec = plan[ids[rid]]
        assert r["status"] == H.HOM_OK
        AH_ref, _, st = solo(N, mat, E, H.SOLVERS[solver], prec, None, 1e-8)
        assert r["stats"]["iterations"] == st["iterations"]
        assert abs(r["AH_EE"] - AH_ref) <= 1e-14 * abs(AH_ref), (solver, prec, N)
        assert r["latency_ms"] >= r["queue_ms"] >= 0


def test_server_keeps_serving_after_a_bucket_empties():
    # first wave drains its bucket completely; later steps must only touch live buckets
    S = H.hom_server_create(1 << 30, max_batch=2)
    wave1 = [(15, 15, 15)] * 2
    wave2 = [(13, 11, 9)] * 3
    seen = {}
    for i, N in enumerate(wave1):
        rid = H.hom_server_submit(S, H.make_request(3, N, material(N, 40 + i, 20.0),
                                                    np.array([1.0, 0.0, 0.0]), H.HOM_CG, 1e-8))
        seen[rid] = None
    for _ in range(5000):
        H.hom_server_step(S, 4)
        for r in H.hom_server_poll(S):
            seen[r["id"]] = r
        if all(v is not None for v in seen.values()):
            break
    assert H.hom_server_status(S)[0] == 0
    for i, N in enumerate(wave2):
        rid = H.hom_server_submit(S, H.make_request(3, N, material(N, 50 + i, 20.0),
                                                    np.array([0.0, 1.0, 0.0]), H.HOM_CHEBYSHEV, 1e-8))
        seen[rid] = None
    for _ in range(5000):
        H.hom_server_step(S, 4)
        for r in H.hom_server_poll(S):
            seen[r["id"]] = r
        if all(v is not None for v in seen.values()):
            break
    H.hom_server_destroy(S)
    assert all(v is not None and v["status"] == H.HOM_OK for v in seen.values())
