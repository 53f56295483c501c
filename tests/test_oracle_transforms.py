"""Pins of the oracle's DFT, projection, double-grid coefficients and prolongation.

Each check compares the oracle with something that is not the oracle: NumPy's FFT (a library
routine the definition reduces to), closed-form derivatives of trigonometric polynomials,
direct quadrature of eq. (FT_def), or algebraic identities of the projection (Section 2).
"""
import numpy as np
import pytest

import microstructure as ms
import oracle as O


@pytest.mark.parametrize("shape", [(3,), (5, 7), (9, 5, 3), (15, 15)])
def test_dft_matches_numpy_fft(shape):
    # eq. (DFT): F_N = (1/|N|) omega^{-mk} is numpy's forward FFT divided by |N|;
    # F_N^{-1} = omega^{mk} is numpy's inverse FFT times |N|.
    rng = np.random.default_rng(1)
    v = rng.standard_normal((2,) + shape) + 1j * rng.standard_normal((2,) + shape)
    nd = len(shape)
    axes = tuple(range(1, nd + 1))
    size = int(np.prod(shape))
    np.testing.assert_allclose(O.dft(v, nd), np.fft.fftn(v, axes=axes) / size, atol=1e-14)
    np.testing.assert_allclose(O.idft(v, nd), np.fft.ifftn(v, axes=axes) * size, atol=1e-12)
    np.testing.assert_allclose(O.idft(O.dft(v, nd), nd), v, atol=1e-13)


def test_dft_plancherel():
    # Scaled forward transform: ||v||^2 (weighted) = sum |v^(k)|^2.
    v = ms.random_field((2, 9, 7), 3)
    vh = O.dft(v, 2)
    assert abs(np.mean(np.sum(v * v, 0)) - np.sum(np.abs(vh) ** 2)) < 1e-13


def _trig_potential(N, seed):
    """A random real trigonometric polynomial phi of order N, its nodal values and the nodal
    values of its exact gradient (closed-form derivative)."""
    rng = np.random.default_rng(seed)
    d = len(N)
    xs = ms.node_coords(N)
    phi = np.zeros(N)
    grad = np.zeros((d,) + tuple(N))
    for _ in range(6):
        k = np.array([rng.integers(-(n - 1) // 2, (n - 1) // 2 + 1) for n in N])
        a, b = rng.standard_normal(2)
        t = sum(2 * np.pi * k[i] * xs[i] for i in range(d))
        t = np.broadcast_to(t, N)
        phi += a * np.cos(t) + b * np.sin(t)
        for i in range(d):
            grad[i] += 2 * np.pi * k[i] * (-a * np.sin(t) + b * np.cos(t))
    return phi, grad


@pytest.mark.parametrize("N", [(9, 7), (5, 7, 9)])
def test_projection_fixes_gradients_and_kills_constants(N):
    d = len(N)
    _, grad = _trig_potential(N, 7)
    np.testing.assert_allclose(O.project(grad), grad, atol=1e-10)
    const = np.broadcast_to(np.arange(1.0, d + 1).reshape((d,) + (1,) * d), (d,) + N).copy()
    assert np.abs(O.project(const)).max() < 1e-13


def test_projection_kills_divergence_free_fields():
    # 2-D: v = (d2 psi, -d1 psi) is divergence free for any trigonometric psi.
    N = (9, 11)
    rng = np.random.default_rng(2)
    xs = ms.node_coords(N)
    v = np.zeros((2,) + N)
    for _ in range(5):
        k = np.array([rng.integers(-4, 5), rng.integers(-5, 6)])
        t = np.broadcast_to(2 * np.pi * (k[0] * xs[0] + k[1] * xs[1]), N)
        # psi = sin(t): d_a psi = 2 pi k_a cos(t)
        v[0] += 2 * np.pi * k[1] * np.cos(t)
        v[1] += -2 * np.pi * k[0] * np.cos(t)
    assert np.abs(O.project(v)).max() < 1e-10


@pytest.mark.parametrize("N", [(7, 9), (5, 5, 7)])
def test_projection_idempotent_selfadjoint_curlfree(N):
    d = len(N)
    u = ms.random_field((d,) + N, 11)
    w = ms.random_field((d,) + N, 12)
    Gu = O.project(u)
    np.testing.assert_allclose(O.project(Gu), Gu, atol=1e-13)
    lhs = np.mean(np.sum(Gu * w, 0))
    rhs = np.mean(np.sum(u * O.project(w), 0))
    assert abs(lhs - rhs) < 1e-13
    # curl-free and zero-mean output: its spectrum (numpy FFT) is parallel to k, zero at k = 0
    sh = np.fft.fftn(Gu, axes=tuple(range(1, d + 1)))
    ks = np.meshgrid(*[np.fft.fftfreq(n) * n for n in N], indexing="ij")
    for a in range(d):
        for b in range(d):
            assert np.abs(ks[a] * sh[b] - ks[b] * sh[a]).max() < 1e-9
    assert np.abs(sh[(slice(None),) + (0,) * d]).max() < 1e-9


def test_double_grid_projection_support_and_fixed_points():
    # G_{N,M} (eq. (discrete_proj)) keeps I_M of gradients of order-N polynomials and removes
    # every frequency outside Z_N.
    N = (7, 9)
    M = O.double_grid(N)
    d = 2
    u = ms.random_field((d,) + M, 5)
    Gu = O.project(u, support=N)
    sh = np.fft.fftn(Gu, axes=(1, 2))
    k0 = np.abs(np.fft.fftfreq(M[0]) * M[0])[:, None]
    k1 = np.abs(np.fft.fftfreq(M[1]) * M[1])[None, :]
    outside = (k0 >= N[0] / 2) | (k1 >= N[1] / 2)
    assert np.abs(sh[:, outside]).max() < 1e-9
    # sample an order-N gradient on M directly (closed form): it must be a fixed point
    rng = np.random.default_rng(4)
    xs = ms.node_coords(M)
    g = np.zeros((d,) + M)
    for _ in range(4):
        k = np.array([rng.integers(-3, 4), rng.integers(-4, 5)])
        t = np.broadcast_to(2 * np.pi * (k[0] * xs[0] + k[1] * xs[1]), M)
        for a in range(d):
            g[a] += -2 * np.pi * k[a] * np.sin(t)
    np.testing.assert_allclose(O.project(g, support=N), g, atol=1e-10)


def test_prolongation_evaluates_the_trigonometric_polynomial():
    # R_{N,M} = I_M o I_N^{-1}: nodal values of phi on N -> values of the same phi on M.
    N = (7, 9)
    M = (13, 17)
    phiN, gN = _trig_potential(N, 21)
    # the same polynomial evaluated on M: rebuild it with identical random draws
    rng = np.random.default_rng(21)
    xs = ms.node_coords(M)
    gM = np.zeros((2,) + M)
    for _ in range(6):
        k = np.array([rng.integers(-(n - 1) // 2, (n - 1) // 2 + 1) for n in N])
        a, b = rng.standard_normal(2)
        t = np.broadcast_to(sum(2 * np.pi * k[i] * xs[i] for i in range(2)), M)
        for i in range(2):
            gM[i] += 2 * np.pi * k[i] * (-a * np.sin(t) + b * np.cos(t))
    np.testing.assert_allclose(O.prolongate(gN, M), gM, atol=1e-10)


def test_box_fourier_coefficients_quadrature():
    # eq. (FT_def) for the box |x| < h/2, integrated by a fine midpoint rule (1-D factor).
    h = 0.6
    M = (29,)
    coef = ms.box_fourier_coefficients(M, h, 0.0, 1.0)
    x = (np.arange(200000) + 0.5) / 200000 - 0.5
    chi = (np.abs(x) < h / 2).astype(float)
    for j, n in enumerate(ms.signed_index(29)):
        ref = np.mean(chi * np.exp(-2j * np.pi * n * x))
        assert abs(coef[j] - ref) < 1e-5


def test_ga_coefficients_mean_is_exact_voigt():
    # The double-grid mean of A_M is A^(0) = a_m + (a_i - a_m) h^d: the exact integral of A.
    N = (15, 15)
    M = O.double_grid(N)
    A_M = O.ga_coefficients(ms.box_fourier_coefficients(M, 0.6, 1.0, 100.0), 2)
    assert abs(A_M.mean() - (1.0 + 99.0 * 0.36)) < 1e-12


def test_voxel_fourier_coefficients_quadrature():
    # eq. (FT_def) for a random voxel image on (3, 5), integrated by a fine midpoint rule whose
    # sub-cells tile every voxel cell [k/N - 1/(2N), k/N + 1/(2N)) (no reuse of the sinc form)
    N = (3, 5)
    M = (7, 11)
    a = np.random.default_rng(3).uniform(1.0, 10.0, N)
    coef = O.voxel_fourier_coefficients(a, M)
    S = 200
    xs = [(np.arange(n * S) + 0.5) / (n * S) - 0.5 / n for n in N]  # sub-cell midpoints
    cell = [np.mod(np.floor(x * n + 0.5).astype(int), n) for x, n in zip(xs, N)]
    f = a[np.ix_(cell[0], cell[1])]
    for j0, n0 in enumerate(O.signed_index(M[0])):
        e0 = np.exp(-2j * np.pi * n0 * xs[0])
        for j1, n1 in enumerate(O.signed_index(M[1])):
            e1 = np.exp(-2j * np.pi * n1 * xs[1])
            ref = np.mean(f * np.outer(e0, e1))
            assert abs(coef[j0, j1] - ref) < 2e-4 * abs(a).max(), (n0, n1)
    assert abs(coef[0, 0] - a.mean()) < 1e-14 * a.mean()


@pytest.mark.parametrize("N,h", [((15, 15), 0.6), ((9, 7, 5), 5 / 9)])
def test_voxel_coefficients_of_whole_voxel_box_are_analytic(N, h):
    # a centred box of whole voxels (side s_a = count_a / N_a on axis a): its voxel image and
    # the analytic coefficients of the box, delta_{n0} a_m + (a_i - a_m) prod_a s_a sinc(pi n_a
    # s_a), are the same function
    d = len(N)
    M = O.double_grid(N)
    ph = ms.box_phase(N, h)
    sides = [int(np.count_nonzero(np.abs(O.signed_index(n)) / n < h / 2)) / n for n in N]
    a = np.where(ph > 0, 10.0, 1.0)
    got = O.voxel_fourier_coefficients(a, M)
    k = O.frequencies(M)
    box = np.ones(M)
    for ax, s_ in enumerate(sides):
        box = box * (s_ * np.sinc(k[ax] * s_))
    delta = np.zeros(M)
    delta[(0,) * d] = 1.0
    np.testing.assert_allclose(got, delta + 9.0 * box, atol=1e-13)
    if np.allclose(sides, h):  # the microstructure module's analytic box coefficients
        np.testing.assert_allclose(got, ms.box_fourier_coefficients(M, h, 1.0, 10.0), atol=1e-13)


def _trig_field_on(shape_eval, N, seed, d):
    """A closed-form vector field of trigonometric order N (sum of a few modes k in Z_N with
    random amplitudes) evaluated at the nodes of the grid `shape_eval`."""
    rng = np.random.default_rng(seed)
    xs = ms.node_coords(shape_eval)
    out = np.zeros((d,) + tuple(shape_eval))
    for _ in range(5):
        k = np.array([rng.integers(-(n - 1) // 2, (n - 1) // 2 + 1) for n in N])
        amp = rng.standard_normal((d, 2))
        t = np.broadcast_to(sum(2 * np.pi * k[i] * xs[i] for i in range(d)), shape_eval)
        for i in range(d):
            out[i] += amp[i, 0] * np.cos(t) + amp[i, 1] * np.sin(t)
    return out


@pytest.mark.parametrize("N,M", [((7, 9), (13, 17)), ((5, 3, 7), (9, 5, 13)), ((9,), (19,))])
def test_restriction_samples_the_trigonometric_polynomial(N, M):
    # R^{-1}: values of a polynomial of order N on the grid M -> its values at the N nodes,
    # checked against the closed form evaluated directly on both grids
    d = len(N)
    vM = _trig_field_on(M, N, 31, d)
    vN = _trig_field_on(N, N, 31, d)
    np.testing.assert_allclose(O.restrict(vM, N), vN, atol=1e-11)


def test_restriction_inverts_prolongation():
    N, M = (7, 5, 9), (13, 11, 17)
    x = ms.random_field((3,) + N, 4)
    np.testing.assert_allclose(O.restrict(O.prolongate(x, M), N), x, atol=1e-12)
    # and the M-grid field of an exact-integration solve lies in the range of G_{N,M}: its
    # restriction, prolonged again, returns it
    y = O.project(ms.random_field((3,) + M, 5), support=N)
    np.testing.assert_allclose(O.prolongate(O.restrict(y, N), M), y, atol=1e-12)
