"""Pins of the 1-D WENO interpolant (Sec. 2) and the tensor-WENO resampling /
arbitrary-scale zoom (Sec. 3.3) in the FP64 oracle, against facts the paper
and the mathematics fix: interpolation at the nodes, the cubic of Eq.
(PolinomZaVelikiStencil) at beta = 0 (numpy's polynomial fit), exactness on
quadratics at any beta, the smoothness indicator by quadrature in physical
units, the ENO choice at a jump, reflection symmetry, fourth-order
convergence (Sec. 2), separable polynomial reproduction and the
endpoint-aligned grid of Sec. 3.3."""
import numpy as np
import pytest
from scipy import integrate

import oracle

BETAS = (0.0, 0.1, 1.0, 2.0, 3.0)


def test_nodes_are_interpolated():
    rng = np.random.default_rng(1)
    V = rng.random(11)
    for beta in BETAS:
        for i in range(V.size):
            assert oracle.weno_spline(V, i, beta=beta) == pytest.approx(V[i], abs=1e-14)
        for i in range(V.size - 1):  # t = 1 end of each cell
            v4 = [V[max(i - 1, 0)], V[i], V[i + 1], V[min(i + 2, V.size - 1)]]
            assert oracle.weno1d_cell(v4, 1.0, beta=beta) == pytest.approx(V[i + 1], abs=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_beta0_is_the_cubic_through_four_nodes(seed):
    """beta = 0 gives the linear weights C_{i,s}, so u_i = q_i (Eq.
    PolinomZaVelikiStencil): the cubic through x_{i-1..i+2}."""
    rng = np.random.default_rng(seed)
    v4 = rng.normal(size=4)
    coef = np.polyfit([-1.0, 0.0, 1.0, 2.0], v4, 3)
    for t in np.linspace(0.0, 1.0, 9):
        assert oracle.weno1d_cell(v4, t, beta=0.0) == pytest.approx(np.polyval(coef, t),
                                                                  abs=1e-13)


@pytest.mark.parametrize("beta", BETAS)
def test_quadratics_are_exact_for_any_beta(beta):
    a, b, c = 0.3, -1.7, 0.45
    x = np.arange(12.0)
    V = a + b * x + c * x * x
    for xx in np.linspace(1.0, 10.0, 37):  # cells whose stencils stay inside
        assert oracle.weno_spline(V, xx, beta=beta) == pytest.approx(a + b * xx + c * xx * xx,
                                                                    abs=1e-11)


def _si_quadrature(nodes, vals, lo, hi, h):
    """SI = sum_{l=1,2} int h^{2l-1} (p^{(l)})^2 dx in physical units."""
    c = np.polyfit(nodes, vals, 2)
    d1, d2 = np.polyder(c, 1), np.polyder(c, 2)
    f = lambda x: h * np.polyval(d1, x) ** 2 + h ** 3 * np.polyval(d2, x) ** 2
    return integrate.quad(f, lo, hi)[0]


@pytest.mark.parametrize("h,k_eps,beta", [(1.0, 1e-8, 2.0), (0.25, 3.0, 1.0), (2.0, 0.05, 1.5)])
def test_weights_from_quadrature_indicators(h, k_eps, beta):
    """Eq. (IzrazOmega) with SI integrated numerically on the physical cell
    [0, h] and eps_h = K_eps h^2: pins the indicator and its h scaling."""
    rng = np.random.default_rng(7)
    v4 = rng.normal(size=4)
    X = np.array([-h, 0.0, h, 2 * h])
    si0 = _si_quadrature(X[:3], v4[:3], 0.0, h, h)
    si1 = _si_quadrature(X[1:], v4[1:], 0.0, h, h)
    p0 = np.polyfit(X[:3], v4[:3], 2)
    p1 = np.polyfit(X[1:], v4[1:], 2)
    q = np.polyfit(X, v4, 3)
    for t in (0.1, 0.5, 0.85):
        x = t * h
        # linear C_{i,s}(x): solve C0 p0 + C1 p1 = q at two points
        M = np.array([[np.polyval(p0, 0.2 * h), np.polyval(p1, 0.2 * h)],
                      [np.polyval(p0, 0.7 * h), np.polyval(p1, 0.7 * h)]])
        # C0 = a + b x, C1 = 1 - C0 ; determine a, b from q = p1 + C0 (p0 - p1)
        xs = np.array([0.2 * h, 0.7 * h])
        C0s = (np.polyval(q, xs) - M[:, 1]) / (M[:, 0] - M[:, 1])
        b = (C0s[1] - C0s[0]) / (xs[1] - xs[0])
        C0 = C0s[0] + b * (x - xs[0])
        eps_h = k_eps * h * h
        a0 = C0 / (eps_h + si0) ** beta
        a1 = (1.0 - C0) / (eps_h + si1) ** beta
        want = (a0 * np.polyval(p0, x) + a1 * np.polyval(p1, x)) / (a0 + a1)
        got = oracle.weno1d_cell(v4, t, beta=beta, k_eps=k_eps, h=h)
        assert got == pytest.approx(want, abs=1e-9, rel=1e-9)


def test_eno_choice_at_a_jump():
    """A jump between x_{i+1} and x_{i+2} leaves p_i flat: the interpolant
    takes p_i; the mirrored jump takes p_{i+1}."""
    for t in np.linspace(0.05, 0.95, 7):
        assert abs(oracle.weno1d_cell([0.0, 0.0, 0.0, 1.0], t, beta=2.0)) < 1e-12
        assert abs(oracle.weno1d_cell([1.0, 0.0, 0.0, 0.0], t, beta=2.0)) < 1e-12
        # beta = 0 follows the cubic instead and overshoots
        assert abs(oracle.weno1d_cell([0.0, 0.0, 0.0, 1.0], t, beta=0.0)) > 1e-3


def test_reflection_symmetry():
    rng = np.random.default_rng(3)
    V = rng.random(9)
    for beta in BETAS:
        for x in np.linspace(0.0, 8.0, 33):
            assert oracle.weno_spline(V, x, beta=beta) == pytest.approx(
                oracle.weno_spline(V[::-1], 8.0 - x, beta=beta), abs=1e-13)


@pytest.mark.parametrize("f", [np.exp, lambda x: np.sin(3 * x + 0.3)])
def test_fourth_order_convergence(f):
    """Sec. 2: u_i is a fourth-order approximation of smooth data."""
    errs = []
    for N in (40, 80, 160, 320):
        x = np.linspace(0.0, 1.0, N)
        h = x[1] - x[0]
        V = f(x)
        xs = np.arange(2, N - 3) + 0.37
        errs.append(max(abs(oracle.weno_spline(V, xx, h=h) - f(xx * h)) for xx in xs))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 3.8, orders


def test_identity_resample_and_endpoint_grid():
    rng = np.random.default_rng(5)
    A = rng.random((2, 7, 9))
    U = oracle.tensor_resample(A, 7, 9)
    assert np.abs(U - A).max() < 1e-14
    for oh, ow in ((3, 4), (13, 17), (2, 2), (20, 5)):
        U = oracle.tensor_resample(A, oh, ow)
        for (r, c), (i, k) in (((0, 0), (0, 0)), ((0, -1), (0, -1)), ((-1, 0), (-1, 0)),
                               ((-1, -1), (-1, -1))):
            assert U[:, r, c] == pytest.approx(A[:, i, k], abs=1e-14)
    # doubling on the endpoint-aligned grid keeps every input sample
    U = oracle.tensor_resample(A, 13, 17)
    assert np.abs(U[:, ::2, ::2] - A).max() < 1e-14


def _interior(n, n_out, margin):
    r = np.arange(n_out)
    y = r * (n - 1) / (n_out - 1)
    return r[(y >= margin) & (y <= n - 1 - margin)], y


@pytest.mark.parametrize("beta", (0.0, 2.0))
def test_tensor_reproduces_separable_polynomials(beta):
    """Columns then rows of 1-D interpolants: products of cubics are exact
    at beta = 0 (bicubic q_i in each direction), products of quadratics at
    any beta, away from the clamped ends."""
    n, m, oh, ow = 10, 12, 23, 31
    i = np.arange(n, dtype=float)[:, None]
    k = np.arange(m, dtype=float)[None, :]
    if beta == 0.0:
        P = lambda y: 0.2 + 0.5 * y - 0.07 * y ** 2 + 0.004 * y ** 3
        Q = lambda x: -0.3 + 0.1 * x + 0.02 * x ** 2 - 0.003 * x ** 3
    else:
        P = lambda y: 0.2 + 0.5 * y - 0.07 * y ** 2
        Q = lambda x: -0.3 + 0.1 * x + 0.02 * x ** 2
    A = P(i) * Q(k)
    U = oracle.tensor_resample(A, oh, ow, beta=beta)
    rows, y = _interior(n, oh, 1.0)
    cols, x = _interior(m, ow, 1.0)
    want = P(y[rows])[:, None] * Q(x[cols])[None, :]
    assert np.abs(U[np.ix_(rows, cols)] - want).max() < 1e-11


def test_tensor_is_columns_then_rows():
    """Eq. (tensor): z_k = w(A(:, k), y), then U = w(Z, x)."""
    rng = np.random.default_rng(11)
    A = rng.random((6, 7))
    A[:, 4:] += 1.0  # an edge makes the two orders differ
    A[3:, :] *= 0.3
    oh, ow = 9, 11
    U = oracle.tensor_resample(A, oh, ow)
    want = np.empty((oh, ow))
    other = np.empty((oh, ow))
    for r in range(oh):
        y = r * 5 / (oh - 1)
        Z = [oracle.weno_spline(A[:, k], y) for k in range(7)]
        for c in range(ow):
            want[r, c] = oracle.weno_spline(Z, c * 6 / (ow - 1))
    for c in range(ow):
        x = c * 6 / (ow - 1)
        Y = [oracle.weno_spline(A[j, :], x) for j in range(6)]
        for r in range(oh):
            other[r, c] = oracle.weno_spline(Y, r * 5 / (oh - 1))
    assert np.abs(U - want).max() < 1e-14
    assert np.abs(U - other).max() > 1e-6


def test_single_row_and_column():
    rng = np.random.default_rng(2)
    A = rng.random((1, 9))
    U = oracle.tensor_resample(A, 3, 17)
    row = [oracle.weno_spline(A[0], c * 8 / 16) for c in range(17)]
    assert np.abs(U - np.array(row)[None, :]).max() < 1e-14
    U = oracle.tensor_resample(A.T, 17, 1)
    assert np.abs(U[:, 0] - np.array(row)).max() < 1e-14


def test_zoom_to_levels_and_quadratic_surface():
    """Arbitrary scale (Sec. 3.3): n -> 2^k (n-1) + 1 until the target is
    covered, then tensor resampling.  A total-degree-2 surface is exact at
    every level (WD WENO and the 1-D interpolant both reproduce it), so the
    result is the surface sampled on the endpoint-aligned 3x grid."""
    from paper_2312_00229_gb300.api import zoom_levels
    assert zoom_levels(24, 20, 72, 60) == 2   # 3x: up to 4n-3, down to 3n
    assert zoom_levels(8, 8, 8, 8) == 0
    assert zoom_levels(2, 2, 6, 6) == 3
    assert zoom_levels(1, 9, 1, 30) == 2
    f = lambda y, x: 0.3 + 0.02 * y - 0.01 * x + 0.004 * x * y + 0.002 * y * y - 0.003 * x * x
    n, m = 24, 20
    A = f(np.arange(n, dtype=float)[:, None], np.arange(m, dtype=float)[None, :])
    U = oracle.zoom_to(A, 3 * n, 3 * m)
    assert U.shape == (3 * n, 3 * m)
    rows, y = _interior(n, 3 * n, 6.0)
    cols, x = _interior(m, 3 * m, 6.0)
    want = f(y[rows][:, None], x[cols][None, :])
    assert np.abs(U[np.ix_(rows, cols)] - want).max() < 1e-10
    # the corners are the input's corners
    assert U[0, 0] == pytest.approx(A[0, 0], abs=1e-12)
    assert U[-1, -1] == pytest.approx(A[-1, -1], abs=1e-12)
