"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an independent quadrature or linear filter, a polynomial the scheme must
reproduce, a symmetry, or the numbers printed in Tables 1 and 2 of
arXiv 2312.00229.  None needs a GPU.
"""
import math
import os

import numpy as np
import pytest
import torch
from scipy import integrate, ndimage

import oracle
from oracle import wdweno_torch as wt
from paper_2312_00229_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


# --------------------------------------------------------------------------
# Per-direction primitives: Eq. (p) and Eq. (2Dsmoothness)
# --------------------------------------------------------------------------
def _si_by_quadrature(n0, n1, n2, step, scale):
    """Eq. (2Dsmoothness) by adaptive quadrature of the interpolating
    polynomial, built with numpy.polyfit in physical arc length."""
    xs = np.array([-1.0, 1.0, 3.0]) * step
    coef = np.polyfit(xs, [n0, n1, n2], 2)
    d1, d2 = np.polyder(coef, 1), np.polyder(coef, 2)
    i1 = integrate.quad(lambda x: np.polyval(d1, x) ** 2, -step, step, epsabs=1e-14)[0]
    i2 = integrate.quad(lambda x: np.polyval(d2, x) ** 2, -step, step, epsabs=1e-14)[0]
    return scale * i1 + scale ** 3 * i2, np.polyval(coef, 0.0)


@pytest.mark.parametrize("h", [1.0, 0.1])
def test_directional_si_matches_quadrature(h):
    for _ in range(50):
        n0, n1, n2 = RNG.normal(size=3)
        # diagonal: |d| = h / sqrt(2), node spacing sqrt(2) h = 2 |d|
        step = h / math.sqrt(2.0)
        si_q, p_q = _si_by_quadrature(n0, n1, n2, step, 2 * step)
        p, si = oracle.directional(n0, n1, n2, 2.0)
        assert abs(si - si_q) <= 1e-10 * max(1.0, abs(si_q))
        assert abs(p - p_q) <= 1e-12 * max(1.0, abs(p_q))
        # literal scaling on an axis: |d| = h / 2, length scale sqrt(2) h
        step = h / 2.0
        si_q, _ = _si_by_quadrature(n0, n1, n2, step, math.sqrt(2.0) * h)
        _, si = oracle.directional(n0, n1, n2, math.sqrt(2.0) * h / step)
        assert abs(si - si_q) <= 1e-10 * max(1.0, abs(si_q))


def test_directional_closed_form():
    """SI = (N1-N0)^2 + 13/12 (N0 - 2 N1 + N2)^2 and p = 3/8 N0 + 3/4 N1 - 1/8 N2."""
    for _ in range(50):
        n0, n1, n2 = RNG.normal(size=3)
        p, si = oracle.directional(n0, n1, n2, 2.0)
        assert abs(p - (3 / 8 * n0 + 3 / 4 * n1 - 1 / 8 * n2)) < 1e-14
        assert abs(si - ((n1 - n0) ** 2 + 13 / 12 * (n0 - 2 * n1 + n2) ** 2)) < 1e-12


def test_directional_quadratic_exact():
    """The stencil quadratic reproduces any quadratic at the centre."""
    for _ in range(20):
        a, b, c = RNG.normal(size=3)
        q = lambda t: a + b * t + c * t * t
        p, _ = oracle.directional(q(-1.0), q(1.0), q(3.0))
        assert abs(p - a) < 1e-13


# --------------------------------------------------------------------------
# Whole-method invariants
# --------------------------------------------------------------------------
SHAPES = [(1, 1), (1, 7), (6, 1), (2, 2), (3, 5), (9, 14), (17, 12)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("beta", [0.0, 1.0, 2.0, 3.5])
def test_constant_image_preserved(shape, beta):
    for mode in (oracle.OUT_2N, oracle.OUT_2N_MINUS_1):
        A = np.full(shape, 0.731)
        U = oracle.zoom2x(A, beta=beta, out_mode=mode)
        assert np.all(U == 0.731) or np.abs(U - 0.731).max() < 1e-15


@pytest.mark.parametrize("shape", SHAPES)
def test_original_samples_kept(shape):
    A = RNG.random(shape)
    for mode in (oracle.OUT_2N, oracle.OUT_2N_MINUS_1):
        U = oracle.zoom2x(A, out_mode=mode)
        assert np.array_equal(U[::2, ::2], A)


def test_2n_minus_1_is_crop_of_2n():
    A = RNG.random((2, 11, 8))
    U2 = oracle.zoom2x(A, out_mode=oracle.OUT_2N)
    U1 = oracle.zoom2x(A, out_mode=oracle.OUT_2N_MINUS_1)
    assert np.array_equal(U2[..., :-1, :-1], U1)


def test_ghost_width_independent():
    A = RNG.random((13, 10))
    assert np.array_equal(oracle.zoom2x(A, ghost=6), oracle.zoom2x(A, ghost=11))


def _poly_grid(n, m, coeffs, h, ghost):
    """Samples of sum c_ab x^a y^b on an (n + 2g) x (m + 2g) grid (x = row)."""
    x = (np.arange(-ghost, n + ghost) * h)[:, None]
    y = (np.arange(-ghost, m + ghost) * h)[None, :]
    return sum(c * x ** a * y ** b for (a, b), c in coeffs.items())


@pytest.mark.parametrize("beta", [0.0, 1.0, 2.0])
def test_quadratics_reproduced_exactly(beta):
    """Total degree <= 2: every directional quadratic is exact, so any convex
    combination is (Sec. 3, Eq. p and Eq. 2dKombinacija)."""
    h = 0.37
    coeffs = {(0, 0): 0.3, (1, 0): -0.7, (0, 1): 0.4, (2, 0): 0.9, (1, 1): -1.3, (0, 2): 0.55}
    n, m, g = 12, 15, 6
    A = _poly_grid(n, m, coeffs, h, g)
    U = oracle.zoom2x(A, beta=beta, h=h, out_mode=oracle.OUT_2N_MINUS_1)
    xf = (np.arange(2 * (n + 2 * g) - 1) * h / 2 - g * h)[:, None]
    yf = (np.arange(2 * (m + 2 * g) - 1) * h / 2 - g * h)[None, :]
    T = sum(c * xf ** a * yf ** b for (a, b), c in coeffs.items())
    # interior: footprint (4 before, 5 after) clear of the clamped ghosts
    s = slice(2 * 5, -2 * 5)
    assert np.abs(U[s, s] - T[s, s]).max() < 1e-12


def test_cubics_reproduced_at_beta0():
    """Prop. 1: with ideal weights the scheme is a blend of cubic
    interpolants along lines and reproduces total-degree-3 polynomials."""
    h = 0.29
    coeffs = {(3, 0): 0.7, (2, 1): -0.4, (1, 2): 1.1, (0, 3): -0.8, (1, 1): 0.5, (0, 0): 0.2}
    n, m, g = 11, 13, 6
    A = _poly_grid(n, m, coeffs, h, g)
    U = oracle.zoom2x(A, beta=0.0, h=h, out_mode=oracle.OUT_2N_MINUS_1)
    xf = (np.arange(2 * (n + 2 * g) - 1) * h / 2 - g * h)[:, None]
    yf = (np.arange(2 * (m + 2 * g) - 1) * h / 2 - g * h)[None, :]
    T = sum(c * xf ** a * yf ** b for (a, b), c in coeffs.items())
    s = slice(2 * 5, -2 * 5)
    assert np.abs(U[s, s] - T[s, s]).max() < 1e-11
    U2 = oracle.zoom2x(A, beta=2.0, h=h, out_mode=oracle.OUT_2N_MINUS_1)
    assert np.abs(U2[s, s] - T[s, s]).max() > 1e-6  # not exact for beta > 0


def test_beta0_is_separately_written_linear_filter():
    """beta = 0 makes every weight 1/4: x points average the two diagonal
    midpoint cubics, + points the row/column midpoint cubics.  Written here
    with scipy.ndimage on the clamp-padded image, independently of the
    oracle's loops."""
    A = RNG.random((19, 23))
    n, m = A.shape
    w = np.array([-1.0, 9.0, 9.0, -1.0]) / 16.0  # cubic at the midpoint
    Ap = np.pad(A, 8, mode="edge")
    # x point between (i, j) and (i+1, j+1): diagonal taps (i-1..i+2, j-1..j+2)
    k1 = np.zeros((4, 4)); k2 = np.zeros((4, 4))
    for t in range(4):
        k1[t, t] = w[t]
        k2[t, 3 - t] = w[t]
    # ndimage.correlate centres a 4x4 kernel at index (2, 2); shift so tap 1
    # (the (i, j) sample) sits on the output index.
    X = 0.5 * ndimage.correlate(Ap, k1, mode="nearest", origin=(-1, -1)) \
        + 0.5 * ndimage.correlate(Ap, k2, mode="nearest", origin=(-1, -1))
    F = np.zeros((2 * Ap.shape[0], 2 * Ap.shape[1]))
    F[::2, ::2] = Ap
    F[1::2, 1::2] = X
    # + points: (even, odd) -> row cubic of samples + column cubic of x values
    Fp = F.copy()
    R, C = F.shape
    for P in range(6, R - 6):
        for Q in range(6, C - 6):
            if (P + Q) % 2 == 1:
                row = sum(w[t] * F[P, Q - 3 + 2 * t] for t in range(4))
                col = sum(w[t] * F[P - 3 + 2 * t, Q] for t in range(4))
                Fp[P, Q] = 0.5 * row + 0.5 * col
    T = Fp[16:16 + 2 * n, 16:16 + 2 * m]
    U = oracle.zoom2x(A, beta=0.0)
    assert np.abs(U - T).max() < 1e-13


def _d4(U, op):
    return {"flip0": U[::-1, :], "flip1": U[:, ::-1], "T": U.T}[op]


@pytest.mark.parametrize("op", ["flip0", "flip1", "T"])
def test_d4_equivariance(op):
    """The direction sets of both phases and the neighbour sets of D are
    closed under flips and the transpose, and so is clamp extension."""
    A = RNG.random((9, 13)) if op != "T" else RNG.random((11, 11))
    U = oracle.zoom2x(A, out_mode=oracle.OUT_2N_MINUS_1)
    Ut = oracle.zoom2x(np.ascontiguousarray(_d4(A, op)), out_mode=oracle.OUT_2N_MINUS_1)
    assert np.abs(_d4(U, op) - Ut).max() < 1e-13


def test_dependency_footprint():
    """Output quad (a, b) depends on input rows a-4..a+5 and columns
    b-4..b+5, and on all of them (brute-force perturbation)."""
    n = m = 24
    A = RNG.random((n, m))
    U0 = oracle.zoom2x(A)
    i0, j0 = 12, 11
    B = A.copy(); B[i0, j0] += 1e-3
    D = np.abs(oracle.zoom2x(B) - U0).reshape(n, 2, m, 2).max(axis=(1, 3))
    a, b = np.nonzero(D > 0)
    assert a.min() == i0 - 5 and a.max() == i0 + 4
    assert b.min() == j0 - 5 and b.max() == j0 + 4


def test_torch_restatement_matches_c_oracle():
    for shape in [(1, 1), (3, 1), (5, 8), (16, 9)]:
        for si in (oracle.SI_NORMALIZED, oracle.SI_LITERAL):
            for beta in (0.0, 1.0, 2.0, 2.5):
                A = RNG.random((2,) + shape)
                Uc = oracle.zoom2x(A, beta=beta, si_scale=si, h=0.5)
                Ut = wt.zoom2x(torch.from_numpy(A), beta=beta, si_scale=si, h=0.5).numpy()
                assert np.abs(Uc - Ut).max() < 1e-12
    # both readings of the neighbour weight, and a mixed one, per phase
    A = RNG.random((2, 7, 10))
    for nc in ((0.25, 0.25), (0.25, 0.125), (0.0, 0.5)):
        Uc = oracle.zoom2x(A, h=1.0, nbr_c=nc)
        Ut = wt.zoom2x(torch.from_numpy(A), h=1.0, nbr_c=nc).numpy()
        assert np.abs(Uc - Ut).max() < 1e-12


def test_encode_u8_half_even():
    vals = np.array([0.5, 1.5, 2.5, 254.5, -3.0, 300.0, 127.49999]) / 255.0
    assert oracle.encode_u8(vals).tolist() == [0, 2, 2, 254, 0, 255, 127]


# --------------------------------------------------------------------------
# Tables 1 and 2 (Sec. 4.1, 4.2)
# --------------------------------------------------------------------------
def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def _table_run(k, f, beta, G=8, nbr_c=None):
    """Row k of the tables: fine spacing 2^-k, coarse spacing 2^(1-k) on
    [-1, 1]^2, samples outside the square taken from f."""
    hc = 2.0 ** (1 - k)
    n = int(round(2 / hc)) + 1
    xe = -1 + hc * np.arange(-G, n + G)
    A = f(xe[:, None], xe[None, :])
    U = oracle.zoom2x(A, beta=beta, h=hc, out_mode=oracle.OUT_2N_MINUS_1, nbr_c=nbr_c)
    r = 2 * n - 1
    U = U[2 * G:2 * G + r, 2 * G:2 * G + r]
    xf = -1 + (hc / 2) * np.arange(r)
    return U - f(xf[:, None], xf[None, :]), xf


def _smooth(x, y):
    return 1.0 / (x * x + y * y + 1.0)


def test_table1_convergence():
    T = _load("table1_convergence.txt")
    linf, l2 = [], []
    for k in range(0, 8):
        E, _ = _table_run(k, _smooth, beta=1.0)
        linf.append(np.abs(E).max())
        l2.append(np.sqrt(np.mean(E ** 2)))
    linf, l2 = np.array(linf), np.array(l2)
    # first row and the asymptotic rows: L_inf within 1.5 %
    assert abs(linf[0] / T[0, 1] - 1) < 0.015
    for k in range(4, 8):
        assert abs(linf[k] / T[k, 1] - 1) < 0.015, (k, linf[k], T[k, 1])
    # row h = 0.5 is the one whose value the neighbour weight of D decides:
    # reproduced to 0.5 % (measured 0.01 %) under the h^2/8 reading
    assert abs(linf[1] / T[1, 1] - 1) < 0.005, (linf[1], T[1, 1])
    # rows h = 0.25, 0.125: within 6 % (measured +5.4 %, +3.6 %; no reading of
    # the weight brings them closer than +3 %)
    for k in range(2, 4):
        assert abs(linf[k] / T[k, 1] - 1) < 0.06, (k, linf[k], T[k, 1])
    # L_2 (root mean square over the fine grid): within 12 % from row 2 on
    for k in range(2, 8):
        assert abs(l2[k] / T[k, 3] - 1) < 0.12, (k, l2[k], T[k, 3])
    # orders -> 4 (Theorem 1; Table 1 orders 3.89..3.92 for these rows)
    orders = np.log2(linf[:-1] / linf[1:])
    for k in range(5, 8):
        assert abs(orders[k - 1] - T[k, 2]) < 0.05, (k, orders[k - 1], T[k, 2])


@pytest.mark.parametrize("nbr_c,ok", [((0.125, 0.125), True), ((0.25, 0.25), False),
                                       ((0.25, 0.125), False), ((0.125, 0.25), False)])
def test_table1_row_h05_decides_the_neighbour_weight(nbr_c, ok):
    """Eq. (2DsmoothnessFinal) and Eq. (tezine) print the neighbour weight of
    D as h^2/4; the proof of Theorem 1 (Eq. DDiffOrder) writes h^2/8.  Only
    Table 1's coarse rows depend on it; at h = 0.5 (coarse spacing 1, where
    the weight is largest against the other terms) h^2/8 in both phases
    gives L_inf 1.3302e-1 against the printed 1.33e-1, and h^2/4 in either
    phase misses by 8-18 %.  The pin that passes for the default reading must
    fail for each of the others."""
    T = _load("table1_convergence.txt")
    E, _ = _table_run(1, _smooth, beta=1.0, nbr_c=nbr_c)
    dev = abs(np.abs(E).max() / T[1, 1] - 1)
    assert (dev < 0.005) == ok, (nbr_c, dev)


def test_oracle_default_neighbour_weight_is_h2_over_8():
    A = np.random.default_rng(3).random((9, 11))
    for h in (1.0, 0.5):
        assert np.array_equal(oracle.zoom2x(A, h=h),
                              oracle.zoom2x(A, h=h, nbr_c=(0.125, 0.125)))
        assert not np.array_equal(oracle.zoom2x(A, h=h),
                                  oracle.zoom2x(A, h=h, nbr_c=(0.25, 0.25)))


def _disc(x, y):
    return _smooth(x, y) + (x < 0)


@pytest.mark.parametrize("col,beta,right", [(0, 2.0, False), (1, 0.0, True), (2, 1.0, True),
                                            (3, 2.0, True)])
def test_table2_discontinuity_orders(col, beta, right):
    T = _load("table2_discontinuity.txt")
    errs = []
    for k in range(3, 9):
        E, xf = _table_run(k, _disc, beta=beta)
        if right:
            E = E[xf >= 0, :]
        errs.append((np.abs(E).max(), np.sqrt(np.mean(E ** 2))))
    errs = np.array(errs)
    o_inf = np.log2(errs[:-1, 0] / errs[1:, 0])
    o_2 = np.log2(errs[:-1, 1] / errs[1:, 1])
    # table rows for k = 4..8 are rows 3..7 of the fixture
    tab = T[3:8, 1 + 2 * col: 3 + 2 * col]
    assert np.all(np.abs(o_inf - tab[:, 0]) < 0.35), (o_inf, tab[:, 0])
    assert np.all(np.abs(o_2 - tab[:, 1]) < 0.2), (o_2, tab[:, 1])
    # Theorem 1: order >= min(3, 2 beta) - slack right of the jump, beta >= 3/2
    if right and beta >= 1.5:
        assert np.all(o_inf[-3:] > 3.4)


def test_config1_smooth_part_converges_at_order4():
    """sin(2 pi x) cos(3 pi y) at pixel centres, clamp extension, interior
    points: order 4 under refinement (Theorem 1)."""
    errs = []
    for n in (32, 64, 128, 256):
        A = scenes.analytic_step(n, with_step=False)
        U = oracle.zoom2x(A, h=1.0 / n)
        T = scenes.analytic_step_truth(2 * n, 2 * n, n, with_step=False)
        s = slice(2 * 6, 2 * (n - 6))
        errs.append(np.abs(U[s, s] - T[s, s]).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > 3.7, orders


# --------------------------------------------------------------------------
# Edges: no new overshoot (the tolerance was set from the oracle and frozen)
# --------------------------------------------------------------------------
def _step(n, angle_deg, offset=0.37):
    i, j = np.mgrid[0:n, 0:n].astype(float)
    a = np.deg2rad(angle_deg)
    return ((j - n / 2) * np.cos(a) + (i - n / 2) * np.sin(a) >= offset).astype(float)


@pytest.mark.parametrize("angle", [0, 45, 30, 16.7, 63])
def test_step_edge_overshoot(angle):
    A = _step(40, angle)
    U2 = oracle.zoom2x(A, beta=2.0, out_mode=oracle.OUT_2N_MINUS_1)
    U0 = oracle.zoom2x(A, beta=0.0, out_mode=oracle.OUT_2N_MINUS_1)
    over2 = max(U2.max() - 1.0, -U2.min())
    over0 = max(U0.max() - 1.0, -U0.min())
    assert over2 <= 0.02          # frozen: measured <= 0.0125 of the jump
    assert over2 <= 0.45 * over0  # well under the linear (beta = 0) scheme


def test_config1_step_no_overshoot():
    n = 64
    A = scenes.analytic_step(n)
    U = oracle.zoom2x(A, beta=2.0, h=1.0 / n)
    Ap = np.pad(A, 2, mode="edge")
    lo = np.full((n, n), np.inf); hi = np.full((n, n), -np.inf)
    for di in range(-1, 3):
        for dj in range(-1, 3):
            w = Ap[2 + di:2 + di + n, 2 + dj:2 + dj + n]
            lo = np.minimum(lo, w); hi = np.maximum(hi, w)
    Q = U.reshape(n, 2, n, 2)
    over = np.maximum(Q - hi[:, None, :, None], 0).max()
    under = np.maximum(lo[:, None, :, None] - Q, 0).max()
    assert over < 0.002 and under < 0.002  # frozen: measured 1.2e-3


# --------------------------------------------------------------------------
# The FP64 reference gradient (autograd of the torch restatement)
# --------------------------------------------------------------------------
def test_reference_gradient_matches_finite_differences():
    """Central differences (step 1e-6) of the C oracle against autograd of
    the independent torch restatement, on a 16 x 16 crop."""
    n = 16
    A = RNG.random((n, n))
    W = RNG.normal(size=(2 * n, 2 * n))
    At = torch.from_numpy(A.copy()).requires_grad_(True)
    loss = (wt.zoom2x(At) * torch.from_numpy(W)).sum()
    (g,) = torch.autograd.grad(loss, At)
    g = g.numpy()
    step = 1e-6
    worst = 0.0
    for (i, j) in [(0, 0), (0, 7), (5, 5), (8, 15), (15, 15), (3, 12), (11, 2)]:
        Ap, Am = A.copy(), A.copy()
        Ap[i, j] += step
        Am[i, j] -= step
        fd = ((oracle.zoom2x(Ap) * W).sum() - (oracle.zoom2x(Am) * W).sum()) / (2 * step)
        worst = max(worst, abs(fd - g[i, j]) / max(1.0, abs(fd)))
    assert worst < 1e-6, worst


def test_reference_gradcheck_tiny():
    A = torch.from_numpy(RNG.random((1, 5, 6))).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a: wt.zoom2x(a, beta=2.0), (A,), eps=1e-6,
                                    atol=1e-7, rtol=1e-5)


@pytest.mark.parametrize("mode", [oracle.OUT_2N, oracle.OUT_2N_MINUS_1])
def test_banded_oracle_equals_whole_image(mode):
    """The banded form (windows with the 4/5-row footprint margins, used to
    time the oracle on all host cores) gives the whole-image result bit for
    bit, for bands down to one quad row."""
    rng = np.random.default_rng(5)
    for shape in [(1, 1, 1), (2, 7, 9), (3, 37, 53), (1, 40, 17)]:
        A = rng.random(shape)
        whole = oracle.zoom2x(A, out_mode=mode)
        for band_rows, threads in [(1, 2), (3, 3), (16, 0), (100, 1)]:
            got = oracle.zoom2x_banded(A, band_rows=band_rows, threads=threads, out_mode=mode)
            assert np.array_equal(got, whole), (shape, band_rows)
