"""Vectorised float64 PyTorch restatement of the WD WENO 2x zoom.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  It exists so that autograd
can produce the FP64 reference gradient of the method; the test-suite checks it
against the C oracle (``wdweno_oracle.c``) to ~1e-13 and its gradient against
central finite differences of the C oracle.

It is written independently of the C oracle: where the C code loops over a
fine-grid array and builds each quadratic from divided differences, this code
works on four interleaved sub-lattices of the fine grid with whole-array
slicing and uses the closed forms below.

Paper: Crnkovic, Skific, Bosner, arXiv 2312.00229.
  Sec. 3, Fig. inputdata: fine point (P, Q) is an input sample if P, Q are
  both even, an "x" point if both odd, a "+" point otherwise.
  Eq. (p): p = l0 N0 + l1 N1 + l2 N2, Lagrange weights of the nodes at
  t = -1, 1, 3 (units of one fine step along gamma) taken at t = 0.
  Eq. (2Dsmoothness) with node spacing L and nodes N0, N1, N2: writing
  g = N1 - N0 and s = N0 - 2 N1 + N2, the quadratic on [N0-node, N1-node] in
  the unit coordinate xi is N0 + g xi + s xi (xi - 1) / 2, so
  int_0^1 p_xi^2 = g^2 + s^2 / 12 and int_0^1 p_xixi^2 = s^2.  With the
  length scale c in place of L the l-th term scales by (c / L)^(2l - 1):
  SI = (c/L) (g^2 + s^2/12) + (c/L)^3 s^2.
  Eqs. (2DsmoothnessFinal), (tezine), (alpha), (IzrazOmega2d), (2dKombinacija),
  (IzrazOmega2dRavno), (2dKombinacijaRavno).
"""
from __future__ import annotations

import math

import torch

SI_NORMALIZED, SI_LITERAL = 0, 1
OUT_2N, OUT_2N_MINUS_1 = 0, 1


def _lagrange_at_zero(nodes):
    """Lagrange basis weights of `nodes` evaluated at 0."""
    w = []
    for i, ti in enumerate(nodes):
        num, den = 1.0, 1.0
        for j, tj in enumerate(nodes):
            if j != i:
                num *= (0.0 - tj)
                den *= (ti - tj)
        w.append(num / den)
    return w


_NODES = (-1.0, 1.0, 3.0)
_LW = _lagrange_at_zero(_NODES)  # (3/8, 3/4, -1/8)


class _Lattice:
    """Values on one parity class of the fine grid.

    Entry [r, c] of ``t`` sits at fine position (P0 + 2 r, Q0 + 2 c)."""

    def __init__(self, t, P0, Q0):
        self.t, self.P0, self.Q0 = t, P0, Q0

    def at(self, P, Q, R, C):
        """Values at fine positions (P + 2 r, Q + 2 c), r < R, c < C."""
        dr, dc = P - self.P0, Q - self.Q0
        assert dr % 2 == 0 and dc % 2 == 0, "parity mismatch"
        r0, c0 = dr // 2, dc // 2
        rows, cols = self.t.shape[-2:]
        if r0 < 0 or c0 < 0 or r0 + R > rows or c0 + C > cols:
            raise IndexError(f"lattice read out of range: origin ({P},{Q}) size ({R},{C})")
        return self.t[..., r0:r0 + R, c0:c0 + C]


class _FineGrid:
    def __init__(self):
        self.lat = {}

    def put(self, lattice):
        self.lat[(lattice.P0 % 2, lattice.Q0 % 2)] = lattice

    def at(self, P, Q, R, C):
        return self.lat[(P % 2, Q % 2)].at(P, Q, R, C)


def _phase(grid, targets, dirs, nbrs, c_over_L, prm):
    """One WD WENO phase on the target lattices.

    targets: list of (P0, Q0, R, C) target regions (one per parity class)
    Returns lattices of new values, each shrunk by one neighbour ring."""
    beta, eps_h, nbr_w = prm
    # p and SI for every direction on every target region.
    P_, SI = {}, {}
    for ti, (P0, Q0, R, C) in enumerate(targets):
        for k, (dP, dQ) in enumerate(dirs):
            n0 = grid.at(P0 - dP, Q0 - dQ, R, C)
            n1 = grid.at(P0 + dP, Q0 + dQ, R, C)
            n2 = grid.at(P0 + 3 * dP, Q0 + 3 * dQ, R, C)
            P_[ti, k] = _LW[0] * n0 + _LW[1] * n1 + _LW[2] * n2
            g = n1 - n0
            s = n0 - 2.0 * n1 + n2
            SI[ti, k] = c_over_L * (g * g + s * s / 12.0) + c_over_L ** 3 * (s * s)
    # SI lattices per direction, so neighbours of any parity can be read.
    si_grids = []
    for k in range(4):
        fg = _FineGrid()
        for ti, (P0, Q0, R, C) in enumerate(targets):
            fg.put(_Lattice(SI[ti, k], P0, Q0))
        si_grids.append(fg)
    out = []
    for ti, (P0, Q0, R, C) in enumerate(targets):
        # Shrink by one lattice step on each side (neighbour offsets reach 2
        # fine steps in phase 1, 1 in phase 2; one lattice step covers both).
        Pn, Qn, Rn, Cn = P0 + 2, Q0 + 2, R - 2, C - 2
        num, den = 0.0, 0.0
        for k in range(4):
            si_c = si_grids[k].at(Pn, Qn, Rn, Cn)
            nsum = 0.0
            for (oP, oQ) in nbrs:
                nsum = nsum + si_grids[k].at(Pn + oP, Qn + oQ, Rn, Cn)
            D = si_c + nbr_w * nsum
            alpha = 0.5 / (eps_h + D) ** beta
            num = num + alpha * P_[ti, k][..., 1:1 + Rn, 1:1 + Cn]
            den = den + alpha
        out.append(_Lattice(num / den, Pn, Qn))
    return out


def _extend_index(n, G):
    return torch.arange(-G, n + G).clamp(0, n - 1)


def zoom2x(A: torch.Tensor, beta=2.0, k_eps=1e-8, h=1.0, si_scale=SI_NORMALIZED,
           out_mode=OUT_2N, ghost=6, nbr_c=(0.125, 0.125)) -> torch.Tensor:
    """WD WENO 2x zoom of ``A`` (..., n, m) with clamp-to-edge extension.

    ``nbr_c`` = (phase 1, phase 2) coefficients c of the neighbour weight
    c h^2 of D.  The definitions (Eqs. 2DsmoothnessFinal, tezine) print
    h^2/4, the proof of Theorem 1 (Eq. DDiffOrder) h^2/8; h^2/8 reproduces
    Table 1's coarse row, so it is the default.

    Differentiable with respect to ``A``; intended for float64."""
    n, m = A.shape[-2:]
    G = int(ghost)
    assert G >= 5
    E = A[..., _extend_index(n, G), :][..., :, _extend_index(m, G)]
    ne, me = n + 2 * G, m + 2 * G
    eps_h = k_eps * h * h
    prm1 = (beta, eps_h, float(nbr_c[0]) * h * h)
    prm2 = (beta, eps_h, float(nbr_c[1]) * h * h)

    grid = _FineGrid()
    grid.put(_Lattice(E, 0, 0))

    # Phase 1: "x" points, gamma_k = pi/4 + k pi/2, one fine step (+-1, +-1).
    diag = [(1, 1), (-1, 1), (-1, -1), (1, -1)]
    diag_nbr = [(0, 2), (2, 0), (0, -2), (-2, 0)]
    # x lattice positions P = 3, 5, ..., 2 ne - 5 (stencil reaches 3 fine steps).
    R1, C1 = ne - 3, me - 3
    # c/L: normalized c = L; literal c = sqrt(2) h = L on diagonals.
    r1 = 1.0
    (X,) = _phase(grid, [(3, 3, R1, C1)], diag, diag_nbr, r1, prm1)
    grid.put(X)

    # Phase 2: "+" points, gamma_k = k pi/2, one fine step (+-1, 0) / (0, +-1).
    axis = [(1, 0), (0, 1), (-1, 0), (0, -1)]
    axis_nbr = [(1, 1), (-1, -1), (-1, 1), (1, -1)]
    # x values exist on fine rows [x0, x1] and columns [y0, y1] (odd).  The
    # axis stencil of a "+" point reaches 3 fine steps along the axis that
    # crosses x points; the D of Eq. (tezine) reads the other "+" class one
    # diagonal step away, so each class keeps one extra step of margin
    # across that axis.
    xr, xc = X.t.shape[-2:]
    x0, y0 = X.P0, X.Q0
    # c/L: normalized c = L; literal c = sqrt(2) h against L = h on axes.
    r2 = 1.0 if si_scale == SI_NORMALIZED else math.sqrt(2.0)
    targets = [
        (x0 + 3, y0 + 2, xr - 3, xc - 2),   # (even, odd): rows x0+3..x1-3
        (x0 + 2, y0 + 3, xr - 2, xc - 3),   # (odd, even): cols y0+3..y1-3
    ]
    plus_e, plus_s = _phase(grid, targets, axis, axis_nbr, r2, prm2)

    # Assemble the 2n x 2m crop; fine output (p, q) is fine (p + 2G, q + 2G).
    P0 = 2 * G
    o = grid.lat[(0, 0)].at(P0, P0, n, m)
    x = X.at(P0 + 1, P0 + 1, n, m)
    e = plus_e.at(P0, P0 + 1, n, m)
    s = plus_s.at(P0 + 1, P0, n, m)
    top = torch.stack([o, e], dim=-1)      # (..., n, m, 2)
    bot = torch.stack([s, x], dim=-1)
    quad = torch.stack([top, bot], dim=-3)  # (..., n, 2, m, 2)
    U = quad.reshape(*A.shape[:-2], 2 * n, 2 * m)
    if out_mode == OUT_2N_MINUS_1:
        U = U[..., : 2 * n - 1, : 2 * m - 1]
    return U
