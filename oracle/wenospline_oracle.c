/*
 * FP64 CPU oracle for the 1-D WENO interpolant of Sec. 2 and the separable
 * "tensor WENO" resampling of Sec. 3.3 (arXiv 2312.00229).
 *
 * TEST INFRASTRUCTURE ONLY (see wdweno_oracle.c): used by the test-suite and
 * the benchmark's CPU leg, never by the CUDA library.
 *
 *   Sec. 2, Eqs. (Tocnost), (Stencil): p_i is the quadratic through
 *     x_{i-1}, x_i, x_{i+1}; p_{i+1} through x_i, x_{i+1}, x_{i+2}.
 *   Eq. (PolinomZaVelikiStencil): the cubic q through the four nodes equals
 *     C_{i,0}(x) p_i(x) + C_{i,1}(x) p_{i+1}(x) on [x_i, x_{i+1}] with linear,
 *     non-negative C_{i,s} summing to one; solved here from that identity.
 *   Eq. (TezinskiPolinom1d): u_i(x) = omega_0 p_i(x) + omega_1 p_{i+1}(x).
 *   Eq. (IzrazOmega): omega_s = alpha_s / (alpha_0 + alpha_1),
 *     alpha_s = C_{i,s}(x) / (eps_h + SI_{i,s})^beta, eps_h = K_eps h^2.
 *   SI_{i,s} = sum_{l=1,2} int_{x_i}^{x_{i+1}} h^{2l-1} (p_{i+s}^{(l)})^2 dx.
 *   Sec. 3.3, WENO spline w(V, x) = u_i(v_{i-1..i+2}, x) on [x_i, x_{i+1}],
 *     evaluated on the grid x_j = j (n-1)/(n*-1), j = 0..n*-1; Eq. (tensor):
 *     z_k = w(A(:,k), y), U(x, y) = w(Z, x).
 * Reading: samples outside 0..n-1 are clamped to the edge (the library's
 * boundary rule); the cell index is min(floor(x), n-2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "wdweno_oracle.h"

/* Lagrange form of the quadratic through (t0,v0), (t1,v1), (t2,v2) and its
 * first two derivatives at t. */
static void quad_eval(const double tn[3], const double v[3], double t, double* p, double* dp,
                      double* d2p) {
  double val = 0.0, d1 = 0.0, d2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double den = (tn[a] - tn[b]) * (tn[a] - tn[c]);
    /* L_a(t) = (t - tb)(t - tc) / den */
    val += v[a] * (t - tn[b]) * (t - tn[c]) / den;
    d1 += v[a] * ((t - tn[b]) + (t - tn[c])) / den;
    d2 += v[a] * 2.0 / den;
  }
  *p = val;
  *dp = d1;
  *d2p = d2;
}

/* SI over [0, 1] in units of h (the h^{2l-1} factors cancel the change of
 * variable x = x_i + h t): int_0^1 p'(t)^2 + p''(t)^2 dt, by 3-point
 * Gauss-Legendre, exact for the quadratic integrand. */
static double si_unit(const double tn[3], const double v[3]) {
  static const double gx[3] = {-0.7745966692414834, 0.0, 0.7745966692414834};
  static const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  double acc = 0.0;
  for (int q = 0; q < 3; ++q) {
    double t = 0.5 + 0.5 * gx[q];
    double p, dp, d2p;
    quad_eval(tn, v, t, &p, &dp, &d2p);
    acc += 0.5 * gw[q] * (dp * dp + d2p * d2p);
  }
  return acc;
}

double oracle_weno1d_cell(const double v4[4], double t, double beta, double k_eps, double h) {
  /* nodes of the cell [x_i, x_{i+1}] in units of h: x_{i-1} = -1 ... x_{i+2} = 2 */
  const double tl[3] = {-1.0, 0.0, 1.0}, tr[3] = {0.0, 1.0, 2.0};
  const double vl[3] = {v4[0], v4[1], v4[2]}, vr[3] = {v4[1], v4[2], v4[3]};
  double p0, p1, d, dd;
  quad_eval(tl, vl, t, &p0, &d, &dd);
  quad_eval(tr, vr, t, &p1, &d, &dd);
  /* Linear C_0 + C_1 = 1 with C_0 (t+1) + C_1 (t-2) = 0 (the cubic terms of
   * q - p_i and q - p_{i+1} cancel), i.e. C_0 = (2-t)/3, C_1 = (1+t)/3. */
  const double C0 = (2.0 - t) / 3.0, C1 = 1.0 - C0;
  const double eps_h = k_eps * h * h;
  const double a0 = C0 / pow(eps_h + si_unit(tl, vl), beta);
  const double a1 = C1 / pow(eps_h + si_unit(tr, vr), beta);
  return (a0 * p0 + a1 * p1) / (a0 + a1);
}

static double sample_clamped(const double* V, int64_t n, int64_t stride, int64_t i) {
  if (i < 0) i = 0;
  if (i > n - 1) i = n - 1;
  return V[i * stride];
}

/* w(V, x) for x in [0, n-1]. */
double oracle_weno_spline(const double* V, int64_t n, int64_t stride, double x, double beta,
                          double k_eps, double h) {
  if (n == 1) return V[0];
  int64_t i = (int64_t)floor(x);
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  const double t = x - (double)i;
  double v4[4];
  for (int q = 0; q < 4; ++q) v4[q] = sample_clamped(V, n, stride, i - 1 + q);
  return oracle_weno1d_cell(v4, t, beta, k_eps, h);
}

/* Eq. (tensor): resample one n x m plane to n_out x m_out on the
 * endpoint-aligned grids.  z_k = w(A(:, k), y) first, then w(Z, x). */
int oracle_tensor_resample(const double* A, int64_t n, int64_t m, double* U, int64_t n_out,
                           int64_t m_out, double beta, double k_eps, double h) {
  if (!A || !U || n < 1 || m < 1 || n_out < 1 || m_out < 1) return ORACLE_EINVAL;
  double* Z = (double*)malloc(sizeof(double) * (size_t)m);
  if (!Z) return ORACLE_ENOMEM;
  for (int64_t r = 0; r < n_out; ++r) {
    const double y = n_out > 1 ? (double)r * (double)(n - 1) / (double)(n_out - 1) : 0.0;
    for (int64_t k = 0; k < m; ++k) Z[k] = oracle_weno_spline(A + k, n, m, y, beta, k_eps, h);
    for (int64_t c = 0; c < m_out; ++c) {
      const double x = m_out > 1 ? (double)c * (double)(m - 1) / (double)(m_out - 1) : 0.0;
      U[r * m_out + c] = oracle_weno_spline(Z, m, 1, x, beta, k_eps, h);
    }
  }
  free(Z);
  return ORACLE_OK;
}
