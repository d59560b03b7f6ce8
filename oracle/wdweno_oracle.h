/*
 * FP64 CPU oracle for the WD WENO 2x zoom (arXiv 2312.00229, Sec. 3).
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the CUDA library.
 */
#ifndef WDWENO_ORACLE_H
#define WDWENO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORACLE_OK = 0,
  ORACLE_EINVAL = -1,
  ORACLE_ENOMEM = -2,
  ORACLE_EFOOTPRINT = -3 /* an output point was left uncomputed */
};

enum { ORACLE_SI_NORMALIZED = 0, ORACLE_SI_LITERAL = 1 };
enum { ORACLE_OUT_2N = 0, ORACLE_OUT_2N_MINUS_1 = 1 };
enum {
  ORACLE_BC_CLAMP = 0,      /* replicate the edge sample (the library's rule) */
  ORACLE_BC_ZERO = 1,       /* zero outside the image */
  ORACLE_BC_REFLECT101 = 2, /* mirror without repeating the edge sample */
  ORACLE_BC_SYMMETRIC = 3   /* mirror repeating the edge sample */
};

typedef struct {
  double beta;  /* exponent of Eq. (alpha) */
  double k_eps; /* eps_h = k_eps * h^2 (Sec. 2) */
  double h;     /* coarse grid spacing */
  int si_scale; /* ORACLE_SI_* */
  int out_mode; /* ORACLE_OUT_*: 2n x 2m or (2n-1) x (2m-1) */
  int boundary; /* ORACLE_BC_* */
  int ghost;    /* coarse ghost cells per side; >= 5 */
  double nbr_c1; /* phase-1 neighbour weight of D is nbr_c1 * h^2 (Eq. 2DsmoothnessFinal) */
  double nbr_c2; /* phase-2 neighbour weight of D is nbr_c2 * h^2 (Eq. tezine) */
} oracle_params;

oracle_params oracle_params_default(void);
int oracle_ghost_default(void);

/* One channel: A is n x m row-major, U is the output (2n or 2n-1 rows, same
 * for columns) row-major.  Returns ORACLE_OK or a negative code. */
int oracle_zoom2x(const double* A, int64_t n, int64_t m, double* U,
                  const oracle_params* p);

/* `planes` independent channels stored back to back. */
int oracle_zoom2x_planes(const double* A, int64_t planes, int64_t n, int64_t m,
                         double* U, const oracle_params* p);

/* oracle_zoom2x_planes computed in bands of `band_rows` quad rows (windows
 * with the footprint's 4/5-row margins), OpenMP over (plane, band) pairs on
 * `threads` threads (0 = OpenMP default).  Same output. */
int oracle_zoom2x_banded(const double* A, int64_t planes, int64_t n, int64_t m, double* U,
                         const oracle_params* p, int64_t band_rows, int threads);

/* p (Eq. p) and SI (Eq. 2Dsmoothness) of one stencil with nodes at
 * t = -1, 1, 3 fine steps; scale_over_step = (length scale) / |d|. */
void oracle_directional(double n0, double n1, double n2, double scale_over_step,
                        double* p, double* si);

/* 1-D WENO interpolant of Sec. 2 on one cell: v4 = samples at x_{i-1..i+2},
 * t = (x - x_i)/h in [0, 1]. */
double oracle_weno1d_cell(const double v4[4], double t, double beta, double k_eps, double h);

/* WENO spline w(V, x), x in [0, n-1], samples V[k * stride] (Sec. 3.3). */
double oracle_weno_spline(const double* V, int64_t n, int64_t stride, double x, double beta,
                          double k_eps, double h);

/* Tensor WENO resampling of one n x m plane to n_out x m_out (Eq. tensor). */
int oracle_tensor_resample(const double* A, int64_t n, int64_t m, double* U, int64_t n_out,
                           int64_t m_out, double beta, double k_eps, double h);

/* Saturate to [0, 1], scale by 255, round half to even. */
void oracle_encode_u8(const double* U, int64_t count, unsigned char* out);

#ifdef __cplusplus
}
#endif

#endif
