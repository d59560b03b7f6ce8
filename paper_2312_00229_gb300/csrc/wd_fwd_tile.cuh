// Tile body of the fused WD WENO forward pass, shared by the one-launch-per-
// image kernel (wd_fwd.cu) and the persistent batched kernel (wd_batched.cu).
//
// Fused WD WENO 2x zoom, forward (arXiv 2312.00229, Sec. 3, Algorithms 1-2).
//
// Work decomposition
//   One CTA = one plane x one strip of TILE_W = 240 coarse columns x one
//   band of `rows_per_band` coarse rows.  128 threads; thread t owns the two
//   coarse columns c0 = b0 - 4 + 2t and c0 + 1, so the CTA spans 256 columns:
//   the 240 output columns plus the 4-before / 5-after dependency halo of the
//   method (an output quad depends on input rows and columns -4..+5).
//   The CTA sweeps its band top to bottom, one coarse row per step.  All
//   per-column state lives in registers as sliding windows over rows; values
//   a thread needs from the neighbouring columns are exchanged through shared
//   memory, so every stage is computed once per (row, column) of its region.
//
// Pipeline of one step s (coarse row s is loaded in this step):
//   stage 1  row s-2  second differences S1/S2 along both diagonals and their
//                     squared, kappa-scaled forms (columns c0..c0+2)
//   stage 2  row s-3  the four phase-1 smoothness indicators (Eq.
//                     2Dsmoothness) of X(s-3, .) and their interpolants
//   stage 3  row s-4  D (Eq. 2DsmoothnessFinal), alpha (Eq. alpha) and the
//                     blend (Eqs. IzrazOmega2d, 2dKombinacija) -> X(s-4, .)
//   stage 4  row s-5  phase-2 indicators of E(s-5, .) and S(s-5, .)
//   stage 5           E(s-5, .) and S(s-6, .) (Eqs. tezine,
//                     IzrazOmega2dRavno, 2dKombinacijaRavno)
//   store             fine row 2(s-5) = [A, E] pairs, fine row 2(s-6)+1 =
//                     [S, X] pairs, four elements per thread and row
// Barrier B1 opens the step (exchange of rows written in the previous step);
// barrier B2 separates the phase-2 indicator exchange inside the step.
#pragma once

#include "wd_common.cuh"
#include "wd_fwd.h"

namespace wdweno {
namespace fwd_tile {

constexpr int THREADS = 128;
constexpr int TILE_W = 2 * THREADS - 16;  // output columns per CTA
constexpr int HALO_L = 4;                 // columns before the strip

struct __align__(16) Exchange {
  float2 A[THREADS + 2];    // input row, both owned columns
  float4 SI0[THREADS + 2];  // phase-1 SIs of column c0 (directions A,B,C,D)
  float4 SI1[THREADS + 2];  // same, column c0+1
  float2 X[THREADS + 2];    // phase-1 values, both columns
  float4 VS[THREADS + 2];   // S-point SIs summed over two rows, column c0
  float4 VE[THREADS + 2];   // E-point SIs summed over two rows, column c0+1
};

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ float sq_eps(float kappa, float s, float eps) {
  float t = kappa * s;
  return fmaf(t, t, eps);
}

// One tile: strip `bx` (columns bx*TILE_W ...), band `by`, plane `plane`.
// Must be called by all THREADS threads of the CTA; the CTA may call it
// repeatedly (persistent kernels): it synchronises before touching `ex`.
template <int BMODE>
__device__ __forceinline__ void zoom2x_fwd_tile(const FwdArgs& a, const MethodConsts& k,
                                                Exchange& ex, int64_t bx, int64_t by,
                                                int64_t plane) {
  const int t = threadIdx.x;
  const int64_t b0 = bx * TILE_W;
  const int64_t a0 = by * a.rows_per_band;
  const int64_t c0 = b0 - HALO_L + 2 * t;
  const int64_t H = a.rows_per_band;

  // Zero the exchange buffers so that reads at the strip edges and before
  // the first writes see finite values.
  __syncthreads();
  {
    float* z = reinterpret_cast<float*>(&ex);
    for (int i = t; i < (int)(sizeof(Exchange) / sizeof(float)); i += THREADS) z[i] = 0.f;
  }

  const int64_t in_off0 = plane * a.in_sc + clamp64(c0, 0, a.m - 1) * a.in_sw;
  const int64_t in_off1 = plane * a.in_sc + clamp64(c0 + 1, 0, a.m - 1) * a.in_sw;
  auto load_row = [&](int64_t r, float& v0, float& v1) {
    const int64_t rr = clamp64(r, 0, a.n - 1) * a.in_sh;
    v0 = load_elem(a.in, rr + in_off0, a.in_dtype);
    v1 = load_elem(a.in, rr + in_off1, a.in_dtype);
  };

  // Output columns this thread stores (fine columns 2c0 .. 2c0+3).
  const bool col_ok0 = (c0 >= b0) && (c0 < b0 + TILE_W) && (c0 < a.m);
  const bool col_ok1 = (c0 + 1 >= b0) && (c0 + 1 < b0 + TILE_W) && (c0 + 1 < a.m);
  const int64_t q0 = 2 * c0;  // first fine column
  const bool vec_ok = a.out_vec && col_ok0 && col_ok1 && (q0 + 3 < a.ocols);
  void* outp = a.out;
  const int64_t out_plane = plane * a.out_sc;

  // ---- register windows -------------------------------------------------
  // Aw[k][u+1] = A(s-k, c0+u): own columns u = 0,1 for k = 0..6,
  // neighbour columns u = -1, 2, 3 for k = 1..5.
  float Aw[7][5];
#pragma unroll
  for (int i = 0; i < 7; ++i)
#pragma unroll
    for (int j = 0; j < 5; ++j) Aw[i][j] = 0.f;
  // stage-1 results of the previous step (row s-3), columns c0..c0+2
  float S1p[3] = {0.f, 0.f, 0.f}, S2p[3] = {0.f, 0.f, 0.f};
  float q1p[3] = {0.f, 0.f, 0.f}, q2p[3] = {0.f, 0.f, 0.f};
  // stage-2 results of the previous step (row s-4): SIs, partial D, p data
  float SIp[2][4], Pp[2][4], pxp[2][6];
  // phase-1 values X(s-5-k, c0+j), k = 0..2
  float Xw[3][2];
  // phase-2 state carried one step: column second differences of X and of
  // A, the E/S indicators of row s-6 and the S-point p data of row s-6
  float sXcp[2] = {0.f, 0.f}, qXcp[2] = {0.f, 0.f};
  float sVcp[2] = {0.f, 0.f}, qVcp[2] = {0.f, 0.f};
  float SIEp[2][4], SISp[2][4], pSp[2][6];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { SIp[j][d] = Pp[j][d] = SIEp[j][d] = SISp[j][d] = 0.f; }
#pragma unroll
    for (int d = 0; d < 6; ++d) { pxp[j][d] = pSp[j][d] = 0.f; }
    Xw[0][j] = Xw[1][j] = Xw[2][j] = 0.f;
  }

  const int64_t s_begin = a0 - 4;
  const int64_t s_end = a0 + H + 5;  // inclusive
  float pf0a, pf0b, pf1a, pf1b;      // prefetched rows s and s+1
  load_row(s_begin, pf0a, pf0b);
  load_row(s_begin + 1, pf1a, pf1b);

  const float w = k.w;

  for (int64_t s = s_begin; s <= s_end; ++s) {
    const int64_t rs = s - a0;
    Aw[0][1] = pf0a;
    Aw[0][2] = pf0b;
    pf0a = pf1a;
    pf0b = pf1b;
    load_row(s + 2, pf1a, pf1b);

    __syncthreads();  // B1: rows written in step s-1 are visible
    {
      float2 l = ex.A[t];
      float2 r = ex.A[t + 2];
      Aw[1][0] = l.y;  // A(s-1, c0-1)
      Aw[1][3] = r.x;  // A(s-1, c0+2)
      Aw[1][4] = r.y;  // A(s-1, c0+3)
    }
    const float4 siL = ex.SI1[t];     // X-SIs of column c0-1, row s-4
    const float4 siR = ex.SI0[t + 2]; // X-SIs of column c0+2, row s-4
    const float2 xl = ex.X[t];        // X(s-5, c0-2), X(s-5, c0-1)
    const float xr = ex.X[t + 2].x;   // X(s-5, c0+2)

    // ---- stage 1: diagonal second differences at row s-2 ----------------
    float S1c[3] = {0.f, 0.f, 0.f}, S2c[3] = {0.f, 0.f, 0.f};
    float q1c[3] = {0.f, 0.f, 0.f}, q2c[3] = {0.f, 0.f, 0.f};
    if (rs >= -1)
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      // S1(i,j) = A(i-1,j-1) - 2A(i,j) + A(i+1,j+1), S2 along (1,-1)
      S1c[u] = fmaf(-2.f, Aw[2][u + 1], Aw[3][u] + Aw[1][u + 2]);
      S2c[u] = fmaf(-2.f, Aw[2][u + 1], Aw[3][u + 2] + Aw[1][u]);
      q1c[u] = sq_eps(k.kappa1, S1c[u], k.eps1);
      q2c[u] = sq_eps(k.kappa1, S2c[u], k.eps1);
    }

    // ---- stage 2: phase-1 SIs of X(s-3, .) -------------------------------
    // X(a,b) sits between A(a,b) and A(a+1,b+1).  Directions:
    //   A (1,1):   nodes A(a,b),   A(a+1,b+1), A(a+2,b+2); s = S1(a+1,b+1)
    //   B (-1,-1): nodes A(a+1,b+1), A(a,b),   A(a-1,b-1); s = S1(a,b)
    //   C (1,-1):  nodes A(a,b+1), A(a+1,b),   A(a+2,b-1); s = S2(a+1,b)
    //   D (-1,1):  nodes A(a+1,b), A(a,b+1),   A(a-1,b+2); s = S2(a,b+1)
    float SIc[2][4] = {}, Pc[2][4] = {}, pxc[2][6] = {};
    if (rs >= 0)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float a_ab = Aw[3][j + 1], a_ab1 = Aw[3][j + 2];
      const float a_a1b = Aw[2][j + 1], a_a1b1 = Aw[2][j + 2];
      const float G1 = a_a1b1 - a_ab;
      const float G2 = a_a1b - a_ab1;
      SIc[j][0] = fmaf(G1, G1, q1c[j + 1]);
      SIc[j][1] = fmaf(G1, G1, q1p[j]);
      SIc[j][2] = fmaf(G2, G2, q2c[j]);
      SIc[j][3] = fmaf(G2, G2, q2p[j + 1]);
#pragma unroll
      for (int d = 0; d < 4; ++d) Pc[j][d] = fmaf(w, SIp[j][d], SIc[j][d]);
      pxc[j][0] = a_ab + a_a1b1;  // N0 + N1 of the (1,1) diagonal pair
      pxc[j][1] = a_ab1 + a_a1b;  // N0 + N1 of the (1,-1) pair
      pxc[j][2] = S1c[j + 1];
      pxc[j][3] = S1p[j];
      pxc[j][4] = S2c[j];
      pxc[j][5] = S2p[j + 1];
    }

    // ---- stage 3: X(s-4, .) ----------------------------------------------
    float Xn[2] = {0.f, 0.f};
    if (rs >= 2) {
      const float hl[4] = {siL.x, siL.y, siL.z, siL.w};
      const float hr[4] = {siR.x, siR.y, siR.z, siR.w};
      float D[2][4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        D[0][d] = fmaf(w, SIc[0][d] + (hl[d] + SIp[1][d]), Pp[0][d]);
        D[1][d] = fmaf(w, SIc[1][d] + (SIp[0][d] + hr[d]), Pp[1][d]);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
        Xn[j] = blend4<BMODE>(D[j][0], D[j][1], D[j][2], D[j][3], pxp[j][0], pxp[j][1],
                              pxp[j][2], pxp[j][3], pxp[j][4], pxp[j][5], k.beta);
    }

    // ---- stage 4: phase-2 indicators at row r = s-5 ----------------------
    // X(r+1) = Xn, X(r) = Xw[0], X(r-1) = Xw[1], X(r-2) = Xw[2]
    // A(r-1) = Aw[6], A(r) = Aw[5], A(r+1) = Aw[4], A(r+2) = Aw[3]
    // Direction order for both classes: (0,1), (0,-1), (1,0), (-1,0).
    float SIE[2][4] = {}, SIS[2][4] = {}, pE[2][6] = {}, pS[2][6] = {};
    float sXcc[2] = {0.f, 0.f}, qXcc[2] = {0.f, 0.f}, sVcc[2] = {0.f, 0.f}, qVcc[2] = {0.f, 0.f};
    // Column second difference of the input centred at A(r+1); carried to
    // the next step as the one centred at A(r), so it starts one row early.
    if (rs >= 3) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        sVcc[j] = fmaf(-2.f, Aw[4][j + 1], Aw[5][j + 1] + Aw[3][j + 1]);
        qVcc[j] = sq_eps(k.kappa2, sVcc[j], k.eps2);
      }
    }
    if (rs >= 4) {
      // E(r,b) horizontal: nodes along input row r
      float sH[3], qH[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        sH[u] = fmaf(-2.f, Aw[5][u + 1], Aw[5][u] + Aw[5][u + 2]);  // centred at c0+u
        qH[u] = sq_eps(k.kappa2, sH[u], k.eps2);
      }
      // S(r,b) horizontal: nodes along phase-1 row r
      const float Xr[5] = {xl.x, xl.y, Xw[0][0], Xw[0][1], xr};  // columns c0-2..c0+2
      float sXr[3], qXr[3];
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        sXr[u] = fmaf(-2.f, Xr[u + 1], Xr[u] + Xr[u + 2]);  // centred at c0+u-1
        qXr[u] = sq_eps(k.kappa2, sXr[u], k.eps2);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        // E(r, b=c0+j): horizontal pair A(r,b), A(r,b+1)
        const float gH = Aw[5][j + 2] - Aw[5][j + 1];
        SIE[j][0] = fmaf(gH, gH, qH[j + 1]);  // (0,1):  s centred at b+1
        SIE[j][1] = fmaf(gH, gH, qH[j]);      // (0,-1): s centred at b
        // E vertical: nodes along phase-1 column b
        sXcc[j] = fmaf(-2.f, Xw[0][j], Xw[1][j] + Xn[j]);  // centred at X(r)
        qXcc[j] = sq_eps(k.kappa2, sXcc[j], k.eps2);
        const float gV = Xw[0][j] - Xw[1][j];
        SIE[j][2] = fmaf(gV, gV, qXcc[j]);  // (1,0):  s centred at X(r)
        SIE[j][3] = fmaf(gV, gV, qXcp[j]);  // (-1,0): s centred at X(r-1)
        pE[j][0] = Aw[5][j + 1] + Aw[5][j + 2];
        pE[j][1] = Xw[1][j] + Xw[0][j];
        pE[j][2] = sH[j + 1];
        pE[j][3] = sH[j];
        pE[j][4] = sXcc[j];
        pE[j][5] = sXcp[j];

        // S(r, b=c0+j): horizontal pair X(r,b-1), X(r,b)
        const float gSh = Xr[j + 2] - Xr[j + 1];
        SIS[j][0] = fmaf(gSh, gSh, qXr[j + 1]);  // (0,1):  s centred at b
        SIS[j][1] = fmaf(gSh, gSh, qXr[j]);      // (0,-1): s centred at b-1
        // S vertical: nodes along input column b
        const float gSv = Aw[4][j + 1] - Aw[5][j + 1];
        SIS[j][2] = fmaf(gSv, gSv, qVcc[j]);  // (1,0):  s centred at A(r+1)
        SIS[j][3] = fmaf(gSv, gSv, qVcp[j]);  // (-1,0): s centred at A(r)
        pS[j][0] = Xr[j + 1] + Xr[j + 2];
        pS[j][1] = Aw[5][j + 1] + Aw[4][j + 1];
        pS[j][2] = sXr[j + 1];
        pS[j][3] = sXr[j];
        pS[j][4] = sVcc[j];
        pS[j][5] = sVcp[j];
      }
    }
    // Row-pair sums for the neighbour terms of Eq. (tezine).
    float VS[2][4], VE[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        VS[j][d] = SISp[j][d] + SIS[j][d];  // S rows r-1, r  (for E(r))
        VE[j][d] = SIEp[j][d] + SIE[j][d];  // E rows r-1, r  (for S(r-1))
      }
    ex.VS[t + 1] = make_float4(VS[0][0], VS[0][1], VS[0][2], VS[0][3]);
    ex.VE[t + 1] = make_float4(VE[1][0], VE[1][1], VE[1][2], VE[1][3]);

    __syncthreads();  // B2

    // ---- stage 5: E(s-5, .) and S(s-6, .) --------------------------------
    float Ev[2] = {0.f, 0.f}, Sv[2] = {0.f, 0.f};
    if (rs >= 5) {
      const float4 vr = ex.VS[t + 2];  // column c0+2
      const float vsr[4] = {vr.x, vr.y, vr.z, vr.w};
      float D[2][4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        D[0][d] = fmaf(w, VS[0][d] + VS[1][d], SIE[0][d]);
        D[1][d] = fmaf(w, VS[1][d] + vsr[d], SIE[1][d]);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
        Ev[j] = blend4<BMODE>(D[j][0], D[j][1], D[j][2], D[j][3], pE[j][0], pE[j][1], pE[j][2],
                              pE[j][3], pE[j][4], pE[j][5], k.beta);
    }
    if (rs >= 6) {
      const float4 vl = ex.VE[t];  // column c0-1
      const float vel[4] = {vl.x, vl.y, vl.z, vl.w};
      float D[2][4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        D[0][d] = fmaf(w, vel[d] + VE[0][d], SISp[0][d]);
        D[1][d] = fmaf(w, VE[0][d] + VE[1][d], SISp[1][d]);
      }
#pragma unroll
      for (int j = 0; j < 2; ++j)
        Sv[j] = blend4<BMODE>(D[j][0], D[j][1], D[j][2], D[j][3], pSp[j][0], pSp[j][1],
                              pSp[j][2], pSp[j][3], pSp[j][4], pSp[j][5], k.beta);
    }

    // ---- stores ------------------------------------------------------------
    {
      const int64_t rE = s - 5;  // fine row 2 rE: [A, E]
      if (rs >= 5 && rE < a0 + H && rE < a.n && 2 * rE < a.orows) {
        const int64_t base = out_plane + (2 * rE) * a.out_sh;
        if (vec_ok) {
          store4_vec(outp, base + q0, Aw[5][1], Ev[0], Aw[5][2], Ev[1], a.out_dtype, k.clamp_float);
        } else {
          if (col_ok0) {
            store_elem(outp, base + q0 * a.out_sw, Aw[5][1], a.out_dtype, k.clamp_float);
            if (q0 + 1 < a.ocols)
              store_elem(outp, base + (q0 + 1) * a.out_sw, Ev[0], a.out_dtype, k.clamp_float);
          }
          if (col_ok1) {
            store_elem(outp, base + (q0 + 2) * a.out_sw, Aw[5][2], a.out_dtype, k.clamp_float);
            if (q0 + 3 < a.ocols)
              store_elem(outp, base + (q0 + 3) * a.out_sw, Ev[1], a.out_dtype, k.clamp_float);
          }
        }
      }
      const int64_t rS = s - 6;  // fine row 2 rS + 1: [S, X]
      if (rs >= 6 && rS < a0 + H && rS < a.n && 2 * rS + 1 < a.orows) {
        const int64_t base = out_plane + (2 * rS + 1) * a.out_sh;
        if (vec_ok) {
          store4_vec(outp, base + q0, Sv[0], Xw[1][0], Sv[1], Xw[1][1], a.out_dtype,
                     k.clamp_float);
        } else {
          if (col_ok0) {
            store_elem(outp, base + q0 * a.out_sw, Sv[0], a.out_dtype, k.clamp_float);
            if (q0 + 1 < a.ocols)
              store_elem(outp, base + (q0 + 1) * a.out_sw, Xw[1][0], a.out_dtype, k.clamp_float);
          }
          if (col_ok1) {
            store_elem(outp, base + (q0 + 2) * a.out_sw, Sv[1], a.out_dtype, k.clamp_float);
            if (q0 + 3 < a.ocols)
              store_elem(outp, base + (q0 + 3) * a.out_sw, Xw[1][1], a.out_dtype, k.clamp_float);
          }
        }
      }
    }

    // ---- publish this step's rows (read after the next B1) ------------------
    ex.A[t + 1] = make_float2(Aw[0][1], Aw[0][2]);
    ex.SI0[t + 1] = make_float4(SIc[0][0], SIc[0][1], SIc[0][2], SIc[0][3]);
    ex.SI1[t + 1] = make_float4(SIc[1][0], SIc[1][1], SIc[1][2], SIc[1][3]);
    ex.X[t + 1] = make_float2(Xn[0], Xn[1]);

    // ---- slide the windows ---------------------------------------------------
#pragma unroll
    for (int i = 6; i >= 1; --i)
#pragma unroll
      for (int j = 0; j < 5; ++j) Aw[i][j] = Aw[i - 1][j];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      S1p[u] = S1c[u]; S2p[u] = S2c[u]; q1p[u] = q1c[u]; q2p[u] = q2c[u];
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        SIp[j][d] = SIc[j][d]; Pp[j][d] = Pc[j][d];
        SIEp[j][d] = SIE[j][d]; SISp[j][d] = SIS[j][d];
      }
#pragma unroll
      for (int d = 0; d < 6; ++d) { pxp[j][d] = pxc[j][d]; pSp[j][d] = pS[j][d]; }
      Xw[2][j] = Xw[1][j]; Xw[1][j] = Xw[0][j]; Xw[0][j] = Xn[j];
      sXcp[j] = sXcc[j]; qXcp[j] = qXcc[j];
      sVcp[j] = sVcc[j]; qVcp[j] = qVcc[j];
    }
  }
}


}  // namespace fwd_tile
}  // namespace wdweno
