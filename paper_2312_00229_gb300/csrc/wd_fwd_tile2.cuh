// Tile body of the fused WD WENO forward pass with two coarse columns per
// thread (arXiv 2312.00229, Sec. 3, Algorithms 1-2).  Same method, stages,
// pipeline and arithmetic as wd_fwd_tile.cuh (every value is formed by the
// same expression, so the output is bit-identical); what changes is the work
// decomposition:
//   thread t owns the adjacent columns c0 = b0 - 4 + 2t and c1 = c0 + 1.
//   NT threads cover 2 NT columns, of which 2 NT - 10 are outputs (an even
//   count, so c0 is even and a thread's four fine output columns start on a
//   multiple of four: one vector store per fine row).
// What the pair shares: the input, phase-1 and indicator values of the
// neighbouring columns that both columns read are loaded once (as aligned
// float2 reads of the shared rows), the second differences centred between
// the two columns are formed once, the neighbour-smoothing sums that cross
// from c0 to c1 stay in registers, and a step's addressing, barrier and
// loop control serve two columns.
#pragma once

#include "wd_fwd_tile.cuh"
#include "wd_packed.cuh"

namespace wdweno {
namespace fwd_tile {

template <int NT>
struct Shape2 {
  static constexpr int COLS = 2 * NT;    // columns of a CTA
  static constexpr int TW = COLS - 10;   // output columns per CTA (even)
  static constexpr int ROW = COLS + 4;   // floats per staged row (2 pad each side)
};

template <int NT>
struct __align__(16) Exchange2 {
  static constexpr int ROW = Shape2<NT>::ROW;
  float A[12][ROW];       // input rows, slot = row & 7 (8..11 repeat 0..3);
                          // column c0 + u of thread t at 2t + 2 + u
  float X[5][ROW];        // phase-1 values, slot = row & 3 (4 repeats 0), same columns
  float4 SI0[2][NT + 2];  // phase-1 SIs of column c0, slot = row & 1, at t + 1
  float4 SI1[2][NT + 2];  // phase-1 SIs of column c1
  float4 VS[2][NT + 2];   // S-point SIs of rows r-1, r summed, column c0, at t + 1
  float4 VE[2][NT + 2];   // E-point SIs of rows r-1, r summed, column c1, at t + 1
  float4 PS[2][3][NT];    // the thread's S blend data, kept two steps (slot = parity)
};

// Values a thread carries from one step to the next (slot = step parity
// where two rows are live).
struct Carry2 {
  float S1[2][3], S2[2][3];                      // stage 1, columns c0 .. c0+2
  float SI[2][2][4];                             // stage 2 SIs [parity][u][direction]
  float P[2][4];                                 // SI + w SI(row above), consumed next step
  float px[2][6];                                // X blend data, consumed next step
  float sXc[2][2], qXc[2][2], sVc[2][2], qVc[2][2];
  float SIE[2][2][4], SIS[2][2][4];
  // stage 4 results that stage 5 uses one step later
  float DE0[4], DEp1[4], DSp0[4], DS1[4], pE[2][6], a5c[2], x6[2];
};

template <int BMODE, class IO, int NT>
struct FwdTile2 {
  static constexpr int TILE_W = Shape2<NT>::TW;
  static constexpr int ROW = Shape2<NT>::ROW;
  const MethodConsts k;
  Exchange2<NT>& ex;
  const int t;
  const void* in;
  void* out;
  int in_dtype, out_dtype;
  int n, a0, H;
  int orows;
  int64_t in_idx0, in_idx1, in_sh;  // element index of (row 0, column c0 / c1); row stride
  int64_t out_base, out_sh;         // element index of (fine row 0, fine column 2 c0)
  int64_t out_sw;
  int64_t oE;                       // element index of (fine row 2(s-6), fine column 2 c0)
  bool col_ok[2], odd_ok[2], vec_ok;

  __device__ __forceinline__ FwdTile2(const FwdArgs& a, const MethodConsts& k_,
                                      Exchange2<NT>& ex_, int64_t bx, int64_t by,
                                      int64_t plane)
      : k(k_), ex(ex_), t(threadIdx.x) {
    in = a.in;
    out = a.out;
    in_dtype = a.in_dtype;
    out_dtype = a.out_dtype;
    n = (int)a.n;
    H = (int)a.rows_per_band;
    a0 = (int)by * H;
    orows = (int)a.orows;
    const int64_t b0 = bx * TILE_W;
    const int64_t c0 = b0 - HALO_L + 2 * t;
    in_idx0 = plane * a.in_sc + clamp64(c0, 0, a.m - 1) * a.in_sw;
    in_idx1 = plane * a.in_sc + clamp64(c0 + 1, 0, a.m - 1) * a.in_sw;
    in_sh = a.in_sh;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t c = c0 + u;
      col_ok[u] = (c >= b0) && (c < b0 + TILE_W) && (c < a.m);
      odd_ok[u] = 2 * c + 1 < a.ocols;
    }
    // one 4-element store: both columns and both fine columns of each inside
    vec_ok = a.out_vec4 && col_ok[0] && col_ok[1] && odd_ok[1];
    out_sw = a.out_sw;
    out_sh = a.out_sh;
    out_base = plane * a.out_sc + 2 * c0 * a.out_sw;
  }

  __device__ __forceinline__ uint32_t load_row(int r, int u) const {
    const int rc = r < 0 ? 0 : (r > n - 1 ? n - 1 : r);
    return IO::load_bits(in, (u ? in_idx1 : in_idx0) + (int64_t)rc * in_sh, in_dtype);
  }

  // fine row at element index `base`: columns 2 c0 .. 2 c0 + 3 hold v0..v3
  __device__ __forceinline__ void store_quad_row(int64_t base, float v0, float v1, float v2,
                                                 float v3) const {
    if (vec_ok) {
      IO::store4(out, base, v0, v1, v2, v3, out_dtype, k.clamp_float);
      return;
    }
    if (col_ok[0]) {
      IO::store1(out, base, v0, out_dtype, k.clamp_float);
      if (odd_ok[0]) IO::store1(out, base + out_sw, v1, out_dtype, k.clamp_float);
    }
    if (col_ok[1]) {
      IO::store1(out, base + 2 * out_sw, v2, out_dtype, k.clamp_float);
      if (odd_ok[1]) IO::store1(out, base + 3 * out_sw, v3, out_dtype, k.clamp_float);
    }
  }

  // Columns c0-2 .. c0+3 of the row at `p` (column c0 - 2): three aligned pairs.
  __device__ __forceinline__ static void row6(const float* p, float (&v)[6]) {
    const float2 l = *reinterpret_cast<const float2*>(p);
    const float2 m = *reinterpret_cast<const float2*>(p + 2);
    const float2 r = *reinterpret_cast<const float2*>(p + 4);
    v[0] = l.x; v[1] = l.y; v[2] = m.x; v[3] = m.y; v[4] = r.x; v[5] = r.y;
  }

  __device__ __forceinline__ void put_row(int r, float v0, float v1) const {
    const int sl = r & 7;
    *reinterpret_cast<float2*>(&ex.A[sl][2 * t + 2]) = make_float2(v0, v1);
    if (sl < 4) *reinterpret_cast<float2*>(&ex.A[sl + 8][2 * t + 2]) = make_float2(v0, v1);
  }

  template <int PH, bool FULL>
  __device__ __forceinline__ void step(int s, uint32_t (&pf)[2], uint32_t (&pf2)[2], Carry2& C) {
    constexpr int Q = PH ^ 1;
    const int rs = s - a0;
    if (!FULL && rs > H + 6) return;
    const float w = k.w;
    oE += 2 * out_sh;

    const uint32_t cur0 = pf[0], cur1 = pf[1];
    pf[0] = pf2[0];
    pf[1] = pf2[1];
    pf2[0] = load_row(s + 2, 0);
    pf2[1] = load_row(s + 2, 1);

    __syncthreads();  // rows published in step s-1 are visible
    put_row(s, IO::value(cur0, in_dtype), IO::value(cur1, in_dtype));

    // ---- stage 5: E(s-6, c0..c1) and S(s-7, c0..c1) ------------------------
    if (FULL || (rs >= 6 && rs <= H + 5)) {
      const float4 v = ex.VS[PH ^ 1][t + 2];  // VS of column c0 + 2 (slot of step s-1)
      float D1[4];
      {
        const f2 a = pk_fma(pk_bc(w), make_float2(v.x, v.y), make_float2(C.DEp1[0], C.DEp1[1]));
        const f2 b = pk_fma(pk_bc(w), make_float2(v.z, v.w), make_float2(C.DEp1[2], C.DEp1[3]));
        D1[0] = a.x; D1[1] = a.y; D1[2] = b.x; D1[3] = b.y;
      }
      const float e0 = blend4_pk<BMODE>(C.DE0[0], C.DE0[1], C.DE0[2], C.DE0[3], C.pE[0][0],
                                     C.pE[0][1], C.pE[0][2], C.pE[0][3], C.pE[0][4],
                                     C.pE[0][5], k.beta);
      const float e1 = blend4_pk<BMODE>(D1[0], D1[1], D1[2], D1[3], C.pE[1][0], C.pE[1][1],
                                     C.pE[1][2], C.pE[1][3], C.pE[1][4], C.pE[1][5], k.beta);
      const int rE = s - 6;  // fine row 2 rE: [A, E] of both columns
      if (FULL || (rE < n && 2 * rE < orows)) store_quad_row(oE, C.a5c[0], e0, C.a5c[1], e1);
    }
    if (FULL || rs >= 7) {
      const float4 v = ex.VE[PH ^ 1][t];  // VE of column c0 - 1
      float D0[4];
      {
        const f2 a = pk_fma(pk_bc(w), make_float2(v.x, v.y), make_float2(C.DSp0[0], C.DSp0[1]));
        const f2 b = pk_fma(pk_bc(w), make_float2(v.z, v.w), make_float2(C.DSp0[2], C.DSp0[3]));
        D0[0] = a.x; D0[1] = a.y; D0[2] = b.x; D0[3] = b.y;
      }
      const float4 ps0 = ex.PS[PH][0][t], ps1 = ex.PS[PH][1][t], ps2 = ex.PS[PH][2][t];
      const float p0[6] = {ps0.x, ps0.y, ps0.z, ps0.w, ps1.x, ps1.y};
      const float p1[6] = {ps1.z, ps1.w, ps2.x, ps2.y, ps2.z, ps2.w};
      const float s0 = blend4_pk<BMODE>(D0[0], D0[1], D0[2], D0[3], p0[0], p0[1], p0[2], p0[3],
                                     p0[4], p0[5], k.beta);
      const float s1 = blend4_pk<BMODE>(C.DS1[0], C.DS1[1], C.DS1[2], C.DS1[3], p1[0], p1[1],
                                     p1[2], p1[3], p1[4], p1[5], k.beta);
      const int rS = s - 7;  // fine row 2 rS + 1: [S, X] of both columns
      if (FULL || (rS < n && 2 * rS + 1 < orows))
        store_quad_row(oE - out_sh, s0, C.x6[0], s1, C.x6[1]);
    }

    // Input rows s-5 .. s-1 sit at consecutive slots from (s-5) & 7.
    const float* A5 = ex.A[(s - 5) & 7] + 2 * t;  // row s-5, column c0 - 2
    // Input rows s-3, s-2, s-1 at columns c0-2 .. c0+3 (index j + 2 = column c0 + j).
    float a1[6], a2[6], a3[6];
    row6(A5 + 4 * ROW, a1);
    row6(A5 + 3 * ROW, a2);
    row6(A5 + 2 * ROW, a3);

    // ---- stage 1: diagonal second differences at row s-2, columns c0..c0+2 --
    // (their squared forms q are formed where stage 2 uses them, for this
    // row and again for the row above, rather than carried)
    if (FULL || rs >= -1) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C.S1[PH][j] = fmaf(-2.f, a2[j + 2], a3[j + 1] + a1[j + 3]);
        C.S2[PH][j] = fmaf(-2.f, a2[j + 2], a3[j + 3] + a1[j + 1]);
      }
    }

    // ---- stage 2: phase-1 SIs of X(s-3, c0..c1) ----------------------------
    if (FULL || rs >= 0) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float G1 = a2[u + 3] - a3[u + 2];  // A(a+1,b+1) - A(a,b)
        const float G2 = a2[u + 2] - a3[u + 3];  // A(a+1,b) - A(a,b+1)
        float* SI = C.SI[PH][u];
        SI[0] = fmaf(G1, G1, sq_eps(k.kappa1, C.S1[PH][u + 1], k.eps1));
        SI[1] = fmaf(G1, G1, sq_eps(k.kappa1, C.S1[Q][u], k.eps1));
        SI[2] = fmaf(G2, G2, sq_eps(k.kappa1, C.S2[PH][u], k.eps1));
        SI[3] = fmaf(G2, G2, sq_eps(k.kappa1, C.S2[Q][u + 1], k.eps1));
        if (u == 0)
          ex.SI0[PH ^ 1][t + 1] = make_float4(SI[0], SI[1], SI[2], SI[3]);
        else
          ex.SI1[PH ^ 1][t + 1] = make_float4(SI[0], SI[1], SI[2], SI[3]);
      }
    }

    // ---- stage 3: X(s-4, c0..c1) -------------------------------------------
    // D = SI(a) + w (SI(a-1) + SI(a+1) + SI(a, c-1) + SI(a, c+1)), with the
    // partial P(a) = SI(a) + w SI(a-1) formed one step earlier.
    float x4[2] = {0.f, 0.f};
    if (FULL || rs >= 2) {
      const float4 l = ex.SI1[PH][t];      // SI(s-4, c0 - 1)
      const float4 r = ex.SI0[PH][t + 2];  // SI(s-4, c0 + 2)
      const float hl0[4] = {l.x, l.y, l.z, l.w};
      const float hr1[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        float D[4];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int d = 2 * p;
          // row s-4 at columns c - 1 and c + 1
          const f2 hl = u == 0 ? make_float2(hl0[d], hl0[d + 1])
                               : make_float2(C.SI[Q][0][d], C.SI[Q][0][d + 1]);
          const f2 hr = u == 0 ? make_float2(C.SI[Q][1][d], C.SI[Q][1][d + 1])
                               : make_float2(hr1[d], hr1[d + 1]);
          const f2 v = pk_fma(pk_bc(w),
                              pk_add(make_float2(C.SI[PH][u][d], C.SI[PH][u][d + 1]),
                                     pk_add(hl, hr)),
                              make_float2(C.P[u][d], C.P[u][d + 1]));
          D[d] = v.x;
          D[d + 1] = v.y;
        }
        const float* px = C.px[u];
        x4[u] = blend4_pk<BMODE>(D[0], D[1], D[2], D[3], px[0], px[1], px[2], px[3], px[4], px[5],
                              k.beta);
      }
      const int xs = (s - 4) & 3;
      *reinterpret_cast<float2*>(&ex.X[xs][2 * t + 2]) = make_float2(x4[0], x4[1]);
      if (xs == 0) *reinterpret_cast<float2*>(&ex.X[4][2 * t + 2]) = make_float2(x4[0], x4[1]);
    }
    // stage 2's values for the next step's stage 3 (after this step's use)
    if (FULL || rs >= 0) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int d = 2 * p;
          const f2 v = pk_fma(pk_bc(w), make_float2(C.SI[Q][u][d], C.SI[Q][u][d + 1]),
                              make_float2(C.SI[PH][u][d], C.SI[PH][u][d + 1]));
          C.P[u][d] = v.x;
          C.P[u][d + 1] = v.y;
        }
        C.px[u][0] = a3[u + 2] + a2[u + 3];  // N0 + N1 of the (1,1) diagonal pair
        C.px[u][1] = a3[u + 3] + a2[u + 2];  // N0 + N1 of the (1,-1) pair
        C.px[u][2] = C.S1[PH][u + 1];
        C.px[u][3] = C.S1[Q][u];
        C.px[u][4] = C.S2[PH][u];
        C.px[u][5] = C.S2[Q][u + 1];
      }
    }

    // ---- stage 4: phase-2 indicators at row r = s-5 -------------------------
    float a5[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, a4[2] = {0.f, 0.f};
    if (FULL || rs >= 3) {
      row6(A5, a5);
      const float2 v4 = *reinterpret_cast<const float2*>(A5 + ROW + 2);
      a4[0] = v4.x;
      a4[1] = v4.y;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        C.sVc[PH][u] = fmaf(-2.f, a4[u], a5[u + 2] + a3[u + 2]);
        C.qVc[PH][u] = sq_eps(k.kappa2, C.sVc[PH][u], k.eps2);
      }
    }
    if (FULL || rs >= 4) {
      // phase-1 rows r-1 (s-6) and r (s-5) at columns c0-2 .. c0+3
      const float* x6p = ex.X[(s - 6) & 3] + 2 * t;
      float xr[6], xu[6];
      row6(x6p + ROW, xr);  // row r
      const float2 xo = *reinterpret_cast<const float2*>(x6p + 2);  // row r-1, own columns
      xu[2] = xo.x;
      xu[3] = xo.y;
      // second differences along row r centred at c0 .. c0+2 (input) and
      // c0-1 .. c0+1 (phase-1 values), shared by the pair
      float sH[3], qH[3], sX[3], qX[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        sH[j] = fmaf(-2.f, a5[j + 2], a5[j + 1] + a5[j + 3]);
        qH[j] = sq_eps(k.kappa2, sH[j], k.eps2);
        sX[j] = fmaf(-2.f, xr[j + 1], xr[j] + xr[j + 2]);
        qX[j] = sq_eps(k.kappa2, sX[j], k.eps2);
      }
      float VSo[2][4], VEo[2][4];
      float2 pS01;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float x6 = xu[u + 2], xr2 = xr[u + 2];
        float* SIE = C.SIE[PH][u];
        float* SIS = C.SIS[PH][u];
        float pS[6];
        // E(r, c) horizontal: nodes along input row r
        const float gH = a5[u + 3] - a5[u + 2];
        SIE[0] = fmaf(gH, gH, qH[u + 1]);  // centred at c + 1
        SIE[1] = fmaf(gH, gH, qH[u]);      // centred at c
        // E vertical: nodes along phase-1 column c
        C.sXc[PH][u] = fmaf(-2.f, xr2, x6 + x4[u]);
        C.qXc[PH][u] = sq_eps(k.kappa2, C.sXc[PH][u], k.eps2);
        const float gV = xr2 - x6;
        SIE[2] = fmaf(gV, gV, C.qXc[PH][u]);
        SIE[3] = fmaf(gV, gV, C.qXc[Q][u]);
        // S(r, c) horizontal: nodes along phase-1 row r
        const float gSh = xr2 - xr[u + 1];
        SIS[0] = fmaf(gSh, gSh, qX[u + 1]);  // centred at c
        SIS[1] = fmaf(gSh, gSh, qX[u]);      // centred at c - 1
        // S vertical: nodes along input column c
        const float gSv = a4[u] - a5[u + 2];
        SIS[2] = fmaf(gSv, gSv, C.qVc[PH][u]);
        SIS[3] = fmaf(gSv, gSv, C.qVc[Q][u]);
        pS[0] = xr[u + 1] + xr2;
        pS[1] = a5[u + 2] + a4[u];
        pS[2] = sX[u + 1];
        pS[3] = sX[u];
        pS[4] = C.sVc[PH][u];
        pS[5] = C.sVc[Q][u];
        if (u == 0) {
          ex.PS[PH][0][t] = make_float4(pS[0], pS[1], pS[2], pS[3]);
          pS01 = make_float2(pS[4], pS[5]);
        } else {
          ex.PS[PH][1][t] = make_float4(pS01.x, pS01.y, pS[0], pS[1]);
          ex.PS[PH][2][t] = make_float4(pS[2], pS[3], pS[4], pS[5]);
        }
        C.pE[u][0] = a5[u + 2] + a5[u + 3];
        C.pE[u][1] = x6 + xr2;
        C.pE[u][2] = sH[u + 1];
        C.pE[u][3] = sH[u];
        C.pE[u][4] = C.sXc[PH][u];
        C.pE[u][5] = C.sXc[Q][u];
        C.a5c[u] = a5[u + 2];
        C.x6[u] = x6;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const int d = 2 * p;
          const f2 vs = pk_add(make_float2(C.SIS[Q][u][d], C.SIS[Q][u][d + 1]),
                               make_float2(SIS[d], SIS[d + 1]));
          const f2 ve = pk_add(make_float2(C.SIE[Q][u][d], C.SIE[Q][u][d + 1]),
                               make_float2(SIE[d], SIE[d + 1]));
          VSo[u][d] = vs.x; VSo[u][d + 1] = vs.y;
          VEo[u][d] = ve.x; VEo[u][d + 1] = ve.y;
        }
      }
      // Row-pair sums for Eq. (tezine): S rows r-1, r feed E(r); E rows
      // r-1, r feed S(r-1).  Neighbours need VS of c0 and VE of c1.
      ex.VS[PH][t + 1] = make_float4(VSo[0][0], VSo[0][1], VSo[0][2], VSo[0][3]);
      ex.VE[PH][t + 1] = make_float4(VEo[1][0], VEo[1][1], VEo[1][2], VEo[1][3]);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int d = 2 * p;
        const f2 W = pk_bc(w);
        const f2 vs0 = make_float2(VSo[0][d], VSo[0][d + 1]);
        const f2 vs1 = make_float2(VSo[1][d], VSo[1][d + 1]);
        const f2 ve0 = make_float2(VEo[0][d], VEo[0][d + 1]);
        const f2 ve1 = make_float2(VEo[1][d], VEo[1][d + 1]);
        const f2 dep0 = pk_fma(W, vs0, make_float2(C.SIE[PH][0][d], C.SIE[PH][0][d + 1]));
        const f2 de0 = pk_fma(W, vs1, dep0);  // E(c0) reads VS of c0 and c1
        const f2 dep1 = pk_fma(W, vs1, make_float2(C.SIE[PH][1][d], C.SIE[PH][1][d + 1]));
        const f2 dsp0 = pk_fma(W, ve0, make_float2(C.SIS[Q][0][d], C.SIS[Q][0][d + 1]));
        const f2 dsp1 = pk_fma(W, ve1, make_float2(C.SIS[Q][1][d], C.SIS[Q][1][d + 1]));
        const f2 ds1 = pk_fma(W, ve0, dsp1);  // S(c1) reads VE of c1 and c0
        C.DE0[d] = de0.x; C.DE0[d + 1] = de0.y;
        C.DEp1[d] = dep1.x; C.DEp1[d + 1] = dep1.y;
        C.DSp0[d] = dsp0.x; C.DSp0[d + 1] = dsp0.y;
        C.DS1[d] = ds1.x; C.DS1[d + 1] = ds1.y;
      }
    }
  }

  __device__ __forceinline__ void run() {
    __syncthreads();
    {
      float* z = reinterpret_cast<float*>(&ex);
      for (int i = t; i < (int)(sizeof(Exchange2<NT>) / sizeof(float)); i += NT) z[i] = 0.f;
    }
    const int s_first = a0 - 4;
    const int s_begin = s_first & ~1;
    const int s_last = a0 + H + 5;
    const int s_end = s_last + 1;
    Carry2 C;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
      for (int j = 0; j < 3; ++j) C.S1[i][j] = C.S2[i][j] = 0.f;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
#pragma unroll
        for (int d = 0; d < 4; ++d) C.SI[i][u][d] = C.SIE[i][u][d] = C.SIS[i][u][d] = 0.f;
        C.sXc[i][u] = C.qXc[i][u] = C.sVc[i][u] = C.qVc[i][u] = 0.f;
      }
#pragma unroll
      for (int d = 0; d < 4; ++d) C.P[i][d] = 0.f;
#pragma unroll
      for (int d = 0; d < 6; ++d) C.px[i][d] = C.pE[i][d] = 0.f;
      C.a5c[i] = C.x6[i] = 0.f;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) C.DE0[d] = C.DEp1[d] = C.DSp0[d] = C.DS1[d] = 0.f;
    uint32_t pf[2] = {load_row(s_begin, 0), load_row(s_begin, 1)};
    uint32_t pf2[2] = {load_row(s_begin + 1, 0), load_row(s_begin + 1, 1)};
    int s = s_begin;
    oE = out_base + 2 * (int64_t)(s_begin - 7) * out_sh;
    for (; s <= s_end && s - a0 < 7; s += 2) {
      step<0, false>(s, pf, pf2, C);
      step<1, false>(s + 1, pf, pf2, C);
    }
    for (; s + 1 - a0 <= H + 4 && s + 1 <= n + 5; s += 2) {
      step<0, true>(s, pf, pf2, C);
      step<1, true>(s + 1, pf, pf2, C);
    }
    for (; s <= s_end; s += 2) {
      step<0, false>(s, pf, pf2, C);
      step<1, false>(s + 1, pf, pf2, C);
    }
  }
};

template <int BMODE, class IO, int NT>
__device__ __forceinline__ void zoom2x_fwd_tile2(const FwdArgs& a, const MethodConsts& k,
                                                 Exchange2<NT>& ex, int64_t bx, int64_t by,
                                                 int64_t plane) {
  FwdTile2<BMODE, IO, NT> tile(a, k, ex, bx, by, plane);
  tile.run();
}

}  // namespace fwd_tile
}  // namespace wdweno
