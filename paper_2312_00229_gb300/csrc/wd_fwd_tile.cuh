// Tile body of the fused WD WENO forward pass, shared by the one-launch-per-
// image kernels (wd_fwd*.cu) and the persistent batched kernels
// (wd_batched.cu).  Method: arXiv 2312.00229, Sec. 3, Algorithms 1-2.
//
// Work decomposition
//   One CTA = one plane x one strip of NT - 9 coarse columns x one band of
//   `rows_per_band` coarse rows.  NT threads (256, or 128 for narrow
//   images); thread t owns coarse column c = b0 - 4 + t, so the CTA spans NT
//   columns: the NT - 9 output columns plus the method's 4-before / 5-after
//   dependency halo (an output quad depends on input rows and columns
//   -4..+5).  The CTA sweeps its band
//   top to bottom, one coarse row per step; every stage is computed once per
//   (row, column) of its region.
//
// Shared memory holds rings of recent rows that neighbouring columns read:
// the decoded input rows (8), the phase-1 values (4), the phase-1
// smoothness indicators (2) and the row-pair sums of the phase-2
// indicators.  The input and phase-1 rings repeat their first slots after
// the last, so the rows a step reads are at constant offsets from one slot
// address.  Registers hold only values a thread carries for its own
// column from one step to the next (period-2 rings; the step loop is
// unrolled twice so their indices are compile-time constants).
//
// Pipeline of one step s (input row s is published, row s+2 prefetched):
//   stage 5  (first, from the previous step's stage 4) E(s-6, c) and S(s-7, c)
//            (Eqs. tezine, IzrazOmega2dRavno, 2dKombinacijaRavno)
//   stage 1  row s-2  second differences S1/S2 along both diagonals and their
//                     squared, kappa-scaled forms (columns c, c+1)
//   stage 2  row s-3  the four phase-1 smoothness indicators (Eq.
//                     2Dsmoothness) of X(s-3, c) and its interpolant data
//   stage 3  row s-4  D (Eq. 2DsmoothnessFinal), alpha (Eq. alpha) and the
//                     blend (Eqs. IzrazOmega2d, 2dKombinacija) -> X(s-4, c)
//   stage 4  row s-5  phase-2 indicators of E(s-5, c) and S(s-5, c), their
//                     row-pair sums published for the neighbours (slot = step
//                     parity) and the data stage 5 needs carried to step s+1
//   store             fine row 2(s-6): [A, E], fine row 2(s-7)+1: [S, X]
// One barrier (B1) opens each step: every shared value a step reads was
// written in an earlier step, in a slot no thread writes in the same step.
//
// Input: each thread loads its (clamped) column of input row s+2 in step s,
// as the element's storage bits, and converts it to FP32 in step s+2, where
// it publishes the row to the ring.  Nothing waits for the load until then:
// the loaded register is only renamed in between (the step loop is unrolled
// twice), and the barriers do not wait for loads in flight.
#pragma once

#include "wd_common.cuh"
#include "wd_fwd.h"

namespace wdweno {
namespace fwd_tile {

// CTA widths: NT threads, one coarse column each, cover NT - 9 output
// columns.  256 is the default; 128 serves narrow images (a smaller part of
// the last strip idles), with four CTAs per SM instead of two.
constexpr int THREADS = 256;
constexpr int THREADS_NARROW = 128;
constexpr int HALO_L = 4;            // columns before the strip
constexpr int TILE_W = THREADS - 9;  // output columns per CTA
template <int NT>
struct Shape {
  static constexpr int TW = NT - 9;   // output columns per CTA
  static constexpr int ROW = NT + 4;  // floats per staged row (2 pad each side)
};

template <int NT>
struct __align__(16) ExchangeT {
  static constexpr int ROW = Shape<NT>::ROW;
  float A[12][ROW];           // input rows, slot = row & 7, column c at t + 2; slots
                              // 8..11 repeat 0..3 so five consecutive rows are
                              // at consecutive slots from any start
  float X[5][ROW];            // phase-1 values, slot = row & 3, column c at t + 2; slot
                              // 4 repeats 0
  float4 SI[2][NT + 2];       // phase-1 SIs (directions A, B, C, D), slot = row & 1,
                              // column c at t + 1
  float4 VS[2][NT + 2];       // S-point SIs summed over rows r-1, r (column c at t + 1),
                              // slot = step parity
  float4 VE[2][NT + 2];       // E-point SIs summed over rows r-1, r
};
using Exchange = ExchangeT<THREADS>;
static_assert(sizeof(Exchange) <= 48 * 1024, "static shared memory");

// Bounded waits that gave up in the kernels of this translation unit (each
// kernel TU has its own counter; see read_wait_timeouts).  The fused
// cascade's waits between levels are the ones that count here.
static __device__ unsigned int g_wait_timeouts;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Host side: this TU's count of abandoned waits (optionally reset to 0).
static inline cudaError_t read_wait_timeouts(unsigned int* v, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(v, g_wait_timeouts, sizeof(unsigned int));
  if (e == cudaSuccess && reset) {
    const unsigned int z = 0;
    e = cudaMemcpyToSymbol(g_wait_timeouts, &z, sizeof(unsigned int));
  }
  return e;
}

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ float sq_eps(float kappa, float s, float eps) {
  float t = kappa * s;
  return fmaf(t, t, eps);
}

// Values a thread carries from one step to the next (slot = step parity).
struct Carry {
  float S1[2][2], S2[2][2], q1[2][2], q2[2][2];  // stage 1, columns c, c+1
  float SI[2][4], P[2][4], px[2][6];             // stage 2
  float sXc[2], qXc[2], sVc[2], qVc[2];          // stage 4 column differences
  float SIE[2][4], SIS[2][4], pS[2][6];          // stage 4
  // stage 4 results that stage 5 uses one step later
  float DEp[4], DSp[4], pE[6], a5c, x6;
};

template <int BMODE, class IO, int NT>
struct FwdTile {
  static constexpr int TILE_W = Shape<NT>::TW;
  static constexpr int ROW = Shape<NT>::ROW;
  // Arguments are held by value so that they stay in registers across the
  // barriers (a reference would be re-read from memory after each one).
  const MethodConsts k;
  ExchangeT<NT>& ex;
  const int t;
  const void* in;
  void* out;
  int in_dtype, out_dtype;
  int n, a0, H;              // coarse rows; band start; band height
  int orows;
  int64_t in_idx, in_sh;     // element index of (row 0, column c); row stride
  int64_t out_base, out_sh;  // element index of (fine row 0, fine column 2c)
  int64_t out_sw;
  int64_t oE;                // element index of (fine row 2(s-6), fine column 2c) in step s
  bool col_ok, vec_ok, odd_ok;

  __device__ __forceinline__ FwdTile(const FwdArgs& a, const MethodConsts& k_, ExchangeT<NT>& ex_,
                                     int64_t bx, int64_t by, int64_t plane)
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
    const int64_t c = b0 - HALO_L + t;
    in_idx = plane * a.in_sc + clamp64(c, 0, a.m - 1) * a.in_sw;
    in_sh = a.in_sh;
    col_ok = (c >= b0) && (c < b0 + TILE_W) && (c < a.m);
    odd_ok = 2 * c + 1 < a.ocols;
    vec_ok = a.out_vec && col_ok && odd_ok;
    out_sw = a.out_sw;
    out_sh = a.out_sh;
    out_base = plane * a.out_sc + 2 * c * a.out_sw;
  }

  // Storage bits of input row r (clamped), column c.
  __device__ __forceinline__ uint32_t load_row(int r) const {
    const int rc = r < 0 ? 0 : (r > n - 1 ? n - 1 : r);
    return IO::load_bits(in, in_idx + (int64_t)rc * in_sh, in_dtype);
  }

  // Element index `base` (fine row, column 2c) and the next column.
  __device__ __forceinline__ void store_pair(int64_t base, float v0, float v1) const {
    if (vec_ok) {
      IO::store2(out, base, v0, v1, out_dtype, k.clamp_float);
    } else if (col_ok) {
      IO::store1(out, base, v0, out_dtype, k.clamp_float);
      if (odd_ok) IO::store1(out, base + out_sw, v1, out_dtype, k.clamp_float);
    }
  }

  // Columns c-1 .. c+2 of the row at `p` (column c-1).
  __device__ __forceinline__ static void row4(const float* p, float (&v)[4]) {
    v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
  }
  // Publishes input row r, column c (and its repeat slot).
  __device__ __forceinline__ void put_row(int r, float v) const {
    const int sl = r & 7;
    ex.A[sl][t + 2] = v;
    if (sl < 4) ex.A[sl + 8][t + 2] = v;
  }

  // FULL: a step in the middle of the band, where every stage's row is
  // inside the band (7 <= rs <= H + 4) and every stored row inside the
  // output: the guards are compiled out so the whole step is one block for
  // the scheduler.
  template <int PH, bool FULL>
  __device__ __forceinline__ void step(int s, uint32_t& pf, uint32_t& pf2, Carry& C) {
    constexpr int Q = PH ^ 1;  // slot written by the previous step
    const int rs = s - a0;
    if (!FULL && rs > H + 6) return;  // padding step past the band (uniform)
    const float w = k.w;
    oE += 2 * out_sh;

    const uint32_t cur = pf;  // input row s, loaded in step s-2 (storage bits)
    pf = pf2;
    pf2 = load_row(s + 2);    // prefetch two rows ahead

    __syncthreads();  // B1: rows published in step s-1 are visible
    put_row(s, IO::value(cur, in_dtype));  // converted here, where it is used

    // ---- stage 5: E(s-6, c) and S(s-7, c) from the previous step's stage 4 --
    // (E row r is stage-4 row s-6 of step s-1; the S blend's data pS was
    // written two steps ago, in the slot of this step's parity, which stage 4
    // below overwrites)
    if (FULL || (rs >= 6 && rs <= H + 5)) {
      const float4 v = ex.VS[PH ^ 1][t + 2];  // column c+1 (slot of step s-1)
      const float vs[4] = {v.x, v.y, v.z, v.w};
      float D[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) D[d] = fmaf(w, vs[d], C.DEp[d]);
      const float e = blend4<BMODE>(D[0], D[1], D[2], D[3], C.pE[0], C.pE[1], C.pE[2], C.pE[3],
                                    C.pE[4], C.pE[5], k.beta);
      const int rE = s - 6;  // fine row 2 rE: [A, E]
      if (FULL || (rE < n && 2 * rE < orows)) store_pair(oE, C.a5c, e);
    }
    if (FULL || rs >= 7) {
      const float4 v = ex.VE[PH ^ 1][t];  // column c-1
      const float ve[4] = {v.x, v.y, v.z, v.w};
      float D[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) D[d] = fmaf(w, ve[d], C.DSp[d]);
      const float* p = C.pS[PH];
      const float sv = blend4<BMODE>(D[0], D[1], D[2], D[3], p[0], p[1], p[2], p[3], p[4], p[5],
                                     k.beta);
      const int rS = s - 7;  // fine row 2 rS + 1: [S, X]
      if (FULL || (rS < n && 2 * rS + 1 < orows)) store_pair(oE - out_sh, sv, C.x6);
    }


    // Input rows s-5 .. s-1 sit at consecutive slots from (s-5) & 7.
    const float* A5 = ex.A[(s - 5) & 7] + t + 1;  // row s-5, column c-1
    // Input rows s-3, s-2, s-1 at columns c-1..c+2 (index u + 1).
    float a1[4], a2[4], a3[4];
    row4(A5 + 4 * ROW, a1);
    row4(A5 + 3 * ROW, a2);
    row4(A5 + 2 * ROW, a3);

    // ---- stage 1: diagonal second differences at row s-2, columns c, c+1 --
    // S1(i,j) = A(i-1,j-1) - 2A(i,j) + A(i+1,j+1);  S2 along (1,-1)
    if (FULL || rs >= -1) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        C.S1[PH][u] = fmaf(-2.f, a2[u + 1], a3[u] + a1[u + 2]);
        C.S2[PH][u] = fmaf(-2.f, a2[u + 1], a3[u + 2] + a1[u]);
        C.q1[PH][u] = sq_eps(k.kappa1, C.S1[PH][u], k.eps1);
        C.q2[PH][u] = sq_eps(k.kappa1, C.S2[PH][u], k.eps1);
      }
    }

    // ---- stage 2: phase-1 SIs of X(s-3, c) ----------------------------------
    // X(a,b) sits between A(a,b) and A(a+1,b+1).  Directions:
    //   A (1,1):   nodes A(a,b),   A(a+1,b+1), A(a+2,b+2); s = S1(a+1,b+1)
    //   B (-1,-1): nodes A(a+1,b+1), A(a,b),   A(a-1,b-1); s = S1(a,b)
    //   C (1,-1):  nodes A(a,b+1), A(a+1,b),   A(a+2,b-1); s = S2(a+1,b)
    //   D (-1,1):  nodes A(a+1,b), A(a,b+1),   A(a-1,b+2); s = S2(a,b+1)
    if (FULL || rs >= 0) {
      const float G1 = a2[2] - a3[1];  // A(a+1,b+1) - A(a,b)
      const float G2 = a2[1] - a3[2];  // A(a+1,b) - A(a,b+1)
      float* SI = C.SI[PH];
      SI[0] = fmaf(G1, G1, C.q1[PH][1]);
      SI[1] = fmaf(G1, G1, C.q1[Q][0]);
      SI[2] = fmaf(G2, G2, C.q2[PH][0]);
      SI[3] = fmaf(G2, G2, C.q2[Q][1]);
      ex.SI[PH ^ 1][t + 1] = make_float4(SI[0], SI[1], SI[2], SI[3]);  // slot (s-3) & 1
#pragma unroll
      for (int d = 0; d < 4; ++d) C.P[PH][d] = fmaf(w, C.SI[Q][d], SI[d]);
      C.px[PH][0] = a3[1] + a2[2];  // N0 + N1 of the (1,1) diagonal pair
      C.px[PH][1] = a3[2] + a2[1];  // N0 + N1 of the (1,-1) pair
      C.px[PH][2] = C.S1[PH][1];
      C.px[PH][3] = C.S1[Q][0];
      C.px[PH][4] = C.S2[PH][0];
      C.px[PH][5] = C.S2[Q][1];
    }

    // ---- stage 3: X(s-4, c) -------------------------------------------------
    // D = SI(a) + w (SI(a-1) + SI(a+1) + SI(a, c-1) + SI(a, c+1)), where the
    // partial P(a) = SI(a) + w SI(a-1) was formed one step earlier.
    float x4 = 0.f;
    if (FULL || rs >= 2) {
      const float4 l = ex.SI[PH][t];  // slot (s-4) & 1
      const float4 r = ex.SI[PH][t + 2];
      const float hl[4] = {l.x, l.y, l.z, l.w};
      const float hr[4] = {r.x, r.y, r.z, r.w};
      float D[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) D[d] = fmaf(w, C.SI[PH][d] + (hl[d] + hr[d]), C.P[Q][d]);
      const float* px = C.px[Q];
      x4 = blend4<BMODE>(D[0], D[1], D[2], D[3], px[0], px[1], px[2], px[3], px[4], px[5],
                         k.beta);
      const int xs = (s - 4) & 3;
      ex.X[xs][t + 2] = x4;
      if (xs == 0) ex.X[4][t + 2] = x4;
    }

    // ---- stage 4: phase-2 indicators at row r = s-5 -------------------------
    // Direction order for both "+" classes: (0,1), (0,-1), (1,0), (-1,0).
    // The column second difference of A centred at A(r+1) is carried to the
    // next step as the one centred at A(r), so it starts one row early.
    float a5[4] = {0.f, 0.f, 0.f, 0.f}, a4 = 0.f;
    if (FULL || rs >= 3) {
      row4(A5, a5);
      a4 = A5[ROW + 1];
      C.sVc[PH] = fmaf(-2.f, a4, a5[1] + a3[1]);
      C.qVc[PH] = sq_eps(k.kappa2, C.sVc[PH], k.eps2);
    }
    float DEp[4], DSp[4], pE[6], x6 = 0.f;
    if (FULL || rs >= 4) {
      // phase-1 row r at columns c-2..c+1, and column c at row r-1
      const float* x6p = ex.X[(s - 6) & 3] + t;  // rows s-6, s-5 at consecutive slots
      const float* xp = x6p + ROW;
      const float xr0 = xp[0], xr1 = xp[1], xr2 = xp[2], xr3 = xp[3];
      x6 = x6p[2];
      float* SIE = C.SIE[PH];
      float* SIS = C.SIS[PH];
      float* pS = C.pS[PH];
      // E(r, c) horizontal: nodes along input row r
      const float sHp = fmaf(-2.f, a5[2], a5[1] + a5[3]);  // centred at c+1
      const float sHm = fmaf(-2.f, a5[1], a5[0] + a5[2]);  // centred at c
      const float gH = a5[2] - a5[1];
      SIE[0] = fmaf(gH, gH, sq_eps(k.kappa2, sHp, k.eps2));
      SIE[1] = fmaf(gH, gH, sq_eps(k.kappa2, sHm, k.eps2));
      // E vertical: nodes along phase-1 column c
      C.sXc[PH] = fmaf(-2.f, xr2, x6 + x4);  // centred at X(r)
      C.qXc[PH] = sq_eps(k.kappa2, C.sXc[PH], k.eps2);
      const float gV = xr2 - x6;
      SIE[2] = fmaf(gV, gV, C.qXc[PH]);
      SIE[3] = fmaf(gV, gV, C.qXc[Q]);
      pE[0] = a5[1] + a5[2];
      pE[1] = x6 + xr2;
      pE[2] = sHp;
      pE[3] = sHm;
      pE[4] = C.sXc[PH];
      pE[5] = C.sXc[Q];
      // S(r, c) horizontal: nodes along phase-1 row r
      const float sXp = fmaf(-2.f, xr2, xr1 + xr3);  // centred at c
      const float sXm = fmaf(-2.f, xr1, xr0 + xr2);  // centred at c-1
      const float gSh = xr2 - xr1;
      SIS[0] = fmaf(gSh, gSh, sq_eps(k.kappa2, sXp, k.eps2));
      SIS[1] = fmaf(gSh, gSh, sq_eps(k.kappa2, sXm, k.eps2));
      // S vertical: nodes along input column c
      const float gSv = a4 - a5[1];
      SIS[2] = fmaf(gSv, gSv, C.qVc[PH]);
      SIS[3] = fmaf(gSv, gSv, C.qVc[Q]);
      pS[0] = xr1 + xr2;
      pS[1] = a5[1] + a4;
      pS[2] = sXp;
      pS[3] = sXm;
      pS[4] = C.sVc[PH];
      pS[5] = C.sVc[Q];
      // Row-pair sums for Eq. (tezine): S rows r-1, r feed E(r); E rows
      // r-1, r feed S(r-1).  Own-column parts of both D sums are added here.
      float VS[4], VE[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        VS[d] = C.SIS[Q][d] + SIS[d];
        VE[d] = C.SIE[Q][d] + SIE[d];
        DEp[d] = fmaf(w, VS[d], SIE[d]);
        DSp[d] = fmaf(w, VE[d], C.SIS[Q][d]);
      }
      ex.VS[PH][t + 1] = make_float4(VS[0], VS[1], VS[2], VS[3]);
      ex.VE[PH][t + 1] = make_float4(VE[0], VE[1], VE[2], VE[3]);
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        C.DEp[d] = DEp[d];
        C.DSp[d] = DSp[d];
      }
#pragma unroll
      for (int d = 0; d < 6; ++d) C.pE[d] = pE[d];
      C.a5c = a5[1];
      C.x6 = x6;
    }
  }

  __device__ __forceinline__ void run() {
    // Zero the shared rings so that reads at the strip edges and before the
    // first writes see finite values.
    __syncthreads();
    {
      float* z = reinterpret_cast<float*>(&ex);
      for (int i = t; i < (int)(sizeof(ExchangeT<NT>) / sizeof(float)); i += NT) z[i] = 0.f;
    }
    // The sweep starts on an even row, so that step<PH> runs on rows of
    // parity PH and the parity-slotted rings have compile-time indices; an
    // odd a0 - 4 adds one leading step in which every stage is idle.
    const int s_first = a0 - 4;          // first input row the band needs
    const int s_begin = s_first & ~1;
    const int s_last = a0 + H + 5;   // last input row of the band's sweep
    const int s_end = s_last + 1;    // inclusive: one more step finishes stage 5
    Carry C;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
      for (int u = 0; u < 2; ++u) C.S1[i][u] = C.S2[i][u] = C.q1[i][u] = C.q2[i][u] = 0.f;
#pragma unroll
      for (int d = 0; d < 4; ++d) C.SI[i][d] = C.P[i][d] = C.SIE[i][d] = C.SIS[i][d] = 0.f;
#pragma unroll
      for (int d = 0; d < 6; ++d) C.px[i][d] = C.pS[i][d] = 0.f;
      C.sXc[i] = C.qXc[i] = C.sVc[i] = C.qVc[i] = 0.f;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) C.DEp[d] = C.DSp[d] = 0.f;
#pragma unroll
    for (int d = 0; d < 6; ++d) C.pE[d] = 0.f;
    C.a5c = C.x6 = 0.f;
    uint32_t pf = load_row(s_begin);
    uint32_t pf2 = load_row(s_begin + 1);
    int s = s_begin;
    oE = out_base + 2 * (int64_t)(s_begin - 7) * out_sh;  // advanced at the top of each step
    for (; s <= s_end && s - a0 < 7; s += 2) {  // pipeline fill
      step<0, false>(s, pf, pf2, C);
      step<1, false>(s + 1, pf, pf2, C);
    }
    // every stage's row inside the band, every stored row inside the output
    for (; s + 1 - a0 <= H + 4 && s + 1 <= n + 5; s += 2) {
      step<0, true>(s, pf, pf2, C);
      step<1, true>(s + 1, pf, pf2, C);
    }
    for (; s <= s_end; s += 2) {  // drain
      step<0, false>(s, pf, pf2, C);
      step<1, false>(s + 1, pf, pf2, C);
    }
  }
};

// Storage access with the types fixed at compile time.
template <class TIn, class TOut>
struct TypedIO {
  __device__ __forceinline__ static uint32_t load_bits(const void* base, int64_t idx, int) {
    return load_elem_bits(base, idx, DTypeOf<TIn>::value);
  }
  __device__ __forceinline__ static float value(uint32_t b, int) {
    return elem_bits_value(b, DTypeOf<TIn>::value);
  }
  __device__ __forceinline__ static void store1(void* out, int64_t idx, float v, int, int clampf) {
    store_typed<TOut>(out, idx, v, clampf);
  }
  __device__ __forceinline__ static void store2(void* out, int64_t idx, float v0, float v1, int,
                                                int clampf) {
    store2_typed<TOut>(out, idx, v0, v1, clampf);
  }
  __device__ __forceinline__ static void store4(void* out, int64_t idx, float v0, float v1,
                                                float v2, float v3, int, int clampf) {
    store4_typed<TOut>(out, idx, v0, v1, v2, v3, clampf);
  }
};

// Storage types chosen at run time (any in/out pair).
struct DynIO {
  __device__ __forceinline__ static uint32_t load_bits(const void* base, int64_t idx, int dt) {
    return load_elem_bits(base, idx, dt);
  }
  __device__ __forceinline__ static float value(uint32_t b, int dt) {
    return elem_bits_value(b, dt);
  }
  __device__ __forceinline__ static void store1(void* out, int64_t idx, float v, int dt,
                                                int clampf) {
    store_elem(out, idx, v, dt, clampf);
  }
  __device__ __forceinline__ static void store2(void* out, int64_t idx, float v0, float v1,
                                                int dt, int clampf) {
    store2_vec(out, idx, v0, v1, dt, clampf);
  }
  __device__ __forceinline__ static void store4(void* out, int64_t idx, float v0, float v1,
                                                float v2, float v3, int dt, int clampf) {
    store4_vec(out, idx, v0, v1, v2, v3, dt, clampf);
  }
};

template <int BMODE, class IO, int NT = THREADS>
__device__ __forceinline__ void zoom2x_fwd_tile(const FwdArgs& a, const MethodConsts& k,
                                                ExchangeT<NT>& ex, int64_t bx, int64_t by,
                                                int64_t plane) {
  FwdTile<BMODE, IO, NT> tile(a, k, ex, bx, by, plane);
  tile.run();
}

}  // namespace fwd_tile
}  // namespace wdweno
