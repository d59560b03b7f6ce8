// Adjoint of the WD WENO 2x zoom (arXiv 2312.00229, Sec. 3), FP32.
//
// For one blend point u = sum_k omega_k p_k with omega_k = alpha_k / sum alpha
// and alpha_k = D_k^-beta (Eqs. alpha, IzrazOmega2d, 2dKombinacija and the
// phase-2 forms), the local adjoints of an incoming u_bar are
//     p_bar_k = u_bar omega_k
//     D_bar_k = -u_bar beta omega_k (p_k - u) / D_k .
// D_k = SI_k(c) + w sum_{nbr} SI_k(c + delta) (Eqs. 2DsmoothnessFinal, tezine),
// so SI_bar_k(c) = D_bar_k(c) + w sum of D_bar_k over the points whose D
// reads c.  With SI = g^2 + kappa^2 s^2 + eps', g = N1 - N0,
// s = N0 - 2 N1 + N2 and p = 3/8 N0 + 3/4 N1 - 1/8 N2 (Eq. p), a stencil
// sends to its nodes
//     N0: 3/8 p_bar + (-2 g + 2 kappa^2 s) SI_bar
//     N1: 3/4 p_bar + ( 2 g - 4 kappa^2 s) SI_bar
//     N2: -1/8 p_bar + 2 kappa^2 s SI_bar .
//
// Two row-sweep kernels, each CTA one plane x one strip of columns x one band
// of rows, sweeping its band top to bottom one coarse row per step with one
// barrier per step; every intermediate lives in shared-memory rings of
// recent rows (slot = row mod ring depth), and a stage at step s works on
// row s - L for its own lag L, reading only rows written in earlier steps.
//
//   k_bwd_plus   recomputes the forward pass (phase-1 indicators and values,
//                phase-2 indicators) and runs the phase-2 adjoint: p_bar,
//                D_bar of every E and S point, their SI_bar and the node
//                coefficients, gathered onto the x points (X_bar, plus the
//                x-point output gradient) and onto the input samples (plus
//                the sample-point output gradient).  Writes X_bar and that
//                partial A_bar on the grid extended by 2 cells per side.
//   k_bwd_cross  recomputes the phase-1 indicators, runs the phase-1 adjoint
//                from X_bar, gathers the node coefficients onto the samples,
//                adds the partial A_bar and folds the clamp-to-edge
//                extension back onto the edge pixels (its adjoint).
// Scatters are gathers: a contribution to a thread's own column is added to
// a short register ring of row accumulators, contributions to other columns
// are published per row in shared memory and gathered one step later.
// In the middle of a band the steps run in groups of four with every ring
// slot a compile-time constant and no stage guards (sweep_band); the global
// values a step needs are loaded three to five (input rows: two or four) steps
// before it.
#include "wd_bwd.h"
#include "wd_packed.cuh"

namespace wdweno {

namespace {

// ---- shared-memory rings ------------------------------------------------------
constexpr int PAD = 2;  // ring columns before / after the CTA's threads

// k_bwd_plus: thread t owns column c = b0 - HL1 + t of a strip whose outputs
// are columns [b0, b0 + NT - HL1 - HR1) of the extended grid.
constexpr int HL1 = 6, HR1 = 7;
// k_bwd_cross: the strip's outputs are image columns [b0, b0 + NT - HL2 - HR2)
// plus, at the image edges, the ghost columns folded onto them.
constexpr int HL2 = 10, HR2 = 10;
// CTA widths built for both sweeps (the host picks one per image width)
constexpr int NT_NARROW = 128, NT_WIDE = 192;
constexpr int GA = 5;  // ghost rows / columns of A_bar (nonzero up to 4)

template <int NT>
struct RingsPlus {
  static constexpr int W = NT + 2 * PAD;
  float A[16][W];     // input rows, slot = row & 15
  float X[16][W];     // phase-1 values
  float4 SIX[4][W];   // phase-1 indicators (4 directions)
  float4 SIE[4][W];   // E-point indicators
  float4 SIS[4][W];   // S-point indicators
  float4 DE[4][W];    // E 2 D_bar
  float4 DS[4][W];    // S 2 D_bar
  // Row stencils' node contributions pre-summed by target column, one array
  // per target so that each gather reads a scalar per thread (no strided
  // component reads of a vector array)
  float EH[4][2][W];  // E along row r: to sample columns c-1, c, c+1, c+2
  float SH[4][4][W];  // S along row r: to x columns c-2, c-1, c, c+1
};

template <int NT>
struct RingsCross {
  static constexpr int W = NT + 2 * PAD;
  float A[16][W];
  float4 SIX[4][W];
  float4 PX[4][W];    // x p_bar
  float4 DX[4][W];    // x 2 D_bar
  float2 C1[2][W];    // contributions to column c+1: rows a, a+1
  float2 C2[2][W];    // to column c+2: rows a+2, a-1
  float2 CM[2][W];    // to column c-1: rows a-1, a+2
  float AF[2][W];     // row-folded A_bar of the row emitted in the previous step
};

// ---- the method's per-point quantities ---------------------------------------
struct Sten {
  float g[4], s[4];  // N1 - N0 and N0 - 2 N1 + N2 per direction
  float M[2];        // N0 + N1 of the direction pairs (0,1) and (2,3)
};

__device__ __forceinline__ void sten(float n0, float n1, float n2, float& g, float& s) {
  g = n1 - n0;
  s = fmaf(-2.f, n1, n0 + n2);
}

// x point X(a,b) (fine (2a+1, 2b+1)).  Directions: 0 (1,1): A(a,b),
// A(a+1,b+1), A(a+2,b+2); 1 (-1,-1): A(a+1,b+1), A(a,b), A(a-1,b-1);
// 2 (1,-1): A(a,b+1), A(a+1,b), A(a+2,b-1); 3 (-1,1): A(a+1,b), A(a,b+1),
// A(a-1,b+2).  am1..a2: rows a-1 .. a+2 at column b.
__device__ __forceinline__ Sten sten_x(const float* am1, const float* a0, const float* a1,
                                       const float* a2) {
  Sten q;
  sten(a0[0], a1[1], a2[2], q.g[0], q.s[0]);
  sten(a1[1], a0[0], am1[-1], q.g[1], q.s[1]);
  sten(a0[1], a1[0], a2[-1], q.g[2], q.s[2]);
  sten(a1[0], a0[1], am1[2], q.g[3], q.s[3]);
  q.M[0] = a0[0] + a1[1];
  q.M[1] = a0[1] + a1[0];
  return q;
}

// E point E(r,c) (fine (2r, 2c+1)).  0 (0,1): A(r,c), A(r,c+1), A(r,c+2);
// 1 (0,-1): A(r,c+1), A(r,c), A(r,c-1); 2 (1,0): X(r-1,c), X(r,c), X(r+1,c);
// 3 (-1,0): X(r,c), X(r-1,c), X(r-2,c).  ar: row r of A at column c;
// xm2..x1: rows r-2 .. r+1 of X at column c.
__device__ __forceinline__ Sten sten_e(const float* ar, float xm2, float xm1, float x0,
                                       float x1) {
  Sten q;
  sten(ar[0], ar[1], ar[2], q.g[0], q.s[0]);
  sten(ar[1], ar[0], ar[-1], q.g[1], q.s[1]);
  sten(xm1, x0, x1, q.g[2], q.s[2]);
  sten(x0, xm1, xm2, q.g[3], q.s[3]);
  q.M[0] = ar[0] + ar[1];
  q.M[1] = xm1 + x0;
  return q;
}

// S point S(r,c) (fine (2r+1, 2c)).  0 (0,1): X(r,c-1), X(r,c), X(r,c+1);
// 1 (0,-1): X(r,c), X(r,c-1), X(r,c-2); 2 (1,0): A(r,c), A(r+1,c), A(r+2,c);
// 3 (-1,0): A(r+1,c), A(r,c), A(r-1,c).  xr: row r of X at column c;
// am1..a2: rows r-1 .. r+2 of A at column c.
__device__ __forceinline__ Sten sten_s(const float* xr, float am1, float a0, float a1,
                                       float a2) {
  Sten q;
  sten(xr[-1], xr[0], xr[1], q.g[0], q.s[0]);
  sten(xr[0], xr[-1], xr[-2], q.g[1], q.s[1]);
  sten(a0, a1, a2, q.g[2], q.s[2]);
  sten(a1, a0, am1, q.g[3], q.s[3]);
  q.M[0] = xr[-1] + xr[0];
  q.M[1] = a0 + a1;
  return q;
}

// The helpers below work on the direction pairs (0, 1) and (2, 3) with the
// packed two-lane FP32 instructions of wd_packed.cuh; every lane takes the
// scalar expression's operations in the scalar order.
__device__ __forceinline__ f2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ f2 pair(const float* v, int p) {
  return make_float2(v[2 * p], v[2 * p + 1]);
}

// SI_k = g_k^2 + (kappa s_k)^2 + eps
__device__ __forceinline__ float4 indicators(const Sten& q, float kap, float eps) {
  f2 si[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const f2 g = pair(q.g, p);
    const f2 ks = pk_mul(pk_bc(kap), pair(q.s, p));
    si[p] = pk_fma(g, g, pk_fma(ks, ks, pk_bc(eps)));
  }
  return make_float4(si[0].x, si[0].y, si[1].x, si[1].y);
}

// D_k = own_k + w (n0 + n1 + n2 + n3)_k
__device__ __forceinline__ void smooth(const float4& own, const float4& n0, const float4& n1,
                                       const float4& n2, const float4& n3, float w, float D[4]) {
  const f2 W = pk_bc(w);
  const f2 d01 =
      pk_fma(W, pk_add(pk_add(lo2(n0), lo2(n1)), pk_add(lo2(n2), lo2(n3))), lo2(own));
  const f2 d23 =
      pk_fma(W, pk_add(pk_add(hi2(n0), hi2(n1)), pk_add(hi2(n2), hi2(n3))), hi2(own));
  D[0] = d01.x; D[1] = d01.y; D[2] = d23.x; D[3] = d23.y;
}

// Normalised weights omega_k from D_k (Eqs. alpha, IzrazOmega2d), and 1/D_k.
template <int BMODE>
__device__ __forceinline__ void weights(const float D[4], float beta, float om[4], float rD[4]) {
  f2 al[2], rd[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) rd[p] = pk_rcp(make_float2(D[2 * p], D[2 * p + 1]));
  if (BMODE == B0) {
    al[0] = al[1] = pk_bc(1.f);
  } else {
    const f2 dmin = pk_bc(fminf(fminf(D[0], D[1]), fminf(D[2], D[3])));
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const f2 r = pk_mul(dmin, rd[p]);
      if (BMODE == B2) {
        al[p] = pk_mul(r, r);
      } else {
        const f2 l = pk_mul(pk_bc(beta), make_float2(lg2_approx(r.x), lg2_approx(r.y)));
        al[p] = make_float2(ex2_approx(l.x), ex2_approx(l.y));
      }
    }
  }
  // the largest alpha is 1, so the sum lies in [1, 4]
  const f2 inv = pk_bc(rcp_approx((al[0].x + al[0].y) + (al[1].x + al[1].y)));
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const f2 o = pk_mul(al[p], inv);
    om[2 * p] = o.x; om[2 * p + 1] = o.y;
    rD[2 * p] = rd[p].x; rD[2 * p + 1] = rd[p].y;
  }
}

// p_k = (N0 + N1)/2 - s_k/8 (Eq. p)
__device__ __forceinline__ void interp4(const Sten& q, float ip[4]) {
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const f2 v = pk_fma(pk_bc(-0.125f), pair(q.s, p), pk_bc(0.5f * q.M[p]));
    ip[2 * p] = v.x; ip[2 * p + 1] = v.y;
  }
}

// p_bar and 2 D_bar of one blend point given its D and stencil data (D_bar
// is carried doubled: the node coefficients' factors of 2 fold into it).
template <int BMODE>
__device__ __forceinline__ void point_adjoint(const Sten& q, const float D[4], float beta,
                                              float ub, float4& pb4, float4& db4) {
  float om[4], rD[4];
  weights<BMODE>(D, beta, om, rD);
  // p_k - u from differences of the stencil data, so that no two O(1)
  // values cancel: d_k = p_k - p_0 = (M_k - M_0)/2 - (s_k - s_0)/8 and
  // u - p_0 = sum_l omega_l d_l, so p_k - u = d_k - sum_l omega_l d_l.
  const float hM = 0.5f * (q.M[1] - q.M[0]);
  const float d1 = -0.125f * (q.s[1] - q.s[0]);
  const float d2 = fmaf(-0.125f, q.s[2] - q.s[0], hM);
  const float d3 = fmaf(-0.125f, q.s[3] - q.s[0], hM);
  const float v = fmaf(om[1], d1, fmaf(om[2], d2, om[3] * d3));
  const f2 pu[2] = {make_float2(-v, d1 - v), pk_sub(make_float2(d2, d3), pk_bc(v))};
  const float ubb = -ub * (2.f * beta);
  f2 pb[2], db[2];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const f2 o = pair(om, p);
    pb[p] = pk_mul(pk_bc(ub), o);
    db[p] = BMODE == B0 ? pk_bc(0.f)
                        : pk_mul(pk_mul(pk_mul(pk_bc(ubb), o), pu[p]), pair(rD, p));
  }
  pb4 = make_float4(pb[0].x, pb[0].y, pb[1].x, pb[1].y);
  db4 = make_float4(db[0].x, db[0].y, db[1].x, db[1].y);
}

// Node coefficients (N0, N1, N2) of the four stencils of a point; sb2 holds
// 2 SI_bar.
__device__ __forceinline__ void node_coefs(const Sten& q, const float4& pb, const float sb2[4],
                                           float k2, float c[4][3]) {
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const f2 pbar = p ? hi2(pb) : lo2(pb);
    const f2 sb = pair(sb2, p);
    const f2 g2 = pk_mul(pair(q.g, p), sb);
    const f2 s2 = pk_mul(pk_mul(pk_bc(k2), pair(q.s, p)), sb);
    const f2 c0 = pk_fma(pk_bc(0.375f), pbar, pk_sub(s2, g2));
    const f2 c1 = pk_fma(pk_bc(0.75f), pbar, pk_fma(pk_bc(-2.f), s2, g2));
    const f2 c2 = pk_fma(pk_bc(-0.125f), pbar, s2);
    c[2 * p][0] = c0.x; c[2 * p + 1][0] = c0.y;
    c[2 * p][1] = c1.x; c[2 * p + 1][1] = c1.y;
    c[2 * p][2] = c2.x; c[2 * p + 1][2] = c2.y;
  }
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

// Extended-grid planes of the workspace: X_bar and the partial A_bar,
// (n + 2 BWD_GHOST) x (m + 2 BWD_GHOST) floats each, per plane.
struct WsPlane {
  float* xb;
  float* ab;
  int64_t ld;  // row stride
  __device__ __forceinline__ int64_t idx(int r, int c) const {
    return (int64_t)(r + BWD_GHOST) * ld + (c + BWD_GHOST);
  }
};

__device__ __forceinline__ WsPlane ws_plane(const BwdArgs& a, int64_t plane) {
  WsPlane w;
  w.ld = a.m + 2 * BWD_GHOST;
  const int64_t cells = (a.n + 2 * BWD_GHOST) * w.ld;
  w.xb = a.ws + plane * 2 * cells;
  w.ab = w.xb + cells;
  return w;
}

// ---- ring addressing of one step ---------------------------------------------
// A step at row s reads ring rows s - L for lags L known at compile time.
// RowsRT computes every slot from s at run time (slot = row mod depth);
// RowsCT<PH> serves the steps s = 4 G + PH of a four-step group: the rows of
// a 16-row ring fall into four groups of four consecutive slots, whose
// addresses (RingGroups) are formed once per group of steps, and row s - L
// lies in group (G - j) mod 4 at position p with j and p compile-time
// constants; the 4- and 2-row rings' slots are constants.
template <int W>
struct RowsRT {
  float* A;  // row slot 0 of a 16-row ring, at the thread's column
  float* X;
  int s;
  template <int L>
  __device__ __forceinline__ float* a() const { return A + ((s - L) & 15) * W; }
  template <int L>
  __device__ __forceinline__ float* x() const { return X + ((s - L) & 15) * W; }
  template <int L>
  __device__ __forceinline__ int m4() const { return (s - L) & 3; }
  template <int L>
  __device__ __forceinline__ int m2() const { return (s - L) & 1; }
};

template <int W>
struct RingGroups {
  float* A[4];  // A[j]: first slot of ring group (G - j) mod 4, G = s >> 2
  float* X[4];
  __device__ __forceinline__ RingGroups(float* a, float* x, int s) {
    const int G = s >> 2;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      A[j] = a + 4 * ((G - j) & 3) * W;
      X[j] = x + 4 * ((G - j) & 3) * W;
    }
  }
};

template <int W, int PH>
struct RowsCT {
  const RingGroups<W>& g;
  template <int L>
  static constexpr int J = PH >= L ? 0 : (L - PH + 3) / 4;  // groups back
  template <int L>
  static constexpr int P = PH - L + 4 * J<L>;  // position inside the group
  template <int L>
  __device__ __forceinline__ float* a() const { return g.A[J<L> & 3] + P<L> * W; }
  template <int L>
  __device__ __forceinline__ float* x() const { return g.X[J<L> & 3] + P<L> * W; }
  template <int L>
  __device__ static constexpr int m4() { return (PH - L) & 3; }
  template <int L>
  __device__ static constexpr int m2() { return (PH - L) & 1; }
};

// Runs a band's steps s_begin .. s_end: four-step groups of FULL steps
// (every stage live, compile-time slots, no guards) where s is a multiple of
// 4 and the group lies inside [s_lo, s_hi], generic steps (run-time slots,
// stage guards) elsewhere.  One instance of each step form.
template <class SW>
__device__ __forceinline__ void sweep_band(SW& sw, float* ringA, float* ringX, int s_begin,
                                           int s_end, int s_lo, int s_hi) {
  constexpr int W = SW::W;
  int s = s_begin;
#pragma unroll 1
  while (s <= s_end) {
    if ((s & 3) == 0 && s >= s_lo && s + 3 <= s_hi) {
      const RingGroups<W> g(ringA, ringX, s);
      sw.template step<true>(s, RowsCT<W, 0>{g});
      sw.template step<true>(s + 1, RowsCT<W, 1>{g});
      sw.template step<true>(s + 2, RowsCT<W, 2>{g});
      sw.template step<true>(s + 3, RowsCT<W, 3>{g});
      s += 4;
    } else {
      sw.template step<false>(s, RowsRT<W>{ringA, ringX, s});
      ++s;
    }
  }
}

// ---- k_bwd_plus ----------------------------------------------------------------
// Output-gradient column of a thread (fine column Q, element pointer at row
// 0), read row by row.
struct GCol {
  const float* p;
  int64_t sh;
  int orows;
  bool ok;
  // FULL steps read rows known to lie inside the output
  template <bool FULL>
  __device__ __forceinline__ float at(int P) const {
    if (FULL) return ok ? __ldg(p + (int64_t)P * sh) : 0.f;
    return (ok && P >= 0 && P < orows) ? __ldg(p + (int64_t)P * sh) : 0.f;
  }
};

__device__ __forceinline__ GCol gcol(const BwdArgs& a, int64_t plane, int64_t Q) {
  GCol g;
  g.ok = Q >= 0 && Q < a.ocols;
  g.p = a.gout + plane * a.g_sc + (g.ok ? Q : 0) * a.g_sw;
  g.sh = a.g_sh;
  g.orows = (int)a.orows;
  return g;
}

__device__ __forceinline__ bool any_nonzero(const float4& v, const float s[4]) {
  return (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) ||
         (s[0] != 0.f || s[1] != 0.f || s[2] != 0.f || s[3] != 0.f);
}

// Lags (row = s - L at step s): input row 0, x indicators 3, x values 5,
// "+" indicators 7, "+" adjoints 9, "+" coefficients 11; the partial A_bar of
// row s - 12 and X_bar of row s - 13 are complete at the end of step s.
// Guarded steps skip the work of points whose incoming adjoints are all zero
// (a sparse output gradient); FULL steps do it, with the same result.
template <int BMODE, int NT1>
struct PlusSweep {
  static constexpr int W = RingsPlus<NT1>::W;
  RingsPlus<NT1>& R;
  const MethodConsts k;
  float w, k2;
  int u, c, n, a0, a1;
  const float* xin;
  int64_t x_sh;
  WsPlane ws;
  bool col_out;
  GCol godd, gevn;  // fine column 2c + 1 (E and x points) and 2c (S points, samples)
  // carried from step to step
  float pf, pf2;              // input rows s+1, s+2 of the column
  // output gradients of the rows the next 5 steps use: [0] the next step's
  float ue[5], us[5], gx[5], ga[5];
  float4 pe1, pe2, ps1, ps2;  // p_bar of the "+" points of rows s-10 (1), s-11 (2)
  float xacc[4], aacc[4];     // own-column accumulators: X_bar rows r-2 .. r+1,
                              // A_bar rows r-1 .. r+2 (r = the coefficient row)

  __device__ __forceinline__ PlusSweep(RingsPlus<NT1>& R_, const BwdArgs& a,
                                       const MethodConsts& k_, int rows)
      : R(R_), k(k_) {
    const int t = threadIdx.x;
    const int64_t plane = blockIdx.z;
    constexpr int TW1 = NT1 - HL1 - HR1;
    n = (int)a.n;
    const int m = (int)a.m;
    const int b0 = -BWD_GHOST + (int)blockIdx.x * TW1;
    const int b1 = min(b0 + TW1, m + BWD_GHOST);
    c = b0 - HL1 + t;
    a0 = -BWD_GHOST + (int)blockIdx.y * rows;
    a1 = min(a0 + rows, n + BWD_GHOST);
    xin = a.x + plane * a.x_sc + (int64_t)clampi(c, 0, m - 1) * a.x_sw;
    x_sh = a.x_sh;
    ws = ws_plane(a, plane);
    col_out = c >= b0 && c < b1;
    godd = gcol(a, plane, 2 * (int64_t)c + 1);
    gevn = gcol(a, plane, 2 * (int64_t)c);
    w = k.w;
    k2 = k.kappa2 * k.kappa2;
    u = t + PAD;
  }

  template <bool FULL, class SL>
  __device__ __forceinline__ void step(const int s, const SL& sl) {
    const float cur = pf;
    pf = pf2;
    pf2 = __ldg(xin + (int64_t)clampi(s + 2, 0, n - 1) * x_sh);
    const float ue_s = ue[0], us_s = us[0], gx_s = gx[0], ga_s = ga[0];
#pragma unroll
    for (int j = 0; j + 1 < 5; ++j) {
      ue[j] = ue[j + 1]; us[j] = us[j + 1]; gx[j] = gx[j + 1]; ga[j] = ga[j + 1];
    }
    ue[5 - 1] = godd.template at<FULL>(2 * (s - 9 + 5));
    us[5 - 1] = gevn.template at<FULL>(2 * (s - 9 + 5) + 1);
    gx[5 - 1] = godd.template at<FULL>(2 * (s - 13 + 5) + 1);
    ga[5 - 1] = gevn.template at<FULL>(2 * (s - 12 + 5));
    __syncthreads();
    *sl.template a<0>() = cur;

    // Each stage runs only on the rows the band's outputs need (the guards
    // are uniform across the CTA): the pipeline's fill and drain steps do
    // just the stages that have work.
    // ---- x indicators, row s-3 ----
    if (FULL || (s - 3 >= a0 - 5 && s - 3 <= a1 + 4)) {
      const Sten q = sten_x(sl.template a<4>(), sl.template a<3>(), sl.template a<2>(),
                            sl.template a<1>());
      R.SIX[sl.template m4<3>()][u] = indicators(q, k.kappa1, k.eps1);
    }
    // ---- x values, row s-5 ----
    if (FULL || (s - 5 >= a0 - 4 && s - 5 <= a1 + 3)) {
      float D[4], om[4];
      smooth(R.SIX[sl.template m4<5>()][u], R.SIX[sl.template m4<6>()][u],
             R.SIX[sl.template m4<4>()][u], R.SIX[sl.template m4<5>()][u - 1],
             R.SIX[sl.template m4<5>()][u + 1], w, D);
      float rD[4], ip[4];
      weights<BMODE>(D, k.beta, om, rD);
      const Sten q = sten_x(sl.template a<6>(), sl.template a<5>(), sl.template a<4>(),
                            sl.template a<3>());
      interp4(q, ip);
      float x = 0.f;
#pragma unroll
      for (int d = 0; d < 4; ++d) x = fmaf(om[d], ip[d], x);
      *sl.template x<5>() = x;
    }
    // ---- "+" indicators, row r = s-7 ----
    if (FULL || (s - 7 >= a0 - 3 && s - 7 <= a1 + 2)) {
      const Sten qe = sten_e(sl.template a<7>(), *sl.template x<9>(), *sl.template x<8>(),
                             *sl.template x<7>(), *sl.template x<6>());
      R.SIE[sl.template m4<7>()][u] = indicators(qe, k.kappa2, k.eps2);
      const Sten qs = sten_s(sl.template x<7>(), *sl.template a<8>(), *sl.template a<7>(),
                             *sl.template a<6>(), *sl.template a<5>());
      R.SIS[sl.template m4<7>()][u] = indicators(qs, k.kappa2, k.eps2);
    }
    // ---- "+" adjoints, row r = s-9 ----
    float4 pe0 = make_float4(0.f, 0.f, 0.f, 0.f), ps0 = pe0;
    if (FULL || (s - 9 >= a0 - 2 && s - 9 <= a1 + 1)) {
      float4 de = pe0, ds = pe0;
      if (FULL || ue_s != 0.f) {
        // E(r,c): D reads S at (r-1,c), (r,c), (r-1,c+1), (r,c+1)
        float D[4];
        smooth(R.SIE[sl.template m4<9>()][u], R.SIS[sl.template m4<10>()][u],
               R.SIS[sl.template m4<9>()][u], R.SIS[sl.template m4<10>()][u + 1],
               R.SIS[sl.template m4<9>()][u + 1], w, D);
        const Sten q = sten_e(sl.template a<9>(), *sl.template x<11>(), *sl.template x<10>(),
                              *sl.template x<9>(), *sl.template x<8>());
        point_adjoint<BMODE>(q, D, k.beta, ue_s, pe0, de);
      }
      if (FULL || us_s != 0.f) {
        // S(r,c): D reads E at (r,c-1), (r,c), (r+1,c-1), (r+1,c)
        float D[4];
        smooth(R.SIS[sl.template m4<9>()][u], R.SIE[sl.template m4<9>()][u - 1],
               R.SIE[sl.template m4<9>()][u], R.SIE[sl.template m4<8>()][u - 1],
               R.SIE[sl.template m4<8>()][u], w, D);
        const Sten q = sten_s(sl.template x<9>(), *sl.template a<10>(), *sl.template a<9>(),
                              *sl.template a<8>(), *sl.template a<7>());
        point_adjoint<BMODE>(q, D, k.beta, us_s, ps0, ds);
      }
      R.DE[sl.template m4<9>()][u] = de;
      R.DS[sl.template m4<9>()][u] = ds;
    }
    // ---- "+" coefficients, row r = s-11 ----
    if (FULL || (s - 11 >= a0 - 2 && s - 11 <= a1 + 1)) {
      // E(r,c) is read by S(r,c), S(r,c+1), S(r-1,c), S(r-1,c+1)
      float sb[4];  // 2 SI_bar
      float eh[4] = {0.f, 0.f, 0.f, 0.f};
      smooth(R.DE[sl.template m4<11>()][u], R.DS[sl.template m4<11>()][u],
             R.DS[sl.template m4<11>()][u + 1], R.DS[sl.template m4<12>()][u],
             R.DS[sl.template m4<12>()][u + 1], w, sb);
      if (FULL || any_nonzero(pe2, sb)) {
        const Sten q = sten_e(sl.template a<11>(), *sl.template x<13>(), *sl.template x<12>(),
                              *sl.template x<11>(), *sl.template x<10>());
        float cf[4][3];
        node_coefs(q, pe2, sb, k2, cf);
        // along row r (samples): targets columns c-1, c, c+1, c+2
        eh[0] = cf[1][2];
        eh[1] = cf[0][0] + cf[1][1];
        eh[2] = cf[0][1] + cf[1][0];
        eh[3] = cf[0][2];
        // along column c (x values): rows r-2 .. r+1
        xacc[0] += cf[3][2];
        xacc[1] += cf[2][0] + cf[3][1];
        xacc[2] += cf[2][1] + cf[3][0];
        xacc[3] += cf[2][2];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) R.EH[j][sl.template m2<11>()][u] = eh[j];
      // S(r,c) is read by E(r,c), E(r+1,c), E(r,c-1), E(r+1,c-1)
      float sh[4] = {0.f, 0.f, 0.f, 0.f};
      smooth(R.DS[sl.template m4<11>()][u], R.DE[sl.template m4<11>()][u],
             R.DE[sl.template m4<10>()][u], R.DE[sl.template m4<11>()][u - 1],
             R.DE[sl.template m4<10>()][u - 1], w, sb);
      if (FULL || any_nonzero(ps2, sb)) {
        const Sten q = sten_s(sl.template x<11>(), *sl.template a<12>(), *sl.template a<11>(),
                              *sl.template a<10>(), *sl.template a<9>());
        float cf[4][3];
        node_coefs(q, ps2, sb, k2, cf);
        // along row r (x values): targets columns c-2, c-1, c, c+1
        sh[0] = cf[1][2];
        sh[1] = cf[0][0] + cf[1][1];
        sh[2] = cf[0][1] + cf[1][0];
        sh[3] = cf[0][2];
        // along column c (samples): rows r-1 .. r+2
        aacc[0] += cf[3][2];
        aacc[1] += cf[2][0] + cf[3][1];
        aacc[2] += cf[2][1] + cf[3][0];
        aacc[3] += cf[2][2];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) R.SH[j][sl.template m4<11>()][u] = sh[j];
    }

    // ---- X_bar of row q = s-13 and the partial A_bar of row p = s-12 are complete ----
    {
      const int q = s - 13, p = s - 12;
      const int sq = sl.template m4<13>(), sp = sl.template m2<12>();
      const float xb = xacc[0] + (R.SH[0][sq][u + 2] + R.SH[1][sq][u + 1]) +
                       (R.SH[2][sq][u] + R.SH[3][sq][u - 1]) + gx_s;
      const float ab = aacc[0] + (R.EH[0][sp][u + 1] + R.EH[1][sp][u]) +
                       (R.EH[2][sp][u - 1] + R.EH[3][sp][u - 2]) + ga_s;
      if (col_out && (FULL || (q >= a0 && q < a1))) ws.xb[ws.idx(q, c)] = xb;
      if (col_out && (FULL || (p >= a0 && p < a1))) ws.ab[ws.idx(p, c)] = ab;
      xacc[0] = xacc[1]; xacc[1] = xacc[2]; xacc[2] = xacc[3]; xacc[3] = 0.f;
      aacc[0] = aacc[1]; aacc[1] = aacc[2]; aacc[2] = aacc[3]; aacc[3] = 0.f;
    }
    pe2 = pe1; pe1 = pe0;
    ps2 = ps1; ps1 = ps0;
  }
};

template <int BMODE, int NT1>
__global__ void __launch_bounds__(NT1, NT1 == NT_NARROW ? 3 : 2)
    k_bwd_plus(BwdArgs a, MethodConsts k, int rows) {
  extern __shared__ __align__(16) unsigned char smem[];
  RingsPlus<NT1>& R = *reinterpret_cast<RingsPlus<NT1>*>(smem);
  {
    float* z = reinterpret_cast<float*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(RingsPlus<NT1>) / sizeof(float)); i += NT1)
      z[i] = 0.f;
  }
  PlusSweep<BMODE, NT1> sw(R, a, k, rows);
  const int s_begin = sw.a0 - 6, s_end = sw.a1 - 1 + 13;
  const int n = sw.n;
  sw.pf = __ldg(sw.xin + (int64_t)clampi(s_begin, 0, n - 1) * sw.x_sh);
  sw.pf2 = __ldg(sw.xin + (int64_t)clampi(s_begin + 1, 0, n - 1) * sw.x_sh);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    sw.ue[j] = sw.godd.template at<false>(2 * (s_begin - 9 + j));
    sw.us[j] = sw.gevn.template at<false>(2 * (s_begin - 9 + j) + 1);
    sw.gx[j] = sw.godd.template at<false>(2 * (s_begin - 13 + j) + 1);
    sw.ga[j] = sw.gevn.template at<false>(2 * (s_begin - 12 + j));
  }
  sw.pe1 = sw.pe2 = sw.ps1 = sw.ps2 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < 4; ++j) sw.xacc[j] = sw.aacc[j] = 0.f;
  // FULL steps: every stage live and every output row written (s in
  // [a0 + 13, a1 + 7]), and the output-gradient rows a step loads inside
  // the output (2 (s - 13 + 5) + 1 >= 0, 2 (s - 9 + 5) + 1 < orows)
  const int s_lo = max(sw.a0 + 13, 8);
  const int s_hi = min(sw.a1 + 7, sw.gevn.orows >= 2 ? (sw.gevn.orows - 2) / 2 + 4 : 3);
  sweep_band(sw, &R.A[0][sw.u], &R.X[0][sw.u], s_begin, s_end, s_lo, s_hi);
}

// ---- k_bwd_cross ---------------------------------------------------------------
// Lags: input row 0, x indicators 3, x adjoints 5, x coefficients 7; A_bar
// of row s - 9 is complete at step s and written (column-folded) at s + 1.
template <int BMODE, int NT2>
struct CrossSweep {
  static constexpr int W = RingsCross<NT2>::W;
  RingsCross<NT2>& R;
  const MethodConsts k;
  float w, k1;
  int u, c, n, a0, a1;
  const float* xin;
  int64_t x_sh;
  WsPlane ws;
  bool cg;  // column on the workspace grid
  // the thread writes grad_in column c; columns 0 and m-1 also sum the ghost
  // columns folded onto them
  bool emit_col, fold_left, fold_right;
  float* gin;  // grad_in column c, row 0
  int64_t gi_sh;
  // carried from step to step
  float pf, pf2, pf3, pf4;  // input rows s .. s+3 of the column
  float xbn, abn;   // workspace values of the next step's rows
  float xbn2, abn2; // and of the step after
  float xbn3, abn3; // and of the one after that
  float acc[4];     // A_bar rows s-9 .. s-6 of this column
  float rowsum;     // ghost rows folded onto an edge row
  int emitted;      // grad_in row published in the previous step (-1: none)

  __device__ __forceinline__ CrossSweep(RingsCross<NT2>& R_, const BwdArgs& a,
                                        const MethodConsts& k_, int rows)
      : R(R_), k(k_) {
    constexpr int TW2 = NT2 - HL2 - HR2;
    const int t = threadIdx.x;
    const int64_t plane = blockIdx.z;
    n = (int)a.n;
    const int m = (int)a.m;
    const int nby = (int)gridDim.y;
    const int b0 = (int)blockIdx.x * TW2;
    const int b1 = min(b0 + TW2, m);
    c = b0 - HL2 + t;
    // A_bar rows of this band: image rows [r0, r1) plus the ghost rows that
    // fold onto row 0 (first band) and row n-1 (last band)
    const int r0 = (int)blockIdx.y * rows, r1 = min(r0 + rows, n);
    a0 = blockIdx.y == 0 ? -GA : r0;
    a1 = (int)blockIdx.y == nby - 1 ? n + GA : r1;
    xin = a.x + plane * a.x_sc + (int64_t)clampi(c, 0, m - 1) * a.x_sw;
    x_sh = a.x_sh;
    ws = ws_plane(a, plane);
    cg = c >= -BWD_GHOST && c < m + BWD_GHOST;
    emit_col = c >= b0 && c < b1;
    fold_left = c == 0;
    fold_right = c == m - 1;
    gin = a.gin + plane * a.gi_sc + (int64_t)(emit_col ? c : 0) * a.gi_sw;
    gi_sh = a.gi_sh;
    w = k.w;
    k1 = k.kappa1 * k.kappa1;
    u = t + PAD;
  }

  // FULL steps read workspace rows known to lie on the workspace grid
  template <bool FULL>
  __device__ __forceinline__ float ws_at(const float* base, int r) const {
    if (FULL) return cg ? base[ws.idx(r, c)] : 0.f;
    return (cg && r >= -BWD_GHOST && r < n + BWD_GHOST) ? base[ws.idx(r, c)] : 0.f;
  }

  template <bool FULL, class SL>
  __device__ __forceinline__ void step(const int s, const SL& sl) {
    const float cur = pf;
    pf = pf2;
    pf2 = pf3;
    pf3 = pf4;
    pf4 = __ldg(xin + (int64_t)clampi(s + 4, 0, n - 1) * x_sh);
    const float xb_s = xbn, ab_s = abn;
    xbn = xbn2;
    abn = abn2;
    xbn2 = xbn3;
    abn2 = abn3;
    xbn3 = ws_at<FULL>(ws.xb, s - 2);
    abn3 = ws_at<FULL>(ws.ab, s - 6);
    __syncthreads();
    *sl.template a<0>() = cur;

    // ---- grad_in row published in the previous step: fold the ghost columns ----
    if ((FULL || emitted >= 0) && emit_col) {
      const float* af = R.AF[sl.template m2<1>()] + u;
      float v = af[0];
      if (fold_left) v += (af[-5] + af[-4]) + (af[-3] + af[-2]) + af[-1];
      if (fold_right) v += (af[1] + af[2]) + (af[3] + af[4]) + af[5];
      gin[(int64_t)(FULL ? s - 10 : emitted) * gi_sh] = v;
    }

    // Stages run only on the rows the band's outputs need (uniform guards).
    // ---- x indicators, row s-3 ----
    if (FULL || (s - 3 >= a0 - 4 && s - 3 <= a1 + 2)) {
      const Sten q = sten_x(sl.template a<4>(), sl.template a<3>(), sl.template a<2>(),
                            sl.template a<1>());
      R.SIX[sl.template m4<3>()][u] = indicators(q, k.kappa1, k.eps1);
    }
    // ---- x adjoints, row s-5 ----
    if (FULL || (s - 5 >= a0 - 3 && s - 5 <= a1 + 1)) {
      float4 px = make_float4(0.f, 0.f, 0.f, 0.f), dx = px;
      if (FULL || xb_s != 0.f) {
        float D[4];
        smooth(R.SIX[sl.template m4<5>()][u], R.SIX[sl.template m4<6>()][u],
               R.SIX[sl.template m4<4>()][u], R.SIX[sl.template m4<5>()][u - 1],
               R.SIX[sl.template m4<5>()][u + 1], w, D);
        const Sten q = sten_x(sl.template a<6>(), sl.template a<5>(), sl.template a<4>(),
                              sl.template a<3>());
        point_adjoint<BMODE>(q, D, k.beta, xb_s, px, dx);
      }
      R.PX[sl.template m4<5>()][u] = px;
      R.DX[sl.template m4<5>()][u] = dx;
    }
    // ---- x coefficients, row s-7 ----
    if (FULL || (s - 7 >= a0 - 2 && s - 7 <= a1)) {
      float sb[4];  // 2 SI_bar
      smooth(R.DX[sl.template m4<7>()][u], R.DX[sl.template m4<8>()][u],
             R.DX[sl.template m4<6>()][u], R.DX[sl.template m4<7>()][u - 1],
             R.DX[sl.template m4<7>()][u + 1], w, sb);
      const float4 pb = R.PX[sl.template m4<7>()][u];
      float2 c1 = make_float2(0.f, 0.f), c2 = c1, cm = c1;
      if (FULL || any_nonzero(pb, sb)) {
        const Sten q = sten_x(sl.template a<8>(), sl.template a<7>(), sl.template a<6>(),
                              sl.template a<5>());
        float cf[4][3];
        node_coefs(q, pb, sb, k1, cf);
        // targets (row offset, column offset): (0,0) d0.N0 + d1.N1,
        // (1,1) d0.N1 + d1.N0, (2,2) d0.N2, (-1,-1) d1.N2, (0,1) d2.N0 + d3.N1,
        // (1,0) d2.N1 + d3.N0, (2,-1) d2.N2, (-1,2) d3.N2
        acc[2] += cf[0][0] + cf[1][1];  // row s-7
        acc[3] += cf[2][1] + cf[3][0];  // row s-6
        c1 = make_float2(cf[2][0] + cf[3][1], cf[0][1] + cf[1][0]);
        c2 = make_float2(cf[0][2], cf[3][2]);
        cm = make_float2(cf[1][2], cf[2][2]);
      }
      R.C1[sl.template m2<7>()][u] = c1;
      R.C2[sl.template m2<7>()][u] = c2;
      R.CM[sl.template m2<7>()][u] = cm;
    }
    // ---- contributions of x row s-8 from the neighbouring columns ----
    if (FULL || (s - 8 >= a0 - 2 && s - 8 <= a1)) {
      const int sp = sl.template m2<8>();
      const float2 c1 = R.C1[sp][u - 1];  // from column c-1: rows s-8, s-7
      const float2 c2 = R.C2[sp][u - 2];  // from column c-2: rows s-6, s-9
      const float2 cm = R.CM[sp][u + 1];  // from column c+1: rows s-9, s-6
      acc[0] += c2.y + cm.x;
      acc[1] += c1.x;
      acc[2] += c1.y;
      acc[3] += c2.x + cm.y;
    }
    // ---- A_bar of row q = s-9 is complete ----
    {
      const int q = s - 9;
      const float ab = acc[0] + ab_s;
      acc[0] = acc[1]; acc[1] = acc[2]; acc[2] = acc[3]; acc[3] = 0.f;
      if (FULL) {
        // an interior row: no ghost rows to fold (rowsum is 0 here)
        R.AF[sl.template m2<0>()][u] = ab;
        emitted = q;
      } else {
        emitted = -1;
        if (q >= a0 && q < a1) {
          rowsum += ab;
          // rows -GA..0 fold onto row 0, rows n-1..n+GA-1 onto row n-1
          if (q >= 0 && (q < n - 1 || q == n - 1 + GA)) {
            emitted = min(q, n - 1);
            R.AF[sl.template m2<0>()][u] = rowsum;
            rowsum = 0.f;
          }
        }
      }
    }
  }
};

template <int BMODE, int NT2>
__global__ void __launch_bounds__(NT2, 3) k_bwd_cross(BwdArgs a, MethodConsts k, int rows) {
  extern __shared__ __align__(16) unsigned char smem[];
  RingsCross<NT2>& R = *reinterpret_cast<RingsCross<NT2>*>(smem);
  {
    float* z = reinterpret_cast<float*>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(RingsCross<NT2>) / sizeof(float)); i += NT2)
      z[i] = 0.f;
  }
  CrossSweep<BMODE, NT2> sw(R, a, k, rows);
  const int s_begin = sw.a0 - 5, s_end = sw.a1 - 1 + 10;
  const int n = sw.n;
  sw.pf = __ldg(sw.xin + (int64_t)clampi(s_begin, 0, n - 1) * sw.x_sh);
  sw.pf2 = __ldg(sw.xin + (int64_t)clampi(s_begin + 1, 0, n - 1) * sw.x_sh);
  sw.pf3 = __ldg(sw.xin + (int64_t)clampi(s_begin + 2, 0, n - 1) * sw.x_sh);
  sw.pf4 = __ldg(sw.xin + (int64_t)clampi(s_begin + 3, 0, n - 1) * sw.x_sh);
  sw.xbn = sw.template ws_at<false>(sw.ws.xb, s_begin - 5);
  sw.abn = sw.template ws_at<false>(sw.ws.ab, s_begin - 9);
  sw.xbn2 = sw.template ws_at<false>(sw.ws.xb, s_begin - 4);
  sw.abn2 = sw.template ws_at<false>(sw.ws.ab, s_begin - 8);
  sw.xbn3 = sw.template ws_at<false>(sw.ws.xb, s_begin - 3);
  sw.abn3 = sw.template ws_at<false>(sw.ws.ab, s_begin - 7);
#pragma unroll
  for (int j = 0; j < 4; ++j) sw.acc[j] = 0.f;
  sw.rowsum = 0.f;
  sw.emitted = -1;
  // FULL steps: every stage live (s in [a0 + 9, a1 + 5]), the previous and
  // the current A_bar rows interior ones (s - 10 >= max(a0, 0),
  // s - 9 < min(a1, n - 1)) and the workspace rows a step loads on the
  // workspace grid (s - 2 < n + 2)
  const int s_lo = max(sw.a0, 0) + 10;
  const int s_hi = min(sw.a1 + 5, sw.n + 3);
  sweep_band(sw, &R.A[0][sw.u], &R.A[0][sw.u], s_begin, s_end, s_lo, s_hi);
}

// Rows per band: the band count that minimises waves x (rows + fill steps).
int band_rows(int64_t rows_total, int64_t ctas_per_band_row, int fill, int resident) {
  int best = (int)rows_total;
  double best_cost = 1e300;
  for (int bands = 1; bands <= 64; ++bands) {
    const int64_t h = (rows_total + bands - 1) / bands;
    if (h < 16 && bands > 1) break;
    const int64_t ctas = ctas_per_band_row * bands;
    const int64_t waves = (ctas + resident - 1) / resident;
    const double cost = double(waves) * double(h + fill);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = (int)h;
    }
  }
  return best;
}

// One sweep kernel with the CTA width, of NT_NARROW and NT_WIDE, that
// spends the least: for each width, the band height band_rows chooses, then
// the per-SM work ceil(CTAs / SMs) x threads x (rows per band + fill).
struct SweepShape {
  const void* fn;
  size_t smem;
  int threads, occ, strips, rows;
  int64_t bands;
};

template <class KN, class KW>
cudaError_t pick_shape(KN kn, KW kw, size_t smem_n, size_t smem_w, int tw_n, int tw_w,
                       int64_t rows_total, int64_t cols_total, int64_t planes, int fill,
                       SweepShape* best) {
  int dev = 0, sms = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  const void* fns[2] = {(const void*)kn, (const void*)kw};
  const size_t smems[2] = {smem_n, smem_w};
  const int nts[2] = {NT_NARROW, NT_WIDE}, tws[2] = {tw_n, tw_w};
  double best_cost = -1.0;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smems[i])) != cudaSuccess)
      return e;
    int occ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[i], nts[i], smems[i])) !=
        cudaSuccess)
      return e;
    if (occ < 1) continue;
    const int64_t strips = (cols_total + tws[i] - 1) / tws[i];
    const int h = band_rows(rows_total, strips * planes, fill, occ * sms);
    const int64_t bands = (rows_total + h - 1) / h;
    const int64_t per_sm = (strips * bands * planes + sms - 1) / sms;
    const double cost = double(per_sm) * nts[i] * double(h + fill);
    if (best_cost < 0.0 || cost < best_cost) {
      best_cost = cost;
      *best = SweepShape{fns[i], smems[i], nts[i], occ, (int)strips, h, bands};
    }
  }
  return best_cost < 0.0 ? cudaErrorInvalidConfiguration : cudaSuccess;
}

template <int BMODE>
cudaError_t launch_all(const BwdArgs& a, const MethodConsts& k, cudaStream_t st) {
  // k_bwd_plus: the extended grid, rows and columns [-2, n+2) x [-2, m+2)
  SweepShape s1, s2;
  cudaError_t e = pick_shape(k_bwd_plus<BMODE, NT_NARROW>, k_bwd_plus<BMODE, NT_WIDE>,
                             sizeof(RingsPlus<NT_NARROW>), sizeof(RingsPlus<NT_WIDE>),
                             NT_NARROW - HL1 - HR1, NT_WIDE - HL1 - HR1,
                             a.n + 2 * BWD_GHOST, a.m + 2 * BWD_GHOST, a.planes, 10, &s1);
  if (e != cudaSuccess) return e;
  const dim3 g1((unsigned)s1.strips, (unsigned)s1.bands, (unsigned)a.planes);
  if (s1.threads == NT_WIDE)
    k_bwd_plus<BMODE, NT_WIDE><<<g1, NT_WIDE, s1.smem, st>>>(a, k, s1.rows);
  else
    k_bwd_plus<BMODE, NT_NARROW><<<g1, NT_NARROW, s1.smem, st>>>(a, k, s1.rows);
  // k_bwd_cross: image rows and columns, ghosts folded at the edges
  e = pick_shape(k_bwd_cross<BMODE, NT_NARROW>, k_bwd_cross<BMODE, NT_WIDE>,
                 sizeof(RingsCross<NT_NARROW>), sizeof(RingsCross<NT_WIDE>),
                 NT_NARROW - HL2 - HR2, NT_WIDE - HL2 - HR2, a.n, a.m, a.planes, 8, &s2);
  if (e != cudaSuccess) return e;
  const dim3 g2((unsigned)s2.strips, (unsigned)s2.bands, (unsigned)a.planes);
  if (s2.threads == NT_WIDE)
    k_bwd_cross<BMODE, NT_WIDE><<<g2, NT_WIDE, s2.smem, st>>>(a, k, s2.rows);
  else
    k_bwd_cross<BMODE, NT_NARROW><<<g2, NT_NARROW, s2.smem, st>>>(a, k, s2.rows);
  return cudaGetLastError();
}

}  // namespace

size_t bwd_workspace_bytes(int64_t n, int64_t m, int64_t planes) {
  // X_bar and the partial A_bar on the grid extended by BWD_GHOST cells
  return sizeof(float) * 2 * (size_t)(n + 2 * BWD_GHOST) * (size_t)(m + 2 * BWD_GHOST) *
         (size_t)planes;
}

cudaError_t launch_zoom2x_bwd(const BwdArgs& a, const MethodConsts& k, int bmode,
                              cudaStream_t stream) {
  switch (bmode) {
    case B2: return launch_all<B2>(a, k, stream);
    case B0: return launch_all<B0>(a, k, stream);
    default: return launch_all<BGEN>(a, k, stream);
  }
}

}  // namespace wdweno
