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
// Every quantity is computed once per cell of a grid extended by BWD_GHOST
// cells per side (clamp-to-edge) and kept in the workspace; scatters are
// written as gathers over these arrays (no atomics):
//   k_xsi      phase-1 indicators (4 directions) of every x point, and the
//              clamp-extended copy of the input that the later kernels read
//              their stencil nodes from (no clamping or 64-bit indexing)
//   k_xval     phase-1 values X
//   k_psi      phase-2 indicators of every E and S point
//   k_padj     p_bar, D_bar of the "+" points that receive an output gradient
//   k_coef<T>  per stencil and node role, the coefficient above
//   k_gather2_xadj  X_bar (plus the x-point output gradient) and A_bar from
//              phase 2 (plus the sample-point output gradient), then the
//              x point's p_bar, D_bar from that X_bar
//   k_gather1  A_bar += phase-1 contributions
//   k_fold     grad_in = A_bar summed over each pixel's clamp preimage
#include "wd_bwd.h"

namespace wdweno {

namespace {

constexpr int G = BWD_GHOST;
// A 32 x 8 block covers 32 columns and R x 8 rows of cells: a thread takes R
// cells of its column, 8 rows apart.  Three light kernels take four cells and
// the x-stencil coefficients two, so a block's start-up is spread over more
// work; the others take one, which keeps their register count (and
// occupancy) down (chosen by measurement).
constexpr int BWD_BY = 8;
constexpr int R_XSI = 4, R_XVAL = 4, R_PSI = 1, R_PADJ = 1, R_COEF2 = 1, R_G2 = 1, R_COEF1 = 2,
              R_G1 = 1, R_FOLD = 4;

// Workspace layout per plane (NE x ME cells, the cell count padded to a
// multiple of 4): seven float4 planes for the four-direction vectors, then
// scalar planes.
enum VGroup {
  G_XSI = 0,  // phase-1 SIs
  G_ESI = 1,  // E-point SIs
  G_SSI = 2,  // S-point SIs
  G_EP = 3,   // E p_bar   (the phase-1 adjoint reuses G_EP, G_ED for x points)
  G_ED = 4,   // E D_bar
  G_SP = 5,   // S p_bar
  G_SD = 6,   // S D_bar
  G_N = 7
};
enum Slot {
  S_X = 0,     // phase-1 values
  S_AB = 1,    // A_bar on the extended grid
  S_ECO = 2,   // 12: E coefficients, index k*3 + t   (phase 1 reuses for x)
  S_SCO = 14,  // 12: S coefficients
  S_A = 26,    // the input, clamp-extended to the work grid
  S_N = 27
};
static_assert(4 * G_N + S_N == BWD_ARRAYS, "workspace slot count");

// Point types: 0 = x point X(a,b) (fine (2a+1, 2b+1)), 1 = E point
// (fine (2a, 2b+1)), 2 = S point (fine (2a+1, 2b)).  For each type and
// direction k the nodes N0, N1, N2 sit at (a, b) + off on the lattice of input
// samples (lattice 0) or of x points (lattice 1).
// x: k = 0 (1,1), 1 (-1,-1), 2 (1,-1), 3 (-1,1)
// E, S: k = 0 (0,1), 1 (0,-1), 2 (1,0), 3 (-1,0)
// Compile-time tables: every call site passes literal or unrolled indices,
// so the lookups fold into immediates.
__device__ __forceinline__ int off_of(int type, int k, int t, int d) {
  constexpr int tab[3][4][3][2] = {
      {{{0, 0}, {1, 1}, {2, 2}}, {{1, 1}, {0, 0}, {-1, -1}},
       {{0, 1}, {1, 0}, {2, -1}}, {{1, 0}, {0, 1}, {-1, 2}}},
      {{{0, 0}, {0, 1}, {0, 2}}, {{0, 1}, {0, 0}, {0, -1}},
       {{-1, 0}, {0, 0}, {1, 0}}, {{0, 0}, {-1, 0}, {-2, 0}}},
      {{{0, -1}, {0, 0}, {0, 1}}, {{0, 0}, {0, -1}, {0, -2}},
       {{0, 0}, {1, 0}, {2, 0}}, {{1, 0}, {0, 0}, {-1, 0}}}};
  return tab[type][k][t][d];
}
__device__ __forceinline__ int lattice_of(int type, int k) {
  constexpr int tab[3][4] = {{0, 0, 0, 0}, {0, 0, 1, 1}, {1, 1, 0, 0}};
  return tab[type][k];
}

struct Ctx {
  const float* x;  // input plane
  int n, m;
  int64_t sh, sw;
  float* ws;       // workspace plane
  int NE, ME;
  int64_t plane_cells;  // NE * ME rounded up to a multiple of 4 (< 2^31, checked on the host)
  float w, kap1, kap2, eps1, eps2, beta;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ float Ahat(const Ctx& c, int i, int j) {
  return __ldg(c.x + (int64_t)clampi(i, 0, c.n - 1) * c.sh + (int64_t)clampi(j, 0, c.m - 1) * c.sw);
}

__device__ __forceinline__ bool in_ext(const Ctx& c, int I, int J) {
  return I >= -G && I < c.n + G && J >= -G && J < c.m + G;
}

// 32-bit: the cell count of a plane is below 2^31.
__device__ __forceinline__ int cell(const Ctx& c, int I, int J) {
  return (I + G) * c.ME + (J + G);
}

__device__ __forceinline__ float& W(const Ctx& c, int slot, int I, int J) {
  return c.ws[(4 * G_N + slot) * c.plane_cells + cell(c, I, J)];
}

// Workspace value, 0 outside the extended grid.
__device__ __forceinline__ float W0(const Ctx& c, int slot, int I, int J) {
  return in_ext(c, I, J) ? W(c, slot, I, J) : 0.f;
}

__device__ __forceinline__ float4& V(const Ctx& c, int g, int I, int J) {
  return reinterpret_cast<float4*>(c.ws)[g * c.plane_cells + cell(c, I, J)];
}

__device__ __forceinline__ float4 V0(const Ctx& c, int g, int I, int J) {
  return in_ext(c, I, J) ? V(c, g, I, J) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float comp(const float4& v, int d) {
  return d == 0 ? v.x : (d == 1 ? v.y : (d == 2 ? v.z : v.w));
}

__device__ __forceinline__ float4 f4(const float a[4]) {
  return make_float4(a[0], a[1], a[2], a[3]);
}

// Stencil node of a point: input samples from the clamp-extended copy (or,
// with COPY = false, clamped reads of the input itself), x points from the
// phase-1 values.  Every caller's nodes lie inside the work grid.
template <bool COPY = true>
__device__ __forceinline__ float node(const Ctx& c, int type, int k, int t, int a, int b) {
  const int i = a + off_of(type, k, t, 0), j = b + off_of(type, k, t, 1);
  if (lattice_of(type, k) == 1) return W(c, S_X, i, j);
  return COPY ? W(c, S_A, i, j) : Ahat(c, i, j);
}

struct Pt {
  float p[4];   // interpolants
  float si[4];  // indicators (eps' included)
  float M[2];   // N0 + N1 of the pairs (0,1) and (2,3)
  float s[4];   // second differences
};

template <bool COPY = true>
__device__ __forceinline__ Pt eval_pt(const Ctx& c, int type, int a, int b) {
  Pt q;
  const float kap = type == 0 ? c.kap1 : c.kap2;
  const float eps = type == 0 ? c.eps1 : c.eps2;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float n0 = node<COPY>(c, type, k, 0, a, b);
    const float n1 = node<COPY>(c, type, k, 1, a, b);
    const float n2 = node<COPY>(c, type, k, 2, a, b);
    const float g = n1 - n0;
    const float s = fmaf(-2.f, n1, n0 + n2);
    const float ks = kap * s;
    q.si[k] = fmaf(g, g, fmaf(ks, ks, eps));
    q.s[k] = s;
    q.p[k] = fmaf(-0.125f, s, 0.5f * (n0 + n1));
    if (k == 0) q.M[0] = n0 + n1;
    if (k == 2) q.M[1] = n0 + n1;
  }
  return q;
}

// Normalised weights omega_k from D_k (Eqs. alpha, IzrazOmega2d).
template <int BMODE>
__device__ __forceinline__ void weights(const float D[4], float beta, float om[4]) {
  float al[4];
  if (BMODE == B0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) al[k] = 1.f;
  } else {
    const float dmin = fminf(fminf(D[0], D[1]), fminf(D[2], D[3]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float r = dmin * rcp_approx(D[k]);
      al[k] = BMODE == B2 ? r * r : ex2_approx(beta * lg2_approx(r));
    }
  }
  // the largest alpha is 1, so the sum lies in [1, 4]
  const float inv = rcp_approx((al[0] + al[1]) + (al[2] + al[3]));
#pragma unroll
  for (int k = 0; k < 4; ++k) om[k] = al[k] * inv;
}

// p_bar, D_bar of one blend point given its D and interpolant data.
template <int BMODE>
__device__ __forceinline__ void point_adjoint(const Pt& q, const float D[4], float beta, float ub,
                                              float pb[4], float db[4]) {
  float om[4];
  weights<BMODE>(D, beta, om);
  // p_k - u = sum_l omega_l (p_k - p_l), each difference formed from the
  // stencil data to avoid cancelling two O(1) values.
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float dM = (kk >> 1) == (l >> 1) ? 0.f : q.M[kk >> 1] - q.M[l >> 1];
      acc = fmaf(om[l], fmaf(0.5f, dM, -0.125f * (q.s[kk] - q.s[l])), acc);
    }
    pb[kk] = ub * om[kk];
    db[kk] = BMODE == B0 ? 0.f : -ub * beta * om[kk] * acc * rcp_approx(D[kk]);
  }
}

// The thread's column J and first row I0; it takes rows I0 + r BWD_BY,
// r < R, that lie on the extended grid.
template <int R>
__device__ __forceinline__ bool setup(const BwdArgs& a, const MethodConsts& k, Ctx& c, int& I0,
                                      int& J) {
  const int64_t plane = blockIdx.z;
  c.n = (int)a.n; c.m = (int)a.m; c.sh = a.x_sh; c.sw = a.x_sw;
  c.x = a.x + plane * a.x_sc;
  c.NE = c.n + 2 * G; c.ME = c.m + 2 * G;
  c.plane_cells = ((int64_t)c.NE * c.ME + 3) & ~int64_t(3);
  c.ws = a.ws + plane * (int64_t)BWD_ARRAYS * c.plane_cells;
  c.w = k.w; c.kap1 = k.kappa1; c.kap2 = k.kappa2; c.eps1 = k.eps1; c.eps2 = k.eps2;
  c.beta = k.beta;
  J = (int)(blockIdx.x * blockDim.x + threadIdx.x) - G;
  I0 = (int)(blockIdx.y * (BWD_BY * R) + threadIdx.y) - G;
  return J < c.m + G;
}

__device__ __forceinline__ float gout_at(const BwdArgs& a, int64_t plane, int64_t P, int64_t Q) {
  if (P < 0 || Q < 0 || P >= a.orows || Q >= a.ocols) return 0.f;
  return __ldg(a.gout + plane * a.g_sc + P * a.g_sh + Q * a.g_sw);
}

// Region where x values, their indicators and the "+" indicators are
// needed: rows/columns -4 .. n+3 (x values feed "+" stencils up to 3 fine
// steps away from the output quads, whose D reads one more ring).
__device__ __forceinline__ bool in_core(const Ctx& c, int I, int J) {
  return I >= -5 && I < c.n + 5 && J >= -5 && J < c.m + 5;
}

// ---- forward recompute ------------------------------------------------------
__global__ void k_xsi(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_XSI>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_XSI; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    float si[4] = {0.f, 0.f, 0.f, 0.f};
    if (in_core(c, I, J)) {
      const Pt q = eval_pt<false>(c, 0, I, J);
  #pragma unroll
      for (int d = 0; d < 4; ++d) si[d] = q.si[d];
    }
    V(c, G_XSI, I, J) = f4(si);
    W(c, S_A, I, J) = Ahat(c, I, J);
  }
}

template <int BMODE>
__device__ __forceinline__ void d_x(const Ctx& c, int I, int J, const float si[4], float D[4]) {
  const float4 u = V0(c, G_XSI, I - 1, J), v = V0(c, G_XSI, I + 1, J);
  const float4 l = V0(c, G_XSI, I, J - 1), r = V0(c, G_XSI, I, J + 1);
#pragma unroll
  for (int d = 0; d < 4; ++d)
    D[d] = fmaf(c.w, comp(u, d) + comp(v, d) + comp(l, d) + comp(r, d), si[d]);
}

template <int BMODE>
__global__ void k_xval(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_XVAL>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_XVAL; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    float v = 0.f;
    if (I >= -4 && I < c.n + 4 && J >= -4 && J < c.m + 4) {
      const Pt q = eval_pt(c, 0, I, J);
      float D[4], om[4];
      d_x<BMODE>(c, I, J, q.si, D);
      weights<BMODE>(D, c.beta, om);
      v = om[0] * q.p[0] + om[1] * q.p[1] + om[2] * q.p[2] + om[3] * q.p[3];
    }
    W(c, S_X, I, J) = v;
  }
}

__global__ void k_psi(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_PSI>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_PSI; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    float e[4] = {0.f, 0.f, 0.f, 0.f}, s[4] = {0.f, 0.f, 0.f, 0.f};
    if (I >= -2 && I < c.n + 2 && J >= -2 && J < c.m + 2) {
      const Pt qe = eval_pt(c, 1, I, J);
      const Pt qs = eval_pt(c, 2, I, J);
  #pragma unroll
      for (int d = 0; d < 4; ++d) { e[d] = qe.si[d]; s[d] = qs.si[d]; }
    }
    V(c, G_ESI, I, J) = f4(e);
    V(c, G_SSI, I, J) = f4(s);
  }
}

// ---- phase-2 adjoint ------------------------------------------------------------
template <int BMODE>
__global__ void k_padj(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_PADJ>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_PADJ; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    float pE[4] = {0.f, 0.f, 0.f, 0.f}, dE[4] = {0.f, 0.f, 0.f, 0.f};
    float pS[4] = {0.f, 0.f, 0.f, 0.f}, dS[4] = {0.f, 0.f, 0.f, 0.f};
    if (I >= 0 && I < c.n && J >= 0 && J < c.m) {
      const int64_t plane = blockIdx.z;
      const float uE = gout_at(a, plane, 2 * (int64_t)I, 2 * (int64_t)J + 1);
      const float uS = gout_at(a, plane, 2 * (int64_t)I + 1, 2 * (int64_t)J);
      if (uE != 0.f) {
        // E(a,b): D reads S at (a-1,b), (a,b), (a-1,b+1), (a,b+1)
        const Pt q = eval_pt(c, 1, I, J);
        float D[4];
        const float4 n0 = V(c, G_SSI, I - 1, J), n1 = V(c, G_SSI, I, J);
        const float4 n2 = V(c, G_SSI, I - 1, J + 1), n3 = V(c, G_SSI, I, J + 1);
        const float4 own = V(c, G_ESI, I, J);
  #pragma unroll
        for (int d = 0; d < 4; ++d)
          D[d] = fmaf(c.w, comp(n0, d) + comp(n1, d) + comp(n2, d) + comp(n3, d), comp(own, d));
        point_adjoint<BMODE>(q, D, c.beta, uE, pE, dE);
      }
      if (uS != 0.f) {
        // S(a,b): D reads E at (a,b-1), (a,b), (a+1,b-1), (a+1,b)
        const Pt q = eval_pt(c, 2, I, J);
        float D[4];
        const float4 n0 = V(c, G_ESI, I, J - 1), n1 = V(c, G_ESI, I, J);
        const float4 n2 = V(c, G_ESI, I + 1, J - 1), n3 = V(c, G_ESI, I + 1, J);
        const float4 own = V(c, G_SSI, I, J);
  #pragma unroll
        for (int d = 0; d < 4; ++d)
          D[d] = fmaf(c.w, comp(n0, d) + comp(n1, d) + comp(n2, d) + comp(n3, d), comp(own, d));
        point_adjoint<BMODE>(q, D, c.beta, uS, pS, dS);
      }
    }
    V(c, G_EP, I, J) = f4(pE);
    V(c, G_ED, I, J) = f4(dE);
    V(c, G_SP, I, J) = f4(pS);
    V(c, G_SD, I, J) = f4(dS);
  }
}

// SI_bar of the four directions at a point: its own D_bar plus w times the
// D_bar of the points whose D reads it (gX, gE, gS: the D_bar groups).
__device__ __forceinline__ void si_bar4(const Ctx& c, int type, int a, int b, int gX, int gE,
                                        int gS, float sb[4]) {
  float4 own, n0, n1, n2, n3;
  if (type == 0) {
    own = V0(c, gX, a, b);
    n0 = V0(c, gX, a - 1, b); n1 = V0(c, gX, a + 1, b);
    n2 = V0(c, gX, a, b - 1); n3 = V0(c, gX, a, b + 1);
  } else if (type == 1) {  // E(a,b) is read by S(a,b), S(a,b+1), S(a-1,b), S(a-1,b+1)
    own = V0(c, gE, a, b);
    n0 = V0(c, gS, a, b); n1 = V0(c, gS, a, b + 1);
    n2 = V0(c, gS, a - 1, b); n3 = V0(c, gS, a - 1, b + 1);
  } else {  // S(a,b) is read by E(a,b), E(a+1,b), E(a,b-1), E(a+1,b-1)
    own = V0(c, gS, a, b);
    n0 = V0(c, gE, a, b); n1 = V0(c, gE, a + 1, b);
    n2 = V0(c, gE, a, b - 1); n3 = V0(c, gE, a + 1, b - 1);
  }
#pragma unroll
  for (int d = 0; d < 4; ++d)
    sb[d] = comp(own, d) + c.w * (comp(n0, d) + comp(n1, d) + comp(n2, d) + comp(n3, d));
}

// Node coefficients of every stencil of `type` at (I, J), stored at scalar
// slot co + k*3 + t (gP: the p_bar group; gX, gE, gS: the D_bar groups).
__device__ __forceinline__ void coef_point(const Ctx& c, int type, int I, int J, int gP, int gX,
                                           int gE, int gS, int co) {
  const float kap = type == 0 ? c.kap1 : c.kap2;
  const float k2 = kap * kap;
  const float4 pb4 = V(c, gP, I, J);
  float sb[4];
  si_bar4(c, type, I, J, gX, gE, gS, sb);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float pbar = comp(pb4, k);
    const float sbar = sb[k];
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    if (pbar != 0.f || sbar != 0.f) {
      const float n0 = node(c, type, k, 0, I, J);
      const float n1 = node(c, type, k, 1, I, J);
      const float n2 = node(c, type, k, 2, I, J);
      const float g = n1 - n0;
      const float s = fmaf(-2.f, n1, n0 + n2);
      c0 = fmaf(0.375f, pbar, (2.f * k2 * s - 2.f * g) * sbar);
      c1 = fmaf(0.75f, pbar, (2.f * g - 4.f * k2 * s) * sbar);
      c2 = fmaf(-0.125f, pbar, 2.f * k2 * s * sbar);
    }
    W(c, co + 3 * k + 0, I, J) = c0;
    W(c, co + 3 * k + 1, I, J) = c1;
    W(c, co + 3 * k + 2, I, J) = c2;
  }
}

__global__ void k_coef2(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_COEF2>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_COEF2; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    // E points whose adjoint can be nonzero: rows 0..n, columns -1..m-1;
    // S points: rows -1..n-1, columns 0..m.  Elsewhere the coefficients are 0.
    const bool e_live = I >= 0 && I <= c.n && J >= -1 && J < c.m;
    const bool s_live = I >= -1 && I < c.n && J >= 0 && J <= c.m;
    if (e_live) {
      coef_point(c, 1, I, J, G_EP, 0, G_ED, G_SD, S_ECO);
    } else {
  #pragma unroll
      for (int q = 0; q < 12; ++q) W(c, S_ECO + q, I, J) = 0.f;
    }
    if (s_live) {
      coef_point(c, 2, I, J, G_SP, 0, G_ED, G_SD, S_SCO);
    } else {
  #pragma unroll
      for (int q = 0; q < 12; ++q) W(c, S_SCO + q, I, J) = 0.f;
    }
  }
}

// Sum over the stencils of `type` whose node on `lattice` sits at (i, j).
__device__ __forceinline__ float gather(const Ctx& c, int type, int lattice, int i, int j,
                                        int co) {
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (lattice_of(type, k) != lattice) continue;
#pragma unroll
    for (int t = 0; t < 3; ++t)
      acc += W0(c, co + 3 * k + t, i - off_of(type, k, t, 0), j - off_of(type, k, t, 1));
  }
  return acc;
}

// X_bar (plus the x-point output gradient) and A_bar from phase 2, then at
// once the x point's own adjoint from that X_bar (phase 1): p_bar, D_bar of
// the x points, into the groups the "+" points used (no thread of this
// kernel reads them).
template <int BMODE>
__global__ void k_gather2_xadj(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_G2>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_G2; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    const int64_t plane = blockIdx.z;
    float xb = gather(c, 1, 1, I, J, S_ECO) + gather(c, 2, 1, I, J, S_SCO);
    float ab = gather(c, 1, 0, I, J, S_ECO) + gather(c, 2, 0, I, J, S_SCO);
    if (I >= 0 && I < c.n && J >= 0 && J < c.m) {
      xb += gout_at(a, plane, 2 * (int64_t)I + 1, 2 * (int64_t)J + 1);
      ab += gout_at(a, plane, 2 * (int64_t)I, 2 * (int64_t)J);
    }
    W(c, S_AB, I, J) = ab;
    // ---- phase-1 adjoint of this x point ----
    float pX[4] = {0.f, 0.f, 0.f, 0.f}, dX[4] = {0.f, 0.f, 0.f, 0.f};
    if (xb != 0.f && I >= -4 && I < c.n + 4 && J >= -4 && J < c.m + 4) {
      const Pt q = eval_pt(c, 0, I, J);
      float D[4];
      d_x<BMODE>(c, I, J, q.si, D);
      point_adjoint<BMODE>(q, D, c.beta, xb, pX, dX);
    }
    V(c, G_EP, I, J) = f4(pX);
    V(c, G_ED, I, J) = f4(dX);
  }
}

__global__ void k_coef1(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_COEF1>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_COEF1; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    if (I >= -5 && I < c.n + 5 && J >= -5 && J < c.m + 5) {
      coef_point(c, 0, I, J, G_EP, G_ED, 0, 0, S_ECO);
    } else {
  #pragma unroll
      for (int q = 0; q < 12; ++q) W(c, S_ECO + q, I, J) = 0.f;
    }
  }
}

__global__ void k_gather1(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_G1>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_G1; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    W(c, S_AB, I, J) += gather(c, 0, 0, I, J, S_ECO);
  }
}

// grad_in(i, j) = sum of A_bar over the extended cells that clamp to (i, j).
__global__ void k_fold(BwdArgs a, MethodConsts k) {
  Ctx c; int I0, J;
  if (!setup<R_FOLD>(a, k, c, I0, J)) return;
  for (int r = 0; r < R_FOLD; ++r) {
    const int I = I0 + r * BWD_BY;
    if (I >= c.n + G) break;
    if (I < 0 || I >= c.n || J < 0 || J >= c.m) continue;
    const int i0 = I == 0 ? -G : I, i1 = I == c.n - 1 ? c.n - 1 + G : I;
    const int j0 = J == 0 ? -G : J, j1 = J == c.m - 1 ? c.m - 1 + G : J;
    float acc = 0.f;
    for (int ii = i0; ii <= i1; ++ii)
      for (int jj = j0; jj <= j1; ++jj) acc += W(c, S_AB, ii, jj);
    const int64_t plane = blockIdx.z;
    a.gin[plane * a.gi_sc + (int64_t)I * a.gi_sh + (int64_t)J * a.gi_sw] = acc;
  }
}

template <int BMODE>
cudaError_t launch_all(const BwdArgs& a, const MethodConsts& k, cudaStream_t st) {
  const dim3 block(32, BWD_BY);
  auto grid = [&](int R) {
    return dim3((unsigned)((a.m + 2 * G + 31) / 32),
                (unsigned)((a.n + 2 * G + BWD_BY * R - 1) / (BWD_BY * R)), (unsigned)a.planes);
  };
  k_xsi<<<grid(R_XSI), block, 0, st>>>(a, k);
  k_xval<BMODE><<<grid(R_XVAL), block, 0, st>>>(a, k);
  k_psi<<<grid(R_PSI), block, 0, st>>>(a, k);
  k_padj<BMODE><<<grid(R_PADJ), block, 0, st>>>(a, k);
  k_coef2<<<grid(R_COEF2), block, 0, st>>>(a, k);
  k_gather2_xadj<BMODE><<<grid(R_G2), block, 0, st>>>(a, k);
  k_coef1<<<grid(R_COEF1), block, 0, st>>>(a, k);
  k_gather1<<<grid(R_G1), block, 0, st>>>(a, k);
  k_fold<<<grid(R_FOLD), block, 0, st>>>(a, k);
  return cudaGetLastError();
}

}  // namespace

size_t bwd_workspace_bytes(int64_t n, int64_t m, int64_t planes) {
  // per plane: the extended cell count padded to a multiple of 4 (float4 planes)
  const size_t cells = ((size_t)(n + 2 * G) * (size_t)(m + 2 * G) + 3) & ~(size_t)3;
  return sizeof(float) * (size_t)BWD_ARRAYS * cells * (size_t)planes;
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
