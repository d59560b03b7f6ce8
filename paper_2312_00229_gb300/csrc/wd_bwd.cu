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
// The kernels below evaluate these scatters as gathers over a grid extended
// by BWD_GHOST cells per side (clamp-to-edge), then fold the ghost cells
// back onto the edge pixels (the adjoint of the extension):
//   k_fwd_x        phase-1 values X on the extended grid
//   k_point2       p_bar, D_bar of every "+" point (phase 2)
//   k_gather2      X_bar (plus the x-point output gradient) and A_bar from
//                  phase 2 (plus the sample-point output gradient)
//   k_point1       p_bar, D_bar of every "x" point (phase 1)
//   k_gather1      A_bar from phase 1
//   k_fold         grad_in = A_bar summed over each pixel's clamp preimage
#include "wd_bwd.h"

namespace wdweno {

namespace {

constexpr int G = BWD_GHOST;
// workspace array slots
enum {
  W_X = 0,     // phase-1 values
  W_PE = 1,    // p_bar of E points, 4 directions (reused for x points)
  W_DE = 5,    // D_bar of E points (reused for x points)
  W_PS = 9,    // p_bar of S points
  W_DS = 13,   // D_bar of S points
  W_XB = 17,   // X_bar
  W_AB = 18    // A_bar on the extended grid
};

struct Ctx {
  const float* x;  // plane base
  int64_t n, m, sh, sw;
  float* ws;       // plane base of the workspace
  int64_t NE, ME;  // extended extents
  MethodConsts k;
};

__device__ __forceinline__ int64_t clampi(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ float Ahat(const Ctx& c, int64_t i, int64_t j) {
  return __ldg(c.x + clampi(i, 0, c.n - 1) * c.sh + clampi(j, 0, c.m - 1) * c.sw);
}

__device__ __forceinline__ int64_t widx(const Ctx& c, int arr, int64_t I, int64_t J) {
  return (int64_t)arr * c.NE * c.ME + (I + G) * c.ME + (J + G);
}

__device__ __forceinline__ bool in_ext(const Ctx& c, int64_t I, int64_t J) {
  return I >= -G && I < c.n + G && J >= -G && J < c.m + G;
}

// Reads a workspace value; 0 outside the extended grid.
__device__ __forceinline__ float W0(const Ctx& c, int arr, int64_t I, int64_t J) {
  return in_ext(c, I, J) ? c.ws[widx(c, arr, I, J)] : 0.f;
}

__device__ __forceinline__ float Xv(const Ctx& c, int64_t a, int64_t b) {
  return c.ws[widx(c, W_X, a, b)];
}

// ---------------------------------------------------------------------------
// Stencil tables.  Point types: 0 = x point, 1 = E point (fine (2a, 2b+1)),
// 2 = S point (fine (2a+1, 2b)).  For each type and direction k the three
// nodes N0, N1, N2 sit at (a, b) + off, on the lattice of input samples
// (lattice 0) or of x points (lattice 1).
// x: k = 0 (1,1), 1 (-1,-1), 2 (1,-1), 3 (-1,1)
// E, S: k = 0 (0,1), 1 (0,-1), 2 (1,0), 3 (-1,0)
// ---------------------------------------------------------------------------
__constant__ int c_off[3][4][3][2] = {
    {{{0, 0}, {1, 1}, {2, 2}}, {{1, 1}, {0, 0}, {-1, -1}},
     {{0, 1}, {1, 0}, {2, -1}}, {{1, 0}, {0, 1}, {-1, 2}}},
    {{{0, 0}, {0, 1}, {0, 2}}, {{0, 1}, {0, 0}, {0, -1}},
     {{-1, 0}, {0, 0}, {1, 0}}, {{0, 0}, {-1, 0}, {-2, 0}}},
    {{{0, -1}, {0, 0}, {0, 1}}, {{0, 0}, {0, -1}, {0, -2}},
     {{0, 0}, {1, 0}, {2, 0}}, {{1, 0}, {0, 0}, {-1, 0}}}};
__constant__ int c_lattice[3][4] = {{0, 0, 0, 0}, {0, 0, 1, 1}, {1, 1, 0, 0}};

__device__ __forceinline__ float node(const Ctx& c, int type, int k, int t, int64_t a, int64_t b) {
  const int64_t i = a + c_off[type][k][t][0], j = b + c_off[type][k][t][1];
  return c_lattice[type][k] == 0 ? Ahat(c, i, j) : Xv(c, i, j);
}

struct Pt {
  float p[4];   // interpolants
  float si[4];  // indicators (eps' included)
  float M[2];   // N0 + N1 of the pairs (0,1) and (2,3)
  float s[4];   // second differences
};

__device__ __forceinline__ Pt eval_pt(const Ctx& c, int type, int64_t a, int64_t b) {
  Pt q;
  const float kap = type == 0 ? c.k.kappa1 : c.k.kappa2;
  const float eps = type == 0 ? c.k.eps1 : c.k.eps2;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float n0 = node(c, type, k, 0, a, b);
    const float n1 = node(c, type, k, 1, a, b);
    const float n2 = node(c, type, k, 2, a, b);
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

__device__ __forceinline__ void si4(const Ctx& c, int type, int64_t a, int64_t b, float out[4]) {
  Pt q = eval_pt(c, type, a, b);
#pragma unroll
  for (int k = 0; k < 4; ++k) out[k] = q.si[k];
}

// D of the four directions at a point (neighbours per Eqs. 2DsmoothnessFinal
// and tezine).
__device__ __forceinline__ void d4(const Ctx& c, int type, int64_t a, int64_t b, const Pt& q,
                                   float D[4]) {
  float acc[4] = {0.f, 0.f, 0.f, 0.f}, t[4];
  if (type == 0) {
    const int64_t nb[4][2] = {{a - 1, b}, {a + 1, b}, {a, b - 1}, {a, b + 1}};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      si4(c, 0, nb[i][0], nb[i][1], t);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += t[k];
    }
  } else if (type == 1) {  // E(a,b): S at (a-1,b), (a,b), (a-1,b+1), (a,b+1)
    const int64_t nb[4][2] = {{a - 1, b}, {a, b}, {a - 1, b + 1}, {a, b + 1}};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      si4(c, 2, nb[i][0], nb[i][1], t);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += t[k];
    }
  } else {  // S(a,b): E at (a,b-1), (a,b), (a+1,b-1), (a+1,b)
    const int64_t nb[4][2] = {{a, b - 1}, {a, b}, {a + 1, b - 1}, {a + 1, b}};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      si4(c, 1, nb[i][0], nb[i][1], t);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] += t[k];
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) D[k] = fmaf(c.k.w, acc[k], q.si[k]);
}

// Normalised weights omega_k from D_k (Eq. alpha, IzrazOmega2d).
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
      const float r = dmin / D[k];
      al[k] = BMODE == B2 ? r * r : ex2_approx(beta * lg2_approx(r));
    }
  }
  const float inv = 1.f / ((al[0] + al[1]) + (al[2] + al[3]));
#pragma unroll
  for (int k = 0; k < 4; ++k) om[k] = al[k] * inv;
}

// p_bar, D_bar of one blend point for the incoming adjoint ub.
template <int BMODE>
__device__ __forceinline__ void point_adjoint(const Ctx& c, int type, int64_t a, int64_t b,
                                              float ub, float pb[4], float db[4]) {
  const Pt q = eval_pt(c, type, a, b);
  float D[4], om[4];
  d4(c, type, a, b, q, D);
  weights<BMODE>(D, c.k.beta, om);
  // p_k - u = sum_l omega_l (p_k - p_l), each difference formed from the
  // stencil data to avoid cancelling two O(1) values.
  float dp[4];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    float acc = 0.f;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float dM = (kk >> 1) == (l >> 1) ? 0.f : q.M[kk >> 1] - q.M[l >> 1];
      acc = fmaf(om[l], fmaf(0.5f, dM, -0.125f * (q.s[kk] - q.s[l])), acc);
    }
    dp[kk] = acc;
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    pb[kk] = ub * om[kk];
    db[kk] = BMODE == B0 ? 0.f : -ub * c.k.beta * om[kk] * dp[kk] / D[kk];
  }
}

// SI_bar of direction k at a point: its own D_bar plus w times the D_bar of
// the points whose D reads it.
__device__ __forceinline__ float si_bar(const Ctx& c, int type, int k, int64_t a, int64_t b,
                                        int dE, int dS) {
  const float w = c.k.w;
  if (type == 0) {
    return W0(c, dE + k, a, b) + w * (W0(c, dE + k, a - 1, b) + W0(c, dE + k, a + 1, b) +
                                      W0(c, dE + k, a, b - 1) + W0(c, dE + k, a, b + 1));
  } else if (type == 1) {  // E(a,b) is read by S(a,b), S(a,b+1), S(a-1,b), S(a-1,b+1)
    return W0(c, dE + k, a, b) + w * (W0(c, dS + k, a, b) + W0(c, dS + k, a, b + 1) +
                                      W0(c, dS + k, a - 1, b) + W0(c, dS + k, a - 1, b + 1));
  } else {  // S(a,b) is read by E(a,b), E(a+1,b), E(a,b-1), E(a+1,b-1)
    return W0(c, dS + k, a, b) + w * (W0(c, dE + k, a, b) + W0(c, dE + k, a + 1, b) +
                                      W0(c, dE + k, a, b - 1) + W0(c, dE + k, a + 1, b - 1));
  }
}

// Sum of the contributions of all stencils of `type` whose node on
// `lattice` sits at (i, j).
__device__ float gather_node(const Ctx& c, int type, int lattice, int64_t i, int64_t j, int pB,
                             int dE, int dS) {
  const float kap = type == 0 ? c.k.kappa1 : c.k.kappa2;
  const float k2 = kap * kap;
  float acc = 0.f;
  for (int k = 0; k < 4; ++k) {
    if (c_lattice[type][k] != lattice) continue;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const int64_t a = i - c_off[type][k][t][0], b = j - c_off[type][k][t][1];
      if (!in_ext(c, a, b)) continue;
      const float pbar = c.ws[widx(c, pB + k, a, b)];
      const float sbar = si_bar(c, type, k, a, b, dE, dS);
      if (pbar == 0.f && sbar == 0.f) continue;
      const float n0 = node(c, type, k, 0, a, b);
      const float n1 = node(c, type, k, 1, a, b);
      const float n2 = node(c, type, k, 2, a, b);
      const float g = n1 - n0;
      const float s = fmaf(-2.f, n1, n0 + n2);
      float coef;
      if (t == 0) coef = fmaf(0.375f, pbar, (2.f * k2 * s - 2.f * g) * sbar);
      else if (t == 1) coef = fmaf(0.75f, pbar, (2.f * g - 4.f * k2 * s) * sbar);
      else coef = fmaf(-0.125f, pbar, 2.f * k2 * s * sbar);
      acc += coef;
    }
  }
  return acc;
}

__device__ __forceinline__ bool setup(const BwdArgs& a, const MethodConsts& k, Ctx& c,
                                      int64_t& I, int64_t& J) {
  const int64_t plane = blockIdx.z;
  c.n = a.n; c.m = a.m; c.sh = a.x_sh; c.sw = a.x_sw;
  c.x = a.x + plane * a.x_sc;
  c.NE = a.n + 2 * G; c.ME = a.m + 2 * G;
  c.ws = a.ws + plane * (int64_t)BWD_ARRAYS * c.NE * c.ME;
  c.k = k;
  J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - G;
  I = (int64_t)blockIdx.y * blockDim.y + threadIdx.y - G;
  return I < a.n + G && J < a.m + G;
}

// x values on the extended grid (rows/columns -4 .. n+3); 0 further out.
template <int BMODE>
__global__ void k_fwd_x(BwdArgs a, MethodConsts k) {
  Ctx c; int64_t I, J;
  if (!setup(a, k, c, I, J)) return;
  float v = 0.f;
  if (I >= -4 && I < c.n + 4 && J >= -4 && J < c.m + 4) {
    const Pt q = eval_pt(c, 0, I, J);
    float D[4], om[4];
    d4(c, 0, I, J, q, D);
    weights<BMODE>(D, k.beta, om);
    v = om[0] * q.p[0] + om[1] * q.p[1] + om[2] * q.p[2] + om[3] * q.p[3];
  }
  c.ws[widx(c, W_X, I, J)] = v;
}

__device__ __forceinline__ float gout_at(const BwdArgs& a, int64_t plane, int64_t P, int64_t Q) {
  if (P < 0 || Q < 0 || P >= a.orows || Q >= a.ocols) return 0.f;
  return __ldg(a.gout + plane * a.g_sc + P * a.g_sh + Q * a.g_sw);
}

template <int BMODE>
__global__ void k_point2(BwdArgs a, MethodConsts k) {
  Ctx c; int64_t I, J;
  if (!setup(a, k, c, I, J)) return;
  float pE[4] = {0.f, 0.f, 0.f, 0.f}, dE[4] = {0.f, 0.f, 0.f, 0.f};
  float pS[4] = {0.f, 0.f, 0.f, 0.f}, dS[4] = {0.f, 0.f, 0.f, 0.f};
  if (I >= 0 && I < c.n && J >= 0 && J < c.m) {
    const int64_t plane = blockIdx.z;
    const float uE = gout_at(a, plane, 2 * I, 2 * J + 1);
    const float uS = gout_at(a, plane, 2 * I + 1, 2 * J);
    if (uE != 0.f) point_adjoint<BMODE>(c, 1, I, J, uE, pE, dE);
    if (uS != 0.f) point_adjoint<BMODE>(c, 2, I, J, uS, pS, dS);
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    c.ws[widx(c, W_PE + kk, I, J)] = pE[kk];
    c.ws[widx(c, W_DE + kk, I, J)] = dE[kk];
    c.ws[widx(c, W_PS + kk, I, J)] = pS[kk];
    c.ws[widx(c, W_DS + kk, I, J)] = dS[kk];
  }
}

__global__ void k_gather2(BwdArgs a, MethodConsts k) {
  Ctx c; int64_t I, J;
  if (!setup(a, k, c, I, J)) return;
  const int64_t plane = blockIdx.z;
  float xb = 0.f, ab = 0.f;
  if (I >= -4 && I < c.n + 4 && J >= -4 && J < c.m + 4) {
    // X_bar: x-point output gradient plus phase-2 stencils on the x lattice
    xb = gather_node(c, 1, 1, I, J, W_PE, W_DE, W_DS) + gather_node(c, 2, 1, I, J, W_PS, W_DE, W_DS);
    ab = gather_node(c, 1, 0, I, J, W_PE, W_DE, W_DS) + gather_node(c, 2, 0, I, J, W_PS, W_DE, W_DS);
    if (I >= 0 && I < c.n && J >= 0 && J < c.m) {
      xb += gout_at(a, plane, 2 * I + 1, 2 * J + 1);
      ab += gout_at(a, plane, 2 * I, 2 * J);
    }
  }
  c.ws[widx(c, W_XB, I, J)] = xb;
  c.ws[widx(c, W_AB, I, J)] = ab;
}

template <int BMODE>
__global__ void k_point1(BwdArgs a, MethodConsts k) {
  Ctx c; int64_t I, J;
  if (!setup(a, k, c, I, J)) return;
  float pX[4] = {0.f, 0.f, 0.f, 0.f}, dX[4] = {0.f, 0.f, 0.f, 0.f};
  const float xb = c.ws[widx(c, W_XB, I, J)];
  if (xb != 0.f && I >= -4 && I < c.n + 4 && J >= -4 && J < c.m + 4)
    point_adjoint<BMODE>(c, 0, I, J, xb, pX, dX);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    c.ws[widx(c, W_PE + kk, I, J)] = pX[kk];
    c.ws[widx(c, W_DE + kk, I, J)] = dX[kk];
  }
}

__global__ void k_gather1(BwdArgs a, MethodConsts k) {
  Ctx c; int64_t I, J;
  if (!setup(a, k, c, I, J)) return;
  if (I >= -G + 1 && I < c.n + G - 1 && J >= -G + 1 && J < c.m + G - 1)
    c.ws[widx(c, W_AB, I, J)] += gather_node(c, 0, 0, I, J, W_PE, W_DE, W_DS);
}

// grad_in(i, j) = sum of A_bar over the extended cells that clamp to (i, j).
__global__ void k_fold(BwdArgs a, MethodConsts k) {
  Ctx c; int64_t I, J;
  if (!setup(a, k, c, I, J)) return;
  if (I < 0 || I >= c.n || J < 0 || J >= c.m) return;
  const int64_t i0 = I == 0 ? -G : I, i1 = I == c.n - 1 ? c.n - 1 + G : I;
  const int64_t j0 = J == 0 ? -G : J, j1 = J == c.m - 1 ? c.m - 1 + G : J;
  float acc = 0.f;
  for (int64_t ii = i0; ii <= i1; ++ii)
    for (int64_t jj = j0; jj <= j1; ++jj)
      if (in_ext(c, ii, jj)) acc += c.ws[widx(c, W_AB, ii, jj)];
  const int64_t plane = blockIdx.z;
  a.gin[plane * a.gi_sc + I * a.gi_sh + J * a.gi_sw] = acc;
}

template <int BMODE>
cudaError_t launch_all(const BwdArgs& a, const MethodConsts& k, cudaStream_t st) {
  const dim3 block(32, 8);
  const dim3 grid((unsigned)((a.m + 2 * G + 31) / 32), (unsigned)((a.n + 2 * G + 7) / 8),
                  (unsigned)a.planes);
  k_fwd_x<BMODE><<<grid, block, 0, st>>>(a, k);
  k_point2<BMODE><<<grid, block, 0, st>>>(a, k);
  k_gather2<<<grid, block, 0, st>>>(a, k);
  k_point1<BMODE><<<grid, block, 0, st>>>(a, k);
  k_gather1<<<grid, block, 0, st>>>(a, k);
  k_fold<<<grid, block, 0, st>>>(a, k);
  return cudaGetLastError();
}

}  // namespace

size_t bwd_workspace_bytes(int64_t n, int64_t m, int64_t planes) {
  return sizeof(float) * (size_t)BWD_ARRAYS * (size_t)(n + 2 * G) * (size_t)(m + 2 * G) *
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
