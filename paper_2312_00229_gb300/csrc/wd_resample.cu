// Tensor-product WENO resampling to an arbitrary size (arXiv 2312.00229,
// Sec. 3.3, Eq. tensor), the second stage of the arbitrary-scale zoom.
//
// The 1-D WENO interpolant of Sec. 2 on the cell [x_i, x_{i+1}], t in [0, 1],
// with samples v0..v3 at x_{i-1..i+2}: writing g = v2 - v1,
// sL = v0 - 2 v1 + v2 and sR = v1 - 2 v2 + v3, the two quadratics are
//     p_i(t)     = v1 + g t + sL (t^2 - t) / 2
//     p_{i+1}(t) = v1 + g t + sR (t^2 - t) / 2
// (Eq. Tocnost), their indicators (Sec. 2) are g^2 + 13/12 sL^2 and
// g^2 + 13/12 sR^2, and the linear weights that recover the cubic (Eq.
// PolinomZaVelikiStencil) are C_0 = (2 - t)/3, C_1 = (1 + t)/3, so
//     u = v1 + g t + (t^2 - t)/2 (alpha_0 sL + alpha_1 sR) / (alpha_0 + alpha_1),
//     alpha_s = C_s / (eps_h + SI_s)^beta                     (Eq. IzrazOmega).
// One thread per output pixel: four 1-D interpolants down the columns of
// the 4x4 input window (z_k = w(A(:,k), y)), then one across them
// (U = w(Z, x)).  Inputs outside the image are clamped to the edge.
#include "wd_common.cuh"
#include "wd_resample.h"

namespace wdweno {

namespace {

template <int BMODE>
__device__ __forceinline__ float weno1d(float v0, float v1, float v2, float v3, float t,
                                        float eps, float beta) {
  const float g = v2 - v1;
  const float sL = fmaf(-2.f, v1, v0 + v2);
  const float sR = fmaf(-2.f, v2, v1 + v3);
  const float C0 = (2.f - t) * (1.f / 3.f);
  const float C1 = 1.f - C0;
  float a0, a1;
  if (BMODE == B0) {
    a0 = C0; a1 = C1;
  } else {
    // alpha_0 : alpha_1 = C_0 eR^beta : C_1 eL^beta with both indicators
    // divided by the larger one, so no power over- or underflows.  eps is
    // at least 1e-30 (host side), so the larger indicator is a normal number.
    const float k2 = 13.f / 12.f;
    const float eL = fmaf(g, g, fmaf(k2 * sL, sL, eps));
    const float eR = fmaf(g, g, fmaf(k2 * sR, sR, eps));
    const float inv = rcp_approx(fmaxf(eL, eR));
    const float rL = eL * inv, rR = eR * inv;
    if (BMODE == B2) {
      a0 = C0 * rR * rR; a1 = C1 * rL * rL;
    } else {
      a0 = C0 * ex2_approx(beta * lg2_approx(rR));
      a1 = C1 * ex2_approx(beta * lg2_approx(rL));
    }
  }
  // a0 + a1 >= 1/3: one ratio is 1 and both C_s are at least 1/3
  const float mix = fmaf(a0, sL, a1 * sR) * rcp_approx(a0 + a1);
  return fmaf(0.5f * fmaf(t, t, -t), mix, fmaf(g, t, v1));
}

// Cell index and offset of output index j on the endpoint-aligned grid of
// n_out points over 0..n-1, in exact integer arithmetic.
__device__ __forceinline__ void grid_pos(int64_t j, int64_t n, int64_t n_out, int64_t& i,
                                         float& t) {
  if (n <= 1 || n_out <= 1) { i = 0; t = 0.f; return; }
  const int64_t num = j * (n - 1), den = n_out - 1;
  i = num / den;
  int64_t rem = num - i * den;
  if (i > n - 2) { i = n - 2; rem = den; }  // last sample: t = 1 on the last cell
  t = (float)((double)rem / (double)den);
}

template <int BMODE>
__global__ void __launch_bounds__(256) resample_kernel(ResampleArgs a, float eps, float beta) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (r >= a.n_out || c >= a.m_out) return;
  const int64_t plane = blockIdx.z;
  int64_t i, j;
  float ty, tx;
  grid_pos(r, a.n, a.n_out, i, ty);
  grid_pos(c, a.m, a.m_out, j, tx);
  const int64_t base = plane * a.in_sc;
  float z[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t col = j - 1 + q < 0 ? 0 : (j - 1 + q > a.m - 1 ? a.m - 1 : j - 1 + q);
    float v[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t row = i - 1 + p < 0 ? 0 : (i - 1 + p > a.n - 1 ? a.n - 1 : i - 1 + p);
      v[p] = load_elem(a.in, base + row * a.in_sh + col * a.in_sw, a.in_dtype);
    }
    z[q] = a.n > 1 ? weno1d<BMODE>(v[0], v[1], v[2], v[3], ty, eps, beta) : v[1];
  }
  const float u = a.m > 1 ? weno1d<BMODE>(z[0], z[1], z[2], z[3], tx, eps, beta) : z[1];
  store_elem(a.out, plane * a.out_sc + r * a.out_sh + c * a.out_sw, u, a.out_dtype,
             a.clamp_float);
}

// Separable tiled form for scales down to 1/2 in x: a CTA owns RS_TR
// output rows x RS_TC output columns of one plane.  Pass 1 forms the column
// interpolants z(r, k) = w(A(:, k), y_r) for the tile's rows and every input
// column its outputs read (at most 2 RS_TC + 5 of them), into shared memory;
// pass 2 interpolates each output across four of them.  Per output this is
// about 1 + (in/out column ratio) + small halo 1-D interpolants instead of 5.
constexpr int RS_TR = 16;
constexpr int RS_TC = 128;
constexpr int RS_WC = 2 * RS_TC + 8;
constexpr int RS_THREADS = 256;

template <int BMODE>
__global__ void __launch_bounds__(RS_THREADS) resample_tiled_kernel(ResampleArgs a, float eps,
                                                                   float beta) {
  __shared__ float z[RS_TR][RS_WC];
  __shared__ int col_j[RS_TC];
  __shared__ float col_t[RS_TC];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * RS_TC;
  const int64_t r0 = (int64_t)blockIdx.y * RS_TR;
  const int64_t plane = blockIdx.z;
  const int nc = (int)(a.m_out - c0 < RS_TC ? a.m_out - c0 : RS_TC);
  const int nr = (int)(a.n_out - r0 < RS_TR ? a.n_out - r0 : RS_TR);
  int64_t jf, jl;
  float tdummy;
  grid_pos(c0, a.m, a.m_out, jf, tdummy);
  grid_pos(c0 + nc - 1, a.m, a.m_out, jl, tdummy);
  const int64_t kfirst = jf - 1;
  const int wc = (int)(jl + 2 - kfirst + 1);  // <= RS_WC (host checks the scale)
  if (tid < nc) {
    int64_t j;
    float t;
    grid_pos(c0 + tid, a.m, a.m_out, j, t);
    col_j[tid] = (int)(j - 1 - kfirst);
    col_t[tid] = t;
  }
  const int64_t base = plane * a.in_sc;
  for (int r = warp; r < nr; r += RS_THREADS / 32) {
    int64_t i;
    float ty;
    grid_pos(r0 + r, a.n, a.n_out, i, ty);
    int64_t rows[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t q = i - 1 + p;
      rows[p] = base + (q < 0 ? 0 : (q > a.n - 1 ? a.n - 1 : q)) * a.in_sh;
    }
    for (int k = lane; k < wc; k += 32) {
      const int64_t kk = kfirst + k;
      const int64_t col = (kk < 0 ? 0 : (kk > a.m - 1 ? a.m - 1 : kk)) * a.in_sw;
      const float v0 = load_elem(a.in, rows[0] + col, a.in_dtype);
      const float v1 = load_elem(a.in, rows[1] + col, a.in_dtype);
      const float v2 = load_elem(a.in, rows[2] + col, a.in_dtype);
      const float v3 = load_elem(a.in, rows[3] + col, a.in_dtype);
      z[r][k] = weno1d<BMODE>(v0, v1, v2, v3, ty, eps, beta);
    }
  }
  __syncthreads();
  for (int r = warp; r < nr; r += RS_THREADS / 32) {
    const int64_t orow = plane * a.out_sc + (r0 + r) * a.out_sh;
    for (int c = lane; c < nc; c += 32) {
      const int k = col_j[c];
      const float u = weno1d<BMODE>(z[r][k], z[r][k + 1], z[r][k + 2], z[r][k + 3], col_t[c],
                                    eps, beta);
      store_elem(a.out, orow + (c0 + c) * a.out_sw, u, a.out_dtype, a.clamp_float);
    }
  }
}

}  // namespace

cudaError_t launch_resample(const ResampleArgs& a, float eps, float beta, int bmode,
                            cudaStream_t stream) {
  // the tiled form needs at most RS_WC input columns per tile: column
  // spacing ratio (m - 1)/(m_out - 1) <= 2
  const bool tiled = a.m_out == 1 || 2 * (a.m_out - 1) >= (a.m - 1);
  if (tiled) {
    const dim3 grid((unsigned)((a.m_out + RS_TC - 1) / RS_TC),
                    (unsigned)((a.n_out + RS_TR - 1) / RS_TR), (unsigned)a.planes);
    switch (bmode) {
      case B2: resample_tiled_kernel<B2><<<grid, RS_THREADS, 0, stream>>>(a, eps, beta); break;
      case B0: resample_tiled_kernel<B0><<<grid, RS_THREADS, 0, stream>>>(a, eps, beta); break;
      default: resample_tiled_kernel<BGEN><<<grid, RS_THREADS, 0, stream>>>(a, eps, beta); break;
    }
    return cudaGetLastError();
  }
  const dim3 block(32, 8);
  const dim3 grid((unsigned)((a.m_out + 31) / 32), (unsigned)((a.n_out + 7) / 8),
                  (unsigned)a.planes);
  switch (bmode) {
    case B2: resample_kernel<B2><<<grid, block, 0, stream>>>(a, eps, beta); break;
    case B0: resample_kernel<B0><<<grid, block, 0, stream>>>(a, eps, beta); break;
    default: resample_kernel<BGEN><<<grid, block, 0, stream>>>(a, eps, beta); break;
  }
  return cudaGetLastError();
}

}  // namespace wdweno
