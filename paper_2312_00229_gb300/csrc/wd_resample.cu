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
#include <type_traits>

#include "wd_common.cuh"
#include "wd_packed.cuh"
#include "wd_resample.h"

namespace wdweno {

namespace {

// With the position's constants given: C0 = (2 - t)/3 and h = (t^2 - t)/2.
template <int BMODE>
__device__ __forceinline__ float weno1d_at(float v0, float v1, float v2, float v3, float t,
                                           float C0, float h, float eps, float beta) {
  const float g = v2 - v1;
  const float sL = fmaf(-2.f, v1, v0 + v2);
  const float sR = fmaf(-2.f, v2, v1 + v3);
  const float C1 = 1.f - C0;
  float a0, a1;
  if (BMODE == B0) {
    a0 = C0; a1 = C1;
  } else if (BMODE == B2R) {
    // alpha_0 : alpha_1 = C_0 eR^2 : C_1 eL^2 as written; the host picks
    // this form only where the storage type bounds the data so that every
    // square, their sum and the numerator below are normal FP32 numbers
    const float k2 = 13.f / 12.f;
    const float eL = fmaf(g, g, fmaf(k2 * sL, sL, eps));
    const float eR = fmaf(g, g, fmaf(k2 * sR, sR, eps));
    a0 = C0 * (eR * eR);
    a1 = C1 * (eL * eL);
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
  // a0 + a1 >= 1/3 in the scaled forms: one ratio is 1 and both C_s are at
  // least 1/3
  const float mix = fmaf(a0, sL, a1 * sR) * rcp_approx(a0 + a1);
  return fmaf(h, mix, fmaf(g, t, v1));
}

// Two interpolants at once on Blackwell's packed two-lane FP32 instructions
// (pk_* helpers of wd_packed.cuh): weno1d_at on lane pairs, the same
// expressions in the same order, each lane rounded as the scalar form.
template <int BMODE>
__device__ __forceinline__ f2 weno1d_at2(f2 v0, f2 v1, f2 v2, f2 v3, f2 t, f2 C0, f2 h,
                                         float eps, float beta) {
  const f2 g = pk_sub(v2, v1);
  const f2 sL = pk_fma(pk_bc(-2.f), v1, pk_add(v0, v2));
  const f2 sR = pk_fma(pk_bc(-2.f), v2, pk_add(v1, v3));
  const f2 C1 = pk_sub(pk_bc(1.f), C0);
  f2 a0, a1;
  if (BMODE == B0) {
    a0 = C0; a1 = C1;
  } else {
    const f2 k2 = pk_bc(13.f / 12.f), e = pk_bc(eps);
    const f2 eL = pk_fma(g, g, pk_fma(pk_mul(k2, sL), sL, e));
    const f2 eR = pk_fma(g, g, pk_fma(pk_mul(k2, sR), sR, e));
    if (BMODE == B2R) {
      a0 = pk_mul(C0, pk_mul(eR, eR));
      a1 = pk_mul(C1, pk_mul(eL, eL));
    } else {
      const f2 inv = pk_rcp(make_float2(fmaxf(eL.x, eR.x), fmaxf(eL.y, eR.y)));
      const f2 rL = pk_mul(eL, inv), rR = pk_mul(eR, inv);
      if (BMODE == B2) {
        a0 = pk_mul(pk_mul(C0, rR), rR);
        a1 = pk_mul(pk_mul(C1, rL), rL);
      } else {
        const f2 b = pk_bc(beta);
        const f2 lR = pk_mul(b, make_float2(lg2_approx(rR.x), lg2_approx(rR.y)));
        const f2 lL = pk_mul(b, make_float2(lg2_approx(rL.x), lg2_approx(rL.y)));
        a0 = pk_mul(C0, make_float2(ex2_approx(lR.x), ex2_approx(lR.y)));
        a1 = pk_mul(C1, make_float2(ex2_approx(lL.x), ex2_approx(lL.y)));
      }
    }
  }
  const f2 mix = pk_mul(pk_fma(a0, sL, pk_mul(a1, sR)), pk_rcp(pk_add(a0, a1)));
  return pk_fma(h, mix, pk_fma(g, t, v1));
}

template <int BMODE>
__device__ __forceinline__ float weno1d(float v0, float v1, float v2, float v3, float t,
                                        float eps, float beta) {
  return weno1d_at<BMODE>(v0, v1, v2, v3, t, (2.f - t) * (1.f / 3.f), 0.5f * fmaf(t, t, -t),
                          eps, beta);
}

// Cell index and offset of output index j on the endpoint-aligned grid of
// n_out points over 0..n-1: i = floor(j (n-1) / (n_out-1)) exactly (by
// multiply-high when the numerator fits 32 bits), t = remainder / (n_out-1).
__device__ __forceinline__ void grid_pos(int64_t j, int64_t n, int64_t n_out, const AxisDiv& d,
                                         int64_t& i, float& t) {
  if (n <= 1 || n_out <= 1) { i = 0; t = 0.f; return; }
  const int64_t den = n_out - 1;
  int64_t q, rem;
  if (d.fast) {
    const uint32_t num = (uint32_t)j * (uint32_t)(n - 1);
    const uint32_t t1 = __umulhi(d.mag, num);
    const uint32_t qq = (t1 + ((num - t1) >> d.sh1)) >> d.sh2;
    q = qq;
    rem = (int64_t)(num - qq * (uint32_t)den);
  } else {
    const int64_t num = j * (n - 1);
    q = num / den;
    rem = num - q * den;
  }
  if (q > n - 2) { q = n - 2; rem = den; }  // last sample: t = 1 on the last cell
  i = q;
  t = rem == den ? 1.f : (float)rem * d.inv;
}

template <int BMODE>
__global__ void __launch_bounds__(256) resample_kernel(ResampleArgs a, float eps, float beta) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (r >= a.n_out || c >= a.m_out) return;
  const int64_t plane = blockIdx.z;
  int64_t i, j;
  float ty, tx;
  grid_pos(r, a.n, a.n_out, a.div_y, i, ty);
  grid_pos(c, a.m, a.m_out, a.div_x, j, tx);
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

// Storage access: a concrete element type, or Dyn for the run-time type.
struct Dyn {};

// Storage bits of one element and their value (the loads of a group are all
// issued before any of them is converted).
template <class T>
__device__ __forceinline__ uint32_t rs_load_bits(const void* base, int64_t idx, int dt) {
  if constexpr (std::is_same<T, Dyn>::value) {
    return load_elem_bits(base, idx, dt);
  } else {
    return load_elem_bits(base, idx, DTypeOf<T>::value);
  }
}

template <class T>
__device__ __forceinline__ float rs_value(uint32_t b, int dt) {
  if constexpr (std::is_same<T, Dyn>::value) {
    return elem_bits_value(b, dt);
  } else {
    return elem_bits_value(b, DTypeOf<T>::value);
  }
}

template <class T>
__device__ __forceinline__ void rs_store(void* base, int64_t idx, float v, int dt, int clampf) {
  if constexpr (std::is_same<T, Dyn>::value) {
    store_elem(base, idx, v, dt, clampf);
  } else {
    store_typed<T>(base, idx, v, clampf);
  }
}

template <class T>
__device__ __forceinline__ void rs_store4(void* base, int64_t idx, const float (&u)[4], int dt,
                                          int clampf) {
  if constexpr (std::is_same<T, Dyn>::value) {
    store4_vec(base, idx, u[0], u[1], u[2], u[3], dt, clampf);
  } else {
    store4_typed<T>(base, idx, u[0], u[1], u[2], u[3], clampf);
  }
}

// Separable tiled form for output/input spacing ratios down to 1/2 on both
// axes: a CTA owns tile_rows (16 or 32) output rows x RS_TC output columns of one
// plane.
//   stage 0  the input window those outputs read (rows i(r0)-1 .. i(r_last)+2,
//            columns j(c0)-1 .. j(c_last)+2, clamped) decoded into shared memory
//   pass 1   the column interpolants z(r, k) = w(A(:, k), y_r) of the tile's
//            rows at every window column (Eq. tensor, first factor)
//   pass 2   each thread interpolates four consecutive outputs of a row across
//            the z values (Eq. tensor, second factor) and stores them together
// Per output this is 1 + (in/out column ratio) + halo 1-D interpolants
// instead of 5.
// Output rows per tile: 32 when the rows are magnified (the per-tile setup
// and window decode spread over more outputs), 16 when they are reduced (the
// window then has up to twice the tile's rows, and taller tiles would leave
// fewer CTAs per SM).
constexpr int RS_TR_UP = 32;
constexpr int RS_TR_DOWN = 16;
constexpr int RS_TC = 128;
constexpr int RS_WC = 2 * RS_TC + 8;  // window columns (>= 2 (RS_TC - 1) + 5)
constexpr int RS_THREADS = 256;

template <int BMODE, class TIn, class TOut>
__global__ void __launch_bounds__(RS_THREADS) resample_tiled_kernel(ResampleArgs a, float eps,
                                                                   float beta) {
  extern __shared__ float rs_smem[];
  float(*win)[RS_WC] = reinterpret_cast<float(*)[RS_WC]>(rs_smem);               // a.win_rows
  float(*z)[RS_WC] = reinterpret_cast<float(*)[RS_WC]>(rs_smem + a.win_rows * RS_WC);  // tile_rows
  __shared__ int col_j[RS_TC];
  __shared__ float col_t[RS_TC];
  __shared__ int row_i[RS_TR_UP];
  __shared__ float row_t[RS_TR_UP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * RS_TC;
  const int tr = a.tile_rows;
  const int64_t r0 = (int64_t)blockIdx.y * tr;
  const int64_t plane = blockIdx.z;
  const int nc = (int)(a.m_out - c0 < RS_TC ? a.m_out - c0 : RS_TC);
  const int nr = (int)(a.n_out - r0 < tr ? a.n_out - r0 : tr);
  // Every output column's and row's cell index (absolute) and offset; the
  // first and last of them bound the input window.
  if (tid < nc) {
    int64_t j;
    float t;
    grid_pos(c0 + tid, a.m, a.m_out, a.div_x, j, t);
    col_j[tid] = (int)j;
    col_t[tid] = t;
  }
  if (tid >= RS_TC && tid - RS_TC < nr) {
    int64_t i;
    float t;
    grid_pos(r0 + tid - RS_TC, a.n, a.n_out, a.div_y, i, t);
    row_i[tid - RS_TC] = (int)i;
    row_t[tid - RS_TC] = t;
  }
  __syncthreads();
  const int64_t kfirst = (int64_t)col_j[0] - 1, ifirst = (int64_t)row_i[0] - 1;
  const int wc = col_j[nc - 1] + 2 - (int)kfirst + 1;  // <= RS_WC (host checks the x scale)
  const int wr = row_i[nr - 1] + 2 - (int)ifirst + 1;  // <= a.win_rows (host sizes it)
  // stage 0: decoded, clamped input window.  A thread takes 2 x 2 elements
  // at a time (rows 8 apart, columns 32 apart) and issues their four loads
  // before it converts any of them, so that the loads overlap.
  constexpr int WR = RS_THREADS / 32;  // rows one pass of the warps covers
  const int64_t pbase = plane * a.in_sc;
  for (int rr0 = warp; rr0 < wr; rr0 += 2 * WR) {
    int64_t rbase[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      int64_t row = ifirst + rr0 + u * WR;
      row = row < 0 ? 0 : (row > a.n - 1 ? a.n - 1 : row);
      rbase[u] = pbase + row * a.in_sh;
    }
    for (int k0 = lane; k0 < wc; k0 += 64) {
      uint32_t b[2][2];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int k = k0 + 32 * v;
          int64_t col = kfirst + k;
          col = col < 0 ? 0 : (col > a.m - 1 ? a.m - 1 : col);
          b[u][v] = (rr0 + u * WR < wr && k < wc)
                        ? rs_load_bits<TIn>(a.in, rbase[u] + col * a.in_sw, a.in_dtype)
                        : 0u;
        }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v)
          if (rr0 + u * WR < wr && k0 + 32 * v < wc)
            win[rr0 + u * WR][k0 + 32 * v] = rs_value<TIn>(b[u][v], a.in_dtype);
    }
  }
  __syncthreads();
  // pass 1: column interpolants
  for (int r = warp; r < nr; r += RS_THREADS / 32) {
    const float* w0 = win[row_i[r] - 1 - (int)ifirst];
    if (a.n > 1) {
      const float ty = row_t[r];
      const float C0 = (2.f - ty) * (1.f / 3.f), h = 0.5f * fmaf(ty, ty, -ty);
      // window columns k and k + 32 in the two lanes (a column past the
      // window repeats k and is not stored)
      for (int k = lane; k < wc; k += 64) {
        const bool two = k + 32 < wc;
        const int kb = two ? k + 32 : k;
        const f2 zz = weno1d_at2<BMODE>(
            make_float2(w0[k], w0[kb]), make_float2(w0[k + RS_WC], w0[kb + RS_WC]),
            make_float2(w0[k + 2 * RS_WC], w0[kb + 2 * RS_WC]),
            make_float2(w0[k + 3 * RS_WC], w0[kb + 3 * RS_WC]), pk_bc(ty), pk_bc(C0), pk_bc(h), eps,
            beta);
        z[r][k] = zz.x;
        if (two) z[r][k + 32] = zz.y;
      }
    } else {
      for (int k = lane; k < wc; k += 32) z[r][k] = w0[k + RS_WC];
    }
  }
  __syncthreads();
  // pass 2: four consecutive outputs per thread; the column positions and
  // their constants are the same for every row of the tile
  const int c = lane * 4;
  if (c >= nc) return;
  const int cn = nc - c < 4 ? nc - c : 4;
  int kq[4];
  float tq[4], cq[4], hq[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int cc = c + (q < cn ? q : 0);  // columns past the tile repeat the first (not stored)
    kq[q] = col_j[cc] - 1 - (int)kfirst;
    tq[q] = col_t[cc];
    cq[q] = (2.f - tq[q]) * (1.f / 3.f);
    hq[q] = 0.5f * fmaf(tq[q], tq[q], -tq[q]);
  }
  const bool interp_x = a.m > 1;
  int64_t o = plane * a.out_sc + (r0 + warp) * a.out_sh + (c0 + c) * a.out_sw;
  const int64_t o_step = (RS_THREADS / 32) * a.out_sh;
  for (int r = warp; r < nr; r += RS_THREADS / 32, o += o_step) {
    float u[4];
    const float* zr = z[r];
    // outputs q and q + 1 in the two lanes
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      const float* za = zr + kq[q];
      const float* zb = zr + kq[q + 1];
      if (interp_x) {
        const f2 uu = weno1d_at2<BMODE>(
            make_float2(za[0], zb[0]), make_float2(za[1], zb[1]), make_float2(za[2], zb[2]),
            make_float2(za[3], zb[3]), make_float2(tq[q], tq[q + 1]),
            make_float2(cq[q], cq[q + 1]), make_float2(hq[q], hq[q + 1]), eps, beta);
        u[q] = uu.x;
        u[q + 1] = uu.y;
      } else {
        u[q] = za[1];
        u[q + 1] = zb[1];
      }
    }
    if (a.out_vec4 && cn == 4) {
      rs_store4<TOut>(a.out, o, u, a.out_dtype, a.clamp_float);
    } else {
      for (int q = 0; q < cn; ++q)
        rs_store<TOut>(a.out, o + q * a.out_sw, u[q], a.out_dtype, a.clamp_float);
    }
  }
}

template <int BMODE, class TIn, class TOut>
cudaError_t launch_tiled(const ResampleArgs& a, float eps, float beta, cudaStream_t stream) {
  const size_t smem = (size_t)(a.win_rows + a.tile_rows) * RS_WC * sizeof(float);
  auto kern = resample_tiled_kernel<BMODE, TIn, TOut>;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((a.m_out + RS_TC - 1) / RS_TC),
                  (unsigned)((a.n_out + a.tile_rows - 1) / a.tile_rows), (unsigned)a.planes);
  kern<<<grid, RS_THREADS, smem, stream>>>(a, eps, beta);
  return cudaGetLastError();
}

template <class TIn, class TOut>
cudaError_t launch_tiled_beta(const ResampleArgs& a, float eps, float beta, int bmode,
                              cudaStream_t stream) {
  switch (bmode) {
    case B2: return launch_tiled<B2, TIn, TOut>(a, eps, beta, stream);
    case B2R: return launch_tiled<B2R, TIn, TOut>(a, eps, beta, stream);
    case B0: return launch_tiled<B0, TIn, TOut>(a, eps, beta, stream);
    default: return launch_tiled<BGEN, TIn, TOut>(a, eps, beta, stream);
  }
}

}  // namespace

static AxisDiv axis_div(int64_t n, int64_t n_out) {
  AxisDiv d{1u, 0, 0, 0, 0.f};
  if (n <= 1 || n_out <= 1) return d;
  const uint64_t den = (uint64_t)(n_out - 1);
  d.inv = (float)(1.0 / (double)den);
  // the largest numerator is (n_out - 1)(n - 1)
  if (den >= (1ull << 32) || (uint64_t)(n - 1) >= (1ull << 32) ||
      den * (uint64_t)(n - 1) >= (1ull << 32))
    return d;
  int l = 0;
  while ((1ull << l) < den) ++l;
  d.mag = (uint32_t)(((1ull << 32) * ((1ull << l) - den)) / den + 1);
  d.sh1 = l < 1 ? l : 1;
  d.sh2 = l > 1 ? l - 1 : 0;
  d.fast = 1;
  return d;
}

cudaError_t launch_resample(const ResampleArgs& a_in, float eps, float beta, int bmode,
                            cudaStream_t stream) {
  ResampleArgs a = a_in;
  a.div_y = axis_div(a.n, a.n_out);
  a.div_x = axis_div(a.m, a.m_out);
  // the tiled form reads at most RS_WC window columns and sizes its window
  // rows from the y ratio: spacing ratios (n - 1)/(n_out - 1) <= 2 per axis
  const bool tiled = (a.m_out == 1 || 2 * (a.m_out - 1) >= (a.m - 1)) &&
                     (a.n_out == 1 || 2 * (a.n_out - 1) >= (a.n - 1));
  if (tiled) {
    a.tile_rows = a.n_out >= a.n ? RS_TR_UP : RS_TR_DOWN;
    a.win_rows =
        (a.n_out > 1 ? (int)((int64_t)(a.tile_rows - 1) * (a.n - 1) / (a.n_out - 1)) : 0) + 5;
    const int i = a.in_dtype, o = a.out_dtype;
    if (i == DT_U8 && o == DT_U8) return launch_tiled_beta<uint8_t, uint8_t>(a, eps, beta, bmode, stream);
    if (i == DT_F16 && o == DT_F16) return launch_tiled_beta<__half, __half>(a, eps, beta, bmode, stream);
    if (i == DT_BF16 && o == DT_BF16)
      return launch_tiled_beta<__nv_bfloat16, __nv_bfloat16>(a, eps, beta, bmode, stream);
    if (i == DT_F32 && o == DT_F32) return launch_tiled_beta<float, float>(a, eps, beta, bmode, stream);
    if (i == DT_U8 && o == DT_F32) return launch_tiled_beta<uint8_t, float>(a, eps, beta, bmode, stream);
    if (i == DT_F32 && o == DT_U8) return launch_tiled_beta<float, uint8_t>(a, eps, beta, bmode, stream);
    return launch_tiled_beta<Dyn, Dyn>(a, eps, beta, bmode, stream);
  }
  const dim3 block(32, 8);
  const dim3 grid((unsigned)((a.m_out + 31) / 32), (unsigned)((a.n_out + 7) / 8),
                  (unsigned)a.planes);
  switch (bmode) {
    case B2: resample_kernel<B2><<<grid, block, 0, stream>>>(a, eps, beta); break;
    case B2R: resample_kernel<B2R><<<grid, block, 0, stream>>>(a, eps, beta); break;
    case B0: resample_kernel<B0><<<grid, block, 0, stream>>>(a, eps, beta); break;
    default: resample_kernel<BGEN><<<grid, block, 0, stream>>>(a, eps, beta); break;
  }
  return cudaGetLastError();
}

}  // namespace wdweno
