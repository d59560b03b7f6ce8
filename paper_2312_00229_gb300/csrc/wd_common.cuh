// Device helpers shared by the WD WENO kernels (arXiv 2312.00229, Sec. 3).
//
// Notation (per channel): the coarse image A is n x m; the zoomed grid has
// fine index (P, Q).  Fine (2a, 2b) is the input sample A(a, b); fine
// (2a+1, 2b+1) is the "x" point X(a, b) of phase 1; fine (2a, 2b+1) is the
// "+" point E(a, b) and fine (2a+1, 2b) the "+" point S(a, b) of phase 2.
// Coarse cell (a, b) therefore owns the output quad
//     [ A(a,b)  E(a,b) ]
//     [ S(a,b)  X(a,b) ].
// Every directional interpolant uses three nodes N0, N1, N2 at -1, +1, +3
// fine steps (Eq. p); with g = N1 - N0 and s = N0 - 2 N1 + N2:
//     p  = (N0 + N1) / 2 - s / 8
//     SI = g^2 + kappa^2 s^2            (Eq. 2Dsmoothness, kappa^2 = 13/12
//                                        for the normalized length scale)
// Opposite directions share the pair (N0, N1), so they share g and N0 + N1
// and differ only in s.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wdweno {

enum DType { DT_U8 = 0, DT_F16 = 1, DT_BF16 = 2, DT_F32 = 3 };

// How Eq. (alpha) is evaluated.
//   B2  : beta == 2, alpha = (D_min / D)^2 (D already holds eps_h).
//   BGEN: any beta > 0, alpha = (D_min / D)^beta (scale-free).
//   B0  : beta == 0, all weights equal.
//   B2R : beta == 2, alpha = 1 / D^2 as written; chosen by the host only
//         where the storage type bounds the data so that every weight, their
//         sum and the blend numerator stay inside the normal FP32 range.
enum BetaMode { B2 = 0, BGEN = 1, B0 = 2, B2R = 3 };

// Constants of the method folded for the kernels.  eps_h is spread over the
// five smoothness indicators that form each D (Eqs. 2DsmoothnessFinal and
// tezine): every SI carries eps_h / (1 + 4 w), so their weighted sum carries
// exactly eps_h.
struct MethodConsts {
  float kappa1;  // sqrt of the s^2 coefficient in phase-1 SIs
  float kappa2;  // same for phase 2 (13/12 normalized, 25/12 literal)
  float eps1;    // eps_h / (1 + 4 w), phase 1
  float eps2;    // phase 2 (divided by sqrt(2) in the literal mode, whose
                 // overall sqrt(2) factor cancels in the weights)
  float w;       // neighbour weight of D: nbr_c h^2
  float beta;
  int clamp_float;
};

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---------------------------------------------------------------------------
// Storage decode / encode
// ---------------------------------------------------------------------------
__device__ __forceinline__ float load_elem(const void* base, int64_t idx, int dt) {
  switch (dt) {
    case DT_U8:
      return (float)__ldg(static_cast<const uint8_t*>(base) + idx) * (1.0f / 255.0f);
    case DT_F16:
      return __half2float(__ldg(static_cast<const __half*>(base) + idx));
    case DT_BF16:
      return __bfloat162float(__ldg(static_cast<const __nv_bfloat16*>(base) + idx));
    default:
      return __ldg(static_cast<const float*>(base) + idx);
  }
}

// The storage bits of one element, zero-extended, and the value they hold.
// A prefetched element is kept in its storage form until its value is used:
// the conversion is then not where the load is issued, so nothing waits for
// the load there.
__device__ __forceinline__ uint32_t load_elem_bits(const void* base, int64_t idx, int dt) {
  switch (dt) {
    case DT_U8:
      return __ldg(static_cast<const uint8_t*>(base) + idx);
    case DT_F16:
    case DT_BF16:
      return __ldg(static_cast<const unsigned short*>(base) + idx);
    default:
      return __float_as_uint(__ldg(static_cast<const float*>(base) + idx));
  }
}

__device__ __forceinline__ float elem_bits_value(uint32_t b, int dt) {
  switch (dt) {
    case DT_U8:
      return (float)b * (1.0f / 255.0f);
    case DT_F16:
      return __half2float(__ushort_as_half((unsigned short)b));
    case DT_BF16:
      return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
    default:
      return __uint_as_float(b);
  }
}

// saturate, scale, round half to even: adding 1.5 * 2^23 inside the FMA
// leaves a float whose unit in the last place is 1, so its low mantissa byte
// is the code, from one rounding of the exact product.
__device__ __forceinline__ uint32_t encode_u8_bits(float v) {
  return __float_as_uint(fmaf(__saturatef(v), 255.0f, 12582912.0f));
}

__device__ __forceinline__ uint32_t encode_u8(float v) { return encode_u8_bits(v) & 0xFFu; }

__device__ __forceinline__ float clamp_opt(float v, int clampf) {
  return clampf ? __saturatef(v) : v;
}

__device__ __forceinline__ void store_elem(void* base, int64_t idx, float v, int dt, int clampf) {
  switch (dt) {
    case DT_U8:
      static_cast<uint8_t*>(base)[idx] = (uint8_t)encode_u8(v);
      break;
    case DT_F16:
      static_cast<__half*>(base)[idx] = __float2half_rn(clamp_opt(v, clampf));
      break;
    case DT_BF16:
      static_cast<__nv_bfloat16*>(base)[idx] = __float2bfloat16_rn(clamp_opt(v, clampf));
      break;
    default:
      static_cast<float*>(base)[idx] = clamp_opt(v, clampf);
      break;
  }
}

// Four consecutive elements at `idx` (idx aligned to 4 elements, unit
// stride) written with one vector store.
__device__ __forceinline__ void store4_vec(void* base, int64_t idx, float v0, float v1, float v2,
                                           float v3, int dt, int clampf) {
  switch (dt) {
    case DT_U8: {
      const uint32_t lo = __byte_perm(encode_u8_bits(v0), encode_u8_bits(v1), 0x0040);
      const uint32_t hi = __byte_perm(encode_u8_bits(v2), encode_u8_bits(v3), 0x0040);
      const uint32_t packed = __byte_perm(lo, hi, 0x5410);
      *reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(base) + idx) = packed;
      break;
    }
    case DT_F16: {
      __half2 lo = __floats2half2_rn(clamp_opt(v0, clampf), clamp_opt(v1, clampf));
      __half2 hi = __floats2half2_rn(clamp_opt(v2, clampf), clamp_opt(v3, clampf));
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&lo);
      u.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(static_cast<__half*>(base) + idx) = u;
      break;
    }
    case DT_BF16: {
      __nv_bfloat162 lo = __floats2bfloat162_rn(clamp_opt(v0, clampf), clamp_opt(v1, clampf));
      __nv_bfloat162 hi = __floats2bfloat162_rn(clamp_opt(v2, clampf), clamp_opt(v3, clampf));
      uint2 u;
      u.x = *reinterpret_cast<uint32_t*>(&lo);
      u.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + idx) = u;
      break;
    }
    default: {
      float4 f = make_float4(clamp_opt(v0, clampf), clamp_opt(v1, clampf), clamp_opt(v2, clampf),
                             clamp_opt(v3, clampf));
      *reinterpret_cast<float4*>(static_cast<float*>(base) + idx) = f;
      break;
    }
  }
}

// Two consecutive elements at `idx` (idx aligned to 2 elements, unit
// stride) written with one vector store.
__device__ __forceinline__ void store2_vec(void* base, int64_t idx, float v0, float v1, int dt,
                                           int clampf) {
  switch (dt) {
    case DT_U8: {
      const uint16_t packed =
          (uint16_t)__byte_perm(encode_u8_bits(v0), encode_u8_bits(v1), 0x0040);
      *reinterpret_cast<uint16_t*>(static_cast<uint8_t*>(base) + idx) = packed;
      break;
    }
    case DT_F16:
      *reinterpret_cast<__half2*>(static_cast<__half*>(base) + idx) =
          __floats2half2_rn(clamp_opt(v0, clampf), clamp_opt(v1, clampf));
      break;
    case DT_BF16:
      *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(base) + idx) =
          __floats2bfloat162_rn(clamp_opt(v0, clampf), clamp_opt(v1, clampf));
      break;
    default:
      *reinterpret_cast<float2*>(static_cast<float*>(base) + idx) =
          make_float2(clamp_opt(v0, clampf), clamp_opt(v1, clampf));
      break;
  }
}

// Typed variants (storage type fixed at compile time).
template <class T> struct DTypeOf;
template <> struct DTypeOf<uint8_t> { static constexpr int value = DT_U8; };
template <> struct DTypeOf<__half> { static constexpr int value = DT_F16; };
template <> struct DTypeOf<__nv_bfloat16> { static constexpr int value = DT_BF16; };
template <> struct DTypeOf<float> { static constexpr int value = DT_F32; };

template <class T>
__device__ __forceinline__ void store_typed(void* base, int64_t idx, float v, int clampf) {
  store_elem(base, idx, v, DTypeOf<T>::value, clampf);  // the switch folds away
}

template <class T>
__device__ __forceinline__ void store2_typed(void* base, int64_t idx, float v0, float v1,
                                             int clampf) {
  store2_vec(base, idx, v0, v1, DTypeOf<T>::value, clampf);
}

template <class T>
__device__ __forceinline__ void store4_typed(void* base, int64_t idx, float v0, float v1,
                                             float v2, float v3, int clampf) {
  store4_vec(base, idx, v0, v1, v2, v3, DTypeOf<T>::value, clampf);
}

// ---------------------------------------------------------------------------
// Directional blend of one new point (Eqs. alpha, IzrazOmega2d,
// 2dKombinacija and their phase-2 counterparts).
//   D0..D3 : neighbour-smoothed indicators of the four directions, already
//            including eps_h; directions (0,1) and (2,3) are opposite pairs
//   M01    : N0 + N1 of the pair (0,1);  M23 likewise
//   s0..s3 : second differences of the four stencils
// Returns sum_k omega_k p_k with omega_k = alpha_k / sum alpha, where
// p_k = M / 2 - s_k / 8 and alpha_k = 0.5 / D_k^beta (the 0.5 cancels).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float combine(float a0, float a1, float a2, float a3, float M01,
                                         float M23, float s0, float s1, float s2, float s3,
                                         float inv_den) {
  float a01 = a0 + a1;
  float a23 = a2 + a3;
  float m = a01 * M01;
  m = fmaf(a23, M23, m);
  float ws = a0 * s0;
  ws = fmaf(a1, s1, ws);
  ws = fmaf(a2, s2, ws);
  ws = fmaf(a3, s3, ws);
  float num = fmaf(ws, -0.25f, m);  // 2 * sum alpha p
  return num * inv_den;             // inv_den = 1 / (2 sum alpha)
}

__device__ __forceinline__ float blend_scale_free(float D0, float D1, float D2, float D3, float M01,
                                                  float M23, float s0, float s1, float s2,
                                                  float s3, float beta) {
  float dmin = fminf(fminf(D0, D1), fminf(D2, D3));
  float r0 = dmin * rcp_approx(D0), r1 = dmin * rcp_approx(D1);
  float r2 = dmin * rcp_approx(D2), r3 = dmin * rcp_approx(D3);
  float a0, a1, a2, a3;
  if (beta == 2.0f) {
    a0 = r0 * r0; a1 = r1 * r1; a2 = r2 * r2; a3 = r3 * r3;
  } else if (beta == 1.0f) {
    a0 = r0; a1 = r1; a2 = r2; a3 = r3;
  } else {
    a0 = ex2_approx(beta * lg2_approx(r0));
    a1 = ex2_approx(beta * lg2_approx(r1));
    a2 = ex2_approx(beta * lg2_approx(r2));
    a3 = ex2_approx(beta * lg2_approx(r3));
  }
  float den = (a0 + a1) + (a2 + a3);
  return combine(a0, a1, a2, a3, M01, M23, s0, s1, s2, s3, rcp_approx(den + den));
}

template <int BMODE>
__device__ __forceinline__ float blend4(float D0, float D1, float D2, float D3, float M01, float M23,
                                        float s0, float s1, float s2, float s3, float beta) {
  if (BMODE == B0) {
    return combine(1.f, 1.f, 1.f, 1.f, M01, M23, s0, s1, s2, s3, 0.125f);
  } else if (BMODE == B2) {
    // alpha_k = (D_min / D_k)^2: the same weights as 1 / D_k^2 up to a common
    // factor, in range for any data magnitude, and without a branch
    return blend_scale_free(D0, D1, D2, D3, M01, M23, s0, s1, s2, s3, 2.0f);
  } else if (BMODE == B2R) {
    const float a0 = rcp_approx(D0 * D0), a1 = rcp_approx(D1 * D1);
    const float a2 = rcp_approx(D2 * D2), a3 = rcp_approx(D3 * D3);
    const float den = (a0 + a1) + (a2 + a3);
    return combine(a0, a1, a2, a3, M01, M23, s0, s1, s2, s3, rcp_approx(den + den));
  } else {
    return blend_scale_free(D0, D1, D2, D3, M01, M23, s0, s1, s2, s3, beta);
  }
}

}  // namespace wdweno
