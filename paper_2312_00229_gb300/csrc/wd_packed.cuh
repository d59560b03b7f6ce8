// Packed two-lane FP32 helpers (Blackwell fma / add / sub / mul .f32x2): one
// instruction for two independent values, each lane rounded exactly as the
// scalar operation (round to nearest even), so a computation written lane by
// lane in the scalar order gives the scalar results bit for bit.
#pragma once

#include "wd_common.cuh"

namespace wdweno {

using f2 = float2;
__device__ __forceinline__ f2 pk_bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ f2 pk_add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 pk_mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 pk_fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 pk_sub(f2 a, f2 b) {
  f2 r;
  asm("{.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ f2 pk_rcp(f2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }

// blend4 of wd_common.cuh with the per-direction steps of the weights (the
// squares, reciprocals and ratios) on the direction pairs (0, 1) and (2, 3);
// the sums stay scalar, in the scalar order, so the result is bit for bit
// that of blend4.
template <int BMODE>
__device__ __forceinline__ float blend4_pk(float D0, float D1, float D2, float D3, float M01,
                                           float M23, float s0, float s1, float s2, float s3,
                                           float beta) {
  if (BMODE == B2R) {
    const f2 a01 = pk_rcp(pk_mul(make_float2(D0, D1), make_float2(D0, D1)));
    const f2 a23 = pk_rcp(pk_mul(make_float2(D2, D3), make_float2(D2, D3)));
    const float den = (a01.x + a01.y) + (a23.x + a23.y);
    return combine(a01.x, a01.y, a23.x, a23.y, M01, M23, s0, s1, s2, s3, rcp_approx(den + den));
  } else if (BMODE == B2) {
    const f2 dmin = pk_bc(fminf(fminf(D0, D1), fminf(D2, D3)));
    const f2 r01 = pk_mul(dmin, pk_rcp(make_float2(D0, D1)));
    const f2 r23 = pk_mul(dmin, pk_rcp(make_float2(D2, D3)));
    const f2 a01 = pk_mul(r01, r01), a23 = pk_mul(r23, r23);
    const float den = (a01.x + a01.y) + (a23.x + a23.y);
    return combine(a01.x, a01.y, a23.x, a23.y, M01, M23, s0, s1, s2, s3, rcp_approx(den + den));
  } else {
    return blend4<BMODE>(D0, D1, D2, D3, M01, M23, s0, s1, s2, s3, beta);
  }
}

}  // namespace wdweno
