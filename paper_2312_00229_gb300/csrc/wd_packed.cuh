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

}  // namespace wdweno
