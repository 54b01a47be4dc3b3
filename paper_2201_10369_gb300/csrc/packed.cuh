// packed.cuh -- two FP32 values in one 64-bit register (low half first) and
// the sm_100-family instructions that work on such pairs.  Each half of
// fma.rn.f32x2 / mul.rn.f32x2 / sub.rn.f32x2 is the IEEE operation with one
// rounding -- exactly fmaf, __fmul_rn, __fsub_rn -- so code written with
// them gives the same bits as the scalar code in half the instructions.
// cvt.rn.{bf16x2,f16x2}.f32 round two FP32 values as two separate RN
// conversions would and pack them into one 32-bit word.
#pragma once

#include <stdint.h>

namespace wino {

__device__ __forceinline__ unsigned long long pack_dup(float a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// RN to BF16 (fp16 = false) or FP16 (fp16 = true) of both halves of v; the
// low half's result in bits 0-15, the high half's in bits 16-31.
__device__ __forceinline__ uint32_t cvt16x2(unsigned long long v, bool fp16) {
  const float2 p = unpack2(v);
  uint32_t r;
  if (fp16)
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(p.y), "f"(p.x));
  else
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(p.y), "f"(p.x));
  return r;
}
// The two 16-bit values of w widened back to FP32 (exact), packed as a pair.
__device__ __forceinline__ unsigned long long widen16x2(uint32_t w, bool fp16) {
  if (fp16) {
    float lo, hi;
    asm("{\n .reg .f16 a, b;\n mov.b32 {a, b}, %2;\n cvt.f32.f16 %0, a;\n cvt.f32.f16 %1, b;\n}"
        : "=f"(lo), "=f"(hi)
        : "r"(w));
    return pack2(lo, hi);
  }
  return pack2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

}  // namespace wino
