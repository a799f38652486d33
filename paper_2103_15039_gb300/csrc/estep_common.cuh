// Device helpers shared by the E-step kernels (FP32 and tensor-core variants).
#pragma once

#include <stdint.h>

namespace lsg {

__device__ __forceinline__ float ex2_neg(float x) {  // 2^-x (the sign folds into MUFU.EX2)
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));
  return y;
}

__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// Cursor over a CTA's units: the source block of unit u, advancing monotonically
// (walks unit_off forward).
struct Cursor {
  int b;
  __device__ __forceinline__ int advance(const int* unit_off, long long u) {
    while (u >= unit_off[b + 1]) ++b;
    return b;
  }
};

}  // namespace lsg
