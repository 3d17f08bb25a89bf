// Device helpers shared by the kernels: typed vector loads/stores and the
// FP64 variant of the plane/weight split.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "opm_internal.h"

namespace opm {

// Same lower plane as plane_weight(), with the weight carried in double so
// that the FP64 forward and adjoint kernels share bit-identical weights.
__device__ __forceinline__ void plane_weight_f64(Split a, Split b, int linear,
                                                 int& n0, double& w) {
  const float df = a.f - b.f;  // its sign equals the sign of the exact difference
  const int neg = df < 0.0f;
  const double d = (double)a.f - (double)b.f;
  n0 = a.i - b.i - neg;
  w = linear ? (neg ? d + 1.0 : d) : 0.0;
}

template <typename Acc>
__device__ __forceinline__ void plane_weight_t(Split a, Split b, int linear, int& n0, Acc& w) {
  if constexpr (std::is_same<Acc, double>::value) {
    plane_weight_f64(a, b, linear, n0, w);
  } else {
    plane_weight(a, b, linear, n0, w);
  }
}

template <typename T>
__device__ __forceinline__ float to_f32(T v) {
  return static_cast<float>(v);
}

// Load VEC consecutive elements starting at p as accumulator values.  `vec`
// selects one aligned vector load; otherwise elements are loaded one by one
// and those at or beyond `lim` read as zero.
template <typename T, int VEC, typename Acc>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, bool vec, int lim, Acc (&out)[VEC]) {
  static_assert(sizeof(T) * VEC == 16, "16-byte vectors");
  if (vec) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
    for (int i = 0; i < VEC; ++i) out[i] = static_cast<Acc>(e[i]);
  } else {
#pragma unroll
    for (int i = 0; i < VEC; ++i) out[i] = i < lim ? static_cast<Acc>(__ldg(p + i)) : Acc(0);
  }
}

__device__ __forceinline__ uint16_t to_u16_rn(float v) {
  // round half to even, clamp to [0, 65535]; NaN maps to 0
  const float c = fminf(fmaxf(v, 0.0f), 65535.0f);
  return static_cast<uint16_t>(__float2uint_rn(c));
}

__device__ __forceinline__ void st_cs_v4(float* p, float a, float b, float c, float d) {
  asm volatile("st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

__device__ __forceinline__ void st_cs_v4u(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.global.cs.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

}  // namespace opm
