// Adjoint of the deskew and backward pass of the z-MIP.
//
// Both are gathers over the transpose of the interpolation map: raw sample
// (n, k, x) collects every output column j of row k whose lower plane n0(j,k)
// is n (weight 1 - w) or n - 1 (weight w), in ascending j.  The weights are
// computed with the forward kernels' own split-table formula, so the adjoint
// is the exact transpose of the map the forward kernels apply.  No atomics:
// results are bitwise reproducible.
#include <cmath>

#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kThreadsX = 32;
constexpr int kThreadsY = 8;

// Search window of columns j whose tent can reach plane n in row k.
__device__ __forceinline__ void j_window(const PlanView& v, Split b, int n, int& jlo, int& jhi) {
  const float bk = (float)b.i + b.f;
  const float lo = (float)v.J0 + ((float)n - 1.0f + bk) * v.rinv;
  const float hi = (float)v.J0 + ((float)n + 1.0f + bk) * v.rinv;
  jlo = max(0, (int)floorf(lo) - 2);
  jhi = min(v.ny - 1, (int)ceilf(hi) + 2);
}

template <typename T, typename Acc, int VEC, bool MIPBWD>
__global__ void __launch_bounds__(kThreadsX* kThreadsY)
k_gather_t(PlanView v, const T* __restrict__ src, const int32_t* __restrict__ argz,
           T* __restrict__ dst, int xtiles, int vec_ok) {
  const int k = blockIdx.x / xtiles;
  const int xt = blockIdx.x - k * xtiles;
  const int x0 = (xt * kThreadsX + threadIdx.x) * VEC;
  const int n = blockIdx.y * kThreadsY + threadIdx.y;
  if (x0 >= v.nx || n >= v.nscan) return;
  const int lim = v.nx - x0;
  const bool vec = vec_ok && lim >= VEC;
  const Split b = v.B[k];
  int jlo, jhi;
  j_window(v, b, n, jlo, jhi);

  Acc acc[VEC];
#pragma unroll
  for (int i = 0; i < VEC; ++i) acc[i] = Acc(0);

#pragma unroll 1
  for (int j = jlo; j <= jhi; ++j) {
    int n0;
    Acc w;
    plane_weight_t<Acc>(v.A[j], b, v.linear, n0, w);
    Acc wt;
    if (n0 == n)
      wt = Acc(1) - w;
    else if (n0 + 1 == n)
      wt = w;
    else
      continue;
    if (wt == Acc(0)) continue;
    Acc val[VEC];
    if constexpr (MIPBWD) {
      // g_zmip[j][x] where argz[j][x] == k, else 0
      const size_t off = (size_t)j * v.nx + x0;
      load_vec<T, VEC, Acc>(src + off, vec, lim, val);
      if (vec) {
        const int4 a4 = __ldg(reinterpret_cast<const int4*>(argz + off));
        const int* ai = reinterpret_cast<const int*>(&a4);
#pragma unroll
        for (int i = 0; i < VEC; ++i) val[i] = ai[i] == k ? val[i] : Acc(0);
      } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) val[i] = (i < lim && __ldg(argz + off + i) == k) ? val[i] : Acc(0);
      }
    } else {
      load_vec<T, VEC, Acc>(src + ((size_t)k * v.ny + j) * v.nx + x0, vec, lim, val);
    }
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc[i] = fma(wt, val[i], acc[i]);
  }

  T* op = dst + ((size_t)n * v.nrows + k) * v.ncols + x0;
  if (vec) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(op) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    } else {
      *reinterpret_cast<double2*>(op) = make_double2(acc[0], acc[1]);
    }
  } else {
    for (int i = 0; i < VEC && i < lim; ++i) op[i] = (T)acc[i];
  }
}

template <typename T, typename Acc, int VEC, bool MIPBWD>
opm_status run(const opm_plan* p, const T* src, const int32_t* argz, T* dst, cudaStream_t s) {
  const PlanView& v = p->view;
  const int xtiles = (v.nx + kThreadsX * VEC - 1) / (kThreadsX * VEC);
  const long long gx = (long long)xtiles * v.nz;
  const long long gy = (v.nscan + kThreadsY - 1) / kThreadsY;
  if (gx > 0x7fffffffLL || gy > 65535)
    return fail(OPM_ERR_UNSUPPORTED, "adjoint grid exceeds launch limits");
  int vec_ok = (v.nx % VEC == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
  if (MIPBWD) vec_ok = vec_ok && ((uintptr_t)argz % 16 == 0);
  dim3 block(kThreadsX, kThreadsY);
  dim3 grid((unsigned)gx, (unsigned)gy);
  k_gather_t<T, Acc, VEC, MIPBWD><<<grid, block, 0, s>>>(v, src, argz, dst, xtiles, vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch adjoint gather");
}

}  // namespace

opm_status launch_adjoint(const opm_plan* p, const void* vol, void* raw_out, opm_dtype t,
                          cudaStream_t s) {
  if (t == OPM_F32)
    return run<float, float, 4, false>(p, static_cast<const float*>(vol), nullptr,
                                       static_cast<float*>(raw_out), s);
  if (t == OPM_F64)
    return run<double, double, 2, false>(p, static_cast<const double*>(vol), nullptr,
                                         static_cast<double*>(raw_out), s);
  return fail(OPM_ERR_UNSUPPORTED, "adjoint dtype");
}

opm_status launch_mip_backward(const opm_plan* p, const float* g, const int32_t* argz,
                               float* g_raw, cudaStream_t s) {
  return run<float, float, 4, true>(p, g, argz, g_raw, s);
}

}  // namespace opm
