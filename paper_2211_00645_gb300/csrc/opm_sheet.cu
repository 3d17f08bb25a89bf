// The paper's own live view: every raw frame n remapped into a larger image,
// shifted along the camera-row axis by its accumulated lateral offset n * s
// rows (Eq. 1 with s = step cos(alpha) / pixel; Fig. 2c), then the
// brightest value over the frames at each pixel (Fig. 2d).  A reduced shear
// factor followed by a 1-D affine warp of the projection changes the viewing
// angle (shear-warp, Fig. 3).  Sub-row shifts interpolate linearly between
// the two neighbouring camera rows (zero outside the frame).
#include <algorithm>
#include <cmath>

#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kShX = 32;    // lanes along x
constexpr int kShY = 8;     // output rows per CTA (one per warp)
constexpr int kShVec = 4;   // columns x per lane

struct ShiftSplit {
  int i;    // floor(n * s)
  float f;  // n * s - floor(n * s), from the FP64 product
};

template <typename T>
__device__ __forceinline__ void load4(const T* __restrict__ p, bool vec, int lim, float (&out)[kShVec]) {
  if constexpr (std::is_same<T, uint16_t>::value) {
    if (vec) {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      out[0] = (float)(u.x & 0xFFFFu);
      out[1] = (float)(u.x >> 16);
      out[2] = (float)(u.y & 0xFFFFu);
      out[3] = (float)(u.y >> 16);
      return;
    }
  } else {
    if (vec) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(p));
      out[0] = f.x;
      out[1] = f.y;
      out[2] = f.z;
      out[3] = f.w;
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < kShVec; ++c) out[c] = c < lim ? (float)__ldg(p + c) : 0.0f;
}

template <typename T>
__global__ void __launch_bounds__(kShX* kShY)
k_sheet_project(const T* __restrict__ raw, int nscan, int nrows, int ncols, double shear, float* __restrict__ out,
                int H, int vec_ok) {
  extern __shared__ ShiftSplit shift[];
  for (int n = threadIdx.y * kShX + threadIdx.x; n < nscan; n += kShX * kShY) {
    const double sh = (double)n * shear;
    const double fl = floor(sh);
    shift[n] = ShiftSplit{(int)fl, (float)(sh - fl)};
  }
  __syncthreads();
  const int Y = blockIdx.y * kShY + threadIdx.y;
  const int x = (blockIdx.x * kShX + threadIdx.x) * kShVec;
  if (Y >= H || x >= ncols) return;
  const int lim = ncols - x;
  const bool vec = vec_ok && lim >= kShVec;
  const size_t plane = (size_t)nrows * ncols;
  float m[kShVec];
#pragma unroll
  for (int c = 0; c < kShVec; ++c) m[c] = -INFINITY;
#pragma unroll 1
  for (int n = 0; n < nscan; ++n) {
    // source row of output row Y: r = Y - n*s = r0 + w
    const ShiftSplit sp = shift[n];
    const bool frac = sp.f > 0.0f;
    const int r0 = Y - sp.i - (frac ? 1 : 0);
    const float w = frac ? 1.0f - sp.f : 0.0f;
    float a[kShVec], b[kShVec];
    const T* fr = raw + (size_t)n * plane + x;
    if (r0 >= 0 && r0 < nrows) {
      load4<T>(fr + (size_t)r0 * ncols, vec, lim, a);
    } else {
#pragma unroll
      for (int c = 0; c < kShVec; ++c) a[c] = 0.0f;
    }
    if (r0 + 1 >= 0 && r0 + 1 < nrows) {
      load4<T>(fr + (size_t)(r0 + 1) * ncols, vec, lim, b);
    } else {
#pragma unroll
      for (int c = 0; c < kShVec; ++c) b[c] = 0.0f;
    }
#pragma unroll
    for (int c = 0; c < kShVec; ++c) m[c] = fmaxf(m[c], fmaf(w, b[c] - a[c], a[c]));
  }
  float* o = out + (size_t)Y * ncols + x;
  if (vec && ((uintptr_t)o % 16 == 0)) {
    *reinterpret_cast<float4*>(o) = make_float4(m[0], m[1], m[2], m[3]);
  } else {
#pragma unroll
    for (int c = 0; c < kShVec; ++c)
      if (c < lim) o[c] = m[c];
  }
}

__global__ void __launch_bounds__(kShX* kShY)
k_warp_rows(const float* __restrict__ in, int H, int ncols, float* __restrict__ out, int Ho, double a, double b,
            int vec_ok) {
  const int Yo = blockIdx.y * kShY + threadIdx.y;
  const int x = (blockIdx.x * kShX + threadIdx.x) * kShVec;
  if (Yo >= Ho || x >= ncols) return;
  const int lim = ncols - x;
  const bool vec = vec_ok && lim >= kShVec;
  const double y = a * (double)Yo + b;
  const double fl = floor(y);
  const int y0 = (int)fmax(fmin(fl, 2.0e9), -2.0e9);
  const float w = (float)(y - fl);
  float lo[kShVec], hi[kShVec];
  if (y0 >= 0 && y0 < H) {
    load4<float>(in + (size_t)y0 * ncols + x, vec, lim, lo);
  } else {
#pragma unroll
    for (int c = 0; c < kShVec; ++c) lo[c] = 0.0f;
  }
  if (y0 + 1 >= 0 && y0 + 1 < H) {
    load4<float>(in + (size_t)(y0 + 1) * ncols + x, vec, lim, hi);
  } else {
#pragma unroll
    for (int c = 0; c < kShVec; ++c) hi[c] = 0.0f;
  }
  float* o = out + (size_t)Yo * ncols + x;
#pragma unroll
  for (int c = 0; c < kShVec; ++c)
    if (c < lim) o[c] = fmaf(w, hi[c] - lo[c], lo[c]);
}

}  // namespace

opm_status launch_sheet_project(const void* raw, opm_dtype in_t, int nscan, int nrows, int ncols, double shear,
                                float* out, int H, cudaStream_t s) {
  const size_t smem = sizeof(ShiftSplit) * (size_t)nscan;
  static int attr_done[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(OPM_ERR_UNSUPPORTED, "device ordinal out of range");
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (smem > (size_t)optin) return fail(OPM_ERR_UNSUPPORTED, "too many scan planes for the shift table");
  if (!attr_done[dev]) {
    e = cudaFuncSetAttribute(k_sheet_project<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sheet_project<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_sheet_project)");
    attr_done[dev] = 1;
  }
  const int es = in_t == OPM_U16 ? 2 : 4;
  const int vec_ok = (ncols % kShVec == 0) && ((uintptr_t)raw % (es * kShVec) == 0);
  dim3 grid((ncols + kShX * kShVec - 1) / (kShX * kShVec), (H + kShY - 1) / kShY), block(kShX, kShY);
  if (grid.y > 65535) return fail(OPM_ERR_UNSUPPORTED, "too many output rows");
  if (in_t == OPM_U16)
    k_sheet_project<uint16_t><<<grid, block, smem, s>>>(static_cast<const uint16_t*>(raw), nscan, nrows, ncols, shear,
                                                        out, H, vec_ok);
  else
    k_sheet_project<float><<<grid, block, smem, s>>>(static_cast<const float*>(raw), nscan, nrows, ncols, shear, out,
                                                     H, vec_ok);
  e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_sheet_project");
}

opm_status launch_warp_rows(const float* in, int H, int ncols, float* out, int Ho, double a, double b,
                            cudaStream_t s) {
  const int vec_ok = (ncols % kShVec == 0) && ((uintptr_t)in % 16 == 0);
  dim3 grid((ncols + kShX * kShVec - 1) / (kShX * kShVec), (Ho + kShY - 1) / kShY), block(kShX, kShY);
  if (grid.y > 65535) return fail(OPM_ERR_UNSUPPORTED, "too many output rows");
  k_warp_rows<<<grid, block, 0, s>>>(in, H, ncols, out, Ho, a, b, vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_warp_rows");
}

}  // namespace opm

using namespace opm;

extern "C" {

opm_status opm_sheet_rows(int64_t nscan, int64_t nrows, double shear, int64_t* rows) {
  if (!rows) return fail(OPM_ERR_INVALID_ARG, "rows is NULL");
  if (nscan < 1 || nrows < 1 || !(shear >= 0.0) || !std::isfinite(shear))
    return fail(OPM_ERR_INVALID_ARG, "need nscan >= 1, nrows >= 1 and a finite shear >= 0");
  const double extra = std::ceil((double)(nscan - 1) * shear - 1e-9);
  if (extra > 2.0e9 || (double)nrows + extra > 2.0e9) return fail(OPM_ERR_UNSUPPORTED, "remapped image too tall");
  *rows = nrows + (int64_t)std::max(0.0, extra);
  return OPM_OK;
}

opm_status opm_sheet_project(const void* raw, opm_dtype in_t, int64_t nscan, int64_t nrows, int64_t ncols,
                             double shear, float* out, int64_t out_rows, void* stream) {
  if (!raw || !out) return fail(OPM_ERR_INVALID_ARG, "raw and out must be non-NULL");
  if (in_t != OPM_U16 && in_t != OPM_F32) return fail(OPM_ERR_UNSUPPORTED, "opm_sheet_project takes U16 or F32");
  if (ncols < 1) return fail(OPM_ERR_INVALID_ARG, "ncols must be >= 1");
  int64_t H = 0;
  opm_status st = opm_sheet_rows(nscan, nrows, shear, &H);
  if (st != OPM_OK) return st;
  if (out_rows != H) return fail(OPM_ERR_INVALID_ARG, "out_rows must equal opm_sheet_rows(nscan, nrows, shear)");
  if (nscan > INT32_MAX || nrows > INT32_MAX || ncols > INT32_MAX)
    return fail(OPM_ERR_UNSUPPORTED, "dimensions exceed 2^31 - 1");
  return launch_sheet_project(raw, in_t, (int)nscan, (int)nrows, (int)ncols, shear, out, (int)H,
                              static_cast<cudaStream_t>(stream));
}

opm_status opm_warp_rows(const float* in, int64_t in_rows, int64_t ncols, float* out, int64_t out_rows, double a,
                         double b, void* stream) {
  if (!in || !out) return fail(OPM_ERR_INVALID_ARG, "in and out must be non-NULL");
  if (in_rows < 1 || ncols < 1 || out_rows < 1 || !std::isfinite(a) || !std::isfinite(b))
    return fail(OPM_ERR_INVALID_ARG, "need positive sizes and finite a, b");
  if (in_rows > INT32_MAX || ncols > INT32_MAX || out_rows > INT32_MAX)
    return fail(OPM_ERR_UNSUPPORTED, "dimensions exceed 2^31 - 1");
  return launch_warp_rows(in, (int)in_rows, (int)ncols, out, (int)out_rows, a, b, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
