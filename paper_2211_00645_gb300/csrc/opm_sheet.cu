// The paper's own live view: every raw frame n remapped into a larger image,
// shifted along the camera-row axis by its accumulated lateral offset n * s
// rows (Eq. 1 with s = step cos(alpha) / pixel; Fig. 2c), then the
// brightest value over the frames at each pixel (Fig. 2d).  A reduced shear
// factor followed by a 1-D affine warp of the projection changes the viewing
// angle (shear-warp, Fig. 3).  Sub-row shifts interpolate linearly between
// the two neighbouring camera rows (zero outside the frame).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "opm_tma.cuh"

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

// ---------------------------------------------------------------------------
// TMA form for uint16 stacks: a CTA owns a tile of kSY output rows x kSX
// columns and a chunk of frames.  Its producer warp stages, per frame, the
// kSY + 1 camera rows that the tile's rows interpolate between (one TMA box
// {kSX, kSY + 1, 1}, zero-filled outside the frame) into a ring; four
// compute warps (64 columns x 16 rows each, two columns per lane) convert
// each staged row once and keep the running maxima in registers, taking
// two frames per step (one 3-input max per voxel and frame pair).  Chunks of
// one tile combine by atomic max into the zeroed output (uint16 views are
// >= 0, so integer order is float order).  Frames whose rows miss the tile
// entirely are skipped: they contribute 0, which the zeroed output holds.
// The arithmetic is that of k_sheet_project, fma(w, b - a, a) and max, so
// the two kernels give the same bits.
constexpr int kSY = 32;                       // output rows per tile
constexpr int kSRows = kSY + 1;               // camera rows staged per frame
constexpr int kSX = 128;                      // columns per tile (TMA box width)
constexpr int kSCW = 4;                       // compute warps
constexpr int kSHalf = kSY / 2;               // output rows per compute warp
constexpr int kSStages = 6;                   // ring depth
constexpr int kSChunk = 50;                   // frames per CTA, at most
constexpr unsigned kSStageBytes = kSRows * kSX * 2;
static_assert(kSStageBytes % 128 == 0, "ring stages stay 128-byte aligned");
constexpr size_t kSOffBar = (size_t)kSStages * kSStageBytes;
constexpr size_t kSOffShift = kSOffBar + 2 * kSStages * sizeof(uint64_t);
constexpr size_t sheet_tma_smem() { return kSOffShift + kSChunk * sizeof(ShiftSplit); }

// Wait-timeout word of the TMA sheet kernel on this device (read and cleared
// by opm_sheet_check).
__device__ unsigned g_sheet_err;

// First staged camera row of frame n for the tile starting at output row Y0,
// and the frame's interpolation weight (as k_sheet_project derives them).
__device__ __forceinline__ int sheet_row0(const ShiftSplit& sp, int Y0) {
  return Y0 - sp.i - (sp.f > 0.0f ? 1 : 0);
}

__global__ void __launch_bounds__(32 * (kSCW + 1))
k_sheet_tma(const __grid_constant__ CUtensorMap map, int nscan, int nrows, int ncols, double shear,
            float* __restrict__ out, int H, int chunk, unsigned* err) {
  extern __shared__ __align__(128) unsigned char ssm[];
  uint64_t* full = reinterpret_cast<uint64_t*>(ssm + kSOffBar);
  uint64_t* sfree = full + kSStages;
  ShiftSplit* shift = reinterpret_cast<ShiftSplit*>(ssm + kSOffShift);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x0 = blockIdx.x * kSX, Y0 = blockIdx.y * kSY;
  const int n0 = blockIdx.z * chunk, n1 = min(nscan, n0 + chunk);
  for (int n = n0 + (int)threadIdx.x; n < n1; n += blockDim.x) {
    const double sh = (double)n * shear;
    const double fl = floor(sh);
    shift[n - n0] = ShiftSplit{(int)fl, (float)(sh - fl)};
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&sfree[s], kSCW);
    }
    fence_barrier_init();
  }
  __syncthreads();
  // a frame feeds the tile when its staged rows [r0, r0 + kSRows) meet the frame
  auto feeds = [&](int n) {
    const int r0 = sheet_row0(shift[n - n0], Y0);
    return r0 < nrows && r0 + kSRows > 0;
  };
  int g = 0;
  bool ok = true;
  if (warp == 0) {
#pragma unroll 1
    for (int n = n0; n < n1 && ok; ++n) {
      if (!feeds(n)) continue;
      const int s = g % kSStages;
      if (g >= kSStages) ok = mbar_wait(&sfree[s], ((g - kSStages) / kSStages) & 1, err);
      if (ok && lane == 0) {
        mbar_arrive_tx(&full[s], kSStageBytes);
        tma_load_3d(ssm + (size_t)s * kSStageBytes, &map, &full[s], x0, sheet_row0(shift[n - n0], Y0), n);
      }
      __syncwarp();
      ++g;
    }
    // the CTA's shared memory must outlive every copy it issued
    for (int q = max(0, g - kSStages); q < g; ++q)
      if (!mbar_wait(&full[q % kSStages], (q / kSStages) & 1, err, ok ? kWaitLimitNs : 50000000ull)) break;
    return;
  }
  const int i = warp - 1;
  const int xl = (i & 1) * 64 + lane * 2;  // this lane's first column within the tile
  const int t0 = (i >> 1) * kSHalf;        // this warp's first output row within the tile
  float m[kSHalf][2];
#pragma unroll
  for (int t = 0; t < kSHalf; ++t) m[t][0] = m[t][1] = 0.0f;
  int n = n0;
#pragma unroll 1
  while (true) {
    while (n < n1 && !feeds(n)) ++n;
    if (n >= n1) break;
    // two frames at a time (one 3-input max per voxel pair), a single one last
    int nb = n + 1;
    while (nb < n1 && !feeds(nb)) ++nb;
    if (nb < n1) {
      const int s = g % kSStages, s2 = (g + 1) % kSStages;
      if (!mbar_wait(&full[s], (g / kSStages) & 1, err) || !mbar_wait(&full[s2], ((g + 1) / kSStages) & 1, err)) {
        ok = false;
        break;
      }
      const ShiftSplit sp = shift[n - n0], sq = shift[nb - n0];
      const float w = sp.f > 0.0f ? 1.0f - sp.f : 0.0f;
      const float w2 = sq.f > 0.0f ? 1.0f - sq.f : 0.0f;
      const f2 ww = pk(w, w), ww2 = pk(w2, w2);
      const unsigned char* row = ssm + (size_t)s * kSStageBytes + (size_t)t0 * (kSX * 2) + xl * 2;
      const unsigned char* row2 = ssm + (size_t)s2 * kSStageBytes + (size_t)t0 * (kSX * 2) + xl * 2;
      f2 a = u16x2_to_f2(*reinterpret_cast<const uint32_t*>(row));
      f2 a2 = u16x2_to_f2(*reinterpret_cast<const uint32_t*>(row2));
#pragma unroll
      for (int t = 0; t < kSHalf; ++t) {
        const f2 b = u16x2_to_f2(*reinterpret_cast<const uint32_t*>(row + (t + 1) * (kSX * 2)));
        const f2 b2 = u16x2_to_f2(*reinterpret_cast<const uint32_t*>(row2 + (t + 1) * (kSX * 2)));
        float v0, v1, u0, u1;
        upk(fma2(ww, sub2(b, a), a), v0, v1);
        upk(fma2(ww2, sub2(b2, a2), a2), u0, u1);
        m[t][0] = max3(m[t][0], v0, u0);
        m[t][1] = max3(m[t][1], v1, u1);
        a = b;
        a2 = b2;
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sfree[s]);
        mbar_arrive(&sfree[s2]);
      }
      g += 2;
      n = nb + 1;
      continue;
    }
    const int s = g % kSStages;
    if (!mbar_wait(&full[s], (g / kSStages) & 1, err)) {
      ok = false;
      break;
    }
    const ShiftSplit sp = shift[n - n0];
    const float w = sp.f > 0.0f ? 1.0f - sp.f : 0.0f;
    const f2 ww = pk(w, w);
    const unsigned char* row = ssm + (size_t)s * kSStageBytes + (size_t)t0 * (kSX * 2) + xl * 2;
    f2 a = u16x2_to_f2(*reinterpret_cast<const uint32_t*>(row));
#pragma unroll
    for (int t = 0; t < kSHalf; ++t) {
      const f2 b = u16x2_to_f2(*reinterpret_cast<const uint32_t*>(row + (t + 1) * (kSX * 2)));
      float v0, v1;
      upk(fma2(ww, sub2(b, a), a), v0, v1);
      m[t][0] = fmaxf(m[t][0], v0);
      m[t][1] = fmaxf(m[t][1], v1);
      a = b;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sfree[s]);
    ++g;
    ++n;
  }
  if (!ok) return;
  const int x = x0 + xl;
#pragma unroll
  for (int t = 0; t < kSHalf; ++t) {
    const int Y = Y0 + t0 + t;
    if (Y >= H) break;
    int* o = reinterpret_cast<int*>(out + (size_t)Y * ncols + x);
    if (x < ncols) atomicMax(o, __float_as_int(m[t][0]));
    if (x + 1 < ncols) atomicMax(o + 1, __float_as_int(m[t][1]));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 sheet_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
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

// The TMA form: uint16 stacks with rows of a multiple of 8 columns (16-byte
// strides), a 16-byte aligned base, and at least one full box of rows and
// columns.  Sets *launched = false (nothing launched) when it does not apply.
opm_status launch_sheet_tma(const void* raw, int nscan, int nrows, int ncols, double shear, float* out, int H,
                            int dev, cudaStream_t s, bool* launched) {
  *launched = false;
  if (ncols % 8 != 0 || (uintptr_t)raw % 16 != 0 || nrows < kSRows || ncols < kSX || !sheet_encode_fn())
    return OPM_OK;
  // per-device set-up, once: the shared-memory limit and the address of the
  // device's error word (taken under the lock, so no launch sees a null one)
  static std::mutex mu;
  static unsigned* err_ptr[64] = {nullptr};
  unsigned* err = nullptr;
  cudaError_t e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!err_ptr[dev]) {
      unsigned* p = nullptr;
      e = cudaFuncSetAttribute(k_sheet_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sheet_tma_smem());
      if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_sheet_err);
      if (e != cudaSuccess) return cuda_fail(e, "set-up of k_sheet_tma");
      err_ptr[dev] = p;
    }
    err = err_ptr[dev];
  }
  CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)ncols, (cuuint64_t)nrows, (cuuint64_t)nscan};
  const cuuint64_t strides[2] = {(cuuint64_t)ncols * 2, (cuuint64_t)nrows * (cuuint64_t)ncols * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kSX, (cuuint32_t)kSRows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult cr = sheet_encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(raw), dims,
                                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return OPM_OK;  // the plain kernel takes it
  const int nchunks = (nscan + kSChunk - 1) / kSChunk;
  const int chunk = (nscan + nchunks - 1) / nchunks;
  const dim3 grid((ncols + kSX - 1) / kSX, (H + kSY - 1) / kSY, nchunks);
  if (grid.y > 65535 || grid.z > 65535) return fail(OPM_ERR_UNSUPPORTED, "too many output rows or frames");
  e = cudaMemsetAsync(out, 0, sizeof(float) * (size_t)H * (size_t)ncols, s);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (sheet view)");
  k_sheet_tma<<<grid, 32 * (kSCW + 1), sheet_tma_smem(), s>>>(map, nscan, nrows, ncols, shear, out, H, chunk, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch k_sheet_tma");
  *launched = true;
  return OPM_OK;
}

opm_status launch_sheet_project(const void* raw, opm_dtype in_t, int nscan, int nrows, int ncols, double shear,
                                float* out, int H, cudaStream_t s) {
  const size_t smem = sizeof(ShiftSplit) * (size_t)nscan;
  static int attr_done[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(OPM_ERR_UNSUPPORTED, "device ordinal out of range");
  if (in_t == OPM_U16) {
    bool launched = false;
    const opm_status st = launch_sheet_tma(raw, nscan, nrows, ncols, shear, out, H, dev, s, &launched);
    if (st != OPM_OK || launched) return st;
  }
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

opm_status opm_sheet_check(void) {
  unsigned v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_sheet_err, sizeof(v));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyFromSymbol (sheet-view error word)");
  if (v == 0) return OPM_OK;
  const unsigned zero = 0;
  e = cudaMemcpyToSymbol(g_sheet_err, &zero, sizeof(zero));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol (sheet-view error word)");
  return fail(OPM_ERR_INTERNAL, "a sheet-view ring wait gave up (result incomplete)");
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
