// Full-volume deskew (Fig. 2c remap with linear interpolation between scan
// planes).  Output-write bound: every voxel is written once with 16-byte
// streaming stores; each thread walks a run of output columns j of one row k
// and keeps the current pair of raw planes in registers, so a raw vector is
// fetched once per plane step rather than once per voxel.
#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kThreadsX = 32;  // lanes along x
constexpr int kThreadsY = 8;   // j-runs per CTA
constexpr int kRunJ = 8;       // output columns per thread

template <typename Tin, typename Tout, typename Acc, int VEC>
__global__ void __launch_bounds__(kThreadsX* kThreadsY)
k_deskew(PlanView v, const Tin* __restrict__ raw, Tout* __restrict__ vol, int xtiles,
         int in_vec_ok, int out_vec_ok) {
  const int k = blockIdx.x / xtiles;
  const int xt = blockIdx.x - k * xtiles;
  const int x0 = (xt * kThreadsX + threadIdx.x) * VEC;
  if (x0 >= v.nx) return;
  const int lim = v.nx - x0;  // valid columns of this vector (>= 1)
  const bool in_vec = in_vec_ok && lim >= VEC;
  const bool out_vec = out_vec_ok && lim >= VEC;
  const int jb = (blockIdx.y * kThreadsY + threadIdx.y) * kRunJ;
  if (jb >= v.ny) return;
  const Split b = v.B[k];
  const size_t plane = (size_t)v.nrows * v.ncols;
  const Tin* rowp = raw + (size_t)k * v.ncols + x0;

  Acc a[VEC], bb[VEC], d[VEC];
#pragma unroll
  for (int i = 0; i < VEC; ++i) a[i] = bb[i] = d[i] = Acc(0);
  int ocur = -0x40000000;  // plane index held in a[] (none yet)

  auto fetch = [&](int n, Acc(&out)[VEC]) {
    if (n >= 0 && n < v.nscan) {
      load_vec<Tin, VEC, Acc>(rowp + (size_t)n * plane, in_vec, lim, out);
    } else {
#pragma unroll
      for (int i = 0; i < VEC; ++i) out[i] = Acc(0);
    }
  };

#pragma unroll 1
  for (int jj = 0; jj < kRunJ; ++jj) {
    const int j = jb + jj;
    if (j >= v.ny) break;
    int n0;
    Acc w;
    plane_weight_t<Acc>(v.A[j], b, v.linear, n0, w);
    if (n0 != ocur) {
      if (n0 == ocur + 1) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) a[i] = bb[i];
      } else {
        fetch(n0, a);
      }
      fetch(n0 + 1, bb);
#pragma unroll
      for (int i = 0; i < VEC; ++i) d[i] = bb[i] - a[i];
      ocur = n0;
    }
    Acc val[VEC];
#pragma unroll
    for (int i = 0; i < VEC; ++i) val[i] = fma(w, d[i], a[i]);

    Tout* op = vol + ((size_t)k * v.ny + j) * v.nx + x0;
    if constexpr (std::is_same<Tout, uint16_t>::value) {
      uint16_t u[VEC];
#pragma unroll
      for (int i = 0; i < VEC; ++i) u[i] = to_u16_rn(val[i]);
      if (out_vec && VEC == 8) {
        const uint32_t* q = reinterpret_cast<const uint32_t*>(u);
        st_cs_v4u(op, q[0], q[1], q[2], q[3]);
      } else {
        for (int i = 0; i < VEC && i < lim; ++i) op[i] = u[i];
      }
    } else if constexpr (std::is_same<Tout, float>::value) {
      if (out_vec) {
#pragma unroll
        for (int i = 0; i < VEC; i += 4) st_cs_v4(op + i, val[i], val[i + 1], val[i + 2], val[i + 3]);
      } else {
        for (int i = 0; i < VEC && i < lim; ++i) op[i] = val[i];
      }
    } else {
      for (int i = 0; i < VEC && i < lim; ++i) op[i] = val[i];
    }
  }
}

template <typename Tin, typename Tout, typename Acc, int VEC>
opm_status run(const opm_plan* p, const void* raw, void* vol, cudaStream_t s) {
  const PlanView& v = p->view;
  const int xtiles = (v.nx + kThreadsX * VEC - 1) / (kThreadsX * VEC);
  const long long gx = (long long)xtiles * v.nz;
  const int gy = (v.ny + kThreadsY * kRunJ - 1) / (kThreadsY * kRunJ);
  if (gx > 0x7fffffffLL || gy > 65535)
    return fail(OPM_ERR_UNSUPPORTED, "deskew grid exceeds launch limits");
  const int in_vec_ok = (v.ncols % VEC == 0) && ((uintptr_t)raw % 16 == 0);
  const int out_vec_ok = (v.nx % VEC == 0) && ((uintptr_t)vol % 16 == 0) &&
                         (sizeof(Tout) * VEC) % 16 == 0;
  dim3 block(kThreadsX, kThreadsY);
  dim3 grid((unsigned)gx, (unsigned)gy);
  k_deskew<Tin, Tout, Acc, VEC><<<grid, block, 0, s>>>(
      v, static_cast<const Tin*>(raw), static_cast<Tout*>(vol), xtiles, in_vec_ok, out_vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_deskew");
}

}  // namespace

opm_status launch_deskew(const opm_plan* p, const void* raw, opm_dtype in_t, void* vol,
                         opm_dtype out_t, cudaStream_t s) {
  if (in_t == OPM_U16 && out_t == OPM_F32) return run<uint16_t, float, float, 8>(p, raw, vol, s);
  if (in_t == OPM_U16 && out_t == OPM_U16) return run<uint16_t, uint16_t, float, 8>(p, raw, vol, s);
  if (in_t == OPM_F32 && out_t == OPM_F32) return run<float, float, float, 4>(p, raw, vol, s);
  if (in_t == OPM_F32 && out_t == OPM_U16) return run<float, uint16_t, float, 4>(p, raw, vol, s);
  if (in_t == OPM_F64 && out_t == OPM_F64) return run<double, double, double, 2>(p, raw, vol, s);
  return fail(OPM_ERR_UNSUPPORTED, "unsupported dtype pair");
}

}  // namespace opm
