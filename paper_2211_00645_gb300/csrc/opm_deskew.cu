// Full-volume deskew (Fig. 2c remap with linear interpolation between scan
// planes).  Output-write bound: every voxel is written once with streaming
// stores.  Each thread walks a run of output columns j of one row k and keeps
// the current pair of raw planes in registers, so a raw vector is fetched once
// per plane step rather than once per voxel.  A lane owns two half-vectors of
// columns 32*HALF apart, so that every store instruction of a warp covers one
// contiguous span of 32*HALF elements.
#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kThreadsX = 32;  // lanes along x
constexpr int kThreadsY = 4;   // j-runs per CTA
constexpr int kRunJ = 32;      // output columns per thread

template <typename T, int N, typename Acc>
__device__ __forceinline__ void load_half(const T* __restrict__ p, bool vec, int lim, Acc (&out)[N]) {
  static_assert(sizeof(T) * N == 8, "8-byte half vectors");
  if (vec) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = static_cast<Acc>(e[i]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = i < lim ? static_cast<Acc>(__ldg(p + i)) : Acc(0);
  }
}

// Stores one half-vector of H output values with streaming stores (16-byte
// FP32 or 8-byte uint16 vectors when `full`), else element by element.
template <typename Tout, int H, typename Acc>
__device__ __forceinline__ void store_half(Tout* op, const Acc (&val)[H], bool full, int lim) {
  if constexpr (std::is_same<Tout, float>::value && H == 4) {
    if (full) {
      st_cs_v4(op, val[0], val[1], val[2], val[3]);
      return;
    }
  }
  if constexpr (std::is_same<Tout, uint16_t>::value && H == 4) {
    if (full) {
      const uint32_t lo = (uint32_t)to_u16_rn(val[0]) | ((uint32_t)to_u16_rn(val[1]) << 16);
      const uint32_t hi = (uint32_t)to_u16_rn(val[2]) | ((uint32_t)to_u16_rn(val[3]) << 16);
      asm volatile("st.global.cs.v2.b32 [%0], {%1, %2};" ::"l"(op), "r"(lo), "r"(hi) : "memory");
      return;
    }
  }
  if constexpr (std::is_same<Tout, float>::value && H == 2) {
    if (full) {
      asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(op), "f"(val[0]), "f"(val[1]) : "memory");
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    if (i >= lim) break;
    if constexpr (std::is_same<Tout, uint16_t>::value)
      op[i] = to_u16_rn(val[i]);
    else
      op[i] = (Tout)val[i];
  }
}

// vol2 (uint16, may be NULL unless DUAL) receives the round-to-nearest-even
// copy of the same values in the same pass.
template <typename Tin, typename Tout, typename Acc, int VEC, bool DUAL>
__global__ void __launch_bounds__(kThreadsX* kThreadsY)
k_deskew(PlanView v, const Tin* __restrict__ raw, Tout* __restrict__ vol, uint16_t* __restrict__ vol2, int xtiles,
         int in_vec_ok, int out_vec_ok, int out2_vec_ok) {
  constexpr int H = VEC / 2;  // elements per half-vector
  const int k = blockIdx.x / xtiles;
  const int xt = blockIdx.x - k * xtiles;
  const int xh[2] = {xt * kThreadsX * VEC + (int)threadIdx.x * H,
                     xt * kThreadsX * VEC + kThreadsX * H + (int)threadIdx.x * H};
  if (xh[0] >= v.nx) return;
  const int lim[2] = {v.nx - xh[0], v.nx - xh[1]};  // valid columns of each half
  const int jb = (blockIdx.y * kThreadsY + threadIdx.y) * kRunJ;
  if (jb >= v.ny) return;
  const Split b = v.B[k];
  const size_t plane = (size_t)v.nrows * v.ncols;
  const Tin* rowp = raw + (size_t)k * v.ncols;

  Acc a[2][H], bb[2][H], d[2][H];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int i = 0; i < H; ++i) a[h][i] = bb[h][i] = d[h][i] = Acc(0);
  int ocur = -0x40000000;  // plane index held in a[] (none yet)

  auto fetch = [&](int n, Acc(&out)[2][H]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (n >= 0 && n < v.nscan && lim[h] > 0) {
        load_half<Tin, H, Acc>(rowp + (size_t)n * plane + xh[h], in_vec_ok && lim[h] >= H, lim[h], out[h]);
      } else {
#pragma unroll
        for (int i = 0; i < H; ++i) out[h][i] = Acc(0);
      }
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
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int i = 0; i < H; ++i) a[h][i] = bb[h][i];
      } else {
        fetch(n0, a);
      }
      fetch(n0 + 1, bb);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int i = 0; i < H; ++i) d[h][i] = bb[h][i] - a[h][i];
      ocur = n0;
    }
    const size_t orow = ((size_t)k * v.ny + j) * v.nx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (lim[h] <= 0) continue;
      Acc val[H];
#pragma unroll
      for (int i = 0; i < H; ++i) val[i] = fma(w, d[h][i], a[h][i]);
      store_half<Tout, H, Acc>(vol + orow + xh[h], val, out_vec_ok && lim[h] >= H, lim[h]);
      if constexpr (DUAL) store_half<uint16_t, H, Acc>(vol2 + orow + xh[h], val, out2_vec_ok && lim[h] >= H, lim[h]);
    }
  }
}

template <typename Tin, typename Tout, typename Acc, int VEC, bool DUAL = false>
opm_status run(const opm_plan* p, const void* raw, void* vol, void* vol2, cudaStream_t s) {
  constexpr int H = VEC / 2;
  const PlanView& v = p->view;
  const int xtiles = (v.nx + kThreadsX * VEC - 1) / (kThreadsX * VEC);
  const long long gx = (long long)xtiles * v.nz;
  const int gy = (v.ny + kThreadsY * kRunJ - 1) / (kThreadsY * kRunJ);
  if (gx > 0x7fffffffLL || gy > 65535)
    return fail(OPM_ERR_UNSUPPORTED, "deskew grid exceeds launch limits");
  const int in_vec_ok = (v.ncols % H == 0) && ((uintptr_t)raw % 8 == 0);
  const int out_vec_ok = (v.nx % H == 0) && ((uintptr_t)vol % (sizeof(Tout) * H) == 0);
  const int out2_vec_ok = (v.nx % H == 0) && ((uintptr_t)vol2 % (sizeof(uint16_t) * H) == 0);
  dim3 block(kThreadsX, kThreadsY);
  dim3 grid((unsigned)gx, (unsigned)gy);
  k_deskew<Tin, Tout, Acc, VEC, DUAL><<<grid, block, 0, s>>>(v, static_cast<const Tin*>(raw), static_cast<Tout*>(vol),
                                                             static_cast<uint16_t*>(vol2), xtiles, in_vec_ok,
                                                             out_vec_ok, out2_vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_deskew");
}

// ---------------------------------------------------------------------------
// Volume and live view in one pass (uint16 input): every voxel is stored as
// k_deskew stores it, and folded into the z-MIP and y-MIP on the way.  CTA
// (32 x 8 threads): 128 columns x (4 per lane) x 32 columns j (4 per warp) x
// a chunk of kMipRows camera rows, 4 CTAs per SM.  The z-maxima of a
// thread's 4 x 4 voxels
// stay in registers across the chunk's rows and are folded into the global
// z-MIP once; the y-maxima of each row are combined across the 8 warps with
// shared-memory atomics and folded into the global y-MIP once per CTA.  All
// combines are maxima of non-negative values on their bit patterns, so the
// result does not depend on their order.
constexpr int kMipRows = 64;
constexpr int kMipWarps = 8;  // warps (runs of kMipJ columns) per CTA
constexpr int kMipJ = 4;     // columns j per thread
constexpr int kMipVec = 4;   // columns x per lane

template <bool F32, bool U16>
__global__ void __launch_bounds__(kThreadsX* kMipWarps, 4)
k_deskew_mip(PlanView v, const uint16_t* __restrict__ raw, float* __restrict__ volf, uint16_t* __restrict__ volh,
             float* __restrict__ zmip, float* __restrict__ ymip, int in_vec_ok, int out_vec_ok) {
  __shared__ float ybuf[kMipRows][kThreadsX * kMipVec];
  const int lane = threadIdx.x, w = threadIdx.y;
  const int x = blockIdx.x * kThreadsX * kMipVec + lane * kMipVec;
  const int jb = (blockIdx.y * kMipWarps + w) * kMipJ;
  const int k0 = blockIdx.z * kMipRows;
  const int k1 = min(k0 + kMipRows, v.nz);
  for (int i = threadIdx.y * kThreadsX + threadIdx.x; i < kMipRows * kThreadsX * kMipVec; i += kThreadsX * kMipWarps)
    (&ybuf[0][0])[i] = 0.0f;
  __syncthreads();
  const bool active = x < v.nx && jb < v.ny;
  const int lim = v.nx - x;  // valid columns of this lane's vector
  const bool vin = in_vec_ok && lim >= kMipVec;
  const bool vout = out_vec_ok && lim >= kMipVec;
  const size_t plane = (size_t)v.nrows * v.ncols;
  float zmax[kMipJ][kMipVec];
#pragma unroll
  for (int j = 0; j < kMipJ; ++j)
#pragma unroll
    for (int c = 0; c < kMipVec; ++c) zmax[j][c] = 0.0f;  // uint16 voxels are >= 0

#pragma unroll 1
  for (int k = k0; active && k < k1; ++k) {
    const Split b = v.B[k];
    const uint16_t* rowp = raw + (size_t)k * v.ncols + x;
    float a[kMipVec], bb[kMipVec], d[kMipVec], ym[kMipVec];
#pragma unroll
    for (int c = 0; c < kMipVec; ++c) a[c] = bb[c] = d[c] = ym[c] = 0.0f;
    int ocur = -0x40000000;
    auto fetch = [&](int n, float(&out)[kMipVec]) {
      if (n >= 0 && n < v.nscan) {
        const uint16_t* p = rowp + (size_t)n * plane;
        if (vin) {
          const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
          out[0] = (float)(u.x & 0xFFFFu);
          out[1] = (float)(u.x >> 16);
          out[2] = (float)(u.y & 0xFFFFu);
          out[3] = (float)(u.y >> 16);
        } else {
#pragma unroll
          for (int c = 0; c < kMipVec; ++c) out[c] = c < lim ? (float)__ldg(p + c) : 0.0f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < kMipVec; ++c) out[c] = 0.0f;
      }
    };
#pragma unroll
    for (int jj = 0; jj < kMipJ; ++jj) {
      const int j = jb + jj;
      if (j >= v.ny) break;
      int n0;
      float wt;
      plane_weight(v.A[j], b, v.linear, n0, wt);
      if (n0 != ocur) {
        if (n0 == ocur + 1) {
#pragma unroll
          for (int c = 0; c < kMipVec; ++c) a[c] = bb[c];
        } else {
          fetch(n0, a);
        }
        fetch(n0 + 1, bb);
#pragma unroll
        for (int c = 0; c < kMipVec; ++c) d[c] = bb[c] - a[c];  // exact: integers below 2^24
        ocur = n0;
      }
      float val[kMipVec];
#pragma unroll
      for (int c = 0; c < kMipVec; ++c) {
        val[c] = fmaf(wt, d[c], a[c]);
        zmax[jj][c] = fmaxf(zmax[jj][c], val[c]);
        ym[c] = fmaxf(ym[c], val[c]);
      }
      const size_t o = ((size_t)k * v.ny + j) * v.nx + x;
      if (vout) {
        if (F32) st_cs_v4(volf + o, val[0], val[1], val[2], val[3]);
        if (U16) {
          const uint32_t lo = (uint32_t)to_u16_rn(val[0]) | ((uint32_t)to_u16_rn(val[1]) << 16);
          const uint32_t hi = (uint32_t)to_u16_rn(val[2]) | ((uint32_t)to_u16_rn(val[3]) << 16);
          asm volatile("st.global.cs.v2.b32 [%0], {%1, %2};" ::"l"(volh + o), "r"(lo), "r"(hi) : "memory");
        }
      } else {
#pragma unroll
        for (int c = 0; c < kMipVec; ++c) {
          if (c >= lim) break;
          if (F32) volf[o + c] = val[c];
          if (U16) volh[o + c] = to_u16_rn(val[c]);
        }
      }
    }
    if (ymip) {
#pragma unroll
      for (int c = 0; c < kMipVec; ++c)
        if (c < lim) atomicMax(reinterpret_cast<int*>(&ybuf[k - k0][lane * kMipVec + c]), __float_as_int(ym[c]));
    }
  }
  if (zmip && active) {
#pragma unroll
    for (int jj = 0; jj < kMipJ; ++jj) {
      const int j = jb + jj;
      if (j >= v.ny) break;
      float* zr = zmip + (size_t)j * v.nx + x;
#pragma unroll
      for (int c = 0; c < kMipVec; ++c)
        if (c < lim) atomicMax(reinterpret_cast<int*>(zr + c), __float_as_int(zmax[jj][c]));
    }
  }
  if (ymip) {
    __syncthreads();
    const int xb = blockIdx.x * kThreadsX * kMipVec;
    for (int i = threadIdx.y * kThreadsX + threadIdx.x; i < (k1 - k0) * kThreadsX * kMipVec;
         i += kThreadsX * kMipWarps) {
      const int kk = i / (kThreadsX * kMipVec), xx = i % (kThreadsX * kMipVec);
      if (xb + xx < v.nx)
        atomicMax(reinterpret_cast<int*>(ymip + (size_t)(k0 + kk) * v.nx + xb + xx), __float_as_int(ybuf[kk][xx]));
    }
  }
}

__global__ void k_zero2(float* a, long long na, float* b, long long nb) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < na || i < nb; i += stride) {
    if (a && i < na) a[i] = 0.0f;
    if (b && i < nb) b[i] = 0.0f;
  }
}

}  // namespace

opm_status launch_deskew(const opm_plan* p, const void* raw, opm_dtype in_t, void* vol,
                         opm_dtype out_t, cudaStream_t s) {
  if (in_t == OPM_U16 && out_t == OPM_F32) return run<uint16_t, float, float, 8>(p, raw, vol, nullptr, s);
  if (in_t == OPM_U16 && out_t == OPM_U16) return run<uint16_t, uint16_t, float, 8>(p, raw, vol, nullptr, s);
  if (in_t == OPM_F32 && out_t == OPM_F32) return run<float, float, float, 4>(p, raw, vol, nullptr, s);
  if (in_t == OPM_F32 && out_t == OPM_U16) return run<float, uint16_t, float, 4>(p, raw, vol, nullptr, s);
  if (in_t == OPM_F64 && out_t == OPM_F64) return run<double, double, double, 2>(p, raw, vol, nullptr, s);
  return fail(OPM_ERR_UNSUPPORTED, "unsupported dtype pair");
}

opm_status launch_deskew_dual(const opm_plan* p, const void* raw, opm_dtype in_t, float* vol_f32, uint16_t* vol_u16,
                              cudaStream_t s) {
  if (in_t == OPM_U16) return run<uint16_t, float, float, 8, true>(p, raw, vol_f32, vol_u16, s);
  if (in_t == OPM_F32) return run<float, float, float, 4, true>(p, raw, vol_f32, vol_u16, s);
  return fail(OPM_ERR_UNSUPPORTED, "dual-output deskew takes uint16 or FP32 input");
}

}  // namespace opm

namespace opm {

namespace {

// The volume on the caller's stream s and the live view beside it on the
// plan's high-priority side stream, forked from and joined back into s.
// The live view's persistent kernel takes a quarter of its usual grid (one
// CTA per SM), so each SM also holds volume CTAs: the issue-bound projection
// then fills the issue slots the write-bound volume leaves idle.  Each
// kernel computes exactly what it computes alone.
opm_status deskew_beside_project(const opm_plan* p, const void* raw, opm_dtype in_t, float* volf, uint16_t* volh,
                                 float* zmip, float* ymip, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(p->side_mu);
  cudaError_t e = cudaEventRecord(p->fork_ev, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->fork_ev, 0);
  if (e != cudaSuccess) return cuda_fail(e, "forking the live view onto the side stream");
  opm_status st = launch_project(p, raw, in_t, zmip, nullptr, ymip, nullptr, p->side, p->lists_per_sm);
  opm_status sv = OPM_OK;
  if (volf && volh)
    sv = launch_deskew_dual(p, raw, in_t, volf, volh, s);
  else
    sv = launch_deskew(p, raw, in_t, volf ? (void*)volf : (void*)volh, volf ? OPM_F32 : OPM_U16, s);
  // join even after a failed launch, so that s never runs ahead of the side stream
  e = cudaEventRecord(p->join_ev, p->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join_ev, 0);
  if (st != OPM_OK) return st;
  if (sv != OPM_OK) return sv;
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "joining the side stream");
}

}  // namespace

opm_status launch_deskew_mip(const opm_plan* p, const void* raw, opm_dtype in_t, float* volf, uint16_t* volh,
                             float* zmip, float* ymip, cudaStream_t s) {
  const PlanView& v = p->view;
  if ((zmip || ymip) && p->side && !p->one_pass_fused)
    return deskew_beside_project(p, raw, in_t, volf, volh, zmip, ymip, s);
  if (in_t != OPM_U16) {
    // FP32 input: the volume, then the projections
    opm_status st = OPM_OK;
    if (volf && volh)
      st = launch_deskew_dual(p, raw, in_t, volf, volh, s);
    else
      st = launch_deskew(p, raw, in_t, volf ? (void*)volf : (void*)volh, volf ? OPM_F32 : OPM_U16, s);
    if (st != OPM_OK || (!zmip && !ymip)) return st;
    return launch_project(p, raw, in_t, zmip, nullptr, ymip, nullptr, s);
  }
  const int xtiles = (v.nx + kThreadsX * kMipVec - 1) / (kThreadsX * kMipVec);
  const int jblocks = (v.ny + kMipWarps * kMipJ - 1) / (kMipWarps * kMipJ);
  const int kchunks = (v.nz + kMipRows - 1) / kMipRows;
  if (jblocks > 65535 || kchunks > 65535) return fail(OPM_ERR_UNSUPPORTED, "deskew grid exceeds launch limits");
  if (zmip || ymip) {
    k_zero2<<<4 * 152, 256, 0, s>>>(zmip, zmip ? (long long)v.ny * v.nx : 0, ymip, ymip ? (long long)v.nz * v.nx : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_zero2");
  }
  const int in_vec_ok = (v.ncols % kMipVec == 0) && ((uintptr_t)raw % 8 == 0);
  const int out_vec_ok = (v.nx % kMipVec == 0) && ((uintptr_t)volf % 16 == 0) && ((uintptr_t)volh % 8 == 0);
  dim3 grid(xtiles, jblocks, kchunks), block(kThreadsX, kMipWarps);
  const uint16_t* r = static_cast<const uint16_t*>(raw);
  if (volf && volh)
    k_deskew_mip<true, true><<<grid, block, 0, s>>>(v, r, volf, volh, zmip, ymip, in_vec_ok, out_vec_ok);
  else if (volf)
    k_deskew_mip<true, false><<<grid, block, 0, s>>>(v, r, volf, volh, zmip, ymip, in_vec_ok, out_vec_ok);
  else
    k_deskew_mip<false, true><<<grid, block, 0, s>>>(v, r, volf, volh, zmip, ymip, in_vec_ok, out_vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_deskew_mip");
}

}  // namespace opm
