// Adjoint of the deskew and backward pass of the z-MIP.
//
// Both apply the transpose of the interpolation map: raw sample (n, k, x)
// collects every output column j of row k whose lower plane n0(j,k) is n
// (weight 1 - w) or n - 1 (weight w), in ascending j.  The weights are
// computed with the forward kernels' own split-table formula, so the adjoint
// is the exact transpose of the map the forward kernels apply.  No atomics:
// results are bitwise reproducible.  The adjoint walks the columns j of a
// row once per block of planes; the z-MIP backward, whose input is non-zero
// on one row per column, scatters.  Both sum every raw sample's terms in
// ascending j, skipping zero weights.
#include <algorithm>
#include <climits>
#include <cmath>

#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kThreadsX = 32;

// Search window of columns j whose tent can reach plane n in row k.
__device__ __forceinline__ void j_window(const PlanView& v, Split b, int n, int& jlo, int& jhi) {
  const float bk = (float)b.i + b.f;
  const float lo = (float)v.J0 + ((float)n - 1.0f + bk) * v.rinv;
  const float hi = (float)v.J0 + ((float)n + 1.0f + bk) * v.rinv;
  jlo = max(0, (int)floorf(lo) - 2);
  jhi = min(v.ny - 1, (int)ceilf(hi) + 2);
}

// ---------------------------------------------------------------- z-MIP backward
//
// The z-MIP gradient reaches the raw grid only through the arg-max row of
// each (j, x): at most 2 ny nx of the nscan nrows ncols raw samples are
// non-zero.  So the output is zero-filled at copy bandwidth and each (j, x)
// then fills the one or two samples it feeds, (n0, k, x) with 1 - w and
// (n0 + 1, k, x) with w, k = argz[j][x].  Several columns j of one x can
// feed the same sample; its smallest such j (inside the sample's search
// window) owns it and sums every feeding column in ascending j (the
// transpose's terms, in the adjoint's order), without atomics.

constexpr int kScX = 32;  // lanes along x (coalesced argz / g reads)
constexpr int kScY = 8;   // columns j per CTA (one per warp)

// Weight of column jj for raw plane n of row b (0 when it does not feed it).
__device__ __forceinline__ float feed_weight(const PlanView& v, Split b, int jj, int n) {
  int n0;
  float w;
  plane_weight(v.A[jj], b, v.linear, n0, w);
  if (n0 == n) return 1.0f - w;
  if (n0 + 1 == n) return w;
  return 0.0f;
}

// A warp is one column j and 32 consecutive x.  Its lanes' arg-max rows
// differ, and so do their search windows; the window scans therefore run
// over offsets d from j, with warp-uniform trip counts (the warp's largest
// window reach), so that every argz / g load is one coalesced row access and
// the lanes stay converged.
__global__ void __launch_bounds__(kScX* kScY)
k_mip_scatter(PlanView v, const float* __restrict__ g, const int32_t* __restrict__ argz, float* __restrict__ g_raw) {
  const int x = blockIdx.x * kScX + threadIdx.x;
  const int j = blockIdx.y * kScY + threadIdx.y;  // warp-uniform
  if (j >= v.ny) return;                          // whole warp
  const bool in = x < v.nx;
  const int k = in ? __ldg(argz + (size_t)j * v.nx + x) : -1;
  const bool live = k >= 0 && k < v.nz;  // out-of-range rows feed no raw sample
  const Split b = v.B[live ? k : 0];
  int n0 = 0;
  float w = 0.0f;
  plane_weight(v.A[j], b, v.linear, n0, w);
  // target t: plane n0 + t with weight wt[t]; own[t] while j may own it
  const float wt[2] = {1.0f - w, w};
  bool own[2];
  int lo[2], hi[2];
  int back = 0, fwd = 0;
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const int n = n0 + t;
    own[t] = live && n >= 0 && n < v.nscan && wt[t] != 0.0f;
    lo[t] = hi[t] = j;
    if (own[t]) {
      j_window(v, b, n, lo[t], hi[t]);
      own[t] = j >= lo[t] && j <= hi[t];
    }
    if (own[t]) {
      back = max(back, j - lo[t]);
      fwd = max(fwd, hi[t] - j);
    }
  }
  back = __reduce_max_sync(0xffffffffu, back);
  fwd = __reduce_max_sync(0xffffffffu, fwd);
  const int32_t* az = argz + x;
  const float* gz = g + x;
  // j owns plane n unless a smaller column of the window feeds it too
#pragma unroll 1
  for (int d = 1; d <= back; ++d) {
    const int jj = j - d;
    const bool c0 = own[0] && jj >= lo[0], c1 = own[1] && jj >= lo[1];
    if ((c0 || c1) && __ldg(az + (size_t)jj * v.nx) == k) {
      const float f0 = feed_weight(v, b, jj, n0), f1 = feed_weight(v, b, jj, n0 + 1);
      if (c0 && f0 != 0.0f) own[0] = false;
      if (c1 && f1 != 0.0f) own[1] = false;
    }
  }
  const float gj = (own[0] || own[1]) ? __ldg(gz + (size_t)j * v.nx) : 0.0f;
  float acc[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) acc[t] = fmaf(wt[t], gj, 0.0f);
  // the owner sums every feeding column in ascending j
#pragma unroll 1
  for (int d = 1; d <= fwd; ++d) {
    const int jj = j + d;
    const bool c0 = own[0] && jj <= hi[0], c1 = own[1] && jj <= hi[1];
    if ((c0 || c1) && __ldg(az + (size_t)jj * v.nx) == k) {
      const float gv = __ldg(gz + (size_t)jj * v.nx);
      const float f0 = feed_weight(v, b, jj, n0), f1 = feed_weight(v, b, jj, n0 + 1);
      if (c0 && f0 != 0.0f) acc[0] = fmaf(f0, gv, acc[0]);
      if (c1 && f1 != 0.0f) acc[1] = fmaf(f1, gv, acc[1]);
    }
  }
#pragma unroll
  for (int t = 0; t < 2; ++t)
    if (own[t]) g_raw[((size_t)(n0 + t) * v.nrows + k) * v.ncols + x] = acc[t];
}

__global__ void k_fill_zero(float* __restrict__ p, long long n, int vec_ok) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec_ok) {
    float4* q = reinterpret_cast<float4*>(p);
    const long long n4 = n / 4;
    for (; i < n4; i += stride) q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  for (; i < n; i += stride) p[i] = 0.0f;
}

// ------------------------------------------------------- adjoint, walking j
//
// A warp owns kWalkPlanes consecutive raw planes [na, nb) of one row k, its
// lanes 4 columns x each.  It walks the output columns j that can feed those
// planes once, in ascending j, reading each V[k][j][x..x+3] once and adding
// it into the two planes its tent touches.  n0(j, k) never decreases along
// j, so the planes complete in order: the warp holds two accumulators
// (planes p and p + 1) and stores a plane as soon as the walk has passed it.
// A plane's sum runs over its window's columns in ascending j, zero weights
// skipped.  Control flow is uniform across the warp (n0 and w depend on j
// and k only), and every load and store is one row of the warp's lanes.
constexpr int kWalkPlanes = 16;
constexpr int kWalkWarps = 4;
constexpr int kWalkUnroll = 2;

template <typename T, typename Acc, int VEC>
__device__ __forceinline__ void walk_store(const PlanView& v, T* __restrict__ raw, int k, int x0, bool vec, int lim,
                                           int n, const Acc (&acc)[VEC]) {
  T* op = raw + ((size_t)n * v.nrows + k) * v.ncols + x0;
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

template <typename T, typename Acc, int VEC>
__global__ void __launch_bounds__(kThreadsX* kWalkWarps)
k_adjoint_walk(PlanView v, const T* __restrict__ vol, T* __restrict__ raw, int xtiles, int vec_ok) {
  const int k = blockIdx.x / xtiles;
  const int xt = blockIdx.x - k * xtiles;
  const int x0 = (xt * kThreadsX + threadIdx.x) * VEC;
  const int na = (blockIdx.y * kWalkWarps + threadIdx.y) * kWalkPlanes;
  if (x0 >= v.nx || na >= v.nscan) return;
  const int nb = min(na + kWalkPlanes, v.nscan);
  const int lim = v.nx - x0;
  const bool vec = vec_ok && lim >= VEC;
  const Split b = v.B[k];
  int jlo, jhi, dummy;
  j_window(v, b, na, jlo, dummy);
  j_window(v, b, nb - 1, dummy, jhi);
  const Acc zero[VEC] = {};
  Acc lo[VEC], hi[VEC];  // planes p and p + 1
#pragma unroll
  for (int i = 0; i < VEC; ++i) lo[i] = hi[i] = Acc(0);
  int p = na - 1;  // no plane of [na, nb) below p + 1 holds a contribution yet
  int nw = na;     // next plane of [na, nb) to store
  // store plane q (when it is this warp's) after zeros for any skipped planes
  auto flush = [&](int q, const Acc(&acc)[VEC]) {
    if (q < na || q >= nb) return;
    for (; nw < q; ++nw) walk_store<T, Acc, VEC>(v, raw, k, x0, vec, lim, nw, zero);
    walk_store<T, Acc, VEC>(v, raw, k, x0, vec, lim, q, acc);
    nw = q + 1;
  };
  const T* vp = vol + (size_t)k * v.ny * v.nx + x0;
  // kWalkUnroll columns per step: their weights first, then their loads (all
  // in flight together), then their terms in ascending j
#pragma unroll 1
  for (int j0 = jlo; j0 <= jhi; j0 += kWalkUnroll) {
    int n0s[kWalkUnroll];
    Acc ws[kWalkUnroll], val[kWalkUnroll][VEC];
    bool tl[kWalkUnroll], th[kWalkUnroll];
#pragma unroll
    for (int u = 0; u < kWalkUnroll; ++u) {
      const int j = j0 + u;
      n0s[u] = INT_MIN;
      ws[u] = Acc(0);
      tl[u] = th[u] = false;
      if (j <= jhi) {
        plane_weight_t<Acc>(v.A[j], b, v.linear, n0s[u], ws[u]);
        const int n0 = n0s[u];
        tl[u] = n0 >= na && n0 < nb && Acc(1) - ws[u] != Acc(0);
        th[u] = n0 + 1 >= na && n0 + 1 < nb && ws[u] != Acc(0);
      }
      if (tl[u] || th[u]) load_vec<T, VEC, Acc>(vp + (size_t)j * v.nx, vec, lim, val[u]);
    }
#pragma unroll
    for (int u = 0; u < kWalkUnroll; ++u) {
      const int n0 = n0s[u];
      if (n0 == INT_MIN) break;  // past jhi
      if (n0 < p) {  // only before the first plane of [na, nb): n0 never decreases along j
        if (n0 + 1 >= na) atomicOr(v.err, kErrOrder);
        continue;
      }
      if (n0 > p) {
        flush(p, lo);
        if (n0 == p + 1) {
#pragma unroll
          for (int i = 0; i < VEC; ++i) {
            lo[i] = hi[i];
            hi[i] = Acc(0);
          }
        } else {
          flush(p + 1, hi);
#pragma unroll
          for (int i = 0; i < VEC; ++i) lo[i] = hi[i] = Acc(0);
        }
        p = n0;
      }
      if (tl[u]) {
        const Acc wl = Acc(1) - ws[u];
#pragma unroll
        for (int i = 0; i < VEC; ++i) lo[i] = fma(wl, val[u][i], lo[i]);
      }
      if (th[u]) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) hi[i] = fma(ws[u], val[u][i], hi[i]);
      }
    }
  }
  flush(p, lo);
  flush(p + 1, hi);
  for (; nw < nb; ++nw) walk_store<T, Acc, VEC>(v, raw, k, x0, vec, lim, nw, zero);
}

template <typename T, typename Acc, int VEC>
opm_status run_walk(const opm_plan* p, const T* src, T* dst, cudaStream_t s) {
  const PlanView& v = p->view;
  const int xtiles = (v.nx + kThreadsX * VEC - 1) / (kThreadsX * VEC);
  const long long gx = (long long)xtiles * v.nz;
  const long long groups = (v.nscan + kWalkPlanes - 1) / kWalkPlanes;
  const long long gy = (groups + kWalkWarps - 1) / kWalkWarps;
  if (gx > 0x7fffffffLL || gy > 65535) return fail(OPM_ERR_UNSUPPORTED, "adjoint grid exceeds launch limits");
  const int vec_ok = (v.nx % VEC == 0) && ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0);
  k_adjoint_walk<T, Acc, VEC><<<dim3((unsigned)gx, (unsigned)gy), dim3(kThreadsX, kWalkWarps), 0, s>>>(
      v, src, dst, xtiles, vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_adjoint_walk");
}

}  // namespace

opm_status launch_adjoint(const opm_plan* p, const void* vol, void* raw_out, opm_dtype t,
                          cudaStream_t s) {
  if (t == OPM_F32)
    return run_walk<float, float, 4>(p, static_cast<const float*>(vol), static_cast<float*>(raw_out), s);
  if (t == OPM_F64)
    return run_walk<double, double, 2>(p, static_cast<const double*>(vol), static_cast<double*>(raw_out), s);
  return fail(OPM_ERR_UNSUPPORTED, "adjoint dtype");
}

opm_status launch_mip_backward(const opm_plan* p, const float* g, const int32_t* argz,
                               float* g_raw, cudaStream_t s) {
  const PlanView& v = p->view;
  const long long nraw = (long long)v.nscan * v.nrows * v.ncols;
  const int vec_ok = (nraw % 4 == 0) && ((uintptr_t)g_raw % 16 == 0);
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  const long long want = ((vec_ok ? nraw / 4 : nraw) + 255) / 256;
  const int zgrid = (int)std::max(1LL, std::min<long long>(want, (long long)nsm * 8));
  k_fill_zero<<<zgrid, 256, 0, s>>>(g_raw, nraw, vec_ok);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch k_fill_zero");
  const long long gx = (v.nx + kScX - 1) / kScX, gy = (v.ny + kScY - 1) / kScY;
  if (gx > 0x7fffffffLL || gy > 65535) return fail(OPM_ERR_UNSUPPORTED, "MIP backward grid exceeds launch limits");
  if (gx == 0 || gy == 0) return OPM_OK;
  k_mip_scatter<<<dim3((unsigned)gx, (unsigned)gy), dim3(kScX, kScY), 0, s>>>(v, g, argz, g_raw);
  e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_mip_scatter");
}

}  // namespace opm
