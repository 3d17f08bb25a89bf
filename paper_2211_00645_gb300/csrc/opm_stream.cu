// Plane-by-plane live view: the projections of a stack accumulated one scan
// plane pair at a time, as the camera delivers frames (the rolling update of
// Fig. 4a).  The call for the pair (n, n + 1) evaluates exactly the voxels
// whose lower interpolation plane is n, V = (1 - w) R~[n] + w R~[n + 1], and
// folds them into the z-MIP, z-sum and y-MIP.  Every voxel has one lower
// plane, so the calls for n = -1 .. nscan - 1 cover the volume once; the
// per-voxel arithmetic (plane, weight, FMA on the plane difference) is the
// fast projection's, so the z-MIP and y-MIP end bit-identical to it.
#include <algorithm>

#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kSVec = 4;         // columns x per thread
constexpr int kSLanesX = 32;     // threads along x (one warp): 128 columns per CTA
constexpr int kSRowsCta = 8;     // camera rows per CTA, one warp each
constexpr int kSTileJ = 32;      // columns j of the CTA's shared z-MIP tile
constexpr int kSearchSteps = 64; // bound on the column search of one row

__global__ void k_stream_zero(float* zmip, float* zsum, long long nj, float* ymip, long long nk) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nj; i += stride) {
    if (zmip) zmip[i] = 0.0f;
    if (zsum) zsum[i] = 0.0f;
  }
  if (ymip)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += stride) ymip[i] = 0.0f;
}

// Loads this thread's kSVec columns of camera row k of one plane (zeros for
// a missing plane or columns past the edge).
__device__ __forceinline__ void load_row(const uint16_t* __restrict__ plane, const PlanView& v, int k, int x0,
                                         bool vec, float (&out)[kSVec]) {
#pragma unroll
  for (int i = 0; i < kSVec; ++i) out[i] = 0.0f;
  if (!plane) return;
  const uint16_t* p = plane + (size_t)k * v.ncols + x0;
  if (vec) {
    const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    out[0] = (float)(u.x & 0xFFFFu);
    out[1] = (float)(u.x >> 16);
    out[2] = (float)(u.y & 0xFFFFu);
    out[3] = (float)(u.y >> 16);
  } else {
#pragma unroll
    for (int i = 0; i < kSVec; ++i)
      if (x0 + i < v.nx) out[i] = (float)__ldg(p + i);
  }
}

// A CTA covers kSRowsCta consecutive camera rows (one warp each, blockIdx.y)
// and kSLanesX x kSVec columns x (blockIdx.x).  The columns j of row k whose
// lower plane is n form one run; it is found from an FP32 estimate and
// corrected with the exact split-table arithmetic.  The runs move up in j
// with k (n0 grows with j and falls with k), so the CTA's rows share a
// narrow band of columns j: their z-MIP values meet in a shared tile of
// kSTileJ columns from the first row's run start (shared atomic max), and
// the tile goes to the global z-MIP once per (j, x) at the end.  Voxels past
// the tile take the global atomic directly.  uint16 voxels are >= 0 and the
// outputs start at 0, so a zero left in the tile is skipped: the maxima are
// the same bits as one global atomic per voxel.
__global__ void __launch_bounds__(kSLanesX * kSRowsCta)
k_stream_pair(PlanView v, const uint16_t* __restrict__ lo, const uint16_t* __restrict__ hi, int n, float* zmip,
              float* zsum, float* ymip, int vec_ok) {
  __shared__ float zt[kSTileJ][kSLanesX * kSVec];
  __shared__ int jbase_s;
  const int lane = threadIdx.x & 31, wrow = threadIdx.x >> 5;
  const int k = blockIdx.y * kSRowsCta + wrow;
  const int xl = lane * kSVec;
  const int x0 = blockIdx.x * (kSLanesX * kSVec) + xl;
  for (int i = threadIdx.x; i < kSTileJ * kSLanesX * kSVec; i += blockDim.x) (&zt[0][0])[i] = 0.0f;
  // first column with lower plane >= n: estimate, then walk (bounded)
  int j = 0, n0 = 0, steps = 0;
  float w = 0.0f;
  const bool row_ok = k < v.nz;
  Split b{0, 0.0f};
  if (row_ok) {
    b = v.B[k];
    const float half = v.linear ? 0.0f : 0.5f;
    const float est = (float)v.J0 + ((float)n - half + (float)b.i + b.f) * v.rinv;
    j = (int)fminf(fmaxf(floorf(est), 0.0f), (float)(v.ny - 1));
    while (j > 0 && steps < kSearchSteps) {
      plane_weight(v.A[j - 1], b, v.linear, n0, w);
      if (n0 < n) break;
      --j;
      ++steps;
    }
    while (j < v.ny && steps < kSearchSteps) {
      plane_weight(v.A[j], b, v.linear, n0, w);
      if (n0 >= n) break;
      ++j;
      ++steps;
    }
  }
  const bool found = row_ok && steps < kSearchSteps;
  if (row_ok && !found && lane == 0) atomicOr(v.err, kErrSearch);
  if (wrow == 0) jbase_s = j;  // the first row's run start (row 0 of a CTA always exists)
  __syncthreads();
  const int jbase = jbase_s;
  if (found && x0 < v.nx) {
    float a[kSVec], d[kSVec];
    const bool vec = vec_ok && x0 + kSVec <= v.nx;
    load_row(lo, v, k, x0, vec, a);
    load_row(hi, v, k, x0, vec, d);
#pragma unroll
    for (int i = 0; i < kSVec; ++i) d[i] = d[i] - a[i];  // exact: integers below 2^24
    float ym[kSVec];
#pragma unroll
    for (int i = 0; i < kSVec; ++i) ym[i] = 0.0f;  // uint16 voxels are >= 0
    bool any = false;
#pragma unroll 1
    for (; j < v.ny; ++j) {
      plane_weight(v.A[j], b, v.linear, n0, w);
      if (n0 != n) break;
      any = true;
      const int jt = j - jbase;  // >= 0: runs move up with k
      const bool in_tile = jt >= 0 && jt < kSTileJ;
      const size_t row = (size_t)j * v.nx + x0;
#pragma unroll
      for (int i = 0; i < kSVec; ++i) {
        if (x0 + i >= v.nx) break;
        const float val = fmaf(w, d[i], a[i]);
        ym[i] = fmaxf(ym[i], val);
        if (zmip) {
          if (in_tile)
            atomicMax(reinterpret_cast<int*>(&zt[jt][xl + i]), __float_as_int(val));
          else
            atomicMax(reinterpret_cast<int*>(zmip + row + i), __float_as_int(val));
        }
        if (zsum) atomicAdd(zsum + row + i, val);
      }
    }
    if (ymip && any) {
      float* yr = ymip + (size_t)k * v.nx + x0;
#pragma unroll
      for (int i = 0; i < kSVec; ++i)
        if (x0 + i < v.nx) yr[i] = fmaxf(yr[i], ym[i]);  // one thread per (k, x) in this launch
    }
  }
  if (!zmip) return;
  __syncthreads();
  const int xb = blockIdx.x * (kSLanesX * kSVec);
  for (int i = threadIdx.x; i < kSTileJ * kSLanesX * kSVec; i += blockDim.x) {
    const int jt = i / (kSLanesX * kSVec), xx = i % (kSLanesX * kSVec);
    const float val = (&zt[0][0])[i];
    if (val != 0.0f && jbase + jt < v.ny && xb + xx < v.nx)
      atomicMax(reinterpret_cast<int*>(zmip + (size_t)(jbase + jt) * v.nx + xb + xx), __float_as_int(val));
  }
}

// out[i] = max(a[i], b[i]) over n FP32 values (out may alias a or b):
// the combine of the sliding view's partial projections.  Four values per
// thread when all three arrays are 16-byte aligned and n is a multiple of 4.
__global__ void __launch_bounds__(256)
k_max_combine(float* out, const float* a, const float* b, long long n, int vec) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const long long n4 = n / 4;
    for (; i < n4; i += stride) {
      const float4 x = reinterpret_cast<const float4*>(a)[i];
      const float4 y = reinterpret_cast<const float4*>(b)[i];
      reinterpret_cast<float4*>(out)[i] =
          make_float4(fmaxf(x.x, y.x), fmaxf(x.y, y.y), fmaxf(x.z, y.z), fmaxf(x.w, y.w));
    }
  } else {
    for (; i < n; i += stride) out[i] = fmaxf(a[i], b[i]);
  }
}

}  // namespace

opm_status launch_stream_begin(const opm_plan* p, float* zmip, float* zsum, float* ymip, cudaStream_t s) {
  const PlanView& v = p->view;
  k_stream_zero<<<4 * 152, 256, 0, s>>>(zmip, zsum, (long long)v.ny * v.nx, ymip, (long long)v.nz * v.nx);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_stream_zero");
}

opm_status launch_stream_pair(const opm_plan* p, const uint16_t* lo, const uint16_t* hi, int n, float* zmip,
                              float* zsum, float* ymip, cudaStream_t s) {
  const PlanView& v = p->view;
  const int xblocks = (v.nx + kSLanesX * kSVec - 1) / (kSLanesX * kSVec);
  if (v.nz > 65535) return fail(OPM_ERR_UNSUPPORTED, "more than 65535 camera rows");
  const int vec_ok = (v.ncols % kSVec == 0) && ((uintptr_t)lo % 8 == 0) && ((uintptr_t)hi % 8 == 0);
  const int rblocks = (v.nz + kSRowsCta - 1) / kSRowsCta;
  k_stream_pair<<<dim3(xblocks, rblocks), kSLanesX * kSRowsCta, 0, s>>>(v, lo, hi, n, zmip, zsum, ymip, vec_ok);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_stream_pair");
}

}  // namespace opm

namespace opm {
namespace {

opm_status launch_max_combine(float* out, const float* a, const float* b, int64_t n, cudaStream_t s) {
  if (n == 0) return OPM_OK;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device query (max combine)");
  const int vec = (n % 4 == 0) && ((uintptr_t)out % 16 == 0) && ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0);
  const long long work = vec ? n / 4 : n;
  const long long blocks = std::min<long long>((work + 255) / 256, (long long)std::max(nsm, 1) * 8);
  k_max_combine<<<(unsigned)blocks, 256, 0, s>>>(out, a, b, (long long)n, vec);
  e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_max_combine");
}

}  // namespace

// The sliding view after frame m of the current stack has been written to
// stack[m] (frames 0..m new, m+1..nscan-1 the previous stack's).  Each
// projection buffer is one z-MIP [ny][nx] followed by one y-MIP [nz][nx];
// `run` holds the maximum of the new stack's complete pairs, slot q of
// `slots` the previous stack's suffix maximum over its pairs q..nscan-1
// until the new stack's pair q replaces it.  The maximum is associative and
// exact, so `view` ends equal to the projection of the whole buffer.
opm_status launch_sliding_push(const opm_plan* p, const uint16_t* stack, int m, float* run, float* slots,
                               float* view, cudaStream_t s) {
  const PlanView& v = p->view;
  const int N = v.nscan;
  const size_t zn = (size_t)v.ny * v.nx, per = zn + (size_t)v.nz * v.nx;
  const size_t frame = (size_t)v.nrows * v.ncols;
  auto F = [&](int n) { return stack + (size_t)n * frame; };
  auto slot = [&](int q) { return slots + (size_t)q * per; };
  opm_status st = OPM_OK;
  // pair q (frames q, q + 1 of the new stack) into slot q, then into run
  auto pair_into_slot = [&](int q) {
    float* b = slot(q);
    opm_status r = launch_stream_begin(p, b, nullptr, b + zn, s);
    if (r == OPM_OK) r = launch_stream_pair(p, F(q), q + 1 < N ? F(q + 1) : nullptr, q, b, nullptr, b + zn, s);
    if (r == OPM_OK) r = launch_max_combine(run, run, b, (int64_t)per, s);
    return r;
  };
  if (m == 0) {  // pair -1: the new stack's first frame alone
    st = launch_stream_begin(p, run, nullptr, run + zn, s);
    if (st == OPM_OK) st = launch_stream_pair(p, nullptr, F(0), -1, run, nullptr, run + zn, s);
  } else if (m == 1) {  // pair 0 is never read from a slot: straight into run
    st = launch_stream_pair(p, F(0), F(1), 0, run, nullptr, run + zn, s);
  } else {
    st = pair_into_slot(m - 1);
  }
  if (st != OPM_OK) return st;
  if (m == N - 1) {  // the last frame closes the stack, then the next suffixes
    st = pair_into_slot(N - 1);
    if (st == OPM_OK) st = launch_max_combine(view, run, run, (int64_t)per, s);
    for (int q = N - 2; q >= 1 && st == OPM_OK; --q) st = launch_max_combine(slot(q), slot(q), slot(q + 1), (int64_t)per, s);
    return st;
  }
  // new pairs, the previous stack's pairs m + 1 .. N - 1, then the mixed pair m
  st = launch_max_combine(view, run, slot(m + 1), (int64_t)per, s);
  if (st == OPM_OK) st = launch_stream_pair(p, F(m), F(m + 1), m, view, nullptr, view + zn, s);
  return st;
}

}  // namespace opm

using namespace opm;

extern "C" opm_status opm_max_combine(float* out, const float* a, const float* b, int64_t n, void* stream) {
  if (!out || !a || !b) return fail(OPM_ERR_INVALID_ARG, "out, a and b must be non-NULL");
  if (n < 0) return fail(OPM_ERR_INVALID_ARG, "n must be >= 0");
  return launch_max_combine(out, a, b, n, static_cast<cudaStream_t>(stream));
}
