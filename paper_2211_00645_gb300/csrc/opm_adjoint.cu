// Adjoint of the deskew and backward pass of the z-MIP.
//
// Both apply the transpose of the interpolation map: raw sample (n, k, x)
// collects every output column j of row k whose lower plane n0(j,k) is n
// (weight 1 - w) or n - 1 (weight w), in ascending j.  The weights are
// computed with the forward kernels' own split-table formula, so the adjoint
// is the exact transpose of the map the forward kernels apply.  No atomics:
// results are bitwise reproducible.  Both kernels walk the columns j of a
// row once per block of planes and write every raw sample exactly once,
// densely: the adjoint's term for column j is vol[k][j][x], the z-MIP
// backward's is g[j][x] when argz[j][x] = k and nothing otherwise.  Every
// raw sample's terms are summed in ascending j, zero weights skipped.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

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

// ------------------------------------------------------- walking j
//
// A warp owns `PLANES` consecutive raw planes [na, nb) of one row k, its
// lanes 4 (FP32) or 2 (FP64) columns x each.  It walks the output columns j
// that can feed those planes once, in ascending j, fetching each column's
// term for its lanes' x once and adding it into the two planes its tent
// touches.  n0(j, k) never decreases along j, so the planes complete in
// order: the warp holds two accumulators (planes p and p + 1) and stores a
// plane as soon as the walk has passed it, zeros for planes nothing feeds.
// A plane's sum runs over its window's columns in ascending j, zero weights
// skipped.  Control flow is uniform across the warp (n0 and w depend on j
// and k only), and every load and store is one row of the warp's lanes.

// Term source of the adjoint: vol[k][j][x].
template <typename T, typename Acc, int VEC>
struct VolTerms {
  const T* vol;
  const T* row;  // vol[k][0][x0]
  __device__ void bind(const PlanView& v, int k, int x0) { row = vol + (size_t)k * v.ny * v.nx + x0; }
  __device__ void load(const PlanView& v, int j, bool vec, int lim, Acc (&val)[VEC]) const {
    load_vec<T, VEC, Acc>(row + (size_t)j * v.nx, vec, lim, val);
  }
};

constexpr int kWalkWarps = 4;
constexpr int kWalkUnroll = 2;
constexpr int kAdjPlanes = 16;  // planes per warp of the adjoint

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

template <typename T, typename Acc, int VEC, int PLANES, typename Src>
__global__ void __launch_bounds__(kThreadsX* kWalkWarps)
k_walk(PlanView v, Src src, T* __restrict__ raw, int xtiles, int vec_ok) {
  const int k = blockIdx.x / xtiles;
  const int xt = blockIdx.x - k * xtiles;
  const int x0 = (xt * kThreadsX + threadIdx.x) * VEC;
  const int na = (blockIdx.y * kWalkWarps + threadIdx.y) * PLANES;
  if (x0 >= v.nx || na >= v.nscan) return;
  const int nb = min(na + PLANES, v.nscan);
  const int lim = v.nx - x0;
  const bool vec = vec_ok && lim >= VEC;
  const Split b = v.B[k];
  src.bind(v, k, x0);
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
      if (tl[u] || th[u]) src.load(v, j, vec, lim, val[u]);
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

// One launch of the walk over every raw sample: grid (row k x x-tile,
// plane groups), kWalkWarps plane groups per CTA.
template <typename T, typename Acc, int VEC, int PLANES, typename Src>
opm_status run_walk(const opm_plan* p, const Src& src, T* dst, bool vec_ok, cudaStream_t s, const char* what) {
  const PlanView& v = p->view;
  const int xtiles = (v.nx + kThreadsX * VEC - 1) / (kThreadsX * VEC);
  const long long gx = (long long)xtiles * v.nz;
  const long long groups = (v.nscan + PLANES - 1) / PLANES;
  const long long gy = (groups + kWalkWarps - 1) / kWalkWarps;
  if (gx > 0x7fffffffLL || gy > 65535) return fail(OPM_ERR_UNSUPPORTED, std::string(what) + " grid exceeds launch limits");
  if (gx == 0 || gy == 0) return OPM_OK;
  k_walk<T, Acc, VEC, PLANES, Src><<<dim3((unsigned)gx, (unsigned)gy), dim3(kThreadsX, kWalkWarps), 0, s>>>(
      v, src, dst, xtiles, vec_ok ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, (std::string("launch ") + what).c_str());
}

// cuTensorMapEncodeTiled through the runtime's driver entry point.
PFN_cuTensorMapEncodeTiled_v12000 mip_encode_fn() {
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

// ---------------------------------------------------------------- z-MIP backward
//
// The z-MIP gradient reaches the raw grid only through the arg-max row of
// each (j, x): column j of x feeds raw samples (n0, k, x) with 1 - w and
// (n0 + 1, k, x) with w, k = argz[j][x], and nothing else.  The raw grid is
// cut into CTA tiles of kMipK rows x 32 columns x (one per lane) x kMipW
// kMipP-plane groups, walked by a persistent grid; each warp holds one
// plane group of the tile in shared memory, zeroed.  Per chunk of the
// columns j that can feed the tile:
//  1. the chunk's argz, g and split-table rows are staged;
//  2. each lane lists, in ascending j, the chunk's columns whose arg-max row
//     of its x falls in the tile's rows and whose lower plane n0 lies in
//     [first plane - 1, last plane], with that n0 (the warps list a quarter
//     of the chunk each, so the four lists in warp order are in ascending j);
//  3. each warp walks its lanes' lists and adds the terms of every listed
//     column that land in its planes.
// Then each warp hands its plane group to the TMA unit, which writes it out
// (clipped at the grid's edges) while the CTA goes on to its next tile:
// every raw sample is written once, densely.  Per sample the terms arrive in
// ascending j from +0, zero weights skipped: the sums of the skew adjoint
// applied to the arg-max volume.
constexpr int kMipP = 4;    // planes per warp
constexpr int kMipK = 8;    // rows per tile
constexpr int kMipW = 4;    // warps (plane groups) per CTA
constexpr int kMipJC = 80;  // columns j staged per chunk
constexpr int kMipCtasPerSm = 5;
constexpr int kMipSeg = kMipJC / kMipW;  // columns j each warp lists per chunk
constexpr int kMipTile = kMipP * kMipK * 32;  // floats per warp tile, [kMipP][kMipK][32]
// list entry: chunk row (7 bits) | row in the tile (4 bits) | n0 - first plane + 1 (5 bits)
static_assert(kMipJC % kMipW == 0 && kMipJC <= 128 && kMipK <= 16 && kMipP * kMipW <= 31, "list entry fields");

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// TMA store of a warp tile at (x, k, n) and the waits on it.
__device__ __forceinline__ void tma_store_tile(const CUtensorMap* map, const float* tile, int x, int k, int n) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
               "r"((unsigned)__cvta_generic_to_shared(tile)), "r"(x), "r"(k), "r"(n)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void tma_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void tma_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// shared memory: warp tiles, staged argz and g [kMipJC][32], split rows,
// lists [kMipW][kMipSeg][32] and their lengths [kMipW][32]
constexpr size_t mip_smem() {
  return (size_t)kMipW * kMipTile * 4 + (size_t)kMipJC * 32 * 8 + (size_t)kMipJC * sizeof(Split) +
         (size_t)kMipK * sizeof(Split) + (size_t)kMipW * kMipSeg * 32 * 2 + (size_t)kMipW * 32 * 4;
}

// `use_tma`: tiles go out through `tmap` (raw as {ncols, nrows, nscan} FP32,
// box {32, kMipK, kMipP}); otherwise with plain stores.  `aligned`: argz and
// g rows start on 16 bytes at every 32-column block.
__global__ void __launch_bounds__(32 * kMipW, kMipCtasPerSm)
k_mip_tile(const __grid_constant__ CUtensorMap tmap, PlanView v, const float* __restrict__ g,
           const int32_t* __restrict__ argz, float* __restrict__ raw, int use_tma, int aligned) {
  extern __shared__ __align__(128) float msm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* tile = msm + warp * kMipTile;
  int* sarg = reinterpret_cast<int*>(msm + kMipW * kMipTile);
  float* sg = reinterpret_cast<float*>(sarg + kMipJC * 32);
  Split* sA = reinterpret_cast<Split*>(sg + kMipJC * 32);
  Split* sB = sA + kMipJC;
  int* cnt = reinterpret_cast<int*>(sB + kMipK);       // [kMipW][32]
  unsigned short* list = reinterpret_cast<unsigned short*>(cnt + kMipW * 32);  // [kMipW][kMipSeg][32]
  const int nxb = (v.nx + 31) / 32, nkb = (v.nz + kMipK - 1) / kMipK;
  const int ntiles = nxb * nkb * ((v.nscan + kMipP * kMipW - 1) / (kMipP * kMipW));
#pragma unroll 1
  for (int tid = blockIdx.x; tid < ntiles; tid += gridDim.x) {
    const int xb = (tid % nxb) * 32;
    const int k0 = ((tid / nxb) % nkb) * kMipK, nk = min(kMipK, v.nz - k0);
    const int nc = (tid / (nxb * nkb)) * (kMipP * kMipW);  // the tile's planes [nc, nce)
    const int nce = min(nc + kMipP * kMipW, v.nscan);
    const int na = nc + warp * kMipP;                    // the warp's planes [na, nb)
    const int np = min(na + kMipP, v.nscan) - na;        // <= 0 for an idle warp
    const int x = xb + lane;
    const bool xin = x < v.nx;
    const bool full = aligned && xb + 32 <= v.nx;
    // the TMA unit has read the warp's previous tile: zero it for this one
    if (use_tma && lane == 0) tma_wait_read();
    __syncwarp();
    for (int i = lane; i < kMipTile / 4; i += 32)
      reinterpret_cast<float4*>(tile)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();  // the previous tile's lists and staged rows are consumed
    if (threadIdx.x < kMipK) sB[threadIdx.x] = v.B[k0 + min((int)threadIdx.x, nk - 1)];
    // columns that can feed the tile: n0 grows with j and falls with k, so
    // the window runs from (first row, first plane) to (last row, last plane)
    int jlo, jhi, d;
    j_window(v, v.B[k0], nc, jlo, d);
    j_window(v, v.B[k0 + nk - 1], nce - 1, d, jhi);
#pragma unroll 1
    for (int c0 = jlo; c0 <= jhi; c0 += kMipJC) {
      const int nr = min(kMipJC, jhi + 1 - c0);
      if (c0 > jlo) __syncthreads();  // the previous chunk is consumed
      // 1. stage: all copies of the chunk in flight at once, then one wait
      if (full) {
        const int q = lane & 7;  // 8 lanes per row, 4 columns each
        for (int r = warp * 4 + (lane >> 3); r < nr; r += kMipW * 4) {
          const size_t o = (size_t)(c0 + r) * v.nx + xb + 4 * q;
          cp_async16(sarg + r * 32 + 4 * q, argz + o);
          cp_async16(sg + r * 32 + 4 * q, g + o);
        }
      } else {
        for (int r = warp; r < nr; r += kMipW) {
          const size_t o = (size_t)(c0 + r) * v.nx + x;
          if (xin) {
            cp_async4(sarg + r * 32 + lane, argz + o);
            cp_async4(sg + r * 32 + lane, g + o);
          } else {
            sarg[r * 32 + lane] = -1;
          }
        }
      }
      for (int r = threadIdx.x; r < nr; r += 32 * kMipW) sA[r] = v.A[c0 + r];
      cp_async_wait_all();
      __syncthreads();
      // 2. list this warp's quarter of the chunk (rows r0 .. r1 - 1)
      {
        const int r0 = warp * kMipSeg, r1 = min(r0 + kMipSeg, nr);
        unsigned short* ls = list + warp * kMipSeg * 32 + lane;
        int c = 0;
#pragma unroll 4
        for (int r = r0; r < r1; ++r) {
          const int kk = sarg[r * 32 + lane] - k0;
          if ((unsigned)kk < (unsigned)nk) {
            int n0;
            float w;
            plane_weight(sA[r], sB[kk], v.linear, n0, w);
            const int tt = n0 - nc + 1;  // 0: the plane before the tile's first
            if (tt >= 0 && tt <= nce - nc) {
              ls[c * 32] = (unsigned short)(r | (kk << 7) | (tt << 11));
              ++c;
            }
          }
        }
        cnt[warp * 32 + lane] = c;
      }
      __syncthreads();
      // 3. this warp's planes: the listed columns, in ascending j
      if (np > 0) {
#pragma unroll 1
        for (int q = 0; q < kMipW; ++q) {
          const unsigned short* ls = list + q * kMipSeg * 32 + lane;
          const int c = cnt[q * 32 + lane];
#pragma unroll 1
          for (int e = 0; e < c; ++e) {
            const unsigned en = ls[e * 32];
            const int t = (int)(en >> 11) - 1 + nc - na;  // n0 - na
            if (t < -1 || t >= np) continue;               // neither plane of this warp
            const int r = en & 127, kk = (en >> 7) & 15;
            int n0;
            float w;
            plane_weight(sA[r], sB[kk], v.linear, n0, w);
            const float gv = sg[r * 32 + lane];
            float* p = tile + (t * kMipK + kk) * 32 + lane;
            const float wl = 1.0f - w;
            if (t >= 0 && wl != 0.0f) p[0] = fmaf(wl, gv, p[0]);
            if (t + 1 < np && w != 0.0f) p[kMipK * 32] = fmaf(w, gv, p[kMipK * 32]);
          }
        }
      }
    }
    // 4. out: the TMA unit clips the tile at the grid's edges
    if (np <= 0) continue;
    if (use_tma) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) tma_store_tile(&tmap, tile, xb, k0, na);
    } else if (xin) {
      __syncwarp();
      for (int t = 0; t < np; ++t)
        for (int kk = 0; kk < nk; ++kk)
          raw[((size_t)(na + t) * v.nrows + k0 + kk) * v.ncols + x] = tile[(t * kMipK + kk) * 32 + lane];
    }
  }
  if (use_tma && lane == 0) tma_wait_all();
}

}  // namespace

opm_status launch_adjoint(const opm_plan* p, const void* vol, void* raw_out, opm_dtype t,
                          cudaStream_t s) {
  const PlanView& v = p->view;
  const bool al = ((uintptr_t)vol % 16 == 0) && ((uintptr_t)raw_out % 16 == 0);
  if (t == OPM_F32) {
    VolTerms<float, float, 4> src{static_cast<const float*>(vol), nullptr};
    return run_walk<float, float, 4, kAdjPlanes>(p, src, static_cast<float*>(raw_out), al && v.nx % 4 == 0, s,
                                                 "k_walk (adjoint)");
  }
  if (t == OPM_F64) {
    VolTerms<double, double, 2> src{static_cast<const double*>(vol), nullptr};
    return run_walk<double, double, 2, kAdjPlanes>(p, src, static_cast<double*>(raw_out), al && v.nx % 2 == 0, s,
                                                   "k_walk (adjoint)");
  }
  return fail(OPM_ERR_UNSUPPORTED, "adjoint dtype");
}

opm_status launch_mip_backward(const opm_plan* p, const float* g, const int32_t* argz,
                               float* g_raw, cudaStream_t s) {
  const PlanView& v = p->view;
  const long long tiles = (long long)((v.nx + 31) / 32) * ((v.nz + kMipK - 1) / kMipK) *
                          ((v.nscan + kMipP * kMipW - 1) / (kMipP * kMipW));
  if (tiles == 0) return OPM_OK;
  if (tiles > 0x7fffffffLL) return fail(OPM_ERR_UNSUPPORTED, "MIP backward grid exceeds launch limits");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  static int done[64] = {0};
  if (e == cudaSuccess && dev >= 0 && dev < 64 && !done[dev]) {
    e = cudaFuncSetAttribute(k_mip_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mip_smem());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_mip_tile, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) done[dev] = 1;
  }
  if (e != cudaSuccess) return cuda_fail(e, "k_mip_tile set-up");
  // TMA stores need 16-byte raw rows; the map clips partial tiles
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  int use_tma = 0;
  if (v.ncols % 4 == 0 && (uintptr_t)g_raw % 16 == 0 && mip_encode_fn()) {
    const cuuint64_t dims[3] = {(cuuint64_t)v.ncols, (cuuint64_t)v.nrows, (cuuint64_t)v.nscan};
    const cuuint64_t strides[2] = {(cuuint64_t)v.ncols * 4, (cuuint64_t)v.nrows * v.ncols * 4};
    const cuuint32_t box[3] = {32u, (cuuint32_t)kMipK, (cuuint32_t)kMipP};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    use_tma = mip_encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, g_raw, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  const int aligned = v.nx % 4 == 0 && (uintptr_t)g % 16 == 0 && (uintptr_t)argz % 16 == 0;
  const int grid = (int)std::min<long long>(tiles, (long long)nsm * kMipCtasPerSm);
  k_mip_tile<<<grid, 32 * kMipW, mip_smem(), s>>>(map, v, g, argz, g_raw, use_tma, aligned);
  e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_mip_tile");
}

}  // namespace opm
