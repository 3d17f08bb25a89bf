// Fused deskew + projection (Fig. 2d): z-MIP, z-sum, y-MIP and argmax-z of
// the deskewed volume, computed straight from the raw stack without ever
// writing the volume.
//
// Work decomposition (one CTA = 32 output columns j x 128 output columns x):
//  * Output row k of the volume reads only camera row k of the raw stack, at
//    planes n0(j,k), n0(j,k)+1 of the CTA's 32 columns: a contiguous slab of P
//    planes.  A producer warp stages that slab, {128 x, 1 row, P planes},
//    into shared memory with one TMA load per row, several rows ahead, on an
//    mbarrier ring.  Planes outside [0, nscan) arrive as TMA zero fill, which
//    is exactly the zero padding of the interpolation.
//  * Four compute warps own 8 columns j each and 4 columns x per lane.  For
//    every staged row they walk their 8 columns in order, keeping the current
//    plane pair (a, b - a) in registers: a column that moves to the next
//    plane costs one shared-memory load, so each staged raw value is
//    converted to FP32 once per warp rather than once per voxel.  Plane steps
//    come as warp-uniform bit masks from the producer.
//  * z-reductions stay in registers across rows; the y-max of each row is
//    reduced over the CTA's 32 columns in shared memory and folded into the
//    global y-MIP with one coalesced atomic max per column (max is order
//    independent, so the result is deterministic).
//  * Only rows whose band can carry non-zero weight for the tile are visited;
//    all other rows are exactly zero and enter the maxima as the value 0.
//
// Three kernels share that structure:
//  k_project_per   the periodic kernel (opm_periodic.cuh) for plans whose
//                  pixel/step is a compiled ratio p/q (1/3): the fast
//                  kernel's producer and schedule, compute warps of 32
//                  columns j x 2 columns x per lane with every plane step
//                  at a compile-time position.
//  k_project_fast  uint16 input, z-MIP and/or y-MIP, full 32-column tiles of
//                  plans whose columns never skip a plane (checked on the
//                  host with the kernel's own arithmetic).  Two rows per stage
//                  (one 3-input max per voxel pair into the z-max), packed
//                  FP32x2 FMAs, one branch per column step, and each tile's
//                  row band split into chunks (256 rows, fewer on narrow
//                  stacks) whose z-maxima combine by atomic max, which
//                  balances tiles of very different band length; a
//                  persistent grid of 4 CTAs per SM walks the chunks.
//  k_project_gen   every output (z-sum, first argmax), uint16 or FP32 input,
//                  any tile (partial last tile, column steps of several
//                  planes), one row per stage, whole band per CTA
//                  (opm_gen.cuh, shared with the batched general kernel).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "opm_gen.cuh"
#include "opm_periodic.cuh"

namespace opm {

namespace {

struct ProjArgs {
  PlanView v;
  float* zmip;
  float* zsum;
  float* ymip;
  int32_t* argz;
  int P;       // staged planes per row
  int jt0;     // first j-tile of this launch
};

// Fast kernel, persistent: one CTA per list of the plan's balanced schedule
// (units of 256 rows of one j-tile at one x-tile).  The stage counter
// carries on across a CTA's units, so the next unit's slabs stream in while
// the current one drains.
__global__ void __launch_bounds__(kThreads, 4)
k_project_fast(const __grid_constant__ CUtensorMap tmap, const ProjArgs args) {
  const PlanView& v = args.v;
  extern __shared__ __align__(128) unsigned char smem[];
  const FastRing ring = fast_ring(smem, args.P);
  fast_ring_init(ring);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int g = 0;
  bool ok = true;
  int l = (int)blockIdx.x - (int)gridDim.x;
  int u = 0, uend = 0;
#pragma unroll 1
  while (ok) {
    if (u >= uend) {
      do {
        l += gridDim.x;
        if (l >= v.nlists) break;
        u = v.lists[l];
        uend = v.lists[l + 1];
      } while (u >= uend);
      if (u >= uend) break;
    }
    const WorkUnit un = v.units[u++];
    FastJob jb;
    jb.ks = un.ks;
    jb.ke = un.ke;
    jb.tmap = &tmap;
    jb.rows = v.frow + (size_t)un.jt * v.nz;
    jb.nlos = v.fnlo + (size_t)un.jt * v.nz;
    jb.zmip = args.zmip;
    jb.ymip = args.ymip;
    jb.nz = v.nz;
    jb.nx = v.nx;
    jb.j0 = tile_j0(un.jt, v.ny);
    jb.xbase = un.xt * kX;
    jb.P = args.P;
    if (warp == 0)
      ok = fast_produce(jb, ring, g, v.err, lane);
    else
      ok = fast_consume(jb, ring, g, v.err, warp - 1, lane);
  }
  if (warp == 0) fast_drain(ring, g, ok, v.err);
}

// Periodic kernel (opm_periodic.cuh): the fast kernel's schedule, tables
// and TMA ring for plans with pixel/step = Pp/Qq, with straight-line compute
// warps per phase pair; MINB CTAs per SM, S ring stages.
template <int Pp, int Qq, int RUN, int MINB, int S>
__global__ void __launch_bounds__(per::Cfg<RUN>::kThreads, MINB)
k_project_per(const __grid_constant__ CUtensorMap tmap, const ProjArgs args) {
  const PlanView& v = args.v;
  extern __shared__ __align__(128) unsigned char smem[];
  const PerRing ring = per_ring(smem, S, args.P);
  per_ring_init(ring, per::Cfg<RUN>::kCW);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int g = 0;
  bool ok = true;
  int l = (int)blockIdx.x - (int)gridDim.x;
  int u = 0, uend = 0;
#pragma unroll 1
  while (ok) {
    if (u >= uend) {
      do {
        l += gridDim.x;
        if (l >= v.nlists) break;
        u = v.lists[l];
        uend = v.lists[l + 1];
      } while (u >= uend);
      if (u >= uend) break;
    }
    const WorkUnit un = v.units[u++];
    FastJob jb;
    jb.ks = un.ks;
    jb.ke = un.ke;
    jb.tmap = &tmap;
    jb.rows = v.frow + (size_t)un.jt * v.nz;
    jb.nlos = v.fnlo + (size_t)un.jt * v.nz;
    jb.zmip = args.zmip;
    jb.ymip = args.ymip;
    jb.nz = v.nz;
    jb.nx = v.nx;
    jb.j0 = tile_j0(un.jt, v.ny);
    jb.xbase = un.xt * kX;
    jb.P = args.P;
    if (warp == 0)
      ok = per_produce(jb, ring, g, v.err, lane);
    else
      ok = per_consume<RUN, Pp, Qq>(jb, ring, g, v.err, warp - 1, lane);
  }
  if (warp == 0) per_drain(ring, g, ok, v.err);
}

// =====================================================================
// General kernel (opm_gen.cuh): every output, uint16 or FP32, any tile, one
// row per stage, one job (a tile's whole row band) per CTA on a grid of
// (x-tile, j-tile).
template <typename T>
__global__ void __launch_bounds__(kThreads, 1)
k_project_gen(const __grid_constant__ CUtensorMap tmap, const ProjArgs args) {
  const PlanView& v = args.v;
  extern __shared__ __align__(128) unsigned char smem[];
  const GenRing<T> ring{smem, args.P};
  gen_ring_init<T>(ring);
  const int jt = blockIdx.y + args.jt0;
  const Band band = v.band[jt];
  GenJob jb;
  jb.tmap = &tmap;
  jb.A = v.A;
  jb.B = v.B;
  jb.linear = v.linear;
  jb.ny = v.ny;
  jb.nz = v.nz;
  jb.nx = v.nx;
  jb.P = args.P;
  jb.j0 = jt * kTileJ;
  jb.xbase = blockIdx.x * kX;
  jb.ks = band.lo;
  jb.ke = band.hi;
  jb.zmip = args.zmip;
  jb.zsum = args.zsum;
  jb.ymip = args.ymip;
  jb.argz = args.argz;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int g = 0;
  if (warp == 0) {
    const bool ok = gen_produce<T>(jb, ring, g, v.err, lane);
    gen_drain<T>(ring, g, ok, v.err, lane);
  } else {
    (void)gen_consume<T>(jb, ring, g, v.err, warp - 1, lane);
  }
}

// =====================================================================
// Plain kernels for shapes the TMA path does not take (unaligned rows,
// very coarse scan steps).  One thread per output pixel, every row visited.
template <typename T>
__global__ void k_zproj_plain(PlanView v, const T* __restrict__ raw, float* zmip, float* zsum,
                              int32_t* argz) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)v.ny * v.nx) return;
  const int j = (int)(idx / v.nx);
  const int x = (int)(idx - (long long)j * v.nx);
  const Split a = v.A[j];
  const size_t plane = (size_t)v.nrows * v.ncols;
  float zm = -INFINITY, zs = 0.0f;
  int az = 0;
  for (int k = 0; k < v.nz; ++k) {
    int n0;
    float w;
    plane_weight(a, v.B[k], v.linear, n0, w);
    const T* rp = raw + (size_t)k * v.ncols + x;
    const float lo = (n0 >= 0 && n0 < v.nscan) ? to_f32(rp[(size_t)n0 * plane]) : 0.0f;
    const float hi = (n0 + 1 >= 0 && n0 + 1 < v.nscan) ? to_f32(rp[(size_t)(n0 + 1) * plane]) : 0.0f;
    const float val = fmaf(w, hi - lo, lo);
    if (val > zm) {
      zm = val;
      az = k;
    }
    zs += val;
  }
  if (zmip) zmip[idx] = zm;
  if (zsum) zsum[idx] = zs;
  if (argz) argz[idx] = az;
}

template <typename T>
__global__ void k_yproj_plain(PlanView v, const T* __restrict__ raw, float* ymip) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)v.nz * v.nx) return;
  const int k = (int)(idx / v.nx);
  const int x = (int)(idx - (long long)k * v.nx);
  const Split b = v.B[k];
  const size_t plane = (size_t)v.nrows * v.ncols;
  const T* rp = raw + (size_t)k * v.ncols + x;
  float ym = -INFINITY;
  for (int j = 0; j < v.ny; ++j) {
    int n0;
    float w;
    plane_weight(v.A[j], b, v.linear, n0, w);
    const float lo = (n0 >= 0 && n0 < v.nscan) ? to_f32(rp[(size_t)n0 * plane]) : 0.0f;
    const float hi = (n0 + 1 >= 0 && n0 + 1 < v.nscan) ? to_f32(rp[(size_t)(n0 + 1) * plane]) : 0.0f;
    ym = fmaxf(ym, fmaf(w, hi - lo, lo));
  }
  ymip[idx] = ym;
}

// Initial values of the atomically combined outputs: the fast kernel folds
// its z-maxima into zeroed z-MIP rows; the y-MIP starts at 0 for uint16
// input (every voxel is >= 0) and at the plan's per-row value otherwise.
__global__ void k_init_outputs(PlanView v, float* zmip, float* ymip, int u16) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nzm = zmip ? (long long)v.ny * v.nx : 0;
  const long long nym = ymip ? (long long)v.nz * v.nx : 0;
  if (idx < nzm) zmip[idx] = 0.0f;
  if (idx < nym) ymip[idx] = u16 ? 0.0f : v.yinit[idx / v.nx];
}

// ------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

int max_optin_smem(int dev) {
  static int cache[64] = {0};
  if (dev < 0 || dev >= 64) return 0;
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      v = 48 * 1024;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

template <typename T>
opm_status encode_raw(const PlanView& v, const void* raw, int P, CUtensorMap* map) {
  std::memset(map, 0, sizeof(*map));
  const cuuint64_t dims[3] = {(cuuint64_t)v.ncols, (cuuint64_t)v.nrows, (cuuint64_t)v.nscan};
  const cuuint64_t strides[2] = {(cuuint64_t)v.ncols * sizeof(T), (cuuint64_t)v.nrows * v.ncols * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)kX, 1u, (cuuint32_t)P};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt =
      std::is_same<T, uint16_t>::value ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult cr = encode_fn()(map, dt, 3, const_cast<void*>(raw), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS)
    return fail(OPM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");
  return OPM_OK;
}

template <typename K>
opm_status prepare_kernel(K kern, int dev, int* done) {
  if (dev >= 0 && dev < 64 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin_smem(dev));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    done[dev] = 1;
  }
  return OPM_OK;
}

// The periodic kernel of the plan's family.
template <int F>
opm_status launch_per_f(const opm_plan* p, const CUtensorMap& map, const ProjArgs& args, cudaStream_t s,
                        int grid_div) {
  if constexpr (F < kNumFamilies) {
    if (p->family - 1 != F) return launch_per_f<F + 1>(p, map, args, s, grid_div);
    constexpr int Pp = kFamilies[F].p, Qq = kFamilies[F].q;
    static int done[64] = {0};
    opm_status st = prepare_kernel(k_project_per<Pp, Qq, kPerRun, kPerCtasPerSm, kPerStages>, p->device, done);
    if (st != OPM_OK) return st;
    const PlanView& v = p->view;
    const int full = std::min(v.nunits, v.nlists);
    if (full == 0) return OPM_OK;
    const int grid = std::max(1, full / std::max(1, grid_div));
    k_project_per<Pp, Qq, kPerRun, kPerCtasPerSm, kPerStages>
        <<<grid, per::Cfg<kPerRun>::kThreads, per::total(kPerStages, args.P), s>>>(map, args);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_project_per");
  } else {
    return fail(OPM_ERR_INTERNAL, "plan names an unknown periodic family");
  }
}

opm_status launch_per(const opm_plan* p, const CUtensorMap& map, const ProjArgs& args, cudaStream_t s,
                      int grid_div) {
  if (!p->view.units || !p->view.lists) return fail(OPM_ERR_INTERNAL, "plan has no fast-kernel schedule");
  return launch_per_f<0>(p, map, args, s, grid_div);
}

opm_status launch_fast(const opm_plan* p, const CUtensorMap& map, const ProjArgs& args, int tiles,
                       cudaStream_t s, int grid_div) {
  static int done[64] = {0};
  if (p->family) return launch_per(p, map, args, s, grid_div);
  opm_status st = prepare_kernel(k_project_fast, p->device, done);
  if (st != OPM_OK) return st;
  const PlanView& v = p->view;
  if (!v.units || !v.lists) return fail(OPM_ERR_INTERNAL, "plan has no fast-kernel schedule");
  const int full = std::min(v.nunits, v.nlists);
  if (full == 0) return OPM_OK;
  const int grid = std::max(1, full / std::max(1, grid_div));
  k_project_fast<<<grid, kThreads, fast::total(args.P), s>>>(map, args);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_project_fast");
}

template <typename T>
opm_status launch_gen(const opm_plan* p, const CUtensorMap& map, const ProjArgs& args, int tiles,
                      cudaStream_t s) {
  static int done[64] = {0};
  opm_status st = prepare_kernel(k_project_gen<T>, p->device, done);
  if (st != OPM_OK) return st;
  const PlanView& v = p->view;
  const int xtiles = (v.nx + kX - 1) / kX;
  if (tiles > 65535) return fail(OPM_ERR_UNSUPPORTED, "projection grid exceeds launch limits");
  dim3 grid(xtiles, tiles, 1);
  k_project_gen<T><<<grid, kThreads, gen::total<T>(args.P), s>>>(map, args);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_project_gen");
}

}  // namespace

opm_status launch_project(const opm_plan* p, const void* raw, opm_dtype in_t, float* zmip, float* zsum,
                          float* ymip, int32_t* argz, cudaStream_t s, int grid_div) {
  const PlanView& v = p->view;
  const bool u16 = in_t == OPM_U16;
  const size_t es = u16 ? 2 : 4;
  const int P = p->P;
  const int smax = max_optin_smem(p->device);
  const bool tma_ok = !p->force_generic && encode_fn() != nullptr && ((uintptr_t)raw % 16 == 0) &&
                      ((size_t)v.ncols * es) % 16 == 0 && P <= 256;
  const bool gen_ok = tma_ok && (int)(u16 ? gen::total<uint16_t>(P) : gen::total<float>(P)) <= smax;
  const bool fast = gen_ok && u16 && !zsum && !argz && p->fast_ok && v.frow &&
                    (int)(p->family ? per::total(kPerStages, P) : fast::total(P)) <= smax;

  if (!gen_ok) {
    const long long nzx = (long long)v.ny * v.nx, nyx = (long long)v.nz * v.nx;
    const int tb = 256;
    if (zmip || zsum || argz) {
      const long long nb = (nzx + tb - 1) / tb;
      if (nb > 0x7fffffffLL) return fail(OPM_ERR_UNSUPPORTED, "grid too large");
      if (u16)
        k_zproj_plain<uint16_t><<<(unsigned)nb, tb, 0, s>>>(v, static_cast<const uint16_t*>(raw), zmip, zsum, argz);
      else
        k_zproj_plain<float><<<(unsigned)nb, tb, 0, s>>>(v, static_cast<const float*>(raw), zmip, zsum, argz);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "launch k_zproj_plain");
    }
    if (ymip) {
      const long long nb = (nyx + tb - 1) / tb;
      if (nb > 0x7fffffffLL) return fail(OPM_ERR_UNSUPPORTED, "grid too large");
      if (u16)
        k_yproj_plain<uint16_t><<<(unsigned)nb, tb, 0, s>>>(v, static_cast<const uint16_t*>(raw), ymip);
      else
        k_yproj_plain<float><<<(unsigned)nb, tb, 0, s>>>(v, static_cast<const float*>(raw), ymip);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "launch k_yproj_plain");
    }
    return OPM_OK;
  }

  // initial values of the atomically combined outputs
  float* zinit = fast ? zmip : nullptr;
  if (zinit || ymip) {
    const long long n = std::max(zinit ? (long long)v.ny * v.nx : 0LL, ymip ? (long long)v.nz * v.nx : 0LL);
    const long long nb = (n + 255) / 256;
    if (nb > 0x7fffffffLL) return fail(OPM_ERR_UNSUPPORTED, "grid too large");
    k_init_outputs<<<(unsigned)nb, 256, 0, s>>>(v, zinit, ymip, u16 ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_init_outputs");
  }

  ProjArgs args;
  args.v = v;
  args.zmip = zmip;
  args.zsum = zsum;
  args.ymip = ymip;
  args.argz = argz;
  args.P = P;
  args.jt0 = 0;
  CUtensorMap map;
  opm_status st = u16 ? encode_raw<uint16_t>(v, raw, P, &map) : encode_raw<float>(v, raw, P, &map);
  if (st != OPM_OK) return st;
  const int jtiles = (v.ny + kTileJ - 1) / kTileJ;
  if (fast) return launch_fast(p, map, args, jtiles, s, grid_div);
  return u16 ? launch_gen<uint16_t>(p, map, args, jtiles, s) : launch_gen<float>(p, map, args, jtiles, s);
}

}  // namespace opm
