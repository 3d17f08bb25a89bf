// Batched live view: persistent launches of the projection kernels over
// many stacks, channels and ROIs of uneven sizes.
//
// The host turns every item into a TMA descriptor (its raw pointer and
// pitches, so a channel can be a strided ROI of a shared frame stack) and its
// tiles into work units.  Items the fast kernels take (a fast-eligible plan,
// z-MIP / y-MIP only) get one unit per (x-tile, j-tile, row chunk); all other
// items (pixel > step, ny < 32, z-sum or arg-max outputs) get one unit per
// (x-tile, j-tile) and whole row band, for the general kernel.  Each kind of
// unit is sorted by decreasing length and dealt onto balanced lists, one per
// persistent CTA of its kernel.  A CTA runs its kernel's producer and
// consumer loops unit after unit on one mbarrier ring whose stage counter
// carries on across units, so the next unit's slabs stream in while the
// current one drains.  The fast items run in the kernel shape the caller
// picks (opm_shape: periodic 32 x 2 or 16 x 2, fast 8 x 4) or all items in
// the general kernel; the results are the same in every shape.
//
// Work-list image (host staging and device copy share it):
//   [0, 256)            BatchHdr: unit and output-segment counts and offsets
//   [256, ...)          BatchItemDev per item (TMA descriptor, tables, outputs)
//   off_segs            BatchSeg per output to zero (y-MIPs, fast items' z-MIPs)
//   off_lists           per fast-kernel CTA list: first unit (n_lists + 1)
//   off_glists          per general-kernel CTA list: first unit
//   off_units           WorkUnit per work unit, list by list (balanced
//                       longest-first schedules, computed on the host): the
//                       fast units, then the general ones
// Only the used prefix is copied per upload.  The kernels read the counts
// from the header, so a launch captured in a CUDA graph stays valid for any
// later content with the same launch shape (kernel shape, slab depths, kinds
// of items, grids).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "opm_sched.h"
#include "opm_gen.cuh"
#include "opm_periodic.cuh"

namespace opm {

namespace {

struct BatchHdr {
  int n_units;          // units of the fast (or periodic) kernel
  int n_segs;
  unsigned off_units;
  unsigned off_segs;
  int n_lists;
  unsigned off_lists;
  int n_gunits;         // units of the general kernel
  unsigned off_gunits;
  int n_glists;
  unsigned off_glists;
  int pad[6];
};
static_assert(sizeof(BatchHdr) == 64, "hdr");

constexpr size_t kOffItems = 256;

struct BatchItemDev {  // 64-byte aligned through its tensor map
  CUtensorMap tmap;      // raw stack of the item, box {128, 1, P}
  const FastRow* frow;   // fast-kernel tables, [ntile][nz] (fast items)
  const int* fnlo;       // [ntile][nz]
  const Split* A;        // split tables (general items)
  const Split* B;
  float* zmip;
  float* ymip;
  float* zsum;
  int32_t* argz;
  int nz, ny, nx, P;
  int linear;
};
static_assert(sizeof(BatchItemDev) == 256, "item");

struct __align__(16) BatchSeg {
  float* ptr;
  long long n;
};

constexpr size_t cal256(size_t v) { return (v + 255) / 256 * 256; }

// Bytes of a work-list image with room for max_items items and max_units
// units (of both kernels together).
constexpr size_t worklist_bytes(size_t max_items, size_t max_units) {
  return kOffItems + cal256(sizeof(BatchItemDev) * max_items) + cal256(sizeof(BatchSeg) * 2 * max_items) +
         2 * cal256(sizeof(int) * (kMaxLists + 1)) + sizeof(WorkUnit) * max_units;
}

__global__ void k_batch_zero(const unsigned char* __restrict__ wl) {
  const BatchHdr hdr = *reinterpret_cast<const BatchHdr*>(wl);
  const BatchSeg* segs = reinterpret_cast<const BatchSeg*>(wl + hdr.off_segs);
  for (int sgi = blockIdx.y; sgi < hdr.n_segs; sgi += gridDim.y) {
    const BatchSeg sg = segs[sgi];
    const long long n4 = ((uintptr_t)sg.ptr % 16 == 0) ? sg.n / 4 : 0;
    float4* p4 = reinterpret_cast<float4*>(sg.ptr);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
      p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = n4 * 4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < sg.n;
         i += (long long)gridDim.x * blockDim.x)
      sg.ptr[i] = 0.0f;
  }
}

__global__ void __launch_bounds__(kThreads, 4)
k_batch_fast(const unsigned char* __restrict__ wl, int Pl, unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const BatchHdr* hdr = reinterpret_cast<const BatchHdr*>(wl);
  const FastRing ring = fast_ring(smem, Pl);
  fast_ring_init(ring);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int g = 0;
  bool ok = true;
  // this CTA's lists: l = blockIdx.x, blockIdx.x + gridDim.x, ... (one list
  // when the grid has a CTA per list), each the unit run [lists[l], lists[l + 1])
  int l = (int)blockIdx.x - (int)gridDim.x;
  int u = 0, uend = 0;
#pragma unroll 1
  while (ok) {
    if (u >= uend) {
      const int* lists = reinterpret_cast<const int*>(wl + hdr->off_lists);
      do {
        l += gridDim.x;
        if (l >= hdr->n_lists) break;
        u = lists[l];
        uend = lists[l + 1];
      } while (u >= uend);
      if (u >= uend) break;
    }
    const WorkUnit un = reinterpret_cast<const WorkUnit*>(wl + hdr->off_units)[u++];
    const BatchItemDev* items = reinterpret_cast<const BatchItemDev*>(wl + kOffItems);
    const BatchItemDev* it = items + un.item;
    FastJob jb;
    jb.tmap = &it->tmap;
    jb.nz = it->nz;
    jb.nx = it->nx;
    jb.rows = it->frow + (size_t)un.jt * jb.nz;
    jb.nlos = it->fnlo + (size_t)un.jt * jb.nz;
    jb.zmip = it->zmip;
    jb.ymip = it->ymip;
    jb.j0 = tile_j0(un.jt, it->ny);
    jb.xbase = un.xt * kX;
    jb.ks = un.ks;
    jb.ke = un.ke;
    jb.P = it->P;
    if (warp == 0) {
      // the descriptor was written by a host copy: order it for the TMA unit
      if (lane == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(jb.tmap) : "memory");
      __syncwarp();
      ok = fast_produce(jb, ring, g, err, lane);
    } else {
      ok = fast_consume(jb, ring, g, err, warp - 1, lane);
    }
  }
  if (warp == 0) fast_drain(ring, g, ok, err);
}

// The same persistent loop with the periodic kernel's producer and compute
// warps (opm_periodic.cuh), for batches whose items all belong to the plan
// family pixel/step = Pp/Qq.
// Resident CTAs per SM the periodic batch kernel is compiled for: 4 with 32
// columns j per warp (96 threads), 3 with 16 (160 threads, whose register
// share at 4 would spill).
template <int RUN>
constexpr int per_minb() { return RUN == 16 ? 3 : kPerCtasPerSm; }

template <int Pp, int Qq, int RUN>
__global__ void __launch_bounds__(per::Cfg<RUN>::kThreads, per_minb<RUN>())
k_batch_per(const unsigned char* __restrict__ wl, int Pl, unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const BatchHdr* hdr = reinterpret_cast<const BatchHdr*>(wl);
  const PerRing ring = per_ring(smem, kPerStages, Pl);
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
      const int* lists = reinterpret_cast<const int*>(wl + hdr->off_lists);
      do {
        l += gridDim.x;
        if (l >= hdr->n_lists) break;
        u = lists[l];
        uend = lists[l + 1];
      } while (u >= uend);
      if (u >= uend) break;
    }
    const WorkUnit un = reinterpret_cast<const WorkUnit*>(wl + hdr->off_units)[u++];
    const BatchItemDev* items = reinterpret_cast<const BatchItemDev*>(wl + kOffItems);
    const BatchItemDev* it = items + un.item;
    FastJob jb;
    jb.tmap = &it->tmap;
    jb.nz = it->nz;
    jb.nx = it->nx;
    jb.rows = it->frow + (size_t)un.jt * jb.nz;
    jb.nlos = it->fnlo + (size_t)un.jt * jb.nz;
    jb.zmip = it->zmip;
    jb.ymip = it->ymip;
    jb.j0 = tile_j0(un.jt, it->ny);
    jb.xbase = un.xt * kX;
    jb.ks = un.ks;
    jb.ke = un.ke;
    jb.P = it->P;
    if (warp == 0) {
      // the descriptor was written by a host copy: order it for the TMA unit
      if (lane == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(jb.tmap) : "memory");
      __syncwarp();
      ok = per_produce(jb, ring, g, err, lane);
    } else {
      ok = per_consume<RUN, Pp, Qq>(jb, ring, g, err, warp - 1, lane);
    }
  }
  if (warp == 0) per_drain(ring, g, ok, err);
}

// The general kernel's persistent loop (opm_gen.cuh) over the items the
// fast kernels do not take: one unit per (x-tile, j-tile) and whole row
// band, on one ring of slab depth Pg whose stage counter carries on across
// units.
constexpr int kGenCtasPerSm = 2;

__global__ void __launch_bounds__(kThreads, kGenCtasPerSm)
k_batch_gen(const unsigned char* __restrict__ wl, int Pg, unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const BatchHdr* hdr = reinterpret_cast<const BatchHdr*>(wl);
  const GenRing<uint16_t> ring{smem, Pg};
  gen_ring_init<uint16_t>(ring);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int g = 0;
  bool ok = true;
  int l = (int)blockIdx.x - (int)gridDim.x;
  int u = 0, uend = 0;
#pragma unroll 1
  while (ok) {
    if (u >= uend) {
      const int* lists = reinterpret_cast<const int*>(wl + hdr->off_glists);
      do {
        l += gridDim.x;
        if (l >= hdr->n_glists) break;
        u = lists[l];
        uend = lists[l + 1];
      } while (u >= uend);
      if (u >= uend) break;
    }
    const WorkUnit un = reinterpret_cast<const WorkUnit*>(wl + hdr->off_gunits)[u++];
    const BatchItemDev* it = reinterpret_cast<const BatchItemDev*>(wl + kOffItems) + un.item;
    GenJob jb;
    jb.tmap = &it->tmap;
    jb.A = it->A;
    jb.B = it->B;
    jb.linear = it->linear;
    jb.ny = it->ny;
    jb.nz = it->nz;
    jb.nx = it->nx;
    jb.P = it->P;
    jb.j0 = un.jt * kTileJ;
    jb.xbase = un.xt * kX;
    jb.ks = un.ks;
    jb.ke = un.ke;
    jb.zmip = it->zmip;
    jb.zsum = it->zsum;
    jb.ymip = it->ymip;
    jb.argz = it->argz;
    if (warp == 0) {
      if (lane == 0)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(jb.tmap) : "memory");
      __syncwarp();
      ok = gen_produce<uint16_t>(jb, ring, g, err, lane);
    } else {
      ok = gen_consume<uint16_t>(jb, ring, g, err, warp - 1, lane);
    }
  }
  if (warp == 0) gen_drain<uint16_t>(ring, g, ok, err, lane);
}

// Shared memory of a batch launch for slab depth Pl (family 0: k_batch_fast).
size_t batch_smem(int Pl, int family) { return family ? per::total(kPerStages, Pl) : fast::total(Pl); }
size_t batch_gen_smem(int Pg) { return gen::total<uint16_t>(Pg); }

PFN_cuTensorMapEncodeTiled_v12000 batch_encode_fn() {
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

struct WorkList {
  size_t used;  // bytes of the image to copy
  int n_items, n_units, n_segs, n_lists, Pl;
  int family;   // kFamilies index + 1 of the periodic kernel, or 0 (fast kernel)
  int n_gunits; // units of the general kernel
  int Pg;       // its slab depth (deepest general item)
  int run;      // columns j per compute warp of the periodic kernel (32 or 16)
  int shape;    // opm_shape the list was built for (never AUTO)
};

constexpr WorkList kEmptyWorkList = {kOffItems, 0, 0, 0, 0, 2, 0, 0, 2, kPerRun, OPM_SHAPE_PER_J32X2};

// Builds the work-list image of `items` into `stage` (room for max_items
// items and max_units units; 64-byte aligned).  Allocates nothing on
// success.  `limit_what` names the capacity in error messages.
//
// An item goes to the fast kernels when its plan is fast-eligible and it
// asks for z-MIP / y-MIP only (units: kchunk-row chunks of every tile's
// band; kchunk 0 takes the single-stack plan's rule over all fast items),
// else to the general kernel (units: whole bands; a tile with an
// empty band still gets a unit when the item has a z output, which the
// unit's epilogue writes).  Zeroed outputs: every y-MIP and the z-MIP of
// fast items (both combined by atomic max); the general kernel writes its
// z outputs outright.
opm_status build_worklist(const opm_batch_item* items, int n_items, int kchunk, int shape, int device, int nlists,
                          unsigned char* stage, int max_items, int64_t max_units, const char* limit_what,
                          WorkList* out) {
  if (n_items < 0) return fail(OPM_ERR_INVALID_ARG, "n_items must be >= 0");
  if (shape < OPM_SHAPE_AUTO || shape > OPM_SHAPE_GEN_J8X4) return fail(OPM_ERR_INVALID_ARG, "unknown shape");
  const bool gen_all = shape == OPM_SHAPE_GEN_J8X4;
  if (n_items > max_items)
    return fail(OPM_ERR_UNSUPPORTED, std::to_string(n_items) + " items exceed the " + limit_what + "'s limit of " +
                                         std::to_string(max_items));
  if (!items && n_items > 0) return fail(OPM_ERR_INVALID_ARG, "items is NULL");
  if (kchunk < 0) return fail(OPM_ERR_INVALID_ARG, "kchunk must be >= 0");
  if (!batch_encode_fn()) return fail(OPM_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is unavailable");
  if (kchunk == 0) {
    // The single-stack rule: the largest of kChunkRows .. kMinChunkRows rows
    // that gives the CTA lists at least kUnitsPerList fast units each, without
    // going past the unit capacity.  Items are validated by the pass below.
    auto nfast_units = [&](int rows) {
      int64_t n = 0;
      for (int i = 0; i < n_items; ++i) {
        const opm_batch_item& it = items[i];
        const opm_plan* p = it.plan;
        if (!p || gen_all || !plan_fast_ok(p) || it.zsum || it.argz || (!it.zmip && !it.ymip)) continue;
        const int64_t xtiles = (p->nx + kX - 1) / kX;
        for (const Band& bd : p->hBand)
          if (bd.lo < bd.hi) n += xtiles * ((bd.hi - 1) / rows - bd.lo / rows + 1);
      }
      return n;
    };
    kchunk = kChunkRows;
    while (kchunk > kMinChunkRows && (double)nfast_units(kchunk) < kUnitsPerList * nlists &&
           nfast_units(kchunk / 2) <= max_units)
      kchunk /= 2;
  }
  const size_t off_segs = cal256(kOffItems + sizeof(BatchItemDev) * (size_t)n_items);
  const size_t off_lists = cal256(off_segs + sizeof(BatchSeg) * 2 * (size_t)n_items);
  const size_t off_glists = cal256(off_lists + sizeof(int) * (size_t)(nlists + 1));
  const size_t off_units = cal256(off_glists + sizeof(int) * (size_t)(nlists + 1));
  BatchItemDev* hitems = reinterpret_cast<BatchItemDev*>(stage + kOffItems);
  BatchSeg* hsegs = reinterpret_cast<BatchSeg*>(stage + off_segs);
  int* hlists = reinterpret_cast<int*>(stage + off_lists);
  int* hglists = reinterpret_cast<int*>(stage + off_glists);
  WorkUnit* hunits = reinterpret_cast<WorkUnit*>(stage + off_units);
  int64_t nunits = 0;
  int Pl = 2, Pg = 2, nseg = 0, family = -1, nfast = 0;
  // first pass: fast items' units; second pass: general items' units after them
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n_items; ++i) {
      const opm_batch_item& it = items[i];
      const opm_plan* p = it.plan;
      if (pass == 0) {
        if (!p || !it.raw) return fail(OPM_ERR_INVALID_ARG, "item " + std::to_string(i) + ": NULL plan or raw");
        if (p->device != device)
          return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) + ": plan on another device");
        if (p->P > 256)
          return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) + ": slab depth beyond 256 planes");
        const int64_t rp = it.row_pitch ? it.row_pitch : p->ncols;
        const int64_t pp = it.plane_pitch ? it.plane_pitch : p->nrows * rp;
        if (rp < p->ncols || pp < p->nrows * rp)
          return fail(OPM_ERR_INVALID_ARG, "item " + std::to_string(i) + ": pitches smaller than the ROI");
        if ((uintptr_t)it.raw % 16 != 0 || rp % 8 != 0 || pp % 8 != 0)
          return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) +
                                               ": raw must be 16-byte aligned and pitches multiples of 8 elements");
        BatchItemDev& d = hitems[i];
        std::memset(&d, 0, sizeof(d));
        const cuuint64_t dims[3] = {(cuuint64_t)p->ncols, (cuuint64_t)p->nrows, (cuuint64_t)p->nscan};
        const cuuint64_t strides[2] = {(cuuint64_t)rp * 2, (cuuint64_t)pp * 2};
        const cuuint32_t box[3] = {(cuuint32_t)kX, 1u, (cuuint32_t)p->P};
        const cuuint32_t estr[3] = {1u, 1u, 1u};
        CUresult cr = batch_encode_fn()(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(it.raw),
                                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS)
          return fail(OPM_ERR_CUDA, "item " + std::to_string(i) + ": cuTensorMapEncodeTiled failed (" +
                                        std::to_string((int)cr) + ")");
        d.frow = p->view.frow;
        d.fnlo = p->view.fnlo;
        d.A = p->view.A;
        d.B = p->view.B;
        d.linear = p->view.linear;
        d.zmip = it.zmip;
        d.ymip = it.ymip;
        d.zsum = it.zsum;
        d.argz = it.argz;
        d.nz = (int)p->nz;
        d.ny = (int)p->ny;
        d.nx = (int)p->nx;
        d.P = p->P;
      }
      const bool fast = !gen_all && plan_fast_ok(p) && !it.zsum && !it.argz;
      if (fast != (pass == 0)) continue;
      const bool zout = it.zmip || it.zsum || it.argz;
      if (!zout && !it.ymip) continue;
      if (fast) {
        Pl = std::max(Pl, p->P);
        family = (family < 0 || family == p->family) ? p->family : 0;
        if (it.zmip) hsegs[nseg++] = BatchSeg{it.zmip, (long long)(p->ny * p->nx)};
      } else {
        Pg = std::max(Pg, p->P);
      }
      if (it.ymip) hsegs[nseg++] = BatchSeg{it.ymip, (long long)(p->nz * p->nx)};
      const int xtiles = (int)((p->nx + kX - 1) / kX);
      const int jtiles = (int)((p->ny + kTileJ - 1) / kTileJ);
      for (int jt = 0; jt < jtiles; ++jt) {
        const Band bd = p->hBand[jt];
        const int step = fast ? kchunk : std::max(1, bd.hi - bd.lo);
        const int cstart = fast ? (bd.lo / kchunk) * kchunk : bd.lo;
        const bool empty_unit = !fast && zout && bd.lo >= bd.hi;
        for (int c0 = cstart; c0 < bd.hi || (empty_unit && c0 == cstart); c0 += step) {
          const int ks = std::max(bd.lo, c0), ke = std::min(bd.hi, c0 + step);
          if (ks >= ke && !empty_unit) continue;
          if (nunits + xtiles > max_units)
            return fail(OPM_ERR_UNSUPPORTED, std::string("the items need more than the ") + limit_what +
                                                 "'s limit of " + std::to_string(max_units) +
                                                 " work units (raise kchunk or split)");
          for (int xt = 0; xt < xtiles; ++xt)
            hunits[nunits++] = WorkUnit{i, xt, jt, ks, std::max(ks, ke), 0, 0, 0};
        }
      }
    }
    if (pass == 0) nfast = (int)nunits;
  }
  const int ngen = (int)nunits - nfast;
  // balanced lists of units, one per persistent CTA, for each kernel
  schedule_lpt(hunits, nfast, nlists, hlists);
  schedule_lpt(hunits + nfast, ngen, nlists, hglists);
  BatchHdr* hdr = reinterpret_cast<BatchHdr*>(stage);
  std::memset(hdr, 0, sizeof(*hdr));
  hdr->n_units = nfast;
  hdr->n_segs = nseg;
  hdr->off_units = (unsigned)off_units;
  hdr->off_segs = (unsigned)off_segs;
  hdr->n_lists = nlists;
  hdr->off_lists = (unsigned)off_lists;
  hdr->n_gunits = ngen;
  hdr->off_gunits = (unsigned)(off_units + sizeof(WorkUnit) * (size_t)nfast);
  hdr->n_glists = nlists;
  hdr->off_glists = (unsigned)off_glists;
  out->used = off_units + sizeof(WorkUnit) * (size_t)nunits;
  out->n_items = n_items;
  out->n_units = nfast;
  out->n_segs = nseg;
  out->n_lists = nlists;
  out->Pl = Pl;
  // the fast items' kernel: the periodic one (32 or 16 columns j per warp)
  // needs one family shared by all of them, else the fast kernel runs them
  if (family < 0) family = 0;
  if (gen_all) {
    family = 0;
  } else if (shape == OPM_SHAPE_AUTO) {
    shape = family ? OPM_SHAPE_PER_J32X2 : OPM_SHAPE_FAST_J8X4;
  } else if (shape == OPM_SHAPE_FAST_J8X4 || family == 0) {
    shape = OPM_SHAPE_FAST_J8X4;
    family = 0;
  }
  out->family = family;
  out->n_gunits = ngen;
  out->Pg = Pg;
  // 16-column runs exist for the first family only; the others run 32
  if (shape == OPM_SHAPE_PER_J16X2 && family != 1) shape = OPM_SHAPE_PER_J32X2;
  out->run = shape == OPM_SHAPE_PER_J16X2 ? 16 : kPerRun;
  out->shape = shape;
  return OPM_OK;
}

// Rows of the zero kernel's grid: its blocks stride over the segments the
// header lists, so one grid shape serves every content.
constexpr int kZeroRows = 32;

template <int F>
void launch_batch_per(const unsigned char* dev_wl, const WorkList& wl, int grid, unsigned* err, cudaStream_t s) {
  if constexpr (F < kNumFamilies) {
    if (wl.family - 1 != F) return launch_batch_per<F + 1>(dev_wl, wl, grid, err, s);
    constexpr int Pp = kFamilies[F].p, Qq = kFamilies[F].q;
    const size_t smem = batch_smem(wl.Pl, wl.family);
    if constexpr (F == 0) {  // 16-column runs are compiled for the first family only
      if (wl.run == 16) {
        k_batch_per<Pp, Qq, 16><<<grid, per::Cfg<16>::kThreads, smem, s>>>(dev_wl, wl.Pl, err);
        return;
      }
    }
    k_batch_per<Pp, Qq, kPerRun><<<grid, per::Cfg<kPerRun>::kThreads, smem, s>>>(dev_wl, wl.Pl, err);
  }
}

// Zero kernel, then the fast (or periodic) kernel's `grid` persistent CTAs
// when the list has fast units, then the general kernel's `ggrid` CTAs when
// it has general units, all on `s`.
cudaError_t launch_worklist(const unsigned char* dev_wl, const WorkList& wl, int grid, int ggrid, unsigned* err,
                            cudaStream_t s) {
  k_batch_zero<<<dim3(64, kZeroRows), 256, 0, s>>>(dev_wl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (grid > 0) {
    if (wl.family)
      launch_batch_per<0>(dev_wl, wl, grid, err, s);
    else
      k_batch_fast<<<grid, kThreads, fast::total(wl.Pl), s>>>(dev_wl, wl.Pl, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (ggrid > 0) {
    k_batch_gen<<<ggrid, kThreads, batch_gen_smem(wl.Pg), s>>>(dev_wl, wl.Pg, err);
    e = cudaGetLastError();
  }
  return e;
}

// Persistent grids of the two kernels for `ctas_per_sm` (the general kernel
// takes at most kGenCtasPerSm per SM); `all` gives full grids whatever the
// unit counts, as a captured graph needs.
void batch_grids(const WorkList& wl, int nsm, int ctas_per_sm, bool all, int* grid, int* ggrid) {
  const int64_t fmax = (int64_t)nsm * ctas_per_sm;
  const int64_t gmax = (int64_t)nsm * std::min(ctas_per_sm, kGenCtasPerSm);
  *grid = wl.n_units == 0 ? 0 : (int)(all ? fmax : std::min<int64_t>(wl.n_units, fmax));
  *ggrid = wl.n_gunits == 0 ? 0 : (int)(all ? gmax : std::min<int64_t>(wl.n_gunits, gmax));
}

// Shared memory check of a prepared list against the device's opt-in limit.
opm_status batch_check_smem(const WorkList& wl, int smem_optin) {
  if (wl.n_units > 0 && (int)batch_smem(wl.Pl, wl.family) > smem_optin)
    return fail(OPM_ERR_UNSUPPORTED, "batch slab depth needs too much shared memory");
  if (wl.n_gunits > 0 && (int)batch_gen_smem(wl.Pg) > smem_optin)
    return fail(OPM_ERR_UNSUPPORTED, "general items' slab depth needs too much shared memory");
  return OPM_OK;
}

template <typename K>
cudaError_t set_kernel_smem(K kern, int smem_optin) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

template <int F>
cudaError_t set_per_attrs(int smem_optin) {
  if constexpr (F < kNumFamilies) {
    cudaError_t e = set_kernel_smem(k_batch_per<kFamilies[F].p, kFamilies[F].q, kPerRun>, smem_optin);
    if constexpr (F == 0)
      if (e == cudaSuccess) e = set_kernel_smem(k_batch_per<kFamilies[F].p, kFamilies[F].q, 16>, smem_optin);
    return e == cudaSuccess ? set_per_attrs<F + 1>(smem_optin) : e;
  }
  return cudaSuccess;
}

cudaError_t set_fast_attrs(int smem_optin) {
  cudaError_t e = set_kernel_smem(k_batch_fast, smem_optin);
  if (e == cudaSuccess) e = set_kernel_smem(k_batch_gen, smem_optin);
  return e == cudaSuccess ? set_per_attrs<0>(smem_optin) : e;
}

}  // namespace

}  // namespace opm

using namespace opm;

constexpr int kGraphCache = 4;  // captured launch shapes kept per batch

struct opm_batch {
  int max_items;
  int64_t max_units;
  int device;
  int nsm;
  int smem_optin;
  size_t bytes;          // work-list capacity; the error word follows at `bytes`
  unsigned char* dev;    // device work list + error word
  unsigned char* host;   // pinned staging
  cudaEvent_t uploaded;  // last upload of the staging has completed
  bool pending;          // an upload was recorded since the last wait
  WorkList wl;           // the prepared content
  int attr_set;
  cudaStream_t capture;  // private stream the graphs are captured on
  // Captured launches (zero kernel + persistent kernels), one per launch
  // shape: kernel shape, periodic family and run, slab depths and grids.
  struct Graph {
    cudaGraphExec_t exec;
    int key[7];
    unsigned long long used;  // launch counter at the last use
  } graphs[kGraphCache];
  unsigned long long launches;
  int graph_captures;
};

extern "C" {

opm_status opm_batch_create(int max_items, int64_t max_units, opm_batch** out) {
  if (!out) return fail(OPM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_items < 1 || max_units < 1 || max_units > (int64_t)1 << 26)
    return fail(OPM_ERR_INVALID_ARG, "need max_items >= 1 and 1 <= max_units <= 2^26");
  opm_batch* b = new (std::nothrow) opm_batch();
  if (!b) return fail(OPM_ERR_OUT_OF_MEMORY, "host allocation of the batch failed");
  b->max_items = max_items;
  b->max_units = max_units;
  b->bytes = worklist_bytes((size_t)max_items, (size_t)max_units);
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->dev), b->bytes + 256);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&b->host), b->bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemset(b->dev, 0, kOffItems);           // empty header
  if (e == cudaSuccess) e = cudaMemset(b->dev + b->bytes, 0, 256);      // error word
  if (e != cudaSuccess) {
    opm_status st = cuda_fail(e, "opm_batch_create");
    if (b->dev) cudaFree(b->dev);
    if (b->host) cudaFreeHost(b->host);
    if (b->uploaded) cudaEventDestroy(b->uploaded);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
    return st;
  }
  std::memset(b->host, 0, kOffItems);
  b->wl = kEmptyWorkList;
  *out = b;
  return OPM_OK;
}

opm_status opm_batch_destroy(opm_batch* b) {
  if (!b) return OPM_OK;
  cudaError_t e = cudaSuccess, e2;
  if (b->uploaded && (e2 = cudaEventSynchronize(b->uploaded)) != cudaSuccess) e = e2;
  for (auto& gr : b->graphs)
    if (gr.exec && (e2 = cudaGraphExecDestroy(gr.exec)) != cudaSuccess) e = e2;
  if (b->capture && (e2 = cudaStreamDestroy(b->capture)) != cudaSuccess) e = e2;
  if (b->dev && (e2 = cudaFree(b->dev)) != cudaSuccess) e = e2;
  if (b->host && (e2 = cudaFreeHost(b->host)) != cudaSuccess) e = e2;
  if (b->uploaded) cudaEventDestroy(b->uploaded);
  delete b;
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "opm_batch_destroy");
}

opm_status opm_batch_set(opm_batch* b, const opm_batch_item* items, int n_items, int kchunk, int shape) {
  if (!b || (!items && n_items > 0)) return fail(OPM_ERR_INVALID_ARG, "batch or items is NULL");
  if (n_items < 0 || n_items > b->max_items)
    return fail(OPM_ERR_INVALID_ARG, "n_items must lie in [0, max_items]");
  // the staging may still be in flight from the previous upload
  if (b->pending) {
    cudaError_t e = cudaEventSynchronize(b->uploaded);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the previous batch upload");
    b->pending = false;
  }
  WorkList wl;
  const int nlists = std::min(b->nsm * 4, kMaxLists);
  opm_status st = build_worklist(items, n_items, kchunk, shape, b->device, nlists, b->host, b->max_items,
                                 b->max_units, "batch", &wl);
  if (st != OPM_OK) {
    // leave an empty, valid image behind
    std::memset(b->host, 0, kOffItems);
    b->wl = kEmptyWorkList;
    return st;
  }
  b->wl = wl;
  return OPM_OK;
}

opm_status opm_batch_upload(opm_batch* b, void* stream) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(b->dev, b->host, b->wl.used, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(b->uploaded, s);
  if (e != cudaSuccess) return cuda_fail(e, "opm_batch_upload");
  b->pending = true;
  return OPM_OK;
}

static opm_status batch_prepare_launch(opm_batch* b, int& ctas_per_sm) {
  if (ctas_per_sm < 0 || ctas_per_sm > 4) return fail(OPM_ERR_INVALID_ARG, "ctas_per_sm must lie in [0, 4]");
  if (ctas_per_sm == 0) ctas_per_sm = 4;
  opm_status st = batch_check_smem(b->wl, b->smem_optin);
  if (st != OPM_OK) return st;
  if (!b->attr_set) {
    cudaError_t e = set_fast_attrs(b->smem_optin);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_batch_fast)");
    b->attr_set = 1;
  }
  return OPM_OK;
}

opm_status opm_batch_launch(opm_batch* b, int ctas_per_sm, void* stream) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  opm_status st = batch_prepare_launch(b, ctas_per_sm);
  if (st != OPM_OK) return st;
  int grid = 0, ggrid = 0;
  batch_grids(b->wl, b->nsm, ctas_per_sm, false, &grid, &ggrid);
  cudaError_t e = launch_worklist(b->dev, b->wl, grid, ggrid, reinterpret_cast<unsigned*>(b->dev + b->bytes),
                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "opm_batch_launch");
}

opm_status opm_batch_launch_graph(opm_batch* b, int ctas_per_sm, void* stream) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  opm_status st = batch_prepare_launch(b, ctas_per_sm);
  if (st != OPM_OK) return st;
  // full grids: every CTA reads the unit counts from the device header
  int grid = 0, ggrid = 0;
  batch_grids(b->wl, b->nsm, ctas_per_sm, true, &grid, &ggrid);
  const int key[7] = {grid ? b->wl.shape : 0, grid ? b->wl.family : 0, grid ? b->wl.run : 0,
                      grid ? b->wl.Pl : 0,    grid,                     ggrid ? b->wl.Pg : 0, ggrid};
  opm_batch::Graph* hit = nullptr;
  for (auto& gr : b->graphs)
    if (gr.exec && std::equal(key, key + 7, gr.key)) hit = &gr;
  b->launches += 1;
  if (!hit) {
    // an empty slot, else the least recently used one
    for (auto& gr : b->graphs)
      if (!hit || (hit->exec && (!gr.exec || gr.used < hit->used))) hit = &gr;
    if (hit->exec) {
      cudaError_t e = cudaGraphExecDestroy(hit->exec);
      hit->exec = nullptr;
      if (e != cudaSuccess) return cuda_fail(e, "cudaGraphExecDestroy");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t le = launch_worklist(b->dev, b->wl, grid, ggrid, reinterpret_cast<unsigned*>(b->dev + b->bytes),
                                     b->capture);
    e = cudaStreamEndCapture(b->capture, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&hit->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      hit->exec = nullptr;
      return cuda_fail(e, "capturing the batch launch");
    }
    std::copy(key, key + 7, hit->key);
    b->graph_captures += 1;
  }
  hit->used = b->launches;
  cudaError_t e = cudaGraphLaunch(hit->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "cudaGraphLaunch");
}

opm_status opm_batch_info(const opm_batch* b, int* n_items, int64_t* n_units, int* smem_bytes, int* graph_captures,
                          int* shape) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  if (shape) *shape = b->wl.shape;
  if (n_items) *n_items = b->wl.n_items;
  if (n_units) *n_units = (int64_t)b->wl.n_units + b->wl.n_gunits;
  if (smem_bytes)
    *smem_bytes = (int)std::max(b->wl.n_units ? batch_smem(b->wl.Pl, b->wl.family) : 0,
                                b->wl.n_gunits ? batch_gen_smem(b->wl.Pg) : 0);
  if (graph_captures) *graph_captures = b->graph_captures;
  return OPM_OK;
}

opm_status opm_batch_check(const opm_batch* b) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  unsigned word = 0;
  unsigned char* errp = b->dev + b->bytes;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, errp, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word) e = cudaMemset(errp, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(e, "opm_batch_check");
  if (word) return fail(OPM_ERR_INTERNAL, "device consistency check failed (bits " + std::to_string(word) + ")");
  return OPM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched live view.
//
// Same kernels and arithmetic as the opm_batch_* path, but the work list
// lives in a fixed file-scope device array instead of memory allocated per
// batch: at most kStaticItems items and kStaticUnits work units, about 2.1 MB
// of device memory reserved when the library is loaded.  The host side
// builds the list in a fixed host array of the same layout, so a successful
// call makes no allocation of any kind.
namespace opm {
namespace {

constexpr int kStaticItems = 64;
constexpr int64_t kStaticUnits = 1 << 16;
constexpr int kStaticDevices = 64;
constexpr size_t kSBytes = worklist_bytes(kStaticItems, kStaticUnits);  // error word follows

struct StaticDevice {
  bool ready;
  unsigned char* scratch;  // device address of the static array on this device
  int nsm, smem_optin;
};

alignas(256) unsigned char g_static_stage[kSBytes];  // host image of the work list
StaticDevice g_static_dev[kStaticDevices];
std::mutex g_static_mu;

}  // namespace
}  // namespace opm

static __device__ __align__(256) unsigned char g_static_scratch[opm::kSBytes + 256];

namespace opm {
namespace {

opm_status static_setup(int dev, StaticDevice** out) {
  if (dev < 0 || dev >= kStaticDevices)
    return fail(OPM_ERR_UNSUPPORTED, "device ordinal " + std::to_string(dev) + " beyond the static table");
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticDevice& d = g_static_dev[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = set_fast_attrs(d.smem_optin);
    if (e != cudaSuccess) return cuda_fail(e, "opm_batch_project_static set-up");
    if ((uintptr_t)p % 256 != 0) return fail(OPM_ERR_INTERNAL, "static scratch is not 256-byte aligned");
    d.scratch = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return OPM_OK;
}

}  // namespace
}  // namespace opm

extern "C" opm_status opm_batch_project_static(const opm_batch_item* items, int n_items, int kchunk,
                                               int ctas_per_sm, int check, void* stream) {
  if (ctas_per_sm < 0 || ctas_per_sm > 4) return fail(OPM_ERR_INVALID_ARG, "ctas_per_sm must lie in [0, 4]");
  if (ctas_per_sm == 0) ctas_per_sm = 4;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  StaticDevice* sd = nullptr;
  opm_status st = static_setup(dev, &sd);
  if (st != OPM_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The host image is one array for the whole process and is copied with a
  // pageable copy, which a stream capture cannot record: refuse capture.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  if (cap != cudaStreamCaptureStatusNone)
    return fail(OPM_ERR_UNSUPPORTED, "opm_batch_project_static cannot be captured in a CUDA graph");
  WorkList wl;
  unsigned char* dv = sd->scratch;
  unsigned* err = reinterpret_cast<unsigned*>(dv + kSBytes);
  {
    // Build and copy under the lock: threads driving other devices share
    // the host image.  The pageable copy returns once its source has been
    // staged, so the image may be rebuilt as soon as it returns.
    std::lock_guard<std::mutex> lk(g_static_mu);
    st = build_worklist(items, n_items, kchunk, OPM_SHAPE_AUTO, dev, std::min(sd->nsm * 4, kMaxLists),
                        g_static_stage, kStaticItems, kStaticUnits, "static work list", &wl);
    if (st != OPM_OK) return st;
    st = batch_check_smem(wl, sd->smem_optin);
    if (st != OPM_OK) return st;
    e = cudaMemcpyAsync(dv, g_static_stage, wl.used, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);  // error word starts at 0
  if (e != cudaSuccess) return cuda_fail(e, "opm_batch_project_static upload");
  int grid = 0, ggrid = 0;
  batch_grids(wl, sd->nsm, ctas_per_sm, false, &grid, &ggrid);
  e = launch_worklist(dv, wl, grid, ggrid, err, s);
  if (e != cudaSuccess) return cuda_fail(e, "opm_batch_project_static launch");
  if (check) {
    unsigned word = 0;
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&word, err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "opm_batch_project_static check");
    if (word) return fail(OPM_ERR_INTERNAL, "device consistency check failed (bits " + std::to_string(word) + ")");
  }
  return OPM_OK;
}
