// Batched live view: one persistent launch of the fast projection over many
// stacks, channels and ROIs of uneven sizes.
//
// The host turns every item into a TMA descriptor (its raw pointer and
// pitches, so a channel can be a strided ROI of a shared frame stack) and
// every item's (x-tile, j-tile, row chunk) into a work unit.  Units are
// sorted by decreasing length and dealt round-robin to a grid of
// ctas_per_sm x SM persistent CTAs; each CTA runs the fast kernel's producer
// and consumer loops unit after unit on one mbarrier ring whose stage counter
// carries on across units, so the next unit's slabs stream in while the
// current one drains.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "opm_tma.cuh"

namespace opm {

namespace {

struct BatchItemDev {  // 64-byte aligned through its tensor map
  CUtensorMap tmap;      // raw stack of the item, box {128, 1, P}
  const FastRow* frow;   // plan tables, [ntile][nz]
  const int* fnlo;       // [ntile][nz]
  float* zmip;
  float* ymip;
  int nz, ny, nx, P;
};

struct __align__(16) BatchUnit {
  int item, xt, jt, ks, ke;
  int pad[3];
};

struct __align__(16) BatchSeg {
  float* ptr;
  long long n;
};

__global__ void k_batch_zero(const BatchSeg* __restrict__ segs, int nseg) {
  for (int sgi = blockIdx.y; sgi < nseg; sgi += gridDim.y) {
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
k_batch_fast(const BatchItemDev* __restrict__ items, const BatchUnit* __restrict__ units, int nunits, int Pl,
             unsigned* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const FastRing ring = fast_ring(smem, Pl);
  fast_ring_init(ring);
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int g = 0;
  bool ok = true;
#pragma unroll 1
  for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
    const BatchUnit un = units[u];
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

size_t al(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

}  // namespace opm

using namespace opm;

struct opm_batch {
  int max_items;
  int64_t max_units;
  int device;
  int nsm;
  int smem_optin;
  size_t off_units, off_segs, off_err, bytes;  // layout shared by host staging and device copy
  unsigned char* dev;   // device work list
  unsigned char* host;  // pinned staging
  cudaEvent_t uploaded; // last upload of the staging has completed
  bool pending;         // an upload was recorded since the last wait
  int n_items, n_segs, Pl;
  int64_t n_units;
  int attr_set;
};

extern "C" {

opm_status opm_batch_create(int max_items, int64_t max_units, opm_batch** out) {
  if (!out) return fail(OPM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_items < 1 || max_units < 1 || max_units > (int64_t)1 << 31)
    return fail(OPM_ERR_INVALID_ARG, "need max_items >= 1 and 1 <= max_units <= 2^31");
  opm_batch* b = new (std::nothrow) opm_batch();
  if (!b) return fail(OPM_ERR_OUT_OF_MEMORY, "host allocation of the batch failed");
  b->max_items = max_items;
  b->max_units = max_units;
  b->off_units = al(sizeof(BatchItemDev) * (size_t)max_items, 256);
  b->off_segs = b->off_units + al(sizeof(BatchUnit) * (size_t)max_units, 256);
  b->off_err = b->off_segs + al(sizeof(BatchSeg) * 2 * (size_t)max_items, 256);
  b->bytes = b->off_err + 256;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->dev), b->bytes);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&b->host), b->bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(b->dev + b->off_err, 0, 256);
  if (e != cudaSuccess) {
    opm_status st = cuda_fail(e, "opm_batch_create");
    if (b->dev) cudaFree(b->dev);
    if (b->host) cudaFreeHost(b->host);
    delete b;
    return st;
  }
  std::memset(b->host, 0, b->bytes);
  *out = b;
  return OPM_OK;
}

opm_status opm_batch_destroy(opm_batch* b) {
  if (!b) return OPM_OK;
  cudaError_t e = cudaSuccess, e2;
  if (b->uploaded && (e2 = cudaEventSynchronize(b->uploaded)) != cudaSuccess) e = e2;
  if (b->dev && (e2 = cudaFree(b->dev)) != cudaSuccess) e = e2;
  if (b->host && (e2 = cudaFreeHost(b->host)) != cudaSuccess) e = e2;
  if (b->uploaded) cudaEventDestroy(b->uploaded);
  delete b;
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "opm_batch_destroy");
}

}  // extern "C"

extern "C" {

opm_status opm_batch_set(opm_batch* b, const opm_batch_item* items, int n_items, int kchunk) {
  if (!b || (!items && n_items > 0)) return fail(OPM_ERR_INVALID_ARG, "batch or items is NULL");
  if (n_items < 0 || n_items > b->max_items)
    return fail(OPM_ERR_INVALID_ARG, "n_items must lie in [0, max_items]");
  if (kchunk < 0) return fail(OPM_ERR_INVALID_ARG, "kchunk must be >= 0");
  if (kchunk == 0) kchunk = 64;
  if (!batch_encode_fn()) return fail(OPM_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is unavailable");
  // the staging may still be in flight from the previous upload
  if (b->pending) {
    cudaError_t e = cudaEventSynchronize(b->uploaded);
    if (e != cudaSuccess) return cuda_fail(e, "waiting for the previous batch upload");
    b->pending = false;
  }
  BatchItemDev* hitems = reinterpret_cast<BatchItemDev*>(b->host);
  BatchSeg* hsegs = reinterpret_cast<BatchSeg*>(b->host + b->off_segs);
  std::vector<BatchUnit> units;
  int Pl = 2, nseg = 0;
  for (int i = 0; i < n_items; ++i) {
    const opm_batch_item& it = items[i];
    const opm_plan* p = it.plan;
    if (!p || !it.raw) return fail(OPM_ERR_INVALID_ARG, "item " + std::to_string(i) + ": NULL plan or raw");
    if (p->device != b->device)
      return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) + ": plan on another device");
    if (!plan_fast_ok(p))
      return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) +
                                           ": plan not eligible (needs pixel <= step and ny >= 32)");
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
    CUresult cr = batch_encode_fn()(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(it.raw), dims,
                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS)
      return fail(OPM_ERR_CUDA, "item " + std::to_string(i) + ": cuTensorMapEncodeTiled failed (" +
                                    std::to_string((int)cr) + ")");
    d.frow = p->view.frow;
    d.fnlo = p->view.fnlo;
    d.zmip = it.zmip;
    d.ymip = it.ymip;
    d.nz = (int)p->nz;
    d.ny = (int)p->ny;
    d.nx = (int)p->nx;
    d.P = p->P;
    Pl = std::max(Pl, p->P);
    if (it.zmip) hsegs[nseg++] = BatchSeg{it.zmip, (long long)(p->ny * p->nx)};
    if (it.ymip) hsegs[nseg++] = BatchSeg{it.ymip, (long long)(p->nz * p->nx)};
    if (!it.zmip && !it.ymip) continue;
    const int xtiles = (int)((p->nx + kX - 1) / kX);
    const int jtiles = (int)((p->ny + kTileJ - 1) / kTileJ);
    for (int jt = 0; jt < jtiles; ++jt) {
      const Band bd = p->hBand[jt];
      for (int c0 = (bd.lo / kchunk) * kchunk; c0 < bd.hi; c0 += kchunk) {
        const int ks = std::max(bd.lo, c0), ke = std::min(bd.hi, c0 + kchunk);
        if (ks >= ke) continue;
        for (int xt = 0; xt < xtiles; ++xt) units.push_back(BatchUnit{i, xt, jt, ks, ke, {0, 0, 0}});
      }
    }
  }
  if ((int64_t)units.size() > b->max_units)
    return fail(OPM_ERR_UNSUPPORTED, "batch needs " + std::to_string(units.size()) + " units, capacity " +
                                         std::to_string(b->max_units));
  // longest units first, dealt round-robin to the persistent CTAs
  std::stable_sort(units.begin(), units.end(),
                   [](const BatchUnit& a, const BatchUnit& c) { return (a.ke - a.ks) > (c.ke - c.ks); });
  if (!units.empty()) std::memcpy(b->host + b->off_units, units.data(), sizeof(BatchUnit) * units.size());
  b->n_items = n_items;
  b->n_units = (int64_t)units.size();
  b->n_segs = nseg;
  b->Pl = Pl;
  return OPM_OK;
}

opm_status opm_batch_upload(opm_batch* b, void* stream) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(b->dev, b->host, b->off_err, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(b->uploaded, s);
  if (e != cudaSuccess) return cuda_fail(e, "opm_batch_upload");
  b->pending = true;
  return OPM_OK;
}

opm_status opm_batch_launch(opm_batch* b, int ctas_per_sm, void* stream) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  if (ctas_per_sm < 0 || ctas_per_sm > 4) return fail(OPM_ERR_INVALID_ARG, "ctas_per_sm must lie in [0, 4]");
  if (ctas_per_sm == 0) ctas_per_sm = 4;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (b->n_segs > 0) {
    dim3 grid(64, std::min(b->n_segs, 65535));
    k_batch_zero<<<grid, 256, 0, s>>>(reinterpret_cast<const BatchSeg*>(b->dev + b->off_segs), b->n_segs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_batch_zero");
  }
  if (b->n_units == 0) return OPM_OK;
  const size_t smem = fast::total(b->Pl);
  if ((int)smem > b->smem_optin) return fail(OPM_ERR_UNSUPPORTED, "batch slab depth needs too much shared memory");
  if (!b->attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, b->smem_optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_batch_fast, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_batch_fast)");
    b->attr_set = 1;
  }
  const int grid = (int)std::min<int64_t>(b->n_units, (int64_t)b->nsm * ctas_per_sm);
  k_batch_fast<<<grid, kThreads, smem, s>>>(reinterpret_cast<const BatchItemDev*>(b->dev),
                                            reinterpret_cast<const BatchUnit*>(b->dev + b->off_units),
                                            (int)b->n_units, b->Pl,
                                            reinterpret_cast<unsigned*>(b->dev + b->off_err));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_batch_fast");
}

opm_status opm_batch_info(const opm_batch* b, int* n_items, int64_t* n_units, int* smem_bytes) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  if (n_items) *n_items = b->n_items;
  if (n_units) *n_units = b->n_units;
  if (smem_bytes) *smem_bytes = (int)fast::total(b->Pl);
  return OPM_OK;
}

opm_status opm_batch_check(const opm_batch* b) {
  if (!b) return fail(OPM_ERR_INVALID_ARG, "batch is NULL");
  unsigned word = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, b->dev + b->off_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word) e = cudaMemset(b->dev + b->off_err, 0, sizeof(unsigned));
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
constexpr size_t cal256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kSOffUnits = cal256(sizeof(BatchItemDev) * kStaticItems);
constexpr size_t kSOffSegs = kSOffUnits + cal256(sizeof(BatchUnit) * kStaticUnits);
constexpr size_t kSOffErr = kSOffSegs + cal256(sizeof(BatchSeg) * 2 * kStaticItems);
constexpr size_t kSBytes = kSOffErr + 256;

struct StaticDevice {
  bool ready;
  unsigned char* scratch;  // device address of the static array on this device
  int nsm, smem_optin;
};

alignas(256) unsigned char g_static_stage[kSBytes];  // host image of the work list
StaticDevice g_static_dev[kStaticDevices];
std::mutex g_static_mu;

bool unit_before(const BatchUnit& a, const BatchUnit& c) {
  // longest first; ties in generation order (item, j-tile, chunk, x-tile),
  // the order the batch path's stable sort keeps
  const int la = a.ke - a.ks, lc = c.ke - c.ks;
  if (la != lc) return la > lc;
  if (a.item != c.item) return a.item < c.item;
  if (a.jt != c.jt) return a.jt < c.jt;
  if (a.ks != c.ks) return a.ks < c.ks;
  return a.xt < c.xt;
}

}  // namespace
}  // namespace opm

static __device__ __align__(256) unsigned char g_static_scratch[opm::kSBytes];

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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_batch_fast, cudaFuncAttributeMaxDynamicSharedMemorySize, d.smem_optin);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_batch_fast, cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
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
  if (!items && n_items > 0) return fail(OPM_ERR_INVALID_ARG, "items is NULL");
  if (n_items < 0) return fail(OPM_ERR_INVALID_ARG, "n_items must be >= 0");
  if (n_items > kStaticItems)
    return fail(OPM_ERR_UNSUPPORTED, std::to_string(n_items) + " items exceed the static limit of " +
                                         std::to_string(kStaticItems));
  if (kchunk < 0) return fail(OPM_ERR_INVALID_ARG, "kchunk must be >= 0");
  if (ctas_per_sm < 0 || ctas_per_sm > 4) return fail(OPM_ERR_INVALID_ARG, "ctas_per_sm must lie in [0, 4]");
  if (kchunk == 0) kchunk = 64;
  if (ctas_per_sm == 0) ctas_per_sm = 4;
  if (!batch_encode_fn()) return fail(OPM_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is unavailable");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  StaticDevice* sd = nullptr;
  opm_status st = static_setup(dev, &sd);
  if (st != OPM_OK) return st;

  BatchItemDev* hitems = reinterpret_cast<BatchItemDev*>(g_static_stage);
  BatchUnit* hunits = reinterpret_cast<BatchUnit*>(g_static_stage + kSOffUnits);
  BatchSeg* hsegs = reinterpret_cast<BatchSeg*>(g_static_stage + kSOffSegs);
  int64_t nunits = 0;
  int Pl = 2, nseg = 0;
  for (int i = 0; i < n_items; ++i) {
    const opm_batch_item& it = items[i];
    const opm_plan* p = it.plan;
    if (!p || !it.raw) return fail(OPM_ERR_INVALID_ARG, "item " + std::to_string(i) + ": NULL plan or raw");
    if (p->device != dev) return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) + ": plan on another device");
    if (!plan_fast_ok(p))
      return fail(OPM_ERR_UNSUPPORTED, "item " + std::to_string(i) +
                                           ": plan not eligible (needs pixel <= step and ny >= 32)");
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
    CUresult cr = batch_encode_fn()(&d.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<uint16_t*>(it.raw), dims,
                                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS)
      return fail(OPM_ERR_CUDA, "item " + std::to_string(i) + ": cuTensorMapEncodeTiled failed (" +
                                    std::to_string((int)cr) + ")");
    d.frow = p->view.frow;
    d.fnlo = p->view.fnlo;
    d.zmip = it.zmip;
    d.ymip = it.ymip;
    d.nz = (int)p->nz;
    d.ny = (int)p->ny;
    d.nx = (int)p->nx;
    d.P = p->P;
    Pl = std::max(Pl, p->P);
    if (it.zmip) hsegs[nseg++] = BatchSeg{it.zmip, (long long)(p->ny * p->nx)};
    if (it.ymip) hsegs[nseg++] = BatchSeg{it.ymip, (long long)(p->nz * p->nx)};
    if (!it.zmip && !it.ymip) continue;
    const int xtiles = (int)((p->nx + kX - 1) / kX);
    const int jtiles = (int)((p->ny + kTileJ - 1) / kTileJ);
    for (int jt = 0; jt < jtiles; ++jt) {
      const Band bd = p->hBand[jt];
      for (int c0 = (bd.lo / kchunk) * kchunk; c0 < bd.hi; c0 += kchunk) {
        const int ks = std::max(bd.lo, c0), ke = std::min(bd.hi, c0 + kchunk);
        if (ks >= ke) continue;
        if (nunits + xtiles > kStaticUnits)
          return fail(OPM_ERR_UNSUPPORTED, "the items need more than the static limit of " +
                                               std::to_string(kStaticUnits) + " work units (raise kchunk or split)");
        for (int xt = 0; xt < xtiles; ++xt) hunits[nunits++] = BatchUnit{i, xt, jt, ks, ke, {0, 0, 0}};
      }
    }
  }
  std::sort(hunits, hunits + nunits, unit_before);

  // Pageable host -> device copies: each returns once its source has been
  // staged, so the host image may be rebuilt by the next call.
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* dv = sd->scratch;
  if (n_items > 0) e = cudaMemcpyAsync(dv, g_static_stage, sizeof(BatchItemDev) * n_items, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nunits > 0)
    e = cudaMemcpyAsync(dv + kSOffUnits, g_static_stage + kSOffUnits, sizeof(BatchUnit) * nunits,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nseg > 0)
    e = cudaMemcpyAsync(dv + kSOffSegs, g_static_stage + kSOffSegs, sizeof(BatchSeg) * nseg, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dv + kSOffErr, 0, sizeof(unsigned), s);  // error word starts at 0
  if (e != cudaSuccess) return cuda_fail(e, "opm_batch_project_static upload");
  if (nseg > 0) {
    dim3 grid(64, std::min(nseg, 65535));
    k_batch_zero<<<grid, 256, 0, s>>>(reinterpret_cast<const BatchSeg*>(dv + kSOffSegs), nseg);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_batch_zero");
  }
  if (nunits > 0) {
    const size_t smem = fast::total(Pl);
    if ((int)smem > sd->smem_optin) return fail(OPM_ERR_UNSUPPORTED, "batch slab depth needs too much shared memory");
    const int grid = (int)std::min<int64_t>(nunits, (int64_t)sd->nsm * ctas_per_sm);
    k_batch_fast<<<grid, kThreads, smem, s>>>(reinterpret_cast<const BatchItemDev*>(dv),
                                              reinterpret_cast<const BatchUnit*>(dv + kSOffUnits), (int)nunits, Pl,
                                              reinterpret_cast<unsigned*>(dv + kSOffErr));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_batch_fast");
  }
  if (check) {
    unsigned word = 0;
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&word, dv + kSOffErr, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "opm_batch_project_static check");
    if (word) return fail(OPM_ERR_INTERNAL, "device consistency check failed (bits " + std::to_string(word) + ")");
  }
  return OPM_OK;
}
