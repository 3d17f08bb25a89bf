// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "opm.h"
#include "opm_sched.h"

namespace opm {

// An FP64 coordinate split into floor (int32) and an FP32 fraction.  The
// per-voxel plane coordinate n_f(j,k) = A_j - B_k is rebuilt on the GPU as
// (A.i - B.i) + (A.f - B.f): the integer part is exact and the fraction keeps
// ~1e-7 absolute error, where a plain FP32 product j*rho would lose ~1e-4 at
// j ~ 2500 (enough to move a uint16 voxel by several counts).
struct Split {
  int32_t i;
  float f;
};

// Row band of one 32-column j-tile: rows [lo, hi) may carry non-zero weight,
// every row outside it is structurally zero for all columns of the tile.
struct Band {
  int32_t lo;
  int32_t hi;
};

constexpr int kTileJ = 32;  // j-columns per CTA tile of the projection kernels

// First column of j-tile t: tiles are 32 columns wide, the last one is
// shifted back to end at ny when ny is not a multiple of 32 (ny >= 32), so
// that every tile is full; columns shared with the previous tile are
// computed twice, which max-combined outputs absorb.
__host__ __device__ inline int tile_j0(int t, int ny) {
  const int j0 = t * kTileJ;
  return (ny >= kTileJ && j0 + kTileJ > ny) ? ny - kTileJ : j0;
}

// Precomputed plane table of one (tile, camera row) for the fast projection
// kernel, fetched by one bulk copy next to the raw slab.  Compute warp g
// (columns 8g..8g+7) reads w[8g..8g+7] and rec[g].
struct FastRec {
  unsigned adv;  // bit j (1..7): column 8g+j sits one plane above column 8g+j-1
  int ofirst;    // slab offset (plane - nlo) of column 8g
};
struct __align__(16) FastRow {
  float w[kTileJ][2];  // (w, w) pairs: interpolation weight of each column
  FastRec rec[4];
};
static_assert(sizeof(FastRow) == 288, "FastRow is copied as 288 bytes");

// Plans whose lower plane advances by p/q planes per output column j
// (pixel/step = p/q) take the periodic live-view kernel (opm_periodic.cuh):
// along a camera row, the 32 columns of a tile sit on planes
// floor((t p + ph)/q) above the first one, t = 0..31, for one phase ph in
// [0, q).  One kernel is compiled per entry of this list; any other plan
// takes k_project_fast.
struct Family {
  int p, q;
};
constexpr Family kFamilies[] = {{1, 3}, {1, 2}};
constexpr int kNumFamilies = (int)(sizeof(kFamilies) / sizeof(kFamilies[0]));
constexpr int kPerRun = 32;       // columns j per compute warp of the periodic kernel
constexpr int kPerCtasPerSm = 4;  // its persistent CTAs per SM
constexpr int kPerStages = 6;     // its TMA ring depth
__host__ __device__ constexpr int per_ofs(int p, int q, int ph, int t) { return (t * p + ph) / q; }

// Error bits recorded by kernels in the plan's device error word.
enum : unsigned {
  kErrSlabRange = 1u,   // a plane offset fell outside the staged slab
  kErrWaitTimeout = 2u, // an mbarrier wait gave up
  kErrSearch = 4u,      // a column search of the plane-pair kernel ran past its bound
  kErrOrder = 8u,       // the adjoint walk met a lower plane that decreased along j
};

void set_error(const std::string& msg);
opm_status fail(opm_status s, const std::string& msg);
opm_status cuda_fail(cudaError_t e, const char* what);

// Device-side view of a plan, passed by value to kernels.
struct PlanView {
  const Split* A;     // [ny]  (j - J0) * pixel/step (+1/2 for NEAREST)
  const Split* B;     // [nz]  k * cos(theta) * pixel/step
  const Band* band;   // [ceil(ny / kTileJ)]
  const float* yinit; // [nz]  0 if row k has a structurally zero voxel, else -inf
  unsigned* err;      // error word
  const FastRow* frow;  // [ntile][nz] fast-kernel tables (NULL unless fast_ok)
  const int* fnlo;      // [ntile][nz] first staged plane of each (tile, row)
  const WorkUnit* units;  // fast-kernel work units, list by list (NULL unless fast_ok)
  const int* lists;       // [nlists + 1] first unit of each persistent CTA's list
  int nunits, nlists;
  int nscan, nrows, ncols, nz, ny, nx, J0;
  int linear;         // 1 LINEAR, 0 NEAREST
  float rinv;         // step / pixel (float), used only to size search windows
};

}  // namespace opm

struct opm_plan {
  int64_t nscan, nrows, ncols, nz, ny, nx, J0;
  double theta, step, pixel, c, rho;
  int interp;
  int force_generic;  // use the plain (non-TMA) kernels for every call
  int P;              // planes staged per row for a 32-column tile
  int fast_ok;        // full tiles never step more than one plane per column
  int family = 0;     // 1 + index into kFamilies when the periodic kernel applies, else 0
  int lists_per_sm = 4;  // persistent CTA lists per SM of the live-view schedule
  int chunk_rows = 0;    // rows per work unit of that schedule (0: no schedule)
  std::vector<opm::Split> hA, hB;
  std::vector<opm::Band> hBand;
  std::vector<float> hYinit;
  std::vector<opm::FastRow> hFrow;  // fast-kernel tables (when fast_ok)
  std::vector<int> hFnlo;
  std::vector<opm::WorkUnit> hUnits;  // fast-kernel schedule (when fast_ok and a device exists)
  std::vector<int> hLists;
  int device;        // -1: created without a device
  void* dmem;        // one allocation holding every device table
  opm::PlanView view;
  // opm_deskew_mip: the live view runs on `side` (highest priority, a
  // quarter of the persistent grid) beside the volume on the caller's stream,
  // forked and joined through the two events; one_pass_fused selects the
  // single fused kernel instead (environment OPM_ONE_PASS_FUSED=1 at plan
  // creation).  `side` is NULL for a plan made without a device.
  int one_pass_fused = 0;
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  mutable std::mutex side_mu;  // one fork/join on `side` at a time
};

namespace opm {

// Kernel launchers (one per translation unit).  Each returns OPM_OK or an
// error already recorded with fail()/cuda_fail().
// grid_div > 1 launches the persistent fast kernel with 1/grid_div of its
// CTAs (each then walks grid_div of the schedule's lists), leaving room on
// every SM for a kernel that runs beside it.
opm_status launch_project(const opm_plan* p, const void* raw, opm_dtype in_t,
                          float* zmip, float* zsum, float* ymip, int32_t* argz,
                          cudaStream_t s, int grid_div = 1);
opm_status launch_deskew(const opm_plan* p, const void* raw, opm_dtype in_t,
                         void* vol, opm_dtype out_t, cudaStream_t s);
opm_status launch_deskew_dual(const opm_plan* p, const void* raw, opm_dtype in_t, float* vol_f32,
                              uint16_t* vol_u16, cudaStream_t s);
opm_status launch_deskew_mip(const opm_plan* p, const void* raw, opm_dtype in_t, float* volf, uint16_t* volh,
                             float* zmip, float* ymip, cudaStream_t s);
opm_status launch_sheet_project(const void* raw, opm_dtype in_t, int nscan, int nrows, int ncols, double shear,
                                float* out, int H, cudaStream_t s);
opm_status launch_warp_rows(const float* in, int H, int ncols, float* out, int Ho, double a, double b,
                            cudaStream_t s);
opm_status launch_stream_begin(const opm_plan* p, float* zmip, float* zsum, float* ymip, cudaStream_t s);
opm_status launch_stream_pair(const opm_plan* p, const uint16_t* lo, const uint16_t* hi, int n, float* zmip,
                              float* zsum, float* ymip, cudaStream_t s);
opm_status launch_sliding_push(const opm_plan* p, const uint16_t* stack, int m, float* run, float* slots,
                               float* view, cudaStream_t s);
opm_status launch_adjoint(const opm_plan* p, const void* vol, void* raw_out,
                          opm_dtype t, cudaStream_t s);
opm_status launch_mip_backward(const opm_plan* p, const float* g,
                               const int32_t* argz, float* g_raw,
                               cudaStream_t s);

// Device-side helpers shared by the kernels -------------------------------
#ifdef __CUDACC__
// Lower plane n0 and weight w of output (j, k): n_f = (A.i - B.i) + (A.f - B.f).
__device__ __forceinline__ void plane_weight(Split a, Split b, int linear,
                                             int& n0, float& w) {
  const float d = a.f - b.f;  // in [-1, 1]
  const int neg = d < 0.0f;
  n0 = a.i - b.i - neg;
  w = linear ? (neg ? d + 1.0f : d) : 0.0f;
}
#endif

}  // namespace opm

namespace opm {
// Fast-projection eligibility and slab depth of a plan (host side).
inline bool plan_fast_ok(const opm_plan* p) { return p && p->fast_ok && p->view.frow != nullptr; }
}  // namespace opm
