// Plan construction (FP64 geometry, split tables) and the C ABI entry points.
//
// Geometry follows Eq. (1) of the paper in the lab frame: a raw sample
// (n, r, x) sits at y = n*step + r*pixel*cos(theta), and output column j of
// row k = r reads the scan-plane coordinate
//   n_f(j, k) = ((j - J0)*pixel - k*pixel*cos(theta)) / step.
// The Fig. 2c remap places every frame into the larger (y', x) image at its
// accumulated offset; here that offset becomes the per-row term B_k.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <string>

#include "opm_internal.h"

namespace opm {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

opm_status fail(opm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

opm_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                 cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? OPM_ERR_OUT_OF_MEMORY : OPM_ERR_CUDA;
}

static double cos_deg(double theta_deg) {
  if (theta_deg == 90.0) return 0.0;
  if (theta_deg == 60.0) return 0.5;
  return std::cos(theta_deg * M_PI / 180.0);
}

static Split split(double v) {
  const double fl = std::floor(v);
  Split s;
  s.i = static_cast<int32_t>(fl);
  s.f = static_cast<float>(v - fl);
  return s;
}

// Host replica of the kernels' lower-plane computation (IEEE single
// subtraction is identical on host and device).
static int host_n0(Split a, Split b) {
  const float d = a.f - b.f;
  return a.i - b.i - (d < 0.0f ? 1 : 0);
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

static opm_status check_plan(const opm_plan* p) {
  if (!p) return fail(OPM_ERR_INVALID_ARG, "plan is NULL");
  if (p->device < 0 || !p->dmem)
    return fail(OPM_ERR_CUDA, "plan was created without a CUDA device");
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != p->device)
    return fail(OPM_ERR_CUDA, "plan belongs to device " + std::to_string(p->device) +
                                  " but device " + std::to_string(cur) + " is current");
  return OPM_OK;
}

}  // namespace opm

using namespace opm;

extern "C" {

int opm_version(void) { return 100; }

const char* opm_last_error(void) { return g_last_error.c_str(); }

opm_status opm_plan_create(int64_t nscan, int64_t nrows, int64_t ncols,
                           double theta_deg, double step, double pixel,
                           opm_interp interp, opm_plan** out) {
  if (!out) return fail(OPM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nscan < 2 || nrows < 1 || ncols < 1)
    return fail(OPM_ERR_INVALID_ARG, "need nscan >= 2, nrows >= 1, ncols >= 1");
  if (!(theta_deg > 0.0 && theta_deg <= 90.0))
    return fail(OPM_ERR_INVALID_ARG, "theta must lie in (0, 90] degrees");
  if (!(step > 0.0) || !(pixel > 0.0) || !std::isfinite(step) || !std::isfinite(pixel))
    return fail(OPM_ERR_INVALID_ARG, "step and pixel must be positive and finite");
  if (interp != OPM_INTERP_LINEAR && interp != OPM_INTERP_NEAREST)
    return fail(OPM_ERR_INVALID_ARG, "interp must be LINEAR or NEAREST");
  const int64_t lim31 = std::numeric_limits<int32_t>::max();
  if (nscan > lim31 / 4 || nrows > lim31 / 4 || ncols > lim31 / 4)
    return fail(OPM_ERR_UNSUPPORTED, "a raw dimension exceeds 2^29");

  const double c = cos_deg(theta_deg);
  const double J0d = std::ceil(step / pixel) - 1.0;
  const double X = J0d + (double)nscan * (step / pixel) + (double)(nrows - 1) * c;
  const double nyd = std::ceil(X - 1e-9);
  if (!(nyd >= 1.0) || nyd > (double)lim31 / 4 || J0d > (double)lim31 / 4)
    return fail(OPM_ERR_UNSUPPORTED, "output grid along y' exceeds 2^29 columns");
  const int64_t ny = (int64_t)nyd;
  const double voxels = (double)nrows * (double)ny * (double)ncols;
  if (voxels > 1099511627776.0)  // 2^40
    return fail(OPM_ERR_UNSUPPORTED, "output grid exceeds 2^40 voxels");

  opm_plan* p = new (std::nothrow) opm_plan();
  if (!p) return fail(OPM_ERR_OUT_OF_MEMORY, "host allocation of the plan failed");
  p->nscan = nscan;
  p->nrows = nrows;
  p->ncols = ncols;
  p->nz = nrows;
  p->ny = ny;
  p->nx = ncols;
  p->J0 = (int64_t)J0d;
  p->theta = theta_deg;
  p->step = step;
  p->pixel = pixel;
  p->c = c;
  p->rho = pixel / step;
  p->interp = interp;
  const char* fg = std::getenv("OPM_FORCE_GENERIC");
  p->force_generic = (fg && fg[0] == '1') ? 1 : 0;
  const char* of = std::getenv("OPM_ONE_PASS_FUSED");
  p->one_pass_fused = (of && of[0] == '1') ? 1 : 0;
  p->device = -1;
  p->dmem = nullptr;

  try {
    // Per-column and per-row terms of n_f, split into int + FP32 fraction.
    // NEAREST folds its +1/2 into A so that floor() picks the nearest plane.
    const double half = (interp == OPM_INTERP_NEAREST) ? 0.5 : 0.0;
    p->hA.resize(ny);
    for (int64_t j = 0; j < ny; ++j) p->hA[j] = split((double)(j - p->J0) * p->rho + half);
    p->hB.resize(nrows);
    for (int64_t k = 0; k < nrows; ++k) p->hB[k] = split((double)k * c * p->rho);

    // Row band of every 32-wide j-tile, from the kernels' own plane formula
    // with a margin of one plane on each side.  n0 is non-increasing in k.
    const int64_t ntile = (ny + kTileJ - 1) / kTileJ;
    p->hBand.resize(ntile);
    for (int64_t t = 0; t < ntile; ++t) {
      const int64_t j0 = tile_j0((int)t, (int)ny);
      const int64_t j1 = std::min<int64_t>(j0 + kTileJ, ny) - 1;
      int64_t lo = nrows, hi = 0;
      for (int64_t k = 0; k < nrows; ++k) {
        const int n_hi = host_n0(p->hA[j1], p->hB[k]);
        const int n_lo = host_n0(p->hA[j0], p->hB[k]);
        if (n_hi >= -2 && n_lo <= nscan) {
          lo = std::min(lo, k);
          hi = std::max(hi, k + 1);
        }
      }
      if (lo >= hi) lo = hi = 0;
      p->hBand[t] = Band{(int32_t)lo, (int32_t)hi};
    }

    // Slab depth of a 32-column tile, and whether the fast projection kernel
    // may assume that, within every full tile, consecutive columns sit on the
    // same or the next plane and the tile spans at most P - 1 planes.  The
    // check replays the kernels' own IEEE single-precision plane formula.
    const double Pd = std::floor((kTileJ - 1) * p->rho) + 4.0;
    p->P = Pd > 256.0 ? 257 : (int)Pd;
    p->fast_ok = (p->rho <= 1.0 && p->P <= 256 && ny >= kTileJ) ? 1 : 0;
    for (int64_t t = 0; p->fast_ok && t < ntile; ++t) {
      const int j0 = tile_j0((int)t, (int)ny);
      for (int64_t k = 0; p->fast_ok && k < nrows; ++k) {
        const int base = host_n0(p->hA[j0], p->hB[k]);
        int prev = base;
        for (int l = 1; l < kTileJ; ++l) {
          const int n0 = host_n0(p->hA[j0 + l], p->hB[k]);
          if ((l % 8) != 0 && n0 != prev && n0 != prev + 1) p->fast_ok = 0;
          if (n0 - base > p->P - 2 || n0 < base) p->fast_ok = 0;
          prev = n0;
        }
      }
    }
    // The fast kernel's per-(tile, row) tables, from the same formula.
    if (p->fast_ok) {
      p->hFrow.resize((size_t)ntile * nrows);
      p->hFnlo.resize((size_t)ntile * nrows);
      for (int64_t t = 0; t < ntile; ++t) {
        const int j0 = tile_j0((int)t, (int)ny);
        for (int64_t k = 0; k < nrows; ++k) {
          FastRow& fr = p->hFrow[t * nrows + k];
          int o[kTileJ];
          const int nlo = host_n0(p->hA[j0], p->hB[k]);
          for (int l = 0; l < kTileJ; ++l) {
            const Split a = p->hA[j0 + l], b = p->hB[k];
            const float d = a.f - b.f;
            const bool neg = d < 0.0f;
            const float w = (interp == OPM_INTERP_LINEAR) ? (neg ? d + 1.0f : d) : 0.0f;
            fr.w[l][0] = w;
            fr.w[l][1] = w;
            o[l] = a.i - b.i - (neg ? 1 : 0) - nlo;
          }
          for (int g = 0; g < 4; ++g) {
            unsigned adv = 0;
            for (int jj = 1; jj < 8; ++jj) {
              if (o[8 * g + jj] == o[8 * g + jj - 1] + 1) adv |= 1u << jj;
              // the fast kernel takes a row's y-max over the first and last
              // column of each plane interval only, which needs the weights
              // to grow along j inside an interval
              if (o[8 * g + jj] == o[8 * g + jj - 1] && fr.w[8 * g + jj][0] < fr.w[8 * g + jj - 1][0])
                p->fast_ok = 0;
            }
            fr.rec[g].adv = adv;
            fr.rec[g].ofirst = o[8 * g];
          }
          p->hFnlo[t * nrows + k] = nlo;
        }
      }
      if (!p->fast_ok) {
        p->hFrow.clear();
        p->hFnlo.clear();
      }
    }
    // The periodic kernel: the first compiled p/q for which every row of
    // every tile steps through its planes as floor((t p + ph) / q),
    // t = 0..31; the phase of each 8-column chunk goes into bits 16..23 of
    // its step word.
    const char* np = std::getenv("OPM_NO_PERIODIC");
    if (p->fast_ok && !(np && np[0] == '1')) {
      // plane of column t (0..31) of a tile row, relative to column 0
      auto tile_ofs = [](const FastRow& fr, int t) {
        const FastRec& rc = fr.rec[t / 8];
        const unsigned below = rc.adv & ((2u << (t % 8)) - 1u) & 0xffu;  // steps at or before column t % 8
        return rc.ofirst + __builtin_popcount(below) - fr.rec[0].ofirst;
      };
      auto phase = [&](const FastRow& fr, int fp, int fq) {
        for (int ph = 0; ph < fq; ++ph) {
          bool same = true;
          for (int t = 1; same && t < kTileJ; ++t) same = tile_ofs(fr, t) == per_ofs(fp, fq, ph, t);
          if (same) return ph;
        }
        return -1;
      };
      for (int f = 0; f < kNumFamilies && !p->family; ++f) {
        bool all = true;
        for (size_t i = 0; all && i < p->hFrow.size(); ++i)
          all = phase(p->hFrow[i], kFamilies[f].p, kFamilies[f].q) >= 0;
        if (all) p->family = f + 1;
      }
      if (p->family) {
        const int fp = kFamilies[p->family - 1].p, fq = kFamilies[p->family - 1].q;
        for (FastRow& fr : p->hFrow) {
          const int ph = phase(fr, fp, fq);
          for (int g = 0; g < 4; ++g) fr.rec[g].adv |= (unsigned)((8 * g * fp + ph) % fq) << 16;
        }
        p->lists_per_sm = kPerCtasPerSm;
      }
    }

    // Row k holds a voxel with no weight at all (so max_j V includes 0)?
    p->hYinit.resize(nrows);
    for (int64_t k = 0; k < nrows; ++k) {
      const double nf0 = (double)(0 - p->J0) * p->rho - (double)k * c * p->rho;
      const double nf1 = (double)(ny - 1 - p->J0) * p->rho - (double)k * c * p->rho;
      bool zero;
      if (interp == OPM_INTERP_NEAREST)
        zero = (nf0 + 0.5 < 0.0) || (nf1 + 0.5 >= (double)nscan);
      else
        zero = (nf0 <= -1.0) || (nf1 >= (double)nscan);
      p->hYinit[k] = zero ? 0.0f : -std::numeric_limits<float>::infinity();
    }
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(OPM_ERR_OUT_OF_MEMORY, "host allocation of the plan tables failed");
  }

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();  // clear the sticky "no device" status
    *out = p;            // host-only plan: shape queries work, compute calls refuse
    return OPM_OK;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaGetDevice");
  }
  // The fast kernel's work units (x-tile, j-tile, chunk of the tile's band)
  // on balanced lists, one per persistent CTA.  A unit is a chain of ring
  // stages that one CTA runs in order, so a plan with fewer units than lists
  // runs for the length of its longest unit with most CTAs idle.  The chunk
  // is the largest of kChunkRows, kChunkRows / 2, ..., kMinChunkRows rows that
  // still gives every list at least kUnitsPerList units on average (larger
  // chunks keep the DRAM locality of LPT's first round and pay the per-unit
  // set-up and z-MIP fold fewer times).
  if (p->fast_ok) {
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      delete p;
      return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    try {
      const int xtiles = (int)((ncols + kUnitX - 1) / kUnitX);
      const int nlists = std::min(std::max(nsm, 1) * p->lists_per_sm, kMaxLists);
      auto nchunks = [&](int rows) {
        int64_t n = 0;
        for (const Band& bd : p->hBand)
          if (bd.lo < bd.hi) n += (bd.hi - 1) / rows - bd.lo / rows + 1;
        return n * xtiles;
      };
      int rows = kChunkRows;
      while (rows > kMinChunkRows && (double)nchunks(rows) < kUnitsPerList * nlists) rows /= 2;
      p->chunk_rows = rows;
      for (int jt = 0; jt < (int)p->hBand.size(); ++jt) {
        const Band bd = p->hBand[jt];
        for (int c0 = (bd.lo / rows) * rows; c0 < bd.hi; c0 += rows) {
          const int ks = std::max(bd.lo, c0), ke = std::min(bd.hi, c0 + rows);
          if (ks >= ke) continue;
          for (int xt = 0; xt < xtiles; ++xt) p->hUnits.push_back(WorkUnit{0, xt, jt, ks, ke, 0, 0, 0});
        }
      }
      if (p->hUnits.size() > (size_t)INT32_MAX) p->fast_ok = 0;
      p->hLists.assign(nlists + 1, 0);
      schedule_lpt(p->hUnits.data(), (int)p->hUnits.size(), nlists, p->hLists.data());
    } catch (const std::bad_alloc&) {
      delete p;
      return fail(OPM_ERR_OUT_OF_MEMORY, "host allocation of the plan schedule failed");
    }
  }
  const size_t szA = align256(sizeof(Split) * p->hA.size());
  const size_t szB = align256(sizeof(Split) * p->hB.size());
  const size_t szT = align256(sizeof(Band) * p->hBand.size());
  const size_t szY = align256(sizeof(float) * p->hYinit.size());
  const size_t szF = align256(sizeof(FastRow) * p->hFrow.size());
  const size_t szN = align256(sizeof(int) * p->hFnlo.size());
  const size_t szU = align256(sizeof(WorkUnit) * p->hUnits.size());
  const size_t szL = align256(sizeof(int) * p->hLists.size());
  const size_t total = szA + szB + szT + szY + szF + szN + szU + szL + 256;
  e = cudaMalloc(&p->dmem, total);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "cudaMalloc(plan tables)");
  }
  char* base = static_cast<char*>(p->dmem);
  Split* dA = reinterpret_cast<Split*>(base);
  Split* dB = reinterpret_cast<Split*>(base + szA);
  Band* dT = reinterpret_cast<Band*>(base + szA + szB);
  float* dY = reinterpret_cast<float*>(base + szA + szB + szT);
  FastRow* dF = reinterpret_cast<FastRow*>(base + szA + szB + szT + szY);
  int* dN = reinterpret_cast<int*>(base + szA + szB + szT + szY + szF);
  WorkUnit* dU = reinterpret_cast<WorkUnit*>(base + szA + szB + szT + szY + szF + szN);
  int* dL = reinterpret_cast<int*>(base + szA + szB + szT + szY + szF + szN + szU);
  unsigned* dE = reinterpret_cast<unsigned*>(base + szA + szB + szT + szY + szF + szN + szU + szL);
  if ((e = cudaMemcpy(dA, p->hA.data(), sizeof(Split) * p->hA.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(dB, p->hB.data(), sizeof(Split) * p->hB.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(dT, p->hBand.data(), sizeof(Band) * p->hBand.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(dY, p->hYinit.data(), sizeof(float) * p->hYinit.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (!p->hFrow.empty() &&
       (e = cudaMemcpy(dF, p->hFrow.data(), sizeof(FastRow) * p->hFrow.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!p->hFnlo.empty() &&
       (e = cudaMemcpy(dN, p->hFnlo.data(), sizeof(int) * p->hFnlo.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (!p->hUnits.empty() &&
       (e = cudaMemcpy(dU, p->hUnits.data(), sizeof(WorkUnit) * p->hUnits.size(), cudaMemcpyHostToDevice)) !=
           cudaSuccess) ||
      (!p->hLists.empty() &&
       (e = cudaMemcpy(dL, p->hLists.data(), sizeof(int) * p->hLists.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemset(dE, 0, 256)) != cudaSuccess) {
    cudaFree(p->dmem);
    delete p;
    return cuda_fail(e, "uploading plan tables");
  }
  int pri_lo = 0, pri_hi = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&pri_lo, &pri_hi)) != cudaSuccess ||
      (e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, pri_hi)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming)) != cudaSuccess) {
    if (p->join_ev) cudaEventDestroy(p->join_ev);
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->side) cudaStreamDestroy(p->side);
    cudaFree(p->dmem);
    delete p;
    return cuda_fail(e, "creating the plan's side stream");
  }
  p->device = dev;
  PlanView& v = p->view;
  v.A = dA;
  v.B = dB;
  v.band = dT;
  v.yinit = dY;
  v.err = dE;
  v.frow = p->hFrow.empty() ? nullptr : dF;
  v.fnlo = p->hFnlo.empty() ? nullptr : dN;
  v.units = p->hUnits.empty() ? nullptr : dU;
  v.lists = p->hLists.empty() ? nullptr : dL;
  v.nunits = (int)p->hUnits.size();
  v.nlists = p->hLists.empty() ? 0 : (int)p->hLists.size() - 1;
  v.nscan = (int)nscan;
  v.nrows = (int)nrows;
  v.ncols = (int)ncols;
  v.nz = (int)nrows;
  v.ny = (int)ny;
  v.nx = (int)ncols;
  v.J0 = (int)p->J0;
  v.linear = interp == OPM_INTERP_LINEAR;
  v.rinv = (float)(step / pixel);
  *out = p;
  return OPM_OK;
}

opm_status opm_plan_path(const opm_plan* p, int* path, int* fam_p, int* fam_q) {
  if (!p) return fail(OPM_ERR_INVALID_ARG, "plan is NULL");
  const bool fast = p->fast_ok && !p->force_generic;
  if (path) *path = !fast ? OPM_PATH_GENERAL : p->family ? OPM_PATH_PERIODIC : OPM_PATH_FAST;
  if (fam_p) *fam_p = (fast && p->family) ? kFamilies[p->family - 1].p : 0;
  if (fam_q) *fam_q = (fast && p->family) ? kFamilies[p->family - 1].q : 0;
  return OPM_OK;
}

opm_status opm_plan_schedule(const opm_plan* p, int64_t* nunits, int* nlists, int* chunk_rows) {
  if (!p) return fail(OPM_ERR_INVALID_ARG, "plan is NULL");
  const bool has = !p->hLists.empty();
  if (nunits) *nunits = has ? (int64_t)p->hUnits.size() : 0;
  if (nlists) *nlists = has ? (int)p->hLists.size() - 1 : 0;
  if (chunk_rows) *chunk_rows = has ? p->chunk_rows : 0;
  return OPM_OK;
}

opm_status opm_plan_shape(const opm_plan* p, int64_t* nz, int64_t* ny,
                          int64_t* nx, int64_t* j0) {
  if (!p) return fail(OPM_ERR_INVALID_ARG, "plan is NULL");
  if (nz) *nz = p->nz;
  if (ny) *ny = p->ny;
  if (nx) *nx = p->nx;
  if (j0) *j0 = p->J0;
  return OPM_OK;
}

opm_status opm_plan_destroy(opm_plan* p) {
  if (!p) return OPM_OK;
  opm_status st = OPM_OK;
  if (p->dmem) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    if (p->join_ev) cudaEventDestroy(p->join_ev);
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->side) cudaStreamDestroy(p->side);
    cudaError_t e = cudaFree(p->dmem);
    if (cur != p->device && cur >= 0) cudaSetDevice(cur);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaFree(plan tables)");
  }
  delete p;
  return st;
}

opm_status opm_plan_check(const opm_plan* p) {
  if (!p) return fail(OPM_ERR_INVALID_ARG, "plan is NULL");
  if (p->device < 0) return OPM_OK;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  unsigned word = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&word, p->view.err, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && word) e = cudaMemset(p->view.err, 0, sizeof(unsigned));
  if (cur != p->device && cur >= 0) cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_fail(e, "opm_plan_check");
  if (word)
    return fail(OPM_ERR_INTERNAL, "device consistency check failed (bits " + std::to_string(word) + ")");
  return OPM_OK;
}

opm_status opm_deskew(const opm_plan* p, const void* raw, opm_dtype in_t,
                      void* vol, opm_dtype out_t, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!raw || !vol) return fail(OPM_ERR_INVALID_ARG, "raw and vol must be non-NULL");
  const bool ok = (in_t == OPM_U16 && (out_t == OPM_F32 || out_t == OPM_U16)) ||
                  (in_t == OPM_F32 && (out_t == OPM_F32 || out_t == OPM_U16)) ||
                  (in_t == OPM_F64 && out_t == OPM_F64);
  if (!ok) return fail(OPM_ERR_UNSUPPORTED, "unsupported (in, out) dtype pair for opm_deskew");
  return launch_deskew(p, raw, in_t, vol, out_t, static_cast<cudaStream_t>(stream));
}

opm_status opm_deskew_mip(const opm_plan* p, const void* raw, opm_dtype in_t, float* vol_f32, uint16_t* vol_u16,
                          float* zmip, float* ymip, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!raw || (!vol_f32 && !vol_u16)) return fail(OPM_ERR_INVALID_ARG, "raw and at least one volume are required");
  if (in_t != OPM_U16 && in_t != OPM_F32) return fail(OPM_ERR_UNSUPPORTED, "opm_deskew_mip takes U16 or F32 input");
  return launch_deskew_mip(p, raw, in_t, vol_f32, vol_u16, zmip, ymip, static_cast<cudaStream_t>(stream));
}

opm_status opm_stream_begin(const opm_plan* p, float* zmip, float* zsum, float* ymip, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!zmip && !zsum && !ymip) return fail(OPM_ERR_INVALID_ARG, "at least one projection output is required");
  return launch_stream_begin(p, zmip, zsum, ymip, static_cast<cudaStream_t>(stream));
}

opm_status opm_stream_pair(const opm_plan* p, const uint16_t* plane_lo, const uint16_t* plane_hi, int64_t n,
                           float* zmip, float* zsum, float* ymip, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!zmip && !zsum && !ymip) return fail(OPM_ERR_INVALID_ARG, "at least one projection output is required");
  if (n < -1 || n > p->nscan - 1) return fail(OPM_ERR_INVALID_ARG, "n must lie in [-1, nscan - 1]");
  if ((n >= 0) != (plane_lo != nullptr))
    return fail(OPM_ERR_INVALID_ARG, "plane_lo must be NULL exactly when n == -1");
  if ((n + 1 < p->nscan) != (plane_hi != nullptr))
    return fail(OPM_ERR_INVALID_ARG, "plane_hi must be NULL exactly when n == nscan - 1");
  return launch_stream_pair(p, plane_lo, plane_hi, (int)n, zmip, zsum, ymip, static_cast<cudaStream_t>(stream));
}

opm_status opm_sliding_push(const opm_plan* p, const uint16_t* stack, int64_t m, float* run, float* slots,
                            float* view, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!stack || !run || !slots || !view) return fail(OPM_ERR_INVALID_ARG, "stack, run, slots and view must be non-NULL");
  if (m < 0 || m > p->nscan - 1) return fail(OPM_ERR_INVALID_ARG, "m must lie in [0, nscan - 1]");
  return launch_sliding_push(p, stack, (int)m, run, slots, view, static_cast<cudaStream_t>(stream));
}

opm_status opm_deskew_dual(const opm_plan* p, const void* raw, opm_dtype in_t, float* vol_f32,
                           uint16_t* vol_u16, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!raw || !vol_f32 || !vol_u16) return fail(OPM_ERR_INVALID_ARG, "raw, vol_f32 and vol_u16 must be non-NULL");
  if (in_t != OPM_U16 && in_t != OPM_F32) return fail(OPM_ERR_UNSUPPORTED, "opm_deskew_dual takes U16 or F32 input");
  return launch_deskew_dual(p, raw, in_t, vol_f32, vol_u16, static_cast<cudaStream_t>(stream));
}

opm_status opm_project(const opm_plan* p, const void* raw, opm_dtype in_t,
                       float* zmip, float* zsum, float* ymip, int32_t* argz,
                       void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!raw) return fail(OPM_ERR_INVALID_ARG, "raw must be non-NULL");
  if (!zmip && !zsum && !ymip && !argz)
    return fail(OPM_ERR_INVALID_ARG, "at least one projection output is required");
  if (in_t != OPM_U16 && in_t != OPM_F32)
    return fail(OPM_ERR_UNSUPPORTED, "opm_project takes U16 or F32 input");
  return launch_project(p, raw, in_t, zmip, zsum, ymip, argz, static_cast<cudaStream_t>(stream));
}

opm_status opm_skew_adjoint(const opm_plan* p, const void* vol, void* raw_out,
                            opm_dtype t, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!vol || !raw_out) return fail(OPM_ERR_INVALID_ARG, "vol and raw_out must be non-NULL");
  if (t != OPM_F32 && t != OPM_F64)
    return fail(OPM_ERR_UNSUPPORTED, "opm_skew_adjoint takes F32 or F64");
  return launch_adjoint(p, vol, raw_out, t, static_cast<cudaStream_t>(stream));
}

opm_status opm_mip_backward(const opm_plan* p, const float* g_zmip,
                            const int32_t* argz, float* g_raw, void* stream) {
  opm_status st = check_plan(p);
  if (st != OPM_OK) return st;
  if (!g_zmip || !argz || !g_raw)
    return fail(OPM_ERR_INVALID_ARG, "g_zmip, argz and g_raw must be non-NULL");
  return launch_mip_backward(p, g_zmip, argz, g_raw, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
