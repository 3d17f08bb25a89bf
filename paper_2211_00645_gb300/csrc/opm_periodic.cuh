// Live view for plans whose plane coordinate advances by a rational p/q
// planes per output column (pixel/step = p/q, p <= q): the periodic path.
//
// Along one camera row, the lower interpolation plane of column j is
// floor((j - J0) p/q - beta_k).  Relative to the first column of a 32-column
// tile it is floor((t p + ph) / q), t = 0..31, for one phase ph in [0, q):
// a tile row steps through its staged planes in one of only q patterns (the
// plan checks every tile and row with the kernels' own IEEE arithmetic and
// records the phase).  Each pattern is compiled into straight-line code:
// the planes a row needs are loaded and converted once, each column's plane
// pair is a fixed register, and a column costs one packed FMA per row, one
// 3-input max per voxel pair into the z-max and, for the y-max, only the
// first and last column of each plane interval (along a row the voxels of
// one interval are a + w (b - a) with w increasing in j, and a correctly
// rounded FMA is monotone in w; the plan checks that the weights increase
// inside every interval).  The arithmetic is that of every other kernel of
// the library (the plan's weights, FMA on the exact plane difference), so
// the outputs are the same bit for bit.
//
// CTA: one producer warp (TMA ring of two camera rows per stage, as in
// opm_tma.cuh) and two compute warps.  Each compute warp owns all 32 columns
// j of the tile for 64 columns x (2 per lane), so a row's y-max over the tile
// is complete in one lane and goes to the global y-MIP with one atomic max;
// the compute warps never wait for each other, only for staged slabs.
#pragma once

#include "opm_tma.cuh"

namespace opm {
namespace {

namespace per {

constexpr int kXL = 2;                  // columns x per lane
constexpr int kXW = 32 * kXL;           // columns x per compute warp
constexpr int kXH = kX / kXW;           // x-halves of the 128-column x-tile
constexpr int kMaxCW = 4;               // compute warps per CTA at most

// A compute warp owns a run of RUN columns j (16 or 32) for kXW columns x.
template <int RUN>
struct Cfg {
  static_assert(RUN == 16 || RUN == 32, "runs of 16 or 32 columns");
  static constexpr int kRuns = kTileJ / RUN;       // column runs per tile
  static constexpr int kCW = kRuns * kXH;          // compute warps per CTA
  static constexpr int kThreads = 32 * (kCW + 1);
};

// Shared memory for S stages of slab depth P.
__host__ __device__ inline size_t off_tab(int S, int P) { return S * fast::stage_slab_bytes(P); }  // FastRow [S][2]
__host__ __device__ inline size_t off_bar(int S, int P) { return off_tab(S, P) + S * 2 * sizeof(FastRow); }
__host__ __device__ inline size_t off_jobs(int S, int P) { return off_bar(S, P) + 2 * S * 8; }  // JobP [kMaxCW]
__host__ __device__ inline size_t total(int S, int P) { return off_jobs(S, P) + kMaxCW * 48; }

struct JobP {  // a compute warp's job fields, parked in shared memory
  float* zmip;
  float* ymip;
  int nx, nz, j0, xbase;
  int k0g;   // camera row of stage g is k0g + 2 g
  int gend;  // stage count at the end of the job
  int pad[2];
};
static_assert(sizeof(JobP) == 48, "JobP layout");

// Plane of column t of a tile row, relative to the tile's first column, for
// pixel/step = p/q at phase ph.
__host__ __device__ constexpr int pofs(int p, int q, int ph, int t) { return per_ofs(p, q, ph, t); }
// Column t is the first or the last of its plane interval within a run of
// `run` columns.
__host__ __device__ constexpr bool pcand(int p, int q, int ph, int t, int run) {
  return t == 0 || t == run - 1 || pofs(p, q, ph, t) != pofs(p, q, ph, t - 1) ||
         pofs(p, q, ph, t + 1) != pofs(p, q, ph, t);
}
// Number of y-max candidates before column t.
__host__ __device__ constexpr int pcount(int p, int q, int ph, int t, int run) {
  int n = 0;
  for (int i = 0; i < t; ++i) n += pcand(p, q, ph, i, run) ? 1 : 0;
  return n;
}

}  // namespace per

// The ring in shared memory: S stages for slab depth Pl.
struct PerRing {
  unsigned char* base;
  int S, Pl;
  __device__ __forceinline__ FastRow* tab() const { return reinterpret_cast<FastRow*>(base + per::off_tab(S, Pl)); }
  // producer -> consumers: slabs and tables of a stage landed
  __device__ __forceinline__ uint64_t* full() const {
    return reinterpret_cast<uint64_t*>(base + per::off_bar(S, Pl));
  }
  // consumers -> producer: slot read by every compute warp
  __device__ __forceinline__ uint64_t* sfree() const { return full() + S; }
  __device__ __forceinline__ per::JobP* jobs() const {
    return reinterpret_cast<per::JobP*>(base + per::off_jobs(S, Pl));
  }
};

__device__ __forceinline__ PerRing per_ring(unsigned char* smem, int S, int Pl) {
  PerRing r;
  r.base = smem;
  r.S = S;
  r.Pl = Pl;
  return r;
}

// Whole CTA: barrier init, then a CTA barrier.
__device__ __forceinline__ void per_ring_init(const PerRing& r, int ncw) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < r.S; ++s) {
      mbar_init(&r.full()[s], 1);
      mbar_init(&r.sfree()[s], ncw);
    }
    fence_barrier_init();
  }
  __syncthreads();
}

// Producer warp: stage the job's rows (two per stage) once the slot is free.
// `g` is the CTA's running stage count, advanced by the job's stage count.
__device__ __forceinline__ bool per_produce(const FastJob& jb, const PerRing& r, int& g, unsigned* err, int lane) {
  const uint32_t pitch = kX * 2;
  const int S = r.S;
  const int nst = (jb.ke - jb.ks + 1) / 2;
  int kbase = jb.ks;  // first staged planes of 32 rows per load, one group ahead
  int ncur = jb.nlos[min(kbase + lane, jb.nz - 1)];
  int nnext = jb.nlos[min(kbase + 32 + lane, jb.nz - 1)];
#pragma unroll 1
  for (int it = 0; it < nst; ++it, ++g) {
    const int s = g % S;
    if (g >= S && !mbar_wait(&r.sfree()[s], ((g - S) / S) & 1, err)) return false;
    int nlo[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = jb.ks + 2 * it + q;
      if (k - kbase >= 32) {  // warp-uniform: rows advance in order
        kbase += 32;
        ncur = nnext;
        nnext = jb.nlos[min(kbase + 32 + lane, jb.nz - 1)];
      }
      nlo[q] = __shfl_sync(0xffffffffu, ncur, k - kbase);
    }
    if (lane == 0) {
      const int k0 = jb.ks + 2 * it;
      const int k1 = k0 + 1;  // k1 == nz: a padding row, staged as TMA zero fill
      unsigned char* slab = r.base + s * fast::stage_slab_bytes(r.Pl);
      mbar_arrive_tx(&r.full()[s], (unsigned)(2 * jb.P * pitch + 2 * sizeof(FastRow)));
      tma_load_3d(slab, jb.tmap, &r.full()[s], jb.xbase, k0, nlo[0]);
      tma_load_3d(slab + fast::slab_row_bytes(r.Pl), jb.tmap, &r.full()[s], jb.xbase, k1, k1 < jb.nz ? nlo[1] : 0);
      bulk_load(&r.tab()[s * 2 + 0], jb.rows + k0, sizeof(FastRow), &r.full()[s]);
      bulk_load(&r.tab()[s * 2 + 1], jb.rows + min(k1, jb.nz - 1), sizeof(FastRow), &r.full()[s]);
    }
    __syncwarp();
  }
  return true;
}

// Producer warp, after its last job: the CTA's shared memory must outlive
// every copy it issued (bounded wait on the last S stages).
__device__ __forceinline__ void per_drain(const PerRing& r, int g, bool ok, unsigned* err) {
  for (int q = max(0, g - r.S); q < g; ++q)
    if (!mbar_wait(&r.full()[q % r.S], (q / r.S) & 1, err, ok ? kWaitLimitNs : 50000000ull)) break;
}

// Two uint16 counts of a staged plane (this lane's 2 columns x) as FP32x2.
__device__ __forceinline__ f2 lds_x2(const unsigned char* smem, uint32_t off) {
  return u16x2_to_f2(*reinterpret_cast<const uint32_t*>(smem + off));
}

// Both camera rows of a stage for one compute warp: a run of RUN columns,
// row 0 at phase PH0 and row 1 at phase PH1.  off0 / off1: shared-memory
// offset of this lane's 2 columns x in the tile's first plane of each row;
// wof0 / wof1: the tile's (w, w) weight pairs of each row.
template <int RUN, int Pp, int Qq, int PH0, int PH1>
__device__ __forceinline__ void per_pair(const unsigned char* __restrict__ smem, uint32_t off0, uint32_t off1,
                                         uint32_t wof0, uint32_t wof1, float (&zmax)[RUN][per::kXL],
                                         float (&ym0)[per::kXL], float (&ym1)[per::kXL]) {
  using namespace per;
  constexpr uint32_t pitch = kX * 2;
  f2 a0 = lds_x2(smem, off0), b0 = lds_x2(smem, off0 + pitch);
  f2 a1 = lds_x2(smem, off1), b1 = lds_x2(smem, off1 + pitch);
  f2 d0 = sub2(b0, a0), d1 = sub2(b1, a1);
  float p0[kXL], p1[kXL];
  ulonglong2 wq0, wq1;
#pragma unroll
  for (int t = 0; t < RUN; ++t) {
    // next plane of a row: integers below 2^24, so the new lower plane is
    // exactly the old upper one
    if (t > 0 && pofs(Pp, Qq, PH0, t) != pofs(Pp, Qq, PH0, t - 1)) {
      a0 = b0;
      b0 = lds_x2(smem, off0 + (uint32_t)(pofs(Pp, Qq, PH0, t) + 1) * pitch);
      d0 = sub2(b0, a0);
    }
    if (t > 0 && pofs(Pp, Qq, PH1, t) != pofs(Pp, Qq, PH1, t - 1)) {
      a1 = b1;
      b1 = lds_x2(smem, off1 + (uint32_t)(pofs(Pp, Qq, PH1, t) + 1) * pitch);
      d1 = sub2(b1, a1);
    }
    if ((t & 1) == 0) {  // weights of columns t and t + 1 of both rows
      wq0 = *reinterpret_cast<const ulonglong2*>(smem + wof0 + 8 * t);
      wq1 = *reinterpret_cast<const ulonglong2*>(smem + wof1 + 8 * t);
    }
    float v0[kXL], v1[kXL];
    upk(fma2((t & 1) ? wq0.y : wq0.x, d0, a0), v0[0], v0[1]);
    upk(fma2((t & 1) ? wq1.y : wq1.x, d1, a1), v1[0], v1[1]);
#pragma unroll
    for (int c = 0; c < kXL; ++c) zmax[t][c] = max3(zmax[t][c], v0[c], v1[c]);
    if (pcand(Pp, Qq, PH0, t, RUN)) {
      if (pcount(Pp, Qq, PH0, t, RUN) % 2 == 0) {
#pragma unroll
        for (int c = 0; c < kXL; ++c) p0[c] = v0[c];
      } else {
#pragma unroll
        for (int c = 0; c < kXL; ++c) ym0[c] = max3(ym0[c], p0[c], v0[c]);
      }
    }
    if (pcand(Pp, Qq, PH1, t, RUN)) {
      if (pcount(Pp, Qq, PH1, t, RUN) % 2 == 0) {
#pragma unroll
        for (int c = 0; c < kXL; ++c) p1[c] = v1[c];
      } else {
#pragma unroll
        for (int c = 0; c < kXL; ++c) ym1[c] = max3(ym1[c], p1[c], v1[c]);
      }
    }
  }
  if (pcount(Pp, Qq, PH0, RUN, RUN) % 2 == 1) {
#pragma unroll
    for (int c = 0; c < kXL; ++c) ym0[c] = fmaxf(ym0[c], p0[c]);
  }
  if (pcount(Pp, Qq, PH1, RUN, RUN) % 2 == 1) {
#pragma unroll
    for (int c = 0; c < kXL; ++c) ym1[c] = fmaxf(ym1[c], p1[c]);
  }
}

// Phase pair idx = PH0 * Qq + PH1 in [LO, HI), by a balanced branch tree.
template <int RUN, int Pp, int Qq, int LO, int HI>
__device__ __forceinline__ void per_tree(int idx, const unsigned char* __restrict__ smem, uint32_t off0,
                                         uint32_t off1, uint32_t wof0, uint32_t wof1, float (&zmax)[RUN][per::kXL],
                                         float (&ym0)[per::kXL], float (&ym1)[per::kXL]) {
  if constexpr (HI - LO == 1) {
    per_pair<RUN, Pp, Qq, LO / Qq, LO % Qq>(smem, off0, off1, wof0, wof1, zmax, ym0, ym1);
  } else {
    constexpr int MID = (LO + HI) / 2;
    if (idx < MID)
      per_tree<RUN, Pp, Qq, LO, MID>(idx, smem, off0, off1, wof0, wof1, zmax, ym0, ym1);
    else
      per_tree<RUN, Pp, Qq, MID, HI>(idx, smem, off0, off1, wof0, wof1, zmax, ym0, ym1);
  }
}

// The phase of each 8-column chunk (its first column's position within the
// period) is kept in bits 16..23 of its step word; a run's is that of its
// first chunk.
constexpr int kPhaseShift = 16;

// Compute warp i: run h = i % kRuns of the job's tile (columns
// j0 + RUN h .. + RUN - 1) for columns x xbase + 64 (i / kRuns) .. + 63,
// both rows of every stage.  z-maxima stay in registers and are folded into
// zmip at the end of the job; each row's y-max over the run goes to ymip
// right away.  Returns false when a bounded wait gave up.
template <int RUN, int Pp, int Qq>
__device__ __forceinline__ bool per_consume(const FastJob& jb, const PerRing& r, int& g, unsigned* err, int i,
                                            int lane) {
  using namespace per;
  constexpr int kRuns = Cfg<RUN>::kRuns;
  const int h = i % kRuns, xh = i / kRuns;
  const uint32_t pitch = kX * 2;
  const int S = r.S;
  const unsigned char* smem = r.base;
  JobP* js = r.jobs() + i;
  if (lane == 0) {
    js->zmip = jb.zmip;
    js->ymip = jb.ymip;
    js->nx = jb.nx;
    js->nz = jb.nz;
    js->j0 = jb.j0;
    js->xbase = jb.xbase;
    js->k0g = jb.ks - 2 * g;
    js->gend = g + (jb.ke - jb.ks + 1) / 2;
  }
  __syncwarp();
  float zmax[RUN][kXL];
#pragma unroll
  for (int t = 0; t < RUN; ++t)
#pragma unroll
    for (int c = 0; c < kXL; ++c) zmax[t][c] = 0.0f;  // uint16 voxels are >= 0
  bool ok = true;
  const uint32_t xoff = (uint32_t)(xh * kXW + lane * kXL) * 2;  // this lane's bytes within a staged plane

#pragma unroll 1
  for (; g < lds_volatile_s32(&js->gend); ++g) {
    const int s = g % S;
    if (!mbar_wait(&r.full()[s], (g / S) & 1, err)) {
      ok = false;
      break;
    }
    const uint32_t tab0 = (uint32_t)(per::off_tab(S, r.Pl) + (size_t)(s * 2) * sizeof(FastRow));
    const uint32_t rec = (uint32_t)(offsetof(FastRow, rec) + (h * RUN / 8) * sizeof(FastRec));
    const uint2 rr0 = *reinterpret_cast<const uint2*>(smem + tab0 + rec);
    const uint2 rr1 = *reinterpret_cast<const uint2*>(smem + tab0 + (uint32_t)sizeof(FastRow) + rec);
    const int c0 = (int)((rr0.x >> kPhaseShift) & 255u);
    const int c1 = (int)((rr1.x >> kPhaseShift) & 255u);
    const uint32_t row0 = (uint32_t)(s * fast::stage_slab_bytes(r.Pl)) + xoff;
    const uint32_t row1 = row0 + (uint32_t)fast::slab_row_bytes(r.Pl);
    float ym0[kXL], ym1[kXL];
#pragma unroll
    for (int c = 0; c < kXL; ++c) ym0[c] = ym1[c] = 0.0f;
    const uint32_t wof0 = tab0 + (uint32_t)(h * RUN * 8);
    per_tree<RUN, Pp, Qq, 0, Qq * Qq>(c0 * Qq + c1, smem, row0 + rr0.y * pitch, row1 + rr1.y * pitch, wof0,
                                      wof0 + (uint32_t)sizeof(FastRow), zmax, ym0, ym1);
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.sfree()[s]);
    float* ymip = lds_volatile_ptr(&js->ymip);
    if (ymip) {
      const int nx = lds_volatile_s32(&js->nx);
      const int k0 = lds_volatile_s32(&js->k0g) + 2 * g;
      const int x = lds_volatile_s32(&js->xbase) + xh * kXW + lane * kXL;
      const bool second = k0 + 1 < lds_volatile_s32(&js->nz);
#pragma unroll
      for (int c = 0; c < kXL; ++c) {
        if (x + c < nx) {
          atomicMax(reinterpret_cast<int*>(ymip + (size_t)k0 * nx + x + c), __float_as_int(ym0[c]));
          if (second) atomicMax(reinterpret_cast<int*>(ymip + (size_t)(k0 + 1) * nx + x + c), __float_as_int(ym1[c]));
        }
      }
    }
  }

  float* zmip = lds_volatile_ptr(&js->zmip);
  if (zmip) {
    const int nx = lds_volatile_s32(&js->nx);
    const int x = lds_volatile_s32(&js->xbase) + xh * kXW + lane * kXL;
    const int j0 = lds_volatile_s32(&js->j0) + h * RUN;
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
      float* row = zmip + (size_t)(j0 + t) * nx;
#pragma unroll
      for (int c = 0; c < kXL; ++c)
        if (x + c < nx) atomicMax(reinterpret_cast<int*>(row + x + c), __float_as_int(zmax[t][c]));
    }
  }
  return ok;
}

}  // namespace
}  // namespace opm
