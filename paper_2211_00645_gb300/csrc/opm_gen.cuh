// General projection kernel's building blocks: its shared-memory ring and
// per-job producer / consumer loops, shared by the one-plan kernel (one job
// per CTA) and the persistent batched kernel (jobs of many stacks, one after
// another on one ring).
//
// One job = one 32-column j-tile of one 128-column x-tile over the tile's
// whole row band [ks, ke) (Fig. 2d).  Every output of the projection is
// produced: z-MIP, z-sum and the first arg-max along z are kept in registers
// over the band and written once at the end of the job; the y-max of every
// staged row is reduced over the tile's 32 columns in shared memory and
// folded into the y-MIP by the producer warp once the compute warps are done
// with the row.  Each ring slot carries its own record of where that fold
// goes (row pointer and column count), because with a stage counter that
// carries on across jobs the fold of a job's last rows happens while the
// producer already stages the next job, maybe of another stack.
//
// Rows come one per stage: the producer computes each column's plane n0 and
// weight w (Eq. 1, split tables A_j + B_k), the slab offsets relative to the
// tile's first column, and warp-uniform step masks, then stages the slab
// {128 x, 1 row, P planes} with one TMA load.  Rows P and P + 1 of every
// slot stay zero: columns outside the output grid (j >= ny) read them.
#pragma once

#include "opm_tma.cuh"

namespace opm {
namespace {
namespace gen {

constexpr int S = kStagesGen;

struct __align__(16) RowHdr {
  int k;           // camera row staged
  int nlo;         // first staged plane
  unsigned adv;    // bit j: column j is one plane above column j-1
  unsigned jump;   // bit j: column j is more than one plane above column j-1
  unsigned valid;  // bit j: column j lies inside the output grid
  int ofirst[kNW]; // slab offset of the first column of each compute warp
  int xn;          // columns of the y-MIP row this slot folds into (<= kX)
  float* yrow;     // y-MIP row k at the tile's first column, or NULL
};
static_assert(sizeof(RowHdr) == 48, "hdr");

// slab rows 0..P-1 come from TMA, rows P and P+1 stay zero (columns j >= ny)
template <typename T>
__host__ __device__ inline size_t slab_bytes(int P) { return (size_t)(P + 2) * kX * sizeof(T); }
template <typename T>
__host__ __device__ inline size_t off_w(int P) { return S * slab_bytes<T>(P); }
template <typename T>
__host__ __device__ inline size_t off_o(int P) { return off_w<T>(P) + S * kTileJ * 4; }
template <typename T>
__host__ __device__ inline size_t off_hdr(int P) { return off_o<T>(P) + S * kTileJ * 4; }
template <typename T>
__host__ __device__ inline size_t off_ybuf(int P) { return off_hdr<T>(P) + S * sizeof(RowHdr); }
template <typename T>
__host__ __device__ inline size_t off_bar(int P) { return off_ybuf<T>(P) + S * kX * 4; }
template <typename T>
__host__ __device__ inline size_t total(int P) { return off_bar<T>(P) + 2 * S * 8; }

}  // namespace gen

// Views of the ring in shared memory for slab depth P (the deepest of the
// jobs the CTA will run).
template <typename T>
struct GenRing {
  unsigned char* base;
  int P;
  __device__ unsigned char* slab(int s) const { return base + (size_t)s * gen::slab_bytes<T>(P); }
  __device__ float* wtab() const { return reinterpret_cast<float*>(base + gen::off_w<T>(P)); }
  __device__ int* otab() const { return reinterpret_cast<int*>(base + gen::off_o<T>(P)); }
  __device__ gen::RowHdr* hdr() const { return reinterpret_cast<gen::RowHdr*>(base + gen::off_hdr<T>(P)); }
  __device__ float* ybuf() const { return reinterpret_cast<float*>(base + gen::off_ybuf<T>(P)); }
  __device__ uint64_t* full() const { return reinterpret_cast<uint64_t*>(base + gen::off_bar<T>(P)); }
  __device__ uint64_t* ydone() const { return full() + gen::S; }
};

// Barriers, the zero rows of every slot and the y-max buffers; ends with a
// CTA barrier.
template <typename T>
__device__ __forceinline__ void gen_ring_init(const GenRing<T>& r) {
  using gen::S;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&r.full()[s], 1);
      mbar_init(&r.ydone()[s], kNW);
    }
    fence_barrier_init();
  }
  const int pitch = kX * (int)sizeof(T);
  for (int s = 0; s < S; ++s) {
    uint4* z = reinterpret_cast<uint4*>(r.slab(s) + (size_t)r.P * pitch);
    for (int i = threadIdx.x; i < 2 * pitch / 16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
  }
  float* yb = r.ybuf();
  for (int i = threadIdx.x; i < S * kX; i += kThreads) yb[i] = -INFINITY;
  __syncthreads();
}

// One job of the general kernel.
struct GenJob {
  const CUtensorMap* tmap;  // raw stack, box {128, 1, P}
  const Split* A;           // [ny] column split table
  const Split* B;           // [nz] row split table
  int linear;               // interpolation mode of the plan
  int ny, nz, nx, P;        // output grid and this stack's slab depth
  int j0, xbase;            // first output column j and x of the tile
  int ks, ke;               // row band of the tile
  float* zmip;              // [ny][nx] or NULL
  float* zsum;              // [ny][nx] or NULL
  float* ymip;              // [nz][nx] or NULL (pre-set, combined by atomic max)
  int32_t* argz;            // [ny][nx] or NULL
};

// Producer's fold of slot s: the row's y-max over the tile's 32 columns
// into the y-MIP, then the slot's buffer back to -inf.
template <typename T>
__device__ __forceinline__ void gen_fold(const GenRing<T>& r, int s, int lane) {
  const gen::RowHdr& h = r.hdr()[s];
  float* yrow = h.yrow;
  const int xn = h.xn;
  float* yb = r.ybuf() + s * kX;
#pragma unroll
  for (int i = 0; i < kVec; ++i) {
    const int xl = 32 * i + lane;
    const int yi = yidx(xl);
    const float val = yb[yi];
    yb[yi] = -INFINITY;
    if (yrow && xl < xn) atomic_max_f(yrow + xl, val);
  }
  __syncwarp();
}

// Producer warp: stages the job's rows on the ring (stage counter g carries
// on across jobs).  Before it reuses a slot it waits until the compute warps
// are done with the slot's previous row and folds that row's y-max.
template <typename T>
__device__ bool gen_produce(const GenJob& jb, const GenRing<T>& r, int& g, unsigned* err, int lane) {
  using gen::S;
  const int pitch = kX * (int)sizeof(T);
  const int nst = jb.ke - jb.ks;
  const int jl = jb.j0 + lane;
  const bool jvalid = jl < jb.ny;
  const Split a = jb.A[jvalid ? jl : jb.ny - 1];
  int kbase = jb.ks;
  Split bcur = jb.B[min(kbase + lane, jb.nz - 1)];
  Split bnext = jb.B[min(kbase + 32 + lane, jb.nz - 1)];
  const int xn = min(kX, jb.nx - jb.xbase);
  float* wtab = r.wtab();
  int* otab = r.otab();
#pragma unroll 1
  for (int it = 0; it < nst; ++it, ++g) {
    const int s = g % S;
    if (g >= S) {
      if (!mbar_wait(&r.ydone()[s], ((g - S) / S) & 1, err)) return false;
      gen_fold<T>(r, s, lane);
    }
    const int k = jb.ks + it;
    if (k - kbase >= 32) {
      kbase += 32;
      bcur = bnext;
      bnext = jb.B[min(kbase + 32 + lane, jb.nz - 1)];
    }
    Split b;
    b.i = __shfl_sync(0xffffffffu, bcur.i, k - kbase);
    b.f = __shfl_sync(0xffffffffu, bcur.f, k - kbase);
    int n0;
    float w;
    plane_weight(a, b, jb.linear, n0, w);
    const int nlo = __shfl_sync(0xffffffffu, n0, 0);
    int o = n0 - nlo;
    if (!jvalid) {
      o = r.P;  // the two zero rows, never written by a load
      w = 0.0f;
    } else if (o < 0 || o > jb.P - 2) {
      atomicOr(err, kErrSlabRange);
      o = min(max(o, 0), jb.P - 2);
    }
    const int op = __shfl_up_sync(0xffffffffu, o, 1);
    const bool first = (lane % kJT) == 0;
    const unsigned adv = __ballot_sync(0xffffffffu, !first && o == op + 1);
    const unsigned jump = __ballot_sync(0xffffffffu, !first && o != op && o != op + 1);
    const unsigned vmask = __ballot_sync(0xffffffffu, jvalid);
    wtab[s * kTileJ + lane] = w;
    otab[s * kTileJ + lane] = o;
    const int of = __shfl_sync(0xffffffffu, o, (lane % kNW) * kJT);
    gen::RowHdr& h = r.hdr()[s];
    if (lane < kNW) h.ofirst[lane] = of;
    if (lane == 0) {
      h.k = k;
      h.nlo = nlo;
      h.adv = adv;
      h.jump = jump;
      h.valid = vmask;
      h.xn = xn;
      h.yrow = jb.ymip ? jb.ymip + (size_t)k * jb.nx + jb.xbase : nullptr;
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive_tx(&r.full()[s], (unsigned)(jb.P * pitch));
      tma_load_3d(r.slab(s), jb.tmap, &r.full()[s], jb.xbase, k, nlo);
    }
    __syncwarp();
  }
  return true;
}

// Producer's end: folds the rows still on the ring (g rows were staged in
// all).  After a failed wait it only waits, with a short limit, for the
// loads still in flight, so that no copy lands after the CTA has exited.
template <typename T>
__device__ void gen_drain(const GenRing<T>& r, int g, bool ok, unsigned* err, int lane) {
  using gen::S;
  for (int q = max(0, g - S); q < g; ++q) {
    const int s = q % S;
    if (ok) {
      ok = mbar_wait(&r.ydone()[s], (q / S) & 1, err);
      if (ok) {
        gen_fold<T>(r, s, lane);
        continue;
      }
    }
    (void)mbar_wait(&r.full()[s], (q / S) & 1, err, 50000000ull);
  }
}

// Compute warp cw (columns j0 + 8 cw .. + 7, 4 columns x per lane): z-max,
// z-sum and first arg-max over the job's band in registers, the y-max of
// each row into the slot's buffer, then the job's outputs.  Rows before the
// band are exactly zero (the z-max starts at 0 with arg-max 0 when the band
// does not start at row 0), and so are rows after it (a z-max still below 0
// at the end becomes 0 at the band's end row).
template <typename T>
__device__ bool gen_consume(const GenJob& jb, const GenRing<T>& r, int& g, unsigned* err, int cw, int lane) {
  using gen::S;
  const int pitch = kX * (int)sizeof(T);
  const int nst = jb.ke - jb.ks;
  const int jg = cw * kJT;
  const unsigned lanebit = (lane < kJT) ? (1u << (jg + lane)) : 0u;
  const float* wtab = r.wtab();
  const int* otab = r.otab();
  float zmax[kJT][kVec], zsum[kJT][kVec];
  int az[kJT][kVec];
  const float zinit = jb.ks > 0 ? 0.0f : -INFINITY;
#pragma unroll
  for (int j = 0; j < kJT; ++j)
#pragma unroll
    for (int c = 0; c < kVec; ++c) {
      zmax[j][c] = zinit;
      zsum[j][c] = 0.0f;
      az[j][c] = 0;
    }
  bool ok = true;
#pragma unroll 1
  for (int it = 0; it < nst; ++it, ++g) {
    const int s = g % S;
    if (!mbar_wait(&r.full()[s], (g / S) & 1, err)) {
      ok = false;
      break;
    }
    const gen::RowHdr& h = r.hdr()[s];
    const int krow = h.k;
    const unsigned adv = __ballot_sync(0xffffffffu, (h.adv & lanebit) != 0);
    const unsigned jump = __ballot_sync(0xffffffffu, (h.jump & lanebit) != 0);
    const unsigned valid = __ballot_sync(0xffffffffu, (h.valid & lanebit) != 0);
    const unsigned char* ls = r.slab(s) + lane * (kVec * (int)sizeof(T));
    Stream st;
    stream_reset<T>(st, ls, pitch, h.ofirst[cw]);
    float ym[kVec];
#pragma unroll
    for (int c = 0; c < kVec; ++c) ym[c] = -INFINITY;
#pragma unroll
    for (int j = 0; j < kJT; ++j) {
      if (j > 0) {
        if (adv & (1u << j))
          stream_step<T>(st, ls, pitch);
        else if (jump & (1u << j))
          stream_reset<T>(st, ls, pitch, otab[s * kTileJ + jg + j]);
      }
      const float w = wtab[s * kTileJ + jg + j];
      const f2 w2 = pk(w, w);
      float val[kVec];
      upk(fma2(w2, st.d[0], st.a[0]), val[0], val[1]);
      upk(fma2(w2, st.d[1], st.a[1]), val[2], val[3]);
#pragma unroll
      for (int c = 0; c < kVec; ++c) {
        if (val[c] > zmax[j][c]) {
          zmax[j][c] = val[c];
          az[j][c] = krow;
        }
        zsum[j][c] += val[c];
      }
      if (valid & (1u << j)) {
#pragma unroll
        for (int c = 0; c < kVec; ++c) ym[c] = fmaxf(ym[c], val[c]);
      }
    }
    float* yb = r.ybuf() + s * kX;
#pragma unroll
    for (int c = 0; c < kVec; ++c) atomic_max_f(yb + yidx(lane * kVec + c), ym[c]);
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.ydone()[s]);
  }

  const int x = jb.xbase + lane * kVec;
#pragma unroll
  for (int j = 0; j < kJT; ++j) {
    const int jj = jb.j0 + jg + j;
    if (jj >= jb.ny) break;
    const size_t row = (size_t)jj * jb.nx;
#pragma unroll
    for (int c = 0; c < kVec; ++c) {
      if (x + c >= jb.nx) break;
      float zm = zmax[j][c];
      int a = az[j][c];
      if (jb.ke < jb.nz && zm < 0.0f) {
        zm = 0.0f;
        a = jb.ke;
      }
      if (jb.zmip) jb.zmip[row + x + c] = zm;
      if (jb.zsum) jb.zsum[row + x + c] = zsum[j][c];
      if (jb.argz) jb.argz[row + x + c] = a;
    }
  }
  return ok;
}

}  // namespace
}  // namespace opm
