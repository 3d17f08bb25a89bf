// Device building blocks shared by the projection kernels: TMA and mbarrier
// wrappers, packed FP32x2 arithmetic, exact uint16 -> FP32 conversion, the
// per-lane plane streams, and the fast kernel's shared-memory layout and
// per-job producer / consumer loops (one job = one 32-column j-tile of one
// 128-column x-tile over a range of camera rows).
#pragma once

#include <cuda.h>

#include "opm_common.cuh"

namespace opm {
namespace {

constexpr int kNW = 4;               // compute warps per CTA
constexpr int kJT = kTileJ / kNW;    // columns j per compute warp (8)
constexpr int kThreads = 32 * (kNW + 1);
constexpr int kVec = 4;              // columns x per lane
constexpr int kX = 32 * kVec;        // columns x per CTA
constexpr int kStagesFast = 6;       // TMA ring depth, fast kernel
constexpr int kStagesGen = 4;        // TMA ring depth, general kernel
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: a launch takes < 10 ms

static_assert(kJT * kNW == kTileJ, "tile");
static_assert(kX == kUnitX, "work units and the fast kernels' x-tiles agree");

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: gives up after `limit_ns`, or at once when another warp of
// any CTA has already recorded a timeout in the plan's error word.  Returns
// false (and records the timeout) when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned* err,
                                          uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (unsigned i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 0) {
      if (*reinterpret_cast<volatile unsigned*>(err) & kErrWaitTimeout) return false;
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicOr(err, kErrWaitTimeout);
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
      "%5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Packed FP32x2 arithmetic (one instruction per pair on sm_100-family parts).
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float lo, float hi) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float max3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Two uint16 counts -> FP32x2, exactly: build 2^23 + u in the float bit
// pattern with a byte permute, then subtract 2^23 from both halves.
__device__ __forceinline__ f2 u16x2_to_f2(uint32_t w) {
  const uint32_t lo = __byte_perm(w, 0x4B000000u, 0x7610);
  const uint32_t hi = __byte_perm(w, 0x4B000000u, 0x7632);
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
  return sub2(r, pk(8388608.0f, 8388608.0f));
}

// Float max on 32-bit words, valid for any sign.
__device__ __forceinline__ void atomic_max_f(float* addr, float v) {
  if (v >= 0.0f)
    atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned*>(addr), __float_as_uint(v));
}

// Conflict-free index of column xl = 4L + c (L = owning lane) in a y-max
// buffer: the compute lanes (fixed c, 32 consecutive L) and the producer
// lanes (32 consecutive xl) both hit 32 distinct banks.
__device__ __forceinline__ int yidx(int xl) {
  const int L = xl >> 2;
  return (L << 2) + ((xl & 3) ^ ((L >> 3) & 3));
}

// 4 raw values of one staged row (this lane's 4 columns) as two FP32 pairs.
template <typename T>
__device__ __forceinline__ void lds_row(const unsigned char* p, f2 (&out)[2]) {
  if constexpr (std::is_same<T, uint16_t>::value) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    out[0] = u16x2_to_f2(u.x);
    out[1] = u16x2_to_f2(u.y);
  } else {
    const float4 f = *reinterpret_cast<const float4*>(p);
    out[0] = pk(f.x, f.y);
    out[1] = pk(f.z, f.w);
  }
}

// One staged row's streaming state for a compute lane: the lower plane a
// and the difference d = b - a at slab offset o.
struct Stream {
  f2 a[2];
  f2 d[2];
  int o;
};

template <typename T>
__device__ __forceinline__ void stream_reset(Stream& st, const unsigned char* lane_slab, int pitch, int o) {
  f2 b[2];
  st.o = o;
  lds_row<T>(lane_slab + o * pitch, st.a);
  lds_row<T>(lane_slab + (o + 1) * pitch, b);
  st.d[0] = sub2(b[0], st.a[0]);
  st.d[1] = sub2(b[1], st.a[1]);
}

template <typename T>
__device__ __forceinline__ void stream_step(Stream& st, const unsigned char* lane_slab, int pitch) {
  f2 b[2];
  st.o += 1;
  lds_row<T>(lane_slab + (st.o + 1) * pitch, b);
  if constexpr (std::is_same<T, uint16_t>::value) {
    // integers below 2^24: a + (b - a) == b exactly
    st.a[0] = add2(st.a[0], st.d[0]);
    st.a[1] = add2(st.a[1], st.d[1]);
  } else {
    lds_row<T>(lane_slab + st.o * pitch, st.a);
  }
  st.d[0] = sub2(b[0], st.a[0]);
  st.d[1] = sub2(b[1], st.a[1]);
}

// Streaming on 32-bit shared-memory offsets for the fast kernel (uint16
// slab): besides the pair (a, d) the lane keeps the raw words of the next
// plane, loaded right after each step, so that a step converts data already
// in registers instead of waiting for a shared-memory load.  `nxo` is the
// offset of those words (plane o + 2).  It may point one plane past the
// row's slab: the ring is followed by its tables, so the load stays inside
// the CTA's shared memory, and a plane past the slab is never stepped onto.
struct StreamPF {
  f2 a[2];
  f2 d[2];
  uint2 nxt;     // raw words of plane o + 2
  uint32_t nxo;  // their shared-memory offset
};

__device__ __forceinline__ void lds_row_u16(const unsigned char* smem, uint32_t off, f2 (&out)[2]) {
  const uint2 u = *reinterpret_cast<const uint2*>(smem + off);
  out[0] = u16x2_to_f2(u.x);
  out[1] = u16x2_to_f2(u.y);
}

__device__ __forceinline__ void stream_reset_u16(StreamPF& st, const unsigned char* smem, uint32_t lane_off,
                                                 uint32_t pitch, int o) {
  f2 b[2];
  const uint32_t off = lane_off + (uint32_t)o * pitch;
  lds_row_u16(smem, off, st.a);
  lds_row_u16(smem, off + pitch, b);
  st.nxo = off + 2 * pitch;
  st.nxt = *reinterpret_cast<const uint2*>(smem + st.nxo);
  st.d[0] = sub2(b[0], st.a[0]);
  st.d[1] = sub2(b[1], st.a[1]);
}

__device__ __forceinline__ void stream_step_u16(StreamPF& st, const unsigned char* smem, uint32_t pitch) {
  f2 b[2];
  b[0] = u16x2_to_f2(st.nxt.x);
  b[1] = u16x2_to_f2(st.nxt.y);
  st.nxo += pitch;
  st.nxt = *reinterpret_cast<const uint2*>(smem + st.nxo);
  // integers below 2^24: a + (b - a) == b exactly
  st.a[0] = add2(st.a[0], st.d[0]);
  st.a[1] = add2(st.a[1], st.d[1]);
  st.d[0] = sub2(b[0], st.a[0]);
  st.d[1] = sub2(b[1], st.a[1]);
}

// =====================================================================
// Fast kernel: uint16, z-MIP and/or y-MIP, plans whose full 32-column
// windows never skip a plane.  Per stage (two camera rows) the producer only
// waits for a free slot and issues four asynchronous copies: the two raw
// slabs (TMA) and the two precomputed plane tables (bulk copies).  The
// compute warps fold the y-max of each stage into the global y-MIP
// themselves, 32 columns per warp, after an mbarrier rendezvous.
namespace fast {

constexpr int S = kStagesFast;

__host__ __device__ inline size_t slab_row_bytes(int P) { return (size_t)P * kX * 2; }
__host__ __device__ inline size_t stage_slab_bytes(int P) { return 2 * slab_row_bytes(P); }
__host__ __device__ inline size_t off_tab(int P) { return S * stage_slab_bytes(P); }        // FastRow [S][2]
__host__ __device__ inline size_t off_ybuf(int P) { return off_tab(P) + S * 2 * sizeof(FastRow); }  // float [S][2][kX]
__host__ __device__ inline size_t off_bar(int P) { return off_ybuf(P) + S * 2 * kX * 4; }
__host__ __device__ inline size_t off_jobs(int P) { return off_bar(P) + 3 * S * 8; }  // JobS [kNW]
__host__ __device__ inline size_t total(int P) { return off_jobs(P) + kNW * 48; }

}  // namespace fast

__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One fast-kernel job: a 32-column j-tile of a 128-column x-tile of one
// stack, over camera rows [ks, ke), staged two rows per ring stage.
struct FastJob {
  const CUtensorMap* tmap;  // the stack's raw tensor map (box {128, 1, P})
  const FastRow* rows;      // plane tables of this j-tile, indexed by camera row
  const int* nlos;          // first staged plane of this j-tile, per camera row
  float* zmip;              // [ny][nx] or NULL
  float* ymip;              // [nz][nx] or NULL
  int nz, nx, j0, xbase, ks, ke, P;
};

// A compute warp's job fields that are only needed at the end of a stage or
// of the job.  They are parked in shared memory and re-read there, so that
// they hold no registers through the column loop.
struct JobS {
  float* zmip;
  float* ymip;
  int nx, nz, j0, xbase;
  int k0g;   // camera row of stage g is k0g + 2 g
  int gend;  // stage count at the end of the job
  int pad[2];
};
static_assert(sizeof(JobS) == 48, "JobS layout");

// The ring in shared memory, laid out for slab depth Pl (>= every job's P).
// Region addresses are recomputed from the base on use rather than held in
// registers.
struct FastRing {
  unsigned char* base;
  int Pl;
  __device__ __forceinline__ FastRow* tab() const { return reinterpret_cast<FastRow*>(base + fast::off_tab(Pl)); }
  __device__ __forceinline__ float* ybuf() const { return reinterpret_cast<float*>(base + fast::off_ybuf(Pl)); }
  // producer -> consumers: slabs and tables landed
  __device__ __forceinline__ uint64_t* full() const { return reinterpret_cast<uint64_t*>(base + fast::off_bar(Pl)); }
  // consumers -> producer: slot free
  __device__ __forceinline__ uint64_t* ydone() const { return full() + fast::S; }
  // consumers -> consumers: y-max of the stage combined
  __device__ __forceinline__ uint64_t* cdone() const { return full() + 2 * fast::S; }
  // one per compute warp
  __device__ __forceinline__ JobS* jobs() const { return reinterpret_cast<JobS*>(base + fast::off_jobs(Pl)); }
};

__device__ __forceinline__ FastRing fast_ring(unsigned char* smem, int Pl) {
  FastRing r;
  r.base = smem;
  r.Pl = Pl;
  return r;
}

// Whole CTA: barrier init and y-max buffer reset, then a CTA barrier.
__device__ __forceinline__ void fast_ring_init(const FastRing& r) {
  using namespace fast;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&r.full()[s], 1);
      mbar_init(&r.ydone()[s], kNW);
      mbar_init(&r.cdone()[s], kNW);
    }
    fence_barrier_init();
  }
  for (int i = threadIdx.x; i < S * 2 * kX; i += blockDim.x) r.ybuf()[i] = 0.0f;
  __syncthreads();
}

// Producer warp: stage the job's rows.  `g` is the CTA's running stage
// count (ring slot and phase), advanced by the job's stage count.
__device__ __forceinline__ bool fast_produce(const FastJob& jb, const FastRing& r, int& g, unsigned* err,
                                             int lane) {
  using namespace fast;
  const uint32_t pitch = kX * 2;
  const int nst = (jb.ke - jb.ks + 1) / 2;
  int kbase = jb.ks;  // first staged planes of 32 rows per load, one group ahead
  int ncur = jb.nlos[min(kbase + lane, jb.nz - 1)];
  int nnext = jb.nlos[min(kbase + 32 + lane, jb.nz - 1)];
#pragma unroll 1
  for (int it = 0; it < nst; ++it, ++g) {
    const int s = g % S;
    if (g >= S && !mbar_wait(&r.ydone()[s], ((g - S) / S) & 1, err)) return false;
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
      unsigned char* slab = r.base + s * stage_slab_bytes(r.Pl);
      mbar_arrive_tx(&r.full()[s], (unsigned)(2 * jb.P * pitch + 2 * sizeof(FastRow)));
      tma_load_3d(slab, jb.tmap, &r.full()[s], jb.xbase, k0, nlo[0]);
      tma_load_3d(slab + slab_row_bytes(r.Pl), jb.tmap, &r.full()[s], jb.xbase, k1, k1 < jb.nz ? nlo[1] : 0);
      bulk_load(&r.tab()[s * 2 + 0], jb.rows + k0, sizeof(FastRow), &r.full()[s]);
      bulk_load(&r.tab()[s * 2 + 1], jb.rows + min(k1, jb.nz - 1), sizeof(FastRow), &r.full()[s]);
    }
    __syncwarp();
  }
  return true;
}

// Producer warp, after its last job: the CTA's shared memory must outlive
// every copy it issued (bounded wait on the last S stages).
__device__ __forceinline__ void fast_drain(const FastRing& r, int g, bool ok, unsigned* err) {
  using namespace fast;
  for (int q = max(0, g - S); q < g; ++q)
    if (!mbar_wait(&r.full()[q % S], (q / S) & 1, err, ok ? kWaitLimitNs : 50000000ull)) break;
}

__device__ __forceinline__ int lds_volatile_s32(const int* p) {
  int v;
  asm volatile("ld.volatile.shared.s32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)));
  return v;
}

__device__ __forceinline__ float* lds_volatile_ptr(float* const* p) {
  unsigned long long v;
  asm volatile("ld.volatile.shared.u64 %0, [%1];" : "=l"(v) : "r"(smem_u32(p)));
  return reinterpret_cast<float*>(v);
}

// Compute warp cw (0..3): columns j0 + 8cw .. + 7 of the job, both rows of
// every stage; z-maxima in registers, folded into zmip at the end of the job;
// the y-max of each stage folded into ymip after the 4-warp rendezvous.
// Returns false when a bounded wait gave up.
__device__ __forceinline__ bool fast_consume(const FastJob& jb, const FastRing& r, int& g, unsigned* err,
                                             int cw, int lane) {
  using namespace fast;
  const uint32_t pitch = kX * 2;
  const unsigned char* smem = r.base;
  JobS* js = r.jobs() + cw;
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
  float zmax[kJT][kVec];
#pragma unroll
  for (int j = 0; j < kJT; ++j)
#pragma unroll
    for (int c = 0; c < kVec; ++c) zmax[j][c] = 0.0f;  // uint16 voxels are >= 0
  bool ok = true;

#pragma unroll 1
  for (; g < lds_volatile_s32(&js->gend); ++g) {
    const int s = g % S;
    const unsigned ph = (g / S) & 1;
    if (!mbar_wait(&r.full()[s], ph, err)) {
      ok = false;
      break;
    }
    const uint32_t lane0 = (uint32_t)(s * stage_slab_bytes(r.Pl)) + lane * (kVec * 2);
    const uint32_t lane1 = lane0 + (uint32_t)slab_row_bytes(r.Pl);
    const FastRec r0 = r.tab()[s * 2 + 0].rec[cw];
    const FastRec r1 = r.tab()[s * 2 + 1].rec[cw];
    // warp-uniform step masks (bit j: step before column j)
    const unsigned adv0 = __ballot_sync(0xffffffffu, lane < kJT && ((r0.adv >> lane) & 1u));
    const unsigned adv1 = __ballot_sync(0xffffffffu, lane < kJT && ((r1.adv >> lane) & 1u));
    StreamPF st0, st1;
    stream_reset_u16(st0, smem, lane0, pitch, r0.ofirst);
    stream_reset_u16(st1, smem, lane1, pitch, r1.ofirst);
    const uint32_t w0off = (uint32_t)(off_tab(r.Pl) + (s * 2 + 0) * sizeof(FastRow)) + cw * kJT * 8;
    const uint32_t w1off = w0off + (uint32_t)sizeof(FastRow);

    float ym0[kVec], ym1[kVec], vp0[kVec], vp1[kVec];
#pragma unroll
    for (int c = 0; c < kVec; ++c) ym0[c] = ym1[c] = 0.0f;

#pragma unroll
    for (int j = 0; j < kJT; ++j) {
      if (j > 0) {
        if (adv0 & (1u << j)) stream_step_u16(st0, smem, pitch);
        if (adv1 & (1u << j)) stream_step_u16(st1, smem, pitch);
      }
      const f2 w0 = *reinterpret_cast<const f2*>(smem + w0off + j * 8);
      const f2 w1 = *reinterpret_cast<const f2*>(smem + w1off + j * 8);
      float v0[kVec], v1[kVec];
      upk(fma2(w0, st0.d[0], st0.a[0]), v0[0], v0[1]);
      upk(fma2(w0, st0.d[1], st0.a[1]), v0[2], v0[3]);
      upk(fma2(w1, st1.d[0], st1.a[0]), v1[0], v1[1]);
      upk(fma2(w1, st1.d[1], st1.a[1]), v1[2], v1[3]);
#pragma unroll
      for (int c = 0; c < kVec; ++c) zmax[j][c] = max3(zmax[j][c], v0[c], v1[c]);
      if (j & 1) {
#pragma unroll
        for (int c = 0; c < kVec; ++c) {
          ym0[c] = max3(ym0[c], vp0[c], v0[c]);
          ym1[c] = max3(ym1[c], vp1[c], v1[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < kVec; ++c) {
          vp0[c] = v0[c];
          vp1[c] = v1[c];
        }
      }
    }
    // y-max: combine the four warps in shared memory, then each warp folds
    // 32 columns of both rows into the global y-MIP
    float* yb0 = r.ybuf() + (s * 2 + 0) * kX;
    float* yb1 = r.ybuf() + (s * 2 + 1) * kX;
#pragma unroll
    for (int c = 0; c < kVec; ++c) {
      const int yi = yidx(lane * kVec + c);
      atomicMax(reinterpret_cast<int*>(yb0 + yi), __float_as_int(ym0[c]));
      atomicMax(reinterpret_cast<int*>(yb1 + yi), __float_as_int(ym1[c]));
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.cdone()[s]);
    if (!mbar_wait(&r.cdone()[s], ph, err)) {
      ok = false;
      break;
    }
    {
      const int xl = 32 * cw + lane;
      const int yi = yidx(xl);
      const float y0 = yb0[yi], y1 = yb1[yi];
      yb0[yi] = 0.0f;
      yb1[yi] = 0.0f;
      float* ymip = lds_volatile_ptr(&js->ymip);
      const int nx = lds_volatile_s32(&js->nx);
      const int x = lds_volatile_s32(&js->xbase) + xl;
      const int k0 = lds_volatile_s32(&js->k0g) + 2 * g;
      if (ymip && x < nx) {
        atomicMax(reinterpret_cast<int*>(ymip + (size_t)k0 * nx + x), __float_as_int(y0));
        if (k0 + 1 < lds_volatile_s32(&js->nz))
          atomicMax(reinterpret_cast<int*>(ymip + (size_t)(k0 + 1) * nx + x), __float_as_int(y1));
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&r.ydone()[s]);
  }

  float* zmip = lds_volatile_ptr(&js->zmip);
  if (zmip) {
    const int nx = lds_volatile_s32(&js->nx);
    const int x = lds_volatile_s32(&js->xbase) + lane * kVec;
    const int jrow = lds_volatile_s32(&js->j0) + cw * kJT;
#pragma unroll
    for (int j = 0; j < kJT; ++j) {
      float* row = zmip + (size_t)(jrow + j) * nx;
#pragma unroll
      for (int c = 0; c < kVec; ++c)
        if (x + c < nx) atomicMax(reinterpret_cast<int*>(row + x + c), __float_as_int(zmax[j][c]));
    }
  }
  return ok;
}

}  // namespace
}  // namespace opm
