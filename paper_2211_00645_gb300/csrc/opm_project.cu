// Fused deskew + projection (Fig. 2d): z-MIP, z-sum, y-MIP and argmax-z of
// the deskewed volume, computed straight from the raw stack without ever
// writing the volume.
//
// Work decomposition (one CTA = 32 output columns j x X output columns x):
//  * Output row k of the volume reads only camera row k of the raw stack, at
//    the planes n0(j,k), n0(j,k)+1 of the CTA's 32 columns: a contiguous slab
//    of P planes.  A producer warp stages that slab, {X cols, 1 row, P planes},
//    into shared memory with one TMA load per row, several rows ahead, on an
//    mbarrier ring.  Planes outside [0, nscan) arrive as TMA zero fill, which
//    is exactly the zero padding of the interpolation.
//  * Four compute warps own 8 columns j each and VEC columns x per lane.  For
//    every staged row they walk their 8 columns in order, keeping the current
//    plane pair (a, b - a) in registers; a column that moves to the next plane
//    costs one shared-memory vector load, so each staged raw value is
//    converted to FP32 once per warp rather than once per voxel.  Plane steps
//    are warp-uniform bit masks computed by the producer.
//  * z-reductions (max, sum, first argmax) stay in registers across rows; the
//    y-max of each row is reduced over the CTA's 32 columns in shared memory
//    and folded into the global y-MIP with one coalesced atomic max per
//    column (max is order independent, so the result is deterministic).
//  * Only rows whose band can carry non-zero weight for the tile are visited;
//    all other rows are exactly zero and enter the maxima as the value 0.
// The fast variant (uint16 input, z-MIP and/or y-MIP only) stages two rows per
// step so that the z-max takes one 3-input max per voxel pair, uses packed
// FP32x2 FMAs, and splits each tile's row band into chunks whose z-maxima are
// combined with atomic max, which balances tiles of very different band length.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "opm_common.cuh"

namespace opm {

namespace {

constexpr int kNW = 4;               // compute warps per CTA
constexpr int kJT = kTileJ / kNW;    // columns j per compute warp (8)
constexpr int kStages = 4;           // TMA ring depth
constexpr int kThreads = 32 * (kNW + 1);
constexpr int kChunkRows = 128;      // rows per work unit in the fast variant
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: the kernel itself takes < 10 ms

static_assert(kJT * kNW == kTileJ, "tile");

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

// Float max on 32-bit words, valid for any sign (+0 and -0 compare equal up
// to their bit patterns; both are exact maxima of the same voxel set).
__device__ __forceinline__ void atomic_max_f(float* addr, float v) {
  if (v >= 0.0f)
    atomicMax(reinterpret_cast<int*>(addr), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned*>(addr), __float_as_uint(v));
}

// --------------------------------------------------------------- layout
struct __align__(16) RowHdr {
  int k;           // camera row staged (>= nz: padding row, all zero)
  int nlo;         // first staged plane
  unsigned adv;    // bit j: column j is one plane above column j-1
  unsigned jump;   // bit j: column j is more than one plane above column j-1
  unsigned valid;  // bit j: column j lies inside the output grid
  int ofirst[kNW]; // slab offset of the first column of each compute warp
  int pad[3];
};
static_assert(sizeof(RowHdr) == 48, "hdr");

template <typename T, int VEC, int ROWS>
struct Layout {
  static constexpr int X = 32 * VEC;  // columns x per CTA
  // slab rows 0..P-1 come from TMA, rows P and P+1 stay zero
  __host__ __device__ static size_t slab_row_bytes(int P) { return (size_t)(P + 2) * X * sizeof(T); }
  __host__ __device__ static size_t slab_stage_bytes(int P) { return ROWS * slab_row_bytes(P); }
  __host__ __device__ static size_t off_w(int P) { return kStages * slab_stage_bytes(P); }
  __host__ __device__ static size_t off_o(int P) { return off_w(P) + kStages * ROWS * kTileJ * 4; }
  __host__ __device__ static size_t off_hdr(int P) { return off_o(P) + kStages * ROWS * kTileJ * 4; }
  __host__ __device__ static size_t off_y(int P) { return off_hdr(P) + kStages * ROWS * sizeof(RowHdr); }
  __host__ __device__ static size_t off_bar(int P) { return off_y(P) + kStages * ROWS * X * 4; }
  __host__ __device__ static size_t total(int P) { return off_bar(P) + 2 * kStages * 8; }
};

// Conflict-free index of column xl (= 8*L + c for VEC = 8) in the y-max
// buffer: both the compute lanes (fixed c, 32 consecutive L) and the
// producer lanes (32 consecutive xl) hit 32 distinct banks.
template <int VEC>
__device__ __forceinline__ int yidx(int xl) {
  if constexpr (VEC == 8) {
    const int L = xl >> 3;
    return (L << 3) + ((xl & 7) ^ ((L >> 2) & 7));
  } else {
    const int L = xl >> 2;
    return (L << 2) + ((xl & 3) ^ ((L >> 3) & 3));
  }
}

struct ProjArgs {
  PlanView v;
  float* zmip;
  float* zsum;
  float* ymip;
  int32_t* argz;
  int P;       // staged planes per row
  int kchunk;  // rows per work unit (fast variant)
};

// Load VEC raw values of one staged row for this lane and return them as
// FP32 pairs.
template <typename T, int VEC>
__device__ __forceinline__ void lds_row(const unsigned char* p, f2 (&out)[VEC / 2]) {
  if constexpr (std::is_same<T, uint16_t>::value && VEC == 8) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    out[0] = u16x2_to_f2(u.x);
    out[1] = u16x2_to_f2(u.y);
    out[2] = u16x2_to_f2(u.z);
    out[3] = u16x2_to_f2(u.w);
  } else if constexpr (std::is_same<T, uint16_t>::value && VEC == 4) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    out[0] = u16x2_to_f2(u.x);
    out[1] = u16x2_to_f2(u.y);
  } else {
    static_assert(std::is_same<T, float>::value && VEC == 4, "vector shape");
    const float4 f = *reinterpret_cast<const float4*>(p);
    out[0] = pk(f.x, f.y);
    out[1] = pk(f.z, f.w);
  }
}

// One staged row's streaming state for a compute lane.
template <int VEC>
struct Stream {
  f2 a[VEC / 2];  // R~[o]
  f2 d[VEC / 2];  // R~[o+1] - R~[o]
  int o;          // slab offset of the current lower plane
};

template <typename T, int VEC>
__device__ __forceinline__ void stream_reset(Stream<VEC>& st, const unsigned char* slab, size_t pitch,
                                             int o) {
  f2 b[VEC / 2];
  st.o = o;
  lds_row<T, VEC>(slab + (size_t)o * pitch, st.a);
  lds_row<T, VEC>(slab + (size_t)(o + 1) * pitch, b);
#pragma unroll
  for (int i = 0; i < VEC / 2; ++i) st.d[i] = sub2(b[i], st.a[i]);
}

template <typename T, int VEC>
__device__ __forceinline__ void stream_step(Stream<VEC>& st, const unsigned char* slab, size_t pitch) {
  f2 b[VEC / 2];
  st.o += 1;
  lds_row<T, VEC>(slab + (size_t)(st.o + 1) * pitch, b);
  if constexpr (std::is_same<T, uint16_t>::value) {
    // integers below 2^24: a + (b - a) == b exactly
#pragma unroll
    for (int i = 0; i < VEC / 2; ++i) {
      st.a[i] = add2(st.a[i], st.d[i]);
      st.d[i] = sub2(b[i], st.a[i]);
    }
  } else {
    f2 a[VEC / 2];
    lds_row<T, VEC>(slab + (size_t)st.o * pitch, a);
#pragma unroll
    for (int i = 0; i < VEC / 2; ++i) {
      st.a[i] = a[i];
      st.d[i] = sub2(b[i], a[i]);
    }
  }
}

// =====================================================================
// TMA kernel.  FAST: uint16, two rows per stage, z-MIP/y-MIP only, row band
// split into chunks (z-MIP combined with atomic max).  !FAST: one row per
// stage, every output, whole row band per CTA.
template <typename T, int VEC, int ROWS, bool FAST>
__global__ void __launch_bounds__(kThreads, 1)
k_project_tma(const __grid_constant__ CUtensorMap tmap, const ProjArgs args) {
  using L = Layout<T, VEC, ROWS>;
  constexpr int X = L::X;
  const PlanView& v = args.v;
  const int P = args.P;
  const int jt = blockIdx.x;
  const int j0 = jt * kTileJ;
  const int xbase = blockIdx.z * X;
  const Band band = v.band[jt];
  int ks = band.lo, ke = band.hi;
  if constexpr (FAST) {
    ks = max(ks, (int)blockIdx.y * args.kchunk);
    ke = min(ke, ((int)blockIdx.y + 1) * args.kchunk);
    if (ks >= ke) return;
  }
  const int nst = (ke - ks + ROWS - 1) / ROWS;

  extern __shared__ __align__(128) unsigned char smem[];
  const size_t pitch = (size_t)X * sizeof(T);
  float* wtab = reinterpret_cast<float*>(smem + L::off_w(P));
  int* otab = reinterpret_cast<int*>(smem + L::off_o(P));
  RowHdr* hdr = reinterpret_cast<RowHdr*>(smem + L::off_hdr(P));
  float* ybuf = reinterpret_cast<float*>(smem + L::off_y(P));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar(P));
  uint64_t* ydone = full + kStages;
  auto slab = [&](int s, int r) { return smem + (size_t)s * L::slab_stage_bytes(P) + (size_t)r * L::slab_row_bytes(P); };
  const float yreset = FAST ? 0.0f : -INFINITY;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ydone[s], kNW);
    }
    fence_barrier_init();
  }
  // zero rows P, P+1 of every staged row; reset the y-max buffers
  for (int s = 0; s < kStages; ++s)
    for (int r = 0; r < ROWS; ++r) {
      uint4* z = reinterpret_cast<uint4*>(slab(s, r) + (size_t)P * pitch);
      for (int i = threadIdx.x; i < (int)(2 * pitch / 16); i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
    }
  for (int i = threadIdx.x; i < kStages * ROWS * X; i += kThreads) ybuf[i] = yreset;
  __syncthreads();

  if (warp == 0) {
    // ------------------------------------------------------ producer warp
    const int jl = j0 + lane;
    const bool jvalid = jl < v.ny;
    const Split a = v.A[jvalid ? jl : v.ny - 1];
    bool ok = true;
    int nst_issued = 0;
    for (int it = 0; it < nst + kStages && ok; ++it) {
      if (it >= kStages) {
        // retire stage it - S: fold its y-max into the global y-MIP
        const int r_it = it - kStages;
        const int s = r_it % kStages;
        ok = mbar_wait(&ydone[s], (r_it / kStages) & 1, v.err);
        if (!ok) break;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int k = hdr[s * ROWS + r].k;
          float* yb = ybuf + (s * ROWS + r) * X;
#pragma unroll
          for (int i = 0; i < VEC; ++i) {
            const int xl = 32 * i + lane;
            const int yi = yidx<VEC>(xl);
            const float val = yb[yi];
            yb[yi] = yreset;
            if (args.ymip && k < v.nz && xbase + xl < v.nx) {
              if constexpr (FAST)
                atomicMax(reinterpret_cast<int*>(args.ymip + (size_t)k * v.nx + xbase + xl), __float_as_int(val));
              else
                atomic_max_f(args.ymip + (size_t)k * v.nx + xbase + xl, val);
            }
          }
        }
        __syncwarp();
      }
      if (it < nst) {
        // issue stage it: plane table of its rows, then the TMA loads
        const int s = it % kStages;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int k = ks + it * ROWS + r;
          const bool kvalid = k < v.nz;
          const Split b = v.B[kvalid ? k : v.nz - 1];
          int n0;
          float w;
          plane_weight(a, b, v.linear, n0, w);
          const int nlo = __shfl_sync(0xffffffffu, n0, 0);
          const bool valid = jvalid && kvalid;
          int o = n0 - nlo;
          if (!valid) {
            o = P;  // the two zero rows
            w = 0.0f;
          } else if (o < 0 || o > P - 2) {
            atomicOr(v.err, kErrSlabRange);
            o = min(max(o, 0), P - 2);
          }
          const int op = __shfl_up_sync(0xffffffffu, o, 1);
          const bool first = (lane % kJT) == 0;
          const unsigned adv = __ballot_sync(0xffffffffu, !first && o == op + 1);
          const unsigned jump = __ballot_sync(0xffffffffu, !first && o != op && o != op + 1);
          const unsigned vmask = __ballot_sync(0xffffffffu, valid);
          wtab[(s * ROWS + r) * kTileJ + lane] = w;
          otab[(s * ROWS + r) * kTileJ + lane] = o;
          const int of = __shfl_sync(0xffffffffu, o, (lane % kNW) * kJT);
          RowHdr& h = hdr[s * ROWS + r];
          if (lane < kNW) h.ofirst[lane] = of;
          if (lane == 0) {
            h.k = k;
            h.nlo = kvalid ? nlo : 0;
            h.adv = adv;
            h.jump = jump;
            h.valid = vmask;
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive_tx(&full[s], (unsigned)(ROWS * P * pitch));
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            const RowHdr& h = hdr[s * ROWS + r];
            tma_load_3d(slab(s, r), &tmap, &full[s], xbase, h.k, h.nlo);
          }
        }
        nst_issued = it + 1;
        __syncwarp();
      }
    }
    if (!ok) {
      // on failure, let the copies this warp issued land (bounded) before the
      // CTA's shared memory is released
      const int issued = min(nst, nst_issued);
      for (int q = max(0, issued - kStages); q < issued; ++q)
        (void)mbar_wait(&full[q % kStages], (q / kStages) & 1, v.err, 50000000ull);
    }
    return;
  }

  // -------------------------------------------------------- compute warps
  const int g = warp - 1;
  const int jg = g * kJT;  // first column of this warp inside the tile
  const unsigned lanebit = (lane < kJT) ? (1u << (jg + lane)) : 0u;

  float zmax[kJT][VEC];
  float zsum[FAST ? 1 : kJT][FAST ? 1 : VEC];
  int az[FAST ? 1 : kJT][FAST ? 1 : VEC];
  {
    const float zinit = (FAST || ks > 0) ? 0.0f : -INFINITY;
#pragma unroll
    for (int j = 0; j < kJT; ++j)
#pragma unroll
      for (int c = 0; c < VEC; ++c) zmax[j][c] = zinit;
    if constexpr (!FAST) {
#pragma unroll
      for (int j = 0; j < kJT; ++j)
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
          zsum[j][c] = 0.0f;
          az[j][c] = 0;
        }
    }
  }

  for (int it = 0; it < nst; ++it) {
    const int s = it % kStages;
    if (!mbar_wait(&full[s], (it / kStages) & 1, v.err)) break;

    Stream<VEC> st[ROWS];
    unsigned adv[ROWS], jump[ROWS], valid[ROWS];
    int krow[ROWS];
    float wv[ROWS][kJT];
    const unsigned char* sl[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const RowHdr& h = hdr[s * ROWS + r];
      krow[r] = h.k;
      // warp-uniform masks (bit j = column jg + j)
      adv[r] = __ballot_sync(0xffffffffu, (h.adv & lanebit) != 0);
      jump[r] = __ballot_sync(0xffffffffu, (h.jump & lanebit) != 0);
      valid[r] = __ballot_sync(0xffffffffu, (h.valid & lanebit) != 0);
      const float4* wp = reinterpret_cast<const float4*>(wtab + (s * ROWS + r) * kTileJ + jg);
#pragma unroll
      for (int q = 0; q < kJT / 4; ++q) {
        const float4 w4 = wp[q];
        wv[r][4 * q + 0] = w4.x;
        wv[r][4 * q + 1] = w4.y;
        wv[r][4 * q + 2] = w4.z;
        wv[r][4 * q + 3] = w4.w;
      }
      sl[r] = slab(s, r) + (size_t)lane * VEC * sizeof(T);
      stream_reset<T, VEC>(st[r], sl[r], pitch, h.ofirst[g]);
    }

    float ym[ROWS][VEC];
    float vprev[ROWS][VEC];
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int c = 0; c < VEC; ++c) ym[r][c] = yreset;

#pragma unroll
    for (int j = 0; j < kJT; ++j) {
      float val[ROWS][VEC];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if (j > 0) {
          if (adv[r] & (1u << j)) {
            stream_step<T, VEC>(st[r], sl[r], pitch);
          } else if (jump[r] & (1u << j)) {
            stream_reset<T, VEC>(st[r], sl[r], pitch, otab[(s * ROWS + r) * kTileJ + jg + j]);
          }
        }
        const f2 w2 = pk(wv[r][j], wv[r][j]);
#pragma unroll
        for (int i = 0; i < VEC / 2; ++i) upk(fma2(w2, st[r].d[i], st[r].a[i]), val[r][2 * i], val[r][2 * i + 1]);
      }
      // z-reductions
      if constexpr (ROWS == 2) {
#pragma unroll
        for (int c = 0; c < VEC; ++c) zmax[j][c] = max3(zmax[j][c], val[0][c], val[1][c]);
      } else if constexpr (FAST) {
#pragma unroll
        for (int c = 0; c < VEC; ++c) zmax[j][c] = fmaxf(zmax[j][c], val[0][c]);
      } else {
#pragma unroll
        for (int c = 0; c < VEC; ++c) {
          const float vv = val[0][c];
          if (vv > zmax[j][c]) {
            zmax[j][c] = vv;
            az[j][c] = krow[0];
          }
          zsum[j][c] += vv;
        }
      }
      // y-max over this warp's columns (pairs of columns per 3-input max)
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        if constexpr (FAST) {
          if (j & 1) {
#pragma unroll
            for (int c = 0; c < VEC; ++c) ym[r][c] = max3(ym[r][c], vprev[r][c], val[r][c]);
          } else {
#pragma unroll
            for (int c = 0; c < VEC; ++c) vprev[r][c] = val[r][c];
          }
        } else {
          if (valid[r] & (1u << j)) {
#pragma unroll
            for (int c = 0; c < VEC; ++c) ym[r][c] = fmaxf(ym[r][c], val[r][c]);
          }
        }
      }
    }
    if constexpr (FAST && (kJT & 1)) {
#pragma unroll
      for (int r = 0; r < ROWS; ++r)
#pragma unroll
        for (int c = 0; c < VEC; ++c) ym[r][c] = fmaxf(ym[r][c], vprev[r][c]);
    }
    // combine the y-max of the CTA's four warps in shared memory
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      float* yb = ybuf + (s * ROWS + r) * X;
#pragma unroll
      for (int c = 0; c < VEC; ++c) {
        float* addr = yb + yidx<VEC>(lane * VEC + c);
        if constexpr (FAST)
          atomicMax(reinterpret_cast<int*>(addr), __float_as_int(ym[r][c]));
        else
          atomic_max_f(addr, ym[r][c]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&ydone[s]);
  }

  // ------------------------------------------------------------ epilogue
  const int x = xbase + lane * VEC;
#pragma unroll
  for (int j = 0; j < kJT; ++j) {
    const int jj = j0 + jg + j;
    if (jj >= v.ny) break;
    const size_t row = (size_t)jj * v.nx;
#pragma unroll
    for (int c = 0; c < VEC; ++c) {
      if (x + c >= v.nx) break;
      if constexpr (FAST) {
        if (args.zmip) atomicMax(reinterpret_cast<int*>(args.zmip + row + x + c), __float_as_int(zmax[j][c]));
      } else {
        float zm = zmax[j][c];
        int a = az[j][c];
        if (ke < v.nz && zm < 0.0f) {  // rows after the band are exactly zero
          zm = 0.0f;
          a = ke;
        }
        if (args.zmip) args.zmip[row + x + c] = zm;
        if (args.zsum) args.zsum[row + x + c] = zsum[j][c];
        if (args.argz) args.argz[row + x + c] = a;
      }
    }
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

// Initial values of the atomically combined outputs.
__global__ void k_init_outputs(PlanView v, float* zmip, float* ymip, int fast) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nzm = zmip ? (long long)v.ny * v.nx : 0;
  const long long nym = ymip ? (long long)v.nz * v.nx : 0;
  if (idx < nzm) zmip[idx] = 0.0f;
  if (idx < nym) ymip[idx] = fast ? 0.0f : v.yinit[idx / v.nx];
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

template <typename T, int VEC, int ROWS, bool FAST>
opm_status run_tma(const opm_plan* p, const void* raw, const ProjArgs& args, cudaStream_t s) {
  using Lt = Layout<T, VEC, ROWS>;
  const PlanView& v = p->view;
  const size_t smem = Lt::total(args.P);
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const cuuint64_t dims[3] = {(cuuint64_t)v.ncols, (cuuint64_t)v.nrows, (cuuint64_t)v.nscan};
  const cuuint64_t strides[2] = {(cuuint64_t)v.ncols * sizeof(T), (cuuint64_t)v.nrows * v.ncols * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)Lt::X, 1u, (cuuint32_t)args.P};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt =
      std::is_same<T, uint16_t>::value ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult cr = encode_fn()(&map, dt, 3, const_cast<void*>(raw), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(OPM_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")");

  auto kern = k_project_tma<T, VEC, ROWS, FAST>;
  static int attr_set[64] = {0};
  const int dev = p->device;
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin_smem(dev));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    attr_set[dev] = 1;
  }
  const int jtiles = (v.ny + kTileJ - 1) / kTileJ;
  const int xtiles = (v.nx + Lt::X - 1) / Lt::X;
  const int chunks = FAST ? (v.nz + args.kchunk - 1) / args.kchunk : 1;
  if (jtiles > 0x7fffffff || chunks > 65535 || xtiles > 65535)
    return fail(OPM_ERR_UNSUPPORTED, "projection grid exceeds launch limits");
  dim3 grid(jtiles, chunks, xtiles);
  kern<<<grid, kThreads, smem, s>>>(map, args);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? OPM_OK : cuda_fail(e, "launch k_project_tma");
}

}  // namespace

opm_status launch_project(const opm_plan* p, const void* raw, opm_dtype in_t, float* zmip, float* zsum,
                          float* ymip, int32_t* argz, cudaStream_t s) {
  const PlanView& v = p->view;
  const size_t es = in_t == OPM_U16 ? 2 : 4;
  const double pd = std::floor((kTileJ - 1) * p->rho) + 4.0;
  const int P = pd > 256.0 ? 257 : (int)pd;
  const bool fast = in_t == OPM_U16 && !zsum && !argz;
  const int smem_need = (int)(fast ? Layout<uint16_t, 8, 2>::total(P)
                                   : (in_t == OPM_U16 ? Layout<uint16_t, 4, 1>::total(P)
                                                      : Layout<float, 4, 1>::total(P)));
  const bool tma_ok = !p->force_generic && encode_fn() != nullptr && ((uintptr_t)raw % 16 == 0) &&
                      ((size_t)v.ncols * es) % 16 == 0 && P <= 256 &&
                      smem_need <= max_optin_smem(p->device);

  if (!tma_ok) {
    const long long nzx = (long long)v.ny * v.nx, nyx = (long long)v.nz * v.nx;
    const int tb = 256;
    if (zmip || zsum || argz) {
      const long long nb = (nzx + tb - 1) / tb;
      if (nb > 0x7fffffffLL) return fail(OPM_ERR_UNSUPPORTED, "grid too large");
      if (in_t == OPM_U16)
        k_zproj_plain<uint16_t><<<(unsigned)nb, tb, 0, s>>>(v, static_cast<const uint16_t*>(raw), zmip, zsum, argz);
      else
        k_zproj_plain<float><<<(unsigned)nb, tb, 0, s>>>(v, static_cast<const float*>(raw), zmip, zsum, argz);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "launch k_zproj_plain");
    }
    if (ymip) {
      const long long nb = (nyx + tb - 1) / tb;
      if (nb > 0x7fffffffLL) return fail(OPM_ERR_UNSUPPORTED, "grid too large");
      if (in_t == OPM_U16)
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
    k_init_outputs<<<(unsigned)nb, 256, 0, s>>>(v, zinit, ymip, fast ? 1 : 0);
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
  args.kchunk = kChunkRows;
  if (fast) return run_tma<uint16_t, 8, 2, true>(p, raw, args, s);
  if (in_t == OPM_U16) return run_tma<uint16_t, 4, 1, false>(p, raw, args, s);
  return run_tma<float, 4, 1, false>(p, raw, args, s);
}

}  // namespace opm
