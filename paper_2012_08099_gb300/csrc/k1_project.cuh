// Step 1 of the Discrete Projection Moment method: one fused pass over the
// volume that writes every projection image at once (Sec. 3.1, Eq. 4 with
// the image set of Eqs. 5-9 and the +-pi/4 families).
//
// Work decomposition.  A CTA owns a tile of XT = 64 columns (x) by BY rows
// (y) and streams it along z.  Its 256 threads form TY = 16 row groups of
// TX = 16 threads (one half-warp per group); a thread holds a micro-tile of
// R = 4 x-values by BYT rows of every z-slice (BY = 16 * BYT = 64, or 32 for
// float volumes with six or more images, whose register state is larger,
// and for integer volumes with nine images).
// Persistent CTAs take contiguous ranges of (tile, z) units.  With 16-byte
// aligned rows each slice of a tile arrives as one tiled tensor copy
// (cp.async.bulk.tensor.3d + mbarrier, issued by one thread) into a ring of
// stages holding ~64 KB in flight per SM; otherwise every thread loads its
// micro-tile from global memory.
//
// Images whose lines leave the z-slice (directions z, (1,0,+-1), (0,1,+-1):
// images 0 and 3-6) accumulate in registers across z:
//   image 0    one accumulator per (x, y);
//   images 3/4 (x+-z, y): a window of R registers per row; after each step
//              the pixel that leaves a thread's window is handed to its
//              neighbour in the half-warp (shuffle), and the tile's edge
//              thread hands it on for emission, complete;
//   images 5/6 (y+-z, x): a window of BYT registers per column, handed to
//              the row group above/below through shared mailboxes.
// Images whose lines lie in the slice (images 1, 2, 7, 8) are reduced per
// step: row sums across the half-warp (image 1), column sums through
// shared slots (image 2), diagonal sums through shared buffers (7, 8).
// After each step a barrier hands these per-step results to all 256 threads,
// which merge them into the global images in an evenly divided task loop
// (for float volumes during the next step, between its sums and its
// in-slice reductions, so the merge's latencies overlap that work).
//
// Float volumes keep every sum compensated: each accumulator is a pair
// (hi, lo) updated with the error-free TwoSum, so a pixel carries float-float
// accuracy whatever the order and signs of its terms.  A pair that leaves
// the CTA is merged into the image's double pixel as two exact float-to-double
// conversions (integer bit operations) and two red.global.add.f64 in the L2;
// the SMs execute no FP64 instruction.  Integer volumes use exact uint32
// sums and red.global.add.u32.
#pragma once
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "dpma_internal.cuh"

namespace dpma {
namespace k1 {

constexpr int R = 4;          // x-values per thread
constexpr int TX = 16;        // threads per row group (a half-warp)
constexpr int TY = 16;        // row groups
constexpr int NT = TX * TY;   // threads per CTA
constexpr int XT = R * TX;    // tile width

// Bounded waits give up after ~2^31 cycles (about a second).
constexpr long long kWaitBudget = 1ll << 31;
constexpr int kStatusTimeout = 5;

// Rows per thread: see BYT below.
template <typename T, int P> struct TileCfg {
  static constexpr bool FL = std::is_same<T, float>::value;
  // 4 x 2 micro-tiles for float volumes with six or more images (register
  // state) and for integer volumes with nine (fewer diagonal cells per
  // thread: measured 6-37% faster at K = 8); 4 x 4 otherwise
  static constexpr int BYT = FL ? (P >= 6 ? 2 : 4) : (P >= 9 ? 2 : 4);
  static constexpr int BY = BYT * TY;
  // resident CTAs per SM (measured): two for every integer case and for
  // float volumes with 4 x 2 micro-tiles, where the extra warps hide more
  // latency than the few spills cost; one for float volumes with 4 or 5
  // images, whose 4 x 4 micro-tiles would spill heavily at 128 registers
  static constexpr int MINB = FL ? ((P == 4 || P == 5) ? 1 : 2) : 2;
  // ring depth: about 64 KB of slices in flight per SM, 4 to 16 stages
  static constexpr int SLICE = BY * XT * (int)sizeof(T);
  static constexpr int FLIGHT = 65536 / MINB;
  static constexpr int STAGES = SLICE * 4 >= FLIGHT ? 4 : (SLICE * 8 >= FLIGHT ? 8 : 16);
  static_assert(R % BYT == 0, "window rotations share the unroll period R");
};

struct K1Params {
  const void* vol;
  int64_t L, M, N;
  int64_t z0, nz;  // the launch projects slices z0 .. z0 + nz - 1
  int64_t nbands, nxt;
  int64_t units;  // nxt * nbands * nz
  int64_t cpt;    // CTAs per x-tile (grid = nxt * cpt), or 0: contiguous ranges
  ImageSet set;
  void* images;
  int* status;
  // when non-null the launch is a fallback: it does nothing unless
  // (*gate & 3) != 0 (the integer-lane projection flagged the volume)
  const int* gate;
};

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of an mbarrier, at most kWaitBudget cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity) {
  if (mbar_try_wait(a, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(a, parity))
    if (clock64() - t0 > kWaitBudget) return false;
  return true;
}
// One box of a 3-D tensor map (coordinates x, y, z; elements outside the
// tensor are filled with zeros and still counted in the transaction bytes).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

// ---------------------------------------------------------------- float helpers

// (hi, lo) += v with the error-free TwoSum: hi + lo stays exact up to the
// rounding of lo (at most one float32 rounding of the accumulated errors).
__device__ __forceinline__ void ts_acc(float& hi, float& lo, float v) {
  const float t = __fadd_rn(hi, v);
  const float bb = __fsub_rn(t, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(v, bb));
  lo = __fadd_rn(lo, e);
  hi = t;
}

// Float pairs held as one 64-bit register (low half first).
__device__ __forceinline__ uint64_t pk(float a, float b) {
  return (uint64_t)__float_as_uint(a) | ((uint64_t)__float_as_uint(b) << 32);
}
__device__ __forceinline__ float half_of(uint64_t p, int h) {
  return __uint_as_float(h ? (uint32_t)(p >> 32) : (uint32_t)p);
}
// (H, Lo) += V for the two pixels of a pair: two scalar TwoSums.  Scalar
// float adds issue to both halves of the FMA pipe, while packed f32x2 adds
// occupy only its heavy half; measured on sm_103a the scalar form is faster
// although it issues more instructions.
__device__ __forceinline__ void ts2(uint64_t& H, uint64_t& Lo, uint64_t V) {
  float h0 = half_of(H, 0), h1 = half_of(H, 1), l0 = half_of(Lo, 0), l1 = half_of(Lo, 1);
  ts_acc(h0, l0, half_of(V, 0));
  ts_acc(h1, l1, half_of(V, 1));
  H = pk(h0, h1);
  Lo = pk(l0, l1);
}

// (h, l) += (bh, bl): bh enters with TwoSum, bl is added to l (the pair is
// not renormalised; h + l keeps the sum to about 2^-48 of its magnitude).
__device__ __forceinline__ void pair_acc(float& h, float& l, float bh, float bl) {
  ts_acc(h, l, bh);
  l = __fadd_rn(l, bl);
}

// The double equal to a float32, from its bits (zero for subnormals, whose
// magnitude is below 2^-126).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0) return 0.0;
  const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// Merge the pair (hi, lo) into a double pixel: two exact conversions and two
// fire-and-forget L2 adds.
__device__ __forceinline__ void emit_ff(double* p, float hi, float lo) {
  if (hi != 0.f) atomicAdd(p, f32_to_f64_bits(hi));
  if (lo != 0.f) atomicAdd(p, f32_to_f64_bits(lo));
}
__device__ __forceinline__ void emit_u(uint32_t* p, uint32_t v) {
  if (v) atomicAdd(p, v);
}

// ---------------------------------------------------------------- loads

__device__ __forceinline__ void load4_global(const float* __restrict__ row, int64_t x, int64_t L,
                                             bool vec, float out[4]) {
  if (vec && x + R <= L) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(row + x));
    out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
    return;
  }
#pragma unroll
  for (int c = 0; c < R; ++c) out[c] = (x + c < L) ? row[x + c] : 0.f;
}
__device__ __forceinline__ void load4_global(const uint16_t* __restrict__ row, int64_t x, int64_t L,
                                             bool vec, uint32_t out[4]) {
  if (vec && x + R <= L) {
    const uint2 q = __ldcs(reinterpret_cast<const uint2*>(row + x));
    out[0] = q.x & 0xffffu; out[1] = q.x >> 16; out[2] = q.y & 0xffffu; out[3] = q.y >> 16;
    return;
  }
#pragma unroll
  for (int c = 0; c < R; ++c) out[c] = (x + c < L) ? (uint32_t)row[x + c] : 0u;
}
__device__ __forceinline__ void load4_global(const uint8_t* __restrict__ row, int64_t x, int64_t L,
                                             bool vec, uint32_t out[4]) {
  if (vec && x + R <= L) {
    const uint32_t q = __ldcs(reinterpret_cast<const unsigned int*>(row + x));
    out[0] = q & 0xffu; out[1] = (q >> 8) & 0xffu; out[2] = (q >> 16) & 0xffu; out[3] = q >> 24;
    return;
  }
#pragma unroll
  for (int c = 0; c < R; ++c) out[c] = (x + c < L) ? (uint32_t)row[x + c] : 0u;
}

__device__ __forceinline__ void load4_smem(const float* p, float out[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
}
__device__ __forceinline__ void load4_smem(const uint16_t* p, uint32_t out[4]) {
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  out[0] = q.x & 0xffffu; out[1] = q.x >> 16; out[2] = q.y & 0xffffu; out[3] = q.y >> 16;
}
__device__ __forceinline__ void load4_smem(const uint8_t* p, uint32_t out[4]) {
  const uint32_t q = *reinterpret_cast<const uint32_t*>(p);
  out[0] = q & 0xffu; out[1] = (q >> 8) & 0xffu; out[2] = (q >> 16) & 0xffu; out[3] = q >> 24;
}

// Float-float sum of BYT per-lane pairs across the 16 lanes of a half-warp,
// scattered so that lane tx with (tx % (16/BYT)) == 0 ends with row
// tx / (16/BYT).
template <int BYT>
__device__ __forceinline__ void ff_rows_half(const float h[BYT], const float l[BYT], int tx,
                                             float& oh, float& ol) {
  float kh, kl;
  if constexpr (BYT == 4) {
    const bool up = tx & 8;
    float k0h = up ? h[2] : h[0], k0l = up ? l[2] : l[0];
    float k1h = up ? h[3] : h[1], k1l = up ? l[3] : l[1];
    const float s0h = up ? h[0] : h[2], s0l = up ? l[0] : l[2];
    const float s1h = up ? h[1] : h[3], s1l = up ? l[1] : l[3];
    const float r0h = __shfl_xor_sync(0xffffffffu, s0h, 8), r0l = __shfl_xor_sync(0xffffffffu, s0l, 8);
    const float r1h = __shfl_xor_sync(0xffffffffu, s1h, 8), r1l = __shfl_xor_sync(0xffffffffu, s1l, 8);
    pair_acc(k0h, k0l, r0h, r0l);
    pair_acc(k1h, k1l, r1h, r1l);
    const bool up2 = tx & 4;
    kh = up2 ? k1h : k0h;
    kl = up2 ? k1l : k0l;
    const float sh = up2 ? k0h : k1h, sl = up2 ? k0l : k1l;
    const float qh = __shfl_xor_sync(0xffffffffu, sh, 4), ql = __shfl_xor_sync(0xffffffffu, sl, 4);
    pair_acc(kh, kl, qh, ql);
#pragma unroll
    for (int m = 2; m >= 1; m >>= 1) {
      const float th = __shfl_xor_sync(0xffffffffu, kh, m), tl = __shfl_xor_sync(0xffffffffu, kl, m);
      pair_acc(kh, kl, th, tl);
    }
  } else {
    const bool up = tx & 8;
    kh = up ? h[1] : h[0];
    kl = up ? l[1] : l[0];
    const float sh = up ? h[0] : h[1], sl = up ? l[0] : l[1];
    const float rh = __shfl_xor_sync(0xffffffffu, sh, 8), rl = __shfl_xor_sync(0xffffffffu, sl, 8);
    pair_acc(kh, kl, rh, rl);
#pragma unroll
    for (int m = 4; m >= 1; m >>= 1) {
      const float th = __shfl_xor_sync(0xffffffffu, kh, m), tl = __shfl_xor_sync(0xffffffffu, kl, m);
      pair_acc(kh, kl, th, tl);
    }
  }
  oh = kh;
  ol = kl;
}

// Integer counterpart: sum of BYT per-lane values across the half-warp,
// lane tx with (tx % (16/BYT)) == 0 ending with row tx / (16/BYT).
template <int BYT>
__device__ __forceinline__ uint32_t u_rows_half(const uint32_t h[BYT], int tx) {
  uint32_t k;
  if constexpr (BYT == 4) {
    const bool up = tx & 8;
    uint32_t k0 = up ? h[2] : h[0], k1 = up ? h[3] : h[1];
    k0 += __shfl_xor_sync(0xffffffffu, up ? h[0] : h[2], 8);
    k1 += __shfl_xor_sync(0xffffffffu, up ? h[1] : h[3], 8);
    const bool up2 = tx & 4;
    k = up2 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, up2 ? k0 : k1, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
  } else {
    const bool up = tx & 8;
    k = up ? h[1] : h[0];
    k += __shfl_xor_sync(0xffffffffu, up ? h[0] : h[1], 8);
#pragma unroll
    for (int m = 4; m >= 1; m >>= 1) k += __shfl_xor_sync(0xffffffffu, k, m);
  }
  return k;
}

// ---------------------------------------------------------------- kernel

// Per-step exit buffer: one slot per merge task, in this order (slot counts
// for a BY x XT tile): image 1 rows (BY), image 3 and image 4 edge pixels
// (BY each), image 5 and image 6 exit rows (XT each), image 7 and image 8
// diagonals (XT + BY - 1 each).  The images present for P images are a
// prefix of this list, so P fixes the task count.
template <int BY> struct ExitLayout {
  static constexpr int kDiag = XT + BY - 1;
  static constexpr int E1 = 0, E3 = BY, E4 = 2 * BY, E5 = 3 * BY, E6 = 3 * BY + XT;
  static constexpr int E7 = 3 * BY + 2 * XT, E8 = E7 + kDiag, ET = E8 + kDiag;
  static constexpr int ES = (ET + 3) & ~3;  // buffer stride: keeps 16-byte vector stores aligned
  __host__ __device__ static constexpr int tasks(int P) {
    return P <= 3 ? E3 : P == 4 ? E4 : P == 5 ? E5 : P == 6 ? E6 : P == 7 ? E7 : P == 8 ? E8 : ET;
  }
};

template <typename T, int P, bool TMA>
__global__ void __launch_bounds__(NT, TileCfg<T, P>::MINB)
    k1_project_kernel(K1Params p, const __grid_constant__ CUtensorMap vmap) {
  if (p.gate && (*p.gate & 3) == 0) return;
  using C = TileCfg<T, P>;
  constexpr bool FL = C::FL;
  using A = typename std::conditional<FL, float, uint32_t>::type;    // accumulators
  using IT = typename std::conditional<FL, double, uint32_t>::type;  // image pixels
  constexpr int BYT = C::BYT, BY = C::BY, STAGES = C::STAGES;
  constexpr bool H3 = P > 3, H4 = P > 4, H5 = P > 5, H6 = P > 6, H7 = P > 7, H8 = P > 8;
  constexpr int PW = FL ? 2 : 1;  // words per slot (float slots hold hi, lo)
  using X = ExitLayout<BY>;
  constexpr int NTASK = X::tasks(P);

  // ---- shared memory (every section 128-byte aligned)
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* at = smem;
  auto take = [&](size_t bytes) {
    unsigned char* r = at;
    at += (bytes + 127) & ~size_t(127);
    return r;
  };
  uint64_t* mbar = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * STAGES));
  T* stage = TMA ? reinterpret_cast<T*>(take(sizeof(T) * STAGES * BY * XT)) : nullptr;
  A* slot2 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * XT));  // [2][TY][XT]
  A* mb5 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * XT));    // [2][TY][XT]
  A* mb6 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * XT));
  A* xb = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * X::ES));       // [2][ES]
  int4* roles = reinterpret_cast<int4*>(take(sizeof(int4) * NTASK));
  // float volumes with seven or more images keep image 0's TwoSum pairs in
  // shared memory ([2 * BYT * R2][NT], one column per thread, conflict-free)
  // instead of registers: image 0 never moves between threads, and the 16
  // registers it frees remove most spills (measured 536 -> 515 us at K=6;
  // with fewer images the registers are not short and it measured slower)
  constexpr bool kImg0Smem = FL && P >= 7;
  uint64_t* s0 =
      kImg0Smem ? reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * 2 * BYT * (R / 2) * NT)) : nullptr;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tx = lane & 15, ty = 2 * warp + (lane >> 4);
  const int xl = tx * R, yl = ty * BYT;
  const T* __restrict__ vol = static_cast<const T*>(p.vol);
  const int64_t L = p.L, M = p.M, N = p.N;
  const ImageSet& set = p.set;
  IT* img = static_cast<IT*>(p.images);
  const bool vec_global =
      (L % R) == 0 && ((reinterpret_cast<uintptr_t>(p.vol) % (R * sizeof(T))) == 0);

  // Units are numbered (tile, band, z), z fastest.  With cpt > 0, CTA b
  // takes tile b % nxt and the (b / nxt)-th of cpt equal ranges of that
  // tile's (band, z) units, so the nxt CTAs of consecutive indexes stream
  // the same rows at the same z and together read whole rows of the volume.
  // unit, slice and step counters are 32-bit (the launcher checks that the
  // units fit): 64-bit ones pushed the float kernels into spills
  int ub, ue;
  if (p.cpt > 0) {
    const int64_t tile = blockIdx.x % p.nxt, c = blockIdx.x / p.nxt;
    const int64_t W = p.nbands * p.nz;
    ub = (int)(tile * W + W * c / p.cpt);
    ue = (int)(tile * W + W * (c + 1) / p.cpt);
  } else {
    ub = (int)(p.units * (int64_t)blockIdx.x / gridDim.x);
    ue = (int)(p.units * (int64_t)(blockIdx.x + 1) / gridDim.x);
  }

  for (int i = tid; i < 2 * X::ES * PW; i += NT) xb[i] = (A)0;
  if constexpr (TMA) {
    if (tid == 0) {
      for (int i = 0; i < STAGES; ++i) mbar_init(smem_u32(&mbar[i]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();

  // unit -> (tile x0, band y0, z); units run z fastest, then band, then tile
  const int zbeg = (int)p.z0, zend = (int)(p.z0 + p.nz);
  auto decode = [&](int u, int& x0, int& y0, int& z) {
    const int seg = u / (int)p.nz;
    z = zbeg + u % (int)p.nz;
    y0 = (seg % p.nbands) * BY;
    x0 = (seg / p.nbands) * XT;
  };

  // Producer cursor, kept by thread 0, which issues every copy.
  int pc_x0 = 0, pc_y0 = 0, pc_z = 0;
  if constexpr (TMA) {
    if (tid == 0) decode(ub, pc_x0, pc_y0, pc_z);
  }
  // thread 0: copy the slice at the cursor into stage st, then advance
  auto issue_next = [&](int st) {
    if constexpr (TMA) {
      const uint32_t mb = smem_u32(&mbar[st]);
      mbar_expect_tx(mb, (uint32_t)C::SLICE);
      tma_load_3d(smem_u32(stage + (size_t)st * BY * XT), &vmap, (int)pc_x0, (int)pc_y0,
                  (int)pc_z, mb);
      if (++pc_z == zend) {
        pc_z = zbeg;
        pc_y0 += BY;
        if (pc_y0 >= M) { pc_y0 = 0; pc_x0 += XT; }
      }
    }
  };

  if constexpr (TMA) {
    if (tid == 0)
      for (int i = 0; i < STAGES && ub + i < ue; ++i) issue_next(i);
  }

  // register state.  Integer volumes: one uint32 per window pixel.  Float
  // volumes: (hi, lo) TwoSum pairs packed two pixels per 64-bit register --
  // adjacent columns for images 0, 5, 6 (their windows never shift in x) and
  // adjacent rows for images 3, 4 (never shift in y) -- so every packed
  // update works on registers that stay paired from step to step.
  constexpr int R2 = R / 2, B2 = (BYT + 1) / 2;
  A a0[BYT][R], w3[BYT][R], w4[BYT][R], w5[BYT][R], w6[BYT][R];
  uint64_t P0h[BYT][R2], P0l[BYT][R2], P5h[BYT][R2], P5l[BYT][R2], P6h[BYT][R2], P6l[BYT][R2];
  uint64_t P3h[R][B2], P3l[R][B2], P4h[R][B2], P4l[R][B2];
  auto clear_state = [&]() {
    if constexpr (FL) {
#pragma unroll
      for (int r = 0; r < BYT; ++r)
#pragma unroll
        for (int c = 0; c < R2; ++c) {
          if constexpr (kImg0Smem) {
            s0[(r * R2 + c) * NT + tid] = 0;
            s0[(BYT * R2 + r * R2 + c) * NT + tid] = 0;
          } else {
            P0h[r][c] = P0l[r][c] = 0;
          }
          P5h[r][c] = P5l[r][c] = P6h[r][c] = P6l[r][c] = 0;
        }
#pragma unroll
      for (int q = 0; q < R; ++q)
#pragma unroll
        for (int b = 0; b < B2; ++b) P3h[q][b] = P3l[q][b] = P4h[q][b] = P4l[q][b] = 0;
    } else {
#pragma unroll
      for (int r = 0; r < BYT; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) {
          a0[r][c] = 0; w3[r][c] = 0; w4[r][c] = 0; w5[r][c] = 0; w6[r][c] = 0;
        }
    }
  };
  clear_state();
  // window pixel (value, compensation) by image, in the scalar index space
  auto g0 = [&](int r, int c, float& lo) -> A {
    if constexpr (kImg0Smem) {
      lo = half_of(s0[(BYT * R2 + r * R2 + c / 2) * NT + tid], c & 1);
      return half_of(s0[(r * R2 + c / 2) * NT + tid], c & 1);
    } else if constexpr (FL) {
      lo = half_of(P0l[r][c / 2], c & 1);
      return half_of(P0h[r][c / 2], c & 1);
    } else {
      lo = 0.f;
      return a0[r][c];
    }
  };
  auto g3 = [&](int r, int q, float& lo) -> A {
    if constexpr (FL) { lo = half_of(P3l[q][r / 2], r & 1); return half_of(P3h[q][r / 2], r & 1); }
    else { lo = 0.f; return w3[r][q]; }
  };
  auto g4 = [&](int r, int q, float& lo) -> A {
    if constexpr (FL) { lo = half_of(P4l[q][r / 2], r & 1); return half_of(P4h[q][r / 2], r & 1); }
    else { lo = 0.f; return w4[r][q]; }
  };
  auto g5 = [&](int q, int c, float& lo) -> A {
    if constexpr (FL) { lo = half_of(P5l[q][c / 2], c & 1); return half_of(P5h[q][c / 2], c & 1); }
    else { lo = 0.f; return w5[q][c]; }
  };
  auto g6 = [&](int q, int c, float& lo) -> A {
    if constexpr (FL) { lo = half_of(P6l[q][c / 2], c & 1); return half_of(P6h[q][c / 2], c & 1); }
    else { lo = 0.f; return w6[q][c]; }
  };

  auto emit = [&](IT* dst, A hi, float lo) {
    if constexpr (FL) emit_ff(dst, hi, lo);
    else emit_u(dst, hi);
  };

  // Emit what the registers hold for the current segment (its last step was
  // z_last; the windows are laid out for step zn = z_last + 1).
  auto drain = [&](int64_t x0, int64_t y0, int64_t z_last) {
    const int64_t xs = x0 + xl, yt = y0 + yl;
    const int64_t zn = z_last + 1;
#pragma unroll
    for (int r = 0; r < BYT; ++r) {
      const int64_t y = yt + r;
      if (y >= M) continue;
#pragma unroll
      for (int c = 0; c < R; ++c) {
        if (xs + c >= L) continue;
        float lo;
        const A hv = g0(r, c, lo);
        emit(img + set.base[0] + y * set.F[0] + xs + c, hv, lo);
      }
    }
    if constexpr (H3) {  // logical k = (q - zn) mod R holds pixel x+z = xs + k + zn
#pragma unroll
      for (int r = 0; r < BYT; ++r) {
        const int64_t y = yt + r;
        if (y >= M) continue;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int k = (int)(((q - zn) % R + R) % R);
          const int64_t f = xs + k + zn;
          float lo;
          const A hv = g3(r, q, lo);
          if (f < set.F[3]) emit(img + set.base[3] + y * set.F[3] + f, hv, lo);
        }
      }
    }
    if constexpr (H4) {  // logical k = (q + zn) mod R holds x-z+N-1 = xs + k - zn + N-1
#pragma unroll
      for (int r = 0; r < BYT; ++r) {
        const int64_t y = yt + r;
        if (y >= M) continue;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int k = (int)(((q + zn) % R + R) % R);
          const int64_t f = xs + k - zn + (N - 1);
          float lo;
          const A hv = g4(r, q, lo);
          if (f >= 0 && f < set.F[4]) emit(img + set.base[4] + y * set.F[4] + f, hv, lo);
        }
      }
    }
    if constexpr (H5) {  // logical k = (q - zn) mod BYT holds row y+z = yt + k + zn
#pragma unroll
      for (int q = 0; q < BYT; ++q) {
        const int k = (int)(((q - zn) % BYT + BYT) % BYT);
        const int64_t srow = yt + k + zn;
        if (srow >= set.S[5]) continue;
#pragma unroll
        for (int c = 0; c < R; ++c)
          if (xs + c < L) {
            float lo;
            const A hv = g5(q, c, lo);
            emit(img + set.base[5] + srow * set.F[5] + xs + c, hv, lo);
          }
      }
    }
    if constexpr (H6) {  // logical k = (q + zn) mod BYT holds row y-z+N-1 = yt + k - zn + N-1
#pragma unroll
      for (int q = 0; q < BYT; ++q) {
        const int k = (int)(((q + zn) % BYT + BYT) % BYT);
        const int64_t srow = yt + k - zn + (N - 1);
        if (srow < 0 || srow >= set.S[6]) continue;
#pragma unroll
        for (int c = 0; c < R; ++c)
          if (xs + c < L) {
            float lo;
            const A hv = g6(q, c, lo);
            emit(img + set.base[6] + srow * set.F[6] + xs + c, hv, lo);
          }
      }
    }
    clear_state();
  };

  // Destination of every merge task for the segment at (x0, y0): pixel index
  // base + z * zs, taken for z >= zmin (zmin = INT_MAX: no pixel).
  auto set_roles = [&](int64_t x0, int64_t y0) {
    constexpr int kNever = 0x7fffffff;
    for (int t = tid; t < NTASK; t += NT) {
      int64_t base = 0;
      int64_t zs = 0;
      int64_t zmin = kNever;
      if (t < X::E3) {  // image 1: pixel (z, y)
        const int64_t y = y0 + t;
        if (y < M) { base = set.base[1] + y; zs = set.F[1]; zmin = 0; }
      } else if (t < X::E5) {  // images 3/4: the pixel leaving the tile edge of row y
        const bool i3 = t < X::E4;
        const int64_t y = y0 + (i3 ? t - X::E3 : t - X::E4);
        if (y < M) {
          if (i3) {  // leaves at x = x0: f = x0 + z
            base = set.base[3] + y * set.F[3] + x0; zs = 1; zmin = 0;
          } else {  // leaves at x = x0 + XT - 1: f = x0 + XT - 1 - z + N - 1 < F4 iff z >= x0 + XT - L
            base = set.base[4] + y * set.F[4] + x0 + XT + N - 2; zs = -1;
            zmin = x0 + XT - L > 0 ? x0 + XT - L : 0;
          }
        }
      } else if (t < X::E7) {  // images 5/6: the row leaving the band edge, column x
        const bool i5 = t < X::E6;
        const int64_t x = x0 + (i5 ? t - X::E5 : t - X::E6);
        if (x < L) {
          if (i5) {  // row y0 + z
            base = set.base[5] + y0 * set.F[5] + x; zs = set.F[5]; zmin = 0;
          } else {  // row y0 + BY - 1 - z + N - 1 < S6 iff z >= y0 + BY - M
            base = set.base[6] + (y0 + BY + N - 2) * set.F[6] + x; zs = -set.F[6];
            zmin = y0 + BY - M > 0 ? y0 + BY - M : 0;
          }
        }
      } else {  // images 7/8: diagonal idx of the tile
        const bool i7 = t < X::E8;
        const int64_t idx = i7 ? t - X::E7 : t - X::E8;
        const int k = i7 ? 7 : 8;
        const int64_t f = i7 ? x0 + y0 + idx : x0 - y0 - (BY - 1) + idx + (M - 1);
        if (f >= 0 && f < set.F[k]) { base = set.base[k] + f; zs = set.F[k]; zmin = 0; }
      }
      roles[t] = make_int4((int)(uint32_t)(uint64_t)base, (int)((uint64_t)base >> 32), (int)zs,
                           (int)zmin);
    }
  };

  // deferred merges pay off with two CTAs per SM (float volumes with six or
  // more images); with one CTA of 4 x 4 micro-tiles they measured slower
  constexpr bool kDeferMerge = FL && BYT == 2;
  bool pend = false;  // a step whose merge is still to do (float volumes)
  int pend_sb = 0;
  int64_t pend_z = 0;
  bool aborted = false;
  int s = 0;   // CTA step counter
  int u = ub;  // next unit
  while (u < ue && !aborted) {
    // one segment: a (tile, band) streamed over z in [za, zb)
    int x0, y0, za;
    decode(u, x0, y0, za);
    const int zb = (zend - za) < (ue - u) ? zend : za + (ue - u);
    const int64_t xs = x0 + xl, yt = y0 + yl;
    // which of the thread's rows and columns hold voxels
    const int ncol = (int)((L - xs) <= 0 ? 0 : ((L - xs) < R ? (L - xs) : R));
    const int nrow = (int)((M - yt) <= 0 ? 0 : ((M - yt) < BYT ? (M - yt) : BYT));
    const bool full = (ncol == R) && (nrow == BYT);
    // image 2 merge: column col2 of the tile, quarter part2 of the row groups
    const int col2 = tid >> 2, part2 = tid & 3;
    const bool ok2 = part2 == 0 && x0 + col2 < L;
    IT* const img2 = img + set.base[2] + x0 + col2;
    const int64_t F2 = set.F[2];
    set_roles(x0, y0);
    __syncthreads();
    // merge of the step results in buffer msb (image 2 slots, exit buffer)
    // for slice mz of this segment
    auto merge_step = [&](int msb, int64_t mz) {
      // (a) image 2, one quarter of a column's TY partials per thread
      {
        // row group r's partials sit at column c ^ (8 * (r / 4)) (see the
        // writes): the 4 threads of a column then read distinct banks
        const A* e0 = slot2 + ((size_t)(msb * TY + part2 * (TY / 4)) * XT + (col2 ^ (part2 << 3))) * PW;
        A h = e0[0];
        float l = 0.f;
        if constexpr (FL) l = e0[1];
#pragma unroll
        for (int g = 1; g < TY / 4; ++g) {
          const A* e = e0 + (size_t)g * XT * PW;
          if constexpr (FL) pair_acc(h, l, e[0], e[1]);
          else h += e[0];
        }
#pragma unroll
        for (int m = 1; m <= 2; m <<= 1) {
          if constexpr (FL) {
            const float oh = __shfl_xor_sync(0xffffffffu, h, m), ol = __shfl_xor_sync(0xffffffffu, l, m);
            pair_acc(h, l, oh, ol);
          } else {
            h += __shfl_xor_sync(0xffffffffu, h, m);
          }
        }
        if (ok2) emit(img2 + mz * F2, h, l);
      }
      // (b) the exit buffer, one slot per task
#pragma unroll
      for (int i = 0; i < (NTASK + NT - 1) / NT; ++i) {
        const int t = tid + i * NT;
        if (t < NTASK) {
          const int4 rd = roles[t];
          A* c = xb + (size_t)msb * X::ES * PW + (size_t)t * PW;
          const A hv = c[0];
          float lv = 0.f;
          if constexpr (FL) lv = c[1];
          if (t >= X::E7) {  // diagonal cells accumulate: clear for the step after next
            c[0] = (A)0;
            if constexpr (FL) c[1] = 0.f;
          }
          if (mz >= rd.w) {
            const int64_t base = (int64_t)(((uint64_t)(uint32_t)rd.y << 32) | (uint32_t)rd.x);
            emit(img + (base + mz * (int64_t)rd.z), hv, lv);
          }
        }
      }
    };
    int z = za;
    while (z < zb && !aborted) {
#pragma unroll
    for (int j = 0; j < R; ++j) {  // unrolled so window slots are static: j == z % R
      if (z >= zb || aborted) break;
      if ((int)(z & (R - 1)) != j) continue;  // align the unroll phase with z
      const int st = (int)(s & (STAGES - 1));
      const int par = (int)((s / STAGES) & 1);
      const int sb = (int)(s & 1);  // shared double-buffer index
      A* const xc = xb + (size_t)sb * X::ES * PW;

      // ---- 1. the micro-tile of slice z
      bool ok = true;
      if constexpr (TMA) ok = mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)par);
      A v[BYT][R];
#pragma unroll
      for (int r = 0; r < BYT; ++r) {
        if constexpr (TMA) {
          load4_smem(stage + ((size_t)st * BY + yl + r) * XT + xl, v[r]);
        } else {
          if (r < nrow && ncol > 0) load4_global(vol + (z * M + yt + r) * L, xs, L, vec_global, v[r]);
        }
        if (!full) {
#pragma unroll
          for (int c = 0; c < R; ++c)
            if (r >= nrow || c >= ncol) v[r][c] = (A)0;
        }
      }
      if (!ok) {
#pragma unroll
        for (int r = 0; r < BYT; ++r)
#pragma unroll
          for (int c = 0; c < R; ++c) v[r][c] = (A)0;
      }

      // ---- 2. images crossing the slice
      // float voxels as pairs: vc = adjacent columns of one row (how the
      // 16-byte loads land), vr = adjacent rows of one column
      uint64_t vc[BYT][R2], vr[R][B2];
      if constexpr (FL) {
#pragma unroll
        for (int r = 0; r < BYT; ++r)
#pragma unroll
          for (int cp = 0; cp < R2; ++cp) vc[r][cp] = pk(v[r][2 * cp], v[r][2 * cp + 1]);
#pragma unroll
        for (int c = 0; c < R; ++c)
#pragma unroll
          for (int rp = 0; rp < B2; ++rp) vr[c][rp] = pk(v[2 * rp][c], v[2 * rp + 1][c]);
#pragma unroll
        for (int r = 0; r < BYT; ++r)
#pragma unroll
          for (int cp = 0; cp < R2; ++cp) {
            if constexpr (kImg0Smem) {
              uint64_t* h0 = s0 + (r * R2 + cp) * NT + tid;
              uint64_t* l0 = s0 + (BYT * R2 + r * R2 + cp) * NT + tid;
              uint64_t hv = *h0, lv = *l0;
              ts2(hv, lv, vc[r][cp]);
              *h0 = hv;
              *l0 = lv;
            } else {
              ts2(P0h[r][cp], P0l[r][cp], vc[r][cp]);
            }
            if constexpr (H5) ts2(P5h[(r + j) % BYT][cp], P5l[(r + j) % BYT][cp], vc[r][cp]);
            if constexpr (H6)
              ts2(P6h[(r - j + R) % BYT][cp], P6l[(r - j + R) % BYT][cp], vc[r][cp]);
          }
#pragma unroll
        for (int c = 0; c < R; ++c)
#pragma unroll
          for (int rp = 0; rp < B2; ++rp) {
            if constexpr (H3) ts2(P3h[(c + j) % R][rp], P3l[(c + j) % R][rp], vr[c][rp]);
            if constexpr (H4) ts2(P4h[(c - j + R) % R][rp], P4l[(c - j + R) % R][rp], vr[c][rp]);
          }
      } else {
#pragma unroll
        for (int r = 0; r < BYT; ++r)
#pragma unroll
          for (int c = 0; c < R; ++c) {
            a0[r][c] += v[r][c];
            if constexpr (H3) w3[r][(c + j) % R] += v[r][c];
            if constexpr (H4) w4[r][(c - j + R) % R] += v[r][c];
            if constexpr (H5) w5[(r + j) % BYT][c] += v[r][c];
            if constexpr (H6) w6[(r - j + R) % BYT][c] += v[r][c];
          }
      }

      if constexpr (kDeferMerge) {  // the previous step's merge
        if (pend) {
          merge_step(pend_sb, pend_z);
          pend = false;
        }
      }
      // ---- 3. images in the slice: column sums (2), row sums (1), diagonals (7, 8)
      {
        // column partials of row group ty at column x ^ (8 * (ty / 4)): the
        // aligned 4-column groups stay contiguous (16-byte stores), and the
        // merge's reads of row groups 4p .. 4p+3 spread over the banks
        A* s2 = slot2 + ((size_t)(sb * TY + ty) * XT + (xl ^ ((ty >> 2) << 3))) * PW;
        A rs[BYT];
        float rsc[BYT];
        if constexpr (FL) {
          uint64_t csh[R2], csl[R2];  // column sums, pairs of adjacent columns
#pragma unroll
          for (int cp = 0; cp < R2; ++cp) {
            csh[cp] = vc[0][cp];
            csl[cp] = 0;
          }
#pragma unroll
          for (int r = 1; r < BYT; ++r)
#pragma unroll
            for (int cp = 0; cp < R2; ++cp) ts2(csh[cp], csl[cp], vc[r][cp]);
          *reinterpret_cast<float4*>(s2) = make_float4(half_of(csh[0], 0), half_of(csl[0], 0),
                                                       half_of(csh[0], 1), half_of(csl[0], 1));
          *reinterpret_cast<float4*>(s2 + 4) = make_float4(half_of(csh[1], 0), half_of(csl[1], 0),
                                                           half_of(csh[1], 1), half_of(csl[1], 1));
          uint64_t rsh[B2], rsl[B2];  // row sums, pairs of adjacent rows
#pragma unroll
          for (int rp = 0; rp < B2; ++rp) {
            rsh[rp] = vr[0][rp];
            rsl[rp] = 0;
          }
#pragma unroll
          for (int c = 1; c < R; ++c)
#pragma unroll
            for (int rp = 0; rp < B2; ++rp) ts2(rsh[rp], rsl[rp], vr[c][rp]);
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            rs[r] = half_of(rsh[r / 2], r & 1);
            rsc[r] = half_of(rsl[r / 2], r & 1);
          }
        } else {
          A cs[R];
#pragma unroll
          for (int c = 0; c < R; ++c) cs[c] = v[0][c];
#pragma unroll
          for (int r = 1; r < BYT; ++r)
#pragma unroll
            for (int c = 0; c < R; ++c) cs[c] += v[r][c];
          *reinterpret_cast<uint4*>(s2) = make_uint4(cs[0], cs[1], cs[2], cs[3]);
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            rs[r] = v[r][0];
            rsc[r] = 0.f;
          }
#pragma unroll
          for (int c = 1; c < R; ++c)
#pragma unroll
            for (int r = 0; r < BYT; ++r) rs[r] += v[r][c];
        }
        constexpr int per = 16 / BYT;
        if constexpr (FL) {
          float oh, ol;
          ff_rows_half<BYT>(rs, rsc, tx, oh, ol);
          if ((tx & (per - 1)) == 0) {
            A* d = xc + (size_t)(X::E1 + yl + tx / per) * PW;
            d[0] = oh;
            d[1] = ol;
          }
        } else {
          const uint32_t t = u_rows_half<BYT>(rs, tx);
          if ((tx & (per - 1)) == 0) xc[X::E1 + yl + tx / per] = t;
        }
      }
      if constexpr (H7 || H8) {
#pragma unroll
        for (int im = 0; im < 2; ++im) {
          if ((im == 0 && !H7) || (im == 1 && !H8)) continue;
#pragma unroll
          for (int k = 0; k < R + BYT - 1; ++k) {
            A d = 0;
            float dc = 0.f;
            bool first = true;
#pragma unroll
            for (int r = 0; r < BYT; ++r) {
              const int c = im == 0 ? k - r : k - (BYT - 1) + r;
              if (c < 0 || c >= R) continue;
              if (first) {
                d = v[r][c];
                first = false;
              } else if constexpr (FL) {
                ts_acc(d, dc, v[r][c]);
              } else {
                d += v[r][c];
              }
            }
            // local index x_l + y_l (image 7) or x_l - y_l + BY - 1 (image 8)
            const int idx = im == 0 ? xl + yl + k : xl - yl + (BY - BYT) + k;
            A* cell = xc + (size_t)((im == 0 ? X::E7 : X::E8) + idx) * PW;
            if constexpr (FL) {
              if (d != 0.f || dc != 0.f) {
                const float old = atomicAdd(cell, d);
                float sum, e;
                two_sum(old, d, sum, e);
                atomicAdd(cell + 1, __fadd_rn(e, dc));
              }
            } else {
              if (d) atomicAdd(cell, d);
            }
          }
        }
      }

      // ---- 4. hand the leaving window pixels on
      if constexpr (H3) {  // logical 0 (slot j) moves to the left neighbour
        if constexpr (FL) {
#pragma unroll
          for (int rp = 0; rp < B2; ++rp) {
            const uint64_t sh = P3h[j][rp], sl = P3l[j][rp];
            const uint64_t rh = __shfl_down_sync(0xffffffffu, (unsigned long long)sh, 1, 16);
            const uint64_t rl = __shfl_down_sync(0xffffffffu, (unsigned long long)sl, 1, 16);
            P3h[j][rp] = (tx == TX - 1) ? 0 : rh;
            P3l[j][rp] = (tx == TX - 1) ? 0 : rl;
            if (tx == 0) {  // leaves the tile: complete for this CTA
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                A* d = xc + (size_t)(X::E3 + yl + 2 * rp + h) * PW;
                d[0] = half_of(sh, h);
                d[1] = half_of(sl, h);
              }
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            const A sv = w3[r][j];
            const A rv = __shfl_down_sync(0xffffffffu, sv, 1, 16);
            w3[r][j] = (tx == TX - 1) ? (A)0 : rv;
            if (tx == 0) xc[X::E3 + yl + r] = sv;  // leaves the tile: complete for this CTA
          }
        }
      }
      if constexpr (H4) {  // logical R-1 moves to the right neighbour
        const int q = (R - 1 - j + R) % R;
        if constexpr (FL) {
#pragma unroll
          for (int rp = 0; rp < B2; ++rp) {
            const uint64_t sh = P4h[q][rp], sl = P4l[q][rp];
            const uint64_t rh = __shfl_up_sync(0xffffffffu, (unsigned long long)sh, 1, 16);
            const uint64_t rl = __shfl_up_sync(0xffffffffu, (unsigned long long)sl, 1, 16);
            P4h[q][rp] = (tx == 0) ? 0 : rh;
            P4l[q][rp] = (tx == 0) ? 0 : rl;
            if (tx == TX - 1) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                A* d = xc + (size_t)(X::E4 + yl + 2 * rp + h) * PW;
                d[0] = half_of(sh, h);
                d[1] = half_of(sl, h);
              }
            }
          }
        } else {
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            const A sv = w4[r][q];
            const A rv = __shfl_up_sync(0xffffffffu, sv, 1, 16);
            w4[r][q] = (tx == 0) ? (A)0 : rv;
            if (tx == TX - 1) xc[X::E4 + yl + r] = sv;
          }
        }
      }
      // images 5/6: the leaving window row goes to the group above (5) or
      // below (6); the band's edge group puts it in the exit buffer
      if constexpr (H5) {
        const int q = j % BYT;
        A* d = ty > 0 ? mb5 + ((size_t)(sb * TY + ty - 1) * XT + xl) * PW
                      : xc + (size_t)(X::E5 + xl) * PW;
        if constexpr (FL) {
          *reinterpret_cast<float4*>(d) = make_float4(half_of(P5h[q][0], 0), half_of(P5l[q][0], 0),
                                                      half_of(P5h[q][0], 1), half_of(P5l[q][0], 1));
          *reinterpret_cast<float4*>(d + 4) =
              make_float4(half_of(P5h[q][1], 0), half_of(P5l[q][1], 0), half_of(P5h[q][1], 1),
                          half_of(P5l[q][1], 1));
#pragma unroll
          for (int cp = 0; cp < R2; ++cp) P5h[q][cp] = P5l[q][cp] = 0;
        } else {
          *reinterpret_cast<uint4*>(d) = make_uint4(w5[q][0], w5[q][1], w5[q][2], w5[q][3]);
#pragma unroll
          for (int c = 0; c < R; ++c) w5[q][c] = 0;
        }
      }
      if constexpr (H6) {
        const int q = (BYT - 1 - j + R) % BYT;
        A* d = ty < TY - 1 ? mb6 + ((size_t)(sb * TY + ty + 1) * XT + xl) * PW
                           : xc + (size_t)(X::E6 + xl) * PW;
        if constexpr (FL) {
          *reinterpret_cast<float4*>(d) = make_float4(half_of(P6h[q][0], 0), half_of(P6l[q][0], 0),
                                                      half_of(P6h[q][0], 1), half_of(P6l[q][0], 1));
          *reinterpret_cast<float4*>(d + 4) =
              make_float4(half_of(P6h[q][1], 0), half_of(P6l[q][1], 0), half_of(P6h[q][1], 1),
                          half_of(P6l[q][1], 1));
#pragma unroll
          for (int cp = 0; cp < R2; ++cp) P6h[q][cp] = P6l[q][cp] = 0;
        } else {
          *reinterpret_cast<uint4*>(d) = make_uint4(w6[q][0], w6[q][1], w6[q][2], w6[q][3]);
#pragma unroll
          for (int c = 0; c < R; ++c) w6[q][c] = 0;
        }
      }

      // ---- 5. step barrier, also agreeing on an abort
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if constexpr (TMA) {  // the slice is consumed: refill its stage
        if (tid == 0 && u + STAGES < ue) issue_next(st);
      }

      // ---- 6. receive the window rows handed over by the neighbouring groups
      if constexpr (H5) {
        if (ty < TY - 1) {
          const int q = j % BYT;
          const A* d = mb5 + ((size_t)(sb * TY + ty) * XT + xl) * PW;
          if constexpr (FL) {
            const float4 e0 = *reinterpret_cast<const float4*>(d);
            const float4 e1 = *reinterpret_cast<const float4*>(d + 4);
            P5h[q][0] = pk(e0.x, e0.z);
            P5l[q][0] = pk(e0.y, e0.w);
            P5h[q][1] = pk(e1.x, e1.z);
            P5l[q][1] = pk(e1.y, e1.w);
          } else {
            const uint4 e0 = *reinterpret_cast<const uint4*>(d);
            w5[q][0] = e0.x; w5[q][1] = e0.y; w5[q][2] = e0.z; w5[q][3] = e0.w;
          }
        }
      }
      if constexpr (H6) {
        if (ty > 0) {
          const int q = (BYT - 1 - j + R) % BYT;
          const A* d = mb6 + ((size_t)(sb * TY + ty) * XT + xl) * PW;
          if constexpr (FL) {
            const float4 e0 = *reinterpret_cast<const float4*>(d);
            const float4 e1 = *reinterpret_cast<const float4*>(d + 4);
            P6h[q][0] = pk(e0.x, e0.z);
            P6l[q][0] = pk(e0.y, e0.w);
            P6h[q][1] = pk(e1.x, e1.z);
            P6l[q][1] = pk(e1.y, e1.w);
          } else {
            const uint4 e0 = *reinterpret_cast<const uint4*>(d);
            w6[q][0] = e0.x; w6[q][1] = e0.y; w6[q][2] = e0.z; w6[q][3] = e0.w;
          }
        }
      }

      // ---- 7. merge this step's complete results into the images: now, or
      // for float volumes with six or more images during the next step (its
      // buffers are not rewritten before the next step's barrier), where the
      // merge's load and shuffle latencies overlap that step's sums
      // (measured 6%)
      if constexpr (kDeferMerge) {
        pend = true;
        pend_sb = sb;
        pend_z = z;
      } else {
        merge_step(sb, z);
      }
      ++s;
      ++u;
      ++z;
    }
    }
    if constexpr (kDeferMerge) {  // the segment's last step
      if (pend && !aborted) merge_step(pend_sb, pend_z);
      pend = false;
    }
    if (!aborted) {
      drain(x0, y0, zb - 1);
      __syncthreads();  // roles are rewritten for the next segment
    }
  }

  if (aborted) {
    // let bulk copies still in flight land before the CTA's shared memory is
    // released (bounded; they were issued for units u .. u+STAGES-1)
    if constexpr (TMA) {
      if (tid == 0) {
        for (int i = 0; i < STAGES && u + i < ue; ++i) {
          const int64_t ss = s + i;
          mbar_wait_bounded(smem_u32(&mbar[ss & (STAGES - 1)]), (uint32_t)((ss / STAGES) & 1));
        }
      }
    }
    if (tid == 0 && p.status) atomicMax(p.status, kStatusTimeout);
  }
}

// Tensor map of the volume as a 3-D tensor (x fastest), box XT x BY x 1.
// cuTensorMapEncodeTiled is reached through the runtime's driver entry point
// (the library links no driver stub).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();  // defined in k1_dispatch.cu

template <typename T>
cudaError_t encode_volume_map(CUtensorMap* map, const void* vol, int64_t L, int64_t M, int64_t N,
                              int box_x, int box_y) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return cudaErrorNotSupported;
  const CUtensorMapDataType dt = std::is_same<T, float>::value
                                     ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                     : (sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT8);
  const cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)M, (cuuint64_t)N};
  const cuuint64_t strides[2] = {(cuuint64_t)(L * (int64_t)sizeof(T)),
                                 (cuuint64_t)(L * M * (int64_t)sizeof(T))};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = fn(map, dt, 3, const_cast<void*>(vol), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int P, bool TMA>
cudaError_t launch_t(const ProjectArgs& a, cudaStream_t st) {
  using C = TileCfg<T, P>;
  constexpr bool FL = C::FL;
  using Acc = typename std::conditional<FL, float, uint32_t>::type;
  constexpr int PW = FL ? 2 : 1;
  constexpr int BY = C::BY, STAGES = C::STAGES;
  K1Params p{};
  p.vol = a.vol;
  p.L = a.L; p.M = a.M; p.N = a.N;
  p.z0 = a.nz > 0 ? a.z0 : 0;
  p.nz = a.nz > 0 ? a.nz : a.N;
  p.nbands = (a.M + BY - 1) / BY;
  p.nxt = (a.L + XT - 1) / XT;
  p.units = p.nxt * p.nbands * p.nz;
  if (p.units >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;  // 32-bit unit counters
  p.set = a.set;
  p.images = a.images;
  p.status = a.status;
  p.gate = a.gate;

  auto rnd = [](size_t b) { return (b + 127) & ~size_t(127); };
  using X = ExitLayout<BY>;
  size_t smem = rnd(sizeof(uint64_t) * STAGES);
  if (TMA) smem += rnd(sizeof(T) * STAGES * BY * XT);
  smem += 3 * rnd(sizeof(Acc) * PW * 2 * TY * XT);  // slot2, mb5, mb6
  smem += rnd(sizeof(Acc) * PW * 2 * X::ES);        // exit buffer
  smem += rnd(sizeof(int4) * X::tasks(P));          // merge roles
  if (FL && P >= 7) smem += rnd(sizeof(uint64_t) * 2 * C::BYT * (R / 2) * NT);  // image 0

  auto kern = k1_project_kernel<T, P, TMA>;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int cached_sms[64] = {0}, cached_per_sm[64] = {0};  // per instantiation
  int sms = dev < 64 ? cached_sms[dev] : 0, per_sm = dev < 64 ? cached_per_sm[dev] : 0;
  if (sms == 0) {
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) { cached_sms[dev] = sms; cached_per_sm[dev] = per_sm; }
  }
  // at least ~8 z-steps per CTA so segment drains stay a small overhead
  const int64_t gmax = (int64_t)sms * per_sm;
  int64_t grid;
  if (p.nxt <= gmax) {  // tile-major ranges, nxt CTAs per (band, z) range
    const int64_t W = p.nbands * p.nz;
    int64_t cpt = gmax / p.nxt;
    if (cpt > (W + 7) / 8) cpt = (W + 7) / 8;
    if (cpt < 1) cpt = 1;
    p.cpt = cpt;
    grid = p.nxt * cpt;
  } else {
    p.cpt = 0;
    grid = gmax;
    const int64_t by_work = (p.units + 7) / 8;
    if (grid > by_work) grid = by_work;
    if (grid < 1) grid = 1;
  }
  CUtensorMap vmap;
  std::memset(&vmap, 0, sizeof(vmap));
  if (TMA) {
    cudaError_t me = encode_volume_map<T>(&vmap, a.vol, a.L, a.M, a.N, XT, BY);
    if (me != cudaSuccess) return me;
  }
  kern<<<(unsigned)grid, NT, smem, st>>>(p, vmap);
  return cudaGetLastError();
}

// Launch for one element type and image count; takes the bulk-copy path
// when rows are 16-byte aligned.
template <typename T, int P>
cudaError_t launch_p(const ProjectArgs& a, cudaStream_t st) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.vol);
  const bool tma = ((a.L * (int64_t)sizeof(T)) % 16 == 0) && (base % 16 == 0);
  return tma ? launch_t<T, P, true>(a, st) : launch_t<T, P, false>(a, st);
}

}  // namespace k1
}  // namespace dpma
