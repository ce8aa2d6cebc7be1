// Step 1 of the Discrete Projection Moment method: one fused pass over the
// volume that writes every projection image at once (Sec. 3.1, Eq. 4 with
// the image set of Eqs. 5-9 and the +-pi/4 families).
//
// Work decomposition.  A CTA owns a tile of XT columns (x) by BY = 16 rows
// (y) and streams it along z.  Its threads form TX columns of R = 4 x-values
// by TY row groups of BYT rows (4 x 4 or 4 x 2 micro-tiles, see TileCfg).  Persistent CTAs take contiguous ranges of
// (tile, z) units.  When rows are 16-byte aligned the slices arrive through
// a 4-stage ring of 1-D bulk copies (cp.async.bulk + mbarrier); otherwise
// every thread loads its micro-tile from global memory.
//
// Images whose lines leave the z-slice (directions z, (1,0,+-1), (0,1,+-1):
// images 0 and 3-6) accumulate in registers across z:
//   image 0    one accumulator per (x, y);
//   images 3/4 (x+-z, y): a window of R registers per row; after each step
//              the pixel that leaves a thread's window is handed to the
//              neighbouring thread (warp shuffle; a shared mailbox between
//              warps), and the tile's edge thread emits it, complete;
//   images 5/6 (y+-z, x): a window of BYT registers per column, handed
//              between row groups through shared mailboxes.
// Images whose lines lie in the slice (images 1, 2, 7, 8) are reduced per
// step: image 2 (sum along y) and image 1 (sum along x) through per-step
// shared slots merged by owner threads, images 7/8 (x+-y) through per-step
// shared buffers.
//
// Float volumes keep every sum compensated: each accumulator is a pair
// (hi, lo) updated with the error-free TwoSum, so a pixel carries float-float
// accuracy whatever the order and signs of its terms.  Partial sums that
// leave a CTA are turned, with integer operations only, into the double that
// equals hi + lo exactly and merged with red.global.add.f64 by the L2 (the
// SMs execute no FP64 instruction).  Integer volumes use exact uint32 sums
// and red.global.add.u32.
#pragma once
#include <cstdint>
#include <type_traits>

#include "dpma_internal.cuh"

namespace dpma {
namespace k1 {

constexpr int R = 4;      // x-values per thread
constexpr int BY = 16;    // rows per tile
constexpr int STAGES = 4;

// Bounded waits give up after ~2^31 cycles (about a second).
constexpr long long kWaitBudget = 1ll << 31;
constexpr int kStatusTimeout = 5;

// Tile shape per element type and image count.  With few images a thread
// holds a 4 x 4 micro-tile; with more windowed images (Kahan pairs for
// floats) the register state needs a 4 x 2 micro-tile.
template <typename T, int P> struct TileCfg {
  static constexpr bool FL = std::is_same<T, float>::value;
  static constexpr bool SMALL = FL && P >= 6;            // 4 x 2 micro-tile
  static constexpr int BYT = SMALL ? 2 : 4;              // rows per thread
  static constexpr int TY = BY / BYT;                    // row groups
  static constexpr int TX = FL ? (SMALL ? 32 : 64) : 64;
  static constexpr int XT = R * TX;
  static constexpr int NT = TX * TY;
  static constexpr int NW = TX / 32;  // warps per row group
  // groups that emit the per-step results
  static constexpr int G_I5 = 0, G_I2 = 1, G_I1 = 2, G_DIAG = 3;
  static constexpr int G_EDGE = TY > 4 ? 4 : 2;
  static constexpr int G_I6 = TY - 1;
  static constexpr int EDGE0 = G_EDGE == G_I1 ? BY : 0;  // first edge thread
  static_assert(EDGE0 + 2 * BY <= TX, "edge emitters must fit in one row group");
  static_assert(R % BYT == 0, "window rotations share the unroll period R");
};

struct K1Params {
  const void* vol;
  int64_t L, M, N;
  int64_t nbands, nxt;
  int64_t units;  // nxt * nbands * N
  ImageSet set;
  void* images;
  int* status;
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
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
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

// Two independent TwoSum accumulations in one set of packed f32x2
// instructions (sm_100 and later): (h0, l0) += v0 and (h1, l1) += v1.
__device__ __forceinline__ void ts_acc2(float& h0, float& l0, float v0, float& h1, float& l1,
                                        float v1) {
  unsigned long long H, Lo, V, t, bb, x, y, e;
  asm("mov.b64 %0, {%1,%2};" : "=l"(H) : "f"(h0), "f"(h1));
  asm("mov.b64 %0, {%1,%2};" : "=l"(Lo) : "f"(l0), "f"(l1));
  asm("mov.b64 %0, {%1,%2};" : "=l"(V) : "f"(v0), "f"(v1));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(H), "l"(V));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(bb) : "l"(t), "l"(H));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(x) : "l"(t), "l"(bb));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(x) : "l"(H), "l"(x));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(y) : "l"(V), "l"(bb));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(e) : "l"(x), "l"(y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(Lo) : "l"(Lo), "l"(e));
  asm("mov.b64 {%0,%1}, %2;" : "=f"(h0), "=f"(h1) : "l"(t));
  asm("mov.b64 {%0,%1}, %2;" : "=f"(l0), "=f"(l1) : "l"(Lo));
}

// The double equal to hi + lo (both float32), built with integer operations.
// hi + lo needs at most 48 significant bits when |lo| <= ulp(hi), so the
// result is exact then; a wider gap rounds lo at 2^-52 relative to hi.
__device__ __forceinline__ double ff_to_f64(float hi, float lo) {
  const uint32_t bh = __float_as_uint(hi), bl = __float_as_uint(lo);
  const int eh = (int)((bh >> 23) & 0xff), el = (int)((bl >> 23) & 0xff);
  // signed integer mantissas and exponents: value = m * 2^e
  long long mh = (long long)((bh & 0x7fffffu) | (eh ? 0x800000u : 0u));
  long long ml = (long long)((bl & 0x7fffffu) | (el ? 0x800000u : 0u));
  if (bh >> 31) mh = -mh;
  if (bl >> 31) ml = -ml;
  const int xh = (eh ? eh : 1) - 150, xl = (el ? el : 1) - 150;
  if (ml == 0 && mh == 0) return 0.0;
  // align both on the smaller exponent, keeping at most 62 bits
  long long S;
  int E;
  if (mh == 0) { S = ml; E = xl; }
  else if (ml == 0) { S = mh; E = xh; }
  else {
    const int lo_e = xh < xl ? xh : xl, hi_e = xh < xl ? xl : xh;
    const long long mbig = xh < xl ? ml : mh, msmall = xh < xl ? mh : ml;
    int d = hi_e - lo_e;
    if (d <= 37) { S = (mbig << d) + msmall; E = lo_e; }
    else { S = (mbig << 37) + (msmall >> (d - 37)); E = hi_e - 37; }
  }
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
  unsigned long long U = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int lz = __clzll(U);
  const int msb = 63 - lz;                 // value = U * 2^E, U in [2^msb, 2^(msb+1))
  if (msb > 52) {                          // round to 53 bits, nearest-even
    const int sh = msb - 52;
    const unsigned long long rem = U & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    U >>= sh;
    E += sh;
    if (rem > half || (rem == half && (U & 1))) ++U;
    if (U >> 53) { U >>= 1; ++E; }
  } else {
    U <<= (52 - msb);
    E -= (52 - msb);
  }
  const long long bexp = (long long)E + 52 + 1023;  // U in [2^52, 2^53)
  if (bexp <= 0) return 0.0;                         // below the double range
  const unsigned long long bits = sign | ((unsigned long long)bexp << 52) | (U & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// Merge the pair (hi, lo) into a global float pixel (a double), fire and forget.
__device__ __forceinline__ void red_ff(double* p, float hi, float lo) {
  if (hi == 0.f && lo == 0.f) return;
  atomicAdd(p, ff_to_f64(hi, lo));
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

// Float-float warp reduction of BYT = 4 per-lane pairs into one pair per
// 8-lane group: lanes 0-7 end with row 0, 8-15 row 1, 16-23 row 2, 24-31 row 3.
__device__ __forceinline__ void ff_reduce4_scatter(const float h[4], const float l[4], int lane,
                                                   float& oh, float& ol) {
  const bool up = lane & 16;
  float k0h = up ? h[2] : h[0], k0l = up ? l[2] : l[0];
  float k1h = up ? h[3] : h[1], k1l = up ? l[3] : l[1];
  const float s0h = up ? h[0] : h[2], s0l = up ? l[0] : l[2];
  const float s1h = up ? h[1] : h[3], s1l = up ? l[1] : l[3];
  const float r0h = __shfl_xor_sync(0xffffffffu, s0h, 16), r0l = __shfl_xor_sync(0xffffffffu, s0l, 16);
  const float r1h = __shfl_xor_sync(0xffffffffu, s1h, 16), r1l = __shfl_xor_sync(0xffffffffu, s1l, 16);
  ff_add(k0h, k0l, r0h, r0l);
  ff_add(k1h, k1l, r1h, r1l);
  const bool up2 = lane & 8;
  float kh = up2 ? k1h : k0h, kl = up2 ? k1l : k0l;
  const float sh = up2 ? k0h : k1h, sl = up2 ? k0l : k1l;
  const float qh = __shfl_xor_sync(0xffffffffu, sh, 8), ql = __shfl_xor_sync(0xffffffffu, sl, 8);
  ff_add(kh, kl, qh, ql);
#pragma unroll
  for (int m = 4; m >= 1; m >>= 1) {
    const float th = __shfl_xor_sync(0xffffffffu, kh, m), tl = __shfl_xor_sync(0xffffffffu, kl, m);
    ff_add(kh, kl, th, tl);
  }
  oh = kh;
  ol = kl;
}

// Same for BYT = 2: lanes 0-15 end with row 0, lanes 16-31 with row 1.
__device__ __forceinline__ void ff_reduce2_scatter(const float h[2], const float l[2], int lane,
                                                   float& oh, float& ol) {
  const bool up = lane & 16;
  float kh = up ? h[1] : h[0], kl = up ? l[1] : l[0];
  const float sh = up ? h[0] : h[1], sl = up ? l[0] : l[1];
  const float rh = __shfl_xor_sync(0xffffffffu, sh, 16), rl = __shfl_xor_sync(0xffffffffu, sl, 16);
  ff_add(kh, kl, rh, rl);
#pragma unroll
  for (int m = 8; m >= 1; m >>= 1) {
    const float th = __shfl_xor_sync(0xffffffffu, kh, m), tl = __shfl_xor_sync(0xffffffffu, kl, m);
    ff_add(kh, kl, th, tl);
  }
  oh = kh;
  ol = kl;
}

// ---------------------------------------------------------------- kernel

template <typename T, int P, bool TMA>
__global__ void __launch_bounds__(TileCfg<T, P>::NT, 1) k1_project_kernel(K1Params p) {
  using C = TileCfg<T, P>;
  constexpr bool FL = C::FL;
  using A = typename std::conditional<FL, float, uint32_t>::type;    // accumulators
  using IT = typename std::conditional<FL, double, uint32_t>::type;  // image pixels
  constexpr int TX = C::TX, XT = C::XT, NT = C::NT, NW = C::NW;
  constexpr int BYT = C::BYT, TY = C::TY;
  constexpr bool H3 = P > 3, H4 = P > 4, H5 = P > 5, H6 = P > 6, H7 = P > 7, H8 = P > 8;
  constexpr int PW = FL ? 2 : 1;  // words per pixel pair in shared buffers
  constexpr int kDiag = XT + BY - 1;

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
  A* slot2 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * XT));        // [2][TY][XT]
  A* slot1 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * NW * BYT));  // [2][TY][NW][BYT]
  A* mb3 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * NW * BYT));    // [2][TY][NW][BYT]
  A* mb4 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * NW * BYT));
  A* mb5 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * XT));          // [2][TY][XT]
  A* mb6 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * TY * XT));
  A* ex34 = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * 2 * BY));          // [2][2][BY]
  A* dg = reinterpret_cast<A*>(take(sizeof(A) * PW * 2 * 2 * kDiag));         // [2][2][kDiag]

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX, lane = tid & 31, wx = tx >> 5;
  const int xl = tx * R, yl = ty * BYT;
  const T* __restrict__ vol = static_cast<const T*>(p.vol);
  const int64_t L = p.L, M = p.M, N = p.N;
  const ImageSet& set = p.set;
  IT* img = static_cast<IT*>(p.images);
  const bool vec_global =
      (L % R) == 0 && ((reinterpret_cast<uintptr_t>(p.vol) % (R * sizeof(T))) == 0);

  const int64_t ub = p.units * (int64_t)blockIdx.x / gridDim.x;
  const int64_t ue = p.units * (int64_t)(blockIdx.x + 1) / gridDim.x;

  for (int i = tid; i < 2 * 2 * kDiag * PW; i += NT) dg[i] = (A)0;
  if constexpr (TMA) {
    if (tid == 0) {
      for (int i = 0; i < STAGES; ++i) mbar_init(smem_u32(&mbar[i]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();

  // unit -> (tile x0, band y0, z)
  auto decode = [&](int64_t u, int64_t& x0, int64_t& y0, int64_t& z) {
    const int64_t seg = u / N;
    z = u % N;
    y0 = (seg % p.nbands) * BY;
    x0 = (seg / p.nbands) * XT;
  };

  // Producer cursor (thread 0): the next unit to copy, advanced without
  // divisions.  Units run z fastest, then band, then tile.
  int64_t pc_x0 = 0, pc_y0 = 0, pc_z = 0;
  if constexpr (TMA) {
    if (tid == 0) decode(ub, pc_x0, pc_y0, pc_z);
  }
  auto advance = [&](int64_t& x0, int64_t& y0, int64_t& z) {
    if (++z == N) {
      z = 0;
      y0 += BY;
      if (y0 >= M) { y0 = 0; x0 += XT; }
    }
  };
  // bulk-copy the slice at the producer cursor into stage buffer st
  auto issue_next = [&](int st) {
    if constexpr (TMA) {
      const int64_t x0 = pc_x0, y0 = pc_y0, z = pc_z;
      advance(pc_x0, pc_y0, pc_z);
      const int64_t rows = (M - y0) < BY ? (M - y0) : BY;
      const int64_t w = (L - x0) < XT ? (L - x0) : XT;
      const uint32_t row_bytes = (uint32_t)(w * sizeof(T));
      const uint32_t mb = smem_u32(&mbar[st]);
      mbar_expect_tx(mb, (uint32_t)(rows * row_bytes));
      for (int64_t r = 0; r < rows; ++r) {
        const T* src = vol + ((z * M + y0 + r) * L + x0);
        bulk_g2s(smem_u32(stage + ((size_t)st * BY + r) * XT), src, row_bytes, mb);
      }
    }
  };

  if constexpr (TMA) {
    if (tid == 0)
      for (int i = 0; i < STAGES && ub + i < ue; ++i) issue_next(i);
  }

  // register state
  A a0[BYT][R], w3[BYT][R], w4[BYT][R], w5[BYT][R], w6[BYT][R];
  float a0c[BYT][R], w3c[BYT][R], w4c[BYT][R], w5c[BYT][R], w6c[BYT][R];
#pragma unroll
  for (int r = 0; r < BYT; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) {
      a0[r][c] = 0; w3[r][c] = 0; w4[r][c] = 0; w5[r][c] = 0; w6[r][c] = 0;
      a0c[r][c] = 0.f; w3c[r][c] = 0.f; w4c[r][c] = 0.f; w5c[r][c] = 0.f; w6c[r][c] = 0.f;
    }

  bool aborted = false;

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
        IT* dst = img + set.base[0] + y * set.F[0] + xs + c;
        if constexpr (FL) red_ff(dst, a0[r][c], a0c[r][c]);
        else if (a0[r][c]) atomicAdd(dst, a0[r][c]);
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
          if (f >= set.F[3]) continue;
          IT* dst = img + set.base[3] + y * set.F[3] + f;
          if constexpr (FL) red_ff(dst, w3[r][q], w3c[r][q]);
          else if (w3[r][q]) atomicAdd(dst, w3[r][q]);
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
          if (f < 0 || f >= set.F[4]) continue;
          IT* dst = img + set.base[4] + y * set.F[4] + f;
          if constexpr (FL) red_ff(dst, w4[r][q], w4c[r][q]);
          else if (w4[r][q]) atomicAdd(dst, w4[r][q]);
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
        for (int c = 0; c < R; ++c) {
          if (xs + c >= L) continue;
          IT* dst = img + set.base[5] + srow * set.F[5] + xs + c;
          if constexpr (FL) red_ff(dst, w5[q][c], w5c[q][c]);
          else if (w5[q][c]) atomicAdd(dst, w5[q][c]);
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
        for (int c = 0; c < R; ++c) {
          if (xs + c >= L) continue;
          IT* dst = img + set.base[6] + srow * set.F[6] + xs + c;
          if constexpr (FL) red_ff(dst, w6[q][c], w6c[q][c]);
          else if (w6[q][c]) atomicAdd(dst, w6[q][c]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < BYT; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) {
        a0[r][c] = 0; w3[r][c] = 0; w4[r][c] = 0; w5[r][c] = 0; w6[r][c] = 0;
        a0c[r][c] = 0.f; w3c[r][c] = 0.f; w4c[r][c] = 0.f; w5c[r][c] = 0.f; w6c[r][c] = 0.f;
      }
  };

  int64_t s = 0;  // CTA step counter
  int64_t u = ub;  // first unit of the current segment
  while (u < ue && !aborted) {
    // one segment: a (tile, band) streamed over z in [za, zb)
    int64_t x0, y0, za;
    decode(u, x0, y0, za);
    const int64_t zb = (N - za) < (ue - u) ? N : za + (ue - u);
    int64_t z = za;
    while (z < zb && !aborted) {
#pragma unroll
    for (int j = 0; j < R; ++j) {  // unrolled so window slots are static: j == z % R
      if (z >= zb || aborted) break;
      if ((int)(z & (R - 1)) != j) continue;  // align the unroll phase with z
      const int st = (int)(s % STAGES);
      const int par = (int)((s / STAGES) & 1);
      const int sb = (int)(s & 1);  // shared double-buffer index
      const int64_t xs = x0 + xl, yt = y0 + yl;

      // ---- 1. wait for the slice (bounded)
      bool ok = true;
      if constexpr (TMA) ok = mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)par);

      // ---- 3. the micro-tile
      A v[BYT][R];
#pragma unroll
      for (int r = 0; r < BYT; ++r) {
        const int64_t y = yt + r;
        const bool row_ok = ok && (y < M) && (xs < L);
        if (row_ok) {
          if constexpr (TMA) {
            load4_smem(stage + ((size_t)st * BY + yl + r) * XT + xl, v[r]);
#pragma unroll
            for (int c = 0; c < R; ++c)
              if (xs + c >= L) v[r][c] = 0;
          } else {
            load4_global(vol + (z * M + y) * L, xs, L, vec_global, v[r]);
          }
        } else {
#pragma unroll
          for (int c = 0; c < R; ++c) v[r][c] = 0;
        }
      }

      // ---- 4. images crossing the slice
      if constexpr (FL) {
        // packed pairs: adjacent columns for images 0, 5, 6; adjacent rows for
        // the x-rotating windows of images 3, 4 (pairs stay fixed across j)
#pragma unroll
        for (int r = 0; r < BYT; ++r)
#pragma unroll
          for (int c = 0; c < R; c += 2) {
            ts_acc2(a0[r][c], a0c[r][c], v[r][c], a0[r][c + 1], a0c[r][c + 1], v[r][c + 1]);
            if constexpr (H5) {
              const int q = (r + j) % BYT;
              ts_acc2(w5[q][c], w5c[q][c], v[r][c], w5[q][c + 1], w5c[q][c + 1], v[r][c + 1]);
            }
            if constexpr (H6) {
              const int q = (r - j + R) % BYT;
              ts_acc2(w6[q][c], w6c[q][c], v[r][c], w6[q][c + 1], w6c[q][c + 1], v[r][c + 1]);
            }
          }
#pragma unroll
        for (int r = 0; r < BYT; r += 2)
#pragma unroll
          for (int c = 0; c < R; ++c) {
            if constexpr (H3) {
              const int q = (c + j) % R;
              ts_acc2(w3[r][q], w3c[r][q], v[r][c], w3[r + 1][q], w3c[r + 1][q], v[r + 1][c]);
            }
            if constexpr (H4) {
              const int q = (c - j + R) % R;
              ts_acc2(w4[r][q], w4c[r][q], v[r][c], w4[r + 1][q], w4c[r + 1][q], v[r + 1][c]);
            }
          }
      }
#pragma unroll
      for (int r = 0; r < BYT; ++r)
#pragma unroll
        for (int c = 0; c < R; ++c) {
          if constexpr (FL) {
          } else {
            a0[r][c] += v[r][c];
            if constexpr (H3) w3[r][(c + j) % R] += v[r][c];
            if constexpr (H4) w4[r][(c - j + R) % R] += v[r][c];
            if constexpr (H5) w5[(r + j) % BYT][c] += v[r][c];
            if constexpr (H6) w6[(r - j + R) % BYT][c] += v[r][c];
          }
        }

      // ---- 5. image 2 (column sums) and image 1 (row sums) of this slice
      {
        A cs[R];
        float csc[R];
#pragma unroll
        for (int c = 0; c < R; ++c) {
          cs[c] = v[0][c];
          csc[c] = 0.f;
#pragma unroll
          for (int r = 1; r < BYT; ++r) {
            if constexpr (FL) ts_acc(cs[c], csc[c], v[r][c]);
            else cs[c] += v[r][c];
          }
        }
        A* s2 = slot2 + ((size_t)(sb * TY + ty) * XT + xl) * PW;
        if constexpr (FL) {
          *reinterpret_cast<float4*>(s2) = make_float4(cs[0], csc[0], cs[1], csc[1]);
          *reinterpret_cast<float4*>(s2 + 4) = make_float4(cs[2], csc[2], cs[3], csc[3]);
        } else {
          *reinterpret_cast<uint4*>(s2) = make_uint4(cs[0], cs[1], cs[2], cs[3]);
        }
        A rs[BYT];
        float rsc[BYT];
#pragma unroll
        for (int r = 0; r < BYT; ++r) {
          rs[r] = v[r][0];
          rsc[r] = 0.f;
#pragma unroll
          for (int c = 1; c < R; ++c) {
            if constexpr (FL) ts_acc(rs[r], rsc[r], v[r][c]);
            else rs[r] += v[r][c];
          }
        }
        if constexpr (FL) {
          float lo[BYT];
#pragma unroll
          for (int r = 0; r < BYT; ++r) lo[r] = rsc[r];
          float oh, ol;
          if constexpr (BYT == 4) ff_reduce4_scatter(rs, lo, lane, oh, ol);
          else ff_reduce2_scatter(rs, lo, lane, oh, ol);
          constexpr int lanes_per_row = 32 / BYT;
          if ((lane & (lanes_per_row - 1)) == 0) {
            A* d = slot1 + ((size_t)((sb * TY + ty) * NW + wx) * BYT + lane / lanes_per_row) * PW;
            d[0] = oh;
            d[1] = ol;
          }
        } else {
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            const uint32_t t = __reduce_add_sync(0xffffffffu, rs[r]);
            if (lane == 0) slot1[(size_t)((sb * TY + ty) * NW + wx) * BYT + r] = t;
          }
        }
      }

      // ---- 6. images 7/8 (x+-y) of this slice: diagonal sums into shared buffers
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
            A* cell = dg + ((size_t)(sb * 2 + im) * kDiag + idx) * PW;
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

      // ---- 7. hand the leaving window pixels on
      if constexpr (H3) {  // logical 0 (slot j) moves to the left neighbour
#pragma unroll
        for (int r = 0; r < BYT; ++r) {
          const A sv = w3[r][j];
          const float sc = w3c[r][j];
          const A rv = __shfl_down_sync(0xffffffffu, sv, 1);
          const float rc = __shfl_down_sync(0xffffffffu, sc, 1);
          w3[r][j] = (lane == 31) ? (A)0 : rv;
          w3c[r][j] = (lane == 31) ? 0.f : rc;
          if (lane == 0) {
            A* d = (wx == 0) ? ex34 + ((size_t)(sb * 2 + 0) * BY + yl + r) * PW
                             : mb3 + ((size_t)((sb * TY + ty) * NW + wx - 1) * BYT + r) * PW;
            d[0] = sv;
            if constexpr (FL) d[1] = sc;
          }
        }
      }
      if constexpr (H4) {  // logical R-1 (slot (R-1-j) % R) moves to the right neighbour
        const int q = (R - 1 - j + R) % R;
#pragma unroll
        for (int r = 0; r < BYT; ++r) {
          const A sv = w4[r][q];
          const float sc = w4c[r][q];
          const A rv = __shfl_up_sync(0xffffffffu, sv, 1);
          const float rc = __shfl_up_sync(0xffffffffu, sc, 1);
          w4[r][q] = (lane == 0) ? (A)0 : rv;
          w4c[r][q] = (lane == 0) ? 0.f : rc;
          if (lane == 31) {
            A* d = (wx == NW - 1) ? ex34 + ((size_t)(sb * 2 + 1) * BY + yl + r) * PW
                                  : mb4 + ((size_t)((sb * TY + ty) * NW + wx + 1) * BYT + r) * PW;
            d[0] = sv;
            if constexpr (FL) d[1] = sc;
          }
        }
      }
      // images 5/6: the leaving window row goes to the row group above (5)
      // or below (6); the band's edge group emits it
      A out5[R], out6[R];
      float out5c[R], out6c[R];
      if constexpr (H5) {
#pragma unroll
        for (int c = 0; c < R; ++c) {
          out5[c] = w5[j % BYT][c]; out5c[c] = w5c[j % BYT][c];
          w5[j % BYT][c] = 0; w5c[j % BYT][c] = 0.f;
        }
        if (ty > 0) {
          A* d = mb5 + ((size_t)(sb * TY + ty - 1) * XT + xl) * PW;
          if constexpr (FL) {
            *reinterpret_cast<float4*>(d) = make_float4(out5[0], out5c[0], out5[1], out5c[1]);
            *reinterpret_cast<float4*>(d + 4) = make_float4(out5[2], out5c[2], out5[3], out5c[3]);
          } else {
            *reinterpret_cast<uint4*>(d) = make_uint4(out5[0], out5[1], out5[2], out5[3]);
          }
        }
      }
      if constexpr (H6) {
        const int q = (BYT - 1 - j + R) % BYT;
#pragma unroll
        for (int c = 0; c < R; ++c) {
          out6[c] = w6[q][c]; out6c[c] = w6c[q][c];
          w6[q][c] = 0; w6c[q][c] = 0.f;
        }
        if (ty < TY - 1) {
          A* d = mb6 + ((size_t)(sb * TY + ty + 1) * XT + xl) * PW;
          if constexpr (FL) {
            *reinterpret_cast<float4*>(d) = make_float4(out6[0], out6c[0], out6[1], out6c[1]);
            *reinterpret_cast<float4*>(d + 4) = make_float4(out6[2], out6c[2], out6[3], out6c[3]);
          } else {
            *reinterpret_cast<uint4*>(d) = make_uint4(out6[0], out6[1], out6[2], out6[3]);
          }
        }
      }

      // ---- 9. step barrier, also agreeing on an abort
      if (__syncthreads_or(!ok)) {
        aborted = true;
        break;
      }
      if constexpr (TMA) {  // the slice is consumed: refill its stage
        if (tid == 0 && u + STAGES < ue) issue_next(st);
      }

      // ---- 10. receive the handed-over window pixels
      if constexpr (H3) {
        if (lane == 31 && wx < NW - 1) {
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            const A* d = mb3 + ((size_t)((sb * TY + ty) * NW + wx) * BYT + r) * PW;
            w3[r][j] = d[0];
            if constexpr (FL) w3c[r][j] = d[1];
          }
        }
      }
      if constexpr (H4) {
        const int q = (R - 1 - j + R) % R;
        if (lane == 0 && wx > 0) {
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            const A* d = mb4 + ((size_t)((sb * TY + ty) * NW + wx) * BYT + r) * PW;
            w4[r][q] = d[0];
            if constexpr (FL) w4c[r][q] = d[1];
          }
        }
      }
      if constexpr (H5) {
        if (ty < TY - 1) {
          const A* d = mb5 + ((size_t)(sb * TY + ty) * XT + xl) * PW;
#pragma unroll
          for (int c = 0; c < R; ++c) {
            w5[j % BYT][c] = d[c * PW];
            if constexpr (FL) w5c[j % BYT][c] = d[c * PW + 1];
          }
        }
      }
      if constexpr (H6) {
        const int q = (BYT - 1 - j + R) % BYT;
        if (ty > 0) {
          const A* d = mb6 + ((size_t)(sb * TY + ty) * XT + xl) * PW;
#pragma unroll
          for (int c = 0; c < R; ++c) {
            w6[q][c] = d[c * PW];
            if constexpr (FL) w6c[q][c] = d[c * PW + 1];
          }
        }
      }

      // ---- 11. emit the pixels this CTA has completed
      if constexpr (H5) {  // image 5: top group's leaving row, pixel row y0 + z
        if (ty == C::G_I5) {
          const int64_t srow = y0 + z;
          if (srow < set.S[5] && xs < L) {
            IT* dst = img + set.base[5] + srow * set.F[5] + xs;
            const int n = (int)((L - xs) < R ? (L - xs) : R);
            if constexpr (FL) {
              for (int c = 0; c < n; ++c) red_ff(dst + c, out5[c], out5c[c]);
            } else {
              for (int c = 0; c < n; ++c)
                if (out5[c]) atomicAdd(dst + c, out5[c]);
            }
          }
        }
      }
      if constexpr (H6) {  // image 6: bottom group's leaving row, y0+BY-1-z+(N-1)
        if (ty == C::G_I6) {
          const int64_t srow = y0 + BY - 1 - z + (N - 1);
          if (srow >= 0 && srow < set.S[6] && xs < L) {
            IT* dst = img + set.base[6] + srow * set.F[6] + xs;
            const int n = (int)((L - xs) < R ? (L - xs) : R);
            if constexpr (FL) {
              for (int c = 0; c < n; ++c) red_ff(dst + c, out6[c], out6c[c]);
            } else {
              for (int c = 0; c < n; ++c)
                if (out6[c]) atomicAdd(dst + c, out6[c]);
            }
          }
        }
      }
      if (ty == C::G_I2 && xs < L) {  // image 2: merge the TY column partials
        const int n = (int)((L - xs) < R ? (L - xs) : R);
        IT* dst = img + set.base[2] + z * set.F[2] + xs;
        if constexpr (FL) {
          float h[R], l[R];
#pragma unroll
          for (int c = 0; c < R; ++c) {
            h[c] = 0.f;
            l[c] = 0.f;
#pragma unroll
            for (int g = 0; g < TY; ++g) {
              const float* e = slot2 + ((size_t)(sb * TY + g) * XT + xl + c) * PW;
              ff_add(h[c], l[c], e[0], e[1]);
            }
          }
          for (int c = 0; c < n; ++c) red_ff(dst + c, h[c], l[c]);
        } else {
#pragma unroll
          for (int c = 0; c < R; ++c) {
            uint32_t t = 0;
#pragma unroll
            for (int g = 0; g < TY; ++g) t += slot2[(size_t)(sb * TY + g) * XT + xl + c];
            if (c < n && t) atomicAdd(dst + c, t);
          }
        }
      }
      if (ty == C::G_I1 && tx < BY) {  // image 1: one thread per row of the band
        {
          const int row = tx;
          const int64_t y = y0 + row;
          if (y < M) {
            IT* dst = img + set.base[1] + z * set.F[1] + y;
            const int g = row / BYT, r = row % BYT;
            if constexpr (FL) {
              float h = 0.f, l = 0.f;
#pragma unroll
              for (int w = 0; w < NW; ++w) {
                const float* e = slot1 + ((size_t)((sb * TY + g) * NW + w) * BYT + r) * PW;
                ff_add(h, l, e[0], e[1]);
              }
              if (p.nxt == 1) dst[0] = ff_to_f64(h, l);  // the row lies in this tile: complete
              else red_ff(dst, h, l);
            } else {
              uint32_t t = 0;
#pragma unroll
              for (int w = 0; w < NW; ++w) t += slot1[(size_t)((sb * TY + g) * NW + w) * BYT + r];
              if (p.nxt == 1) dst[0] = t;
              else if (t) atomicAdd(dst, t);
            }
          }
        }
      }
      if (ty == C::G_EDGE && tx >= C::EDGE0 && tx < C::EDGE0 + 2 * BY) {  // image 3/4 edges
        {
          const int e = tx - C::EDGE0;
          const int im = e / BY, row = e % BY;
          const int64_t y = y0 + row;
          if (((im == 0 && H3) || (im == 1 && H4)) && y < M) {
            // image 3 leaves at x = x0: f = x0 + z; image 4 at x = x0+XT-1:
            // f = x0 + XT - 1 - z + (N - 1)
            const int k = im == 0 ? 3 : 4;
            const int64_t f = im == 0 ? x0 + z : x0 + XT - 1 - z + (N - 1);
            const A* cell = ex34 + ((size_t)(sb * 2 + im) * BY + row) * PW;
            if (f >= 0 && f < set.F[k]) {
              IT* dst = img + set.base[k] + y * set.F[k] + f;
              if constexpr (FL) {
                red_ff(dst, cell[0], cell[1]);
              } else {
                if (cell[0]) atomicAdd(dst, cell[0]);
              }
            }
          }
        }
      }
      if constexpr (H7 || H8) {  // images 7/8: group 3 emits the diagonal buffers
        if (ty == C::G_DIAG) {
          for (int e = tx; e < 2 * kDiag; e += TX) {
            const int im = e / kDiag, idx = e % kDiag;
            if ((im == 0 && !H7) || (im == 1 && !H8)) continue;
            A* cell = dg + ((size_t)(sb * 2 + im) * kDiag + idx) * PW;
            const int k = 7 + im;
            const int64_t f = im == 0 ? x0 + y0 + idx : x0 - y0 - (BY - 1) + idx + (M - 1);
            if (f >= 0 && f < set.F[k]) {
              IT* dst = img + set.base[k] + z * set.F[k] + f;
              if constexpr (FL) red_ff(dst, cell[0], cell[1]);
              else if (cell[0]) atomicAdd(dst, cell[0]);
            }
            cell[0] = (A)0;
            if constexpr (FL) cell[1] = 0.f;
          }
        }
      }

      ++s;
      ++u;
      ++z;
    }
    }
    if (!aborted) drain(x0, y0, zb - 1);
  }

  if (aborted) {
    // let bulk copies still in flight land before the CTA's shared memory is
    // released (bounded; they were issued for units u .. u+STAGES-1)
    if constexpr (TMA) {
      if (tid == 0) {
        for (int i = 0; i < STAGES && u + i < ue; ++i) {
          const int64_t ss = s + i;
          mbar_wait_bounded(smem_u32(&mbar[ss % STAGES]), (uint32_t)((ss / STAGES) & 1));
        }
      }
    }
    if (tid == 0 && p.status) atomicMax(p.status, kStatusTimeout);
  }
}

template <typename T, int P, bool TMA>
cudaError_t launch_t(const ProjectArgs& a, cudaStream_t st) {
  using C = TileCfg<T, P>;
  constexpr int BYT = C::BYT, TY = C::TY;
  constexpr bool FL = C::FL;
  using Acc = typename std::conditional<FL, float, uint32_t>::type;
  constexpr int PW = FL ? 2 : 1;
  K1Params p{};
  p.vol = a.vol;
  p.L = a.L; p.M = a.M; p.N = a.N;
  p.nbands = (a.M + BY - 1) / BY;
  p.nxt = (a.L + C::XT - 1) / C::XT;
  p.units = p.nxt * p.nbands * a.N;
  p.set = a.set;
  p.images = a.images;
  p.status = a.status;

  auto rnd = [](size_t b) { return (b + 127) & ~size_t(127); };
  constexpr int NW = C::NW, XT = C::XT, kDiag = XT + BY - 1;
  size_t smem = rnd(sizeof(uint64_t) * STAGES);
  if (TMA) smem += rnd(sizeof(T) * STAGES * BY * XT);
  smem += rnd(sizeof(Acc) * PW * 2 * TY * XT);               // slot2
  smem += 3 * rnd(sizeof(Acc) * PW * 2 * TY * NW * BYT);     // slot1, mb3, mb4
  smem += 2 * rnd(sizeof(Acc) * PW * 2 * TY * XT);           // mb5, mb6
  smem += rnd(sizeof(Acc) * PW * 2 * 2 * BY);                // ex34
  smem += rnd(sizeof(Acc) * PW * 2 * 2 * kDiag);             // dg

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
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) { cached_sms[dev] = sms; cached_per_sm[dev] = per_sm; }
  }
  // at least ~8 z-steps per CTA so segment drains stay a small overhead
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t by_work = (p.units + 7) / 8;
  if (grid > by_work) grid = by_work;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, C::NT, smem, st>>>(p);
  return cudaGetLastError();
}

// Launch for one element type and image count; picks the bulk-copy path
// when rows are 16-byte aligned.
template <typename T, int P>
cudaError_t launch_p(const ProjectArgs& a, cudaStream_t st) {
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.vol);
  const bool tma = ((a.L * (int64_t)sizeof(T)) % 16 == 0) && (base % 16 == 0);
  return tma ? launch_t<T, P, true>(a, st) : launch_t<T, P, false>(a, st);
}

}  // namespace k1
}  // namespace dpma
