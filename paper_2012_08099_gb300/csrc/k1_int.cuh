// Step 1 of the Discrete Projection Moment method on integer lanes: one fused
// pass over the volume that writes every projection image at once (Sec. 3.1,
// Eq. 4 with the image set of Eqs. 5-9 and the +-pi/4 family about x).
//
// Every sum is an exact 32-bit integer sum.  Integer volumes add their voxels
// directly.  A float32 voxel v is first quantised exactly onto a power-of-two
// grid in two signed limbs,
//     v ~= h1 * 2^-e1 + h2 * 2^-(e1 + B + 1),   |h1|, |h2| <= 2^B,
// (h1 = round(v 2^e1), h2 = round((v - h1 2^-e1) 2^(e1+B+1)), both by the
// round-to-nearest of a single float addition of 1.5 * 2^23), and each limb
// is projected like an integer volume into its own set of images.  The
// images, and everything computed from them, are then exact integers; the
// only rounding of the whole float pipeline is this quantisation (at most
// half a grid step 2^-(e1+B+1) per voxel) and the final conversion of the
// moments to double.  B is chosen on the host so that no line sum can leave
// the int32 range; e1 comes from a sample of the volume taken while the
// images are cleared (with 2x headroom).  A voxel beyond the grid's range or
// a non-finite voxel raises a flag; the pipeline then recomputes the volume
// with the compensated float kernels, which it queues behind this one and
// which do nothing unless the flag is set.
//
// Work decomposition.  A CTA owns a tile of 64 columns (x) by TYc rows (y)
// and streams it along z two slices at a time; persistent CTAs take ranges
// of (tile, z-pair) units, interleaved over the x-tiles so that the CTAs of
// one band read whole rows of the volume together.  Each z-pair of a tile
// arrives as one tiled tensor copy (cp.async.bulk.tensor.3d, box 64 x TYc x
// 2, zero filled outside the volume) into a ring of stages.  The CTA's 16
// warps form two groups, each with the lane order that makes its images'
// hand-overs shuffles inside a lane group:
//   group A (warps 0-7) reads the stage: groups of GA lanes along x, lane tx
//     owning RA consecutive x-values of BYA rows; images 1 (sum along x) and
//     3/4 (x+-z, y).  It also writes the z-pair, as 32-bit lanes (limbs for
//     a float volume), into a transposed buffer in blocks of 2 rows x BB
//     columns x NL limbs (16 bytes), whose order is XOR-swizzled so that both
//     these writes and group B's reads are free of bank conflicts;
//   group B (warps 8-15), one z-pair behind, reads that buffer: groups of GB
//     lanes along y, lane gl owning RYB = 8 consecutive rows of BB columns;
//     images 0 (x, y), 2 (sum along y) and 5/6 (y+-z, x).
// Images whose lines leave the slice accumulate in registers across z in
// windows of RA pixels per owned row (3/4) or RYB pixels per owned column
// (5/6): the two slices of a step land on neighbouring pixels, so a pixel
// takes both voxels in one 3-input add; after the step the two pixels that
// leave a lane's window go to its neighbour lane.  At the tile edge they are
// complete for this tile: images 3/4 stage them into runs of 16 consecutive
// pixels, merged by one coalesced reduction every 8 steps; images 5/6 stage
// the edge rows, which all warps of group B merge together after the next
// barrier.  Images whose lines lie in the slice
// (1 and 2) are reduced per step across the lane group.  Partial pixels go to
// the images in L2 with red.global.add.u32 (wrapping 32-bit adds are exact
// because every complete pixel fits in int32).
#pragma once
#include <cuda.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "dpma_internal.cuh"

namespace dpma {
namespace k1i {

constexpr int kStatusTimeout = 5;
constexpr int kFlagRange = 1;  // a float voxel outside the quantisation grid

constexpr float kMagic = 12582912.0f;         // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;  // its bit pattern

template <typename T, int P> struct Cfg {
  static constexpr bool FL = std::is_same<T, float>::value;
  static constexpr int NL = FL ? 2 : 1;  // limbs per voxel
  static constexpr int TXc = 64;         // tile width
  static constexpr int NWG = 8;          // warps per group
  static constexpr int NT = 64 * NWG;    // both groups
  // group A: GA lanes along x, RA x-values by BYA rows per lane
  static constexpr int GA = FL ? 16 : 8;
  static constexpr int RA = TXc / GA;
  static constexpr int BYA = 2;
  static constexpr int TYc = (32 / GA) * NWG * BYA;
  // group B: GB lanes along y, RYB rows by BXB columns per lane
  static constexpr int RYB = 8;
  static constexpr int GB = TYc / RYB;
  static constexpr int BXB = TXc / (NWG * (32 / GB));
  // transposed buffer: 16-byte blocks of 2 rows x BB columns x NL limbs
  static constexpr int BB = 2 / NL;
  static constexpr int NBR = TYc / 2, NBC = TXc / BB;  // blocks per column / row
  // group B keeps image 0's sums in shared memory (in its own blocks of the
  // transposed layout) rather than in registers
  static constexpr bool A0SMEM = !FL;
  static constexpr int SLICE = TXc * TYc * (int)sizeof(T);
  static constexpr int STAGE = 2 * SLICE;  // one z-pair
  // ring depth: about 96 KB of z-pairs in flight
  static constexpr int STAGES = (98304 / STAGE) < 2 ? 2 : (98304 / STAGE > 16 ? 16 : 98304 / STAGE);
  static constexpr bool H3 = P > 3, H4 = P > 4, H5 = P > 5, H6 = P > 6, H7 = P > 7, H8 = P > 8;
  // the in-slice diagonal images 7 (x+y) and 8 (x-y) of one slice of a tile
  // span DW pixels
  static constexpr int DW = TXc + TYc - 1;
  static_assert(P >= 3 && P <= 9, "images 9 and 10 are projected by a second kernel");
  static_assert(GB * RYB == TYc && BXB == BB, "group B covers the tile with one block column");
  static_assert(RA % BB == 0 && NBR % 8 == 0 && BYA == 2, "transposed-buffer blocks");
  static_assert(RA <= 8 && RYB == 8, "windows of up to 8 positions");
};

struct Params {
  const void* vol;
  int L, M, N;
  int z0, nz;          // slices z0 .. z0 + nz - 1 (nz even unless the range ends at N)
  int nxt, nyt, nzp;   // tiles along x and y, z-pairs
  int units;           // nxt * nyt * nzp
  int cpt;             // CTAs per x-tile (grid = nxt * cpt), or 0: contiguous ranges
  ImageSet set;        // geometry; base[k] indexes limb 0
  int64_t limb_stride; // pixels from one limb's images to the next
  uint32_t* images;
  int* status;         // max(status, 5) when a bounded wait gives up
  int* flags;          // float volumes: |= kFlagRange
  // float volumes: the quantisation grid
  const uint32_t* sample;  // float bits of |v| maxima of a sample of the volume
  int nsample;
  int limb_bits;       // B
  int* scale_out;      // block 0 stores e1 and B here (may be null)
  long long wait_budget;
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
__device__ __forceinline__ bool mbar_test_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity`, giving up after `budget` cycles.  try_wait may
// suspend the thread for a while inside one probe, so a budget shorter than
// that (the fault-injection hook of the tests) polls with test_wait instead.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t a, uint32_t parity, long long budget) {
  if (budget < 65536) {
    const long long t0 = clock64();
    while (!mbar_test_wait(a, parity))
      if (clock64() - t0 > budget) return false;
    return true;
  }
  if (mbar_try_wait(a, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(a, parity))
    if (clock64() - t0 > budget) return false;
  return true;
}
// One box of the volume as a 3-D tensor, streamed through L2 with an
// evict-first policy so that the images being reduced there stay resident.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            int z, uint32_t mbar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// The limb images of a float32 volume are reduced in the L2 with an
// evict-last hint (H, policy `pol` made once per thread by keep_policy), so
// that the streaming volume (loaded evict-first) rather than the images
// leaves the L2 first: their DRAM write-backs halve (a 512^3 launch moves
// about 563 instead of 567 MB).  Integer images take plain reductions: the
// hinted form measured slower there.
__device__ __forceinline__ uint64_t keep_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
template <bool H>
__device__ __forceinline__ void red_always(uint32_t* p, uint32_t v, uint64_t pol) {
  if constexpr (H)
    asm volatile("red.global.add.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
                 : "memory");
  else
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
template <bool H>
__device__ __forceinline__ void red_add(uint32_t* p, uint32_t v, uint64_t pol) {
  if (v) red_always<H>(p, v, pol);
}
// without the zero test (per-step sums, which are rarely zero)
template <bool H>
__device__ __forceinline__ void red_add_always(uint32_t* p, uint32_t v, uint64_t pol) {
  red_always<H>(p, v, pol);
}
// Two neighbouring pixels p[0], p[1] (p 8-byte aligned) in one 64-bit
// reduction.  Unsigned integer images: every partial sum of a pixel stays
// below its final value, which is below 2^32, so the low word never carries
// into the high one.  Limb images (SG): the low word holds kLimbPairBias plus
// a partial sum of magnitude below 2^30, and `a` is added sign-extended, so
// again the low word stays inside [0, 2^32) and the high word is exact.
template <bool SG, bool H>
__device__ __forceinline__ void red_add_pair(uint32_t* p, uint32_t a, uint32_t b, uint64_t pol) {
  const unsigned long long v =
      ((unsigned long long)b << 32) +
      (SG ? (unsigned long long)(long long)(int32_t)a : (unsigned long long)a);
  if (!(a | b)) return;
  if constexpr (H)
    asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol)
                 : "memory");
  else
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// v[k] into p[k] for lo <= k < hi, neighbouring pixels paired where p + k is
// 8-byte aligned.
template <int W, bool SG, bool H>
__device__ __forceinline__ void red_add_run(uint32_t* p, const uint32_t (&v)[W], int lo, int hi,
                                            uint64_t pol) {
  auto go = [&](auto par) {
    constexpr int o = decltype(par)::value;  // 1: p[0] is the high word of a pair
    auto one = [&](int k) {
      if (k >= lo && k < hi) red_add<H>(p + k, v[k], pol);
    };
    if constexpr (o == 1) one(0);
#pragma unroll
    for (int k = o; k + 1 < W; k += 2) {
      const bool in_k = k >= lo && k < hi, in_n = k + 1 >= lo && k + 1 < hi;
      if (in_k && in_n) {
        red_add_pair<SG, H>(p + k, v[k], v[k + 1], pol);
      } else {
        one(k);
        one(k + 1);
      }
    }
    if constexpr (((W - o) & 1) == 1) one(W - 1);
  };
  if (reinterpret_cast<uintptr_t>(p) & 4) go(std::integral_constant<int, 1>{});
  else go(std::integral_constant<int, 0>{});
}
// Shared-memory reduction (no return value).
__device__ __forceinline__ void red_shared(uint32_t* p, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
__device__ __forceinline__ float max_nan(float a, float b) {
  float d;
  asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
  return d;
}


// W consecutive voxels of one row from shared memory, as 32-bit lanes.
template <int W> __device__ __forceinline__ void load_row(const float* p, float out[W]) {
  static_assert(W == 4, "four floats");
  const float4 q = *reinterpret_cast<const float4*>(p);
  out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
}
template <int W> __device__ __forceinline__ void load_row(const uint16_t* p, uint32_t out[W]) {
  static_assert(W == 8, "eight uint16 values");
  const uint4 q = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) { out[2 * i] = w[i] & 0xffffu; out[2 * i + 1] = w[i] >> 16; }
}
template <int W> __device__ __forceinline__ void load_row(const uint8_t* p, uint32_t out[W]) {
  static_assert(W == 8, "eight uint8 values");
  const uint2 q = *reinterpret_cast<const uint2*>(p);
  const uint32_t w[2] = {q.x, q.y};
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int b = 0; b < 4; ++b) out[4 * i + b] = (w[i] >> (8 * b)) & 0xffu;
}

// Sum over a group of G aligned lanes (G a power of two, the group given by
// `gl` = lane % G) of NV values per lane (NV a power of two).  The values are
// scattered while they are reduced: on return the lane holds the totals of
// values idx .. idx + NOUT - 1, NOUT = max(1, NV / G), in out[]; with NV < G
// each total is held by G / NV lanes.
template <int G, int NV> struct Scatter {
  static constexpr int NOUT = NV > G ? NV / G : 1;  // totals per lane
  static constexpr int REP = NV >= G ? 1 : G / NV;  // lanes holding each total
};
template <int G, int NV>
__device__ __forceinline__ void group_scatter_sum(const uint32_t (&v)[NV], int gl, int& idx,
                                                  uint32_t (&out)[Scatter<G, NV>::NOUT]) {
  static_assert(NV >= 1 && NV <= 16 && (NV & (NV - 1)) == 0, "NV: a power of two up to 16");
  uint32_t cur[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) cur[i] = v[i];
  int off = 0;
  int cnt = NV;
#pragma unroll
  for (int m = G / 2; m >= 1; m >>= 1) {
    if (cnt > 1) {
      const int half = cnt / 2;
      const bool up = (gl & m) != 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (i < half) {
          const uint32_t keep = up ? cur[i + half] : cur[i];
          const uint32_t send = up ? cur[i] : cur[i + half];
          cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
      }
      if (up) off += half;
      cnt = half;
    } else {
      cur[0] += __shfl_xor_sync(0xffffffffu, cur[0], m);
    }
  }
  idx = off;
#pragma unroll
  for (int i = 0; i < Scatter<G, NV>::NOUT; ++i) out[i] = cur[i];
}

// The first total index group_scatter_sum leaves with lane gl.
template <int G, int NV>
__device__ __forceinline__ int scatter_index(int gl) {
  int idx = 0;
#pragma unroll
  for (int m = G / 2, cnt = NV; m >= 1 && cnt > 1; m >>= 1, cnt >>= 1)
    if (gl & m) idx += cnt / 2;
  return idx;
}

// One float voxel as its two quantisation limbs; tracks max |v| (NaN sticks).
__device__ __forceinline__ void quantise(float x, float s1, float g1, float s2, uint32_t& h1,
                                         uint32_t& h2, float& vmax) {
  vmax = max_nan(vmax, fabsf(x));
  const float t1 = __fmaf_rn(x, s1, kMagic);
  h1 = __float_as_uint(t1) - kMagicBits;
  const float hf = __fsub_rn(t1, kMagic);
  const float rem = __fmaf_rn(-hf, g1, x);
  const float t2 = __fmaf_rn(rem, s2, kMagic);
  h2 = __float_as_uint(t2) - kMagicBits;
}

// A window of W + 1 pixels along the lane direction for a "+" image (pixel
// coordinate = position + z): slot k holds the pixel at position k of the
// lane's first voxel; a[j] / b[j] are the voxels at position j of the two
// slices.  Slice 0 lands on slot j, slice 1 on slot j + 1.  Slot W is empty
// at the start of every step, so S keeps slots 0..W-1.  Afterwards the two
// leaving pixels (returned in out0, out1) have moved to the previous lane of
// the group of G lanes and the window is laid out for the next z-pair.
template <int G, int W>
__device__ __forceinline__ void window_plus(uint32_t (&S)[W], const uint32_t (&a)[W],
                                            const uint32_t (&b)[W], int gl, uint32_t& out0,
                                            uint32_t& out1) {
  uint32_t u[W];
  u[0] = S[0] + a[0];
#pragma unroll
  for (int k = 1; k < W; ++k) u[k] = S[k] + a[k] + b[k - 1];
  uint32_t r0 = __shfl_down_sync(0xffffffffu, u[0], 1, G);
  uint32_t r1 = __shfl_down_sync(0xffffffffu, u[1], 1, G);
  if (gl == G - 1) { r0 = 0; r1 = 0; }
  out0 = u[0];
  out1 = u[1];
#pragma unroll
  for (int k = 0; k + 2 < W; ++k) S[k] = u[k + 2];
  S[W - 2] = b[W - 1] + r0;
  S[W - 1] = r1;
}

// The same for a "-" image (pixel coordinate = position - z + offset): slot
// k holds the pixel at position k - 1; slice 0 lands on slot j + 1, slice 1
// on slot j.  Slot 0 is empty at the start of every step, so S keeps slots
// 1..W (S[j] is slot j + 1); the two leaving pixels (slots W-1, W) move to
// the next lane.
template <int G, int W>
__device__ __forceinline__ void window_minus(uint32_t (&S)[W], const uint32_t (&a)[W],
                                             const uint32_t (&b)[W], int gl, uint32_t& outA,
                                             uint32_t& outB) {
  uint32_t u[W + 1];  // u[k]: slot k after the step's voxels (u[0] = b[0])
#pragma unroll
  for (int j = 0; j + 1 < W; ++j) u[j + 1] = S[j] + a[j] + b[j + 1];
  u[W] = S[W - 1] + a[W - 1];
  uint32_t rA = __shfl_up_sync(0xffffffffu, u[W - 1], 1, G);
  uint32_t rB = __shfl_up_sync(0xffffffffu, u[W], 1, G);
  if (gl == 0) { rA = 0; rB = 0; }
  outA = u[W - 1];
  outB = u[W];
  S[0] = rA;           // slot 1
  S[1] = b[0] + rB;    // slot 2
#pragma unroll
  for (int j = 2; j < W; ++j) S[j] = u[j - 1];  // slot j + 1
}

// Block position of (block row br, block column bc) inside its column of the
// transposed buffer: the low three bits of br are XORed with those of
// (br / 4) ^ (bc / 4).  Group A's lanes (one block row, block columns
// 4 tx + j) and group B's lanes (block rows 4 gl + i, one block column) then
// both hit distinct 16-byte bank groups.
__device__ __forceinline__ int block_pos(int br, int bc) {
  return br ^ (((br >> 2) ^ (bc >> 2)) & 7);
}

// The micro-tile of a group-A lane, both slices: NR rows of NC voxels
// starting at (row y, column x) of the stage, as NL limbs each.  After a wait
// that gave up the stage holds undefined values; they feed only the sums of
// that step, after which every thread leaves and the call reports the
// timeout, so they are not masked.
template <typename T, int NR, int NC, int NL, int TXc, int TYc>
__device__ __forceinline__ void load_tile(const T* sb, int y, int x, float s1, float g1,
                                          float s2, float& vmax, uint32_t (&v)[2][NR][NC][NL]) {
  constexpr bool FL = std::is_same<T, float>::value;
  using V = typename std::conditional<FL, float, uint32_t>::type;
#pragma unroll
  for (int sl = 0; sl < 2; ++sl)
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      V raw[NC];
      load_row<NC>(sb + ((size_t)sl * TYc + y + r) * TXc + x, raw);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if constexpr (FL) {
          quantise(raw[c], s1, g1, s2, v[sl][r][c][0], v[sl][r][c][NL - 1], vmax);
        } else {
          v[sl][r][c][0] = raw[c];
        }
      }
    }
}

template <typename T, int P>
__global__ void __launch_bounds__(Cfg<T, P>::NT, 1)
    k1_int_kernel(Params p, const __grid_constant__ CUtensorMap vmap) {
  using C = Cfg<T, P>;
  constexpr bool FL = C::FL;
  constexpr int NL = C::NL, NT = C::NT, NWG = C::NWG;
  constexpr int TXc = C::TXc, TYc = C::TYc, STAGES = C::STAGES;
  constexpr int GA = C::GA, RA = C::RA, BYA = C::BYA, RYB = C::RYB, GB = C::GB, BXB = C::BXB;
  constexpr int BB = C::BB, NBR = C::NBR, NBC = C::NBC;
  constexpr bool H3 = C::H3, H4 = C::H4, H5 = C::H5, H6 = C::H6, H7 = C::H7, H8 = C::H8;
  constexpr int DW = C::DW;
  constexpr int NTRA = (32 / GA) * NWG;  // group A thread-rows

  // ---- shared memory (sections 128-byte aligned)
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* at = smem;
  auto take = [&](size_t bytes) {
    unsigned char* r = at;
    at += (bytes + 127) & ~size_t(127);
    return r;
  };
  uint64_t* mbar = reinterpret_cast<uint64_t*>(take(sizeof(uint64_t) * STAGES));
  T* stage = reinterpret_cast<T*>(take((size_t)C::STAGE * STAGES));
  // exit runs of images 3 and 4, [thread-row][row][limb][16]
  uint32_t* run3 = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * NTRA * BYA * NL * 16));
  uint32_t* run4 = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * NTRA * BYA * NL * 16));
  // edge rows of images 5 and 6 leaving the tile, [buf][image][row][limb][column]
  uint32_t* edge = reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 2 * 2 * 2 * NL * TXc));
  // the z-pair for group B, [buf][slice][block column][block position] of
  // 16-byte blocks (2 rows x BB columns x NL limbs, row-major)
  uint4* xbuf = reinterpret_cast<uint4*>(take(sizeof(uint4) * 2 * 2 * NBC * NBR));
  // image 0 sums of group B (A0SMEM), [block column][block position]
  uint4* a0buf = C::A0SMEM ? reinterpret_cast<uint4*>(take(sizeof(uint4) * NBC * NBR)) : nullptr;
  // the step's partial diagonal rows of images 7 (group A) and 8 (group B),
  // [buf][slice][limb][DW], merged into the images one step later
  uint32_t* diag7 = H7 ? reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 2 * 2 * NL * DW))
                       : nullptr;
  uint32_t* diag8 = H8 ? reinterpret_cast<uint32_t*>(take(sizeof(uint32_t) * 2 * 2 * NL * DW))
                       : nullptr;
  float* red_f = reinterpret_cast<float*>(take(sizeof(float) * 32));
  int* abort_flag = reinterpret_cast<int*>(take(sizeof(int)));

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool isA = warp < NWG;
  // group A: lane tx of thread-row ty owns x = xl .. xl+RA-1, rows yl, yl+1
  const int tx = lane % GA;
  const int ty = (32 / GA) * warp + lane / GA;
  // group B: lane gl of column group cg owns rows yl .. yl+7, columns xl .. xl+BXB-1
  const int gl = lane % GB;
  const int cg = (warp - NWG) * (32 / GB) + lane / GB;
  const int xl = isA ? RA * tx : BXB * cg;
  const int yl = isA ? BYA * ty : RYB * gl;
  const int L = p.L, M = p.M, N = p.N;
  const ImageSet& set = p.set;
  uint32_t* const img = p.images;
  const int64_t lstride = p.limb_stride;
  const int zend = p.z0 + p.nz;
  const int c4 = N - 1, c6 = N - 1;  // offsets of the "-" images

  // ---- float volumes: the quantisation grid from the sample
  float s1 = 1.f, g1 = 1.f, s2 = 1.f, vcap = 0.f;
  if constexpr (FL) {
    float m = 0.f;
    for (int i = tid; i < p.nsample; i += NT) m = max_nan(m, __uint_as_float(p.sample[i]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = max_nan(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red_f[warp] = m;
    __syncthreads();
    m = 0.f;
    for (int i = 0; i < NT / 32; ++i) m = max_nan(m, red_f[i]);
    // headroom 2x (at least); an all-zero sample gets the grid of values up to 1
    float est = m > 0.f ? m * 2.f : 1.f;
    if (!(est < 3.0e38f)) est = 3.0e38f;
    int E;  // est < 2^E
    frexpf(est, &E);
    int e1 = p.limb_bits - E;
    const int e1max = 126 - p.limb_bits;
    if (e1 > e1max) e1 = e1max;
    if (e1 < -126) e1 = -126;
    s1 = ldexpf(1.f, e1);
    g1 = ldexpf(1.f, -e1);
    s2 = ldexpf(1.f, e1 + p.limb_bits + 1);
    vcap = ldexpf(1.f, p.limb_bits - e1);
    if (blockIdx.x == 0 && tid == 0 && p.scale_out) {
      p.scale_out[0] = e1;
      p.scale_out[1] = p.limb_bits;
    }
  }
  float vmax = 0.f;

  // Units are numbered x-tile-major: u = xtile * W + band * nzp + zpair with
  // W = nyt * nzp.  With cpt > 0, CTA b takes x-tile b % nxt and the
  // (b / nxt)-th of cpt equal ranges of that tile's (band, z-pair) units, so
  // the nxt CTAs of consecutive indexes stream the same rows of the volume
  // at the same time (whole rows per DRAM page, and the L2's 256-byte
  // promotion of each box row serves the neighbouring tile).
  const int W = p.nyt * p.nzp;
  int ub, ue;
  if (p.cpt > 0) {
    const int xtile = blockIdx.x % p.nxt, c = blockIdx.x / p.nxt;
    ub = xtile * W + (int)((int64_t)W * c / p.cpt);
    ue = xtile * W + (int)((int64_t)W * (c + 1) / p.cpt);
  } else {
    ub = (int)((int64_t)p.units * blockIdx.x / gridDim.x);
    ue = (int)((int64_t)p.units * (blockIdx.x + 1) / gridDim.x);
  }
  auto decode = [&](int u, int& x0, int& y0, int& z) {
    const int xtile = u / W, rem = u - xtile * W;
    const int band = rem / p.nzp;
    z = p.z0 + 2 * (rem - band * p.nzp);
    x0 = xtile * TXc;
    y0 = band * TYc;
  };

  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(smem_u32(&mbar[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
  }
  for (int i = tid; i < NTRA * BYA * NL * 16; i += NT) {
    run3[i] = 0;
    run4[i] = 0;
  }
  if constexpr (H7)
    for (int i = tid; i < 2 * 2 * NL * DW; i += NT) diag7[i] = 0;
  if constexpr (H8)
    for (int i = tid; i < 2 * 2 * NL * DW; i += NT) diag8[i] = 0;
  __syncthreads();

  const uint64_t policy = evict_first_policy();
  const uint64_t l2keep = FL ? keep_policy() : 0;
  int pc_u = ub;  // producer cursor (thread 0)
  auto issue = [&](int st) {
    int x0, y0, z;
    decode(pc_u, x0, y0, z);
    const uint32_t mb = smem_u32(&mbar[st]);
    mbar_expect_tx(mb, (uint32_t)C::STAGE);
    tma_load_3d(smem_u32(stage + (size_t)st * 2 * TYc * TXc), &vmap, x0, y0, z, mb, policy);
    ++pc_u;
  };
  if (tid == 0)
    for (int i = 0; i < STAGES && pc_u < ue; ++i) issue(i);

  // image pixel pointers (limb 0; limb l adds l * lstride)
  auto pix = [&](int k, int64_t s, int64_t f) -> uint32_t* {
    return img + set.base[k] + s * set.F[k] + f;
  };
  // One step's partial diagonal rows (buffer buf, z-pair at zb, tile x0, y0)
  // into image k (7: f = x0 + y0 + d; 8: f = x0 - y0 + d - (TYc - 1) + M - 1),
  // shared out over the 256 threads of one group (gt = thread in the group);
  // each entry is zeroed for the buffer's next use.
  auto merge_diag = [&](uint32_t* dg, int k, int buf, int zb, int x0, int y0, int gt) {
    const int64_t f0 = k == 7 ? (int64_t)x0 + y0 : (int64_t)x0 - y0 - (TYc - 1) + (M - 1);
    for (int e = gt; e < 2 * NL * DW; e += 32 * NWG) {
      const int d = e % DW, l = (e / DW) % NL, sl = e / (DW * NL);
      uint32_t* src = dg + ((buf * 2 + sl) * NL + l) * DW + d;
      const uint32_t val = *src;
      if (val) {
        *src = 0;
        const int64_t f = f0 + d;
        const int zz = zb + sl;
        if (f >= 0 && f < set.F[k] && zz < zend && zz < N)
          red_add_always<FL>(img + set.base[k] + (int64_t)zz * set.F[k] + f + l * lstride, val,
                         l2keep);
      }
    }
  };
  // the block of (block row br, block column bc), slice sl, buffer buf
  auto xblk = [&](int buf, int sl, int br, int bc) -> uint4* {
    return xbuf + (((size_t)buf * 2 + sl) * NBC + bc) * NBR + block_pos(br, bc);
  };

  bool aborted = false;
  int s = 0;   // CTA step counter
  int u = ub;  // next unit
  if (isA) {
    // ================= group A: images 1, 3, 4 (lanes along x)
    uint32_t w3[BYA][NL][RA], w4[BYA][NL][RA];
    auto clear_a = [&]() {
#pragma unroll
      for (int r = 0; r < BYA; ++r)
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int k = 0; k < RA; ++k) { w3[r][l][k] = 0; w4[r][l][k] = 0; }
    };
    clear_a();
    // exit runs of this lane group: image 3 pixels f3 + j, image 4 pixels
    // f4 + j (j < 16) of rows yt + r; positions [lo, hi) were written
    auto flush_runs = [&](int yt, int64_t f3, int lo3, int hi3, int64_t f4, int lo4, int hi4) {
      __syncwarp();
#pragma unroll
      for (int r = 0; r < BYA; ++r) {
        const int y = yt + r;
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
          for (int q = 0; q < 16 / GA; ++q) {
            const int j = tx + GA * q;
            if constexpr (H3) {
              uint32_t* slot = run3 + ((ty * BYA + r) * NL + l) * 16 + j;
              const int64_t f = f3 + j;
              if (j >= lo3 && j < hi3 && y < M && f < set.F[3])
                red_add<FL>(pix(3, y, f) + l * lstride, *slot, l2keep);
              *slot = 0;
            }
            if constexpr (H4) {
              uint32_t* slot = run4 + ((ty * BYA + r) * NL + l) * 16 + j;
              const int64_t f = f4 + j;
              if (j >= lo4 && j < hi4 && y < M && f >= 0 && f < set.F[4])
                red_add<FL>(pix(4, y, f) + l * lstride, *slot, l2keep);
              *slot = 0;
            }
          }
      }
      __syncwarp();
    };
    // this lane's blocks of the transposed buffer (buffer 0; buffer 1 follows)
    uint4* xwr[2][RA / BB];
#pragma unroll
    for (int sl = 0; sl < 2; ++sl)
#pragma unroll
      for (int j = 0; j < RA / BB; ++j) xwr[sl][j] = xblk(0, sl, ty, xl / BB + j);
    while (u < ue && !aborted) {
      int x0, y0, za;
      decode(u, x0, y0, za);
      const int tile_units = p.nzp - (za - p.z0) / 2;
      const int nsteps = tile_units < (ue - u) ? tile_units : (ue - u);
      const int yt = y0 + yl;
      int run_start = za, run_len = 0;
      // image 1 pixel (z, y) of this lane's total: base + z * M (see the emit below)
      constexpr int NV1 = NL * 2 * BYA;
      uint32_t* p1[Scatter<GA, NV1>::NOUT];
      {
        // the lane's total indices depend only on tx (group_scatter_sum)
        const int i0 = scatter_index<GA, NV1>(tx);
#pragma unroll
        for (int j = 0; j < Scatter<GA, NV1>::NOUT; ++j) {
          const int idx = i0 + j;
          const int r = idx % BYA, sl = (idx / BYA) & 1, l = idx / (2 * BYA);
          p1[j] = img + set.base[1] + (int64_t)sl * set.F[1] + (yt + r) + l * lstride;
        }
      }
      int z = za;
      for (int i = 0; i < nsteps; ++i) {
        // the previous step's diagonal rows of image 7 (complete since the
        // step barrier) into the image, while this step's copy may still land
        if constexpr (H7) {
          if (i > 0) merge_diag(diag7, 7, (s - 1) & 1, z - 2, x0, y0, tid);
        }
        const int st = s % STAGES;
        const bool ok = mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)((s / STAGES) & 1),
                                          p.wait_budget);
        if (!ok) *abort_flag = 1;
        uint32_t v[2][BYA][RA][NL];
        load_tile<T, BYA, RA, NL, TXc, TYc>(stage + (size_t)st * 2 * TYc * TXc, yl, xl, s1, g1,
                                            s2, vmax, v);
        // the micro-tile for group B, as blocks of 2 rows x BB columns
#pragma unroll
        for (int sl = 0; sl < 2; ++sl)
#pragma unroll
          for (int j = 0; j < RA / BB; ++j) {
            uint32_t e[4];
#pragma unroll
            for (int ri = 0; ri < 2; ++ri)
#pragma unroll
              for (int cj = 0; cj < BB; ++cj)
#pragma unroll
                for (int l = 0; l < NL; ++l) e[(ri * BB + cj) * NL + l] = v[sl][ri][BB * j + cj][l];
            xwr[sl][j][(s & 1) * 2 * NBC * NBR] = make_uint4(e[0], e[1], e[2], e[3]);
          }
        if constexpr (H7) {
          // image 7 (z, x+y): the micro-tile's RA + 1 diagonals (x - x0) +
          // (y - y0) = xl + yl + k, per slice and limb, into the step's row
#pragma unroll
          for (int sl = 0; sl < 2; ++sl)
#pragma unroll
            for (int l = 0; l < NL; ++l) {
              uint32_t* row = diag7 + (((s & 1) * 2 + sl) * NL + l) * DW + xl + yl;
              red_shared(row, v[sl][0][0][l]);
#pragma unroll
              for (int k = 1; k < RA; ++k) red_shared(row + k, v[sl][0][k][l] + v[sl][1][k - 1][l]);
              red_shared(row + RA, v[sl][1][RA - 1][l]);
            }
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) {
#pragma unroll
          for (int r = 0; r < BYA; ++r) {
            uint32_t a[RA], b[RA];
#pragma unroll
            for (int c = 0; c < RA; ++c) {
              a[c] = v[0][r][c][l];
              b[c] = v[1][r][c][l];
            }
            if constexpr (H3) {  // (x+z, y): slot k holds pixel xt + z + k
              uint32_t o0, o1;
              window_plus<GA, RA>(w3[r][l], a, b, tx, o0, o1);
              if (tx == 0) {  // leave the tile: pixels x0 + z, x0 + z + 1
                uint32_t* q = run3 + ((ty * BYA + r) * NL + l) * 16 + 2 * run_len;
                q[0] = o0;
                q[1] = o1;
              }
            }
            if constexpr (H4) {  // (x-z+N-1, y): slot k holds xt - 1 + k - z + N-1
              uint32_t o3, o4;
              window_minus<GA, RA>(w4[r][l], a, b, tx, o3, o4);
              if (tx == GA - 1) {  // leave the tile: pixels x0 + 62 - z + N-1 + {0, 1}
                uint32_t* q = run4 + ((ty * BYA + r) * NL + l) * 16 + 14 - 2 * run_len;
                q[0] = o3;
                q[1] = o4;
              }
            }
          }
        }
        // image 1 (z, y): row sums, reduced over the lane group
        {
          constexpr int NV = NL * 2 * BYA;
          uint32_t rs[NV];
#pragma unroll
          for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int sl = 0; sl < 2; ++sl)
#pragma unroll
              for (int r = 0; r < BYA; ++r) {
                uint32_t t = v[sl][r][0][l];
#pragma unroll
                for (int c = 1; c < RA; ++c) t += v[sl][r][c][l];
                rs[(l * 2 + sl) * BYA + r] = t;
              }
          int idx;
          uint32_t tot[Scatter<GA, NV>::NOUT];
          group_scatter_sum<GA, NV>(rs, tx, idx, tot);
          if ((tx & (Scatter<GA, NV>::REP - 1)) == 0) {
#pragma unroll
            for (int j = 0; j < Scatter<GA, NV>::NOUT; ++j) {
              const int r = (idx + j) % BYA, sl = ((idx + j) / BYA) & 1;
              const int y = yt + r, zz = z + sl;
              if (y < M && zz < zend && zz < N)
                red_add_always<FL>(p1[j] + (int64_t)z * M, tot[j], l2keep);
            }
          }
        }
        if (++run_len == 8) {
          flush_runs(yt, (int64_t)x0 + run_start, 0, 16, (int64_t)x0 + TXc - 16 - run_start + c4,
                     0, 16);
          run_start = z + 2;
          run_len = 0;
        }
        // step barrier (with group B); any failed wait aborts everyone
        __syncthreads();
        if (*abort_flag) {
          aborted = true;
          break;
        }
        if (tid == 0 && pc_u < ue) issue(st);
        ++s;
        ++u;
        z += 2;
      }
      if (aborted) break;
      __syncthreads();  // group B finishes the segment's last z-pair
      if constexpr (H7) merge_diag(diag7, 7, (s - 1) & 1, z - 2, x0, y0, tid);
      // segment end: exit runs and windows into the images
      flush_runs(yt, (int64_t)x0 + run_start, 0, 2 * run_len,
                 (int64_t)x0 + TXc - 16 - run_start + c4, 16 - 2 * run_len, 16);
      const int zn = z;  // the windows are laid out for the next z-pair
      const int xt = x0 + xl;
#pragma unroll
      for (int r = 0; r < BYA; ++r) {
        const int y = yt + r;
        if (y >= M) continue;
        // consecutive pixels: paired 64-bit reductions
#pragma unroll
        for (int l = 0; l < NL; ++l) {
          if constexpr (H3) {  // slot k: pixel f3 + k
            const int64_t f3 = (int64_t)xt + zn;
            const int64_t hi = set.F[3] - f3;
            red_add_run<RA, FL, FL>(pix(3, y, f3) + l * lstride, w3[r][l], 0,
                                    hi < RA ? (int)hi : RA, l2keep);
          }
          if constexpr (H4) {  // slot k + 1: pixel f4 + k
            const int64_t f4 = (int64_t)xt - zn + c4;
            const int64_t hi = set.F[4] - f4;
            red_add_run<RA, FL, FL>(pix(4, y, f4) + l * lstride, w4[r][l],
                                    f4 < 0 ? (int)-f4 : 0, hi < RA ? (int)hi : RA, l2keep);
          }
        }
      }
      clear_a();
    }
  } else {
    // ================= group B: images 0, 2, 5, 6 (lanes along y), one
    // z-pair behind group A: after the barrier of step s it takes step s's
    // voxels from the transposed buffer, which group A wrote before it
    const int bw = warp - NWG;
    uint32_t a0[RYB][BXB][NL];
    uint32_t w5[BXB][NL][RYB], w6[BXB][NL][RYB];
    auto clear_b = [&]() {
#pragma unroll
      for (int c = 0; c < BXB; ++c)
#pragma unroll
        for (int l = 0; l < NL; ++l) {
#pragma unroll
          for (int k = 0; k < RYB; ++k) { w5[c][l][k] = 0; w6[c][l][k] = 0; a0[k][c][l] = 0; }
        }
    };
    clear_b();
    // edge[buf][image 5 / 6][row k][limb][column]
    auto edge_at = [&](int buf, int im, int k, int l, int col) -> uint32_t* {
      return edge + ((((size_t)buf * 2 + im) * 2 + k) * NL + l) * TXc + col;
    };
    // the edge rows of the z-pair at z (tile x0, y0) into images 5 and 6:
    // images x 2 rows x NL limbs x TXc columns, shared out over the group's
    // warps (32 consecutive columns per warp and pass: coalesced)
    auto emit_edges = [&](int buf, int z, int x0, int y0) {
      constexpr int NIM = (H5 ? 1 : 0) + (H6 ? 1 : 0);
      constexpr int E = NIM * 2 * NL * TXc;
      constexpr int PER = (E + 32 * NWG - 1) / (32 * NWG);
#pragma unroll
      for (int j = 0; j < PER; ++j) {
        const int e = (j * NWG + bw) * 32 + lane;
        if (E % (32 * NWG) != 0 && e >= E) continue;
        const int col = e % TXc;
        const int l = (e / TXc) % NL;
        const int k = (e / (TXc * NL)) & 1;
        const int im = NIM == 2 ? e / (TXc * NL * 2) : (H5 ? 0 : 1);
        const int k5 = im == 0 ? 5 : 6;
        const int64_t sr = im == 0 ? (int64_t)y0 + z + k : (int64_t)y0 + TYc - 2 + k - z + c6;
        if (sr >= 0 && sr < set.S[k5] && x0 + col < L)
          red_add<FL>(pix(k5, sr, x0 + col) + l * lstride, *edge_at(buf, im, k, l, col), l2keep);
      }
    };
    // this lane's blocks of the transposed buffer (buffer 0) and of image 0
    const uint4* xrd[2][RYB / 2];
    uint4* a0p[RYB / 2];
#pragma unroll
    for (int bi = 0; bi < RYB / 2; ++bi) {
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) xrd[sl][bi] = xblk(0, sl, (RYB / 2) * gl + bi, cg);
      if constexpr (C::A0SMEM) {
        a0p[bi] = a0buf + (size_t)cg * NBR + block_pos((RYB / 2) * gl + bi, cg);
        *a0p[bi] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    while (u < ue && !aborted) {
      int x0, y0, za;
      decode(u, x0, y0, za);
      const int tile_units = p.nzp - (za - p.z0) / 2;
      const int nsteps = tile_units < (ue - u) ? tile_units : (ue - u);
      const int xt = x0 + xl, yt = y0 + yl;
      int z = za;
      // image 2 pixel (z, x) of this lane's total: base + z * L
      constexpr int NV2 = NL * 2 * BXB;
      uint32_t* p2[Scatter<GB, NV2>::NOUT];
      {
        const int i0 = scatter_index<GB, NV2>(gl);
#pragma unroll
        for (int j = 0; j < Scatter<GB, NV2>::NOUT; ++j) {
          const int idx = i0 + j;
          const int c = idx % BXB, sl = (idx / BXB) & 1, l = idx / (2 * BXB);
          p2[j] = img + set.base[2] + (int64_t)sl * set.F[2] + (xt + c) + l * lstride;
        }
      }
      for (int i = 0; i < nsteps; ++i) {
        const int buf = s & 1;
        // step barrier (with group A), which also publishes an abort
        __syncthreads();
        if (*abort_flag) {
          aborted = true;
          break;
        }
        // the previous z-pair's edge rows
        if ((H5 || H6) && i > 0) emit_edges(buf ^ 1, z - 2, x0, y0);
        if constexpr (H8) {
          if (i > 0) merge_diag(diag8, 8, buf ^ 1, z - 2, x0, y0, tid - 32 * NWG);
        }
        uint32_t v[2][RYB][BXB][NL];
#pragma unroll
        for (int sl = 0; sl < 2; ++sl)
#pragma unroll
          for (int bi = 0; bi < RYB / 2; ++bi) {
            const uint4 q = xrd[sl][bi][buf * 2 * NBC * NBR];
            const uint32_t e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int ri = 0; ri < 2; ++ri)
#pragma unroll
              for (int cj = 0; cj < BB; ++cj)
#pragma unroll
                for (int l = 0; l < NL; ++l) v[sl][2 * bi + ri][cj][l] = e[(ri * BB + cj) * NL + l];
          }
        if constexpr (H8) {
          // image 8 (z, x-y): the micro-tile's RYB + BXB - 1 diagonals
          // (x - x0) - (y - y0) + TYc - 1 = xl - yl - (RYB - 1) + TYc - 1 + k,
          // per slice and limb, into the step's row
#pragma unroll
          for (int sl = 0; sl < 2; ++sl)
#pragma unroll
            for (int l = 0; l < NL; ++l) {
              uint32_t dsum[RYB + BXB - 1];
#pragma unroll
              for (int k = 0; k < RYB + BXB - 1; ++k) dsum[k] = 0;
#pragma unroll
              for (int q = 0; q < RYB; ++q)
#pragma unroll
                for (int c = 0; c < BXB; ++c) dsum[c - q + RYB - 1] += v[sl][q][c][l];
              uint32_t* row = diag8 + ((buf * 2 + sl) * NL + l) * DW + xl - yl - (RYB - 1) + TYc - 1;
#pragma unroll
              for (int k = 0; k < RYB + BXB - 1; ++k) red_shared(row + k, dsum[k]);
            }
        }
#pragma unroll
        for (int c = 0; c < BXB; ++c)
#pragma unroll
          for (int l = 0; l < NL; ++l) {
            uint32_t a[RYB], b[RYB];
#pragma unroll
            for (int q = 0; q < RYB; ++q) {
              a[q] = v[0][q][c][l];
              b[q] = v[1][q][c][l];
              if constexpr (!C::A0SMEM) a0[q][c][l] += a[q] + b[q];  // image 0
            }
            if constexpr (H5) {  // (y+z, x): slot k holds row yt + z + k
              uint32_t o0, o1;
              window_plus<GB, RYB>(w5[c][l], a, b, gl, o0, o1);
              if (gl == 0) {  // leave the tile's top edge: rows y0 + z, y0 + z + 1
                *edge_at(buf, 0, 0, l, xl + c) = o0;
                *edge_at(buf, 0, 1, l, xl + c) = o1;
              }
            }
            if constexpr (H6) {  // (y-z+N-1, x): slot k holds row yt - 1 + k - z + N-1
              uint32_t o3, o4;
              window_minus<GB, RYB>(w6[c][l], a, b, gl, o3, o4);
              if (gl == GB - 1) {  // leave the bottom edge: rows y0 + TYc - 2 - z + N-1 + {0, 1}
                *edge_at(buf, 1, 0, l, xl + c) = o3;
                *edge_at(buf, 1, 1, l, xl + c) = o4;
              }
            }
          }
        if constexpr (C::A0SMEM) {  // image 0: the blocks' sums in shared memory
#pragma unroll
          for (int bi = 0; bi < RYB / 2; ++bi) {
            uint4 q = *a0p[bi];
            uint32_t e[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int ri = 0; ri < 2; ++ri)
#pragma unroll
              for (int cj = 0; cj < BB; ++cj)
#pragma unroll
                for (int l = 0; l < NL; ++l)
                  e[(ri * BB + cj) * NL + l] += v[0][2 * bi + ri][cj][l] + v[1][2 * bi + ri][cj][l];
            *a0p[bi] = make_uint4(e[0], e[1], e[2], e[3]);
          }
        }
        // image 2 (z, x): column sums, reduced over the lane group
        {
          constexpr int NV = NL * 2 * BXB;
          uint32_t cs[NV];
#pragma unroll
          for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int sl = 0; sl < 2; ++sl)
#pragma unroll
              for (int c = 0; c < BXB; ++c) {
                uint32_t t = v[sl][0][c][l];
#pragma unroll
                for (int q = 1; q < RYB; ++q) t += v[sl][q][c][l];
                cs[(l * 2 + sl) * BXB + c] = t;
              }
          int idx;
          uint32_t tot[Scatter<GB, NV>::NOUT];
          group_scatter_sum<GB, NV>(cs, gl, idx, tot);
          if ((gl & (Scatter<GB, NV>::REP - 1)) == 0) {
#pragma unroll
            for (int j = 0; j < Scatter<GB, NV>::NOUT; ++j) {
              const int c = (idx + j) % BXB, sl = ((idx + j) / BXB) & 1;
              const int x = xt + c, zz = z + sl;
              if (x < L && zz < zend && zz < N)
                red_add_always<FL>(p2[j] + (int64_t)z * L, tot[j], l2keep);
            }
          }
        }
        ++s;
        ++u;
        z += 2;
      }
      if (aborted) break;
      __syncthreads();  // matches group A's segment-end barrier: edge rows visible
      if (H5 || H6) emit_edges((s - 1) & 1, z - 2, x0, y0);
      if constexpr (H8) merge_diag(diag8, 8, (s - 1) & 1, z - 2, x0, y0, tid - 32 * NWG);
      // segment end: windows into the images
      const int zn = z;
      if constexpr (!FL && BXB == 2) {
        // the lane's two columns are neighbouring pixels of images 0, 5 and 6:
        // paired 64-bit reductions
        const bool in1 = xt + 1 < L;
        auto pair = [&](uint32_t* q, uint32_t a, uint32_t b) {
          if (in1 && (reinterpret_cast<uintptr_t>(q) & 7) == 0) {
            red_add_pair<false, FL>(q, a, b, l2keep);
          } else {
            red_add<FL>(q, a, l2keep);
            if (in1) red_add<FL>(q + 1, b, l2keep);
          }
        };
        if (xt < L) {
#pragma unroll
          for (int k = 0; k < RYB; ++k) {
            if (yt + k < M) {
              if constexpr (C::A0SMEM) {
                const uint32_t* e = reinterpret_cast<const uint32_t*>(a0p[k / 2]);
                pair(pix(0, yt + k, xt), e[(k & 1) * BB], e[(k & 1) * BB + 1]);
              } else {
                pair(pix(0, yt + k, xt), a0[k][0][0], a0[k][1][0]);
              }
            }
            if constexpr (H5) {  // slot k
              const int64_t sr = (int64_t)yt + zn + k;
              if (sr < set.S[5]) pair(pix(5, sr, xt), w5[0][0][k], w5[1][0][k]);
            }
            if constexpr (H6) {  // slot k + 1
              const int64_t sr = (int64_t)yt + k - zn + c6;
              if (sr >= 0 && sr < set.S[6]) pair(pix(6, sr, xt), w6[0][0][k], w6[1][0][k]);
            }
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < BXB; ++c) {
          const int x = xt + c;
          if (x >= L) continue;
#pragma unroll
          for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int k = 0; k < RYB; ++k) {
              if (yt + k < M) {
                if constexpr (C::A0SMEM) {
                  const uint32_t* e = reinterpret_cast<const uint32_t*>(a0p[k / 2]);
                  red_add<FL>(pix(0, yt + k, x) + l * lstride, e[((k & 1) * BB + c) * NL + l],
                          l2keep);
                } else {
                  red_add<FL>(pix(0, yt + k, x) + l * lstride, a0[k][c][l], l2keep);
                }
              }
              if constexpr (H5) {  // slot k
                const int64_t sr = (int64_t)yt + zn + k;
                if (sr < set.S[5]) red_add<FL>(pix(5, sr, x) + l * lstride, w5[c][l][k], l2keep);
              }
              if constexpr (H6) {  // slot k + 1
                const int64_t sr = (int64_t)yt + k - zn + c6;
                if (sr >= 0 && sr < set.S[6])
                  red_add<FL>(pix(6, sr, x) + l * lstride, w6[c][l][k], l2keep);
              }
            }
        }
      }
      clear_b();
      if constexpr (C::A0SMEM) {
#pragma unroll
        for (int bi = 0; bi < RYB / 2; ++bi) *a0p[bi] = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }

  if (aborted) {
    // let bulk copies still in flight land before the CTA's shared memory is
    // released (bounded; they were issued for units u .. pc_u - 1)
    if (tid == 0) {
      for (int ss = s; ss < s + (pc_u - u); ++ss)
        mbar_wait_bounded(smem_u32(&mbar[ss % STAGES]), (uint32_t)((ss / STAGES) & 1),
                          1ll << 31);
    }
    if (tid == 0 && p.status) atomicMax(p.status, kStatusTimeout);
  }
  if constexpr (FL) {
    // the range check of the quantisation grid
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) vmax = max_nan(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if (lane == 0 && !(vmax <= vcap)) atomicOr(p.flags, kFlagRange);
  }
}

// Tensor map of the volume (x fastest), box 64 x TYc x 2.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();  // defined in k1_int_dispatch.cu

template <typename T>
cudaError_t encode_map(CUtensorMap* map, const void* vol, int64_t L, int64_t M, int64_t N,
                       int box_x, int box_y, int box_z) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return cudaErrorNotSupported;
  const CUtensorMapDataType dt = std::is_same<T, float>::value
                                     ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                     : (sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT8);
  const cuuint64_t dims[3] = {(cuuint64_t)L, (cuuint64_t)M, (cuuint64_t)N};
  const cuuint64_t strides[2] = {(cuuint64_t)(L * (int64_t)sizeof(T)),
                                 (cuuint64_t)(L * M * (int64_t)sizeof(T))};
  const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_z};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = fn(map, dt, 3, const_cast<void*>(vol), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T, int P>
size_t smem_bytes() {
  using C = Cfg<T, P>;
  auto rnd = [](size_t b) { return (b + 127) & ~size_t(127); };
  size_t b = rnd(sizeof(uint64_t) * C::STAGES);
  b += rnd((size_t)C::STAGE * C::STAGES);
  b += 2 * rnd(sizeof(uint32_t) * (32 / C::GA) * C::NWG * C::BYA * C::NL * 16);
  b += rnd(sizeof(uint32_t) * 2 * 2 * 2 * C::NL * C::TXc);
  b += rnd(sizeof(uint4) * 2 * 2 * C::NBC * C::NBR);
  if (C::A0SMEM) b += rnd(sizeof(uint4) * C::NBC * C::NBR);
  if (C::H7) b += rnd(sizeof(uint32_t) * 2 * 2 * C::NL * C::DW);
  if (C::H8) b += rnd(sizeof(uint32_t) * 2 * 2 * C::NL * C::DW);
  b += rnd(sizeof(float) * 32);
  b += rnd(sizeof(int));
  return b;
}

// Launch of one element type and image count.  The caller guarantees
// 16-byte aligned rows and P <= 7.
template <typename T, int P>
cudaError_t launch(const IntProjectArgs& a, cudaStream_t st) {
  using C = Cfg<T, P>;
  Params p{};
  p.vol = a.vol;
  p.L = (int)a.L; p.M = (int)a.M; p.N = (int)a.N;
  p.z0 = (int)(a.nz > 0 ? a.z0 : 0);
  p.nz = (int)(a.nz > 0 ? a.nz : a.N);
  p.nxt = (int)((a.L + C::TXc - 1) / C::TXc);
  p.nyt = (int)((a.M + C::TYc - 1) / C::TYc);
  p.nzp = (p.nz + 1) / 2;
  const int64_t units = (int64_t)p.nxt * p.nyt * p.nzp;
  if (units >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  p.units = (int)units;
  p.set = a.set;
  p.limb_stride = a.set.total_elems;
  p.images = static_cast<uint32_t*>(a.images);
  p.status = a.status;
  p.flags = a.flags;
  p.sample = a.sample;
  p.nsample = a.nsample;
  p.limb_bits = a.limb_bits;
  p.scale_out = a.scale_out;
  p.wait_budget = a.wait_budget;

  const size_t smem = smem_bytes<T, P>();
  auto kern = k1_int_kernel<T, P>;
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
  // at least a few z-pairs per CTA so segment ends stay a small overhead:
  // 4, or 1 for volumes of at most 64 units, where latency rules (measured
  // K1: 64^3 u8 K=3 16.2 / 12.3 / 10.1 / 9.2 us at 8 / 4 / 2 / 1; 128^3 u16
  // K=6 21.7 / 16.9 / 18.7 us at 8 / 4 / 2; 128^3 f32 K=6 22.8 / 17.5 / 18.7
  // us; 256^3 and larger unchanged)
  const int64_t gmax = (int64_t)sms * per_sm;
  const int64_t W = (int64_t)p.nyt * p.nzp;
  const int64_t min_steps = units <= 64 ? 1 : 4;
  int64_t grid;
  if (p.nxt <= gmax) {  // nxt CTAs per (band, z-pair) range
    int64_t cpt = gmax / p.nxt;
    if (cpt > (W + min_steps - 1) / min_steps) cpt = (W + min_steps - 1) / min_steps;
    if (cpt < 1) cpt = 1;
    p.cpt = (int)cpt;
    grid = p.nxt * cpt;
  } else {
    p.cpt = 0;
    grid = gmax;
    const int64_t by_work = (units + min_steps - 1) / min_steps;
    if (grid > by_work) grid = by_work;
    if (grid < 1) grid = 1;
  }
  CUtensorMap vmap;
  std::memset(&vmap, 0, sizeof(vmap));
  e = encode_map<T>(&vmap, a.vol, a.L, a.M, a.N, C::TXc, C::TYc, 2);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)grid, C::NT, smem, st>>>(p, vmap);
  return cudaGetLastError();
}

}  // namespace k1i
}  // namespace dpma
