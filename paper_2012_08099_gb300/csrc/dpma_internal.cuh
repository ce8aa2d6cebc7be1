// Internal declarations shared by the kernels and the C ABI of the Discrete
// Projection Moment library (Diggin & Diggin 2020, Sec. 3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "plan.h"

namespace dpma {

// A named range on the host timeline of a profiler (NVTX), for the scope of
// the object; costs a pointer test when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

using i128 = __int128;
using u128 = unsigned __int128;

// Geometry of the P images of one volume, packed for kernels.
struct ImageSet {
  int P;
  int64_t S[kMaxImages], F[kMaxImages];
  int64_t off_s[kMaxImages], off_f[kMaxImages];
  // pixel offset of image k inside the image buffer (uint32 pixels for
  // integer volumes, IEEE double pixels for float volumes)
  int64_t base[kMaxImages];
  int64_t total_elems;  // pixels of all images
};

inline ImageSet make_image_set(int64_t L, int64_t M, int64_t N, int K, bool /*is_float*/) {
  ImageSet s{};
  s.P = num_images(K);
  int64_t at = 0;
  for (int k = 0; k < s.P; ++k) {
    ImageGeom g;
    image_geom(k, L, M, N, &g);
    s.S[k] = g.S; s.F[k] = g.F; s.off_s[k] = g.off_s; s.off_f[k] = g.off_f;
    s.base[k] = at;
    at += g.S * g.F;
  }
  s.total_elems = at;
  return s;
}

// Signed Stirling numbers times factorials, (-1)^(b-j) S(b,j) j! for
// j <= b <= kMaxK (S: Stirling numbers of the second kind).  They turn the
// cascaded sums A_j = sum_w w^(j)/j! I (w^(j) the rising factorial) into the
// power sums sum_w w^b I = sum_j (-1)^(b-j) S(b,j) j! A_j.
struct StirlingTable {
  int64_t v[kMaxK + 1][kMaxK + 1];
};
constexpr StirlingTable make_stirling() {
  StirlingTable t{};
  int64_t S[kMaxK + 1][kMaxK + 1] = {};
  S[0][0] = 1;
  for (int b = 1; b <= kMaxK; ++b)
    for (int j = 1; j <= b; ++j) S[b][j] = j * S[b - 1][j] + S[b - 1][j - 1];
  for (int b = 0; b <= kMaxK; ++b) {
    int64_t fact = 1;
    for (int j = 0; j <= b; ++j) {
      if (j > 0) fact *= j;
      t.v[b][j] = ((b - j) & 1 ? -1 : 1) * S[b][j] * fact;
    }
  }
  return t;
}

// ---------------- float-float helpers (error-free transformations) ----------

// s + e == a + b exactly (Knuth's TwoSum, 6 flops, no ordering condition).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// p + e == a * b exactly (fused multiply-add based TwoProd).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// (hi, lo) += (bh, bl), renormalised.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// ---------------- kernel launchers (defined in the .cu files) ----------------

struct ProjectArgs {
  const void* vol;
  int64_t L, M, N;
  int dtype;  // 0 u8, 1 u16, 2 f32
  int K;
  void* images;
  ImageSet set;
  int* status;  // device status word for bounded-wait timeouts (may be null)
  // slices z0 .. z0 + nz - 1 only (nz = 0: the whole volume); the images
  // are accumulated, so launches over disjoint ranges add up to the volume
  int64_t z0 = 0, nz = 0;
  // fallback launches: the kernel does nothing unless (*gate & 3) != 0
  const int* gate = nullptr;
};

// Zeroes `bytes` (a multiple of 4) at `p` and, if non-null, the status word,
// in one launch: 16-byte stores when p is 16-byte aligned, 4-byte stores for
// the tail.  Falls back to cudaMemsetAsync for a misaligned p.
cudaError_t launch_clear(void* p, size_t bytes, int* status, cudaStream_t st,
                         const int* gate = nullptr);

// Step 1: images must be zeroed by the caller (the launcher does not clear).
// Orders 9 and 10 (integer volumes) add images 9 and 10 in a second kernel.
cudaError_t launch_project(const ProjectArgs& a, cudaStream_t st);
// Images 9 and 10 of an integer volume (nothing if a.set.P <= 9).
cudaError_t launch_project_extra(const ProjectArgs& a, cudaStream_t st);

// Step 1 on integer lanes (k1_int.cuh): uint32 images for integer volumes;
// for float32 volumes two sets of int32 images, one per quantisation limb
// (limb l of image k at base[k] + l * set.total_elems).
struct IntProjectArgs {
  const void* vol;
  int64_t L, M, N;
  int dtype;  // 0 u8, 1 u16, 2 f32
  void* images;
  ImageSet set;
  int* status;               // bounded-wait timeouts (may be null)
  int* flags;                // float volumes: |= 1 when a voxel leaves the grid
  const uint32_t* sample;    // float volumes: sampled |v| maxima (float bits)
  int nsample;
  int limb_bits;             // float volumes: B, |limb| <= 2^B
  int* scale_out;            // float volumes: receives e1 (may be null)
  long long wait_budget;     // cycles a bounded wait may spin
  int64_t z0 = 0, nz = 0;    // slices z0 .. z0 + nz - 1 (nz = 0: all; nz even unless it ends at N)
};
// Whether the integer-lane kernel takes this volume (16-byte aligned rows
// and at most 7 images).
bool project_int_supported(const void* vol, int64_t L, int dtype, int P);
cudaError_t launch_project_int(const IntProjectArgs& a, cudaStream_t st);
// Zeroes `bytes` at p (16-byte aligned, a multiple of 16), as many at p2
// (same rules; may be null), the status and flags words, and for float volumes (sample != null) writes into
// sample[0 .. nsample) the maxima of |v| over a sample of rows of slices
// z0 .. z0 + nz - 1: about 4096 rows spread over them, or, with row_stride
// > 0, exactly the rows 0, row_stride, 2 row_stride, ... (row r = z * M + y
// counted from slice z0).  Returns the sample length through *nsample.
cudaError_t launch_clear_sample(void* p, size_t bytes, int* status, int* flags, const float* vol,
                                int64_t L, int64_t M, int64_t z0, int64_t nz, uint32_t* sample,
                                int* nsample, cudaStream_t st, int64_t row_stride = 0,
                                void* p2 = nullptr, size_t bytes2 = 0, uint32_t even_fill = 0);
// The limb images of a float32 volume start with every pixel at an 8-byte
// aligned address (the low word of a pixel pair) at kLimbPairBias instead of
// 0; step 2 removes it.  With it the low word of a pair stays inside
// [0, 2^32) under any order of additions (|partial sums| < 2^30), so 32-bit
// reductions and paired 64-bit reductions of sign-extended sums can mix.
constexpr uint32_t kLimbPairBias = 0x80000000u;
constexpr int kMaxSample = 2048;  // sample slots

// Step 2 by the discrete Radon route (k2_drt.cu): integer images only.
size_t drt_workspace_bytes(int64_t L, int64_t M, int64_t N, int K);
cudaError_t launch_image_moments_drt(const void* images, int64_t L, int64_t M, int64_t N, int K,
                                     void* workspace, void* m2d, int* status, cudaStream_t st);
// Host: direction j of the 1-D integrals, and the exact solve of degree n
// (E row-major [b][j], (n+1) x (n+1); D[b]); false if unavailable.
int drt_direction(int j, int* alpha, int* beta);
bool drt_plan_degree(int n, int64_t* E, int64_t* D);

// Step 2: block partials of every image's 2-D moments into `partials`
// (int128 or float pairs), then a reduction into `m2d`.  For integer images
// whose `m2d` the caller has zeroed on the same stream (m2d_zeroed), each
// block adds its sums into `m2d` itself and the reduction launch is skipped.
size_t moments2d_partials_bytes(const ImageSet& set, int K, bool is_float);
cudaError_t launch_image_moments(const void* images, const ImageSet& set, int K, bool is_float,
                                 void* partials, void* m2d, cudaStream_t st,
                                 const int* gate = nullptr, bool m2d_zeroed = false);
// Step 2 on nl limb sets of int32 images (image i of the nl * P is image
// i % P of limb i / P, at base[i % P] + (i / P) * limb_stride); `m2d`
// receives nl * P rows of int128 moments.
constexpr int kMaxLimbImages = 2 * kMaxImages;
size_t moments2d_partials_bytes_limbs(const ImageSet& set, int K, int nl);
cudaError_t launch_image_moments_limbs(const void* images, const ImageSet& set, int64_t limb_stride,
                                       int K, int nl, void* partials, void* m2d, cudaStream_t st,
                                       bool m2d_zeroed = false);

// Step 3: combine into 3-D moments.
cudaError_t launch_combine(const void* m2d, int K, bool is_float, void* out, int* status,
                           cudaStream_t st, const int* gate = nullptr);
// Step 3 for the limb images of a float volume: exact combine of both limbs,
// the join of the limbs, the conversion to double and the guaranteed-error
// check (flags |= 2 when the quantisation error bound exceeds tol of a moment).
// scale[0] = e1 and scale[1] = B as the projection stored them.
cudaError_t launch_combine_fixed(const void* m2d, int K, int P, double* out, int* status,
                                 int* flags, const int* scale, int64_t L, int64_t M, int64_t N,
                                 double tol, cudaStream_t st);

// Bits B of the quantisation limbs of a float32 volume (|limb| <= 2^B):
// every line sum fits in int32 and every limb moment in int128; below
// kMinLimbBits the float volume takes the compensated float kernel.
int float_limb_bits(int64_t L, int64_t M, int64_t N, int K);
constexpr int kMinLimbBits = 12;

}  // namespace dpma
