// Host-side plan of the Discrete Projection Moment method: image geometry,
// the exact combine matrices of the final step, and magnitude bounds.
#pragma once
#include <cstdint>
#include <cstddef>

namespace dpma {

// Single-volume pipeline: integer volumes up to order 10 (11 images: the
// axis and +-pi/4 families plus the arctan(1/2) and isometric images),
// float32 volumes up to order 8.
constexpr int kMaxK = 10;
constexpr int kMaxKFloat = 8;
constexpr int kMaxImages = 11;
constexpr int kMaxMono = 66;            // (10+1)(10+2)/2 monomials of degree 10
constexpr int kMax2D = 66;              // 2-D moments a+b <= 10 per image
// Batched launches, the server and the allocation-free entry: order <= 8.
constexpr int kMaxKBatch = 8;
constexpr int kMaxImagesBatch = 9;
constexpr int kMax2DBatch = 45;

// Linear forms of one projection image: the voxel (x,y,z) lands on row
// s = slow.(x,y,z) + off_s and column f = fast.(x,y,z) + off_f of an
// [S][F] row-major image (Sec. 3.1, Eq. 4; Eqs. 5-9, the +-pi/4 families and,
// for orders 9 and 10, the arctan(1/2) image about y and the isometric image).
struct ImageGeom {
  int slow[3];
  int fast[3];
  int64_t S, F, off_s, off_f;
};

int num_images(int K);
int num_moments(int K);
int num_2d(int K);                      // (K+1)(K+2)/2
bool image_geom(int k, int64_t L, int64_t M, int64_t N, ImageGeom* g);

// Index of the 2-D moment T_ab (a = slow exponent) in an image's moment
// vector: degree ascending, a descending.
inline int idx2d(int a, int b) { int n = a + b; return n * (n + 1) / 2 + (n - a); }
// Index of M_pqr in graded order: degree ascending, p descending, q descending.
int idx3d(int p, int q, int r);

// Combine of one degree n: M_n = (1/D) * C * t_sel, where t_sel[j] is the
// 2-D moment T_{a_j, n-a_j} of image img_j.  C is nmono x nmono, row-major;
// rows follow the graded order of the degree-n monomials.
struct DegreePlan {
  int n;
  int nmono;
  int64_t D;
  int img[kMaxMono];
  int a[kMaxMono];
  int64_t C[kMaxMono * kMaxMono];
};

struct CombinePlan {
  int K;
  int P;
  DegreePlan deg[kMaxK + 1];
};

// Builds (once, cached) and returns the plan for order K; nullptr if K is
// out of range or the exact verification fails.
const CombinePlan* combine_plan(int K);

// log2 of an upper bound on |T_ab| over all images and a+b <= K for a volume
// whose voxels are at most vmax in magnitude.
double log2_bound_2d(int64_t L, int64_t M, int64_t N, double vmax, int K);
// log2 of an upper bound on |M_pqr| for p+q+r <= K.
double log2_bound_3d(int64_t L, int64_t M, int64_t N, double vmax, int K);

}  // namespace dpma
