// Features derived from the raw moments: the post-step the paper describes
// after the combine (Sec. 4): the centroid (M100/M000, M010/M000, M001/M000),
// the central moments
//     mu_pqr = sum V (x - xbar)^p (y - ybar)^q (z - zbar)^r,
// the normalised central moments of Eq. 17,
//     eta_pqr = mu_pqr / mu_000^((p+q+r)/3 + 1),
// and the central moments in physical units for voxel spacings (a, b, c),
//     mu'_pqr = a^(1+p) b^(1+q) c^(1+r) mu_pqr.
//
// mu_pqr is the binomial expansion of (x - xbar)^p (y - ybar)^q (z - zbar)^r
// over the raw moments, whose terms cancel heavily (an odd central moment of
// a symmetric object is 0 while its terms are of the size of M_pqr).  Every
// step therefore runs in double-double arithmetic (about 106 significant
// bits) from the exact int128 moments, and only the results are rounded to
// double.  The double-double operations are the error-free TwoSum and the
// fused-multiply-add TwoProduct with Dekker's normalisation.
#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/dpma.h"
#include "dpma_internal.cuh"

namespace dpma {
void set_last_error(const char* msg);
}

using namespace dpma;

namespace {

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_norm(double s, double e) {  // |s| >= |e|
  const double h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const double s = a.hi + b.hi;
  const double bb = s - a.hi;
  const double e = (a.hi - (s - bb)) + (b.hi - bb);
  return dd_norm(s, e + a.lo + b.lo);
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const double p = a.hi * b.hi;
  const double e = fma(a.hi, b.hi, -p);
  return dd_norm(p, e + (a.hi * b.lo + a.lo * b.hi));
}
__device__ __forceinline__ dd dd_scale(dd a, double k) {  // k exact (a small integer)
  const double p = a.hi * k;
  const double e = fma(a.hi, k, -p);
  return dd_norm(p, e + a.lo * k);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
// a / b by long division: three quotient digits
__device__ dd dd_div(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  dd r = dd_add(a, dd_neg(dd_mul(b, {q1, 0.0})));
  const double q2 = r.hi / b.hi;
  r = dd_add(r, dd_neg(dd_mul(b, {q2, 0.0})));
  const double q3 = r.hi / b.hi;
  dd q = dd_norm(q1, q2);
  return dd_add(q, {q3, 0.0});
}
__device__ __forceinline__ dd dd_from_i128(i128 v) {
  const double hi = (double)v;
  const i128 rest = v - (i128)hi;  // |hi| < 2^126: exact
  return dd_norm(hi, (double)rest);
}

struct DerivedParams {
  const void* m;    // raw moments: int128 or double, graded order
  bool is_float;
  int K, nm;
  double sa, sb, sc;  // voxel spacings
  double* out;        // [centroid 3 | mu nm | eta nm | mu' nm]
};

__device__ __forceinline__ int idx3(int p, int q, int r) {
  const int n = p + q + r;
  // graded order: degree n, then p descending, then q descending
  const int before = n * (n + 1) * (n + 2) / 6;
  const int pp = n - p;  // rows with a larger p come first
  return before + pp * (pp + 1) / 2 + (n - p - q);
}

__device__ dd load_m(const DerivedParams& d, int i) {
  if (d.is_float) return {static_cast<const double*>(d.m)[i], 0.0};
  return dd_from_i128(static_cast<const i128*>(d.m)[i]);
}

__global__ void derived_kernel(DerivedParams d) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= d.nm) return;
  int n = 0;
  while ((n + 1) * (n + 2) * (n + 3) / 6 <= m) ++n;
  int row = m - n * (n + 1) * (n + 2) / 6;
  int p = n, q = 0;
  // row enumerates (p, q) with p descending, then q descending
  for (p = n; p >= 0; --p) {
    const int cnt = n - p + 1;
    if (row < cnt) { q = n - p - row; break; }
    row -= cnt;
  }
  const int r = n - p - q;
  const dd m000 = load_m(d, 0);
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (m000.hi == 0.0) {
    if (m == 0) d.out[0] = d.out[1] = d.out[2] = nan;
    d.out[3 + m] = nan;
    d.out[3 + d.nm + m] = nan;
    d.out[3 + 2 * d.nm + m] = nan;
    return;
  }
  dd c[3];
  c[0] = d.K >= 1 ? dd_div(load_m(d, 1), m000) : dd{0.0, 0.0};
  c[1] = d.K >= 1 ? dd_div(load_m(d, 2), m000) : dd{0.0, 0.0};
  c[2] = d.K >= 1 ? dd_div(load_m(d, 3), m000) : dd{0.0, 0.0};
  if (m == 0) {  // the centroid needs the first-degree moments
    for (int i = 0; i < 3; ++i) d.out[i] = d.K >= 1 ? c[i].hi + c[i].lo : nan;
  }
  // powers of -xbar, -ybar, -zbar
  dd px[kMaxK + 1], py[kMaxK + 1], pz[kMaxK + 1];
  px[0] = py[0] = pz[0] = {1.0, 0.0};
  for (int a = 1; a <= n; ++a) {
    px[a] = dd_mul(px[a - 1], dd_neg(c[0]));
    py[a] = dd_mul(py[a - 1], dd_neg(c[1]));
    pz[a] = dd_mul(pz[a - 1], dd_neg(c[2]));
  }
  // mu_pqr = sum_{i,j,k} C(p,i) C(q,j) C(r,k) (-xbar)^(p-i) (-ybar)^(q-j) (-zbar)^(r-k) M_ijk
  dd acc = {0.0, 0.0};
  double bi = 1.0;
  for (int i = 0; i <= p; ++i) {
    double bj = 1.0;
    for (int j = 0; j <= q; ++j) {
      double bk = 1.0;
      for (int k = 0; k <= r; ++k) {
        dd t = dd_mul(dd_mul(px[p - i], py[q - j]), pz[r - k]);
        t = dd_mul(t, load_m(d, idx3(i, j, k)));
        acc = dd_add(acc, dd_scale(t, bi * bj * bk));
        bk = bk * (r - k) / (k + 1);
      }
      bj = bj * (q - j) / (j + 1);
    }
    bi = bi * (p - i) / (i + 1);
  }
  const double mu = acc.hi + acc.lo;
  d.out[3 + m] = mu;
  // Eq. 17 (mu_000 = M_000)
  const double m0 = m000.hi + m000.lo;
  d.out[3 + d.nm + m] = mu / pow(m0, (double)n / 3.0 + 1.0);
  d.out[3 + 2 * d.nm + m] =
      mu * pow(d.sa, 1.0 + p) * pow(d.sb, 1.0 + q) * pow(d.sc, 1.0 + r);
}

}  // namespace

extern "C" dpma_status dpma_derived_moments(const void* moments, dpma_dtype dtype, int K,
                                            const double* spacing, double* out, void* stream) {
  if (!moments || !out) {
    set_last_error("null moments or output pointer");
    return DPMA_ERR_INVALID_ARG;
  }
  if (K < 0 || K > DPMA_MAX_K || (dtype != DPMA_U8 && dtype != DPMA_U16 && dtype != DPMA_F32)) {
    set_last_error("K must lie in 0..10 and dtype be a library dtype");
    return DPMA_ERR_INVALID_ARG;
  }
  DerivedParams d{};
  d.m = moments;
  d.is_float = dtype == DPMA_F32;
  d.K = K;
  d.nm = num_moments(K);
  d.sa = spacing ? spacing[0] : 1.0;
  d.sb = spacing ? spacing[1] : 1.0;
  d.sc = spacing ? spacing[2] : 1.0;
  if (!(d.sa > 0 && d.sb > 0 && d.sc > 0)) {
    set_last_error("spacings must be positive");
    return DPMA_ERR_INVALID_ARG;
  }
  d.out = out;
  const int threads = 64;
  derived_kernel<<<(d.nm + threads - 1) / threads, threads, 0, static_cast<cudaStream_t>(stream)>>>(d);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error((std::string("derived moments kernel: ") + cudaGetErrorString(e)).c_str());
    return DPMA_ERR_CUDA;
  }
  return DPMA_OK;
}
