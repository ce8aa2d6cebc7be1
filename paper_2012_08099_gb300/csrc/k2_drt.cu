// Step 2 by the discrete Radon route of Sec. 3.2: every projection image is
// summed once more, onto 1-D integrals along n+1 lattice directions, the
// 1-D moments of those integrals are taken, and the 2-D moments of degree n
// of the image follow from them by an exact rational solve.  Like the 3-D
// step above it, the 2-D identity is exact: for a direction (alpha, beta) and
// the signed image coordinates (s', f') of Eq. 1 with the origin shift of
// Sec. 5,
//
//   mu_n = sum_t t^n P(t),  P(t) = sum over the pixels with alpha f' + beta s' = t,
//        = sum_b C(n,b) alpha^b beta^(n-b) T_{n-b,b},   T_ab = sum I s'^a f'^b,
//
// so n+1 directions, pairwise non-proportional, determine the n+1 moments
// T_{n-b,b} of degree n.  The paper's five directions (columns, rows, the
// diagonal, the anti-diagonal and x + 2y) serve orders up to 4; six more
// extend the route to order 10.
//
// The solve is written in Lagrange form: with the binary forms
// L_j(X, Y) = prod_{i != j} (beta_i X - alpha_i Y) / d_j,
// d_j = prod_{i != j} (beta_i alpha_j - alpha_i beta_j), the degree-n form
// p(X, Y) = sum_b C(n,b) T_{n-b,b} X^b Y^(n-b) equals sum_j mu_j L_j(X, Y).
// Its coefficients give T_{n-b,b} = (sum_j E[b][j] mu_j) / D[b] with small
// integers E, D (below 2^27 at n = 10), which the host builds and checks
// exactly.
//
// Integer images only (the uint32 images of uint8/uint16 volumes).  The
// 1-D integrals are exact int64 sums (a pixel is below 2^32 and a line holds
// fewer than 2^17 of them); the 1-D moments and the solve run in exact
// 256-bit two's complement, and the division by D[b] is checked to leave no
// remainder (status 7 otherwise).  The result is bit-identical to the power
// sums of k2_moments.cu.
//
// Kernels: (1) drt_profile_kernel, one CTA per tile of 16 rows x 1024
// columns of one image, holds the tile's pixels in registers and, per
// direction, accumulates the tile's part of the integral in shared memory
// (64-bit shared atomics; the row direction by a lane-group sum) and adds it
// to the global integral; (2) drt_moment_kernel, one CTA per (image,
// direction), the 1-D moments t^n P(t) of n = 0..K in 256 bits; (3)
// drt_solve_kernel, one thread per 2-D moment.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <utility>

#include "../../include/dpma.h"
#include "dpma_internal.cuh"

namespace dpma {
namespace {

constexpr int kDirs = kMaxK + 1;
// (alpha, beta) of the integral t = alpha * f' + beta * s'.
constexpr int kDir[kDirs][2] = {{1, 0}, {0, 1}, {1, 1},  {1, -1}, {1, 2}, {2, 1},
                                {1, -2}, {2, -1}, {1, 3}, {3, 1}, {1, -3}};

constexpr int kTileRows = 16;     // rows of a profile tile
constexpr int kTileCols = 1024;   // columns of a profile tile
constexpr int kThreads = 256;
// widest tile part of one integral: |alpha| (cols - 1) + |beta| (rows - 1) + 1
constexpr int kSpanMax = 3 * (kTileCols - 1) + 3 * (kTileRows - 1) + 1;

struct DrtDegree {
  int64_t E[kDirs][kDirs];  // [b][j]
  int64_t D[kDirs];         // [b]
};
struct DrtPlan {
  DrtDegree deg[kMaxK + 1];
};

// Host: the exact solve of degree n over the first n+1 directions, reduced
// by the gcd of each row; false if the exact check fails.
bool build_drt_degree(int n, DrtDegree* out) {
  std::memset(out, 0, sizeof(*out));
  int64_t d[kDirs], N[kDirs][kDirs];
  for (int j = 0; j <= n; ++j) {
    int64_t poly[kDirs] = {1};  // coefficients of X^b
    int deg = 0;
    int64_t dj = 1;
    for (int i = 0; i <= n; ++i) {
      if (i == j) continue;
      const int64_t ai = kDir[i][0], bi = kDir[i][1];
      int64_t next[kDirs] = {0};
      for (int b = 0; b <= deg; ++b) {
        next[b] += -ai * poly[b];    // times -alpha_i Y
        next[b + 1] += bi * poly[b];  // times beta_i X
      }
      ++deg;
      std::memcpy(poly, next, sizeof(poly));
      dj *= bi * kDir[j][0] - ai * kDir[j][1];
    }
    if (dj == 0) return false;
    d[j] = dj;
    for (int b = 0; b <= n; ++b) N[j][b] = poly[b];
  }
  auto gcd = [](int64_t a, int64_t b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) { const int64_t t = a % b; a = b; b = t; }
    return a;
  };
  int64_t lam = 1;
  for (int j = 0; j <= n; ++j) {
    const int64_t a = d[j] < 0 ? -d[j] : d[j];
    lam = lam / gcd(lam, a) * a;
    if (lam > ((int64_t)1 << 40)) return false;
  }
  for (int b = 0; b <= n; ++b) {
    int64_t binom = 1;
    for (int i = 0; i < b; ++i) binom = binom * (n - i) / (i + 1);
    int64_t D = lam * binom, g = D;
    int64_t row[kDirs];
    for (int j = 0; j <= n; ++j) {
      const int64_t q = lam / (d[j] < 0 ? -d[j] : d[j]);
      row[j] = N[j][b] * (d[j] < 0 ? -q : q);
      g = gcd(g, row[j]);
    }
    for (int j = 0; j <= n; ++j) out->E[b][j] = row[j] / g;
    out->D[b] = D / g;
  }
  // exact check: sum_j E[b][j] C(n,b') alpha_j^b' beta_j^(n-b') = D[b] [b == b']
  for (int b = 0; b <= n; ++b)
    for (int bb = 0; bb <= n; ++bb) {
      i128 s = 0;
      int64_t binom = 1;
      for (int i = 0; i < bb; ++i) binom = binom * (n - i) / (i + 1);
      for (int j = 0; j <= n; ++j) {
        i128 a = binom;
        for (int e = 0; e < bb; ++e) a *= kDir[j][0];
        for (int e = 0; e < n - bb; ++e) a *= kDir[j][1];
        s += (i128)out->E[b][j] * a;
      }
      if (s != (b == bb ? (i128)out->D[b] : (i128)0)) return false;
    }
  return true;
}

const DrtPlan* drt_plan() {
  static DrtPlan plan;
  static int state = 0;  // 0 unbuilt, 1 ok, -1 failed
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (state == 0) {
    state = 1;
    for (int n = 0; n <= kMaxK; ++n)
      if (!build_drt_degree(n, &plan.deg[n])) state = -1;
  }
  return state == 1 ? &plan : nullptr;
}

// Geometry of the integral of image k along direction j: u = alpha f + beta s
// + c (u >= 0) over `len` entries; the signed coordinate is t = u + t0.
struct Integral {
  int64_t c, len, t0;
};
__host__ __device__ inline Integral integral_geom(int64_t S, int64_t F, int64_t off_s, int64_t off_f,
                                                  int a, int b) {
  Integral g;
  g.c = (a < 0 ? -(int64_t)a * (F - 1) : 0) + (b < 0 ? -(int64_t)b * (S - 1) : 0);
  g.len = (int64_t)(a < 0 ? -a : a) * (F - 1) + (int64_t)(b < 0 ? -b : b) * (S - 1) + 1;
  g.t0 = -g.c - (int64_t)a * off_f - (int64_t)b * off_s;
  return g;
}

struct DrtParams {
  const uint32_t* images;
  ImageSet set;
  int K, ndir, npairs;
  int dir[kDirs][2];                        // (alpha, beta) of each integral
  int64_t tile_base[kMaxImages + 1];        // first tile of each image
  int64_t prof_base[kMaxImages][kDirs];     // first entry of each integral
  unsigned long long* prof;                 // int64 entries (two's complement)
  uint64_t* mu;                             // [k][j][n] 256-bit moments, 4 words each
  void* m2d;                                // [k][npairs] int128
  int* status;
};

// ---------------- 256-bit helpers (two's complement, little-endian words)

struct W256 {
  uint64_t w[4];
};
__device__ __forceinline__ W256 w256_from_i64(int64_t v) {
  const uint64_t s = v < 0 ? ~0ull : 0ull;
  return W256{{(uint64_t)v, s, s, s}};
}
__device__ __forceinline__ void w256_add(W256& a, const W256& b) {
  uint64_t c = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t s = a.w[i] + b.w[i];
    const uint64_t c1 = s < a.w[i];
    const uint64_t r = s + c;
    const uint64_t c2 = r < s;
    a.w[i] = r;
    c = c1 | c2;
  }
}
__device__ __forceinline__ void w256_neg(W256& a) {
  uint64_t c = 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t v = ~a.w[i] + c;
    c = (c && v == 0) ? 1 : 0;
    a.w[i] = v;
  }
}
// a * m modulo 2^256 (exact while the product fits in 255 bits plus sign)
__device__ __forceinline__ W256 w256_mul_i64(W256 a, int64_t m) {
  const bool neg = m < 0;
  const uint64_t um = neg ? (uint64_t)0 - (uint64_t)m : (uint64_t)m;
  W256 r;
  uint64_t carry = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t lo = a.w[i] * um;
    const uint64_t hi = __umul64hi(a.w[i], um);
    const uint64_t s = lo + carry;
    carry = hi + (s < lo);
    r.w[i] = s;
  }
  if (neg) w256_neg(r);
  return r;
}
__device__ __forceinline__ W256 w256_shfl_xor(const W256& a, int m) {
  W256 r;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    r.w[i] = __shfl_xor_sync(0xffffffffu, (unsigned long long)a.w[i], m);
  return r;
}
// a / d exactly (d > 0); false on a remainder or a quotient outside int128.
__device__ bool w256_div_exact(W256 a, int64_t d, i128* q) {
  const bool neg = (a.w[3] >> 63) != 0;
  if (neg) w256_neg(a);
  uint64_t qw[4];
  u128 rem = 0;
  for (int i = 3; i >= 0; --i) {
    const u128 cur = (rem << 64) | a.w[i];
    qw[i] = (uint64_t)(cur / (uint64_t)d);
    rem = cur % (uint64_t)d;
  }
  if (rem != 0 || qw[3] != 0 || qw[2] != 0) return false;
  const u128 mag = ((u128)qw[1] << 64) | qw[0];
  if (!neg && (mag >> 127)) return false;
  if (neg && mag > ((u128)1 << 127)) return false;
  *q = neg ? (i128)(~mag + 1) : (i128)mag;
  return true;
}

// ---------------- kernels

__global__ void __launch_bounds__(kThreads) drt_profile_kernel(DrtParams p) {
  __shared__ unsigned long long acc[kSpanMax];
  const int tile = blockIdx.x;
  int k = 0;
  while (k + 1 < p.set.P && tile >= p.tile_base[k + 1]) ++k;
  const int64_t S = p.set.S[k], F = p.set.F[k];
  const int64_t ntc = (F + kTileCols - 1) / kTileCols;
  const int64_t rel = tile - p.tile_base[k];
  const int64_t s0 = (rel / ntc) * kTileRows, f0 = (rel % ntc) * kTileCols;
  const uint32_t* img = p.images + p.set.base[k];
  const int tid = threadIdx.x, r = tid >> 4, g = tid & 15;
  const int64_t s = s0 + r;
  // the thread's pixels: row s, columns f0 + 64 i + 4 g + q
  uint32_t px[16][4];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int64_t f = f0 + 64 * i + 4 * g;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      px[i][q] = (s < S && f + q < F) ? __ldg(img + s * F + f + q) : 0u;
  }
  for (int j = 0; j < p.ndir; ++j) {
    const int a = p.dir[j][0], b = p.dir[j][1];
    const Integral ig = integral_geom(S, F, p.set.off_s[k], p.set.off_f[k], a, b);
    const int span = (a < 0 ? -a : a) * (kTileCols - 1) + (b < 0 ? -b : b) * (kTileRows - 1) + 1;
    const int lc = (a < 0 ? -a * (kTileCols - 1) : 0) + (b < 0 ? -b * (kTileRows - 1) : 0);
    // global entry of local index e: e + ubase
    const int64_t ubase = (int64_t)a * f0 + (int64_t)b * s0 + ig.c - lc;
    unsigned long long* out = p.prof + p.prof_base[k][j];
    if (a == 0) {
      // the row integral: the 16 lanes of a row sum their pixels
      unsigned long long t = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) t += px[i][q];
#pragma unroll
      for (int m = 8; m >= 1; m >>= 1) t += __shfl_xor_sync(0xffffffffu, t, m);
      if (g == 0 && s < S && t) {
        const int64_t u = (int64_t)b * s + ig.c;
        atomicAdd(out + u, t);
      }
      continue;
    }
    for (int e = tid; e < span; e += kThreads) acc[e] = 0;
    __syncthreads();
    const int lrow = b * r + lc;
#pragma unroll
    for (int i = 0; i < 16; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (px[i][q]) atomicAdd(&acc[a * (64 * i + 4 * g + q) + lrow], (unsigned long long)px[i][q]);
    __syncthreads();
    for (int e = tid; e < span; e += kThreads) {
      const unsigned long long v = acc[e];
      if (v) atomicAdd(out + (ubase + e), v);
    }
    __syncthreads();
  }
}

template <int K>
__global__ void __launch_bounds__(kThreads) drt_moment_kernel(DrtParams p) {
  constexpr int NB = K + 1;
  const int k = blockIdx.x / p.ndir, j = blockIdx.x % p.ndir;
  const Integral ig = integral_geom(p.set.S[k], p.set.F[k], p.set.off_s[k], p.set.off_f[k],
                                    p.dir[j][0], p.dir[j][1]);
  const long long* prof = reinterpret_cast<const long long*>(p.prof + p.prof_base[k][j]);
  W256 acc[NB];
#pragma unroll
  for (int n = 0; n < NB; ++n) acc[n] = W256{{0, 0, 0, 0}};
  for (int64_t u = threadIdx.x; u < ig.len; u += kThreads) {
    const int64_t v = prof[u];
    if (v == 0) continue;
    const int64_t t = u + ig.t0;
    W256 pw = w256_from_i64(v);
#pragma unroll
    for (int n = 0; n < NB; ++n) {
      w256_add(acc[n], pw);
      if (n + 1 < NB) pw = w256_mul_i64(pw, t);
    }
  }
  __shared__ W256 part[kThreads / 32][NB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int n = 0; n < NB; ++n) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) w256_add(acc[n], w256_shfl_xor(acc[n], m));
    if (lane == 0) part[warp][n] = acc[n];
  }
  __syncthreads();
  if (threadIdx.x < NB) {
    const int n = threadIdx.x;
    W256 s = part[0][n];
    for (int w = 1; w < kThreads / 32; ++w) w256_add(s, part[w][n]);
    uint64_t* dst = p.mu + ((size_t)blockIdx.x * NB + n) * 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i] = s.w[i];
  }
}

__global__ void drt_solve_kernel(DrtParams p, DrtPlan plan) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= p.set.P * p.npairs) return;
  const int k = id / p.npairs, pair = id % p.npairs;
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= pair) ++n;
  const int bexp = pair - n * (n + 1) / 2;  // f exponent: T_{n-b, b} sits at n(n+1)/2 + b
  const DrtDegree& dg = plan.deg[n];
  W256 s{{0, 0, 0, 0}};
  for (int j = 0; j <= n; ++j) {
    const uint64_t* m = p.mu + (((size_t)k * p.ndir + j) * (p.K + 1) + n) * 4;
    W256 v{{m[0], m[1], m[2], m[3]}};
    w256_add(s, w256_mul_i64(v, dg.E[bexp][j]));
  }
  i128 q = 0;
  if (!w256_div_exact(s, dg.D[bexp], &q)) {
    if (p.status) atomicCAS(p.status, 0, 7);
    q = 0;
  }
  static_cast<i128*>(p.m2d)[(size_t)k * p.npairs + pair] = q;
}

using MomentKernel = void (*)(DrtParams);
template <int... Ks>
MomentKernel pick_moment_kernel(int K, std::integer_sequence<int, Ks...>) {
  MomentKernel r = nullptr;
  ((r = (K == Ks ? drt_moment_kernel<Ks> : r)), ...);
  return r;
}

struct DrtLayout {
  int64_t prof_base[kMaxImages][kDirs];
  int64_t prof_entries;
  size_t off_mu, total;
};

DrtLayout drt_layout(const ImageSet& set, int K) {
  DrtLayout w{};
  const int ndir = K + 1;
  int64_t at = 0;
  for (int k = 0; k < set.P; ++k)
    for (int j = 0; j < ndir; ++j) {
      w.prof_base[k][j] = at;
      at += integral_geom(set.S[k], set.F[k], set.off_s[k], set.off_f[k], kDir[j][0],
                          kDir[j][1]).len;
    }
  w.prof_entries = at;
  w.off_mu = ((size_t)at * 8 + 255) & ~size_t(255);
  w.total = w.off_mu + (size_t)set.P * ndir * (K + 1) * 32;
  return w;
}

}  // namespace

size_t drt_workspace_bytes(int64_t L, int64_t M, int64_t N, int K) {
  return drt_layout(make_image_set(L, M, N, K, false), K).total;
}

bool drt_plan_degree(int n, int64_t* E, int64_t* D) {
  const DrtPlan* pl = drt_plan();
  if (!pl || n < 0 || n > kMaxK) return false;
  for (int b = 0; b <= n; ++b) {
    if (D) D[b] = pl->deg[n].D[b];
    for (int j = 0; j <= n; ++j)
      if (E) E[b * (n + 1) + j] = pl->deg[n].E[b][j];
  }
  return true;
}

int drt_direction(int j, int* alpha, int* beta) {
  if (j < 0 || j >= kDirs) return 0;
  *alpha = kDir[j][0];
  *beta = kDir[j][1];
  return 1;
}

// The discrete Radon step 2 of integer images into m2d ([P][npairs] int128),
// workspace of drt_workspace_bytes, status (may be null) set to 7 on a
// remainder.
cudaError_t launch_image_moments_drt(const void* images, int64_t L, int64_t M, int64_t N, int K,
                                     void* workspace, void* m2d, int* status, cudaStream_t st) {
  const DrtPlan* plan = drt_plan();
  if (!plan) return cudaErrorInvalidValue;
  const ImageSet set = make_image_set(L, M, N, K, false);
  const DrtLayout w = drt_layout(set, K);
  DrtParams p{};
  p.images = static_cast<const uint32_t*>(images);
  p.set = set;
  p.K = K;
  p.ndir = K + 1;
  p.npairs = num_2d(K);
  std::memcpy(p.dir, kDir, sizeof(p.dir));
  int64_t tiles = 0;
  for (int k = 0; k < set.P; ++k) {
    p.tile_base[k] = tiles;
    tiles += ((set.S[k] + kTileRows - 1) / kTileRows) * ((set.F[k] + kTileCols - 1) / kTileCols);
  }
  p.tile_base[set.P] = tiles;
  std::memcpy(p.prof_base, w.prof_base, sizeof(p.prof_base));
  p.prof = static_cast<unsigned long long*>(workspace);
  p.mu = reinterpret_cast<uint64_t*>(static_cast<unsigned char*>(workspace) + w.off_mu);
  p.m2d = m2d;
  p.status = status;
  if (tiles >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(workspace, 0, (size_t)w.prof_entries * 8, st);
  if (e != cudaSuccess) return e;
  drt_profile_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  MomentKernel mk = pick_moment_kernel(K, std::make_integer_sequence<int, kMaxK + 1>{});
  if (!mk) return cudaErrorInvalidValue;
  mk<<<set.P * p.ndir, kThreads, 0, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nthr = set.P * p.npairs;
  drt_solve_kernel<<<(nthr + 127) / 128, 128, 0, st>>>(p, *plan);
  return cudaGetLastError();
}

}  // namespace dpma
