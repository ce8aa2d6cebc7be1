// Multithreaded CPU implementation of the Discrete Projection Moment method.
//
// The chain of Sec. 3, as the paper runs it on a CPU:
//   1. one pass over the volume adds every voxel into each projection image
//      (Sec. 3.1, Eq. 4 and the rotated projections that follow it): the
//      threads take slabs of z and accumulate private images, which are
//      then added together;
//   2. every image is collapsed into 1-D integrals along K + 1 directions
//      (the discrete Radon transform route to 2-D moments of Sec. 3.2 and
//      Sec. 4, additions only), and the power moments of those 1-D integrals
//      give the image's 2-D moments by a small linear solve per degree;
//   3. the 2-D moments of all images give the 3-D raw moments M_pqr of
//      Eq. 2 by one more linear solve per degree (the relations of
//      Eqs. 10-16, generalised: each 2-D moment of an image is a fixed
//      integer combination of 3-D moments of the same degree).
//
// Exactness.  Voxel, pixel and 1-D integral sums are exact 64-bit integer
// sums.  A float32 volume is first rounded onto the grid 2^-e (e chosen from
// its largest magnitude so that no sum can leave the int64 range), which is
// the only rounding of the float pipeline before the final conversion.
// Everything after the 1-D integrals runs modulo three primes just below
// 2^62; the moments, which are integers on that grid, come back from their
// residues by the Chinese remainder theorem in Garner's mixed-radix form.
//
// The image set is chosen per order: the three axis projections, then
// rotated projections (+-pi/4 about each axis, then +-arctan(1/2) and
// +-arctan 2 about each axis) added one at a time while they raise the rank
// of some degree's system, until every degree up to K has full rank.
#include "cpu_dpma.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace {

using u64 = uint64_t;
using i64 = int64_t;
using u128 = unsigned __int128;
using i128 = __int128;

constexpr int kMaxOrder = 12;

// ------------------------------------------------------------ modular

u64 mul_mod(u64 a, u64 b, u64 p) { return (u64)((u128)a * b % p); }

u64 pow_mod(u64 a, u64 e, u64 p) {
  u64 r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mul_mod(r, a, p);
    a = mul_mod(a, a, p);
    e >>= 1;
  }
  return r;
}

u64 inv_mod(u64 a, u64 p) { return pow_mod(a, p - 2, p); }  // p prime, a != 0

u64 to_mod(i64 v, u64 p) {
  const i64 r = v % (i64)p;
  return (u64)(r < 0 ? r + (i64)p : r);
}

// Miller-Rabin; these twelve bases decide every 64-bit integer.
bool is_prime(u64 n) {
  if (n < 2) return false;
  static const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (u64 q : small)
    if (n % q == 0) return n == q;
  u64 d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (u64 a : small) {
    u64 x = pow_mod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < s; ++i) {
      x = mul_mod(x, x, n);
      if (x == n - 1) { comp = false; break; }
    }
    if (comp) return false;
  }
  return true;
}

struct Primes {
  u64 p[3];
  u64 inv01;   // p0^-1 mod p1
  u64 inv012;  // (p0 p1)^-1 mod p2
};

const Primes& primes() {
  static Primes P = [] {
    Primes q{};
    u64 c = ((u64)1 << 62) - 1;
    for (int i = 0; i < 3; ++i) {
      while (!is_prime(c)) c -= 2;
      q.p[i] = c;
      c -= 2;
    }
    q.inv01 = inv_mod(q.p[0] % q.p[1], q.p[1]);
    q.inv012 = inv_mod(mul_mod(q.p[0] % q.p[2], q.p[1] % q.p[2], q.p[2]), q.p[2]);
    return q;
  }();
  return P;
}

// Solve the consistent system A u = b (mod p) for u, A with `rows` rows and
// `cols` columns of full column rank (row-major, augmented in place as
// [A | b]).  Returns false if the rank is short.
bool solve_mod(std::vector<u64>& Ab, int rows, int cols, u64 p, u64* u) {
  const int w = cols + 1;
  int r = 0;
  std::vector<int> piv(cols, -1);
  for (int c = 0; c < cols && r < rows; ++c) {
    int sel = -1;
    for (int i = r; i < rows; ++i)
      if (Ab[(size_t)i * w + c]) { sel = i; break; }
    if (sel < 0) return false;
    if (sel != r)
      for (int j = 0; j < w; ++j) std::swap(Ab[(size_t)sel * w + j], Ab[(size_t)r * w + j]);
    const u64 iv = inv_mod(Ab[(size_t)r * w + c], p);
    for (int j = 0; j < w; ++j) Ab[(size_t)r * w + j] = mul_mod(Ab[(size_t)r * w + j], iv, p);
    for (int i = 0; i < rows; ++i) {
      if (i == r) continue;
      const u64 f = Ab[(size_t)i * w + c];
      if (!f) continue;
      for (int j = 0; j < w; ++j) {
        const u64 t = mul_mod(f, Ab[(size_t)r * w + j], p);
        u64& x = Ab[(size_t)i * w + j];
        x = x >= t ? x - t : x + p - t;
      }
    }
    piv[c] = r++;
  }
  for (int c = 0; c < cols; ++c) u[c] = Ab[(size_t)piv[c] * w + cols];
  return true;
}

// Rank of a matrix mod p (row-major, rows x cols).
int rank_mod(std::vector<u64> A, int rows, int cols, u64 p) {
  int r = 0;
  for (int c = 0; c < cols && r < rows; ++c) {
    int sel = -1;
    for (int i = r; i < rows; ++i)
      if (A[(size_t)i * cols + c]) { sel = i; break; }
    if (sel < 0) continue;
    if (sel != r)
      for (int j = 0; j < cols; ++j) std::swap(A[(size_t)sel * cols + j], A[(size_t)r * cols + j]);
    const u64 iv = inv_mod(A[(size_t)r * cols + c], p);
    for (int i = r + 1; i < rows; ++i) {
      const u64 f = mul_mod(A[(size_t)i * cols + c], iv, p);
      if (!f) continue;
      for (int j = c; j < cols; ++j) {
        const u64 t = mul_mod(f, A[(size_t)r * cols + j], p);
        u64& x = A[(size_t)i * cols + j];
        x = x >= t ? x - t : x + p - t;
      }
    }
    ++r;
  }
  return r;
}

// ------------------------------------------------------------ geometry

// A linear form c . (x, y, z) with small integer coefficients.
struct Form {
  int cx, cy, cz;
};

// A projection image: the pixel of voxel (x, y, z) is (s, t) = (S . v, T . v);
// the image sums the voxels along the direction orthogonal to both forms.
struct Image {
  Form s, t;
};

// Candidates in the order they are tried (s carries the x term whenever
// one of the two forms has one, so that a row of voxels walks along s).
const Image kCandidates[] = {
    {{1, 0, 0}, {0, 1, 0}},   // along z: (x, y)
    {{0, 1, 0}, {0, 0, 1}},   // along x: (y, z)
    {{1, 0, 0}, {0, 0, 1}},   // along y: (x, z)
    {{1, 0, 1}, {0, 1, 0}},   // +pi/4 about y: (x + z, y)
    {{1, 0, -1}, {0, 1, 0}},  // -pi/4 about y: (x - z, y)
    {{1, 1, 0}, {0, 0, 1}},   // +pi/4 about z: (x + y, z)
    {{1, -1, 0}, {0, 0, 1}},  // -pi/4 about z: (x - y, z)
    {{1, 0, 0}, {0, 1, 1}},   // +pi/4 about x: (x, y + z)
    {{1, 0, 0}, {0, 1, -1}},  // -pi/4 about x: (x, y - z)
    {{1, 0, 2}, {0, 1, 0}},   // arctan(1/2), arctan 2 about y
    {{1, 0, -2}, {0, 1, 0}},
    {{2, 0, 1}, {0, 1, 0}},
    {{2, 0, -1}, {0, 1, 0}},
    {{1, 2, 0}, {0, 0, 1}},   // ... about z
    {{1, -2, 0}, {0, 0, 1}},
    {{2, 1, 0}, {0, 0, 1}},
    {{2, -1, 0}, {0, 0, 1}},
    {{1, 0, 0}, {0, 1, 2}},   // ... about x
    {{1, 0, 0}, {0, 1, -2}},
    {{1, 0, 0}, {0, 2, 1}},
    {{1, 0, 0}, {0, 2, -1}},
};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

// Directions (a, b) of the 1-D integrals of an image: u = a s + b t.  Any
// n + 1 of them with distinct ratios a : b resolve the degree-n moments.
const int kDirections[][2] = {{1, 0}, {0, 1}, {1, 1}, {1, -1}, {1, 2}, {2, 1}, {1, -2},
                              {2, -1}, {1, 3}, {3, 1}, {1, -3}, {3, -1}, {2, 3}};
static_assert(sizeof(kDirections) / sizeof(kDirections[0]) >= kMaxOrder + 1, "directions");

int num_monos(int n) { return (n + 1) * (n + 2) / 2; }

// position of x^p y^q z^(n-p-q) among the degree-n monomials (p descending,
// then q descending)
int mono_pos(int n, int p, int q) {
  int pos = 0;
  for (int pp = n; pp > p; --pp) pos += n - pp + 1;
  return pos + (n - p - q);
}

// Exact integer coefficients of the degree-n monomials in s^i t^(n-i):
// out[mono_pos(n, p, q)].
void expand(const Image& im, int i, int n, std::vector<i64>& out) {
  // dense (n+1)^3 polynomial, multiplied factor by factor
  const int D = n + 1;
  std::vector<i64> a((size_t)D * D * D, 0), b;
  a[0] = 1;
  int deg = 0;
  for (int f = 0; f < n; ++f) {
    const Form& F = f < i ? im.s : im.t;
    b.assign(a.size(), 0);
    for (int x = 0; x <= deg; ++x)
      for (int y = 0; x + y <= deg; ++y) {
        const int z = deg - x - y;
        const i64 c = a[((size_t)x * D + y) * D + z];
        if (!c) continue;
        b[((size_t)(x + 1) * D + y) * D + z] += c * F.cx;
        b[((size_t)x * D + y + 1) * D + z] += c * F.cy;
        b[((size_t)x * D + y) * D + z + 1] += c * F.cz;
      }
    a.swap(b);
    ++deg;
  }
  out.assign(num_monos(n), 0);
  for (int p = 0; p <= n; ++p)
    for (int q = 0; p + q <= n; ++q) out[mono_pos(n, p, q)] = a[((size_t)p * D + q) * D + (n - p - q)];
}

// Rows of degree n contributed by image im (n + 1 of them), mod p.
void image_rows(const Image& im, int n, u64 p, std::vector<u64>& rows) {
  std::vector<i64> c;
  for (int i = n; i >= 0; --i) {
    expand(im, i, n, c);
    for (i64 v : c) rows.push_back(to_mod(v, p));
  }
}

struct Plan {
  bool ok = false;
  std::vector<Image> images;
};

Plan build_plan(int K) {
  Plan pl;
  const u64 p = primes().p[0];
  std::vector<int> rank(K + 1, 0);
  for (int c = 0; c < kNumCandidates; ++c) {
    bool full = true;
    for (int n = 0; n <= K; ++n) full = full && rank[n] == num_monos(n);
    if (full) break;
    std::vector<Image> trial = pl.images;
    trial.push_back(kCandidates[c]);
    bool gain = false;
    std::vector<int> nr(K + 1);
    for (int n = 0; n <= K; ++n) {
      std::vector<u64> A;
      for (const Image& im : trial) image_rows(im, n, p, A);
      nr[n] = rank_mod(A, (int)trial.size() * (n + 1), num_monos(n), p);
      gain = gain || nr[n] > rank[n];
    }
    // the three axis images are always taken
    if (gain || c < 3) {
      pl.images = trial;
      rank = nr;
    }
  }
  pl.ok = true;
  for (int n = 0; n <= K; ++n) pl.ok = pl.ok && rank[n] == num_monos(n);
  return pl;
}

const Plan& plan_for(int K) {
  static std::mutex mu;
  static Plan plans[kMaxOrder + 1];
  static bool built[kMaxOrder + 1] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (!built[K]) {
    plans[K] = build_plan(K);
    built[K] = true;
  }
  return plans[K];
}

// extent of a form over the box [0, L) x [0, M) x [0, N)
void form_range(const Form& f, i64 L, i64 M, i64 N, i64* lo, i64* hi) {
  const i64 d[3] = {L - 1, M - 1, N - 1};
  const int c[3] = {f.cx, f.cy, f.cz};
  *lo = *hi = 0;
  for (int k = 0; k < 3; ++k) {
    if (c[k] > 0) *hi += c[k] * d[k];
    else *lo += c[k] * d[k];
  }
}

struct ImgGeom {
  Image im;
  i64 smin, tmin, S, T;  // pixel (s, t) at [(t - tmin) * S + (s - smin)]
  i64 stride;            // pixel step for x -> x + 1
  size_t offset;         // of this image in the image block
};

std::vector<ImgGeom> geometry(const Plan& pl, i64 L, i64 M, i64 N, size_t* total) {
  std::vector<ImgGeom> g;
  size_t off = 0;
  for (const Image& im : pl.images) {
    ImgGeom x{};
    x.im = im;
    i64 smax, tmax;
    form_range(im.s, L, M, N, &x.smin, &smax);
    form_range(im.t, L, M, N, &x.tmin, &tmax);
    x.S = smax - x.smin + 1;
    x.T = tmax - x.tmin + 1;
    x.stride = im.s.cx + (i64)im.t.cx * x.S;
    x.offset = off;
    off += (size_t)(x.S * x.T);
    g.push_back(x);
  }
  *total = off;
  return g;
}

// ------------------------------------------------------------ step 1

// Voxel rows [r0, r1) (row r = z * M + y) added into the images at `img`.
template <typename T>
void project_rows(const T* vol, i64 L, i64 M, i64 r0, i64 r1, const std::vector<ImgGeom>& g,
                  i64* img, double scale) {
  std::vector<i64> q((size_t)L);
  for (i64 r = r0; r < r1; ++r) {
    const i64 z = r / M, y = r - z * M;
    const T* row = vol + (size_t)r * L;
    if constexpr (sizeof(T) == 4) {
      for (i64 x = 0; x < L; ++x) q[x] = (i64)std::nearbyint((double)row[x] * scale);
    } else {
      for (i64 x = 0; x < L; ++x) q[x] = (i64)row[x];
    }
    bool have_sum = false;
    i64 sum = 0;
    for (const ImgGeom& G : g) {
      const i64 s0 = (i64)G.im.s.cy * y + (i64)G.im.s.cz * z - G.smin;
      const i64 t0 = (i64)G.im.t.cy * y + (i64)G.im.t.cz * z - G.tmin;
      i64* base = img + G.offset + t0 * G.S + s0;
      if (G.stride == 0) {
        if (!have_sum) {
          for (i64 x = 0; x < L; ++x) sum += q[x];
          have_sum = true;
        }
        base[0] += sum;
      } else if (G.stride == 1) {
        for (i64 x = 0; x < L; ++x) base[x] += q[x];
      } else {
        const i64 st = G.stride;
        for (i64 x = 0; x < L; ++x) base[x * st] += q[x];
      }
    }
  }
}

template <typename F>
void parallel_for(int threads, i64 n, F&& f) {
  if (threads <= 1 || n <= 1) {
    f(0, (i64)0, n);
    return;
  }
  std::vector<std::thread> pool;
  const i64 T = std::min<i64>(threads, n);
  for (i64 t = 0; t < T; ++t) {
    const i64 a = n * t / T, b = n * (t + 1) / T;
    pool.emplace_back([&f, t, a, b] { f((int)t, a, b); });
  }
  for (auto& th : pool) th.join();
}

// ------------------------------------------------------------ step 2

// Residues of the 2-D moments of one image, for every prime: m[prime][n]
// holds the n + 1 moments of degree n, s-power descending.
struct ImageMoments {
  std::vector<u64> m[3][kMaxOrder + 1];
};

// The 1-D integral of image G along direction (a, b) and its power moments
// mu[prime][n] = sum_u g(u) u^n, n <= K.
void radon_moments(const i64* I, const ImgGeom& G, int a, int b, int K, u64 mu[3][kMaxOrder + 1]) {
  const i64 smax = G.smin + G.S - 1, tmax = G.tmin + G.T - 1;
  const i64 c[4] = {a * G.smin + b * G.tmin, a * G.smin + b * tmax, a * smax + b * G.tmin,
                    a * smax + b * tmax};
  const i64 umin = *std::min_element(c, c + 4), umax = *std::max_element(c, c + 4);
  std::vector<i64> g((size_t)(umax - umin + 1), 0);
  for (i64 t = 0; t < G.T; ++t) {
    const i64* row = I + G.offset + t * G.S;
    i64* dst = g.data() + (a * G.smin + b * (G.tmin + t) - umin);
    if (a == 1) {
      for (i64 s = 0; s < G.S; ++s) dst[s] += row[s];
    } else if (a == 0) {
      i64 sum = 0;
      for (i64 s = 0; s < G.S; ++s) sum += row[s];
      dst[0] += sum;
    } else {
      for (i64 s = 0; s < G.S; ++s) dst[s * a] += row[s];
    }
  }
  const Primes& P = primes();
  for (int k = 0; k < 3; ++k) {
    const u64 p = P.p[k];
    for (int n = 0; n <= K; ++n) mu[k][n] = 0;
    for (size_t j = 0; j < g.size(); ++j) {
      if (!g[j]) continue;
      const u64 um = to_mod(umin + (i64)j, p);
      u64 w = to_mod(g[j], p);
      for (int n = 0; n <= K; ++n) {
        mu[k][n] += w;
        if (mu[k][n] >= p) mu[k][n] -= p;
        w = mul_mod(w, um, p);
      }
    }
  }
}

u64 binom_mod(int n, int k, u64 p) {
  u64 r = 1;
  for (int i = 1; i <= k; ++i) r = r * (u64)(n - k + i) / (u64)i;  // exact, small n
  return r % p;
}

u64 pow_small(int a, int e, u64 p) {
  u64 r = 1 % p;
  const u64 am = to_mod(a, p);
  for (int i = 0; i < e; ++i) r = mul_mod(r, am, p);
  return r;
}

// The 2-D moments of degree n from the 1-D moments of directions 0..n:
// mu_n(a, b) = sum_i C(n, i) a^i b^(n-i) m_{i, n-i}.
bool moments_2d(const u64 mu[kMaxOrder + 1][3][kMaxOrder + 1], int n, int k, u64 p,
                std::vector<u64>& out) {
  const int w = n + 2;
  std::vector<u64> Ab((size_t)(n + 1) * w);
  for (int j = 0; j <= n; ++j) {
    const int a = kDirections[j][0], b = kDirections[j][1];
    for (int c = 0; c <= n; ++c) {
      const int i = n - c;  // column c holds m_{i, n-i}, i descending
      Ab[(size_t)j * w + c] = mul_mod(binom_mod(n, i, p),
                                      mul_mod(pow_small(a, i, p), pow_small(b, n - i, p), p), p);
    }
    Ab[(size_t)j * w + n + 1] = mu[j][k][n];
  }
  out.assign(n + 1, 0);
  return solve_mod(Ab, n + 1, n + 1, p, out.data());
}

// ------------------------------------------------------------ CRT

struct Mixed {
  u64 d0, d1, d2;  // value = d0 + p0 d1 + p0 p1 d2, in [0, p0 p1 p2)
};

Mixed garner(const u64 r[3]) {
  const Primes& P = primes();
  Mixed m;
  m.d0 = r[0];
  const u64 a1 = (r[1] + P.p[1] - m.d0 % P.p[1]) % P.p[1];
  m.d1 = mul_mod(a1, P.inv01, P.p[1]);
  u64 a2 = (r[2] + P.p[2] - m.d0 % P.p[2]) % P.p[2];
  const u64 t = mul_mod(P.p[0] % P.p[2], m.d1, P.p[2]);
  a2 = (a2 + P.p[2] - t) % P.p[2];
  m.d2 = mul_mod(a2, P.inv012, P.p[2]);
  return m;
}

// Values in the upper half of the range are negative (the magnitudes in
// play are far below p0 p1 p2 / 2 ~ 2^185).
bool is_negative(const Mixed& m) { return m.d2 > primes().p[2] / 2; }

// |value| as mixed-radix digits
Mixed magnitude(const Mixed& m) {
  if (!is_negative(m)) return m;
  const Primes& P = primes();
  // P - x = (P - 1 - x) + 1, digit by digit, then the +1 with carries
  Mixed r{P.p[0] - 1 - m.d0, P.p[1] - 1 - m.d1, P.p[2] - 1 - m.d2};
  if (++r.d0 == P.p[0]) {
    r.d0 = 0;
    if (++r.d1 == P.p[1]) { r.d1 = 0; ++r.d2; }
  }
  return r;
}

bool to_i128(const Mixed& m, i128* out) {
  const Primes& P = primes();
  const Mixed a = magnitude(m);
  const u128 p01 = (u128)P.p[0] * P.p[1];
  const u128 lim = ((u128)1 << 127) - 1;
  if (a.d2 > 7) return false;
  u128 v = p01 * a.d2;
  const u128 mid = (u128)P.p[0] * a.d1 + a.d0;
  if (v > lim - mid) return false;
  v += mid;
  *out = is_negative(m) ? -(i128)v : (i128)v;
  return true;
}

double to_double(const Mixed& m) {
  const Primes& P = primes();
  const Mixed a = magnitude(m);
  const double v = (double)a.d0 + (double)P.p[0] * ((double)a.d1 + (double)P.p[1] * (double)a.d2);
  return is_negative(m) ? -v : v;
}

thread_local int g_last_e = 0;

}  // namespace

extern "C" int cpu_dpma_max_order(void) { return kMaxOrder; }

extern "C" int cpu_dpma_num_images(int K) {
  if (K < 0 || K > kMaxOrder) return 0;
  const Plan& pl = plan_for(K);
  return pl.ok ? (int)pl.images.size() : 0;
}

extern "C" int cpu_dpma_last_float_exponent(void) { return g_last_e; }

extern "C" int cpu_dpma_moments(const void* vol, int64_t L, int64_t M, int64_t N, int dtype, int K,
                                int threads, void* out, int* threads_used) {
  if (!vol || !out || L <= 0 || M <= 0 || N <= 0 || K < 0 || K > kMaxOrder || dtype < 0 ||
      dtype > 2)
    return 1;
  const Plan& pl = plan_for(K);
  if (!pl.ok) return 4;
  int T = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (T < 1) T = 1;
  const i64 rows = M * N;
  if (T > rows) T = (int)rows;
  size_t total = 0;
  const std::vector<ImgGeom> geo = geometry(pl, L, M, N, &total);
  // private images per thread, at most ~8 GB in all
  const size_t cap = ((size_t)8 << 30) / (total * sizeof(i64) + 1);
  if ((size_t)T > cap) T = (int)std::max<size_t>(1, cap);
  if (threads_used) *threads_used = T;

  // float32: the quantisation grid 2^-e from the largest magnitude
  double scale = 1.0;
  int e = 0;
  if (dtype == 2) {
    const float* f = static_cast<const float*>(vol);
    const i64 nvox = L * M * N;
    std::vector<float> part(T, 0.f);
    std::vector<int> bad(T, 0);
    parallel_for(T, nvox, [&](int t, i64 a, i64 b) {
      float m = 0.f;
      int nf = 0;
      for (i64 i = a; i < b; ++i) {
        const float v = std::fabs(f[i]);
        if (!(v <= 3.4028235e38f)) nf = 1;  // NaN or infinite
        else if (v > m) m = v;
      }
      part[t] = m;
      bad[t] = nf;
    });
    float vmax = 0.f;
    for (int t = 0; t < T; ++t) {
      if (bad[t]) return 2;
      vmax = std::max(vmax, part[t]);
    }
    if (vmax > 0.f) {
      int Ev, En = 0;
      std::frexp((double)vmax, &Ev);  // vmax < 2^Ev
      while (((i64)1 << En) < nvox) ++En;
      e = 62 - Ev - En;               // sum |q| <= nvox (2^(62-En) + 1/2) < 2^63
      scale = std::ldexp(1.0, e);
    }
    g_last_e = e;
  }

  // step 1: the projection images
  std::vector<i64*> priv(T, nullptr);
  for (int t = 0; t < T; ++t) {
    priv[t] = new (std::nothrow) i64[total];
    if (!priv[t]) {
      for (int u = 0; u < t; ++u) delete[] priv[u];
      return 5;
    }
  }
  parallel_for(T, rows, [&](int t, i64 a, i64 b) {
    std::memset(priv[t], 0, total * sizeof(i64));
    if (dtype == 0)
      project_rows(static_cast<const uint8_t*>(vol), L, M, a, b, geo, priv[t], scale);
    else if (dtype == 1)
      project_rows(static_cast<const uint16_t*>(vol), L, M, a, b, geo, priv[t], scale);
    else
      project_rows(static_cast<const float*>(vol), L, M, a, b, geo, priv[t], scale);
  });
  i64* img = priv[0];
  if (T > 1)
    parallel_for(T, (i64)total, [&](int, i64 a, i64 b) {
      for (int u = 1; u < T; ++u)
        for (i64 i = a; i < b; ++i) img[i] += priv[u][i];
    });
  for (int u = 1; u < T; ++u) delete[] priv[u];

  // step 2: 1-D integrals of every image along K + 1 directions, their
  // power moments, and the images' 2-D moments
  const int P = (int)geo.size();
  const int nd = K + 1;
  std::vector<u64> mu((size_t)P * nd * 3 * (kMaxOrder + 1));
  auto mu_at = [&](int k, int j) {
    return reinterpret_cast<u64(*)[kMaxOrder + 1]>(mu.data() + ((size_t)k * nd + j) * 3 * (kMaxOrder + 1));
  };
  parallel_for(T, (i64)P * nd, [&](int, i64 a, i64 b) {
    for (i64 w = a; w < b; ++w) {
      const int k = (int)(w / nd), j = (int)(w % nd);
      radon_moments(img, geo[k], kDirections[j][0], kDirections[j][1], K, mu_at(k, j));
    }
  });
  delete[] img;
  const Primes& PR = primes();
  std::vector<ImageMoments> im2(P);
  for (int k = 0; k < P; ++k) {
    u64 m1[kMaxOrder + 1][3][kMaxOrder + 1];
    for (int j = 0; j < nd; ++j) std::memcpy(m1[j], mu_at(k, j), sizeof(m1[j]));
    for (int pi = 0; pi < 3; ++pi)
      for (int n = 0; n <= K; ++n)
        if (!moments_2d(m1, n, pi, PR.p[pi], im2[k].m[pi][n])) return 4;
  }

  // step 3: the 3-D moments of each degree from the images' 2-D moments
  int base = 0;
  for (int n = 0; n <= K; ++n) {
    const int nm = num_monos(n);
    std::vector<std::vector<u64>> res(3, std::vector<u64>(nm));
    for (int pi = 0; pi < 3; ++pi) {
      const u64 p = PR.p[pi];
      std::vector<u64> Ab;
      Ab.reserve((size_t)P * (n + 1) * (nm + 1));
      for (int k = 0; k < P; ++k) {
        std::vector<u64> rws;
        image_rows(geo[k].im, n, p, rws);
        for (int i = 0; i <= n; ++i) {
          Ab.insert(Ab.end(), rws.begin() + (size_t)i * nm, rws.begin() + (size_t)(i + 1) * nm);
          Ab.push_back(im2[k].m[pi][n][i]);
        }
      }
      if (!solve_mod(Ab, P * (n + 1), nm, p, res[pi].data())) return 4;
    }
    for (int c = 0; c < nm; ++c) {
      const u64 r[3] = {res[0][c], res[1][c], res[2][c]};
      const Mixed mx = garner(r);
      if (dtype == 2) {
        static_cast<double*>(out)[base + c] = std::ldexp(to_double(mx), -e);
      } else {
        i128 v;
        if (!to_i128(mx, &v)) return 3;
        int64_t* o = static_cast<int64_t*>(out) + 2 * (size_t)(base + c);
        o[0] = (int64_t)(u64)v;
        o[1] = (int64_t)(u64)((u128)v >> 64);
      }
    }
    base += nm;
  }
  return 0;
}
