// Exact combine plan for the final step of the Discrete Projection Moment
// method (Sec. 3.2, Eqs. 10-16, generalised to any order K <= 10).
//
// An image with forms (u, w) has 2-D moments
//     T_ab = sum_voxels V (u.x)^a (w.x)^b,
// a homogeneous polynomial identity of degree n = a+b in the 3-D moments
// (the expansion the paper performs for Eq. 13).  Stacking, for each degree
// n, the rows of every image's (a, n-a) expansions gives an integer system
// A_n m_n = t_n; K+1 distinct line directions give it full column rank for
// every n <= K (the axis family of Eqs. 5-7 plus the +-pi/4 family named
// after Eq. 9 hold 9 directions, enough for K <= 8; the arctan(1/2) image
// about y and the isometric image of the further families extend it to
// K = 10).  The plan keeps, in a
// fixed order, the rows that raise the rank, inverts the square system
// exactly and stores it as an integer matrix C over a common denominator D:
//     m_n = (1/D) C t_sel.
// The inverse is computed modulo the prime 2^61-1, lifted to rationals by
// rational reconstruction and then checked exactly (C A_sel == D I in
// integer arithmetic), so a wrong lift cannot go unnoticed.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace dpma {

namespace {

using u64 = uint64_t;
using i128 = __int128;
using u128 = unsigned __int128;

constexpr u64 kPrime = (1ull << 61) - 1;

u64 mulmod(u64 a, u64 b) {
  u128 p = (u128)a * b;
  u64 lo = (u64)(p & kPrime), hi = (u64)(p >> 61);
  u64 s = lo + hi;
  return s >= kPrime ? s - kPrime : s;
}
u64 submod(u64 a, u64 b) { return a >= b ? a - b : a + kPrime - b; }
u64 powmod(u64 a, u64 e) {
  u64 r = 1;
  while (e) { if (e & 1) r = mulmod(r, a); a = mulmod(a, a); e >>= 1; }
  return r;
}
u64 invmod(u64 a) { return powmod(a, kPrime - 2); }
u64 tomod(int64_t v) {
  int64_t m = v % (int64_t)kPrime;
  return m < 0 ? (u64)(m + (int64_t)kPrime) : (u64)m;
}

// Recover num/den with |num|, den <= sqrt(p/2) from r = num/den mod p.
bool rational_reconstruct(u64 r, int64_t* num, int64_t* den) {
  const i128 bound = (i128)1 << 29;  // 2 * bound^2 < p: the lift is unique
  i128 r0 = kPrime, r1 = r, t0 = 0, t1 = 1;
  while (r1 >= bound) {
    i128 q = r0 / r1;
    i128 r2 = r0 - q * r1; r0 = r1; r1 = r2;
    i128 t2 = t0 - q * t1; t0 = t1; t1 = t2;
  }
  if (t1 == 0) return false;
  if (t1 < 0) { t1 = -t1; r1 = -r1; }
  if (t1 >= bound) return false;
  *num = (int64_t)r1;
  *den = (int64_t)t1;
  return true;
}

int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}

// Degree-n monomials in graded order (p descending, then q descending).
void monomials(int n, std::vector<int>& p, std::vector<int>& q, std::vector<int>& r) {
  for (int pp = n; pp >= 0; --pp)
    for (int qq = n - pp; qq >= 0; --qq) { p.push_back(pp); q.push_back(qq); r.push_back(n - pp - qq); }
}

// Coefficients of (u.x)^a (w.x)^b over the degree-(a+b) monomials.
void expand_row(const int u[3], const int w[3], int a, int b, const std::vector<int>& mp,
                const std::vector<int>& mq, int64_t* row) {
  const int n = a + b;
  // dense polynomial over exponents (p, q) with r implied, size (n+1)^2
  std::vector<int64_t> poly((n + 1) * (n + 1), 0), next;
  poly[0] = 1;
  int deg = 0;
  auto mul = [&](const int f[3]) {
    next.assign((n + 1) * (n + 1), 0);
    for (int p = 0; p <= deg; ++p)
      for (int q = 0; q + p <= deg; ++q) {
        int64_t c = poly[p * (n + 1) + q];
        if (!c) continue;
        if (f[0]) next[(p + 1) * (n + 1) + q] += c * f[0];
        if (f[1]) next[p * (n + 1) + q + 1] += c * f[1];
        if (f[2]) next[p * (n + 1) + q] += c * f[2];
      }
    poly.swap(next);
    ++deg;
  };
  for (int i = 0; i < a; ++i) mul(u);
  for (int i = 0; i < b; ++i) mul(w);
  for (size_t m = 0; m < mp.size(); ++m) row[m] = poly[mp[m] * (n + 1) + mq[m]];
}

bool build_degree(int n, int P, DegreePlan* out) {
  std::vector<int> mp, mq, mr;
  monomials(n, mp, mq, mr);
  const int nm = (int)mp.size();
  out->n = n;
  out->nmono = nm;

  // candidate rows in fixed order: image 0..P-1, slow exponent a = n..0
  std::vector<std::vector<int64_t>> sel_rows;
  std::vector<std::vector<u64>> basis;  // echelon basis mod p
  std::vector<int> pivots;
  for (int k = 0; k < P && (int)sel_rows.size() < nm; ++k) {
    ImageGeom g;
    image_geom(k, 1, 1, 1, &g);
    for (int a = n; a >= 0 && (int)sel_rows.size() < nm; --a) {
      std::vector<int64_t> row(nm);
      expand_row(g.slow, g.fast, a, n - a, mp, mq, row.data());
      std::vector<u64> v(nm);
      for (int j = 0; j < nm; ++j) v[j] = tomod(row[j]);
      for (size_t b = 0; b < basis.size(); ++b) {
        u64 c = v[pivots[b]];
        if (!c) continue;
        for (int j = 0; j < nm; ++j) v[j] = submod(v[j], mulmod(c, basis[b][j]));
      }
      int piv = -1;
      for (int j = 0; j < nm; ++j) if (v[j]) { piv = j; break; }
      if (piv < 0) continue;  // does not raise the rank
      u64 inv = invmod(v[piv]);
      for (int j = 0; j < nm; ++j) v[j] = mulmod(v[j], inv);
      basis.push_back(v);
      pivots.push_back(piv);
      out->img[sel_rows.size()] = k;
      out->a[sel_rows.size()] = a;
      sel_rows.push_back(row);
    }
  }
  if ((int)sel_rows.size() != nm) return false;

  // Solve A_sel m = t: C = A_sel^{-1} (mod p) by Gauss-Jordan on [A | I].
  std::vector<u64> aug(nm * 2 * nm, 0);
  for (int i = 0; i < nm; ++i) {
    for (int j = 0; j < nm; ++j) aug[i * 2 * nm + j] = tomod(sel_rows[i][j]);
    aug[i * 2 * nm + nm + i] = 1;
  }
  for (int c = 0; c < nm; ++c) {
    int piv = -1;
    for (int i = c; i < nm; ++i) if (aug[i * 2 * nm + c]) { piv = i; break; }
    if (piv < 0) return false;
    if (piv != c)
      for (int j = 0; j < 2 * nm; ++j) std::swap(aug[piv * 2 * nm + j], aug[c * 2 * nm + j]);
    u64 inv = invmod(aug[c * 2 * nm + c]);
    for (int j = 0; j < 2 * nm; ++j) aug[c * 2 * nm + j] = mulmod(aug[c * 2 * nm + j], inv);
    for (int i = 0; i < nm; ++i) {
      if (i == c) continue;
      u64 f = aug[i * 2 * nm + c];
      if (!f) continue;
      for (int j = 0; j < 2 * nm; ++j)
        aug[i * 2 * nm + j] = submod(aug[i * 2 * nm + j], mulmod(f, aug[c * 2 * nm + j]));
    }
  }
  // A_sel^{-1}[m][j] maps selected 2-D moments j to monomial m.
  std::vector<int64_t> num(nm * nm), den(nm * nm);
  int64_t D = 1;
  for (int m = 0; m < nm; ++m)
    for (int j = 0; j < nm; ++j) {
      if (!rational_reconstruct(aug[m * 2 * nm + nm + j], &num[m * nm + j], &den[m * nm + j]))
        return false;
      int64_t d = den[m * nm + j];
      D = D / gcd64(D, d) * d;
      if (D > ((int64_t)1 << 40)) return false;
    }
  out->D = D;
  for (int m = 0; m < nm; ++m)
    for (int j = 0; j < nm; ++j) out->C[m * nm + j] = num[m * nm + j] * (D / den[m * nm + j]);

  // Exact check: C * A_sel == D * I.
  for (int m = 0; m < nm; ++m)
    for (int c = 0; c < nm; ++c) {
      i128 s = 0;
      for (int j = 0; j < nm; ++j) s += (i128)out->C[m * nm + j] * sel_rows[j][c];
      if (s != (m == c ? (i128)D : 0)) return false;
    }
  return true;
}

std::mutex g_plan_mu;
CombinePlan* g_plans[kMaxK + 1] = {nullptr};
bool g_plan_failed[kMaxK + 1] = {false};

}  // namespace

int num_images(int K) { return K + 1 < 3 ? 3 : K + 1; }
int num_moments(int K) { return (K + 1) * (K + 2) * (K + 3) / 6; }
int num_2d(int K) { return (K + 1) * (K + 2) / 2; }

int idx3d(int p, int q, int r) {
  int n = p + q + r;
  int base = n * (n + 1) * (n + 2) / 6;  // moments of degree < n
  // within degree n: p descending then q descending
  int off = 0;
  for (int pp = n; pp > p; --pp) off += n - pp + 1;
  off += (n - p) - q;
  return base + off;
}

bool image_geom(int k, int64_t L, int64_t M, int64_t N, ImageGeom* g) {
  static const int forms[kMaxImages][2][3] = {
      {{0, 1, 0}, {1, 0, 0}},   // 0: (x, y), line along z          Eq. 5
      {{0, 0, 1}, {0, 1, 0}},   // 1: (y, z), line along x          Eq. 6
      {{0, 0, 1}, {1, 0, 0}},   // 2: (z, x), line along y          Eq. 7
      {{0, 1, 0}, {1, 0, 1}},   // 3: (x+z, y)                      Eq. 8
      {{0, 1, 0}, {1, 0, -1}},  // 4: (x-z, y)                      Eq. 9
      {{0, 1, 1}, {1, 0, 0}},   // 5: (y+z, x)   +-pi/4 about x
      {{0, 1, -1}, {1, 0, 0}},  // 6: (y-z, x)
      {{0, 0, 1}, {1, 1, 0}},   // 7: (x+y, z)   +-pi/4 about z
      {{0, 0, 1}, {1, -1, 0}},  // 8: (x-y, z)
      {{0, 1, 0}, {1, 0, 2}},   // 9: (x+2z, y)  arctan(1/2) about y, line (2,0,-1)
      {{1, 0, 1}, {1, 2, -1}},  // 10: isometric (x+z, 2y+x-z), line (1,-1,-1)
  };
  if (k < 0 || k >= kMaxImages) return false;
  std::memcpy(g->slow, forms[k][0], sizeof(g->slow));
  std::memcpy(g->fast, forms[k][1], sizeof(g->fast));
  const int64_t dims[3] = {L, M, N};
  auto extent = [&](const int f[3], int64_t* lo) {
    int64_t mn = 0, mx = 0;
    for (int d = 0; d < 3; ++d) {
      if (f[d] > 0) mx += f[d] * (dims[d] - 1);
      if (f[d] < 0) mn += f[d] * (dims[d] - 1);
    }
    *lo = mn;
    return mx - mn + 1;
  };
  int64_t lo_s, lo_f;
  g->S = extent(g->slow, &lo_s);
  g->F = extent(g->fast, &lo_f);
  g->off_s = -lo_s;
  g->off_f = -lo_f;
  return true;
}

const CombinePlan* combine_plan(int K) {
  if (K < 0 || K > kMaxK) return nullptr;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  if (g_plans[K]) return g_plans[K];
  if (g_plan_failed[K]) return nullptr;
  CombinePlan* p = new CombinePlan();
  p->K = K;
  p->P = num_images(K);
  for (int n = 0; n <= K; ++n)
    if (!build_degree(n, p->P, &p->deg[n])) {
      delete p;
      g_plan_failed[K] = true;
      return nullptr;
    }
  g_plans[K] = p;
  return p;
}

double log2_bound_2d(int64_t L, int64_t M, int64_t N, double vmax, int K) {
  const double mass = std::log2(vmax > 1 ? vmax : 1.0) + std::log2((double)L) +
                      std::log2((double)M) + std::log2((double)N);
  double worst = mass;
  for (int k = 0; k < num_images(K); ++k) {
    ImageGeom g;
    image_geom(k, L, M, N, &g);
    // largest |signed coordinate| along each axis of the image
    double smax = (double)std::max<int64_t>(g.S - 1 - g.off_s, g.off_s);
    double fmax = (double)std::max<int64_t>(g.F - 1 - g.off_f, g.off_f);
    double ls = smax > 1 ? std::log2(smax) : 0.0, lf = fmax > 1 ? std::log2(fmax) : 0.0;
    for (int a = 0; a <= K; ++a)
      for (int b = 0; a + b <= K; ++b) worst = std::max(worst, mass + a * ls + b * lf);
  }
  return worst;
}

double log2_bound_3d(int64_t L, int64_t M, int64_t N, double vmax, int K) {
  const double mass = std::log2(vmax > 1 ? vmax : 1.0) + std::log2((double)L) +
                      std::log2((double)M) + std::log2((double)N);
  double lx = L > 2 ? std::log2((double)(L - 1)) : 0.0;
  double ly = M > 2 ? std::log2((double)(M - 1)) : 0.0;
  double lz = N > 2 ? std::log2((double)(N - 1)) : 0.0;
  double worst = mass;
  for (int p = 0; p <= K; ++p)
    for (int q = 0; p + q <= K; ++q)
      for (int r = 0; p + q + r <= K; ++r) worst = std::max(worst, mass + p * lx + q * ly + r * lz);
  return worst;
}

int float_limb_bits(int64_t L, int64_t M, int64_t N, int K) {
  // every line holds at most max(L, M, N) voxels: line sums of limbs up to
  // 2^B stay below 2^30
  const int64_t nmax = std::max<int64_t>(L, std::max<int64_t>(M, N));
  int lg = 0;
  while (((int64_t)1 << lg) < nmax) ++lg;
  int B = 30 - lg;
  if (B > 22) B = 22;  // the rounding by 1.5 * 2^23 needs |x| <= 2^22
  // limb moments (2-D and 3-D) of a volume of values up to 2^B within int128
  const double unit = std::max(log2_bound_2d(L, M, N, 1.0, K), log2_bound_3d(L, M, N, 1.0, K));
  const int cap = (int)std::floor(124.0 - unit);
  if (B > cap) B = cap;
  return B;
}

}  // namespace dpma
