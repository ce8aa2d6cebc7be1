// Step 3 of the Discrete Projection Moment method: the 3-D moments from the
// 2-D moments of the projection images (Sec. 3.2, Eqs. 10-16, generalised to
// every degree n <= K with an exact integer combine per degree).
//
// Integer volumes: the 2-D moments are exact int128 values; each 3-D moment
// is  (sum_j C[m][j] T_j) / D  with the sum accumulated in 256-bit two's
// complement and divided exactly (a non-zero remainder means the images
// were not those of any volume and is reported as a self-check failure).
// Float volumes: the float-float 2-D moments are widened to FP64 here, the
// only FP64 arithmetic of the pipeline, because the combine cancels terms.
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "dpma_internal.cuh"

namespace dpma {
namespace {

constexpr int kStatusInternal = 7;

// ---------------- partial reduction ----------------

struct RedParams {
  const void* partials;
  int64_t blk_base[kMaxLimbImages + 1];
  int P, npairs;  // P: image rows to reduce
  void* m2d;
  const int* gate;  // fallback launch: nothing unless (*gate & 3)
};

// One CTA per (image k, pair t): the threads stride over the image's block
// partials (all loads independent), then a shared-memory tree adds the
// thread sums.  Integer sums are exact in int128; float pairs meet in
// float-float additions.
constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads) reduce_int_kernel(RedParams p) {
  const int k = blockIdx.x / p.npairs, t = blockIdx.x % p.npairs;
  const i128* part = static_cast<const i128*>(p.partials);
  i128 acc = 0;
  for (int64_t b = p.blk_base[k] + threadIdx.x; b < p.blk_base[k + 1]; b += kRedThreads)
    acc += part[b * p.npairs + t];
  __shared__ i128 sh[kRedThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) static_cast<i128*>(p.m2d)[k * p.npairs + t] = sh[0];
}

__global__ void __launch_bounds__(kRedThreads) reduce_f32_kernel(RedParams p) {
  if (p.gate && (*p.gate & 3) == 0) return;
  const int k = blockIdx.x / p.npairs, t = blockIdx.x % p.npairs;
  const float2* part = static_cast<const float2*>(p.partials);
  float h = 0.f, l = 0.f;
  for (int64_t b = p.blk_base[k] + threadIdx.x; b < p.blk_base[k + 1]; b += kRedThreads) {
    const float2 v = part[b * p.npairs + t];
    ff_add(h, l, v.x, v.y);
  }
  __shared__ float2 sh[kRedThreads];
  sh[threadIdx.x] = make_float2(h, l);
  __syncthreads();
  for (int w = kRedThreads / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) {
      float2 a = sh[threadIdx.x];
      const float2 c = sh[threadIdx.x + w];
      ff_add(a.x, a.y, c.x, c.y);
      sh[threadIdx.x] = a;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) static_cast<float2*>(p.m2d)[k * p.npairs + t] = sh[0];
}

// ---------------- 256-bit helpers ----------------

struct I256 {
  uint64_t w[4];
};

__device__ __forceinline__ void neg256(I256& a) {
  uint64_t carry = 1;
  for (int i = 0; i < 4; ++i) {
    uint64_t v = ~a.w[i] + carry;
    carry = (carry && v == 0) ? 1 : 0;
    a.w[i] = v;
  }
}

__device__ __forceinline__ void add256(I256& a, const I256& b) {
  unsigned long long carry = 0;
  for (int i = 0; i < 4; ++i) {
    u128 s = (u128)a.w[i] + b.w[i] + carry;
    a.w[i] = (uint64_t)s;
    carry = (unsigned long long)(s >> 64);
  }
}

// a += c * t   (c: int64, t: int128)
__device__ __forceinline__ void mac256(I256& a, int64_t c, i128 t) {
  if (c == 0 || t == 0) return;
  const bool neg = (c < 0) != (t < 0);
  const uint64_t uc = c < 0 ? (uint64_t)(-(c + 1)) + 1 : (uint64_t)c;
  const u128 ut = t < 0 ? (u128)(-(t + 1)) + 1 : (u128)t;
  const u128 p0 = (u128)uc * (uint64_t)ut;
  const u128 p1 = (u128)uc * (uint64_t)(ut >> 64);
  const u128 mid = (p0 >> 64) + (u128)(uint64_t)p1;
  I256 prod;
  prod.w[0] = (uint64_t)p0;
  prod.w[1] = (uint64_t)mid;
  prod.w[2] = (uint64_t)(p1 >> 64) + (uint64_t)(mid >> 64);
  prod.w[3] = 0;
  if (neg) neg256(prod);
  add256(a, prod);
}

// q = a / d exactly for d = odd << sh, with inv the inverse of odd modulo
// 2^128: when the division is exact the quotient is the low 128 bits of
// (a >> sh) * inv, and multiplying back reproduces a in 256 bits; a
// remainder or a quotient outside int128 fails that check.  Two 128-bit
// products instead of four long divisions.
__device__ bool div_exact_inv(const I256& a, int64_t d, int sh, u128 inv, i128* q) {
  const u128 lo = ((u128)a.w[1] << 64) | a.w[0];
  const u128 hi = ((u128)a.w[3] << 64) | a.w[2];
  const u128 as = sh ? ((lo >> sh) | (hi << (128 - sh))) : lo;
  const i128 qc = (i128)(as * inv);
  I256 back = {{0, 0, 0, 0}};
  mac256(back, d, qc);
  if (back.w[0] != a.w[0] || back.w[1] != a.w[1] || back.w[2] != a.w[2] || back.w[3] != a.w[3])
    return false;
  *q = qc;
  return true;
}

// ---------------- combine ----------------

// Packed plan (int64 words): for n = 0..K at word off[n]:
//   D, nmono, img[nmono], a[nmono], C[nmono * nmono]
struct CombParams {
  const int64_t* plan;
  int off[kMaxK + 1];
  int dshift[kMaxK + 1];       // D_n = odd << dshift[n]
  uint64_t dinv[kMaxK + 1][2];  // odd^-1 mod 2^128 (low, high)
  int K, npairs;
  const void* m2d;
  void* out;
  int* status;
  const int* gate;  // fallback launch: nothing unless (*gate & 3)
};

// One warp per moment: the lanes take the terms j = lane, lane + 32, ... of
// the degree's combination, their partial sums meet in a warp reduction and
// lane 0 divides by D (exactly, for integers) and writes the moment.
__device__ __forceinline__ bool moment_of_warp(const CombParams& p, int& n, int& row) {
  const int m = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nmom = (p.K + 1) * (p.K + 2) * (p.K + 3) / 6;
  if (m >= nmom) return false;
  n = 0;
  while ((n + 1) * (n + 2) * (n + 3) / 6 <= m) ++n;
  row = m - n * (n + 1) * (n + 2) / 6;
  return true;
}

__global__ void combine_int_kernel(CombParams p) {
  int n, row;
  if (!moment_of_warp(p, n, row)) return;  // uniform across the warp
  const int lane = threadIdx.x & 31;
  const int64_t* pl = p.plan + p.off[n];
  const int64_t D = pl[0];
  const int nm = (int)pl[1];
  const int64_t* img = pl + 2;
  const int64_t* aa = img + nm;
  const int64_t* C = aa + nm;
  const i128* T = static_cast<const i128*>(p.m2d);
  I256 acc = {{0, 0, 0, 0}};
  for (int j = lane; j < nm; j += 32) {
    const int a = (int)aa[j];
    const int pair = n * (n + 1) / 2 + (n - a);
    mac256(acc, C[row * nm + j], T[img[j] * p.npairs + pair]);
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    I256 o;
#pragma unroll
    for (int w = 0; w < 4; ++w)
      o.w[w] = __shfl_xor_sync(0xffffffffu, (unsigned long long)acc.w[w], m);
    add256(acc, o);
  }
  if (lane != 0) return;
  i128 q = 0;
  const u128 inv = ((u128)p.dinv[n][1] << 64) | p.dinv[n][0];
  if (!div_exact_inv(acc, D, p.dshift[n], inv, &q)) {
    if (p.status) atomicCAS(p.status, 0, kStatusInternal);  // a timeout (5) stays
    q = 0;
  }
  const int mi = n * (n + 1) * (n + 2) / 6 + row;
  static_cast<i128*>(p.out)[mi] = q;
}

__global__ void combine_f32_kernel(CombParams p) {
  if (p.gate && (*p.gate & 3) == 0) return;
  int n, row;
  if (!moment_of_warp(p, n, row)) return;
  const int lane = threadIdx.x & 31;
  const int64_t* pl = p.plan + p.off[n];
  const double D = (double)pl[0];
  const int nm = (int)pl[1];
  const int64_t* img = pl + 2;
  const int64_t* aa = img + nm;
  const int64_t* C = aa + nm;
  const float2* T = static_cast<const float2*>(p.m2d);
  double acc = 0.0;
  for (int j = lane; j < nm; j += 32) {
    const int a = (int)aa[j];
    const int pair = n * (n + 1) / 2 + (n - a);
    const float2 t = T[img[j] * p.npairs + pair];
    acc += (double)C[row * nm + j] * ((double)t.x + (double)t.y);
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
  if (lane == 0) static_cast<double*>(p.out)[n * (n + 1) * (n + 2) / 6 + row] = acc / D;
}

// Float volumes projected on quantisation limbs: the m2d rows hold the exact
// int128 2-D moments of limb 0 (rows 0..P-1) and limb 1 (rows P..2P-1).
// One warp per moment combines both limbs exactly, joins them into the
// moment of the quantised volume, Q = M0 * 2^(B+1) + M1 in units of
// 2^-(e1+B+1), and converts it to double: the only rounding after the
// quantisation.  It also bounds the quantisation error of the moment,
//   |M_pqr(V) - M_pqr(Q)| <= 2^-(e1+B+2) * sum_{x<L} x^p sum_{y<M} y^q sum_{z<N} z^r,
// each power sum bounded from above in closed form, and raises flag 2 when that bound
// (plus the final rounding) exceeds `tol` times |M_pqr(Q)| minus the bound,
// i.e. when the result cannot be guaranteed within tol of the moment of |V|.
struct FixedParams {
  const int64_t* plan;
  int off[kMaxK + 1];
  int dshift[kMaxK + 1];
  uint64_t dinv[kMaxK + 1][2];
  int K, npairs, P;
  const void* m2d;
  double* out;
  int* status;
  int* flags;
  const int* scale;  // e1, B
  double L, M, N;
  double tol;
};

// Upper bound on sum_{t<n} t^p: n for p = 0, else the last term (n-1)^p plus
// the integral of t^p over [0, n-1] (t^p increases); zero when n = 1.
__device__ __forceinline__ double power_sum_bound(double n, int p) {
  if (p == 0) return n;
  const double m = n - 1.0;
  double v = 1.0;
  for (int i = 0; i < p; ++i) v *= m;
  return v + v * m / (double)(p + 1);
}

// double nearest (within a few ulps) to a 256-bit two's complement value
__device__ __forceinline__ double i256_to_double(I256 a) {
  const bool neg = (a.w[3] >> 63) != 0;
  if (neg) neg256(a);
  double d = (double)a.w[3];
  d = d * 18446744073709551616.0 + (double)a.w[2];
  d = d * 18446744073709551616.0 + (double)a.w[1];
  d = d * 18446744073709551616.0 + (double)a.w[0];
  return neg ? -d : d;
}

__global__ void combine_fixed_kernel(FixedParams p) {
  const int m = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nmom = (p.K + 1) * (p.K + 2) * (p.K + 3) / 6;
  if (m >= nmom) return;  // uniform across the warp
  int n = 0;
  while ((n + 1) * (n + 2) * (n + 3) / 6 <= m) ++n;
  const int row = m - n * (n + 1) * (n + 2) / 6;
  const int lane = threadIdx.x & 31;
  const int64_t* pl = p.plan + p.off[n];
  const int64_t D = pl[0];
  const int nm = (int)pl[1];
  const int64_t* img = pl + 2;
  const int64_t* aa = img + nm;
  const int64_t* Cm = aa + nm;
  const i128* T = static_cast<const i128*>(p.m2d);
  I256 acc0 = {{0, 0, 0, 0}}, acc1 = {{0, 0, 0, 0}};
  for (int j = lane; j < nm; j += 32) {
    const int a = (int)aa[j];
    const int pair = n * (n + 1) / 2 + (n - a);
    const int64_t c = Cm[row * nm + j];
    mac256(acc0, c, T[img[j] * p.npairs + pair]);
    mac256(acc1, c, T[(p.P + img[j]) * p.npairs + pair]);
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    I256 x, y;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      x.w[w] = __shfl_xor_sync(0xffffffffu, (unsigned long long)acc0.w[w], o);
      y.w[w] = __shfl_xor_sync(0xffffffffu, (unsigned long long)acc1.w[w], o);
    }
    add256(acc0, x);
    add256(acc1, y);
  }
  if (lane != 0) return;
  i128 q0 = 0, q1 = 0;
  // a remainder (impossible for images of a volume) also sends the volume
  // to the fallback, which recomputes it
  const u128 inv = ((u128)p.dinv[n][1] << 64) | p.dinv[n][0];
  const bool ok = div_exact_inv(acc0, D, p.dshift[n], inv, &q0) &&
                  div_exact_inv(acc1, D, p.dshift[n], inv, &q1);
  // Q = q0 * 2^(B+1) + q1, exactly, in 256 bits
  I256 q;
  {
    const int sh = p.scale[1] + 1;  // B + 1 <= 22
    const u128 lo = (u128)q0 << sh;
    const i128 hi = q0 >> (128 - sh);  // arithmetic: the bits shifted out, sign-extended
    q.w[0] = (uint64_t)lo;
    q.w[1] = (uint64_t)(lo >> 64);
    q.w[2] = (uint64_t)hi;
    q.w[3] = (uint64_t)(hi >> 64);
    I256 b;
    b.w[0] = (uint64_t)(u128)q1;
    b.w[1] = (uint64_t)((u128)q1 >> 64);
    b.w[2] = b.w[3] = (q1 < 0) ? ~0ull : 0ull;
    add256(q, b);
  }
  const int e = p.scale[0] + p.scale[1] + 1;  // Q counts units of 2^-e
  const double val = ldexp(i256_to_double(q), -e);
  const int mi = n * (n + 1) * (n + 2) / 6 + row;
  p.out[mi] = val;
  // (p, q, r) of row `row` of degree n: p descending, then q descending
  int pp = n, rr = row;
  while (rr > n - pp) { rr -= n - pp + 1; --pp; }
  const int qq = n - pp - rr, rz = rr;
  const double bound = ldexp(power_sum_bound(p.L, pp) * power_sum_bound(p.M, qq) *
                                 power_sum_bound(p.N, rz), -e - 1) +
                       fabs(val) * 0x1p-50;
  if (!ok || !(bound <= p.tol * (fabs(val) - bound))) atomicOr(p.flags, 2);
}

// For every degree of plan cp: D_n = odd << dshift[n] and odd^-1 modulo
// 2^128 (Newton's iteration x <- x (2 - odd x), which doubles the correct
// low bits from 3 at x = odd).  Host only.
bool divisor_inverses(const CombinePlan& cp, int dshift[kMaxK + 1], uint64_t dinv[kMaxK + 1][2]) {
  for (int n = 0; n <= kMaxK; ++n) { dshift[n] = 0; dinv[n][0] = dinv[n][1] = 0; }
  for (int n = 0; n <= cp.K; ++n) {
    uint64_t odd = (uint64_t)cp.deg[n].D;
    int sh = 0;
    while (odd && (odd & 1) == 0) { odd >>= 1; ++sh; }
    if (odd == 0) return false;
    u128 x = odd;
    for (int it = 0; it < 7; ++it) x *= (u128)2 - (u128)odd * x;
    dshift[n] = sh;
    dinv[n][0] = (uint64_t)x;
    dinv[n][1] = (uint64_t)(x >> 64);
  }
  return true;
}

struct DevPlan {
  int64_t* words;
  int off[kMaxK + 1];
  int dshift[kMaxK + 1];
  uint64_t dinv[kMaxK + 1][2];
};

std::mutex g_mu;
std::unordered_map<int64_t, DevPlan> g_dev_plans;  // key: device * 16 + K

cudaError_t device_plan(int K, DevPlan* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int64_t key = (int64_t)dev * 16 + K;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_dev_plans.find(key);
  if (it != g_dev_plans.end()) { *out = it->second; return cudaSuccess; }
  const CombinePlan* cp = combine_plan(K);
  if (!cp) return cudaErrorInvalidValue;
  std::vector<int64_t> w;
  DevPlan dp{};
  if (!divisor_inverses(*cp, dp.dshift, dp.dinv)) return cudaErrorInvalidValue;
  for (int n = 0; n <= K; ++n) {
    const DegreePlan& d = cp->deg[n];
    dp.off[n] = (int)w.size();
    w.push_back(d.D);
    w.push_back(d.nmono);
    for (int j = 0; j < d.nmono; ++j) w.push_back(d.img[j]);
    for (int j = 0; j < d.nmono; ++j) w.push_back(d.a[j]);
    for (int j = 0; j < d.nmono * d.nmono; ++j) w.push_back(d.C[j]);
  }
  e = cudaMalloc(&dp.words, w.size() * sizeof(int64_t));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(dp.words, w.data(), w.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(dp.words); return e; }
  g_dev_plans[key] = dp;
  *out = dp;
  return cudaSuccess;
}

}  // namespace

namespace {
__global__ void clear_kernel(uint32_t* p, int64_t n32, int* status, const int* gate) {
  if (gate && (*gate & 3) == 0) return;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (status && gid == 0) *status = 0;
  const int64_t n16 = n32 >> 2;
  uint4* q = reinterpret_cast<uint4*>(p);
  for (int64_t i = gid; i < n16; i += stride) q[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t i = (n16 << 2) + gid; i < n32; i += stride) p[i] = 0u;
}
}  // namespace

cudaError_t launch_clear(void* p, size_t bytes, int* status, cudaStream_t st, const int* gate) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) != 0 || (bytes & 3) != 0) {
    if (gate) return cudaErrorInvalidValue;  // gated clears need the kernel
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, st);
    if (e == cudaSuccess && status) e = cudaMemsetAsync(status, 0, sizeof(int), st);
    return e;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t n32 = (int64_t)(bytes / 4);
  int64_t blocks = (n32 / 4 + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  clear_kernel<<<(unsigned)blocks, 256, 0, st>>>(static_cast<uint32_t*>(p), n32, status, gate);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const void* partials, const int64_t* blk_base, int P, int K,
                                   bool is_float, void* m2d, cudaStream_t st, const int* gate) {
  RedParams p{};
  p.gate = gate;
  p.partials = partials;
  p.m2d = m2d;
  for (int k = 0; k <= P; ++k) p.blk_base[k] = blk_base[k];
  p.P = P;
  p.npairs = num_2d(K);
  if (is_float) reduce_f32_kernel<<<P * p.npairs, kRedThreads, 0, st>>>(p);
  else reduce_int_kernel<<<P * p.npairs, kRedThreads, 0, st>>>(p);
  return cudaGetLastError();
}

// Ensures the plan of order K is resident on the current device (host call,
// synchronous the first time).
cudaError_t prepare_combine(int K) {
  DevPlan dp{};
  return device_plan(K, &dp);
}

cudaError_t launch_combine(const void* m2d, int K, bool is_float, void* out, int* status,
                           cudaStream_t st, const int* gate) {
  DevPlan dp{};
  cudaError_t e = device_plan(K, &dp);
  if (e != cudaSuccess) return e;
  CombParams p{};
  p.gate = gate;
  p.plan = dp.words;
  for (int n = 0; n <= kMaxK; ++n) {
    p.off[n] = dp.off[n];
    p.dshift[n] = dp.dshift[n];
    p.dinv[n][0] = dp.dinv[n][0];
    p.dinv[n][1] = dp.dinv[n][1];
  }
  p.K = K;
  p.npairs = num_2d(K);
  p.m2d = m2d;
  p.out = out;
  p.status = status;
  const int nmom = num_moments(K);
  const int threads = 128;  // four moments per block, one warp each
  const int blocks = (nmom * 32 + threads - 1) / threads;
  if (is_float) combine_f32_kernel<<<blocks, threads, 0, st>>>(p);
  else combine_int_kernel<<<blocks, threads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_combine_fixed(const void* m2d, int K, int P, double* out, int* status,
                                 int* flags, const int* scale, int64_t L, int64_t M, int64_t N,
                                 double tol, cudaStream_t st) {
  DevPlan dp{};
  cudaError_t e = device_plan(K, &dp);
  if (e != cudaSuccess) return e;
  FixedParams p{};
  p.plan = dp.words;
  for (int n = 0; n <= kMaxK; ++n) {
    p.off[n] = dp.off[n];
    p.dshift[n] = dp.dshift[n];
    p.dinv[n][0] = dp.dinv[n][0];
    p.dinv[n][1] = dp.dinv[n][1];
  }
  p.K = K;
  p.npairs = num_2d(K);
  p.P = P;
  p.m2d = m2d;
  p.out = out;
  p.status = status;
  p.flags = flags;
  p.scale = scale;
  p.L = (double)L; p.M = (double)M; p.N = (double)N;
  p.tol = tol;
  const int nmom = num_moments(K);
  const int threads = 128;
  const int blocks = (nmom * 32 + threads - 1) / threads;
  combine_fixed_kernel<<<blocks, threads, 0, st>>>(p);
  return cudaGetLastError();
}

// Packs the combine plan of order K into `words` (capacity in int64 words)
// with the layout the combine kernels read; returns the word count, 0 if the
// plan is unavailable or does not fit.  Host only, allocates no device memory.
size_t pack_combine_plan(int K, int64_t* words, size_t capacity, int off[kMaxK + 1]) {
  const CombinePlan* cp = combine_plan(K);
  if (!cp) return 0;
  size_t n = 0;
  for (int k = 0; k <= kMaxK; ++k) off[k] = 0;
  for (int d = 0; d <= K; ++d) {
    const DegreePlan& g = cp->deg[d];
    const size_t need = 2 + 2 * (size_t)g.nmono + (size_t)g.nmono * g.nmono;
    if (n + need > capacity) return 0;
    off[d] = (int)n;
    words[n++] = g.D;
    words[n++] = g.nmono;
    for (int j = 0; j < g.nmono; ++j) words[n++] = g.img[j];
    for (int j = 0; j < g.nmono; ++j) words[n++] = g.a[j];
    for (int j = 0; j < g.nmono * g.nmono; ++j) words[n++] = g.C[j];
  }
  return n;
}

// Combine with a packed plan already resident at `dev_words` (device memory).
cudaError_t launch_combine_packed(const int64_t* dev_words, const int off[kMaxK + 1],
                                  const void* m2d, int K, bool is_float, void* out, int* status,
                                  cudaStream_t st) {
  CombParams p{};
  p.plan = dev_words;
  for (int n = 0; n <= kMaxK; ++n) p.off[n] = off[n];
  const CombinePlan* cp = combine_plan(K);
  if (!cp || !divisor_inverses(*cp, p.dshift, p.dinv)) return cudaErrorInvalidValue;
  p.K = K;
  p.npairs = num_2d(K);
  p.m2d = m2d;
  p.out = out;
  p.status = status;
  const int nmom = num_moments(K);
  const int threads = 128;  // four moments per block, one warp each
  const int blocks = (nmom * 32 + threads - 1) / threads;
  if (is_float) combine_f32_kernel<<<blocks, threads, 0, st>>>(p);
  else combine_int_kernel<<<blocks, threads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace dpma
