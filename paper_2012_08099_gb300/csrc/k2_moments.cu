// Step 2 of the Discrete Projection Moment method: the 2-D moments of every
// projection image (Sec. 1, Eq. 1; Sec. 3.2), with signed coordinates so
// the origin shift of the negative-index images (Sec. 5) is built in:
//
//     T_ab = sum_s (s - off_s)^a * F_b(s),   F_b(s) = sum_f I[s][f] (f - off_f)^b.
//
// The paper obtains the same values from 1-D Discrete Radon integrals of
// each image (its DRT listing); on a GPU the separable power sums above are
// cheaper and exact, and they give identical results.
//
// Integer images: one thread per row segment of 16-64 pixels runs
// cascaded sums (additions only) and converts them exactly to the
// segment's power sums F_b; the CTA then folds s^a F_b over its segments.
// Float images (doubles): the same segments; each double is split into a
// float32 pair with integer operations and F_b accumulates in float-float
// (no FP64 arithmetic), then the same fold in float-float.
// Every CTA writes one partial vector; a small kernel sums them per image.
#include <cstdint>

#include "dpma_internal.cuh"

namespace dpma {
namespace {


struct K2Params {
  const void* images;
  ImageSet set;
  int nimg;     // images to reduce: nl * P (image i is image i % P of limb i / P)
  int K;
  int npairs;
  int seg_len;  // integer images: pixels per row segment
  int64_t blk_base[kMaxLimbImages + 1];  // first block of each image; [nimg] = total
  void* partials;                        // [block][npairs] int128 or float2
  const int* gate;                       // fallback launch: nothing unless (*gate & 3)
  // integer images: when set, each CTA adds its sums into these zeroed
  // [nimg][npairs] int128 moments itself and no reduction launch follows
  i128* m2d_atomic;
};

// dst += v modulo 2^128 with two 64-bit atomic adds: the low word's carry,
// known from its value before the add, goes into the high word, so any
// interleaving of such adds leaves the exact sum.
__device__ __forceinline__ void atomic_add_u128(i128* dst, u128 v) {
  unsigned long long* w = reinterpret_cast<unsigned long long*>(dst);
  const unsigned long long lo = (unsigned long long)v;
  const unsigned long long hi = (unsigned long long)(v >> 64);
  const unsigned long long old = atomicAdd(w, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi + carry) atomicAdd(w + 1, hi + carry);
}

// The signed product a * b of two 64-bit values, as 128 bits.
__device__ __forceinline__ u128 mul_s64(int64_t a, int64_t b) {
  const uint64_t lo = (uint64_t)a * (uint64_t)b;
  const uint64_t hi = (uint64_t)__mul64hi((long long)a, (long long)b);
  return ((u128)hi << 64) | lo;
}
// x * d modulo 2^128 for a signed 64-bit d (d sign-extended to 128 bits is
// du - 2^64 for d < 0, du = d modulo 2^64).
__device__ __forceinline__ u128 mul_u128_s64(u128 x, int64_t d) {
  const uint64_t xl = (uint64_t)x, xh = (uint64_t)(x >> 64), du = (uint64_t)d;
  uint64_t hi = __umul64hi(xl, du) + xh * du;
  if (d < 0) hi -= xl;
  return ((u128)hi << 64) | (xl * du);
}

// Integer images by cascaded sums -------------------------------------------
//
// For a row segment of n pixels I_0 .. I_{n-1}, running A_0 += I_i,
// A_1 += A_0, ..., A_K += A_{K-1} (each with the value just updated) leaves
// A_j = sum_i C(n-1-i+j, j) I_i, which is sum_w w^(j)/j! I with w = n - i and
// w^(j) the rising factorial.  Rising factorials expand in powers through the
// Stirling numbers of the second kind, w^b = sum_j (-1)^(b-j) S(b,j) w^(j),
// so Q_b = sum_w w^b I = sum_j (-1)^(b-j) S(b,j) j! A_j.  The signed image
// coordinate is c = f - off_f = D - w with D = f_start + n - off_f, and the
// row power sums F_b = sum (D - w)^b I follow from the Q_k by a binomial
// shift.  Every step is a ring operation, so all of it is exact modulo
// 2^128, and the 2-D moments, which fit in int128, come out exact.  Per pixel
// this costs K + 1 additions instead of K products.
//
// Pixels per segment at most: |A_j| <= max|I| * C(n + j, j + 1), which for
// n = 64 and |I| < 2^32 (or limb pixels of magnitude at most 2^31) stays
// below 2^63 up to j = 6, so A_0 .. A_6 run in signed 64-bit words.
constexpr int kSegLenMax = 64;
constexpr int kCascade64 = 7;  // cascade sums kept in 64 bits
static_assert(kSegLenMax <= 64, "the 64-bit cascade bound holds for segments of at most 64 pixels");
constexpr int kUnitThreads = 128;  // segments per CTA
// The segments of one CTA are consecutive in memory (rows follow each other),
// so the CTA first copies its pixels, at most kUnitThreads * kSegLenMax, into
// shared memory with coalesced loads; pixel i goes to word i + i / seg, which
// keeps the threads' sequential reads of their own segments on distinct banks.
constexpr int kStageWords = kUnitThreads * kSegLenMax + kUnitThreads;

__constant__ StirlingTable c_stirling = make_stirling();

// SGN: the pixels are two's complement int32 (the limb images of a float
// volume) instead of uint32.
template <int K, bool SGN>
__global__ void __launch_bounds__(kUnitThreads) k2_int_cascade_kernel(K2Params p) {
  constexpr int NB = K + 1;
  constexpr int CH = kUnitThreads / NB;  // unit chunks per power b in the fold
  const int blk = blockIdx.x;
  int kk = 0;
  while (kk + 1 < p.nimg && blk >= p.blk_base[kk + 1]) ++kk;
  const int k = kk % p.set.P, limb = kk / p.set.P;
  const int64_t chunk = blk - p.blk_base[kk];
  const int64_t S = p.set.S[k], F = p.set.F[k];
  const int64_t off_s = p.set.off_s[k], off_f = p.set.off_f[k];
  const int64_t seg = p.seg_len;
  const int lgseg = 31 - __clz((int)seg);  // seg is a power of two
  // segments per row; S * nseg < 2^31 (checked on the host), so the
  // divisions by nseg below run in 32 bits
  const uint32_t nseg = (uint32_t)((F + seg - 1) >> lgseg);
  const uint32_t* img =
      static_cast<const uint32_t*>(p.images) + p.set.base[k] + limb * p.set.total_elems;
  const int t = threadIdx.x;

  // limb images: the pixels at 8-byte aligned addresses carry kLimbPairBias
  auto unbias = [](const uint32_t* at, uint32_t v) -> uint32_t {
    return (SGN && (reinterpret_cast<uintptr_t>(at) & 4) == 0) ? v ^ kLimbPairBias : v;
  };
  // the staged pixels, and after the cascades the segments' power sums and
  // the fold partials in the same memory
  struct Sums {
    u128 Fs[kUnitThreads][NB];  // row power sums of each segment
    u128 part[NB][CH][NB];      // fold partials [b][chunk][a]
  };
  __shared__ union Smem {
    uint32_t stage[kStageWords];
    Sums sums;
  } sm;
  __shared__ int64_t Cs[kUnitThreads];  // each segment's signed row coordinate
  auto& Fs = sm.sums.Fs;
  auto& part = sm.sums.part;

  // 0. the CTA's pixels into shared memory (segments of more than 16
  // pixels; shorter ones, which only small image sets use, are read in
  // place, where the extra copy phase would only add latency)
  const bool staged = seg > 16;
  const int64_t units = S * nseg;
  const int64_t u_first = chunk * kUnitThreads;
  const int64_t u_last = (u_first + kUnitThreads < units ? u_first + kUnitThreads : units) - 1;
  int64_t p0, plen;
  {
    const int64_t s0 = (uint32_t)u_first / nseg, sl = (uint32_t)u_last / nseg;
    const int64_t gl = u_last - sl * nseg;
    p0 = s0 * F + (u_first - s0 * nseg) * seg;
    plen = sl * F + ((gl + 1) * seg < F ? (gl + 1) * seg : F) - p0;
  }
  if (staged) {
    // pixels up to the first 16-byte boundary and after the last one one by
    // one, the rest as 16-byte loads, all issued before they are stored
    const uint32_t* src = img + p0;
    int head = (int)((16 - (reinterpret_cast<uintptr_t>(src) & 15)) & 15) / 4;
    if (head > plen) head = (int)plen;
    const int nvec = (int)((plen - head) / 4);
    const int tail0 = head + 4 * nvec;
    auto put = [&](int i, uint32_t v) { sm.stage[i + (i >> lgseg)] = v; };
    if (t < head) put(t, unbias(src + t, __ldg(src + t)));
    if (tail0 + t < plen) put(tail0 + t, unbias(src + tail0 + t, __ldg(src + tail0 + t)));
    const uint4* vsrc = reinterpret_cast<const uint4*>(src + head);
    constexpr int kVecPerThread = kSegLenMax / 4;  // nvec <= kUnitThreads * kSegLenMax / 4
    constexpr int kBatch = 8;
#pragma unroll
    for (int j0 = 0; j0 < kVecPerThread; j0 += kBatch) {
      uint4 q[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int vi = t + (j0 + j) * kUnitThreads;
        if (vi < nvec) q[j] = __ldg(vsrc + vi);
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int vi = t + (j0 + j) * kUnitThreads;
        if (vi < nvec) {
          const int i = head + 4 * vi;
          // words 0 and 2 of an aligned 16-byte block are 8-byte aligned
          put(i, SGN ? q[j].x ^ kLimbPairBias : q[j].x);
          put(i + 1, q[j].y);
          put(i + 2, SGN ? q[j].z ^ kLimbPairBias : q[j].z);
          put(i + 3, q[j].w);
        }
      }
    }
  }
  __syncthreads();

  // 1. one segment per thread
  const int64_t u = u_first + t;
  u128 Fb[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) Fb[b] = 0;
  int64_t cs = 0;
  if (u < units) {
    const int64_t s = (uint32_t)u / nseg, g = u - s * nseg;
    const int64_t fs = g * seg;
    const int n = (int)(F - fs < seg ? F - fs : seg);
    const int o = (int)(s * F + fs - p0);  // the segment's first pixel in the stage
    const uint32_t* row = img + s * F + fs;
    constexpr int N64 = NB < kCascade64 ? NB : kCascade64;  // A_0 .. A_6 in 64 bits
    constexpr int N128 = NB > kCascade64 ? NB - kCascade64 : 1;
    uint64_t a64[N64];
    u128 a128[N128];
#pragma unroll
    for (int j = 0; j < N64; ++j) a64[j] = 0;
#pragma unroll
    for (int j = 0; j < N128; ++j) a128[j] = 0;
    auto step = [&](uint32_t px) {
      a64[0] += SGN ? (uint64_t)(int64_t)(int32_t)px : (uint64_t)px;
#pragma unroll
      for (int j = 1; j < N64; ++j) a64[j] += a64[j - 1];
      if constexpr (NB > kCascade64) {
        a128[0] += (u128)(i128)(int64_t)a64[kCascade64 - 1];
#pragma unroll
        for (int j = 1; j < NB - kCascade64; ++j) a128[j] += a128[j - 1];
      }
    };
    // eight loads ahead of their eight dependent cascade steps
    auto cascade = [&](auto pixel) {
      int i = 0;
      for (; i + 8 <= n; i += 8) {
        uint32_t q[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) q[j] = pixel(i + j);
#pragma unroll
        for (int j = 0; j < 8; ++j) step(q[j]);
      }
      for (; i < n; ++i) step(pixel(i));
    };
    if (staged) {
      cascade([&](int i) -> uint32_t {
        const int w = o + i;
        return sm.stage[w + (w >> lgseg)];
      });
    } else {
      cascade([&](int i) -> uint32_t { return unbias(row + i, __ldg(row + i)); });
    }
    u128 A[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j)
      A[j] = j < kCascade64 ? (u128)(i128)(int64_t)a64[j < kCascade64 ? j : 0]
                            : a128[j >= kCascade64 ? j - kCascade64 : 0];
    // Q_b = sum_j (-1)^(b-j) S(b,j) j! A_j, then the shift to c = D - w:
    // with m_k = (-1)^k Q_k, F_b = sum_k C(b,k) D^(b-k) m_k, built by the
    // Pascal recurrence m_b += D m_(b-1) applied K times
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      u128 q = 0;
#pragma unroll
      for (int j = 0; j <= b; ++j)
        q += j < kCascade64 ? mul_s64((int64_t)a64[j < kCascade64 ? j : 0], c_stirling.v[b][j])
                            : mul_u128_s64(A[j], c_stirling.v[b][j]);
      Fb[b] = (b & 1) ? (u128)0 - q : q;
    }
    const int64_t D = fs + n - off_f;
#pragma unroll
    for (int i = 1; i < NB; ++i)
#pragma unroll
      for (int b = NB - 1; b >= i; --b) Fb[b] += mul_u128_s64(Fb[b - 1], D);
    cs = s - off_s;
  }
  __syncthreads();  // every cascade has read the stage, which Fs overwrites
#pragma unroll
  for (int b = 0; b < NB; ++b) Fs[t][b] = Fb[b];
  Cs[t] = cs;
  __syncthreads();

  // 2. fold: thread (b, chunk c) takes a contiguous range of the CTA's
  // segments, sums the segments of each row, and adds s^a F_b(row) for
  // a <= K - b
  if (t < NB * CH) {
    const int b = t / CH, c = t - b * CH;
    constexpr int per = (kUnitThreads + CH - 1) / CH;
    const int u0 = c * per, u1 = (u0 + per < kUnitThreads) ? u0 + per : kUnitThreads;
    u128 T[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) T[a] = 0;
    auto fold = [&](u128 pw, int64_t srow) {

      T[0] += pw;
#pragma unroll
      for (int a = 1; a < NB; ++a) {
        if (a > K - b) break;
        pw = mul_u128_s64(pw, srow);
        T[a] += pw;
      }
    };
    if (u0 < u1) {
      u128 cur = Fs[u0][b];
      int64_t cur_s = Cs[u0];
      for (int uu = u0 + 1; uu < u1; ++uu) {
        if (Cs[uu] == cur_s) {
          cur += Fs[uu][b];
        } else {
          fold(cur, cur_s);
          cur = Fs[uu][b];
          cur_s = Cs[uu];
        }
      }
      fold(cur, cur_s);
    }
#pragma unroll
    for (int a = 0; a < NB; ++a) part[b][c][a] = T[a];
  }
  __syncthreads();

  // 3. pair (a, b), number n (n + 1) / 2 + b with n = a + b, sums the chunks
  for (int j = t; j < p.npairs; j += kUnitThreads) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= j) ++n;
    const int b = j - n * (n + 1) / 2, a = n - b;
    u128 acc = 0;
    for (int c = 0; c < CH; ++c) acc += part[b][c][a];
    if (p.m2d_atomic) atomic_add_u128(p.m2d_atomic + (int64_t)kk * p.npairs + j, acc);
    else static_cast<i128*>(p.partials)[(int64_t)blk * p.npairs + j] = (i128)acc;
  }
}

// float-float helpers -------------------------------------------------------

// Split a double pixel (raw bits) into float32 hi + lo with integer
// operations: hi is the mantissa rounded to 24 bits, lo the signed remainder
// (rounded to 24 bits, i.e. 2^-48 relative to hi).  Pixels outside the
// float32 exponent range are not produced by the projection of a float32
// volume whose values stay below 2^110.
__device__ __forceinline__ void f64_to_ff(unsigned long long b, float& hi, float& lo) {
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7ff);
  hi = 0.f;
  lo = 0.f;
  if (e == 0) return;  // zero (or a double far below the float range)
  const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);  // value = m * 2^(e-1075)
  unsigned long long mh = m >> 29;
  long long rem = (long long)(m & ((1ull << 29) - 1));
  if (rem >= (1ll << 28)) { mh += 1; rem -= (1ll << 29); }
  int eh = e - 1075 + 29;  // hi = mh * 2^eh
  if (mh == (1ull << 24)) { mh >>= 1; eh += 1; }
  const int bexp = eh + 23 + 127;
  if (bexp <= 0 || bexp >= 255) return;
  hi = __uint_as_float(sign | ((unsigned int)bexp << 23) | (unsigned int)(mh & 0x7fffffu));
  if (rem != 0) {
    const float r = __int2float_rn((int)rem);          // |rem| < 2^29
    const unsigned int rb = __float_as_uint(r);
    const int re = (int)((rb >> 23) & 0xff) + (e - 1075);  // scale by 2^(e-1075)
    if (re > 0 && re < 255) lo = __uint_as_float((rb & 0x807fffffu) ^ sign | ((unsigned int)re << 23));
  }
}

// (hi, lo) * c for a float c whose products stay finite.
__device__ __forceinline__ void ff_mul_f(float hi, float lo, float c, float& rh, float& rl) {
  float p, e;
  two_prod(hi, c, p, e);
  e = __fmaf_rn(lo, c, e);
  rh = __fadd_rn(p, e);
  rl = __fsub_rn(e, __fsub_rn(rh, p));
}

// Float images: one thread per row segment (the layout of the integer
// kernel).  The double pixels are split into float pairs with integer
// operations; F_b of the segment accumulates in float-float (the power
// chain I c^b by the FMA-based TwoProd); the CTA sums the segments of each
// row in float-float and folds s^a F_b.
template <int K>
__global__ void __launch_bounds__(kUnitThreads) k2_f32_seg_kernel(K2Params p) {
  if (p.gate && (*p.gate & 3) == 0) return;
  constexpr int NB = K + 1;
  constexpr int CH = kUnitThreads / NB;
  const int blk = blockIdx.x;
  int k = 0;
  while (k + 1 < p.nimg && blk >= p.blk_base[k + 1]) ++k;
  const int64_t chunk = blk - p.blk_base[k];
  const int64_t S = p.set.S[k], F = p.set.F[k];
  const int64_t off_s = p.set.off_s[k], off_f = p.set.off_f[k];
  const int64_t seg = p.seg_len;
  const int64_t nseg = (F + seg - 1) / seg;
  const unsigned long long* img = static_cast<const unsigned long long*>(p.images) + p.set.base[k];
  const int t = threadIdx.x;

  __shared__ float2 Fs[kUnitThreads][NB];
  __shared__ int64_t Cs[kUnitThreads];
  __shared__ float2 part[NB][CH][NB];

  // 1. one segment per thread
  float Fh[NB], Fl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) { Fh[b] = 0.f; Fl[b] = 0.f; }
  const int64_t u = chunk * kUnitThreads + t;
  int64_t cs = 0;
  if (u < S * nseg) {
    const int64_t s = u / nseg, g = u - s * nseg;
    const int64_t fs = g * seg;
    const int n = (int)(F - fs < seg ? F - fs : seg);
    const unsigned long long* row = img + s * F + fs;
    for (int i = 0; i < n; ++i) {
      float th, tl;
      f64_to_ff(__ldg(row + i), th, tl);
      if (th == 0.f && tl == 0.f) continue;
      const float c = (float)(fs + i - off_f);
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        ff_add(Fh[b], Fl[b], th, tl);
        if (b < K) ff_mul_f(th, tl, c, th, tl);
      }
    }
    cs = s - off_s;
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) Fs[t][b] = make_float2(Fh[b], Fl[b]);
  Cs[t] = cs;
  __syncthreads();

  // 2. fold: thread (b, chunk c) takes a contiguous range of segments, sums
  // the segments of each row, and adds s^a F_b(row) for a <= K - b
  if (t < NB * CH) {
    const int b = t / CH, c = t - b * CH;
    constexpr int per = (kUnitThreads + CH - 1) / CH;
    const int u0 = c * per, u1 = (u0 + per < kUnitThreads) ? u0 + per : kUnitThreads;
    float Th[NB], Tl[NB];
#pragma unroll
    for (int a = 0; a < NB; ++a) { Th[a] = 0.f; Tl[a] = 0.f; }
    auto fold = [&](float ph, float pl, int64_t srow) {
      const float sv = (float)srow;
      ff_add(Th[0], Tl[0], ph, pl);
#pragma unroll
      for (int a = 1; a < NB; ++a) {
        if (a > K - b) break;
        ff_mul_f(ph, pl, sv, ph, pl);
        ff_add(Th[a], Tl[a], ph, pl);
      }
    };
    if (u0 < u1) {
      float ch = Fs[u0][b].x, cl = Fs[u0][b].y;
      int64_t cur_s = Cs[u0];
      for (int uu = u0 + 1; uu < u1; ++uu) {
        if (Cs[uu] == cur_s) {
          ff_add(ch, cl, Fs[uu][b].x, Fs[uu][b].y);
        } else {
          fold(ch, cl, cur_s);
          ch = Fs[uu][b].x;
          cl = Fs[uu][b].y;
          cur_s = Cs[uu];
        }
      }
      fold(ch, cl, cur_s);
    }
#pragma unroll
    for (int a = 0; a < NB; ++a) part[b][c][a] = make_float2(Th[a], Tl[a]);
  }
  __syncthreads();

  // 3. pair (a, b), number n (n + 1) / 2 + b with n = a + b, sums the chunks
  for (int j = t; j < p.npairs; j += kUnitThreads) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= j) ++n;
    const int b = j - n * (n + 1) / 2, a = n - b;
    float ah = 0.f, al = 0.f;
    for (int c = 0; c < CH; ++c) ff_add(ah, al, part[b][c][a].x, part[b][c][a].y);
    static_cast<float2*>(p.partials)[(int64_t)blk * p.npairs + j] = make_float2(ah, al);
  }
}

// Pixels per row segment: 16 .. 64, the largest power of two that still
// gives about 78 K segments (16 warps per SM) over all images of all nl limb
// sets (measured at 512^3, K = 6: float32 limbs 46.7 -> 37.5 us with the
// eight-load prefetch, uint16 28.7 -> 27.0 us).
int int_seg_len(const ImageSet& set, int nl) {
  int64_t pixels = 0;
  for (int k = 0; k < set.P; ++k) pixels += set.S[k] * set.F[k] * nl;
  int seg = kSegLenMax;
  while (seg > 16 && pixels / seg < 152 * 16 * 32) seg >>= 1;
  return seg;
}

// CTAs of step 2 per image: kUnitThreads row segments per CTA; nl limb sets
// of the P images (image i is image i % P of limb i / P).
int64_t blocks_of(const ImageSet& set, int nl, int64_t* base) {
  const int64_t seg = int_seg_len(set, nl);
  int64_t at = 0;
  for (int i = 0; i < nl * set.P; ++i) {
    const int k = i % set.P;
    if (base) base[i] = at;
    const int64_t units = set.S[k] * ((set.F[k] + seg - 1) / seg);
    at += (units + kUnitThreads - 1) / kUnitThreads;
  }
  if (base) base[nl * set.P] = at;
  return at;
}

}  // namespace

size_t moments2d_partials_bytes(const ImageSet& set, int K, bool is_float) {
  return (size_t)blocks_of(set, 1, nullptr) * num_2d(K) *
         (is_float ? sizeof(float2) : sizeof(i128));
}

size_t moments2d_partials_bytes_limbs(const ImageSet& set, int K, int nl) {
  return (size_t)blocks_of(set, nl, nullptr) * num_2d(K) * sizeof(i128);
}

// defined in k3_combine.cu: sums the block partials into per-image moments
cudaError_t launch_reduce_partials(const void* partials, const int64_t* blk_base, int nimg, int K,
                                   bool is_float, void* m2d, cudaStream_t st, const int* gate);

namespace {
cudaError_t launch_k2(const void* images, const ImageSet& set, int K, bool is_float, int nl,
                      bool sgn, void* partials, void* m2d, cudaStream_t st, const int* gate,
                      bool m2d_zeroed) {
  K2Params p{};
  p.gate = gate;
  const bool atomic = m2d_zeroed && !is_float;
  p.m2d_atomic = atomic ? static_cast<i128*>(m2d) : nullptr;
  p.images = images;
  p.set = set;
  p.nimg = nl * set.P;
  p.K = K;
  p.npairs = num_2d(K);
  p.seg_len = int_seg_len(set, nl);
  // the kernels divide segment numbers (S * nseg of them per image) in 32 bits
  for (int k = 0; k < set.P; ++k)
    if (set.S[k] * ((set.F[k] + p.seg_len - 1) / p.seg_len) >= ((int64_t)1 << 31))
      return cudaErrorInvalidValue;
  const int64_t nblk = blocks_of(set, nl, p.blk_base);
  p.partials = partials;
  const unsigned g = (unsigned)nblk;
  switch (K) {
#define DPMA_K2_CASE(k)                                                              \
  case k:                                                                            \
    if (is_float) k2_f32_seg_kernel<k><<<g, kUnitThreads, 0, st>>>(p);               \
    else if (sgn) k2_int_cascade_kernel<k, true><<<g, kUnitThreads, 0, st>>>(p);     \
    else k2_int_cascade_kernel<k, false><<<g, kUnitThreads, 0, st>>>(p);             \
    break;
    DPMA_K2_CASE(0) DPMA_K2_CASE(1) DPMA_K2_CASE(2) DPMA_K2_CASE(3) DPMA_K2_CASE(4)
    DPMA_K2_CASE(5) DPMA_K2_CASE(6) DPMA_K2_CASE(7) DPMA_K2_CASE(8)
#undef DPMA_K2_CASE
#define DPMA_K2_INT_CASE(k)                                                          \
  case k:                                                                            \
    if (is_float) return cudaErrorInvalidValue;                                      \
    if (sgn) k2_int_cascade_kernel<k, true><<<g, kUnitThreads, 0, st>>>(p);          \
    else k2_int_cascade_kernel<k, false><<<g, kUnitThreads, 0, st>>>(p);             \
    break;
    DPMA_K2_INT_CASE(9) DPMA_K2_INT_CASE(10)
#undef DPMA_K2_INT_CASE
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || atomic) return e;
  return launch_reduce_partials(partials, p.blk_base, p.nimg, K, is_float, m2d, st, gate);
}
}  // namespace

cudaError_t launch_image_moments(const void* images, const ImageSet& set, int K, bool is_float,
                                 void* partials, void* m2d, cudaStream_t st, const int* gate,
                                 bool m2d_zeroed) {
  return launch_k2(images, set, K, is_float, 1, false, partials, m2d, st, gate, m2d_zeroed);
}

cudaError_t launch_image_moments_limbs(const void* images, const ImageSet& set, int64_t limb_stride,
                                       int K, int nl, void* partials, void* m2d, cudaStream_t st,
                                       bool m2d_zeroed) {
  ImageSet s2 = set;
  s2.total_elems = limb_stride;  // the kernel steps from limb to limb by total_elems
  return launch_k2(images, s2, K, false, nl, true, partials, m2d, st, nullptr, m2d_zeroed);
}

}  // namespace dpma
