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
// One warp handles one image row: lanes stride over the row (four loads in
// flight per lane) and accumulate F_b for b = 0..K, a butterfly reduction
// gives every lane the row totals, and lane t then adds (s - off_s)^a F_b
// for the (a, b) pairs it owns.  A CTA covers kRowsPerBlock = 8 rows of one
// image, so a 512^3 volume's seven images give ~450 CTAs; each CTA writes
// one partial vector and a small kernel sums the partials per image.
// Integer images accumulate exactly in int128; float images (doubles) are
// split into float32 pairs with integer operations and accumulate in
// float-float, so no FP64 arithmetic happens here.
#include <cstdint>

#include "dpma_internal.cuh"

namespace dpma {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRowsPerBlock = kWarps;  // one image row per warp

struct K2Params {
  const void* images;
  ImageSet set;
  int K;
  int npairs;
  int64_t blk_base[kMaxImages + 1];  // first block of each image; [P] = total
  void* partials;                    // [block][npairs] int128 or float2
};

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int m) {
  unsigned long long lo = (unsigned long long)(u128)v;
  unsigned long long hi = (unsigned long long)((u128)v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, m);
  hi = __shfl_xor_sync(0xffffffffu, hi, m);
  return (i128)(((u128)hi << 64) | lo);
}

template <int K>
__global__ void __launch_bounds__(kThreads) k2_int_kernel(K2Params p) {
  const int blk = blockIdx.x;
  int k = 0;
  while (k + 1 < p.set.P && blk >= p.blk_base[k + 1]) ++k;
  const int64_t chunk = blk - p.blk_base[k];
  const int64_t S = p.set.S[k], F = p.set.F[k];
  const int64_t off_s = p.set.off_s[k], off_f = p.set.off_f[k];
  const uint32_t* img = static_cast<const uint32_t*>(p.images) + p.set.base[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // pairs owned by this lane: index lane and lane + 32
  int pa[2], pb[2];
  for (int t = 0; t < 2; ++t) {
    int idx = lane + 32 * t;
    pa[t] = -1; pb[t] = -1;
    if (idx < p.npairs) {
      int n = 0;
      while ((n + 1) * (n + 2) / 2 <= idx) ++n;
      int a = n - (idx - n * (n + 1) / 2);
      pa[t] = a; pb[t] = n - a;
    }
  }
  i128 T[2] = {0, 0};

  const int64_t r0 = chunk * kRowsPerBlock;
  const int64_t r1 = (r0 + kRowsPerBlock < S) ? r0 + kRowsPerBlock : S;
  for (int64_t s = r0 + warp; s < r1; s += kWarps) {
    i128 Fb[K + 1];
#pragma unroll
    for (int b = 0; b <= K; ++b) Fb[b] = 0;
    const uint32_t* row = img + s * F;
    for (int64_t f0 = lane; f0 < F; f0 += 4 * 32) {
      uint32_t vv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t f = f0 + q * 32;
        vv[q] = f < F ? __ldg(row + f) : 0u;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!vv[q]) continue;
        const int64_t c = f0 + q * 32 - off_f;
        i128 t = (i128)vv[q];
#pragma unroll
        for (int b = 0; b <= K; ++b) {
          Fb[b] += t;
          if (b < K) t *= (i128)c;
        }
      }
    }
#pragma unroll
    for (int b = 0; b <= K; ++b) {
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) Fb[b] += shfl_xor_i128(Fb[b], m);
    }
    const i128 cs = (i128)(s - off_s);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (pa[t] < 0) continue;
      i128 w = 1;
      for (int e = 0; e < pa[t]; ++e) w *= cs;
      i128 fb = 0;
#pragma unroll
      for (int b = 0; b <= K; ++b)
        if (b == pb[t]) fb = Fb[b];
      T[t] += w * fb;
    }
  }

  // reduce the kWarps partial vectors of this CTA
  __shared__ i128 red[kWarps][64];
  red[warp][lane] = T[0];
  red[warp][lane + 32] = T[1];
  __syncthreads();
  if (warp == 0) {
    for (int t = 0; t < 2; ++t) {
      const int idx = lane + 32 * t;
      if (idx >= p.npairs) continue;
      i128 acc = 0;
      for (int w = 0; w < kWarps; ++w) acc += red[w][idx];
      static_cast<i128*>(p.partials)[(int64_t)blk * p.npairs + idx] = acc;
    }
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

template <int K>
__global__ void __launch_bounds__(kThreads) k2_f32_kernel(K2Params p) {
  const int blk = blockIdx.x;
  int k = 0;
  while (k + 1 < p.set.P && blk >= p.blk_base[k + 1]) ++k;
  const int64_t chunk = blk - p.blk_base[k];
  const int64_t S = p.set.S[k], F = p.set.F[k];
  const int64_t off_s = p.set.off_s[k], off_f = p.set.off_f[k];
  const unsigned long long* plane = static_cast<const unsigned long long*>(p.images) + p.set.base[k];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int pa[2], pb[2];
  for (int t = 0; t < 2; ++t) {
    int idx = lane + 32 * t;
    pa[t] = -1; pb[t] = -1;
    if (idx < p.npairs) {
      int n = 0;
      while ((n + 1) * (n + 2) / 2 <= idx) ++n;
      int a = n - (idx - n * (n + 1) / 2);
      pa[t] = a; pb[t] = n - a;
    }
  }
  float Th[2] = {0.f, 0.f}, Tl[2] = {0.f, 0.f};

  const int64_t r0 = chunk * kRowsPerBlock;
  const int64_t r1 = (r0 + kRowsPerBlock < S) ? r0 + kRowsPerBlock : S;
  for (int64_t s = r0 + warp; s < r1; s += kWarps) {
    float Fh[K + 1], Fl[K + 1];
#pragma unroll
    for (int b = 0; b <= K; ++b) { Fh[b] = 0.f; Fl[b] = 0.f; }
    const unsigned long long* row = plane + s * F;
    for (int64_t f0 = lane; f0 < F; f0 += 4 * 32) {
      unsigned long long raw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t f = f0 + q * 32;
        raw[q] = f < F ? __ldg(row + f) : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float th, tl;
        f64_to_ff(raw[q], th, tl);
        if (th == 0.f && tl == 0.f) continue;
        const float c = (float)(f0 + q * 32 - off_f);
#pragma unroll
        for (int b = 0; b <= K; ++b) {
          ff_add(Fh[b], Fl[b], th, tl);
          if (b < K) ff_mul_f(th, tl, c, th, tl);
        }
      }
    }
#pragma unroll
    for (int b = 0; b <= K; ++b) {
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) {
        float oh = __shfl_xor_sync(0xffffffffu, Fh[b], m);
        float ol = __shfl_xor_sync(0xffffffffu, Fl[b], m);
        ff_add(Fh[b], Fl[b], oh, ol);
      }
    }
    const float cs = (float)(s - off_s);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (pa[t] < 0) continue;
      float fh = 0.f, fl = 0.f;
#pragma unroll
      for (int b = 0; b <= K; ++b)
        if (b == pb[t]) { fh = Fh[b]; fl = Fl[b]; }
      for (int e = 0; e < pa[t]; ++e) ff_mul_f(fh, fl, cs, fh, fl);
      ff_add(Th[t], Tl[t], fh, fl);
    }
  }

  __shared__ float2 red[kWarps][64];
  red[warp][lane] = make_float2(Th[0], Tl[0]);
  red[warp][lane + 32] = make_float2(Th[1], Tl[1]);
  __syncthreads();
  if (warp == 0) {
    for (int t = 0; t < 2; ++t) {
      const int idx = lane + 32 * t;
      if (idx >= p.npairs) continue;
      float ah = 0.f, al = 0.f;
      for (int w = 0; w < kWarps; ++w) ff_add(ah, al, red[w][idx].x, red[w][idx].y);
      static_cast<float2*>(p.partials)[(int64_t)blk * p.npairs + idx] = make_float2(ah, al);
    }
  }
}

int64_t blocks_of(const ImageSet& set, int64_t* base) {
  int64_t at = 0;
  for (int k = 0; k < set.P; ++k) {
    if (base) base[k] = at;
    at += (set.S[k] + kRowsPerBlock - 1) / kRowsPerBlock;
  }
  if (base) base[set.P] = at;
  return at;
}

}  // namespace

size_t moments2d_partials_bytes(const ImageSet& set, int K, bool is_float) {
  return (size_t)blocks_of(set, nullptr) * num_2d(K) * (is_float ? sizeof(float2) : sizeof(i128));
}

// defined in k3_combine.cu: sums the block partials into per-image moments
cudaError_t launch_reduce_partials(const void* partials, const int64_t* blk_base, int P, int K,
                                   bool is_float, void* m2d, cudaStream_t st);

cudaError_t launch_image_moments(const void* images, const ImageSet& set, int K, bool is_float,
                                 void* partials, void* m2d, cudaStream_t st) {
  K2Params p{};
  p.images = images;
  p.set = set;
  p.K = K;
  p.npairs = num_2d(K);
  const int64_t nblk = blocks_of(set, p.blk_base);
  p.partials = partials;
  switch (K) {
#define DPMA_K2_CASE(k)                                                   \
  case k:                                                                 \
    if (is_float) k2_f32_kernel<k><<<(unsigned)nblk, kThreads, 0, st>>>(p); \
    else k2_int_kernel<k><<<(unsigned)nblk, kThreads, 0, st>>>(p);          \
    break;
    DPMA_K2_CASE(0) DPMA_K2_CASE(1) DPMA_K2_CASE(2) DPMA_K2_CASE(3) DPMA_K2_CASE(4)
    DPMA_K2_CASE(5) DPMA_K2_CASE(6) DPMA_K2_CASE(7) DPMA_K2_CASE(8)
#undef DPMA_K2_CASE
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(partials, p.blk_base, set.P, K, is_float, m2d, st);
}

}  // namespace dpma
