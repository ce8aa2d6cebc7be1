// Batched moments of many small volumes (regions of interest) in one
// persistent launch.
//
// The three steps of the Discrete Projection Moment method (Sec. 3: the
// images of Eq. 4 / Eqs. 5-9 and the +-pi/4 families, their 2-D moments by
// Eq. 1 with the origin shift of Sec. 5, and the exact combine of Eqs. 10-16
// generalised) run for every volume of the batch, but the first two are
// fused and kept on chip: a persistent CTA takes one volume at a time from a
// device work queue (largest first), builds all of its images in shared
// memory and reduces them to 2-D moments there; only the 2-D moments reach
// global memory.  One more launch combines them for every volume.
//
// Inside a CTA each warp owns image rows y (y = warp, warp + NW, ...) of every
// z-slice, so the images whose pixels stay within one row (0, 1, 3, 4) are
// updated with plain shared-memory read-modify-writes ordered by __syncwarp;
// the others (2, 5, 6, 7, 8) use shared-memory atomic adds.  Pixels are 16-bit
// when the longest line times the largest voxel value stays below 2^16 (two
// pixels per 32-bit word; an atomic add of v << 16 never carries into the
// neighbour because the sum is bounded), 32-bit otherwise.
//
// Volumes the fused kernel does not take (float32, rows wider than 256, or
// images larger than the shared-memory budget) run through the single-volume
// pipeline on the same stream, one after another.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dpma.h"
#include "batch_internal.cuh"
#include "dpma_internal.cuh"

namespace dpma {
cudaError_t prepare_combine(int K);
size_t pack_combine_plan(int K, int64_t* words, size_t capacity, int off[kMaxK + 1]);
void set_last_error(const char* msg);
}  // namespace dpma

using namespace dpma;
using dpma::batch::BTask;

namespace {

constexpr int kMaxXSlots = 8;            // fused path: L <= 256 (8 x-values per lane)
constexpr int kMaxWarps = 16;            // up to 512 threads per CTA
constexpr int kPartBytes = kMaxWarps * kMax2D * 16;  // per-warp 2-D moment partials
constexpr int kSmemLimit = 227 * 1024;
constexpr int kStatusInternal = 7;


struct FusedParams {
  const BTask* tasks;
  const int* order;  // processing order (largest first)
  int ntasks;
  int* counter;      // work queue head (zeroed before each run)
  i128* T;           // 2-D moments of every volume
};

// ---------------------------------------------------------------- pixels

template <bool WIDE>
__device__ __forceinline__ void pix_add(uint32_t* sm, int idx, uint32_t v) {
  if constexpr (WIDE) {
    sm[idx] += v;
  } else {
    uint16_t* p = reinterpret_cast<uint16_t*>(sm);
    p[idx] = (uint16_t)(p[idx] + v);
  }
}
template <bool WIDE>
__device__ __forceinline__ void pix_atomic(uint32_t* sm, int idx, uint32_t v) {
  if constexpr (WIDE) atomicAdd(sm + idx, v);
  else atomicAdd(sm + (idx >> 1), v << (16 * (idx & 1)));
}
template <bool WIDE>
__device__ __forceinline__ uint32_t pix_get(const uint32_t* sm, int idx) {
  if constexpr (WIDE) return sm[idx];
  else return reinterpret_cast<const uint16_t*>(sm)[idx];
}

// ---------------------------------------------------------------- step 1

// Every image of one volume into shared memory (Eq. 4 for the image table of
// dpma.h): warp w handles rows y = w, w + NW, ... of each z-slice, lane l the
// columns x = l + 32k.
template <typename T, bool WIDE, int NT>
__device__ void project_volume(const BTask& t, uint32_t* sm) {
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* __restrict__ vol = static_cast<const T*>(t.vol);
  const int L = t.L, M = t.M, N = t.N, P = t.P;
  const int F3 = L + N - 1, F7 = L + M - 1;
  const int nxs = (L + 31) >> 5;
  const int* o = t.img_off;
  for (int z = 0; z < N; ++z) {
    uint32_t col[kMaxXSlots];
#pragma unroll
    for (int k = 0; k < kMaxXSlots; ++k) col[k] = 0;
    for (int y = warp; y < M; y += NW) {
      const T* row = vol + ((size_t)z * M + y) * L;
      uint32_t rsum = 0;
#pragma unroll
      for (int k = 0; k < kMaxXSlots; ++k) {
        const int x = lane + 32 * k;
        if (k < nxs && x < L) {
          const uint32_t v = row[x];
          if (v) {
            rsum += v;
            col[k] += v;
            pix_add<WIDE>(sm, o[0] + y * L + x, v);                          // (y, x)
            if (P > 3) pix_add<WIDE>(sm, o[3] + y * F3 + x + z, v);          // (y, x+z)
            if (P > 4) pix_add<WIDE>(sm, o[4] + y * F3 + x - z + N - 1, v);  // (y, x-z)
            if (P > 5) pix_atomic<WIDE>(sm, o[5] + (y + z) * L + x, v);      // (y+z, x)
            if (P > 6) pix_atomic<WIDE>(sm, o[6] + (y - z + N - 1) * L + x, v);
            if (P > 7) pix_atomic<WIDE>(sm, o[7] + z * F7 + x + y, v);      // (z, x+y)
            if (P > 8) pix_atomic<WIDE>(sm, o[8] + z * F7 + x - y + M - 1, v);
          }
        }
      }
      rsum = __reduce_add_sync(0xffffffffu, rsum);
      if (lane == 0 && rsum) pix_add<WIDE>(sm, o[1] + z * M + y, rsum);  // (z, y)
      __syncwarp();  // row y's pixels of images 3 and 4 move between lanes with z
    }
#pragma unroll
    for (int k = 0; k < kMaxXSlots; ++k) {
      const int x = lane + 32 * k;
      if (k < nxs && x < L && col[k]) pix_atomic<WIDE>(sm, o[2] + z * L + x, col[k]);  // (z, x)
    }
  }
}

// ---------------------------------------------------------------- step 2

__device__ __forceinline__ int64_t shfl_xor_i64(int64_t v, int m) {
  return __shfl_xor_sync(0xffffffffu, (long long)v, m);
}
__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int m) {
  const uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
  const uint64_t l2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)lo, m);
  const uint64_t h2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)hi, m);
  return (i128)(((u128)h2 << 64) | l2);
}
template <typename RT>
__device__ __forceinline__ RT warp_sum(RT v) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    if constexpr (sizeof(RT) == 8) v += shfl_xor_i64(v, m);
    else v += shfl_xor_i128(v, m);
  }
  return v;
}

// 2-D moments T_ab (a + b <= K, signed coordinates) of one image held in
// shared memory (Eq. 1): per row s, the power sums R_b(s) = sum_f I f^b, then
// T_ab = sum_s s^a R_b(s).  Lane j accumulates pairs j and j + 32.
template <typename RT, bool WIDE, int NT>
__device__ void image_moments(const uint32_t* sm, int base, int64_t S, int64_t F, int64_t off_s,
                              int64_t off_f, int K, i128* part, i128* Tout) {
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int npairs = (K + 1) * (K + 2) / 2;
  // the (a, b) of this lane's pairs
  int ja[2], jb[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    int n = 0;
    while ((n + 1) * (n + 2) / 2 <= j) ++n;
    ja[h] = n - (j - n * (n + 1) / 2);
    jb[h] = n - ja[h];
  }
  i128 acc[2] = {0, 0};
  for (int64_t s = warp; s < S; s += NW) {
    RT R[kMaxK + 1];
#pragma unroll
    for (int b = 0; b <= kMaxK; ++b) R[b] = 0;
    for (int64_t f = lane; f < F; f += 32) {
      const uint32_t v = pix_get<WIDE>(sm, base + (int)(s * F + f));
      if (v) {
        const RT fs = (RT)(f - off_f);
        RT pw = (RT)v;
#pragma unroll
        for (int b = 0; b <= kMaxK; ++b) {
          if (b > K) break;
          R[b] += pw;
          pw *= fs;
        }
      }
    }
    bool any = false;
#pragma unroll
    for (int b = 0; b <= kMaxK; ++b) {
      if (b > K) break;
      R[b] = warp_sum<RT>(R[b]);
      any = any || R[b] != 0;
    }
    if (!any) continue;
    const i128 ss = (i128)(s - off_s);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (lane + 32 * h >= npairs) continue;
      i128 sp = 1;
      for (int a = 0; a < ja[h]; ++a) sp *= ss;
      RT rb = 0;
#pragma unroll
      for (int b = 0; b <= kMaxK; ++b)
        if (b == jb[h]) rb = R[b];
      acc[h] += sp * (i128)rb;
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (lane + 32 * h < npairs) part[warp * kMax2D + lane + 32 * h] = acc[h];
  __syncthreads();
  for (int j = threadIdx.x; j < npairs; j += NT) {
    i128 sum = 0;
    for (int w = 0; w < NW; ++w) sum += part[w * kMax2D + j];
    Tout[j] = sum;
  }
  __syncthreads();
}

template <typename T, bool WIDE, int NT>
__device__ void run_task(const BTask& t, uint32_t* sm, i128* part, i128* Tout) {
  project_volume<T, WIDE, NT>(t, sm);
  __syncthreads();
  const int npairs = (t.K + 1) * (t.K + 2) / 2;
  for (int k = 0; k < t.P; ++k) {
    // geometry of image k (the table of dpma.h)
    const int64_t L = t.L, M = t.M, N = t.N;
    int64_t S, F, os = 0, of = 0;
    switch (k) {
      case 0: S = M; F = L; break;
      case 1: S = N; F = M; break;
      case 2: S = N; F = L; break;
      case 3: S = M; F = L + N - 1; break;
      case 4: S = M; F = L + N - 1; of = N - 1; break;
      case 5: S = M + N - 1; F = L; break;
      case 6: S = M + N - 1; F = L; os = N - 1; break;
      case 7: S = N; F = L + M - 1; break;
      default: S = N; F = L + M - 1; of = M - 1; break;
    }
    if (t.r64) image_moments<int64_t, WIDE, NT>(sm, t.img_off[k], S, F, os, of, t.K, part, Tout + k * npairs);
    else image_moments<i128, WIDE, NT>(sm, t.img_off[k], S, F, os, of, t.K, part, Tout + k * npairs);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) batch_fused_kernel(FusedParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  i128* part = reinterpret_cast<i128*>(smem_raw);
  uint32_t* sm = reinterpret_cast<uint32_t*>(smem_raw + kPartBytes);
  __shared__ int s_task;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(p.counter, 1);
    __syncthreads();
    const int ti = s_task;
    if (ti >= p.ntasks) break;
    const BTask t = p.tasks[p.order[ti]];
    for (int w = threadIdx.x; w < t.words; w += NT) sm[w] = 0;
    __syncthreads();
    i128* Tout = p.T + t.t_off;
    if (t.dtype == DPMA_U8) {
      if (t.wide) run_task<uint8_t, true, NT>(t, sm, part, Tout);
      else run_task<uint8_t, false, NT>(t, sm, part, Tout);
    } else {
      if (t.wide) run_task<uint16_t, true, NT>(t, sm, part, Tout);
      else run_task<uint16_t, false, NT>(t, sm, part, Tout);
    }
    // run_task ends with a barrier: s_task may be rewritten
  }
}

// ---------------------------------------------------------------- step 3

struct BCombParams {
  const BTask* tasks;
  int ntasks;
  const int64_t* plans;        // packed plans of every K present
  int off[kMaxK + 1][kMaxK + 1];  // off[K][n]: word offset of degree n of order K
  const i128* T;
  unsigned char* out;
  int* status;
};

struct I256 { uint64_t w[4]; };

__device__ __forceinline__ void neg256(I256& a) {
  uint64_t carry = 1;
  for (int i = 0; i < 4; ++i) {
    const uint64_t v = ~a.w[i] + carry;
    carry = (carry && v == 0) ? 1 : 0;
    a.w[i] = v;
  }
}
__device__ __forceinline__ void add256(I256& a, const I256& b) {
  unsigned long long carry = 0;
  for (int i = 0; i < 4; ++i) {
    const u128 s = (u128)a.w[i] + b.w[i] + carry;
    a.w[i] = (uint64_t)s;
    carry = (unsigned long long)(s >> 64);
  }
}
// a += c * t (c: int64, t: int128), exact in 256 bits
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
// q = a / d exactly; false on a remainder or if q leaves int128
__device__ bool div256_exact(I256 a, int64_t d, i128* q) {
  const bool neg = (a.w[3] >> 63) != 0;
  if (neg) neg256(a);
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

// One thread per (volume, moment): M = (C t_sel) / D for the moment's degree.
__global__ void batch_combine_kernel(BCombParams p) {
  constexpr int kStride = 165;  // moments of order 8
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ti = gid / kStride;
  const int m = (int)(gid % kStride);
  if (ti >= p.ntasks) return;
  const BTask& t = p.tasks[ti];
  const int K = t.K;
  if (m >= (K + 1) * (K + 2) * (K + 3) / 6) return;
  int n = 0;
  while ((n + 1) * (n + 2) * (n + 3) / 6 <= m) ++n;
  const int row = m - n * (n + 1) * (n + 2) / 6;
  const int64_t* pl = p.plans + p.off[K][n];
  const int64_t D = pl[0];
  const int nm = (int)pl[1];
  const int64_t* img = pl + 2;
  const int64_t* aa = img + nm;
  const int64_t* C = aa + nm;
  const int npairs = (K + 1) * (K + 2) / 2;
  const i128* T = p.T + t.t_off;
  I256 acc = {{0, 0, 0, 0}};
  for (int j = 0; j < nm; ++j) {
    const int a = (int)aa[j];
    const int pair = n * (n + 1) / 2 + (n - a);
    mac256(acc, C[row * nm + j], T[img[j] * npairs + pair]);
  }
  i128 q = 0;
  if (!div256_exact(acc, D, &q)) {
    atomicMax(p.status, kStatusInternal);
    q = 0;
  }
  reinterpret_cast<i128*>(p.out + t.out_off)[m] = q;
}

// Folds a single-volume run's device status into the batch's.
__global__ void merge_status_kernel(const int* src, int* dst) {
  if (*src) atomicMax(dst, *src);
}

// ---------------------------------------------------------------- host side

dpma_status bfail(dpma_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

// Upper bound on the voxels one pixel sums (the longest line of any image).
int64_t longest_line(int64_t L, int64_t M, int64_t N) { return std::max({N, L, M}); }

template <int NT>
cudaError_t set_smem(size_t smem) {
  return cudaFuncSetAttribute(batch_fused_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

struct DevPlans {
  int64_t* words = nullptr;
  int off[kMaxK + 1][kMaxK + 1] = {};
};
std::mutex g_plans_mu;
std::vector<DevPlans> g_plans;  // per device

cudaError_t plans_for_device(const DevPlans** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_plans_mu);
  if ((int)g_plans.size() <= dev) g_plans.resize(dev + 1);
  DevPlans& dp = g_plans[dev];
  if (!dp.words) {
    std::vector<int64_t> words;
    for (int K = 0; K <= kMaxK; ++K) {
      std::vector<int64_t> w(8192);
      int off[kMaxK + 1];
      const size_t n = pack_combine_plan(K, w.data(), w.size(), off);
      if (n == 0) return cudaErrorInvalidValue;
      for (int d = 0; d <= kMaxK; ++d) dp.off[K][d] = (int)words.size() + off[d];
      words.insert(words.end(), w.begin(), w.begin() + n);
    }
    int64_t* dw = nullptr;
    e = cudaMalloc(&dw, sizeof(int64_t) * words.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(dw, words.data(), sizeof(int64_t) * words.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(dw); return e; }
    dp.words = dw;
  }
  *out = &dp;
  return cudaSuccess;
}

}  // namespace

namespace dpma {
namespace batch {

void classify(const dpma_volume_desc* descs, int count, Classified* c) {
  *c = Classified{};
  for (int i = 0; i < count; ++i) {
    const dpma_volume_desc& d = descs[i];
    const int P = num_images(d.K);
    bool fused = d.dtype != DPMA_F32 && d.L <= 32 * kMaxXSlots;
    BTask t{};
    if (fused) {
      const double vmax = d.dtype == DPMA_U8 ? 255.0 : 65535.0;
      const int64_t line = longest_line(d.L, d.M, d.N);
      t.wide = vmax * (double)line >= 65536.0 ? 1 : 0;
      int64_t pix = 0, maxF = 1;
      for (int k = 0; k < P; ++k) {
        ImageGeom g;
        image_geom(k, d.L, d.M, d.N, &g);
        t.img_off[k] = (int)std::min<int64_t>(pix, 1 << 30);
        pix += (g.S * g.F + 1) & ~int64_t(1);  // even: 16-bit pixels pair up in words
        maxF = std::max(maxF, std::max(g.F, g.S));
      }
      const int64_t words = t.wide ? pix : pix / 2;
      if (pix > (1ll << 30) || (size_t)words * 4 + kPartBytes > (size_t)kSmemLimit) fused = false;
      if (fused) {
        t.vol = d.volume;
        t.L = (int)d.L; t.M = (int)d.M; t.N = (int)d.N;
        t.dtype = d.dtype; t.K = d.K; t.P = P;
        t.words = (int)words;
        // a row power sum is at most (vmax * line) * maxF^K * maxF
        const double bits = std::log2(vmax * (double)line + 1) + d.K * std::log2((double)maxF + 1) +
                            std::log2((double)maxF + 1);
        t.r64 = bits < 62.0 ? 1 : 0;
        t.t_off = c->t_total;
        t.out_off = d.out_offset;
        c->t_total += (int64_t)P * num_2d(d.K);
        c->tasks.push_back(t);
        c->fused_index.push_back(i);
        c->max_words = std::max(c->max_words, (size_t)words);
      }
    }
    if (!fused) c->single.push_back(i);
  }
}

std::vector<int> lpt_order(const std::vector<BTask>& tasks) {
  std::vector<int> order(tasks.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const BTask &a = tasks[x], &c = tasks[y];
    return (int64_t)a.L * a.M * a.N > (int64_t)c.L * c.M * c.N;
  });
  return order;
}

size_t fused_smem(size_t max_words) { return (size_t)kPartBytes + max_words * 4; }

int fused_grid(size_t smem, int threads, int ntasks) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (threads == 512) {
    set_smem<512>(smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fused_kernel<512>, 512, smem);
  } else {
    set_smem<256>(smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fused_kernel<256>, 256, smem);
  }
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  return std::max(1, std::min(sms * per_sm, ntasks));
}

cudaError_t prepare_plans() {
  const DevPlans* dp = nullptr;
  return plans_for_device(&dp);
}

cudaError_t enqueue_fused(const BTask* d_tasks, const int* d_order, int n, int* d_counter,
                          i128* d_T, size_t smem, int threads, int grid, void* out,
                          int* d_status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const DevPlans* dp = nullptr;
  cudaError_t e = plans_for_device(&dp);
  if (e != cudaSuccess) return e;
  FusedParams p{};
  p.tasks = d_tasks;
  p.order = d_order;
  p.ntasks = n;
  p.counter = d_counter;
  p.T = d_T;
  if (threads == 512) {
    e = set_smem<512>(smem);
    if (e != cudaSuccess) return e;
    batch_fused_kernel<512><<<grid, 512, smem, st>>>(p);
  } else {
    e = set_smem<256>(smem);
    if (e != cudaSuccess) return e;
    batch_fused_kernel<256><<<grid, 256, smem, st>>>(p);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  BCombParams cp{};
  cp.tasks = d_tasks;
  cp.ntasks = n;
  cp.plans = dp->words;
  std::memcpy(cp.off, dp->off, sizeof(cp.off));
  cp.T = d_T;
  cp.out = static_cast<unsigned char*>(out);
  cp.status = d_status;
  const int64_t nt = 128, total = (int64_t)n * 165;
  batch_combine_kernel<<<(unsigned)((total + nt - 1) / nt), (unsigned)nt, 0, st>>>(cp);
  return cudaGetLastError();
}

cudaError_t enqueue_merge_status(const int* src, int* dst, cudaStream_t st) {
  merge_status_kernel<<<1, 1, 0, st>>>(src, dst);
  return cudaGetLastError();
}

}  // namespace batch
}  // namespace dpma

struct dpma_batch {
  int device = 0;
  std::vector<dpma_volume_desc> descs;
  batch::Classified cls;
  BTask* d_tasks = nullptr;
  int* d_order = nullptr;
  int* d_counter = nullptr;
  int* d_status = nullptr;
  i128* d_T = nullptr;
  size_t smem = 0;
  int threads = 512;
  int grid = 0;
  void* d_ws = nullptr;  // workspace of the single-volume path
  size_t ws_bytes = 0;
};

namespace {

void free_plan(dpma_batch* b) {
  if (!b) return;
  cudaFree(b->d_tasks);
  cudaFree(b->d_order);
  cudaFree(b->d_counter);
  cudaFree(b->d_status);
  cudaFree(b->d_T);
  cudaFree(b->d_ws);
  delete b;
}

dpma_status enqueue_batch(dpma_batch* b, void* out, cudaStream_t st, bool singles = true) {
  unsigned char* o = static_cast<unsigned char*>(out);
  cudaError_t e = cudaMemsetAsync(b->d_status, 0, sizeof(int), st);
  if (e != cudaSuccess) return bfail(DPMA_ERR_CUDA, std::string("clear status: ") + cudaGetErrorString(e));
  const int n = (int)b->cls.tasks.size();
  if (n > 0) {
    e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = batch::enqueue_fused(b->d_tasks, b->d_order, n, b->d_counter, b->d_T, b->smem,
                               b->threads, b->grid, out, b->d_status, st);
    if (e != cudaSuccess)
      return bfail(DPMA_ERR_CUDA, std::string("batched kernels: ") + cudaGetErrorString(e));
  }
  if (!singles) return DPMA_OK;
  for (int i : b->cls.single) {
    const dpma_volume_desc& d = b->descs[i];
    dpma_status s = dpma_moments_async(d.volume, d.L, d.M, d.N, (dpma_dtype)d.dtype, d.K,
                                       o + d.out_offset, st, b->d_ws, b->ws_bytes);
    if (s != DPMA_OK) return s;
    // a single-volume layout keeps its status word in its last 256 bytes
    const size_t total = dpma_workspace_size(d.L, d.M, d.N, (dpma_dtype)d.dtype, d.K);
    e = batch::enqueue_merge_status(
        reinterpret_cast<const int*>(static_cast<unsigned char*>(b->d_ws) + total - 256),
        b->d_status, st);
    if (e != cudaSuccess) return bfail(DPMA_ERR_CUDA, std::string("status merge: ") + cudaGetErrorString(e));
  }
  return DPMA_OK;
}

// Host-only validation of a descriptor array.
dpma_status validate(const dpma_volume_desc* descs, int count) {
  if (count < 0 || (count > 0 && !descs)) return bfail(DPMA_ERR_INVALID_ARG, "bad descriptor array");
  for (int i = 0; i < count; ++i) {
    const dpma_volume_desc& d = descs[i];
    const std::string at = "descriptor " + std::to_string(i) + ": ";
    if (!d.volume) return bfail(DPMA_ERR_INVALID_ARG, at + "null volume");
    if (d.out_offset < 0 || d.out_offset % 16 != 0)
      return bfail(DPMA_ERR_INVALID_ARG, at + "out_offset must be a non-negative multiple of 16");
    if (dpma_workspace_size(d.L, d.M, d.N, (dpma_dtype)d.dtype, d.K) == 0)
      return bfail(DPMA_ERR_INVALID_ARG, at + "bad dimensions, dtype or K");
    if (d.dtype != DPMA_F32) {
      const double vmax = d.dtype == DPMA_U8 ? 255.0 : 65535.0;
      if (log2_bound_2d(d.L, d.M, d.N, vmax, d.K) > 125.0 ||
          log2_bound_3d(d.L, d.M, d.N, vmax, d.K) > 125.0)
        return bfail(DPMA_ERR_OVERFLOW, at + "moments could exceed the int128 range");
    }
  }
  return DPMA_OK;
}

}  // namespace

namespace dpma {
// Shared with the serving loop: host-only descriptor checks.
dpma_status validate_descs(const dpma_volume_desc* descs, int count) { return validate(descs, count); }
}  // namespace dpma

extern "C" {

dpma_status dpma_batch_create(const dpma_volume_desc* descs, int count, int flags,
                              dpma_batch** plan) {
  if (!plan) return bfail(DPMA_ERR_INVALID_ARG, "null plan pointer");
  *plan = nullptr;
  if (count < 0 || (count > 0 && !descs)) return bfail(DPMA_ERR_INVALID_ARG, "bad descriptor array");
  if (flags & ~DPMA_BATCH_AUTOTUNE) return bfail(DPMA_ERR_INVALID_ARG, "unknown flags");
  dpma_status vs = validate(descs, count);
  if (vs != DPMA_OK) return vs;
  dpma_batch* b = new dpma_batch();
  b->descs.assign(descs, descs + count);
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) { free_plan(b); return bfail(DPMA_ERR_CUDA, "no current CUDA device"); }
  batch::classify(descs, count, &b->cls);

  auto oom = [&](cudaError_t err, const char* what) {
    free_plan(b);
    if (err == cudaErrorMemoryAllocation) { cudaGetLastError(); return bfail(DPMA_ERR_OOM, what); }
    return bfail(DPMA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
  };
  e = cudaMalloc(&b->d_status, sizeof(int));
  if (e != cudaSuccess) return oom(e, "batch status");
  const std::vector<BTask>& tasks = b->cls.tasks;
  if (!tasks.empty()) {
    const std::vector<int> order = batch::lpt_order(tasks);
    e = cudaMalloc(&b->d_tasks, sizeof(BTask) * tasks.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * order.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
    if (e == cudaSuccess)
      e = cudaMalloc(&b->d_T, sizeof(i128) * (size_t)std::max<int64_t>(1, b->cls.t_total));
    if (e != cudaSuccess) return oom(e, "batch buffers");
    e = cudaMemcpy(b->d_tasks, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = batch::prepare_plans();
    if (e != cudaSuccess) return oom(e, "batch upload");
    b->smem = batch::fused_smem(b->cls.max_words);
    b->threads = 512;
    b->grid = batch::fused_grid(b->smem, 512, (int)tasks.size());
  }
  if (!b->cls.single.empty()) {
    size_t ws = 0;
    for (int i : b->cls.single) {
      const dpma_volume_desc& d = descs[i];
      ws = std::max(ws, dpma_workspace_size(d.L, d.M, d.N, (dpma_dtype)d.dtype, d.K));
      e = prepare_combine(d.K);  // resident before any stream capture
      if (e != cudaSuccess) return oom(e, "combine plan");
    }
    e = cudaMalloc(&b->d_ws, ws);
    if (e != cudaSuccess) return oom(e, "single-volume workspace");
    b->ws_bytes = ws;
  }

  if ((flags & DPMA_BATCH_AUTOTUNE) && !tasks.empty()) {
    // time both CTA sizes of the fused launch on the real inputs, keep the faster
    void* scratch = nullptr;
    size_t ob = 16;
    for (const dpma_volume_desc& d : b->descs)
      ob = std::max(ob, (size_t)d.out_offset + (size_t)num_moments(d.K) * 16);
    e = cudaMalloc(&scratch, ob);
    if (e != cudaSuccess) return oom(e, "autotune scratch");
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_nt = 512, best_grid = b->grid;
    for (int nt : {256, 512}) {
      b->threads = nt;
      b->grid = batch::fused_grid(b->smem, nt, (int)tasks.size());
      enqueue_batch(b, scratch, st, false);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) enqueue_batch(b, scratch, st, false);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_nt = nt; best_grid = b->grid; }
    }
    b->threads = best_nt;
    b->grid = best_grid;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) { free_plan(b); return bfail(DPMA_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e)); }
  }
  *plan = b;
  return DPMA_OK;
}

dpma_status dpma_batch_run(dpma_batch* plan, void* out, void* stream) {
  if (!plan || !out) return bfail(DPMA_ERR_INVALID_ARG, "null plan or output pointer");
  return enqueue_batch(plan, out, static_cast<cudaStream_t>(stream));
}

dpma_status dpma_batch_status(dpma_batch* plan, void* stream) {
  if (!plan) return bfail(DPMA_ERR_INVALID_ARG, "null plan");
  int status = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(&status, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bfail(DPMA_ERR_CUDA, std::string("batch status: ") + cudaGetErrorString(e));
  if (status == DPMA_ERR_TIMEOUT) return bfail(DPMA_ERR_TIMEOUT, "a bounded device wait gave up");
  if (status) return bfail(DPMA_ERR_INTERNAL, "combine division left a remainder");
  return DPMA_OK;
}

int dpma_batch_info(const dpma_batch* plan, int what) {
  if (!plan) return -1;
  switch (what) {
    case 0: return (int)plan->cls.tasks.size();
    case 1: return (int)plan->cls.single.size();
    case 2: return plan->threads;
    case 3: return plan->grid;
    case 4: return (int)plan->smem;
  }
  return -1;
}

dpma_status dpma_batch_destroy(dpma_batch* plan) {
  free_plan(plan);
  return DPMA_OK;
}

dpma_status dpma_moments_batched(const dpma_volume_desc* descs, int count, void* out,
                                 void* stream) {
  if (!out) return bfail(DPMA_ERR_INVALID_ARG, "null output pointer");
  dpma_batch* b = nullptr;
  dpma_status s = dpma_batch_create(descs, count, 0, &b);
  if (s != DPMA_OK) return s;
  s = dpma_batch_run(b, out, stream);
  if (s == DPMA_OK) s = dpma_batch_status(b, stream);
  else cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  dpma_batch_destroy(b);
  return s;
}

}  // extern "C"
