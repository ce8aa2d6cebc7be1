// Step 1 of the Discrete Projection Moment method: one fused pass over the
// volume that writes every projection image at once (Sec. 3.1, Eq. 4 with
// the image set of Eqs. 5-9 and the +-pi/4 families; the paper's own CPU
// loop appears as its projection listing in Sec. 5).
//
// Work decomposition.  A CTA owns a tile of XT = 512 columns (x) by BY = 16
// rows (y) and streams it along z.  Its 512 threads form TX = 128 columns of
// R = 4 x-elements by TY = 4 row groups of BYT = 4 rows, so each thread
// holds a 4 x 4 micro-tile of every z-slice.  Persistent CTAs take
// contiguous ranges of (tile, z) units, so every CTA streams one or two
// long z-segments.
//
// Per voxel and per image the thread does one addition into a register:
//  * image 0 (sum along z)   : a register accumulator per (x, y), Kahan-
//                              compensated for float volumes;
//  * images 3/4 (x+-z, y)    : a rotating window of R registers per row; the
//                              pixel leaving the window each z-step is added
//                              into a rolling shared-memory row of XT slots
//                              (Kahan-compensated for float volumes);
//  * images 7/8 (y+-z, x)    : a rotating window of BYT registers per column;
//                              leaving pixels go to global memory;
//  * images 1, 2, 5, 6 (one z-slice each): the micro-tile is reduced in
//                              registers (row sums, column sums, diagonal
//                              sums) and added into a per-step shared buffer.
// After each z-step a barrier hands the per-step buffer and the completed
// rolling pixels to all threads, which add them into the global images with
// L2 atomics (red.global.add).  Integer images are uint32 and exact; float
// images are (hi, lo) planes whose sum is the compensated value.
#include <cstdint>
#include <type_traits>

#include "dpma_internal.cuh"

namespace dpma {
namespace {

constexpr int R = 4;           // x elements per thread
constexpr int BYT = 4;         // rows per thread
constexpr int TX = 128;        // thread columns
constexpr int TY = 4;          // thread row groups
constexpr int XT = R * TX;     // tile width
constexpr int BY = BYT * TY;   // tile height
constexpr int NT = TX * TY;    // threads per CTA
static_assert(R == BYT, "window rotations share one unroll period");

// per-step buffer sections (words)
constexpr int kS1 = 0;                        // image 1: BY row sums
constexpr int kS2 = kS1 + BY;                 // image 2: XT column sums
constexpr int kS5 = kS2 + XT;                 // image 5: XT+BY-1 diagonals
constexpr int kS6 = kS5 + XT + BY - 1;        // image 6
constexpr int kStep = kS6 + XT + BY - 1;      // words per step buffer

template <typename T> struct AccT { using type = uint32_t; };
template <> struct AccT<float> { using type = float; };

struct K1Params {
  const void* vol;
  int64_t L, M, N;
  int64_t nbands;
  int64_t units;  // nxt * nbands * N
  ImageSet set;
  void* images;
  int vec;        // rows allow R-element vector loads
};

__device__ __forceinline__ void gadd(uint32_t* p, uint32_t v) {
  if (v) atomicAdd(p, v);
}
__device__ __forceinline__ void gadd(float* p, float v) {
  if (v != 0.0f) atomicAdd(p, v);
}

// Load R elements of one row starting at x (masked to [0, L)).
template <typename T, typename A>
__device__ __forceinline__ void load_run(const T* __restrict__ row, int64_t x, int64_t L, bool vec,
                                         A out[R]) {
  if (vec && x + R <= L) {
    if constexpr (std::is_same<T, float>::value) {
      float4 q = __ldcs(reinterpret_cast<const float4*>(row + x));
      out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
    } else if constexpr (std::is_same<T, uint16_t>::value) {
      uint2 q = __ldcs(reinterpret_cast<const uint2*>(row + x));
      out[0] = q.x & 0xffffu; out[1] = q.x >> 16; out[2] = q.y & 0xffffu; out[3] = q.y >> 16;
    } else {
      uint32_t q = __ldcs(reinterpret_cast<const unsigned int*>(row + x));
      out[0] = q & 0xffu; out[1] = (q >> 8) & 0xffu; out[2] = (q >> 16) & 0xffu; out[3] = q >> 24;
    }
  } else {
#pragma unroll
    for (int c = 0; c < R; ++c) out[c] = (x + c < L) ? (A)row[x + c] : (A)0;
  }
}

// Warp reduction of BYT = 4 per-lane values into one value per 8-lane group:
// lanes 0-7 end with row 0, 8-15 row 1, 16-23 row 2, 24-31 row 3.
__device__ __forceinline__ float reduce4_scatter(float a0, float a1, float a2, float a3, int lane) {
  const bool up = lane & 16;
  float k0 = up ? a2 : a0, k1 = up ? a3 : a1;
  float s0 = up ? a0 : a2, s1 = up ? a1 : a3;
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool up2 = lane & 8;
  float k = up2 ? k1 : k0, s = up2 ? k0 : k1;
  k += __shfl_xor_sync(0xffffffffu, s, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

template <typename T, int P>
__global__ void __launch_bounds__(NT, 1) k1_project_kernel(K1Params p) {
  using A = typename AccT<T>::type;
  constexpr bool FL = std::is_same<T, float>::value;
  constexpr bool H3 = P > 3, H4 = P > 4, H5 = P > 5, H6 = P > 6, H7 = P > 7, H8 = P > 8;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* stepbuf = reinterpret_cast<A*>(smem_raw);            // [2][kStep]
  A* roll = stepbuf + 2 * kStep;                          // rolling rows, see below
  // rolling buffers: image 3 then image 4; each [BY][XT] sums, then (float)
  // [BY][XT] Kahan compensations
  constexpr int kRollWords = BY * XT * (FL ? 2 : 1);
  A* roll3 = roll;
  A* roll4 = roll + (H3 ? kRollWords : 0);

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX, lane = tid & 31;
  const T* __restrict__ vol = static_cast<const T*>(p.vol);
  const int64_t L = p.L, M = p.M, N = p.N;
  const ImageSet& set = p.set;
  A* img = static_cast<A*>(p.images);
  const int xl = tx * R;        // thread's first column inside the tile
  const int yl = ty * BYT;      // thread's first row inside the tile

  // zero shared state once; every segment leaves it zeroed again
  {
    const int words = 2 * kStep + (H3 ? kRollWords : 0) + (H4 ? kRollWords : 0);
    for (int i = tid; i < words; i += NT) stepbuf[i] = (A)0;
  }
  __syncthreads();

  const int64_t ub = p.units * (int64_t)blockIdx.x / gridDim.x;
  const int64_t ue = p.units * (int64_t)(blockIdx.x + 1) / gridDim.x;

  for (int64_t u = ub; u < ue;) {
    const int64_t seg = u / N;
    const int64_t za = u % N;
    const int64_t Z = (N - za) < (ue - u) ? (N - za) : (ue - u);
    const int64_t band = seg % p.nbands;
    const int64_t x0 = (seg / p.nbands) * XT;
    const int64_t y0 = band * BY;
    const int64_t xs = x0 + xl;      // thread's first x
    const int64_t yt = y0 + yl;      // thread's first y

    A a0[BYT][R];
    float a0c[BYT][R];
    A w3[BYT][R], w4[BYT][R], w7[BYT][R], w8[BYT][R];
#pragma unroll
    for (int r = 0; r < BYT; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) {
        a0[r][c] = 0; a0c[r][c] = 0.f; w3[r][c] = 0; w4[r][c] = 0; w7[r][c] = 0; w8[r][c] = 0;
      }

    // Z real steps plus R-1 trailing steps that only drain the windows.
    const int64_t Zext = Z + ((H3 || H7) ? (R - 1) : 0);
    int64_t s = 0;
    for (int64_t s0 = 0; s0 < Zext; s0 += R) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        s = s0 + j;
        if (s < Zext) {
          const bool real = s < Z;
          const int64_t z = za + s;
          A* buf = stepbuf + (s & 1) * kStep;
          A v[BYT][R];
#pragma unroll
          for (int r = 0; r < BYT; ++r) {
            const int64_t y = yt + r;
            if (real && y < M && xs < L) {
              load_run<T, A>(vol + (z * M + y) * L, xs, L, p.vec != 0, v[r]);
            } else {
#pragma unroll
              for (int c = 0; c < R; ++c) v[r][c] = 0;
            }
          }

          // image 0: sum along z
#pragma unroll
          for (int r = 0; r < BYT; ++r)
#pragma unroll
            for (int c = 0; c < R; ++c) {
              if constexpr (FL) {
                float yk = v[r][c] - a0c[r][c];
                float t = a0[r][c] + yk;
                a0c[r][c] = (t - a0[r][c]) - yk;
                a0[r][c] = t;
              } else {
                a0[r][c] += v[r][c];
              }
            }

          // images 3 / 4: rotating windows along x (logical k = column c)
          if constexpr (H3) {
#pragma unroll
            for (int r = 0; r < BYT; ++r)
#pragma unroll
              for (int c = 0; c < R; ++c) w3[r][(c + j) % R] += v[r][c];
          }
          if constexpr (H4) {
#pragma unroll
            for (int r = 0; r < BYT; ++r)
#pragma unroll
              for (int c = 0; c < R; ++c) w4[r][(c - j + R) % R] += v[r][c];
          }
          // images 7 / 8: rotating windows along y (logical k = row r)
          if constexpr (H7) {
#pragma unroll
            for (int r = 0; r < BYT; ++r)
#pragma unroll
              for (int c = 0; c < R; ++c) w7[(r + j) % BYT][c] += v[r][c];
          }
          if constexpr (H8) {
#pragma unroll
            for (int r = 0; r < BYT; ++r)
#pragma unroll
              for (int c = 0; c < R; ++c) w8[(r - j + BYT) % BYT][c] += v[r][c];
          }

          // leaving pixels of the x windows -> rolling rows (exclusive slots)
          if constexpr (H3) {
            const int slot = (int)((xl + s) % XT);  // pixel xl + s of image 3
#pragma unroll
            for (int r = 0; r < BYT; ++r) {
              A wv = w3[r][j];
              w3[r][j] = 0;
              A* cell = roll3 + (yl + r) * XT + slot;
              if constexpr (FL) {
                float* comp = reinterpret_cast<float*>(roll3 + BY * XT) + (yl + r) * XT + slot;
                float sum = *cell, cc = *comp;
                float yk = wv - cc;
                float t = sum + yk;
                *comp = (t - sum) - yk;
                *cell = t;
              } else {
                *cell += wv;
              }
            }
          }
          if constexpr (H4) {
            const int lk = (R - 1 - j + R) % R;  // physical index of logical R-1
            // pixel xl + R-1 - s of image 4 (may be negative: rolling index)
            const int slot = (int)((((int64_t)xl + R - 1 - s) % XT + XT) % XT);
#pragma unroll
            for (int r = 0; r < BYT; ++r) {
              A wv = w4[r][lk];
              w4[r][lk] = 0;
              A* cell = roll4 + (yl + r) * XT + slot;
              if constexpr (FL) {
                float* comp = reinterpret_cast<float*>(roll4 + BY * XT) + (yl + r) * XT + slot;
                float sum = *cell, cc = *comp;
                float yk = wv - cc;
                float t = sum + yk;
                *comp = (t - sum) - yk;
                *cell = t;
              } else {
                *cell += wv;
              }
            }
          }
          // leaving pixels of the y windows -> global
          if constexpr (H7) {
            const int64_t srow = yt + z;  // slow index y + z of image 7
            if (srow < set.S[7]) {
              A* dst = img + set.base[7] + srow * set.F[7];
#pragma unroll
              for (int c = 0; c < R; ++c)
                if (xs + c < L) gadd(dst + xs + c, w7[j][c]);
            }
#pragma unroll
            for (int c = 0; c < R; ++c) w7[j][c] = 0;
          }
          if constexpr (H8) {
            const int lk = (BYT - 1 - j + BYT) % BYT;
            const int64_t srow = yt + (BYT - 1) - z + (N - 1);  // y - z + N - 1
            if (srow >= 0 && srow < set.S[8]) {
              A* dst = img + set.base[8] + srow * set.F[8];
#pragma unroll
              for (int c = 0; c < R; ++c)
                if (xs + c < L) gadd(dst + xs + c, w8[lk][c]);
            }
#pragma unroll
            for (int c = 0; c < R; ++c) w8[lk][c] = 0;
          }

          // images on the current z-slice -> per-step shared buffer
          if (real) {
            // image 1 (sum along x): row sums
            A rs[BYT];
#pragma unroll
            for (int r = 0; r < BYT; ++r) {
              rs[r] = v[r][0];
#pragma unroll
              for (int c = 1; c < R; ++c) rs[r] += v[r][c];
            }
            if constexpr (FL) {
              float k = reduce4_scatter(rs[0], rs[1], rs[2], rs[3], lane);
              if ((lane & 7) == 0) atomicAdd(buf + kS1 + yl + (lane >> 3), k);
            } else {
#pragma unroll
              for (int r = 0; r < BYT; ++r) {
                uint32_t t = __reduce_add_sync(0xffffffffu, rs[r]);
                if (lane == 0 && t) atomicAdd(buf + kS1 + yl + r, t);
              }
            }
            // image 2 (sum along y): column sums
#pragma unroll
            for (int c = 0; c < R; ++c) {
              A cs = v[0][c];
#pragma unroll
              for (int r = 1; r < BYT; ++r) cs += v[r][c];
              atomicAdd(buf + kS2 + xl + c, cs);
            }
            // image 5 (x + y) and image 6 (x - y): diagonal sums
            if constexpr (H5) {
#pragma unroll
              for (int k = 0; k < R + BYT - 1; ++k) {
                A d = 0;
#pragma unroll
                for (int r = 0; r < BYT; ++r) {
                  const int c = k - r;
                  if (c >= 0 && c < R) d += v[r][c];
                }
                atomicAdd(buf + kS5 + xl + yl + k, d);
              }
            }
            if constexpr (H6) {
#pragma unroll
              for (int k = 0; k < R + BYT - 1; ++k) {
                A d = 0;
#pragma unroll
                for (int r = 0; r < BYT; ++r) {
                  const int c = k - (BYT - 1) + r;
                  if (c >= 0 && c < R) d += v[r][c];
                }
                // local index x_l - y_l + BY - 1
                atomicAdd(buf + kS6 + xl - yl + (BY - BYT) + k, d);
              }
            }
          }

          __syncthreads();

          // flush: per-step buffer and completed rolling pixels -> global
          {
            constexpr int kRet3 = kStep;            // BY retiring pixels of image 3
            constexpr int kRet4 = kStep + BY;       // BY retiring pixels of image 4
            constexpr int kTot = kStep + 2 * BY;
            for (int e = tid; e < kTot; e += NT) {
              if (e < kStep) {
                if (!real) continue;
                A val = buf[e];
                if (val == (A)0) continue;
                buf[e] = (A)0;
                int64_t k, srow, f;
                if (e < kS2) { k = 1; srow = z; f = y0 + (e - kS1); }
                else if (e < kS5) { k = 2; srow = z; f = x0 + (e - kS2); }
                else if (e < kS6) { k = 5; srow = z; f = x0 + y0 + (e - kS5); }
                else { k = 6; srow = z; f = x0 - y0 - (BY - 1) + (e - kS6) + (M - 1); }
                if ((k == 5 && !H5) || (k == 6 && !H6)) continue;
                if (f < 0 || f >= set.F[k]) continue;
                A* dst = img + set.base[k] + srow * set.F[k] + f;
                if constexpr (FL) gadd(dst, val);
                else gadd(dst, val);
              } else if (e < kRet4) {
                if constexpr (H3) {
                  const int rr = e - kRet3;
                  const int slot = (int)(s % XT);
                  A* cell = roll3 + rr * XT + slot;
                  A val = *cell;
                  float comp = 0.f;
                  if constexpr (FL) {
                    float* cp = reinterpret_cast<float*>(roll3 + BY * XT) + rr * XT + slot;
                    comp = *cp;
                    *cp = 0.f;
                  }
                  *cell = (A)0;
                  const int64_t y = y0 + rr;
                  const int64_t f = x0 + za + s;  // x + z of pixel s
                  if (y < M && f < set.F[3]) {
                    A* dst = img + set.base[3] + y * set.F[3] + f;
                    gadd(dst, val);
                    if constexpr (FL) gadd(reinterpret_cast<float*>(dst) + set.S[3] * set.F[3], -comp);
                  }
                }
              } else {
                if constexpr (H4) {
                  const int rr = e - kRet4;
                  const int64_t pix = (int64_t)XT - 1 - s;  // rolling index of image 4
                  const int slot = (int)(((pix % XT) + XT) % XT);
                  A* cell = roll4 + rr * XT + slot;
                  A val = *cell;
                  float comp = 0.f;
                  if constexpr (FL) {
                    float* cp = reinterpret_cast<float*>(roll4 + BY * XT) + rr * XT + slot;
                    comp = *cp;
                    *cp = 0.f;
                  }
                  *cell = (A)0;
                  const int64_t y = y0 + rr;
                  const int64_t f = (x0 - za + N - 1) + pix;  // x - z + N - 1
                  if (y < M && f >= 0 && f < set.F[4]) {
                    A* dst = img + set.base[4] + y * set.F[4] + f;
                    gadd(dst, val);
                    if constexpr (FL) gadd(reinterpret_cast<float*>(dst) + set.S[4] * set.F[4], -comp);
                  }
                }
              }
            }
          }
        }
      }
    }

    // ---- segment end ----
    // image 0: registers -> global
#pragma unroll
    for (int r = 0; r < BYT; ++r) {
      const int64_t y = yt + r;
      if (y >= M) continue;
      A* dst = img + set.base[0] + y * set.F[0];
#pragma unroll
      for (int c = 0; c < R; ++c) {
        if (xs + c >= L) continue;
        gadd(dst + xs + c, a0[r][c]);
        if constexpr (FL) gadd(reinterpret_cast<float*>(dst + xs + c) + set.S[0] * set.F[0], -a0c[r][c]);
      }
    }
    __syncthreads();  // last retire reads are done before the final sweep
    // rolling rows still holding live pixels -> global, then zero
    const int64_t sf = Zext - 1;  // last step index
    if constexpr (H3 || H4) {
      for (int e = tid; e < BY * XT * ((H3 ? 1 : 0) + (H4 ? 1 : 0)); e += NT) {
        const bool is4 = H3 ? (e >= BY * XT) : true;
        const int ee = H3 ? (e % (BY * XT)) : e;
        const int rr = ee / XT, slot = ee % XT;
        A* rb = is4 ? roll4 : roll3;
        A* cell = rb + rr * XT + slot;
        A val = *cell;
        float comp = 0.f;
        if constexpr (FL) {
          float* cp = reinterpret_cast<float*>(rb + BY * XT) + rr * XT + slot;
          comp = *cp;
          *cp = 0.f;
        }
        *cell = (A)0;
        if (val == (A)0 && comp == 0.f) continue;
        const int64_t y = y0 + rr;
        if (y >= M) continue;
        int64_t pix, f;
        int k;
        if (!is4) {
          pix = sf + 1 + ((slot - (sf + 1)) % XT + XT) % XT;
          f = x0 + za + pix;
          k = 3;
        } else {
          pix = -(sf + 1) + ((slot + sf + 1) % XT);
          f = (x0 - za + N - 1) + pix;
          k = 4;
        }
        if (f < 0 || f >= set.F[k]) continue;
        A* dst = img + set.base[k] + y * set.F[k] + f;
        gadd(dst, val);
        if constexpr (FL) gadd(reinterpret_cast<float*>(dst) + set.S[k] * set.F[k], -comp);
      }
    }
    __syncthreads();
    u += Z;
  }
}

template <typename T, int P>
cudaError_t launch_t(const ProjectArgs& a, cudaStream_t st) {
  constexpr bool FL = std::is_same<T, float>::value;
  K1Params p{};
  p.vol = a.vol;
  p.L = a.L; p.M = a.M; p.N = a.N;
  p.nbands = (a.M + BY - 1) / BY;
  const int64_t nxt = (a.L + XT - 1) / XT;
  p.units = nxt * p.nbands * a.N;
  p.set = a.set;
  p.images = a.images;
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.vol);
  p.vec = ((a.L % R) == 0 && (base % (R * sizeof(T))) == 0) ? 1 : 0;

  const int roll_imgs = (P > 3 ? 1 : 0) + (P > 4 ? 1 : 0);
  const size_t smem = (size_t)(2 * kStep + roll_imgs * BY * XT * (FL ? 2 : 1)) * 4;
  auto kern = k1_project_kernel<T, P>;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static int cached_sms[64] = {0}, cached_per_sm[64] = {0};  // per instantiation
  int sms = dev < 64 ? cached_sms[dev] : 0, per_sm = dev < 64 ? cached_per_sm[dev] : 0;
  if (sms == 0) {
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (dev < 64) { cached_sms[dev] = sms; cached_per_sm[dev] = per_sm; }
  }
  // at least ~8 z-steps per CTA so the window drain stays a small overhead
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t by_work = (p.units + 7) / 8;
  if (grid > by_work) grid = by_work;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, NT, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dtype(const ProjectArgs& a, cudaStream_t st) {
  switch (a.set.P) {
    case 3: return launch_t<T, 3>(a, st);
    case 4: return launch_t<T, 4>(a, st);
    case 5: return launch_t<T, 5>(a, st);
    case 6: return launch_t<T, 6>(a, st);
    case 7: return launch_t<T, 7>(a, st);
    case 8: return launch_t<T, 8>(a, st);
    case 9: return launch_t<T, 9>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_project(const ProjectArgs& a, cudaStream_t st) {
  switch (a.dtype) {
    case 0: return launch_dtype<uint8_t>(a, st);
    case 1: return launch_dtype<uint16_t>(a, st);
    case 2: return launch_dtype<float>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dpma
