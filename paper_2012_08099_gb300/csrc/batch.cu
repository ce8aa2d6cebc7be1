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
// Inside a CTA a slice is cut into chunks of four consecutive voxels of one
// row; each thread loads its chunk as one word and adds it to every image with
// shared-memory atomic adds (two or three 32-bit words per image).  Pixels
// are 16-bit when the longest line times the largest voxel value stays below
// 2^16 (two pixels per 32-bit word; a packed add never carries into the
// neighbour because every sum is bounded), 32-bit otherwise.  The 2-D moments
// are then taken per image from row power sums of row segments, one thread
// per segment, folded into T_ab by one warp per image and power b.
//
// Volumes the fused kernel does not take (float32, slices over 24 KB, or
// images larger than the shared-memory budget) run through the single-volume
// pipeline on the same stream, one after another.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
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

// the 2-D moments T_ab of every image of the volume being reduced (int128)
constexpr int kPartBytes = kMaxImagesBatch * kMax2DBatch * 16;
constexpr int kSlabWords = 6144;  // one stage buffer (24 KB), double-buffered
// stage buffers of a one-CTA-per-SM launch whose images leave room (48 KB):
// half as many stages, so half as many stage barriers
constexpr int kSlabWordsBig = 12288;
constexpr int kChunk = 8;  // voxels of one row per projection position
// words past the last image: the zero adds of a ragged chunk reach up to
// kChunk - 1 pixels past a row
constexpr int kSlackWords = 8;
constexpr int kSmemLimit = 227 * 1024 - 512;  // dynamic bytes: the rest is static (meta, task id)
constexpr int kStatusInternal = 7;


struct FusedParams {
  const BTask* tasks;
  const int* order;  // processing order (largest first)
  int ntasks;
  int* counter;      // work queue head (zeroed before each run)
  i128* T;           // 2-D moments of every volume
  int slab_words;    // words of one stage buffer: kSlabWords or kSlabWordsBig
};

// Which of a task's z-block choices a launch uses: 256 threads, or 512
// threads with standard or big stage buffers.
__host__ __device__ __forceinline__ int zblock_index(int nt, int sw) {
  return nt == 256 ? 0 : (sw == kSlabWordsBig ? 2 : 1);
}

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

// Adds the four consecutive pixels b .. b+3 of one image row, given as the
// packed pairs p01 = v0 | v1 << 16 and p23 = v2 | v3 << 16 (every v < 2^16).
// With 16-bit pixels the pairs are shifted onto the pixel words (three words
// from word b/2) and added with one shared atomic per word; a halfword's sum
// is bounded below 2^16, so no carry crosses into its neighbour.  The adds
// are unconditional: a word past the row (a ragged chunk) gets zero, and the
// image area ends with kSlackWords spare words for the last image.
template <bool WIDE>
__device__ __forceinline__ void add4(uint32_t* sm, int b, uint32_t p01, uint32_t p23) {
  if constexpr (WIDE) {
    atomicAdd(sm + b, p01 & 0xffffu);
    atomicAdd(sm + b + 1, p01 >> 16);
    atomicAdd(sm + b + 2, p23 & 0xffffu);
    atomicAdd(sm + b + 3, p23 >> 16);
  } else {
    const int w = b >> 1;
    const uint32_t sh = (uint32_t)(b & 1) << 4;
    atomicAdd(sm + w, p01 << sh);
    atomicAdd(sm + w + 1, __funnelshift_l(p01, p23, sh));
    atomicAdd(sm + w + 2, __funnelshift_l(p23, 0u, sh));
  }
}

// Adds the eight consecutive pixels b .. b+7 of one image row, given as the
// packed pairs p01, p23, q01, q23 (pixels 0-1, 2-3, 4-5, 6-7; every v <
// 2^16): with 16-bit pixels five shifted words from word b/2, one shared
// atomic each (no carry crosses a halfword, as in add4).
template <bool WIDE>
__device__ __forceinline__ void add8(uint32_t* sm, int b, uint32_t p01, uint32_t p23,
                                     uint32_t q01, uint32_t q23) {
  if constexpr (WIDE) {
    add4<true>(sm, b, p01, p23);
    add4<true>(sm, b + 4, q01, q23);
  } else {
    const int w = b >> 1;
    const uint32_t sh = (uint32_t)(b & 1) << 4;
    atomicAdd(sm + w, p01 << sh);
    atomicAdd(sm + w + 1, __funnelshift_l(p01, p23, sh));
    atomicAdd(sm + w + 2, __funnelshift_l(p23, q01, sh));
    atomicAdd(sm + w + 3, __funnelshift_l(q01, q23, sh));
    atomicAdd(sm + w + 4, __funnelshift_l(q23, 0u, sh));
  }
}

// Slices per projection stage: as many as fit in one buffer with the 16-byte
// alignment head and the bytes a chunk load may read past the stage (the
// aligned words covering a chunk: up to 18 bytes past its last voxel).
__host__ __device__ __forceinline__ int stage_slices(int64_t slice_bytes, int N, int sw) {
  const int64_t g = ((int64_t)(sw - 8) * 4 - 30) / slice_bytes;
  return (int)(g < 1 ? 1 : (g < N ? g : N));
}

// Starts the copy of the stage of volume t that begins at slice z0 into the
// stage buffer dst (cp.async, 16-byte blocks, one commit group); returns the
// byte offset of slice z0 in the buffer.
template <int NT>
__device__ __forceinline__ int fetch_stage(const BTask& t, int z0, uint32_t* dst, int sw) {
  const int esize = t.dtype == DPMA_U8 ? 1 : 2;
  const int slice_bytes = t.L * t.M * esize;
  const int G = stage_slices(slice_bytes, t.N, sw);
  const uintptr_t a = reinterpret_cast<uintptr_t>(t.vol) + (uintptr_t)z0 * slice_bytes;
  const uintptr_t a16 = a & ~(uintptr_t)15;
  const int hd = (int)(a - a16);
  const int nb = (hd + min(G, t.N - z0) * slice_bytes + 15) >> 4;
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  for (int i = threadIdx.x; i < nb; i += NT)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16 * i),
                 "l"(a16 + 16 * (uintptr_t)i)
                 : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  return hd;
}

// Every image of one volume into shared memory (Eq. 4 for the image table of
// dpma.h).  The volume streams through shared buffers in stages of G whole
// z-slices (as many as fit in one buffer): the 16-byte aligned blocks
// covering the next stage are copied with cp.async while the current stage
// is processed (a 16-byte block holding a byte of the volume lies in the same
// mapped page).  Stage 0 arrives in `first` (copied ahead, during the
// previous volume's moment stage, and complete on entry: it is slab buffer
// 1); stage s uses slab buffer (s + 1) & 1.  A position is a chunk of
// kChunk = 8 consecutive voxels of one row, (y, c) with x0 = 8c; the stage's
// slices are split into Zg blocks so that positions x blocks fill the CTA,
// and a thread walks its position through the z of its block.  The chunk's
// voxels land on eight consecutive pixels of every image but image 1 (z, y),
// which takes the chunk's sum (eight voxels per atomic: the lanes of one row
// share that pixel); image 0 (y, x) does not move with z and is summed in
// registers over the block.  Every shared update is an atomic add; image k's
// pixel index moves by a constant per z-step.
template <typename T, bool WIDE, bool MANY, int NT>
__device__ __forceinline__ void project_volume(const BTask& t, uint32_t* sm, uint32_t* slab,
                                               const uint32_t* first, int head0, int sw) {
  const int L = t.L, M = t.M, N = t.N, P = t.P;
  const int F3 = L + N - 1, F7 = L + M - 1;
  const int* o = t.img_off;
  const int slice_bytes = L * M * (int)sizeof(T);
  const int G = stage_slices(slice_bytes, N, sw);
  const int nc = (L + kChunk - 1) / kChunk, npos = M * nc;
  const int Zg = t.zblocks[zblock_index(NT, sw)];  // z-blocks per stage
  int head = head0, head_next = 0;
  const uint32_t* cur = first;
  for (int z0 = 0, si = 0; z0 < N; z0 += G, ++si) {
    // in flight while this stage is processed: buffer si & 1 was last read
    // in stage si - 1 (or by the previous volume's moment stage), before a
    // barrier
    uint32_t* nxt = slab + (si & 1) * sw;
    if (z0 + G < N) head_next = fetch_stage<NT>(t, z0 + G, nxt, sw);
    const unsigned char* S = reinterpret_cast<const unsigned char*>(cur);
    const int gz = min(G, N - z0), zlen = (gz + Zg - 1) / Zg;
    for (int it = threadIdx.x; it < npos * Zg; it += NT) {
      const int zg = it / npos, pos = it - zg * npos;
      const int y = pos / nc, x0 = (pos - y * nc) * kChunk;
      const int zs = z0 + zg * zlen, ze = min(z0 + gz, zs + zlen);
      if (zs >= ze) continue;
      const int rem = L - x0;
      // byte offset of the chunk in the stage, and the pixel indices at z = zs
      int off = head + (((zs - z0) * M + y) * L + x0) * (int)sizeof(T);
      int b1 = o[1] + zs * M + y, b2 = o[2] + zs * L + x0;
      int b3 = o[3] + y * F3 + x0 + zs, b4 = o[4] + y * F3 + x0 - zs + N - 1;
      int b5 = o[5] + (y + zs) * L + x0, b6 = o[6] + (y - zs + N - 1) * L + x0;
      int b7 = o[7] + zs * F7 + x0 + y, b8 = o[8] + zs * F7 + x0 - y + M - 1;
      // image 0 over the block: packed pairs, or one word per pixel
      uint32_t i0[WIDE ? 8 : 4] = {};
      for (int z = zs; z < ze; ++z) {
        const uint32_t* W = reinterpret_cast<const uint32_t*>(S + (off & ~3));
        const uint32_t sh = (uint32_t)(off & 3) << 3;
        uint32_t p01, p23, q01, q23, rs;
        if constexpr (sizeof(T) == 1) {
          const uint32_t w1 = W[1];
          uint32_t wa = __funnelshift_r(W[0], w1, sh), wb = __funnelshift_r(w1, W[2], sh);
          if (rem < 8) {  // bytes past the row end are zero
            if (rem < 4) { wa &= (1u << (rem << 3)) - 1u; wb = 0u; }
            else wb &= (1u << ((rem - 4) << 3)) - 1u;
          }
          p01 = __byte_perm(wa, 0u, 0x4140);
          p23 = __byte_perm(wa, 0u, 0x4342);
          q01 = __byte_perm(wb, 0u, 0x4140);
          q23 = __byte_perm(wb, 0u, 0x4342);
          rs = __dp4a(wa, 0x01010101u, __dp4a(wb, 0x01010101u, 0u));
        } else {  // off is even: the volume and its slices are 2-byte aligned
          const uint32_t w1 = W[1], w2 = W[2], w3 = W[3];
          p01 = __funnelshift_r(W[0], w1, sh);
          p23 = __funnelshift_r(w1, w2, sh);
          q01 = __funnelshift_r(w2, w3, sh);
          q23 = __funnelshift_r(w3, W[4], sh);
          if (rem < 8) {  // halfwords past the row end are zero
            const uint32_t keep[4] = {p01, p23, q01, q23};
            uint32_t m[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int lo = 2 * i;  // pixels lo, lo + 1 of the chunk
              m[i] = rem > lo + 1 ? keep[i] : (rem == lo + 1 ? (keep[i] & 0xffffu) : 0u);
            }
            p01 = m[0]; p23 = m[1]; q01 = m[2]; q23 = m[3];
          }
          rs = (p01 & 0xffffu) + (p01 >> 16) + (p23 & 0xffffu) + (p23 >> 16) +
               (q01 & 0xffffu) + (q01 >> 16) + (q23 & 0xffffu) + (q23 >> 16);
        }
        if (rs) {
          pix_atomic<WIDE>(sm, b1, rs);                       // (z, y)
          add8<WIDE>(sm, b2, p01, p23, q01, q23);             // (z, x)
          if (P > 3) add8<WIDE>(sm, b3, p01, p23, q01, q23);  // (y, x+z)
          if (P > 4) add8<WIDE>(sm, b4, p01, p23, q01, q23);  // (y, x-z)
          if constexpr (MANY) {
            add8<WIDE>(sm, b5, p01, p23, q01, q23);             // (y+z, x)
            if (P > 6) add8<WIDE>(sm, b6, p01, p23, q01, q23);  // (y-z, x)
            if (P > 7) add8<WIDE>(sm, b7, p01, p23, q01, q23);  // (z, x+y)
            if (P > 8) add8<WIDE>(sm, b8, p01, p23, q01, q23);  // (z, x-y)
          }
          if constexpr (WIDE) {
            i0[0] += p01 & 0xffffu; i0[1] += p01 >> 16; i0[2] += p23 & 0xffffu; i0[3] += p23 >> 16;
            i0[4] += q01 & 0xffffu; i0[5] += q01 >> 16; i0[6] += q23 & 0xffffu; i0[7] += q23 >> 16;
          } else {  // packed: every pixel sum stays below 2^16
            i0[0] += p01; i0[1] += p23; i0[2] += q01; i0[3] += q23;
          }
        }
        off += slice_bytes;
        b1 += M; b2 += L; b3 += 1; b4 -= 1;
        if constexpr (MANY) { b5 += L; b6 -= L; b7 += F7; b8 += F7; }
      }
      const int b0 = o[0] + y * L + x0;  // (y, x)
      if constexpr (WIDE) {
#pragma unroll
        for (int i = 0; i < 8; ++i) atomicAdd(sm + b0 + i, i0[i]);
      } else {
        add8<false>(sm, b0, i0[0], i0[1], i0[2], i0[3]);
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    head = head_next;
    cur = nxt;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- step 2

// Units per round of the moment stage: a unit's K + 1 power sums (rt_bytes
// each) and its row coordinate fit stage buffer 0 (buffer 1 takes a
// prefetch), at most one unit per thread.
__host__ __device__ __forceinline__ int moment_units(int nt, int K, int rt_bytes) {
  const int u = kSlabWords * 4 / ((K + 1) * rt_bytes + 4);
  return u < nt ? u : nt;
}

// Geometry of image k (the table of dpma.h): S rows of F pixels, and the
// offsets that make its coordinates signed (Sec. 5).
__device__ __forceinline__ void image_geom_dev(const BTask& t, int k, int& S, int& F, int& os, int& of) {
  const int L = t.L, M = t.M, N = t.N;
  os = 0;
  of = 0;
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
}

// Per-image plan of the moment stage, built once per volume.
struct ImgMeta {
  int S, F, os, of;
  int nseg;    // interleaved segments per row
  int ustart;  // first unit of the image ([P] = all units)
};

__device__ __forceinline__ int64_t shfl_xor_v(int64_t v, int m) {
  return __shfl_xor_sync(0xffffffffu, (long long)v, m);
}
__device__ __forceinline__ i128 shfl_xor_v(i128 v, int m) {
  const uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
  const uint64_t l2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)lo, m);
  const uint64_t h2 = __shfl_xor_sync(0xffffffffu, (unsigned long long)hi, m);
  return (i128)(((u128)h2 << 64) | l2);
}

__constant__ StirlingTable c_stir_b = make_stirling();

template <typename UT>
__device__ __forceinline__ UT ring_of(int64_t v) {
  if constexpr (sizeof(UT) == 16) return (UT)(i128)v;
  else return (UT)v;
}

// Power sums R_b = sum_f I(f) (f - of)^b, b <= KK, of the interleaved
// segment f = g, g + nseg, ... < F of one image row, by cascaded sums.  For
// its n pixels I_0 .. I_{n-1}, running A_0 += I_i, A_1 += A_0, ...,
// A_KK += A_{KK-1} leaves A_j = sum_w w^(j)/j! I with w = n - i and w^(j)
// the rising factorial, so Q_b = sum_w w^b I = sum_j (-1)^(b-j) S(b,j) j! A_j
// (Stirling numbers of the second kind).  The signed coordinate is
// f - of = D - nseg w with D = g + nseg n - of, so R_b = sum_k C(b,k)
// D^(b-k) (-nseg)^k Q_k, built by the Pascal recurrence.  Every step is ring
// arithmetic modulo 2^64 (UT = uint64_t) or 2^128, exact because each R_b
// fits RT (the host's bound).  Per pixel: KK + 1 additions, no products.
template <int KK, typename UT, bool WIDE>
__device__ __forceinline__ void seg_power_sums(const uint32_t* sm, int row, int g, int nseg,
                                               int F, int of, UT* R) {
  UT A[KK + 1];
#pragma unroll
  for (int j = 0; j <= KK; ++j) A[j] = 0;
  for (int f = g; f < F; f += nseg) {
    A[0] += (UT)pix_get<WIDE>(sm, row + f);
#pragma unroll
    for (int j = 1; j <= KK; ++j) A[j] += A[j - 1];
  }
  const int n = (F - g + nseg - 1) / nseg;
  const UT step = (UT)0 - (UT)(uint32_t)nseg;  // -nseg in the ring
  UT sc = 1;
#pragma unroll
  for (int b = 0; b <= KK; ++b) {
    UT q = 0;
#pragma unroll
    for (int j = 0; j <= b; ++j) q += ring_of<UT>(c_stir_b.v[b][j]) * A[j];
    R[b] = q * sc;
    sc *= step;
  }
  const UT D = ring_of<UT>((int64_t)g + (int64_t)nseg * n - of);
#pragma unroll
  for (int i = 1; i <= KK; ++i)
#pragma unroll
    for (int b = KK; b >= i; --b) R[b] += D * R[b - 1];
}

// One unit of the moment stage: its power sums into dst[0..K].
template <int KK, typename RT, bool WIDE>
__device__ __forceinline__ void unit_sums(const uint32_t* sm, int row, int g, int nseg, int F,
                                          int of, RT* dst) {
  using UT = typename std::conditional<sizeof(RT) == 16, u128, uint64_t>::type;
  UT R[KK + 1];
  seg_power_sums<KK, UT, WIDE>(sm, row, g, nseg, F, of, R);
#pragma unroll
  for (int b = 0; b <= KK; ++b) dst[b] = (RT)R[b];
}

// Sum of V values over the 32 lanes of a warp by recursive halving: at each
// of the first levels (lane masks 16, 8, ...) a lane keeps half of its values
// and adds its partner's copy of that half, so the shuffles per level halve
// with the values; the last levels are plain butterflies.  On return x[0] is
// the warp total of value *index (index >= V: an empty slot), held by every
// lane whose plain-level bits are the same; *owner marks one of them.
template <int V, typename AT>
__device__ __forceinline__ void warp_sum_halving(AT (&x)[V], int lane, int* index, bool* owner) {
  int base = 0, plain = 0;
  int c = V;
#pragma unroll
  for (int lev = 0; lev < 5; ++lev) {
    const int m = 16 >> lev;
    if (c > 1) {
      const int h = (c + 1) / 2;
      const bool up = (lane & m) != 0;
#pragma unroll
      for (int j = 0; j < h; ++j) {
        const AT hi = (j + h < c) ? x[j + h] : (AT)0;
        const AT send = up ? x[j] : hi;
        const AT keep = up ? hi : x[j];
        x[j] = keep + shfl_xor_v(send, m);
      }
      if (up) base += h;
      c = h;
    } else {
      x[0] += shfl_xor_v(x[0], m);
      plain |= m;
    }
  }
  *index = base;
  *owner = (lane & plain) == 0;
}

// Fold of one round of units into the 2-D moments: T_ab += sum over the
// round's units of image k of s^a R_b.  Job (k, j) takes the powers b1 = j
// and b2 = KK - j together (b1 = b2 = KK / 2 alone), so an image needs
// KK / 2 + 1 jobs and each unit's row powers s^a are formed once per job.
// Its KK + 2 slots: slot i <= KK - b1 is (a = i, b1); slot i > KK - b1 is
// (a = KK + 1 - i, b2).
template <int KK, typename RT, typename AT, int NT>
__device__ __forceinline__ void fold_round(const RT* Rs, const int* Ss, const ImgMeta* meta, int P,
                                           int u0, int nu, i128* Tacc) {
  constexpr int NW = NT / 32, V = KK + 2, JP = KK / 2 + 1;
  constexpr int npairs = (KK + 1) * (KK + 2) / 2, stride = KK + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int job = warp; job < P * JP; job += NW) {
    const int k = job / JP, b1 = job - k * JP, b2 = KK - b1;
    const int lo = max(meta[k].ustart - u0, 0), hi = min(meta[k + 1].ustart - u0, nu);
    if (lo >= hi) continue;  // uniform across the warp
    const bool pair = b1 < b2;
    AT acc[V];
#pragma unroll
    for (int i = 0; i < V; ++i) acc[i] = 0;
    for (int u = lo + lane; u < hi; u += 32) {
      const RT* R = Rs + (size_t)u * stride;
      const AT r1 = (AT)R[b1];
      const AT r2 = pair ? (AT)R[b2] : (AT)0;
      const AT sv = (AT)Ss[u];
      AT sp[KK + 1];
      sp[0] = 1;
#pragma unroll
      for (int a = 1; a <= KK; ++a) sp[a] = sp[a - 1] * sv;
#pragma unroll
      for (int i = 0; i < V; ++i) {
        const bool first = i <= KK - b1;
        const AT w = first ? sp[i <= KK ? i : 0] : sp[i == 0 ? 0 : KK + 1 - i];
        acc[i] += (first ? r1 : r2) * w;
      }
    }
    int idx;
    bool own;
    warp_sum_halving<V, AT>(acc, lane, &idx, &own);
    if (own && idx < V) {
      const bool first = idx <= KK - b1;
      if (first || pair) {
        const int a = first ? idx : KK + 1 - idx, b = first ? b1 : b2;
        // pair (a, b) is number n (n + 1) / 2 + b with n = a + b
        Tacc[k * npairs + (a + b) * (a + b + 1) / 2 + b] += (i128)acc[0];
      }
    }
  }
}

// 2-D moments T_ab (a + b <= K, signed coordinates) of every image of one
// volume held in shared memory (Eq. 1 with the origin shift of Sec. 5), in
// rounds of at most U units:
//  1. unit u = (image k, row s, segment g): row s of image k is cut into
//     nseg_k interleaved segments of about Lseg pixels; the unit's partial
//     power sums R_b = sum over its pixels f of I f^b (by cascaded sums) are
//     stored with s;
//  2. the fold (fold_round): warps take the jobs (k, {b, K - b}); their
//     lanes run over image k's units of the round, accumulating s^a R_b,
//     and the warp totals go into T_ab.
// RT holds a row power sum exactly, AT a 2-D moment (int64 when the host's
// bounds allow, int128 otherwise).
template <typename RT, typename AT, bool WIDE, int NT>
__device__ __forceinline__ void volume_moments(const BTask& t, const uint32_t* sm, void* scratch,
                                               i128* Tacc, ImgMeta* meta, i128* Tout) {
  const int K = t.K, P = t.P;
  const int npairs = (K + 1) * (K + 2) / 2;
  const int stride = K + 1;  // RT words per unit
  const int U = moment_units(NT, K, (int)sizeof(RT));
  RT* Rs = static_cast<RT*>(scratch);
  int* Ss = reinterpret_cast<int*>(Rs + (size_t)U * stride);
  if (threadIdx.x == 0) {
    for (int k = 0; k < P; ++k) {
      ImgMeta& m = meta[k];
      image_geom_dev(t, k, m.S, m.F, m.os, m.of);
    }
    const int Lseg = t.lseg[NT == 512 ? 1 : 0];  // chosen on the host: one round when possible
    int u = 0;
    for (int k = 0; k < P; ++k) {
      meta[k].nseg = (meta[k].F + Lseg - 1) / Lseg;
      meta[k].ustart = u;
      u += meta[k].S * meta[k].nseg;
    }
    meta[P].ustart = u;
  }
  for (int j = threadIdx.x; j < P * npairs; j += NT) Tacc[j] = 0;
  __syncthreads();
  const int units = meta[P].ustart;
  for (int u0 = 0; u0 < units; u0 += U) {
    const int nu = min(U, units - u0);
    if ((int)threadIdx.x < nu) {
      int v = u0 + (int)threadIdx.x, k = 0;
      while (v >= meta[k + 1].ustart) ++k;
      const ImgMeta m = meta[k];
      v -= m.ustart;
      const int s = v / m.nseg, g = v - s * m.nseg;
      const int row = t.img_off[k] + s * m.F;
      RT* dst = Rs + (size_t)threadIdx.x * stride;
      switch (K) {
#define DPMA_UNIT_CASE(kk) \
  case kk: unit_sums<kk, RT, WIDE>(sm, row, g, m.nseg, m.F, m.of, dst); break;
        DPMA_UNIT_CASE(0) DPMA_UNIT_CASE(1) DPMA_UNIT_CASE(2) DPMA_UNIT_CASE(3)
        DPMA_UNIT_CASE(4) DPMA_UNIT_CASE(5) DPMA_UNIT_CASE(6) DPMA_UNIT_CASE(7)
        default: unit_sums<8, RT, WIDE>(sm, row, g, m.nseg, m.F, m.of, dst); break;
#undef DPMA_UNIT_CASE
      }
      Ss[threadIdx.x] = s - m.os;
    }
    __syncthreads();
    switch (K) {
#define DPMA_FOLD_CASE(kk) \
  case kk: fold_round<kk, RT, AT, NT>(Rs, Ss, meta, P, u0, nu, Tacc); break;
      DPMA_FOLD_CASE(0) DPMA_FOLD_CASE(1) DPMA_FOLD_CASE(2) DPMA_FOLD_CASE(3)
      DPMA_FOLD_CASE(4) DPMA_FOLD_CASE(5) DPMA_FOLD_CASE(6) DPMA_FOLD_CASE(7)
      default: fold_round<8, RT, AT, NT>(Rs, Ss, meta, P, u0, nu, Tacc); break;
#undef DPMA_FOLD_CASE
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < P * npairs; j += NT) Tout[j] = Tacc[j];
}

template <typename T, bool WIDE, int NT>
__device__ __forceinline__ void project_any(const BTask& t, uint32_t* sm, uint32_t* slab,
                                            const uint32_t* first, int head0, int sw) {
  if (t.P > 5) project_volume<T, WIDE, true, NT>(t, sm, slab, first, head0, sw);
  else project_volume<T, WIDE, false, NT>(t, sm, slab, first, head0, sw);
}

template <bool WIDE, int NT>
__device__ __forceinline__ void moments_any(const BTask& t, const uint32_t* sm, uint32_t* slab,
                                            i128* Tacc, ImgMeta* meta, i128* Tout) {
  if (t.r64 && t.t64) volume_moments<int64_t, int64_t, WIDE, NT>(t, sm, slab, Tacc, meta, Tout);
  else if (t.r64) volume_moments<int64_t, i128, WIDE, NT>(t, sm, slab, Tacc, meta, Tout);
  else volume_moments<i128, i128, WIDE, NT>(t, sm, slab, Tacc, meta, Tout);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 2 : 1) batch_fused_kernel(FusedParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  i128* Tacc = reinterpret_cast<i128*>(smem_raw);
  __shared__ ImgMeta meta[kMaxImages + 1];
  const int sw = p.slab_words;
  uint32_t* slab = reinterpret_cast<uint32_t*>(smem_raw + kPartBytes);  // [2][sw]
  // stage buffer 1 receives the next volume's stage 0 while the moment
  // stage uses (the first kSlabWords of) buffer 0 as its scratch area
  uint32_t* pre = slab + sw;
  uint32_t* sm = slab + 2 * sw;  // images
  __shared__ int s_first, s_next;
  if (threadIdx.x == 0) s_first = atomicAdd(p.counter, 1);
  __syncthreads();
  int ti = s_first;  // s_first is never written again
  int head_pre = ti < p.ntasks ? fetch_stage<NT>(p.tasks[p.order[ti]], 0, pre, sw) : 0;
  while (ti < p.ntasks) {
    const BTask t = p.tasks[p.order[ti]];
    // the next volume is claimed now and its first stage is copied during
    // this volume's moment stage, so neither latency is exposed
    // (s_next was last read before the previous volume's final barrier)
    if (threadIdx.x == 0) s_next = atomicAdd(p.counter, 1);
    for (int w = threadIdx.x; w < t.words + kSlackWords; w += NT) sm[w] = 0;
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();  // images zeroed, stage 0 in `pre`, s_next visible
    const int next = s_next;
    i128* Tout = p.T + t.t_off;
    if (t.dtype == DPMA_U8) {
      if (t.wide) project_any<uint8_t, true, NT>(t, sm, slab, pre, head_pre, sw);
      else project_any<uint8_t, false, NT>(t, sm, slab, pre, head_pre, sw);
    } else {
      if (t.wide) project_any<uint16_t, true, NT>(t, sm, slab, pre, head_pre, sw);
      else project_any<uint16_t, false, NT>(t, sm, slab, pre, head_pre, sw);
    }
    // the projection ended with a barrier: `pre` is free
    if (next < p.ntasks) head_pre = fetch_stage<NT>(p.tasks[p.order[next]], 0, pre, sw);
    if (t.wide) moments_any<true, NT>(t, sm, slab, Tacc, meta, Tout);
    else moments_any<false, NT>(t, sm, slab, Tacc, meta, Tout);
    __syncthreads();  // s_next, the images and the scratch area are rewritten next
    ti = next;
  }
}

// ---------------------------------------------------------------- step 3

struct BCombParams {
  const BTask* tasks;
  int ntasks;
  int stride;                  // moments per task slot (those of the highest order)
  const int64_t* plans;        // packed plans of every K present
  int off[kMaxK + 1][kMaxK + 1];  // off[K][n]: word offset of degree n of order K
  // divisor D of degree n of order K as odd << shift, with the inverse of odd
  // modulo 2^128 (two words, low first)
  int dshift[kMaxK + 1][kMaxK + 1];
  uint64_t dinv[kMaxK + 1][kMaxK + 1][2];
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
// q = a / d exactly for d = odd << sh (sh < 64): the candidate q is the low
// 128 bits of (a >> sh) times the inverse of odd modulo 2^128, which is the
// quotient whenever the division is exact; q * d == a (in 256 bits) holds
// exactly then, so a remainder or a quotient outside int128 fails the check.
__device__ bool div_exact(const I256& a, int64_t d, int sh, u128 inv, i128* q) {
  const u128 lo = ((u128)a.w[1] << 64) | a.w[0];
  const u128 hi = ((u128)a.w[3] << 64) | a.w[2];
  const u128 as = sh ? ((lo >> sh) | (hi << (128 - sh))) : lo;
  const i128 qc = (i128)(as * inv);
  I256 chk = {{0, 0, 0, 0}};
  mac256(chk, d, qc);
  if (chk.w[0] != a.w[0] || chk.w[1] != a.w[1] || chk.w[2] != a.w[2] || chk.w[3] != a.w[3])
    return false;
  *q = qc;
  return true;
}

// One thread per (volume, moment): M = (C t_sel) / D for the moment's degree.
__global__ void batch_combine_kernel(BCombParams p) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ti = gid / p.stride;
  const int m = (int)(gid % p.stride);
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
  const u128 inv = ((u128)p.dinv[K][n][1] << 64) | p.dinv[K][n][0];
  if (!div_exact(acc, D, p.dshift[K][n], inv, &q)) {
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
  int dshift[kMaxK + 1][kMaxK + 1] = {};
  uint64_t dinv[kMaxK + 1][kMaxK + 1][2] = {};
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
    for (int K = 0; K <= kMaxKBatch; ++K) {
      std::vector<int64_t> w(8192);
      int off[kMaxK + 1];
      const size_t n = pack_combine_plan(K, w.data(), w.size(), off);
      if (n == 0) return cudaErrorInvalidValue;
      for (int d = 0; d <= kMaxK; ++d) dp.off[K][d] = (int)words.size() + off[d];
      for (int d = 0; d <= K; ++d) {
        // D = odd << shift; the inverse of odd modulo 2^128 by Newton's
        // iteration x <- x (2 - odd x), exact to 3 bits at x = odd
        uint64_t D = (uint64_t)w[off[d]];
        if (D == 0) return cudaErrorInvalidValue;
        int sh = 0;
        while ((D & 1) == 0) { D >>= 1; ++sh; }
        const u128 odd = D;
        u128 x = odd;
        for (int it = 0; it < 7; ++it) x *= (u128)2 - odd * x;
        dp.dshift[K][d] = sh;
        dp.dinv[K][d][0] = (uint64_t)x;
        dp.dinv[K][d][1] = (uint64_t)(x >> 64);
      }
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
    bool fused = d.dtype != DPMA_F32;
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
      // one slice with its 16-byte alignment head and the two words a chunk
      // load may read past it fits in one stage buffer
      const int64_t slice_b = d.L * d.M * (int64_t)(d.dtype == DPMA_U8 ? 1 : 2);
      if (pix > (1ll << 30) || slice_b + 30 > (int64_t)(kSlabWords - 8) * 4 ||
          (size_t)(words + kSlackWords) * 4 + kPartBytes + 2 * kSlabWords * 4 > (size_t)kSmemLimit)
        fused = false;
      if (fused) {
        t.vol = d.volume;
        t.L = (int)d.L; t.M = (int)d.M; t.N = (int)d.N;
        t.dtype = d.dtype; t.K = d.K; t.P = P;
        t.words = (int)words;
        // z-blocks per stage: the fewest chunk loads on the busiest thread,
        // counting two loads of overhead per work item
        const int64_t slice_bytes = d.L * d.M * (int64_t)(d.dtype == DPMA_U8 ? 1 : 2);
        const int64_t npos = d.M * ((d.L + kChunk - 1) / kChunk);
        for (int v = 0; v < 3; ++v) {  // the launch shapes of zblock_index
          const int64_t nt = v ? 512 : 256;
          const int64_t G = stage_slices(slice_bytes, (int)d.N, v == 2 ? kSlabWordsBig : kSlabWords);
          int64_t best = -1, bz = 1;
          for (int64_t zg = 1; zg <= std::min<int64_t>(G, 32); ++zg) {
            const int64_t cost = ((npos * zg + nt - 1) / nt) * ((G + zg - 1) / zg + 2);
            if (best < 0 || cost < best) { best = cost; bz = zg; }
          }
          t.zblocks[v] = (int)bz;
        }
        // a row power sum is at most (vmax * line) * maxF^K * maxF
        const double bits = std::log2(vmax * (double)line + 1) + d.K * std::log2((double)maxF + 1) +
                            std::log2((double)maxF + 1);
        t.r64 = bits < 62.0 ? 1 : 0;
        // every 2-D moment and partial sum of absolute terms fits int64
        t.t64 = log2_bound_2d(d.L, d.M, d.N, vmax, d.K) < 62.0 ? 1 : 0;
        // moment-stage segment length: about all pixels over the units of a
        // round (at least 4), raised until every unit fits one round (each
        // round costs a pass of the fold and two barriers) or every row is
        // one segment
        int64_t S_[kMaxImages], F_[kMaxImages], pixels = 0, fmax = 1;
        for (int k = 0; k < P; ++k) {
          ImageGeom g;
          image_geom(k, d.L, d.M, d.N, &g);
          S_[k] = g.S; F_[k] = g.F;
          pixels += g.S * g.F;
          fmax = std::max(fmax, g.F);
        }
        for (int v = 0; v < 2; ++v) {
          const int64_t U = moment_units(v ? 512 : 256, d.K, t.r64 ? 8 : 16);
          int64_t Ls = pixels > 4 * U ? (pixels + U - 1) / U : 4;
          for (;;) {
            int64_t units = 0, next = fmax;
            for (int k = 0; k < P; ++k) {
              const int64_t ns = (F_[k] + Ls - 1) / Ls;
              units += S_[k] * ns;
              if (ns > 1) next = std::min(next, (F_[k] + ns - 2) / (ns - 1));
            }
            if (units <= U || Ls >= fmax) break;
            Ls = std::max(Ls + 1, next);
          }
          t.lseg[v] = (int)Ls;
        }
        t.t_off = c->t_total;
        t.out_off = d.out_offset;
        c->t_total += (int64_t)P * num_2d(d.K);
        c->tasks.push_back(t);
        c->fused_index.push_back(i);
        c->max_words = std::max(c->max_words, (size_t)words);
        c->max_K = std::max(c->max_K, d.K);
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

size_t fused_smem(size_t max_words, int slab_words) {
  return (size_t)kPartBytes + 2 * (size_t)slab_words * 4 + (max_words + kSlackWords) * 4;
}

int slab_words_for(size_t max_words, int threads) {
  return threads == 512 && fused_smem(max_words, kSlabWordsBig) <= (size_t)kSmemLimit ? kSlabWordsBig
                                                                                        : kSlabWords;
}

int fused_per_sm(size_t smem, int threads) {
  int per_sm = 0;
  cudaError_t e;
  if (threads == 512) {
    set_smem<512>(smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fused_kernel<512>, 512, smem);
  } else {
    set_smem<256>(smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_fused_kernel<256>, 256, smem);
  }
  return (e != cudaSuccess || per_sm < 1) ? 1 : per_sm;
}

int fused_grid(size_t smem, int threads, int ntasks) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(sms * fused_per_sm(smem, threads), ntasks));
}

size_t two_cta_smem_limit() {
  int dev = 0, per_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, batch_fused_kernel<256>);
  const int64_t lim = (int64_t)per_sm / 2 - reserved - (int64_t)fa.sharedSizeBytes;
  size_t out = lim > 0 ? (size_t)lim : 0;
  // the occupancy calculator has the last word
  while (out > 0 && fused_per_sm(out, 256) < 2) out = out > 1024 ? out - 1024 : 0;
  return out;
}

cudaError_t prepare_plans() {
  const DevPlans* dp = nullptr;
  return plans_for_device(&dp);
}

cudaError_t enqueue_fused(const BTask* d_tasks, const int* d_order, int n, int max_K,
                          int* d_counters, i128* d_T, const FusedGroup* groups, int ngroups,
                          void* out, int* d_status, cudaStream_t st, const Fork* fk) {
  if (n <= 0) return cudaSuccess;
  const DevPlans* dp = nullptr;
  cudaError_t e = plans_for_device(&dp);
  if (e != cudaSuccess) return e;
  // Two groups run concurrently when a fork is given: the second group's
  // CTAs take each SM as soon as the first group's CTA there has drained its
  // queue, so the first launch's tail overlaps the second launch.
  const bool concurrent = fk && fk->side && ngroups == 2 && groups[0].count > 0 &&
                          groups[1].count > 0;
  if (concurrent) {
    e = cudaEventRecord(fk->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(fk->side, fk->fork, 0);
    if (e != cudaSuccess) return e;
  }
  for (int g = 0; g < ngroups; ++g) {
    const FusedGroup& G = groups[g];
    if (G.count <= 0) continue;
    const cudaStream_t gs = (concurrent && g == 1) ? fk->side : st;
    FusedParams p{};
    p.tasks = d_tasks;
    p.order = d_order + G.first;
    p.ntasks = G.count;
    p.counter = d_counters + g;
    p.T = d_T;
    p.slab_words = G.slab_words;
    if (G.threads == 512) {
      e = set_smem<512>(G.smem);
      if (e != cudaSuccess) return e;
      batch_fused_kernel<512><<<G.grid, 512, G.smem, gs>>>(p);
    } else {
      e = set_smem<256>(G.smem);
      if (e != cudaSuccess) return e;
      batch_fused_kernel<256><<<G.grid, 256, G.smem, gs>>>(p);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (concurrent) {
    e = cudaEventRecord(fk->join, fk->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, fk->join, 0);
    if (e != cudaSuccess) return e;
  }
  BCombParams cp{};
  cp.tasks = d_tasks;
  cp.ntasks = n;
  cp.stride = (int)num_moments(max_K);
  cp.plans = dp->words;
  std::memcpy(cp.off, dp->off, sizeof(cp.off));
  std::memcpy(cp.dshift, dp->dshift, sizeof(cp.dshift));
  std::memcpy(cp.dinv, dp->dinv, sizeof(cp.dinv));
  cp.T = d_T;
  cp.out = static_cast<unsigned char*>(out);
  cp.status = d_status;
  const int64_t nt = 128, total = (int64_t)n * cp.stride;
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
  int* d_counter = nullptr;  // one queue counter per fused group
  int* d_status = nullptr;
  i128* d_T = nullptr;
  batch::FusedGroup groups[batch::kMaxGroups];
  int ngroups = 0;
  std::vector<int> order;  // fused queue: large-footprint volumes, then the others, each largest first
  int n_over = 0;          // volumes whose footprint rules out two CTAs per SM
  int sms = 1;
  void* d_ws = nullptr;  // workspace of the single-volume path
  size_t ws_bytes = 0;
  batch::Fork fork;      // side stream and events of the concurrent second launch
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
  if (b->fork.side) cudaStreamDestroy(b->fork.side);
  if (b->fork.fork) cudaEventDestroy(b->fork.fork);
  if (b->fork.join) cudaEventDestroy(b->fork.join);
  delete b;
}

// Fused launches of plan b: order[0 .. X) in one launch of nt0-thread CTAs
// and order[X .. n) in a second of 256-thread CTAs (none when X = n), each
// with the shared memory of its largest footprint.
void set_split(dpma_batch* b, int X, int nt0) {
  const std::vector<BTask>& tasks = b->cls.tasks;
  const int n = (int)b->order.size();
  size_t w0 = 0, w1 = 0;
  for (int i = 0; i < n; ++i) {
    const size_t w = (size_t)tasks[b->order[i]].words;
    if (i < X) w0 = std::max(w0, w);
    else w1 = std::max(w1, w);
  }
  b->ngroups = 0;
  if (X > 0) {
    batch::FusedGroup& g = b->groups[b->ngroups++];
    g.first = 0; g.count = X; g.threads = nt0;
    g.slab_words = batch::slab_words_for(w0, nt0);
    g.smem = batch::fused_smem(w0, g.slab_words);
    g.grid = batch::fused_grid(g.smem, nt0, X);
  }
  if (X < n) {
    batch::FusedGroup& g = b->groups[b->ngroups++];
    g.first = X; g.count = n - X; g.threads = 256;
    g.slab_words = batch::slab_words_for(w1, 256);
    g.smem = batch::fused_smem(w1, g.slab_words);
    g.grid = batch::fused_grid(g.smem, 256, n - X);
  }
}

// Split used without autotuning: the large-footprint volumes and then the
// largest of the rest up to eight volumes per SM in the first launch (on
// 4096 ROI masks of sizes 8..96, 2, 4, 8 volumes per SM or one launch
// measured 0.468, 0.424, 0.382 and 0.419 ms).
int default_split(const dpma_batch* b) {
  const int n = (int)b->order.size();
  if (b->n_over == 0) return 0;
  return std::min(n, std::max(b->n_over, 8 * b->sms));
}

dpma_status enqueue_batch(dpma_batch* b, void* out, cudaStream_t st, bool singles = true) {
  unsigned char* o = static_cast<unsigned char*>(out);
  cudaError_t e = cudaMemsetAsync(b->d_status, 0, sizeof(int), st);
  if (e != cudaSuccess) return bfail(DPMA_ERR_CUDA, std::string("clear status: ") + cudaGetErrorString(e));
  const int n = (int)b->cls.tasks.size();
  if (n > 0) {
    e = cudaMemsetAsync(b->d_counter, 0, sizeof(int) * batch::kMaxGroups, st);
    if (e == cudaSuccess && b->ngroups == 2 && !b->fork.side) {
      e = cudaStreamCreateWithFlags(&b->fork.side, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork.fork, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork.join, cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
      e = batch::enqueue_fused(b->d_tasks, b->d_order, n, b->cls.max_K, b->d_counter, b->d_T,
                               b->groups, b->ngroups, out, b->d_status, st, &b->fork);
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
    if (d.K > DPMA_MAX_K_BATCH ||
        dpma_workspace_size(d.L, d.M, d.N, (dpma_dtype)d.dtype, d.K) == 0)
      return bfail(DPMA_ERR_INVALID_ARG, at + "bad dimensions, dtype or K (batches: K <= 8)");
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
    // Two launches when the batch mixes footprints: the volumes whose launch
    // fits two 256-thread CTAs per SM run after the others in a launch that
    // keeps two volumes in flight per SM (their barriers and latency-bound
    // moment stages overlap); each group takes its volumes largest first.
    // The first launch also takes the largest of the small-footprint volumes
    // until it holds a few volumes per SM, so that its tail stays short.
    const std::vector<int> lpt = batch::lpt_order(tasks);
    const size_t small_limit = batch::two_cta_smem_limit();
    std::vector<int> small;
    b->order.clear();
    for (int i : lpt) {
      if (batch::fused_smem((size_t)tasks[i].words, kSlabWords) <= small_limit) small.push_back(i);
      else b->order.push_back(i);
    }
    b->n_over = (int)b->order.size();
    b->order.insert(b->order.end(), small.begin(), small.end());
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->sms = std::max(1, sms);
    set_split(b, default_split(b), 512);
    e = cudaMalloc(&b->d_tasks, sizeof(BTask) * tasks.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_order, sizeof(int) * b->order.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int) * batch::kMaxGroups);
    if (e == cudaSuccess)
      e = cudaMalloc(&b->d_T, sizeof(i128) * (size_t)std::max<int64_t>(1, b->cls.t_total));
    if (e != cudaSuccess) return oom(e, "batch buffers");
    e = cudaMemcpy(b->d_tasks, tasks.data(), sizeof(BTask) * tasks.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_order, b->order.data(), sizeof(int) * b->order.size(),
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = batch::prepare_plans();
    if (e != cudaSuccess) return oom(e, "batch upload");
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
    // time the candidate launch shapes on the real inputs, keep the fastest:
    // the large-footprint group at 512 or 256 threads, or all volumes in one
    // launch at either size
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
    // candidates: the split after X volumes (X = the large-footprint ones,
    // or 2 to 24 volumes per SM) with the first launch at 512 or 256
    // threads, or all volumes in one launch (X = n)
    std::vector<std::vector<batch::FusedGroup>> cand;
    const int n = (int)tasks.size();
    std::vector<int> splits = {b->n_over, 2 * b->sms, 4 * b->sms, 8 * b->sms,
                               12 * b->sms, 16 * b->sms, 24 * b->sms, n};
    std::sort(splits.begin(), splits.end());
    splits.erase(std::unique(splits.begin(), splits.end()), splits.end());
    for (int X : splits) {
      if (X < b->n_over || X > n) continue;
      for (int nt : {512, 256}) {
        set_split(b, X, nt);
        cand.emplace_back(b->groups, b->groups + b->ngroups);
      }
    }
    float best = 1e30f;
    std::vector<batch::FusedGroup> keep(b->groups, b->groups + b->ngroups);
    for (const auto& c : cand) {
      std::copy(c.begin(), c.end(), b->groups);
      b->ngroups = (int)c.size();
      enqueue_batch(b, scratch, st, false);
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) enqueue_batch(b, scratch, st, false);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; keep = c; }
    }
    std::copy(keep.begin(), keep.end(), b->groups);
    b->ngroups = (int)keep.size();
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
  const NvtxRange range("dpma: batch run");
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
    case 2: return plan->ngroups ? plan->groups[0].threads : 0;
    case 3: return plan->ngroups ? plan->groups[0].grid : 0;
    case 4: return plan->ngroups ? (int)plan->groups[0].smem : 0;
    case 5: return plan->ngroups;
    case 6: return plan->ngroups > 1 ? plan->groups[1].count : 0;
    case 7: return plan->ngroups > 1 ? plan->groups[1].threads : 0;
    case 8: return plan->ngroups > 1 ? plan->groups[1].grid : 0;
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
