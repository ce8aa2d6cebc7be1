// Step 1 on integer lanes: dispatch by element type and image count, the
// tensor-map encoder, and the kernel that clears the images and samples a
// float volume's magnitude for the quantisation grid.
#include <mutex>

#include "k1_int.cuh"

namespace dpma {
namespace k1i {

EncodeTiledFn encode_tiled_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

cudaError_t launch_u8(int P, const IntProjectArgs& a, cudaStream_t st);
cudaError_t launch_u16(int P, const IntProjectArgs& a, cudaStream_t st);
cudaError_t launch_f32(int P, const IntProjectArgs& a, cudaStream_t st);

namespace {

// Grid-stride zeroing with 16-byte stores; warp w of the grid also takes
// sampled rows w, w + W, ... (W warps) of the float volume (row j of the
// sample is volume row j * rows / nsr, jittered inside its stride), and
// block b stores the largest |v| its warps saw (float bits; NaN propagates)
// in sample[b].
__global__ void clear_sample_kernel(uint4* p, int64_t n16, uint4* p2, int64_t n2,
                                    int* status, int* flags,
                                    const float* vol, int64_t L, int64_t M, int64_t z0,
                                    int64_t nz, uint32_t* sample, int64_t nsr,
                                    int64_t row_stride, uint32_t even_fill) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (gid == 0) {
    if (status) *status = 0;
    if (flags) *flags = 0;
  }
  // one sampled row per warp at a time, its loads (16 per lane) in flight
  // together; the first row's loads are issued before the zero stores
  const int64_t rows = M * nz;
  const int64_t step = sample ? rows / nsr : 1;  // >= 1
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31;
  constexpr int kBatch = 16;
  auto row_ptr = [&](int64_t j) {
    const int64_t row =
        row_stride > 0 ? j * row_stride : j * rows / nsr + (step > 1 ? (j * 7919) % step : 0);
    const int64_t y = row % M, z = z0 + row / M;
    return vol + (z * M + y) * L;
  };
  auto absmax = [](float a, float b) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(fabsf(b)));
    return d;
  };
  float m = 0.f;
  int64_t j = gid >> 5;
  float pre[kBatch];
  const float* first = (sample && j < nsr) ? row_ptr(j) : nullptr;
  if (first) {
#pragma unroll
    for (int k = 0; k < kBatch; ++k) {
      const int64_t x = lane + 32 * k;
      pre[k] = x < L ? __ldcs(first + x) : 0.f;
    }
  }
  // words 0 and 2 of each 16-byte block sit at 8-byte aligned addresses
  for (int64_t i = gid; i < n16; i += stride) p[i] = make_uint4(even_fill, 0u, even_fill, 0u);
  for (int64_t i = gid; i < n2; i += stride) p2[i] = make_uint4(0u, 0u, 0u, 0u);
  if (!sample) return;
  // the rest of a row from column c on
  auto rest = [&](const float* src, int64_t c) {
    int64_t x = c + lane;
    for (; x + 32 * (kBatch - 1) < L; x += 32 * kBatch) {
      float v[kBatch];
#pragma unroll
      for (int k = 0; k < kBatch; ++k) v[k] = __ldcs(src + x + 32 * k);
#pragma unroll
      for (int k = 0; k < kBatch; ++k) m = absmax(m, v[k]);
    }
    for (; x < L; x += 32) m = absmax(m, __ldcs(src + x));
  };
  if (first) {
#pragma unroll
    for (int k = 0; k < kBatch; ++k) m = absmax(m, pre[k]);
    rest(first, 32 * kBatch);
  }
  for (j += warps; j < nsr; j += warps) rest(row_ptr(j), 0);
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    float d;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(m), "f"(__shfl_xor_sync(0xffffffffu, m, o)));
    m = d;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      float d;
      asm("max.NaN.f32 %0, %1, %2;" : "=f"(d) : "f"(m), "f"(red[w]));
      m = d;
    }
    sample[blockIdx.x] = __float_as_uint(m);
  }
}

}  // namespace
}  // namespace k1i

bool project_int_supported(const void* vol, int64_t L, int dtype, int P) {
  const int64_t es = dtype == 0 ? 1 : (dtype == 1 ? 2 : 4);
  // images 9 and 10 (integer volumes) come from the second kernel
  const int Pmax = dtype == 2 ? 9 : 11;
  return P >= 3 && P <= Pmax && (L * es) % 16 == 0 &&
         (reinterpret_cast<uintptr_t>(vol) % 16) == 0;
}

cudaError_t launch_project_int(const IntProjectArgs& a, cudaStream_t st) {
  const int P = a.set.P;
  if (!project_int_supported(a.vol, a.L, a.dtype, P)) return cudaErrorInvalidValue;
  const int P9 = P < 9 ? P : 9;  // images 0-8 in the fused pass
  cudaError_t e;
  switch (a.dtype) {
    case 0: e = k1i::launch_u8(P9, a, st); break;
    case 1: e = k1i::launch_u16(P9, a, st); break;
    case 2: e = k1i::launch_f32(P9, a, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || P <= 9) return e;
  // images 9 and 10 of an integer volume
  ProjectArgs pa{};
  pa.vol = a.vol;
  pa.L = a.L; pa.M = a.M; pa.N = a.N;
  pa.dtype = a.dtype;
  pa.images = a.images;
  pa.set = a.set;
  pa.status = a.status;
  pa.z0 = a.z0;
  pa.nz = a.nz;
  return launch_project_extra(pa, st);
}

cudaError_t launch_clear_sample(void* p, size_t bytes, int* status, int* flags, const float* vol,
                                int64_t L, int64_t M, int64_t z0, int64_t nz, uint32_t* sample,
                                int* nsample, cudaStream_t st, int64_t row_stride, void* p2,
                                size_t bytes2, uint32_t even_fill) {
  if ((reinterpret_cast<uintptr_t>(p) & 15) != 0 || (bytes & 15) != 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(p2) & 15) != 0 || (bytes2 & 15) != 0) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t n16 = (int64_t)(bytes / 16);
  int64_t blocks = (n16 + 255) / 256;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
  if (blocks > cap) blocks = cap;
  int64_t nsr = 0;
  if (sample) {
    // about 4096 sampled rows (every row of a small volume), or every
    // row_stride-th row
    const int64_t rows = M * nz;
    nsr = row_stride > 0 ? (rows + row_stride - 1) / row_stride : (rows < 4096 ? rows : 4096);
    if (blocks < 64) blocks = 64;
    if (blocks > kMaxSample) blocks = kMaxSample;
    if (blocks > nsr) blocks = nsr;
  }
  if (blocks < 1) blocks = 1;
  if (nsample) *nsample = sample ? (int)blocks : 0;
  k1i::clear_sample_kernel<<<(unsigned)blocks, 256, 0, st>>>(
      static_cast<uint4*>(p), n16, static_cast<uint4*>(p2), p2 ? (int64_t)(bytes2 / 16) : 0,
      status, flags, vol, L, M, z0, nz, sample, nsr, row_stride, even_fill);
  return cudaGetLastError();
}

}  // namespace dpma
