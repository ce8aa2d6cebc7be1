// Step 1 for the images of orders 9 and 10 (Sec. 3.1, the further families
// named after Eq. 9): image 9, the arctan(1/2) rotation about y with pixel
// (y, x+2z), and image 10, the isometric projection with pixel
// (x+z, 2y+x-z+N-1).  Integer volumes only.
//
// These images run as a second pass beside the fused projection of images
// 0-8: a CTA takes rows (y, z) of the volume, its threads walk x, and every
// non-zero voxel goes to its pixel with red.global.add.u32 (exact: a line of
// these directions holds at most 65536 voxels, so pixel sums of uint16 data
// stay below 2^32).  Image 9's pixels are consecutive along x, so a warp's
// reductions coalesce; image 10's step F_10 + 1 along x and do not.
#include "dpma_internal.cuh"

namespace dpma {

namespace {

constexpr int kExtraThreads = 128;

__device__ __forceinline__ void red_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(kExtraThreads)
    k1_extra_kernel(const T* __restrict__ vol, int64_t L, int64_t M, int64_t z0, int64_t nrows,
                    int k_end, ImageSet set, uint32_t* __restrict__ img) {
  uint32_t* const im9 = img + set.base[9];
  uint32_t* const im10 = k_end > 10 ? img + set.base[10] : nullptr;
  const int64_t F9 = set.F[9], F10 = k_end > 10 ? set.F[10] : 0;
  const int64_t of10 = k_end > 10 ? set.off_f[10] : 0;
  for (int64_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int64_t z = z0 + r / M, y = r % M;
    const T* row = vol + (z * M + y) * L;
    // image 9: row y, column x + 2z;  image 10: row x + z, column 2y + x - z + N-1
    uint32_t* const p9 = im9 + y * F9 + 2 * z;
    uint32_t* const p10 = im10 ? im10 + z * F10 + (2 * y - z + of10) : nullptr;
    for (int64_t x = threadIdx.x; x < L; x += kExtraThreads) {
      const uint32_t v = (uint32_t)row[x];
      if (v == 0) continue;
      red_add_u32(p9 + x, v);
      if (p10) red_add_u32(p10 + x * (F10 + 1), v);
    }
  }
}

}  // namespace

cudaError_t launch_project_extra(const ProjectArgs& a, cudaStream_t st) {
  if (a.set.P <= 9) return cudaSuccess;
  if (a.dtype != 0 && a.dtype != 1) return cudaErrorInvalidValue;
  const int64_t z0 = a.nz > 0 ? a.z0 : 0;
  const int64_t nz = a.nz > 0 ? a.nz : a.N;
  const int64_t nrows = nz * a.M;
  if (nrows <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 16;
  const unsigned grid = (unsigned)(nrows < cap ? nrows : cap);
  uint32_t* img = static_cast<uint32_t*>(a.images);
  if (a.dtype == 0)
    k1_extra_kernel<uint8_t><<<grid, kExtraThreads, 0, st>>>(
        static_cast<const uint8_t*>(a.vol), a.L, a.M, z0, nrows, a.set.P, a.set, img);
  else
    k1_extra_kernel<uint16_t><<<grid, kExtraThreads, 0, st>>>(
        static_cast<const uint16_t*>(a.vol), a.L, a.M, z0, nrows, a.set.P, a.set, img);
  return cudaGetLastError();
}

}  // namespace dpma
