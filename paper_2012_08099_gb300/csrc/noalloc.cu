// dpma_moments_noalloc: the whole moment computation with no device memory
// allocation at all.
//
// Some callers cannot call cudaMalloc: an application whose own memory pool
// already holds the device memory it may use, or a latency-critical loop in
// which the device-wide synchronisation and possible failure of cudaMalloc
// cannot be tolerated.  This entry point runs the same three kernels as
// dpma_moments_async, but its workspace (projection images, partial sums,
// combine tables and status word) lives in one file-scope __device__ array
// of kScratchBytes, which every GPU that loads the library holds until the
// process exits.  The caller still passes the volume and the output.
//
// Set-up: the first call on a device, with that device current, looks up
// the array's device address with cudaGetSymbolAddress (the host-side name
// of a __device__ array is only a stand-in and must never be handed to a
// kernel).  That first call should therefore come before any stream capture.
//
// Sharing: every call uses the same array and finds the previous call's
// contents there; the call clears what must start at zero.  Two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on the array; callers must serialise them.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "../../include/dpma.h"
#include "dpma_internal.cuh"

namespace dpma {
void set_last_error(const char* msg);
size_t pack_combine_plan(int K, int64_t* words, size_t capacity, int off[kMaxK + 1]);
cudaError_t launch_combine_packed(const int64_t* dev_words, const int off[kMaxK + 1],
                                  const void* m2d, int K, bool is_float, void* out, int* status,
                                  cudaStream_t st);
}  // namespace dpma

using namespace dpma;

namespace {

constexpr size_t kScratchBytes = 32ull << 20;  // 32 MiB in total
constexpr size_t kPlanBytes = 64ull << 10;     // combine tables at the front
constexpr size_t kWorkBytes = kScratchBytes - kPlanBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
std::unordered_map<int, unsigned char*> g_scratch_addr;  // device -> address

size_t up(size_t v) { return (v + 255) / 256 * 256; }

dpma_status fail_with(dpma_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

}  // namespace

extern "C" dpma_status dpma_moments_noalloc(const void* volume, int64_t L, int64_t M, int64_t N,
                                            dpma_dtype dtype, int K, void* out, void* stream) {
  if (!volume || !out) return fail_with(DPMA_ERR_INVALID_ARG, "null volume or output pointer");
  if (L < 1 || M < 1 || N < 1 || L > DPMA_MAX_DIM || M > DPMA_MAX_DIM || N > DPMA_MAX_DIM)
    return fail_with(DPMA_ERR_INVALID_ARG, "dimensions must lie in 1..65536");
  if (K < 0 || K > DPMA_MAX_K) return fail_with(DPMA_ERR_INVALID_ARG, "K must lie in 0..8");
  if (dtype != DPMA_U8 && dtype != DPMA_U16 && dtype != DPMA_F32)
    return fail_with(DPMA_ERR_INVALID_ARG, "unknown dtype");
  const bool fl = dtype == DPMA_F32;
  if (fl) {
    if (K * std::log2((double)(L + M + N)) > 100.0)
      return fail_with(DPMA_ERR_OVERFLOW, "coordinate powers exceed the float32 range");
  } else {
    const double vmax = dtype == DPMA_U8 ? 255.0 : 65535.0;
    if (log2_bound_2d(L, M, N, vmax, K) > 125.0 || log2_bound_3d(L, M, N, vmax, K) > 125.0)
      return fail_with(DPMA_ERR_OVERFLOW, "moments could exceed the int128 range");
  }

  // workspace layout inside the array (same sections as dpma_moments_async)
  const ImageSet set = make_image_set(L, M, N, K, fl);
  const size_t img_bytes = (size_t)set.total_elems * (fl ? 8 : 4);
  const size_t part_bytes = moments2d_partials_bytes(set, K, fl);
  const size_t m2d_bytes = (size_t)set.P * num_2d(K) * (fl ? 8 : 16);
  const size_t off_img = 0, off_part = up(off_img + img_bytes);
  const size_t off_m2d = up(off_part + part_bytes), off_status = up(off_m2d + m2d_bytes);
  const size_t need = off_status + 256;
  if (need > kWorkBytes)
    return fail_with(DPMA_ERR_REJECTED,
                     "volume needs " + std::to_string(need) + " bytes of workspace; the static "
                     "scratch of dpma_moments_noalloc holds " + std::to_string(kWorkBytes));

  // per-device set-up: the array's device address
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_with(DPMA_ERR_CUDA, cudaGetErrorString(e));
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch_addr.find(dev);
    if (it == g_scratch_addr.end()) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return fail_with(DPMA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      it = g_scratch_addr.emplace(dev, static_cast<unsigned char*>(ptr)).first;
    }
    base = it->second;
  }
  int64_t* plan_words = reinterpret_cast<int64_t*>(base);
  unsigned char* ws = base + kPlanBytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // combine tables of order K into the front of the array (host-built)
  int64_t host_words[kPlanBytes / sizeof(int64_t)];
  int off[kMaxK + 1];
  const size_t nw = pack_combine_plan(K, host_words, kPlanBytes / sizeof(int64_t), off);
  if (nw == 0) return fail_with(DPMA_ERR_INTERNAL, "combine plan unavailable");
  e = cudaMemcpyAsync(plan_words, host_words, nw * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail_with(DPMA_ERR_CUDA, cudaGetErrorString(e));

  // the three steps; images and the status word must start at zero
  e = launch_clear(ws + off_img, img_bytes, reinterpret_cast<int*>(ws + off_status), st);
  if (e != cudaSuccess) return fail_with(DPMA_ERR_CUDA, cudaGetErrorString(e));
  ProjectArgs a{};
  a.vol = volume;
  a.L = L; a.M = M; a.N = N;
  a.dtype = (int)dtype;
  a.K = K;
  a.images = ws + off_img;
  a.set = set;
  a.status = reinterpret_cast<int*>(ws + off_status);
  e = launch_project(a, st);
  if (e == cudaSuccess)
    e = launch_image_moments(ws + off_img, set, K, fl, ws + off_part, ws + off_m2d, st);
  if (e == cudaSuccess)
    e = launch_combine_packed(plan_words, off, ws + off_m2d, K, fl, out,
                              reinterpret_cast<int*>(ws + off_status), st);
  if (e != cudaSuccess) return fail_with(DPMA_ERR_CUDA, cudaGetErrorString(e));
  return DPMA_OK;
}

