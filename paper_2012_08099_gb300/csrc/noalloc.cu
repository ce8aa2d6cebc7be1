// dpma_moments_noalloc: the whole moment computation with no device memory
// allocation at all.
//
// Some callers cannot call cudaMalloc: an application whose own memory pool
// already holds the device memory it may use, or a latency-critical loop in
// which the device-wide synchronisation and possible failure of cudaMalloc
// cannot be tolerated.  This entry point runs the same three kernels as
// dpma_moments_async, but its workspace (projection images, partial sums and
// status word) lives in one file-scope __device__ array of kScratchBytes, and
// the combine tables of every order in a second one of kPlanBytes; every GPU
// that loads the library holds both until the process exits.  The caller
// still passes the volume and the output.
//
// Set-up: the first call on a device, with that device current, looks up
// both arrays' device addresses with cudaGetSymbolAddress (the host-side name
// of a __device__ array is only a stand-in and must never be handed to a
// kernel) and copies the combine tables of K = 0..8 into the second array
// (synchronous).  That first call should therefore come before any stream
// capture.  Later calls issue only kernel launches.
//
// Sharing: every call uses the same workspace array and finds the previous
// call's contents there; the call clears what must start at zero.  Two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on the array; callers must serialise them.
//
// Failures on the device (a bounded wait that gave up, a combine division
// that left a remainder) set the status word; a last kernel then overwrites
// every output moment with a sentinel (NaN for float volumes, the most
// negative int128 for integer volumes), so the caller sees them in `out`.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

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

constexpr size_t kScratchBytes = 32ull << 20;  // workspace: 32 MiB
constexpr size_t kWorkBytes = kScratchBytes;
constexpr size_t kPlanWords = 16384;            // combine tables of K = 0..8: 128 KiB
constexpr size_t kPlanBytes = kPlanWords * sizeof(int64_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];
static __device__ __align__(256) int64_t g_noalloc_plans[kPlanWords];

// Per device: both arrays' device addresses and where each order's tables
// start inside the plan array.
struct NoallocDevice {
  unsigned char* scratch = nullptr;
  int64_t* plans = nullptr;
  int off[kMaxK + 1][kMaxK + 1] = {};  // [K][n]: word offset of degree n of order K
};

std::mutex g_mu;
std::unordered_map<int, NoallocDevice> g_devices;

// Overwrites the nm output moments with the failure sentinel when the
// status word is non-zero.
__global__ void poison_on_failure(const int* status, void* out, int nm, int is_float) {
  if (*status == 0) return;
  for (int i = threadIdx.x; i < nm; i += blockDim.x) {
    if (is_float) {
      static_cast<double*>(out)[i] = __longlong_as_double(0x7ff8000000000000ll);
    } else {
      uint64_t* w = static_cast<uint64_t*>(out) + 2 * i;
      w[0] = 0;
      w[1] = 0x8000000000000000ull;
    }
  }
}

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
  if (K < 0 || K > DPMA_MAX_K_BATCH) return fail_with(DPMA_ERR_INVALID_ARG, "K must lie in 0..8");
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

  // per-device set-up: both arrays' device addresses and the combine tables
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_with(DPMA_ERR_CUDA, cudaGetErrorString(e));
  NoallocDevice nd;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_devices.find(dev);
    if (it == g_devices.end()) {
      NoallocDevice fresh;
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return fail_with(DPMA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      fresh.scratch = static_cast<unsigned char*>(ptr);
      ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_plans);
      if (e != cudaSuccess || !ptr)
        return fail_with(DPMA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      fresh.plans = static_cast<int64_t*>(ptr);
      std::vector<int64_t> words;
      std::vector<int64_t> buf(8192);
      for (int k = 0; k <= kMaxKBatch; ++k) {
        int off[kMaxK + 1];
        const size_t nw = pack_combine_plan(k, buf.data(), buf.size(), off);
        if (nw == 0) return fail_with(DPMA_ERR_INTERNAL, "combine plan unavailable");
        for (int n = 0; n <= kMaxK; ++n) fresh.off[k][n] = off[n] + (int)words.size();
        words.insert(words.end(), buf.begin(), buf.begin() + nw);
      }
      if (words.size() > kPlanWords) return fail_with(DPMA_ERR_INTERNAL, "combine tables too large");
      e = cudaMemcpyToSymbol(g_noalloc_plans, words.data(), words.size() * sizeof(int64_t));
      if (e != cudaSuccess)
        return fail_with(DPMA_ERR_CUDA, std::string("cudaMemcpyToSymbol: ") + cudaGetErrorString(e));
      it = g_devices.emplace(dev, fresh).first;
    }
    nd = it->second;
  }
  unsigned char* ws = nd.scratch;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

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
    e = launch_combine_packed(nd.plans, nd.off[K], ws + off_m2d, K, fl, out,
                              reinterpret_cast<int*>(ws + off_status), st);
  if (e == cudaSuccess) {
    poison_on_failure<<<1, 256, 0, st>>>(reinterpret_cast<const int*>(ws + off_status), out,
                                         num_moments(K), fl ? 1 : 0);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return fail_with(DPMA_ERR_CUDA, cudaGetErrorString(e));
  return DPMA_OK;
}

