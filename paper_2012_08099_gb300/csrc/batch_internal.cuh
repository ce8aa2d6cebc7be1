// Internal interface of the batched path (batch.cu), shared by the batch plan
// of the C ABI and the serving loop (server.cu).
#pragma once
#include <vector>

#include "../../include/dpma.h"
#include "dpma_internal.cuh"

namespace dpma {
namespace batch {

// One volume of a fused launch (device-resident task table entry).
struct BTask {
  const void* vol;
  int L, M, N;
  int dtype, K, P;
  int wide;   // 1: 32-bit pixels, 0: 16-bit pixels
  int r64;    // 1: row power sums fit int64
  int t64;    // 1: 2-D moments fit int64
  int words;  // 32-bit words of shared memory the images take
  int zblocks[3];  // z-blocks per projection stage at 256 threads, and at 512 with standard or big stage buffers
  int lseg[2];     // pixels per row segment of the moment stage at 256 and 512 threads
  int img_off[kMaxImages];  // first pixel of each image (even, in pixel units)
  int64_t t_off;            // first 2-D moment of this volume in T (int128 units)
  int64_t out_off;          // byte offset of this volume's moments in the output
};

struct Classified {
  std::vector<BTask> tasks;       // fused volumes, in descriptor order
  std::vector<int> fused_index;   // descriptor index of each task
  std::vector<int> single;        // descriptors for the single-volume path
  int64_t t_total = 0;            // int128 2-D moments of all tasks
  size_t max_words = 0;           // largest image footprint in 32-bit words
  int max_K = 0;                  // highest order among the fused tasks
};

// Sorts valid descriptors into fused tasks (integer volumes whose z-slice and
// images fit in shared memory) and single-volume ones.  Host only.
void classify(const dpma_volume_desc* d, int n, Classified* c);
// Processing order of the fused queue: largest volumes first.
std::vector<int> lpt_order(const std::vector<BTask>& tasks);
// Dynamic shared memory of a fused launch whose largest task takes max_words
// and whose two stage buffers hold slab_words words each.
size_t fused_smem(size_t max_words, int slab_words);
// Stage-buffer words of a fused launch: big buffers for a 512-thread launch
// whose images leave room for them, the standard size otherwise.
int slab_words_for(size_t max_words, int threads);
// CTAs of a fused launch: resident capacity, at most ntasks.
int fused_grid(size_t smem, int threads, int ntasks);
// Resident CTAs per SM of a fused launch.
int fused_per_sm(size_t smem, int threads);
// Largest dynamic shared memory of a 256-thread fused launch with two CTAs
// resident per SM.
size_t two_cta_smem_limit();
// Packed combine plans of every order 0..8 resident on the current device
// (built once per device; synchronous the first time).
cudaError_t prepare_plans();

// One persistent fused launch over the tasks order[first .. first + count).
struct FusedGroup {
  int first = 0, count = 0;
  size_t smem = 0;
  int threads = 512, grid = 0;
  int slab_words = 0;
};
constexpr int kMaxGroups = 2;

// Enqueues the fused projection + 2-D moment launches of the groups (each
// with its own queue counter d_counters[g], which must be zero when the
// launch starts: the caller clears them) and the batched combine for all n
// tasks already in device memory, whose highest order is max_K; `out` is the
// base the tasks' out_off refer to; *d_status becomes 7 if an exact division
// left a remainder.  With a side stream and two events (fork, join) the
// second group runs on `side`, concurrently with the first, and the combine
// waits for both; otherwise the groups run one after another on st.
struct Fork {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
cudaError_t enqueue_fused(const BTask* d_tasks, const int* d_order, int n, int max_K,
                          int* d_counters, i128* d_T, const FusedGroup* groups, int ngroups,
                          void* out, int* d_status, cudaStream_t st, const Fork* fk = nullptr);
// Enqueues *dst = max(*dst, *src) on the device.
cudaError_t enqueue_merge_status(const int* src, int* dst, cudaStream_t st);

}  // namespace batch
}  // namespace dpma
