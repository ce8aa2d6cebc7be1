// Serving loop: continuous batching of moment requests (the method of Sec. 3
// applied per request).
//
// submit() copies the caller's host volume into a pooled pinned buffer and
// queues the request.  One scheduler thread admits queued requests in
// arrival order whenever an in-flight slot and enough of the server's device
// arena are free, then launches them at once: the admitted volumes that fit
// on chip go into one fused launch (batch.cu), the others run through the
// single-volume pipeline; launches are spread over several non-blocking
// streams, so uploads, kernels and downloads of different groups overlap.
// A host callback at the end of each group only records completion; the
// scheduler then releases the group's device memory and slots, which admits
// the next requests.  Waiters block on the request's completion.
//
// Requests may name their volume with a key.  The images of a keyed
// single-volume run of an integer volume stay resident in the arena after it
// completes (a float32 run's images are limbs on the volume's own
// quantisation grid, or the fallback's, so float32 keys are not cached); a
// later request for the same key at an order K no higher than the resident one
// needs no upload and no projection (the image set of order K is a prefix of
// every larger order's set, with the same geometry) and runs only the image
// moments and the combine.  Resident images are evicted, least recently used
// first, when admission needs their memory.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dpma.h"
#include "batch_internal.cuh"
#include "dpma_internal.cuh"

namespace dpma {
cudaError_t prepare_combine(int K);
void set_last_error(const char* msg);
dpma_status validate_descs(const dpma_volume_desc* descs, int count);
}  // namespace dpma

using namespace dpma;
using dpma::batch::BTask;

namespace {

dpma_status sfail(dpma_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

size_t elem_size(int dt) { return dt == DPMA_U8 ? 1 : (dt == DPMA_U16 ? 2 : 4); }

// First-fit allocator over one device region (host-side bookkeeping only, so
// releasing memory never synchronises the device).
class Arena {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
    size_ = bytes;
    free_[0] = bytes;
    return true;
  }
  ~Arena() { if (base_) cudaFree(base_); }
  // offset of a block of `bytes` (256-aligned), or SIZE_MAX
  size_t alloc(size_t bytes) {
    bytes = align256(std::max<size_t>(bytes, 256));
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, rest = it->second - bytes;
        free_.erase(it);
        if (rest) free_[off + bytes] = rest;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        sizes_[off] = bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off) {
    auto s = sizes_.find(off);
    if (s == sizes_.end()) return;
    size_t bytes = s->second;
    sizes_.erase(s);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  unsigned char* base() const { return static_cast<unsigned char*>(base_); }
  size_t size() const { return size_; }
  size_t peak() const { return peak_; }

 private:
  void* base_ = nullptr;
  size_t size_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
  std::unordered_map<size_t, size_t> sizes_;
};

// Copies of submitted host volumes into pinned buffers, split over worker
// threads: one thread's memcpy runs well below the host memory bandwidth,
// and submit() must finish the copy before it returns.
class CopyPool {
 public:
  explicit CopyPool(int workers) {
    for (int i = 0; i < workers; ++i) threads_.emplace_back([this] { run(); });
  }
  ~CopyPool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (std::thread& t : threads_) t.join();
  }
  // dst <- src (bytes); returns when the whole copy is done
  void copy(void* dst, const void* src, size_t bytes) {
    constexpr size_t kMinPart = 1u << 20;
    size_t parts = bytes / kMinPart;
    if (parts > threads_.size() + 1) parts = threads_.size() + 1;
    if (parts <= 1) {
      std::memcpy(dst, src, bytes);
      return;
    }
    Done done;
    done.left = (int)parts - 1;
    const size_t step = ((bytes + parts - 1) / parts + 4095) & ~size_t(4095);
    unsigned char* d = static_cast<unsigned char*>(dst);
    const unsigned char* sp = static_cast<const unsigned char*>(src);
    size_t first = step < bytes ? step : bytes;
    {
      std::lock_guard<std::mutex> lk(mu_);
      int queued = 0;
      for (size_t at = first; at < bytes; at += step) {
        const size_t n = (bytes - at) < step ? (bytes - at) : step;
        jobs_.push_back(Part{d + at, sp + at, n, &done});
        ++queued;
      }
      done.left = queued;  // parts past the first, which this thread copies
    }
    cv_.notify_all();
    std::memcpy(d, sp, first);
    std::unique_lock<std::mutex> lk(done.mu);
    done.cv.wait(lk, [&] { return done.left == 0; });
  }

 private:
  struct Done {
    std::mutex mu;
    std::condition_variable cv;
    int left = 0;
  };
  struct Part {
    unsigned char* dst;
    const unsigned char* src;
    size_t n;
    Done* done;
  };
  void run() {
    for (;;) {
      Part p;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || !jobs_.empty(); });
        if (jobs_.empty()) return;  // stop requested and nothing left
        p = jobs_.front();
        jobs_.pop_front();
      }
      std::memcpy(p.dst, p.src, p.n);
      std::lock_guard<std::mutex> lk(p.done->mu);
      if (--p.done->left == 0) p.done->cv.notify_all();
    }
  }
  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_;
  std::deque<Part> jobs_;
  bool stop_ = false;
};

int copy_workers() {
  const unsigned hw = std::thread::hardware_concurrency();
  const int n = hw > 2 ? (int)(hw / 2) : 1;
  return n > 8 ? 8 : n;
}

// Pinned host buffers reused by size class (powers of two from 4 KiB).
class PinnedPool {
 public:
  ~PinnedPool() {
    for (auto& kv : free_)
      for (void* p : kv.second) cudaFreeHost(p);
  }
  void* get(size_t bytes, size_t* cls_out) {
    size_t cls = 4096;
    while (cls < bytes) cls <<= 1;
    *cls_out = cls;
    {
      std::lock_guard<std::mutex> lk(mu_);
      auto& v = free_[cls];
      if (!v.empty()) {
        void* p = v.back();
        v.pop_back();
        return p;
      }
    }
    void* p = nullptr;
    if (cudaHostAlloc(&p, cls, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t cls) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu_);
    free_[cls].push_back(p);
  }

 private:
  std::mutex mu_;
  std::map<size_t, std::vector<void*>> free_;
};

enum State { kPending = 0, kInFlight = 1, kDone = 2 };

// Images of a completed keyed single-volume run kept in the arena.
struct CacheEntry {
  uint64_t key = 0;
  int64_t L = 0, M = 0, N = 0;
  int dtype = 0, K = 0;
  size_t blk = SIZE_MAX;  // arena block [moments | workspace]; images start the workspace
  size_t off_img = 0;
  int refs = 0;           // requests in flight reading the images
  bool stale = false;     // replaced by a newer entry: free once unused
  uint64_t last_use = 0;
};

struct Request {
  uint64_t id = 0;
  uint64_t key = 0;
  dpma_volume_desc d{};  // d.volume: the pinned host copy
  size_t vbytes = 0, obytes = 0, in_cls = 0, out_cls = 0;
  void* h_in = nullptr;
  void* h_out = nullptr;
  bool fused = false;
  size_t ws_bytes = 0;         // single-volume workspace
  size_t t_bytes = 0;          // fused: this volume's 2-D moments
  // arena blocks: fused: blk = [volume | moments | 2-D moments]; single:
  // vblk = [volume], blk = [moments | workspace]; resident hit: blk =
  // [moments | partials | 2-D moments | status] and src holds the images
  size_t blk = SIZE_MAX, vblk = SIZE_MAX;
  size_t off_vol = 0, off_out = 0, off_ws = 0;
  CacheEntry* src = nullptr;
  size_t part_bytes = 0, m2d_bytes = 0;
  double t_submit = 0, t_done = 0;
  State state = kPending;
  dpma_status status = DPMA_OK;
};

// One launch: a fused group of small volumes or one single-volume run.  Its
// control block (device [tasks | order | counter | status] and the pinned host
// staging of the same bytes) is one of the server's preallocated blocks.
struct Group {
  std::vector<Request*> reqs;
  int stream = 0;
  int ctrl = -1;
  dpma_server* srv = nullptr;
};

}  // namespace

struct dpma_server {
  dpma_server_config cfg{};
  int device = 0;
  Arena arena;
  PinnedPool pinned;
  CopyPool copier{copy_workers()};
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  // one control block per in-flight slot (a group holds at least one request)
  unsigned char* ctrl_dev = nullptr;
  unsigned char* ctrl_host = nullptr;
  size_t ctrl_bytes = 0;
  std::vector<int> ctrl_free;

  std::mutex mu;
  std::condition_variable cv_sched;  // scheduler: new requests or completions
  std::condition_variable cv_done;   // waiters
  bool stop = false;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<Group*> completed;  // groups whose callback ran
  int inflight = 0;
  int groups_inflight = 0;
  bool mem_blocked = false;  // the queue head waits for device memory
  std::vector<CacheEntry*> cache;  // resident images of keyed volumes
  uint64_t use_clock = 0;
  uint64_t next_id = 1;

  // statistics
  int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_rejected = 0, n_launches = 0;
  int64_t n_cache_hits = 0;
  int64_t voxels_done = 0;
  double t_first_submit = -1, t_last_done = -1;
  std::vector<double> lat_ms;

  std::thread sched;
};

namespace {

void CUDART_CB on_group_done(void* arg) {
  Group* g = static_cast<Group*>(arg);
  dpma_server* s = g->srv;
  const double t = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  for (Request* r : g->reqs) r->t_done = t;
  s->completed.push_back(g);
  s->cv_sched.notify_all();
}

// Device bytes of a request's main block (see Request::blk) and of its
// separate volume block (single-volume runs only).
size_t main_bytes(const Request* r) {
  if (r->src) return align256(r->obytes) + align256(r->part_bytes) + align256(r->m2d_bytes) + 256;
  if (r->fused) return align256(r->vbytes) + align256(r->obytes) + align256(r->t_bytes);
  return align256(r->obytes) + align256(r->ws_bytes);
}
size_t volume_bytes(const Request* r) { return (r->fused || r->src) ? 0 : align256(r->vbytes); }

// A resident entry for the request's key that serves its order (lock held).
CacheEntry* find_entry(dpma_server* s, const Request* r) {
  if (!r->key || r->fused || r->d.dtype == DPMA_F32) return nullptr;
  for (CacheEntry* e : s->cache)
    if (!e->stale && e->key == r->key && e->L == r->d.L && e->M == r->d.M && e->N == r->d.N &&
        e->dtype == r->d.dtype && e->K >= r->d.K)
      return e;
  return nullptr;
}

// Frees the least recently used idle entry; false if none (lock held).
bool evict_one(dpma_server* s) {
  int best = -1;
  for (int i = 0; i < (int)s->cache.size(); ++i)
    if (s->cache[i]->refs == 0 && (best < 0 || s->cache[i]->last_use < s->cache[best]->last_use))
      best = i;
  if (best < 0) return false;
  s->arena.release(s->cache[best]->blk);
  delete s->cache[best];
  s->cache.erase(s->cache.begin() + best);
  return true;
}

size_t alloc_evicting(dpma_server* s, size_t bytes) {
  size_t off = s->arena.alloc(bytes);
  while (off == SIZE_MAX && evict_one(s)) off = s->arena.alloc(bytes);
  return off;
}

// Layout of a control block for groups of up to max_group requests.
size_t ctrl_tasks_bytes(int max_group) { return align256(sizeof(BTask) * max_group); }
size_t ctrl_order_bytes(int max_group) { return align256(sizeof(int) * max_group); }
size_t ctrl_block_bytes(int max_group) {
  return ctrl_tasks_bytes(max_group) + ctrl_order_bytes(max_group) + 512;  // + counter, status
}

// Marks a group's requests finished and frees what they hold (lock held).
void retire_group(dpma_server* s, Group* g) {
  const int* h_status = g->ctrl >= 0
      ? reinterpret_cast<const int*>(s->ctrl_host + (size_t)g->ctrl * s->ctrl_bytes +
                                     ctrl_tasks_bytes(s->cfg.max_group) +
                                     ctrl_order_bytes(s->cfg.max_group) + 256)
      : nullptr;
  for (size_t i = 0; i < g->reqs.size(); ++i) {
    Request* r = g->reqs[i];
    const int st = h_status ? *h_status : 0;
    if (r->status == DPMA_OK && st != 0)
      r->status = st == DPMA_ERR_TIMEOUT ? DPMA_ERR_TIMEOUT : DPMA_ERR_INTERNAL;
    r->state = kDone;
    const bool was_hit = r->src != nullptr;
    if (r->vblk != SIZE_MAX) s->arena.release(r->vblk);
    r->vblk = SIZE_MAX;
    if (r->src) {  // read resident images: release them
      r->src->refs--;
      if (r->src->stale && r->src->refs == 0) {
        s->arena.release(r->src->blk);
        s->cache.erase(std::find(s->cache.begin(), s->cache.end(), r->src));
        delete r->src;
      }
      r->src = nullptr;
    }
    if (r->key && !r->fused && r->d.dtype != DPMA_F32 && !was_hit && r->status == DPMA_OK &&
        r->blk != SIZE_MAX) {
      // keep this run's images resident for later requests with the same key
      for (CacheEntry* e : s->cache)
        if (e->key == r->key && !e->stale) e->stale = true;
      for (size_t i = 0; i < s->cache.size();) {
        CacheEntry* e = s->cache[i];
        if (e->stale && e->refs == 0) {
          s->arena.release(e->blk);
          delete e;
          s->cache.erase(s->cache.begin() + i);
        } else {
          ++i;
        }
      }
      CacheEntry* e = new CacheEntry();
      e->key = r->key;
      e->L = r->d.L; e->M = r->d.M; e->N = r->d.N;
      e->dtype = r->d.dtype;
      e->K = r->d.K;
      e->blk = r->blk;
      e->off_img = r->off_ws;
      e->last_use = ++s->use_clock;
      s->cache.push_back(e);
      r->blk = SIZE_MAX;
    }
    if (r->blk != SIZE_MAX) s->arena.release(r->blk);
    r->blk = SIZE_MAX;
    s->pinned.put(r->h_in, r->in_cls);
    r->h_in = nullptr;
    s->inflight--;
    if (r->status == DPMA_OK) {
      s->n_completed++;
      s->voxels_done += r->d.L * r->d.M * r->d.N;
      s->lat_ms.push_back(r->t_done - r->t_submit);
      s->t_last_done = std::max(s->t_last_done, r->t_done);
    } else {
      s->n_failed++;
    }
  }
  if (g->ctrl >= 0) s->ctrl_free.push_back(g->ctrl);
  s->groups_inflight--;
  s->mem_blocked = false;
  delete g;
}

void fail_group(dpma_server*, Group* g, dpma_status st) {
  for (Request* r : g->reqs) r->status = st;
}

// Enqueues one group on its stream (no lock held).  Returns false if it
// failed before its completion callback was queued (the caller retires it).
bool launch_group(dpma_server* s, Group* g, bool fused) {
  cudaStream_t st = s->streams[g->stream];
  const int n = (int)g->reqs.size();
  const int mg = s->cfg.max_group;
  unsigned char* cdev = s->ctrl_dev + (size_t)g->ctrl * s->ctrl_bytes;
  unsigned char* chost = s->ctrl_host + (size_t)g->ctrl * s->ctrl_bytes;
  const size_t tb = ctrl_tasks_bytes(mg), ob = ctrl_order_bytes(mg);
  int* h_status = reinterpret_cast<int*>(chost + tb + ob + 256);
  *h_status = 0;
  unsigned char* base = s->arena.base();
  cudaError_t e = cudaSuccess;
  for (Request* r : g->reqs) {
    if (r->src) continue;  // resident images: nothing to upload
    e = cudaMemcpyAsync(base + r->off_vol, r->h_in, r->vbytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess && !fused && g->reqs[0]->src) {
    // steps 2 and 3 on the resident images (the first P images of the order
    // they were made at, with the same geometry)
    Request* r = g->reqs[0];
    const bool fl = r->d.dtype == DPMA_F32;
    const ImageSet set = make_image_set(r->d.L, r->d.M, r->d.N, r->d.K, fl);
    unsigned char* part = base + r->off_ws;
    unsigned char* m2d = part + align256(r->part_bytes);
    int* status = reinterpret_cast<int*>(m2d + align256(r->m2d_bytes));
    e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = launch_image_moments(base + r->src->off_img, set, r->d.K, fl, part, m2d, st);
    if (e == cudaSuccess) e = launch_combine(m2d, r->d.K, fl, base + r->off_out, status, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  } else if (e == cudaSuccess && fused) {
    // descriptors of the device copies; moments land at arena offsets and each
    // volume's 2-D moments in its own block (T is the arena seen as int128)
    std::vector<dpma_volume_desc> dd(n);
    for (int i = 0; i < n; ++i) {
      dd[i] = g->reqs[i]->d;
      dd[i].volume = base + g->reqs[i]->off_vol;
      dd[i].out_offset = (int64_t)g->reqs[i]->off_out;
    }
    batch::Classified c;
    batch::classify(dd.data(), n, &c);
    if ((int)c.tasks.size() != n) { fail_group(s, g, DPMA_ERR_INTERNAL); return false; }
    for (int i = 0; i < n; ++i) c.tasks[i].t_off = (int64_t)(g->reqs[i]->off_ws / sizeof(i128));
    const std::vector<int> order = batch::lpt_order(c.tasks);
    std::memcpy(chost, c.tasks.data(), sizeof(BTask) * n);
    std::memcpy(chost + tb, order.data(), sizeof(int) * n);
    e = cudaMemcpyAsync(cdev, chost, tb + ob, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cdev + tb + ob, 0, 512, st);
    if (e == cudaSuccess) {
      batch::FusedGroup grp;
      grp.count = n;
      grp.slab_words = batch::slab_words_for(c.max_words, 512);
      grp.smem = batch::fused_smem(c.max_words, grp.slab_words);
      grp.threads = 512;
      grp.grid = batch::fused_grid(grp.smem, 512, n);
      e = batch::enqueue_fused(reinterpret_cast<const BTask*>(cdev),
                               reinterpret_cast<const int*>(cdev + tb), n, c.max_K,
                               reinterpret_cast<int*>(cdev + tb + ob),
                               reinterpret_cast<i128*>(base), &grp, 1, base,
                               reinterpret_cast<int*>(cdev + tb + ob + 256), st);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_status, cdev + tb + ob + 256, sizeof(int), cudaMemcpyDeviceToHost, st);
  } else if (e == cudaSuccess) {
    Request* r = g->reqs[0];
    const dpma_status ds =
        dpma_moments_async(base + r->off_vol, r->d.L, r->d.M, r->d.N, (dpma_dtype)r->d.dtype,
                           r->d.K, base + r->off_out, st, base + r->off_ws, r->ws_bytes);
    if (ds != DPMA_OK) {
      fail_group(s, g, ds);
      cudaStreamSynchronize(st);
      return false;
    }
    // a single-volume layout keeps its status word in its last 256 bytes
    e = cudaMemcpyAsync(h_status, base + r->off_ws + r->ws_bytes - 256, sizeof(int),
                        cudaMemcpyDeviceToHost, st);
  }
  for (Request* r : g->reqs) {
    if (e != cudaSuccess) break;
    e = cudaMemcpyAsync(r->h_out, base + r->off_out, r->obytes, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaLaunchHostFunc(st, on_group_done, g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail_group(s, g, DPMA_ERR_CUDA);
    cudaStreamSynchronize(st);  // queued work must finish before its memory is reused
    return false;
  }
  return true;
}

void scheduler(dpma_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_sched.wait(lk, [&] {
        if (!s->completed.empty()) return true;
        if (s->stop && s->groups_inflight == 0) return true;
        return !s->stop && !s->mem_blocked && !s->pending.empty() &&
               s->inflight < s->cfg.max_inflight;
      });
      for (Group* g : s->completed) retire_group(s, g);
      const bool had_completions = !s->completed.empty();
      s->completed.clear();
      if (had_completions) s->cv_done.notify_all();
      if (s->stop) {
        if (s->groups_inflight == 0) {
          for (Request* r : s->pending) {
            r->status = DPMA_ERR_REJECTED;
            r->state = kDone;
            s->pinned.put(r->h_in, r->in_cls);
            r->h_in = nullptr;
            s->n_failed++;
          }
          s->pending.clear();
          s->cv_done.notify_all();
          return;
        }
        continue;
      }
      // admission in arrival order while a slot and device memory are free
      const NvtxRange admit_range("dpma: server admission");
      while (!s->pending.empty() && s->inflight + (int)admitted.size() < s->cfg.max_inflight) {
        Request* r = s->pending.front();
        CacheEntry* hit = find_entry(s, r);
        if (hit) {  // size the block for steps 2 and 3 alone; pin the images
          const bool fl = r->d.dtype == DPMA_F32;
          const ImageSet set = make_image_set(r->d.L, r->d.M, r->d.N, r->d.K, fl);
          r->part_bytes = moments2d_partials_bytes(set, r->d.K, fl);
          r->m2d_bytes = (size_t)set.P * num_2d(r->d.K) * (fl ? 8 : 16);
          r->src = hit;
          hit->refs++;
        }
        const size_t off = alloc_evicting(s, main_bytes(r));
        size_t voff = SIZE_MAX;
        if (off != SIZE_MAX && volume_bytes(r)) {
          voff = alloc_evicting(s, volume_bytes(r));
          if (voff == SIZE_MAX) s->arena.release(off);
        }
        if (off == SIZE_MAX || (volume_bytes(r) && voff == SIZE_MAX)) {
          if (hit) {
            hit->refs--;
            r->src = nullptr;
          }
          s->mem_blocked = true;  // wait for a completion to free memory
          break;
        }
        r->blk = off;
        r->vblk = voff;
        if (r->fused) {  // [volume | moments | 2-D moments]
          r->off_vol = off;
          r->off_out = off + align256(r->vbytes);
          r->off_ws = r->off_out + align256(r->obytes);
        } else {  // [moments | workspace] (+ the volume block), or [moments | step 2-3 scratch]
          r->off_vol = voff;
          r->off_out = off;
          r->off_ws = off + align256(r->obytes);
        }
        if (hit) {
          hit->last_use = ++s->use_clock;
          s->n_cache_hits++;
        }
        r->state = kInFlight;
        s->pending.pop_front();
        admitted.push_back(r);
      }
      s->inflight += (int)admitted.size();
    }
    if (admitted.empty()) continue;
    // fused groups of up to max_group small volumes; one group per large one
    std::vector<Group*> groups;
    std::vector<bool> fused_flag;
    Group* cur = nullptr;
    for (Request* r : admitted) {
      if (r->fused) {
        if (!cur || (int)cur->reqs.size() >= s->cfg.max_group) {
          cur = new Group();
          groups.push_back(cur);
          fused_flag.push_back(true);
        }
        cur->reqs.push_back(r);
      } else {
        Group* g = new Group();
        g->reqs.push_back(r);
        groups.push_back(g);
        fused_flag.push_back(false);
      }
    }
    for (size_t i = 0; i < groups.size(); ++i) {
      Group* g = groups[i];
      g->srv = s;
      g->stream = s->next_stream;
      s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->groups_inflight++;
        s->n_launches++;
        g->ctrl = s->ctrl_free.back();  // groups in flight <= requests in flight <= slots
        s->ctrl_free.pop_back();
      }
      if (!launch_group(s, g, fused_flag[i])) {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request* r : g->reqs) r->t_done = now_ms();
        s->completed.push_back(g);
      }
    }
  }
}

}  // namespace

extern "C" {

dpma_status dpma_server_create(const dpma_server_config* cfg, dpma_server** out) {
  if (!out) return sfail(DPMA_ERR_INVALID_ARG, "null server pointer");
  *out = nullptr;
  dpma_server_config c{};
  if (cfg) c = *cfg;
  if (c.device_bytes < 0 || c.max_inflight < 0 || c.streams < 0 || c.max_group < 0 ||
      c.max_pending < 0)
    return sfail(DPMA_ERR_INVALID_ARG, "negative configuration value");
  if (c.max_inflight == 0) c.max_inflight = 64;
  if (c.streams == 0) c.streams = 4;
  if (c.max_group == 0) c.max_group = 256;
  if (c.max_pending == 0) c.max_pending = 4096;
  if (c.streams > 64) return sfail(DPMA_ERR_INVALID_ARG, "at most 64 streams");
  dpma_server* s = new dpma_server();
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) { delete s; return sfail(DPMA_ERR_CUDA, "no current CUDA device"); }
  if (c.device_bytes == 0) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) { delete s; return sfail(DPMA_ERR_CUDA, "cudaMemGetInfo failed"); }
    c.device_bytes = (int64_t)(fr / 4);
  }
  s->cfg = c;
  if (!s->arena.init((size_t)c.device_bytes)) {
    delete s;
    return sfail(DPMA_ERR_OOM, "server device arena");
  }
  s->ctrl_bytes = ctrl_block_bytes(c.max_group);
  e = cudaMalloc(&s->ctrl_dev, s->ctrl_bytes * c.max_inflight);
  if (e == cudaSuccess) e = cudaHostAlloc(&s->ctrl_host, s->ctrl_bytes * c.max_inflight, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    cudaFree(s->ctrl_dev);
    delete s;
    return sfail(DPMA_ERR_OOM, "server control blocks");
  }
  for (int i = 0; i < c.max_inflight; ++i) s->ctrl_free.push_back(i);
  for (int i = 0; i < c.streams; ++i) {
    cudaStream_t st = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) break;
    s->streams.push_back(st);
  }
  // every plan resident before serving starts: nothing synchronises later
  for (int K = 0; K <= DPMA_MAX_K_BATCH && e == cudaSuccess; ++K) e = prepare_combine(K);
  if (e == cudaSuccess) e = batch::prepare_plans();
  if (e != cudaSuccess) {
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    cudaFree(s->ctrl_dev);
    cudaFreeHost(s->ctrl_host);
    delete s;
    return sfail(DPMA_ERR_CUDA, std::string("server setup: ") + cudaGetErrorString(e));
  }
  s->sched = std::thread(scheduler, s);
  *out = s;
  return DPMA_OK;
}

dpma_status dpma_server_submit(dpma_server* s, const dpma_volume_desc* desc, uint64_t* ticket) {
  return dpma_server_submit_keyed(s, desc, 0, ticket);
}

dpma_status dpma_server_submit_keyed(dpma_server* s, const dpma_volume_desc* desc, uint64_t key,
                                     uint64_t* ticket) {
  // latency runs from entry to this call (before the pinned copy) to completion
  const double t_entry = now_ms();
  const NvtxRange range("dpma: server submit");
  if (!s || !desc || !ticket) return sfail(DPMA_ERR_INVALID_ARG, "null argument");
  dpma_volume_desc d = *desc;
  d.out_offset = 0;
  dpma_status vs = validate_descs(&d, 1);
  if (vs != DPMA_OK) return vs;
  Request* r = new Request();
  r->vbytes = (size_t)d.L * d.M * d.N * elem_size(d.dtype);
  // moments as the caller receives them: int128 for integer volumes, double for float32
  r->obytes = (size_t)num_moments(d.K) * (d.dtype == DPMA_F32 ? 8 : 16);
  batch::Classified c;
  batch::classify(&d, 1, &c);
  r->fused = !c.tasks.empty();
  if (r->fused) r->t_bytes = (size_t)c.t_total * sizeof(i128);
  else r->ws_bytes = dpma_workspace_size(d.L, d.M, d.N, (dpma_dtype)d.dtype, d.K);
  r->key = key;
  if (main_bytes(r) + volume_bytes(r) > s->arena.size()) {
    delete r;
    std::lock_guard<std::mutex> lk(s->mu);
    s->n_rejected++;
    return sfail(DPMA_ERR_REJECTED, "request needs more device memory than the server holds");
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->pending.size() >= s->cfg.max_pending || s->stop) {
      s->n_rejected++;
      delete r;
      return sfail(DPMA_ERR_REJECTED, "server queue is full");
    }
  }
  r->h_in = s->pinned.get(r->vbytes, &r->in_cls);
  r->h_out = s->pinned.get(r->obytes, &r->out_cls);
  if (!r->h_in || !r->h_out) {
    s->pinned.put(r->h_in, r->in_cls);
    s->pinned.put(r->h_out, r->out_cls);
    delete r;
    return sfail(DPMA_ERR_OOM, "pinned host memory");
  }
  s->copier.copy(r->h_in, d.volume, r->vbytes);  // the caller's buffer is free on return
  r->d = d;
  r->d.volume = r->h_in;
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = t_entry;
  if (s->t_first_submit < 0) s->t_first_submit = r->t_submit;
  s->n_submitted++;
  s->reqs[r->id] = r;
  s->pending.push_back(r);
  *ticket = r->id;
  s->cv_sched.notify_all();
  return DPMA_OK;
}

int dpma_server_poll(dpma_server* s, uint64_t ticket) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return -1;
  return it->second->state == kDone ? 1 : 0;
}

dpma_status dpma_server_wait(dpma_server* s, uint64_t ticket, int64_t timeout_ms, void* host_out) {
  if (!s) return sfail(DPMA_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(DPMA_ERR_INVALID_ARG, "unknown ticket");
  Request* r = it->second;
  auto done = [&] { return r->state == kDone; };
  if (timeout_ms < 0) s->cv_done.wait(lk, done);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
    return sfail(DPMA_ERR_TIMEOUT, "request not finished yet");
  const dpma_status st = r->status;
  if (st == DPMA_OK && host_out) std::memcpy(host_out, r->h_out, r->obytes);
  s->reqs.erase(it);
  lk.unlock();
  s->pinned.put(r->h_out, r->out_cls);
  delete r;
  if (st != DPMA_OK) return sfail(st, "request failed");
  return DPMA_OK;
}

dpma_status dpma_server_stats(dpma_server* s, dpma_server_counters* out, int reset) {
  if (!s || !out) return sfail(DPMA_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  dpma_server_counters r{};
  r.submitted = s->n_submitted;
  r.completed = s->n_completed;
  r.failed = s->n_failed;
  r.rejected = s->n_rejected;
  r.pending = (int64_t)s->pending.size();
  r.inflight = s->inflight;
  r.launches = s->n_launches;
  r.cache_hits = s->n_cache_hits;
  r.resident_volumes = (int64_t)s->cache.size();
  r.device_bytes_peak = (int64_t)s->arena.peak();
  std::vector<double> v = s->lat_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, q * v.size() - 1e-9));
      return v[i];
    };
    r.p50_ms = pct(0.50);
    r.p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    r.mean_ms = sum / v.size();
    r.max_ms = v.back();
  }
  if (s->n_completed > 0 && s->t_last_done > s->t_first_submit) {
    const double span_s = (s->t_last_done - s->t_first_submit) * 1e-3;
    r.volumes_per_s = s->n_completed / span_s;
    r.voxels_per_s = s->voxels_done / span_s;
  }
  *out = r;
  if (reset) {
    s->n_submitted = s->n_completed = s->n_failed = s->n_rejected = s->n_launches = 0;
    s->n_cache_hits = 0;
    s->voxels_done = 0;
    s->lat_ms.clear();
    s->t_first_submit = s->t_last_done = -1;
  }
  return DPMA_OK;
}

dpma_status dpma_server_destroy(dpma_server* s) {
  if (!s) return DPMA_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_sched.notify_all();
  }
  if (s->sched.joinable()) s->sched.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& kv : s->reqs) {
    s->pinned.put(kv.second->h_in, kv.second->in_cls);
    s->pinned.put(kv.second->h_out, kv.second->out_cls);
    delete kv.second;
  }
  for (CacheEntry* e : s->cache) delete e;  // their memory goes with the arena
  cudaFree(s->ctrl_dev);
  cudaFreeHost(s->ctrl_host);
  delete s;
  return DPMA_OK;
}

}  // extern "C"
