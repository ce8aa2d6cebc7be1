// C ABI of the Discrete Projection Moment library (declared in include/dpma.h).
//
// Host-side argument checks, magnitude bounds, workspace layout and stream
// handling around the three device steps:
//   step 1  launch_project        (Sec. 3.1, Eqs. 4-9)
//   step 2  launch_image_moments  (Eq. 1 with signed coordinates)
//   step 3  launch_combine        (Eqs. 10-16 generalised)
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/dpma.h"
#include "dpma_internal.cuh"

namespace dpma {
cudaError_t prepare_combine(int K);
}

using namespace dpma;

namespace {

thread_local std::string t_last_error;
// flags word of the calling thread's last synchronous float32 call: 0 when
// the quantised pipeline gave the result, 1 / 2 when the compensated
// fallback recomputed it (a voxel beyond the grid / an error bound above the
// tolerance)
thread_local int t_last_flags = 0;

dpma_status fail(dpma_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}

dpma_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(DPMA_ERR_OOM, std::string(where) + ": " + cudaGetErrorString(e));
  }
  return fail(DPMA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool is_float(dpma_dtype d) { return d == DPMA_F32; }

dpma_status check_args(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K) {
  if (L < 1 || M < 1 || N < 1 || L > DPMA_MAX_DIM || M > DPMA_MAX_DIM || N > DPMA_MAX_DIM)
    return fail(DPMA_ERR_INVALID_ARG, "dimensions must lie in 1..65536");
  if (dtype != DPMA_U8 && dtype != DPMA_U16 && dtype != DPMA_F32)
    return fail(DPMA_ERR_INVALID_ARG, "unknown dtype");
  if (K < 0 || K > (dtype == DPMA_F32 ? DPMA_MAX_K_FLOAT : DPMA_MAX_K))
    return fail(DPMA_ERR_INVALID_ARG, "K must lie in 0..10 (0..8 for float32)");
  if (dtype == DPMA_F32) {
    // float-float coordinate powers must stay well inside the float range
    const double maxc = (double)(L + M + N);
    if (K * std::log2(maxc) > 100.0)
      return fail(DPMA_ERR_OVERFLOW, "coordinate powers exceed the float32 range");
  } else {
    const double vmax = dtype == DPMA_U8 ? 255.0 : 65535.0;
    if (log2_bound_2d(L, M, N, vmax, K) > 125.0 || log2_bound_3d(L, M, N, vmax, K) > 125.0)
      return fail(DPMA_ERR_OVERFLOW, "moments could exceed the int128 range");
  }
  return DPMA_OK;
}

struct Layout {
  ImageSet set;
  size_t img_bytes, part_bytes, m2d_bytes;
  size_t off_img, off_part, off_m2d, off_sample, off_status, total;
  // status block: [0] status, [1] flags, [2] e1, [3] B
};

// One workspace serves both float32 pipelines: the quantised-limb one (two
// int32 image sets, int128 partials and moments for 2P images) and its
// compensated fallback (double images, float-pair partials and moments).
Layout layout(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K) {
  Layout w;
  const bool fl = is_float(dtype);
  w.set = make_image_set(L, M, N, K, fl);
  w.img_bytes = (size_t)w.set.total_elems * (fl ? 8 : 4);
  w.part_bytes = moments2d_partials_bytes(w.set, K, fl);
  w.m2d_bytes = (size_t)w.set.P * num_2d(K) * (fl ? 8 : 16);
  if (fl) {
    w.part_bytes = std::max(w.part_bytes, moments2d_partials_bytes_limbs(w.set, K, 2));
    w.m2d_bytes = std::max(w.m2d_bytes, (size_t)2 * w.set.P * num_2d(K) * 16);
  }
  w.off_img = 0;
  w.off_part = align_up(w.off_img + w.img_bytes, 256);
  w.off_m2d = align_up(w.off_part + w.part_bytes, 256);
  w.off_sample = align_up(w.off_m2d + w.m2d_bytes, 256);
  w.off_status = align_up(w.off_sample + (fl ? kMaxSample * sizeof(uint32_t) : 0), 256);
  w.total = w.off_status + 256;
  return w;
}

// Cycles a bounded device wait of the projection may spin (a test hook can
// shorten it).
std::atomic<long long> g_wait_budget{1ll << 31};

// Float32 results of the quantised pipeline are guaranteed within this
// fraction of the moment of |V| (the method's tolerance is 1e-6); a moment
// whose error bound is larger sends the volume to the compensated fallback.
constexpr double kFloatTolerance = 1e-7;

// Library-owned per-device resources.
struct DeviceState {
  std::mutex mu;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* host_vol = nullptr;  // device buffers of dpma_moments_host
  size_t host_vol_bytes = 0;
  void* host_out = nullptr;
  cudaStream_t copy_stream = nullptr;  // host-to-device chunks of dpma_moments_host
  cudaEvent_t chunk_ready = nullptr;
  int* h_status = nullptr;  // pinned: the synchronous calls read the status word here
  void* drt_ws = nullptr;   // workspace of dpma_image_moments_drt without a caller workspace
  size_t drt_ws_bytes = 0;
};

// The pinned host word that receives the device status (a pageable
// destination would make every synchronous call pay a staged copy).
cudaError_t ensure_host_status(DeviceState* s) {
  if (s->h_status) return cudaSuccess;
  return cudaMallocHost(reinterpret_cast<void**>(&s->h_status), 2 * sizeof(int));
}

std::mutex g_states_mu;
std::unordered_map<int, DeviceState*> g_states;

DeviceState* state_for_current_device(int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  if (dev_out) *dev_out = dev;
  std::lock_guard<std::mutex> lk(g_states_mu);
  auto it = g_states.find(dev);
  if (it != g_states.end()) return it->second;
  DeviceState* s = new DeviceState();
  g_states[dev] = s;
  return s;
}

cudaError_t ensure_stream(DeviceState* s) {
  if (s->stream) return cudaSuccess;
  // a blocking stream: it waits for work queued on the legacy default stream
  return cudaStreamCreateWithFlags(&s->stream, cudaStreamDefault);
}

cudaError_t ensure_buffer(void** p, size_t* have, size_t need) {
  if (*have >= need && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, need);
  if (e == cudaSuccess) *have = need;
  return e;
}

// Optional per-stage event timing (profiling aid, off by default).
struct StageEvent {
  int stage;
  int kernels;  // kernel launches the stage made
  cudaEvent_t a, b;
  bool free_a;  // a is the call's first event (b of a stage is a of the next)
};
std::mutex g_timing_mu;
bool g_timing = false;
std::vector<StageEvent> g_pending;
std::vector<cudaEvent_t> g_free_events;
double g_stage_ms[4] = {0, 0, 0, 0};
int64_t g_stage_launches[4] = {0, 0, 0, 0};

cudaEvent_t take_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// One event per stage boundary: the event that ends a stage starts the next.
struct StageRecorder {
  bool on;
  bool first = true;
  cudaStream_t st;
  cudaEvent_t last = nullptr;
  explicit StageRecorder(cudaStream_t s) : st(s) {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    on = g_timing;
    if (on) { last = take_event(); cudaEventRecord(last, st); }
  }
  void mark(int stage, int kernels) {
    if (!on) return;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    cudaEvent_t e = take_event();
    cudaEventRecord(e, st);
    g_pending.push_back({stage, kernels, last, e, first});
    first = false;
    last = e;
  }
  ~StageRecorder() {
    if (!on || !first) return;
    std::lock_guard<std::mutex> lk(g_timing_mu);
    g_free_events.push_back(last);  // recorded but never used
  }
};

// Enqueue the three steps on `st` with workspace `ws` (layout `w`).
size_t elem_size(dpma_dtype d) { return d == DPMA_U8 ? 1 : (d == DPMA_U16 ? 2 : 4); }

// Host volumes arrive in z-chunks: about 4 MB each, at most 16.
int64_t host_chunk_slices(int64_t N, size_t vbytes) {
  int64_t n = (int64_t)(vbytes / (4u << 20));
  n = n < 1 ? 1 : (n > 16 ? 16 : n);
  if (n > N) n = N;
  return (N + n - 1) / n;
}

// The float32 fallback: the compensated float kernels over the whole volume,
// each launch gated on the flags word, so it costs nothing but its launches
// unless the quantised pipeline flagged the volume (a voxel beyond the grid,
// a non-finite voxel, or a moment whose guaranteed error exceeds the
// tolerance).  Then it overwrites images, moments and `out`.
dpma_status enqueue_float_fallback(const void* volume, int64_t L, int64_t M, int64_t N, int K,
                                   void* out, cudaStream_t st, unsigned char* ws, const Layout& w) {
  int* status = reinterpret_cast<int*>(ws + w.off_status);
  const int* gate = status + 1;
  void* images = ws + w.off_img;
  cudaError_t e = launch_clear(images, w.img_bytes, nullptr, st, gate);
  if (e != cudaSuccess) return cuda_fail(e, "clear images (fallback)");
  ProjectArgs a{};
  a.vol = volume;
  a.L = L; a.M = M; a.N = N;
  a.dtype = (int)DPMA_F32;
  a.K = K;
  a.images = images;
  a.set = w.set;
  a.status = status;
  a.gate = gate;
  e = launch_project(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "projection kernel (fallback)");
  e = launch_image_moments(images, w.set, K, true, ws + w.off_part, ws + w.off_m2d, st, gate);
  if (e != cudaSuccess) return cuda_fail(e, "image moment kernel (fallback)");
  e = launch_combine(ws + w.off_m2d, K, true, out, status, st, gate);
  if (e != cudaSuccess) return cuda_fail(e, "combine kernel (fallback)");
  return DPMA_OK;
}

// The fallback as one graph launch.  Five gated launches cost about 25 us of
// stream time even when the gate is closed, so a pipeline that repeats with
// the same buffers runs them as a cached executable graph instead: a
// one-thread gate kernel reads the flags word and sets the condition of an
// IF node whose body is the five launches (captured from
// enqueue_float_fallback; the body's kernels keep their own gate test).  The
// graph bakes in every pointer and size, so it is keyed by all of them, and
// a key is promoted to a graph only when it is seen a second time: one-off
// calls keep the plain gated launches and pay no graph construction.
__global__ void fallback_gate_kernel(const int* flags, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, (*flags & 3) ? 1u : 0u);
}

struct FallbackKey {
  int dev;
  const void* vol;
  int64_t L, M, N;
  int K;
  void* out;
  unsigned char* ws;
  bool operator==(const FallbackKey& o) const {
    return dev == o.dev && vol == o.vol && L == o.L && M == o.M && N == o.N && K == o.K &&
           out == o.out && ws == o.ws;
  }
};
struct FallbackGraph {
  FallbackKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
constexpr size_t kFallbackGraphs = 8;   // cached executable graphs (least recently used out)
constexpr size_t kFallbackSeen = 16;    // keys seen once
std::mutex g_fb_mu;
std::vector<FallbackGraph> g_fb_graphs;  // most recently used last
std::vector<FallbackKey> g_fb_seen;

cudaError_t build_fallback_graph(const FallbackKey& k, cudaStream_t cap, const Layout& w,
                                 FallbackGraph* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  auto fail = [&](cudaError_t err) {
    cudaGraphDestroy(g);
    return err;
  };
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e != cudaSuccess) return fail(e);
  const int* flags = reinterpret_cast<const int*>(k.ws + w.off_status) + 1;
  void* args[] = {&flags, &h};
  cudaKernelNodeParams kp{};
  kp.func = reinterpret_cast<void*>(fallback_gate_kernel);
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.kernelParams = args;
  cudaGraphNode_t gate;
  e = cudaGraphAddKernelNode(&gate, g, nullptr, 0, &kp);
  if (e != cudaSuccess) return fail(e);
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t cond;
  e = cudaGraphAddNode(&cond, g, &gate, nullptr, 1, &np);
  if (e != cudaSuccess) return fail(e);
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(e);
  const dpma_status fs = enqueue_float_fallback(k.vol, k.L, k.M, k.N, k.K, k.out, cap, k.ws, w);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(cap, &captured);
  if (fs != DPMA_OK) return fail(cudaErrorUnknown);
  if (e != cudaSuccess) return fail(e);
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) return fail(e);
  out->key = k;
  out->graph = g;
  out->exec = exec;
  return cudaSuccess;
}

// The fallback into a graph that st is capturing: the gate kernel, then an
// IF node whose body is the five launches (captured on a stream of its own),
// so a replay of the captured graph runs one gate kernel instead of five
// gated launches while the gate is closed.
dpma_status capture_fallback_conditional(const void* volume, int64_t L, int64_t M, int64_t N,
                                         int K, void* out, cudaStream_t st, unsigned char* ws,
                                         const Layout& w, int* launches) {
  *launches = 1;
  // the body's stream first: without it the graph stays as it is and the
  // plain gated launches go into the capture
  cudaStream_t side = nullptr;
  if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    *launches = 5;
    return enqueue_float_fallback(volume, L, M, N, K, out, st, ws, w);
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t cg = nullptr;
  auto fail = [&](cudaError_t err, const char* where) {
    cudaStreamDestroy(side);
    return cuda_fail(err, where);
  };
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return fail(e, "capture info (fallback)");
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, cg, 0, 0);
  if (e != cudaSuccess) return fail(e, "conditional handle (fallback)");
  const int* flags = reinterpret_cast<const int*>(ws + w.off_status) + 1;
  fallback_gate_kernel<<<1, 1, 0, st>>>(flags, h);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(e, "fallback gate kernel");
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &nd);
  if (e != cudaSuccess) return fail(e, "capture info (fallback)");
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t cond;
  e = cudaGraphAddNode(&cond, cg, deps, nullptr, nd, &np);
  if (e != cudaSuccess) return fail(e, "conditional node (fallback)");
  e = cudaStreamBeginCaptureToGraph(side, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  dpma_status fs = DPMA_OK;
  if (e == cudaSuccess) {
    fs = enqueue_float_fallback(volume, L, M, N, K, out, side, ws, w);
    cudaGraph_t body = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(side, &body);
    if (e2 != cudaSuccess && fs == DPMA_OK) fs = cuda_fail(e2, "capture (fallback body)");
  } else {
    fs = cuda_fail(e, "capture (fallback body)");
  }
  cudaStreamDestroy(side);
  if (fs != DPMA_OK) return fs;
  e = cudaStreamUpdateCaptureDependencies(st, &cond, nullptr, 1,
                                          cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return cuda_fail(e, "capture dependencies (fallback)");
  return DPMA_OK;
}

// Enqueues the fallback on st: inside a stream capture the conditional form
// above; otherwise the cached graph of this key, else (building it on a key's
// second use) the plain gated launches.  *launches receives the kernel
// launches issued from the host.
dpma_status enqueue_fallback(const void* volume, int64_t L, int64_t M, int64_t N, int K,
                             void* out, cudaStream_t st, unsigned char* ws, const Layout& w,
                             int* launches) {
  FallbackKey k{};
  if (cudaGetDevice(&k.dev) != cudaSuccess) k.dev = -1;
  k.vol = volume; k.L = L; k.M = M; k.N = N; k.K = K; k.out = out; k.ws = ws;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
                         cs != cudaStreamCaptureStatusNone;
  if (capturing) return capture_fallback_conditional(volume, L, M, N, K, out, st, ws, w, launches);
  if (k.dev >= 0) {
    std::lock_guard<std::mutex> lk(g_fb_mu);
    cudaGraphExec_t exec = nullptr;
    for (size_t i = 0; i < g_fb_graphs.size(); ++i)
      if (g_fb_graphs[i].key == k) {
        FallbackGraph fg = g_fb_graphs[i];
        g_fb_graphs.erase(g_fb_graphs.begin() + i);
        g_fb_graphs.push_back(fg);
        exec = fg.exec;
        break;
      }
    if (!exec) {
      bool seen = false;
      for (const FallbackKey& o : g_fb_seen) seen = seen || (o == k);
      if (seen) {
        cudaStream_t cap = nullptr;
        FallbackGraph fg;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = build_fallback_graph(k, cap, w, &fg);
        if (cap) cudaStreamDestroy(cap);
        if (e == cudaSuccess) {
          if (g_fb_graphs.size() >= kFallbackGraphs) {
            cudaGraphExecDestroy(g_fb_graphs.front().exec);
            cudaGraphDestroy(g_fb_graphs.front().graph);
            g_fb_graphs.erase(g_fb_graphs.begin());
          }
          g_fb_graphs.push_back(fg);
          exec = fg.exec;
        } else {
          cudaGetLastError();  // a failed build leaves the plain launches in use
        }
      } else {
        if (g_fb_seen.size() >= kFallbackSeen) g_fb_seen.erase(g_fb_seen.begin());
        g_fb_seen.push_back(k);
      }
    }
    if (exec) {
      const cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) return cuda_fail(e, "fallback graph launch");
      *launches = 1;
      return DPMA_OK;
    }
  }
  *launches = 5;
  return enqueue_float_fallback(volume, L, M, N, K, out, st, ws, w);
}

// The pipeline on stream st.  With a host source (host_src non-null) the
// volume is copied into `volume` in z-chunks on copy_st, and the projection
// of each chunk starts as soon as its copy has landed, so the copy of the
// next chunk overlaps it; launches over disjoint z-ranges add up to the
// images of the whole volume.
//
// Volumes with 16-byte aligned rows and at most 7 images take the
// integer-lane projection (exact integer images; float32 volumes as two
// quantisation limbs, with the gated compensated fallback behind them); the
// others take the compensated/integer projection of k1_project.cuh.
dpma_status enqueue(const void* volume, int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K,
                    void* out, cudaStream_t st, unsigned char* ws, const Layout& w,
                    const void* host_src = nullptr, cudaStream_t copy_st = nullptr,
                    cudaEvent_t ev = nullptr) {
  const NvtxRange range("dpma: moments");
  cudaError_t e = prepare_combine(K);
  if (e != cudaSuccess) return cuda_fail(e, "combine plan");
  StageRecorder rec(st);
  const bool fl = is_float(dtype);
  void* images = ws + w.off_img;
  int* status = reinterpret_cast<int*>(ws + w.off_status);
  int* flags = status + 1;
  int* scale = status + 2;
  uint32_t* sample = reinterpret_cast<uint32_t*>(ws + w.off_sample);
  const int B = fl ? float_limb_bits(L, M, N, K) : 0;
  const bool lanes = project_int_supported(volume, L, (int)dtype, w.set.P) &&
                     (!fl || B >= kMinLimbBits);
  int ia_nsample = 0;
  int k1_launches = 0;
  if (!lanes) {
    e = launch_clear(images, w.img_bytes, status, st);
  } else {
    // the images (rounded up to 16 bytes: the padding before the next
    // section), the 2-D moments (step 2 adds into them), the status words
    // and, for a device-resident float volume, the magnitude sample
    e = launch_clear_sample(images, align_up(w.img_bytes, 16), status, flags,
                            fl && !host_src ? static_cast<const float*>(volume) : nullptr, L, M,
                            0, N, fl && !host_src ? sample : nullptr, &ia_nsample, st, 0,
                            ws + w.off_m2d, align_up(w.m2d_bytes, 16), fl ? kLimbPairBias : 0u);
  }
  if (e != cudaSuccess) return cuda_fail(e, "clear images");
  rec.mark(0, 1);
  ProjectArgs a{};
  a.vol = volume;
  a.L = L; a.M = M; a.N = N;
  a.dtype = (int)dtype;
  a.K = K;
  a.images = images;
  a.set = w.set;
  a.status = status;
  IntProjectArgs ia{};
  ia.vol = volume;
  ia.L = L; ia.M = M; ia.N = N;
  ia.dtype = (int)dtype;
  ia.images = images;
  ia.set = w.set;
  ia.status = status;
  ia.flags = flags;
  ia.sample = fl ? sample : nullptr;
  ia.limb_bits = B;
  ia.scale_out = fl ? scale : nullptr;
  ia.wait_budget = g_wait_budget.load();
  ia.nsample = ia_nsample;
  if (host_src) {
    const size_t slice = (size_t)L * M * elem_size(dtype);
    int64_t zc = host_chunk_slices(N, slice * N);
    zc += zc & 1;  // even chunks: the integer-lane projection takes z-pairs
    // the staging buffer is rewritten only after all earlier work on st
    e = cudaEventRecord(ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_st, ev, 0);
    if (e == cudaSuccess && lanes && fl) {
      // The quantisation grid must be fixed before the first chunk is
      // projected, yet come from the whole volume: about 1024 rows evenly
      // spread over it are copied ahead of the chunks (one strided copy into
      // their places in the device buffer) and sampled; the chunk copies,
      // which rewrite those rows with the same bytes, wait for the sample.
      const int64_t rows = M * N;
      const int64_t rs = rows > 1024 ? rows / 1024 : 1;
      const size_t row_bytes = (size_t)L * sizeof(float);
      e = cudaMemcpy2DAsync(const_cast<void*>(volume), rs * row_bytes, host_src, rs * row_bytes,
                            row_bytes, (size_t)((rows + rs - 1) / rs), cudaMemcpyHostToDevice,
                            copy_st);
      if (e == cudaSuccess) e = cudaEventRecord(ev, copy_st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
      if (e != cudaSuccess) return cuda_fail(e, "copy sample rows to device");
      e = launch_clear_sample(images, 0, nullptr, nullptr, static_cast<const float*>(volume), L, M,
                              0, N, sample, &ia.nsample, st, rs);
      if (e != cudaSuccess) return cuda_fail(e, "magnitude sample");
      ++k1_launches;
      e = cudaEventRecord(ev, st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(copy_st, ev, 0);
    }
    for (int64_t z0 = 0; z0 < N && e == cudaSuccess; z0 += zc) {
      const int64_t nz = (N - z0) < zc ? (N - z0) : zc;
      e = cudaMemcpyAsync(static_cast<unsigned char*>(const_cast<void*>(volume)) + z0 * slice,
                          static_cast<const unsigned char*>(host_src) + z0 * slice, nz * slice,
                          cudaMemcpyHostToDevice, copy_st);
      if (e == cudaSuccess) e = cudaEventRecord(ev, copy_st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
      if (e != cudaSuccess) return cuda_fail(e, "copy volume chunk to device");
      k1_launches += w.set.P > 9 ? 2 : 1;  // images 9, 10 in a second kernel
      if (lanes) {
        ia.z0 = z0;
        ia.nz = nz;
        e = launch_project_int(ia, st);
      } else {
        a.z0 = z0;
        a.nz = nz;
        e = launch_project(a, st);
      }
      if (e != cudaSuccess) return cuda_fail(e, "projection kernel");
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy volume to device");
  } else {
    if (lanes) {
      e = launch_project_int(ia, st);
    } else {
      e = launch_project(a, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "projection kernel");
    k1_launches = w.set.P > 9 ? 2 : 1;
  }
  rec.mark(1, k1_launches);
  if (lanes && fl) {
    e = launch_image_moments_limbs(images, w.set, w.set.total_elems, K, 2, ws + w.off_part,
                                   ws + w.off_m2d, st, true);
    if (e != cudaSuccess) return cuda_fail(e, "image moment kernel");
    rec.mark(2, 1);
    e = launch_combine_fixed(ws + w.off_m2d, K, w.set.P, static_cast<double*>(out), status, flags,
                             scale, L, M, N, kFloatTolerance, st);
    if (e != cudaSuccess) return cuda_fail(e, "combine kernel");
    // the combine and the gated fallback (five launches, or one graph
    // launch of a one-thread gate and a conditional body) count as the last
    // stage
    int fb_launches = 0;
    const dpma_status fs = enqueue_fallback(volume, L, M, N, K, out, st, ws, w, &fb_launches);
    rec.mark(3, 1 + fb_launches);
    return fs;
  }
  // on the integer-lane path the clear above zeroed the 2-D moments, so the
  // image moment kernel accumulates them itself (no reduction launch)
  e = launch_image_moments(images, w.set, K, fl, ws + w.off_part, ws + w.off_m2d, st, nullptr,
                           lanes && !fl);
  if (e != cudaSuccess) return cuda_fail(e, "image moment kernel");
  rec.mark(2, lanes && !fl ? 1 : 2);
  e = launch_combine(ws + w.off_m2d, K, fl, out, status, st);
  if (e != cudaSuccess) return cuda_fail(e, "combine kernel");
  rec.mark(3, 1);
  return DPMA_OK;
}

// The whole device-resident pipeline as one cached graph launch.  Small
// volumes spend most of a call in the gaps between five to eleven dependent
// launches; a caller that repeats the call with the same buffers (a loop over
// frames, a benchmark) gets the captured sequence replayed by one graph
// launch instead.  Keyed by every pointer and size the kernels bake in and by
// the wait budget; a key becomes a graph on its second use, never while
// stage timing is on (its events belong to each call) or while the caller's
// stream is itself being captured.
struct PipeKey {
  int dev;
  const void* vol;
  int64_t L, M, N;
  int dtype, K;
  void* out;
  unsigned char* ws;
  long long budget;
  bool operator==(const PipeKey& o) const {
    return dev == o.dev && vol == o.vol && L == o.L && M == o.M && N == o.N && dtype == o.dtype &&
           K == o.K && out == o.out && ws == o.ws && budget == o.budget;
  }
};
struct PipeGraph {
  PipeKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};
constexpr size_t kPipeGraphs = 8;
constexpr size_t kPipeSeen = 16;
std::mutex g_pipe_mu;
std::vector<PipeGraph> g_pipe_graphs;  // most recently used last
std::vector<PipeKey> g_pipe_seen;

dpma_status enqueue_device(const void* volume, int64_t L, int64_t M, int64_t N, dpma_dtype dtype,
                           int K, void* out, cudaStream_t st, unsigned char* ws, const Layout& w) {
  bool timing;
  {
    std::lock_guard<std::mutex> lk(g_timing_mu);
    timing = g_timing;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturing = cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
                         cs != cudaStreamCaptureStatusNone;
  const NvtxRange range("dpma: pipeline call");
  PipeKey k{};
  if (timing || capturing || cudaGetDevice(&k.dev) != cudaSuccess)
    return enqueue(volume, L, M, N, dtype, K, out, st, ws, w);
  k.vol = volume; k.L = L; k.M = M; k.N = N; k.dtype = (int)dtype; k.K = K;
  k.out = out; k.ws = ws; k.budget = g_wait_budget.load();
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    for (size_t i = 0; i < g_pipe_graphs.size(); ++i)
      if (g_pipe_graphs[i].key == k) {
        const PipeGraph pg = g_pipe_graphs[i];
        g_pipe_graphs.erase(g_pipe_graphs.begin() + i);
        g_pipe_graphs.push_back(pg);
        exec = pg.exec;
        break;
      }
    if (!exec) {
      bool seen = false;
      for (const PipeKey& o : g_pipe_seen) seen = seen || (o == k);
      if (!seen) {
        if (g_pipe_seen.size() >= kPipeSeen) g_pipe_seen.erase(g_pipe_seen.begin());
        g_pipe_seen.push_back(k);
      } else {
        // host-side preparations that must not happen during the capture
        cudaError_t e = prepare_combine(K);
        cudaStream_t cap = nullptr;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        PipeGraph pg;
        pg.key = k;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const dpma_status ps = enqueue(volume, L, M, N, dtype, K, out, cap, ws, w);
          cudaGraph_t g = nullptr;
          e = cudaStreamEndCapture(cap, &g);
          if (ps != DPMA_OK && e == cudaSuccess) e = cudaErrorUnknown;
          if (e == cudaSuccess) e = cudaGraphInstantiate(&pg.exec, g, 0);
          if (e == cudaSuccess) pg.graph = g;
          else if (g) cudaGraphDestroy(g);
        }
        if (cap) cudaStreamDestroy(cap);
        if (e == cudaSuccess) {
          if (g_pipe_graphs.size() >= kPipeGraphs) {
            cudaGraphExecDestroy(g_pipe_graphs.front().exec);
            cudaGraphDestroy(g_pipe_graphs.front().graph);
            g_pipe_graphs.erase(g_pipe_graphs.begin());
          }
          g_pipe_graphs.push_back(pg);
          exec = pg.exec;
        } else {
          cudaGetLastError();  // a failed capture leaves the plain launches in use
        }
      }
    }
  }
  if (!exec) return enqueue(volume, L, M, N, dtype, K, out, st, ws, w);
  const cudaError_t e = cudaGraphLaunch(exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline graph launch");
  return DPMA_OK;
}

}  // namespace

namespace dpma {
// Records `msg` as the calling thread's last error (used by entry points
// defined in other translation units).
void set_last_error(const char* msg) { t_last_error = msg; }
}  // namespace dpma

extern "C" {

int dpma_num_moments(int K) { return (K < 0 || K > DPMA_MAX_K) ? 0 : num_moments(K); }

int dpma_num_images(int K) { return (K < 0 || K > DPMA_MAX_K) ? 0 : num_images(K); }

int dpma_moment_index(int p, int q, int r) {
  if (p < 0 || q < 0 || r < 0 || p + q + r > DPMA_MAX_K) return -1;
  return idx3d(p, q, r);
}

const char* dpma_status_string(dpma_status s) {
  switch (s) {
    case DPMA_OK: return "ok";
    case DPMA_ERR_INVALID_ARG: return "invalid argument";
    case DPMA_ERR_OVERFLOW: return "exact range exceeded";
    case DPMA_ERR_OOM: return "out of device memory";
    case DPMA_ERR_CUDA: return "CUDA error";
    case DPMA_ERR_TIMEOUT: return "device wait timed out";
    case DPMA_ERR_REJECTED: return "request rejected";
    case DPMA_ERR_INTERNAL: return "internal self-check failed";
  }
  return "unknown status";
}

const char* dpma_last_error(void) { return t_last_error.c_str(); }

int dpma_last_float_path(void) { return t_last_flags; }

dpma_status dpma_set_wait_budget(int64_t cycles) {
  if (cycles < 0) return fail(DPMA_ERR_INVALID_ARG, "negative wait budget");
  g_wait_budget.store(cycles == 0 ? (1ll << 31) : cycles);
  return DPMA_OK;
}

dpma_status dpma_image_geometry(int k, int64_t L, int64_t M, int64_t N, int64_t* S, int64_t* F,
                                int64_t* off_s, int64_t* off_f) {
  if (k < 0 || k >= kMaxImages || L < 1 || M < 1 || N < 1)
    return fail(DPMA_ERR_INVALID_ARG, "bad image index or dimensions");
  ImageGeom g;
  image_geom(k, L, M, N, &g);
  if (S) *S = g.S;
  if (F) *F = g.F;
  if (off_s) *off_s = g.off_s;
  if (off_f) *off_f = g.off_f;
  return DPMA_OK;
}

size_t dpma_images_size(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K) {
  if (check_args(L, M, N, dtype, K) == DPMA_ERR_INVALID_ARG) return 0;
  return layout(L, M, N, dtype, K).img_bytes;
}

size_t dpma_workspace_size(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K) {
  if (check_args(L, M, N, dtype, K) == DPMA_ERR_INVALID_ARG) return 0;
  return layout(L, M, N, dtype, K).total;
}

dpma_status dpma_combine_plan(int K, int n, int* nmono, int64_t* D, int32_t* img, int32_t* a,
                              int64_t* C) {
  if (K < 0 || K > DPMA_MAX_K || n < 0 || n > K)
    return fail(DPMA_ERR_INVALID_ARG, "need 0 <= n <= K <= 10");
  const CombinePlan* cp = combine_plan(K);
  if (!cp) return fail(DPMA_ERR_INTERNAL, "combine plan failed its exact check");
  const DegreePlan& d = cp->deg[n];
  if (nmono) *nmono = d.nmono;
  if (D) *D = d.D;
  for (int j = 0; j < d.nmono; ++j) {
    if (img) img[j] = d.img[j];
    if (a) a[j] = d.a[j];
  }
  if (C) std::memcpy(C, d.C, sizeof(int64_t) * d.nmono * d.nmono);
  return DPMA_OK;
}

dpma_status dpma_moments_async(const void* volume, int64_t L, int64_t M, int64_t N,
                               dpma_dtype dtype, int K, void* out, void* stream, void* workspace,
                               size_t workspace_bytes) {
  if (!volume || !out) return fail(DPMA_ERR_INVALID_ARG, "null volume or output pointer");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK) return s;
  const Layout w = layout(L, M, N, dtype, K);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (workspace) {
    if (workspace_bytes < w.total) return fail(DPMA_ERR_INVALID_ARG, "workspace too small");
    return enqueue_device(volume, L, M, N, dtype, K, out, st,
                          static_cast<unsigned char*>(workspace), w);
  }
  DeviceState* ds = state_for_current_device(nullptr);
  if (!ds) return fail(DPMA_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(ds->mu);
  cudaError_t e = ensure_buffer(&ds->ws, &ds->ws_bytes, w.total);
  if (e != cudaSuccess) return cuda_fail(e, "workspace");
  return enqueue_device(volume, L, M, N, dtype, K, out, st, static_cast<unsigned char*>(ds->ws), w);
}

dpma_status dpma_moments(const void* volume, int64_t L, int64_t M, int64_t N, dpma_dtype dtype,
                         int K, void* out) {
  if (!volume || !out) return fail(DPMA_ERR_INVALID_ARG, "null volume or output pointer");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK) return s;
  DeviceState* ds = state_for_current_device(nullptr);
  if (!ds) return fail(DPMA_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(ds->mu);
  cudaError_t e = ensure_stream(ds);
  if (e != cudaSuccess) return cuda_fail(e, "stream");
  const Layout w = layout(L, M, N, dtype, K);
  e = ensure_buffer(&ds->ws, &ds->ws_bytes, w.total);
  if (e != cudaSuccess) return cuda_fail(e, "workspace");
  unsigned char* ws = static_cast<unsigned char*>(ds->ws);
  e = ensure_host_status(ds);
  if (e != cudaSuccess) return cuda_fail(e, "pinned status word");
  s = enqueue_device(volume, L, M, N, dtype, K, out, ds->stream, ws, w);
  if (s != DPMA_OK) return s;
  e = cudaMemcpyAsync(ds->h_status, ws + w.off_status, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                      ds->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ds->stream);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  t_last_flags = ds->h_status[1];
  const int status = *ds->h_status;
  if (status == DPMA_ERR_TIMEOUT) return fail(DPMA_ERR_TIMEOUT, "a bounded device wait gave up");
  if (status) return fail(DPMA_ERR_INTERNAL, "combine division left a remainder");
  return DPMA_OK;
}

dpma_status dpma_moments_host(const void* host_volume, int64_t L, int64_t M, int64_t N,
                              dpma_dtype dtype, int K, void* host_out) {
  if (!host_volume || !host_out) return fail(DPMA_ERR_INVALID_ARG, "null host pointer");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK) return s;
  DeviceState* ds = state_for_current_device(nullptr);
  if (!ds) return fail(DPMA_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(ds->mu);
  cudaError_t e = ensure_stream(ds);
  if (e != cudaSuccess) return cuda_fail(e, "stream");
  const Layout w = layout(L, M, N, dtype, K);
  const size_t vbytes = (size_t)L * M * N * elem_size(dtype);
  const size_t obytes = (size_t)num_moments(DPMA_MAX_K) * 16;
  // one allocation: [volume | moments] so the workspace can stay separate
  size_t need = align_up(vbytes, 256) + obytes;
  e = ensure_buffer(&ds->host_vol, &ds->host_vol_bytes, need);
  if (e != cudaSuccess) return cuda_fail(e, "staging buffer");
  ds->host_out = static_cast<unsigned char*>(ds->host_vol) + align_up(vbytes, 256);
  e = ensure_buffer(&ds->ws, &ds->ws_bytes, w.total);
  if (e != cudaSuccess) return cuda_fail(e, "workspace");
  if (!ds->copy_stream) {
    e = cudaStreamCreateWithFlags(&ds->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "copy stream");
  }
  if (!ds->chunk_ready) {
    e = cudaEventCreateWithFlags(&ds->chunk_ready, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "chunk event");
  }
  unsigned char* ws = static_cast<unsigned char*>(ds->ws);
  s = enqueue(ds->host_vol, L, M, N, dtype, K, ds->host_out, ds->stream, ws, w, host_volume,
              ds->copy_stream, ds->chunk_ready);
  if (s != DPMA_OK) return s;
  const size_t out_bytes = (size_t)num_moments(K) * (is_float(dtype) ? 8 : 16);
  e = ensure_host_status(ds);
  if (e != cudaSuccess) return cuda_fail(e, "pinned status word");
  e = cudaMemcpyAsync(host_out, ds->host_out, out_bytes, cudaMemcpyDeviceToHost, ds->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ds->h_status, ws + w.off_status, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                        ds->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ds->stream);
  if (e != cudaSuccess) return cuda_fail(e, "copy moments to host");
  t_last_flags = ds->h_status[1];
  const int status = *ds->h_status;
  if (status == DPMA_ERR_TIMEOUT) return fail(DPMA_ERR_TIMEOUT, "a bounded device wait gave up");
  if (status) return fail(DPMA_ERR_INTERNAL, "combine division left a remainder");
  return DPMA_OK;
}

dpma_status dpma_project(const void* volume, int64_t L, int64_t M, int64_t N, dpma_dtype dtype,
                         int K, void* images, void* stream) {
  if (!volume || !images) return fail(DPMA_ERR_INVALID_ARG, "null volume or image pointer");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK && s != DPMA_ERR_OVERFLOW) return s;  // images alone are always exact
  const Layout w = layout(L, M, N, dtype, K);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(images, 0, w.img_bytes, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear images");
  if (!is_float(dtype) && project_int_supported(volume, L, (int)dtype, w.set.P)) {
    // integer volumes: the integer-lane kernel of the fused pipeline
    IntProjectArgs ia{};
    ia.vol = volume;
    ia.L = L; ia.M = M; ia.N = N;
    ia.dtype = (int)dtype;
    ia.images = images;
    ia.set = w.set;
    ia.wait_budget = g_wait_budget.load();
    e = launch_project_int(ia, st);
    if (e != cudaSuccess) return cuda_fail(e, "projection kernel");
    return DPMA_OK;
  }
  ProjectArgs a{};
  a.vol = volume;
  a.L = L; a.M = M; a.N = N;
  a.dtype = (int)dtype;
  a.K = K;
  a.images = images;
  a.set = w.set;
  e = launch_project(a, st);
  if (e != cudaSuccess) return cuda_fail(e, "projection kernel");
  return DPMA_OK;
}

dpma_status dpma_image_moments(const void* images, int64_t L, int64_t M, int64_t N,
                               dpma_dtype dtype, int K, void* moments2d, void* stream,
                               void* workspace, size_t workspace_bytes) {
  if (!images || !moments2d) return fail(DPMA_ERR_INVALID_ARG, "null image or output pointer");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK) return s;
  const Layout w = layout(L, M, N, dtype, K);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* part = nullptr;
  if (workspace) {
    if (workspace_bytes < w.total) return fail(DPMA_ERR_INVALID_ARG, "workspace too small");
    part = static_cast<unsigned char*>(workspace) + w.off_part;
    cudaError_t e = launch_image_moments(images, w.set, K, is_float(dtype), part, moments2d, st);
    if (e != cudaSuccess) return cuda_fail(e, "image moment kernel");
    return DPMA_OK;
  }
  DeviceState* ds = state_for_current_device(nullptr);
  if (!ds) return fail(DPMA_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(ds->mu);
  cudaError_t e = ensure_buffer(&ds->ws, &ds->ws_bytes, w.total);
  if (e != cudaSuccess) return cuda_fail(e, "workspace");
  part = static_cast<unsigned char*>(ds->ws) + w.off_part;
  e = launch_image_moments(images, w.set, K, is_float(dtype), part, moments2d, st);
  if (e != cudaSuccess) return cuda_fail(e, "image moment kernel");
  return DPMA_OK;
}

size_t dpma_drt_workspace_size(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K) {
  if (check_args(L, M, N, dtype, K) != DPMA_OK || is_float(dtype)) return 0;
  return drt_workspace_bytes(L, M, N, K);
}

dpma_status dpma_image_moments_drt(const void* images, int64_t L, int64_t M, int64_t N,
                                   dpma_dtype dtype, int K, void* moments2d, void* stream,
                                   void* workspace, size_t workspace_bytes, int* status) {
  if (!images || !moments2d) return fail(DPMA_ERR_INVALID_ARG, "null image or output pointer");
  if (is_float(dtype))
    return fail(DPMA_ERR_INVALID_ARG, "the discrete Radon step takes integer images only");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK) return s;
  const size_t need = drt_workspace_bytes(L, M, N, K);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (workspace) {
    if (workspace_bytes < need) return fail(DPMA_ERR_INVALID_ARG, "workspace too small");
    cudaError_t e = launch_image_moments_drt(images, L, M, N, K, workspace, moments2d, status, st);
    if (e != cudaSuccess) return cuda_fail(e, "discrete Radon moment kernels");
    return DPMA_OK;
  }
  DeviceState* ds = state_for_current_device(nullptr);
  if (!ds) return fail(DPMA_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(ds->mu);
  cudaError_t e = ensure_buffer(&ds->drt_ws, &ds->drt_ws_bytes, need);
  if (e != cudaSuccess) return cuda_fail(e, "discrete Radon workspace");
  e = launch_image_moments_drt(images, L, M, N, K, ds->drt_ws, moments2d, status, st);
  if (e != cudaSuccess) return cuda_fail(e, "discrete Radon moment kernels");
  return DPMA_OK;
}

dpma_status dpma_drt_plan(int n, int* alpha, int* beta, int64_t* E, int64_t* D) {
  if (n < 0 || n > DPMA_MAX_K) return fail(DPMA_ERR_INVALID_ARG, "degree out of range");
  for (int j = 0; j <= n; ++j) {
    int a = 0, b = 0;
    drt_direction(j, &a, &b);
    if (alpha) alpha[j] = a;
    if (beta) beta[j] = b;
  }
  if (!drt_plan_degree(n, E, D)) return fail(DPMA_ERR_INTERNAL, "discrete Radon solve unavailable");
  return DPMA_OK;
}

dpma_status dpma_combine(const void* moments2d, dpma_dtype dtype, int K, void* out, void* stream,
                         int* status) {
  if (!moments2d || !out) return fail(DPMA_ERR_INVALID_ARG, "null pointer");
  if (dtype != DPMA_U8 && dtype != DPMA_U16 && dtype != DPMA_F32)
    return fail(DPMA_ERR_INVALID_ARG, "unknown dtype");
  if (K < 0 || K > (dtype == DPMA_F32 ? DPMA_MAX_K_FLOAT : DPMA_MAX_K))
    return fail(DPMA_ERR_INVALID_ARG, "K must lie in 0..10 (0..8 for float32)");
  cudaError_t e = prepare_combine(K);
  if (e != cudaSuccess) return cuda_fail(e, "combine plan");
  e = launch_combine(moments2d, K, is_float(dtype), out, status, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "combine kernel");
  return DPMA_OK;
}

dpma_status dpma_moments_from_projections(const void* images, int64_t L, int64_t M, int64_t N,
                                          dpma_dtype dtype, int K, void* out, void* stream) {
  if (!images || !out) return fail(DPMA_ERR_INVALID_ARG, "null image or output pointer");
  dpma_status s = check_args(L, M, N, dtype, K);
  if (s != DPMA_OK) return s;
  cudaError_t e = prepare_combine(K);
  if (e != cudaSuccess) return cuda_fail(e, "combine plan");
  DeviceState* ds = state_for_current_device(nullptr);
  if (!ds) return fail(DPMA_ERR_CUDA, "no current CUDA device");
  std::lock_guard<std::mutex> lk(ds->mu);
  const Layout w = layout(L, M, N, dtype, K);
  e = ensure_buffer(&ds->ws, &ds->ws_bytes, w.total);
  if (e != cudaSuccess) return cuda_fail(e, "workspace");
  unsigned char* ws = static_cast<unsigned char*>(ds->ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* status = reinterpret_cast<int*>(ws + w.off_status);
  e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "clear status");
  const bool fl = is_float(dtype);
  e = launch_image_moments(images, w.set, K, fl, ws + w.off_part, ws + w.off_m2d, st);
  if (e != cudaSuccess) return cuda_fail(e, "image moment kernel");
  e = launch_combine(ws + w.off_m2d, K, fl, out, status, st);
  if (e != cudaSuccess) return cuda_fail(e, "combine kernel");
  int h = 0;
  e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "synchronize");
  if (h) return fail(DPMA_ERR_INTERNAL,
                     "the projections are not those of any integer volume (a combine division "
                     "left a remainder)");
  return DPMA_OK;
}

dpma_status dpma_stage_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timing = enable != 0;
  return DPMA_OK;
}

dpma_status dpma_stage_times(double* ms, int64_t* launches, int reset) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (const StageEvent& se : g_pending) {
    cudaError_t e = cudaEventSynchronize(se.b);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, se.a, se.b);
    if (e != cudaSuccess) {
      g_pending.clear();
      return cuda_fail(e, "stage timing events");
    }
    g_stage_ms[se.stage] += t;
    g_stage_launches[se.stage] += se.kernels;
    if (se.free_a) g_free_events.push_back(se.a);
    g_free_events.push_back(se.b);
  }
  g_pending.clear();
  for (int i = 0; i < 4; ++i) {
    if (ms) ms[i] = g_stage_ms[i];
    if (launches) launches[i] = g_stage_launches[i];
    if (reset) { g_stage_ms[i] = 0; g_stage_launches[i] = 0; }
  }
  return DPMA_OK;
}

}  // extern "C"
