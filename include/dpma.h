/*
 * dpma.h -- C ABI of the GB300 (sm_103a) Discrete Projection Moment library.
 *
 * The library computes every raw 3-D moment
 *
 *     M_pqr = sum_{x<L, y<M, z<N} V(x,y,z) x^p y^q z^r ,   p+q+r <= K        (Eq. 2)
 *
 * of a volume by the Discrete Projection Moment method of Diggin & Diggin,
 * "Fast 3D Image Moments" (2020), Sec. 3:
 *   1. project the volume into P = max(3, K+1) discrete line-sum images in one
 *      pass over the voxels, with additions only (Sec. 3.1, Eqs. 4-9);
 *   2. take the 2-D moments of every image (Sec. 1, Eq. 1; Sec. 3.2);
 *   3. combine them linearly into the 3-D moments (Eqs. 10-16, generalised to
 *      any K <= 10 by an exact integer combine matrix per degree).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * Volume layout: V[(z*M + y)*L + x], x contiguous, 0-based coordinates with
 *   the origin at voxel (0,0,0) and 0^0 = 1 (Eq. 2).
 * Element types: DPMA_U8 (uint8), DPMA_U16 (uint16), DPMA_F32 (float32).
 * Moment order ("graded"): degree n = p+q+r ascending, then p descending,
 *   then q descending: 000,100,010,001,200,110,101,020,011,002,...
 *   dpma_num_moments(K) = (K+1)(K+2)(K+3)/6 values (20, 35, 84, 165 for
 *   K = 3, 4, 6, 8).
 * Moment types: integer volumes give exact signed 128-bit integers stored
 *   little-endian in 16 bytes (low 64 bits first); float32 volumes give
 *   IEEE doubles.
 * Images: image k holds the sums of V along one lattice direction and is a
 *   row-major [S_k][F_k] array; a voxel lands on row
 *   s = slow_k(x,y,z) + off_s and column f = fast_k(x,y,z) + off_f:
 *
 *     k  sums along  slow        fast          S_k      F_k      paper
 *     0  z           y           x             M        L        Eq. 5
 *     1  x           z           y             N        M        Eq. 6
 *     2  y           z           x             N        L        Eq. 7
 *     3  (1,0,-1)    y           x+z           M        L+N-1    Eq. 8
 *     4  (1,0,1)     y           x-z+(N-1)     M        L+N-1    Eq. 9
 *     5  (0,1,-1)    y+z         x             M+N-1    L        +-pi/4 about x
 *     6  (0,1,1)     y-z+(N-1)   x             M+N-1    L        (Sec. 3.1)
 *     7  (1,-1,0)    z           x+y           N        L+M-1    +-pi/4 about z
 *     8  (1,1,0)     z           x-y+(M-1)     N        L+M-1    (Sec. 3.1)
 *     9  (2,0,-1)    y           x+2z          M        L+2N-2   arctan(1/2) about y
 *    10  (1,-1,-1)   x+z         2y+x-z+(N-1)  L+N-1    L+2M+N-3 isometric (Sec. 3.1)
 *
 *   Order K uses images 0..max(2, K); images 9 and 10 (orders 9 and 10)
 *   are taken for integer volumes only.
 *
 *   Integer volumes: uint32 pixels (exact: dimensions are capped at 65536,
 *   so a line sum of uint16 voxels stays below 2^32).  Float32 volumes:
 *   IEEE double pixels holding the compensated float32 line sum (float-float
 *   accuracy, about 2^-46 relative to the sum of |V| along the line).
 * 2-D moments: T_ab = sum I[s][f] (s-off_s)^a (f-off_f)^b for a+b <= K (signed
 *   coordinates, the origin shift of Sec. 5), ordered degree ascending then
 *   a descending; (K+1)(K+2)/2 values per image, int128 for integer volumes,
 *   (hi, lo) float32 pairs for float volumes.
 * Pointers: "device" pointers must come from cudaMalloc (or be otherwise
 *   addressable by the current CUDA device); "host" pointers are ordinary
 *   process memory (pinned memory makes the copies asynchronous and faster).
 *   The library keeps no pointer after a call returns, except where stated.
 * Streams: arguments named `stream` are cudaStream_t values passed as void*;
 *   NULL means the legacy default stream.
 * Errors: every call returns a dpma_status; nothing is thrown across the
 *   ABI.  dpma_last_error() returns a thread-local message for the last
 *   failing call of the calling thread.
 * Devices: calls run on the CUDA device current in the calling thread.
 */
#ifndef DPMA_H
#define DPMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dpma_status {
  DPMA_OK = 0,
  DPMA_ERR_INVALID_ARG = 1, /* null pointer, dimension < 1 or > 65536, K out of range, bad dtype */
  DPMA_ERR_OVERFLOW = 2,    /* an exact intermediate could exceed the int128 range */
  DPMA_ERR_OOM = 3,         /* device memory allocation failed */
  DPMA_ERR_CUDA = 4,        /* a CUDA runtime call failed; see dpma_last_error() */
  DPMA_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  DPMA_ERR_REJECTED = 6,    /* the request was refused (capacity) */
  DPMA_ERR_INTERNAL = 7     /* a self-check failed (e.g. a combine division left a remainder) */
} dpma_status;

typedef enum dpma_dtype { DPMA_U8 = 0, DPMA_U16 = 1, DPMA_F32 = 2 } dpma_dtype;

/* Largest order K: 10 for uint8/uint16 volumes through the single-volume
 * entry points (dpma_moments, _async, _host, dpma_project,
 * dpma_image_moments, dpma_combine, dpma_moments_from_projections,
 * dpma_derived_moments); 8 for float32 volumes and for the batched
 * launches, the server and dpma_moments_noalloc. */
#define DPMA_MAX_K 10
#define DPMA_MAX_K_FLOAT 8
#define DPMA_MAX_K_BATCH 8
#define DPMA_MAX_DIM 65536

/* ---------------- helpers (host only, no GPU needed) ---------------- */

/* Number of moments with p+q+r <= K, i.e. C(K+3,3); 0 if K is out of range. */
int dpma_num_moments(int K);
/* Number of projection images the method uses for order K: max(3, K+1). */
int dpma_num_images(int K);
/* Position of M_pqr in graded order; -1 if p, q or r is negative or p+q+r > DPMA_MAX_K. */
int dpma_moment_index(int p, int q, int r);
/* Static text for a status code. */
const char* dpma_status_string(dpma_status s);
/* Thread-local message describing the calling thread's last failure ("" if none). */
const char* dpma_last_error(void);
/*
 * Which float32 pipeline produced the calling thread's last synchronous
 * float32 result (dpma_moments, dpma_moments_host): 0 the quantised
 * integer-lane pipeline; otherwise the compensated float pipeline recomputed
 * it because bit 0: a voxel lay beyond the sampled quantisation grid or was
 * not finite, bit 1: a moment's guaranteed error bound exceeded the
 * tolerance.  Integer volumes leave it 0.
 */
int dpma_last_float_path(void);
/*
 * Fault-injection hook for tests of the bounded device waits: the number of
 * clock cycles a wait of the projection kernel spins before it gives up and
 * the call reports DPMA_ERR_TIMEOUT (0 restores the default, about 2^31).
 * Copies already issued still land before a CTA leaves.  Process-wide.
 */
dpma_status dpma_set_wait_budget(int64_t cycles);
/* Geometry of image k (0..10) of an L x M x N volume (table above). */
dpma_status dpma_image_geometry(int k, int64_t L, int64_t M, int64_t N, int64_t* S, int64_t* F,
                                int64_t* off_s, int64_t* off_f);
/* Bytes of the image buffer dpma_project writes (all P images, layout above). */
size_t dpma_images_size(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K);
/* Bytes of device workspace dpma_moments_async needs (images + partial sums + status). */
size_t dpma_workspace_size(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K);
/*
 * The exact combine of degree n for order K (Sec. 3.2 generalised):
 *   M_n = (1/D) * C * t,   t[j] = T_{a[j], n-a[j]} of image img[j],
 * M_n being the degree-n moments in graded order.  C is nmono x nmono
 * row-major (nmono = (n+1)(n+2)/2; capacity of C: 45*45, of img and a: 45).
 * Any output pointer may be NULL.  Returns DPMA_ERR_INVALID_ARG unless
 * 0 <= n <= K <= 8.
 */
dpma_status dpma_combine_plan(int K, int n, int* nmono, int64_t* D, int32_t* img, int32_t* a,
                              int64_t* C);

/* ---------------- the hot path ---------------- */

/*
 * All moments of a device-resident volume; synchronous.  `volume` and `out`
 * are device pointers (out: dpma_num_moments(K) entries of 16 bytes for
 * integer volumes, 8 bytes for float volumes).  Runs on a library-owned
 * stream with a library-owned workspace and returns after the result is in
 * `out`.  The library's stream is a blocking stream, so work queued on the
 * legacy default stream (e.g. the copy that filled `volume`) completes
 * first.  Errors: INVALID_ARG, OVERFLOW (only for integer volumes whose
 * bound exceeds int128), OOM, CUDA, INTERNAL.
 */
dpma_status dpma_moments(const void* volume, int64_t L, int64_t M, int64_t N, dpma_dtype dtype,
                         int K, void* out);

/*
 * Same, enqueued on `stream`; returns once enqueued.  `workspace` is a
 * device buffer of at least dpma_workspace_size(...) bytes owned by the
 * caller (it must stay untouched until the stream has finished the call);
 * if it is NULL the library uses its own buffer and the call serialises
 * with other NULL-workspace calls on the same device.  A combine self-check
 * failure is reported by the next synchronous call, not by this one.
 */
dpma_status dpma_moments_async(const void* volume, int64_t L, int64_t M, int64_t N,
                               dpma_dtype dtype, int K, void* out, void* stream, void* workspace,
                               size_t workspace_bytes);

/*
 * End to end from host memory: copies the volume host->device, computes,
 * copies the moments device->host, and returns when `host_out` holds them.
 * `host_volume` and `host_out` are host pointers; device buffers are owned
 * and reused by the library.  The volume is copied in z-chunks (about 4 MB,
 * at most 16) on a separate stream, and the projection of each chunk runs
 * while the next one is copied; pinned host memory gives the full link rate.
 * Float results may differ from the device-resident call in the last bits
 * (partial sums merge in another order), within the library's tolerance.
 */
dpma_status dpma_moments_host(const void* host_volume, int64_t L, int64_t M, int64_t N,
                              dpma_dtype dtype, int K, void* host_out);

/*
 * Step 1 alone (Sec. 3.1, Eqs. 4-9): writes the P = dpma_num_images(K)
 * images of the device volume into the device buffer `images`
 * (dpma_images_size bytes; zeroed by the call), enqueued on `stream`.
 */
dpma_status dpma_project(const void* volume, int64_t L, int64_t M, int64_t N, dpma_dtype dtype,
                         int K, void* images, void* stream);

/*
 * Step 2 alone (Eq. 1 with signed coordinates): the 2-D moments of images
 * laid out as dpma_project writes them, into the device buffer `moments2d`
 * (P * (K+1)(K+2)/2 values; int128 or float32 pairs), enqueued on `stream`.
 * `workspace` as for dpma_moments_async.
 */
dpma_status dpma_image_moments(const void* images, int64_t L, int64_t M, int64_t N,
                               dpma_dtype dtype, int K, void* moments2d, void* stream,
                               void* workspace, size_t workspace_bytes);

/*
 * Step 2 by the discrete Radon route (Sec. 3.2 and its DRT integral
 * listing): every image is summed once more onto 1-D integrals along n+1
 * lattice directions t = alpha f' + beta s' (the paper's five: (1,0), (0,1),
 * (1,1), (1,-1), (1,2); then (2,1), (1,-2), (2,-1), (1,3), (3,1), (1,-3) for
 * orders 5..10), their 1-D moments are taken, and the degree-n 2-D moments
 * follow by an exact rational solve (dpma_drt_plan).  Integer volumes only
 * (uint32 images as dpma_project writes them); the output `moments2d`
 * (device, P * (K+1)(K+2)/2 int128) is bit-identical to dpma_image_moments.
 * `workspace` (device, dpma_drt_workspace_size bytes) may be NULL: the
 * library then uses its own buffer.  `status` (device int, may be NULL) is
 * set to 7 if a division of the solve leaves a remainder (images that are
 * not line sums of any integer volume cannot cause this; a corrupted buffer
 * can).  Enqueued on `stream`.  DPMA_ERR_INVALID_ARG for float32.
 */
dpma_status dpma_image_moments_drt(const void* images, int64_t L, int64_t M, int64_t N,
                                   dpma_dtype dtype, int K, void* moments2d, void* stream,
                                   void* workspace, size_t workspace_bytes, int* status);
/* Bytes of device workspace dpma_image_moments_drt needs (0 for float32 or bad arguments). */
size_t dpma_drt_workspace_size(int64_t L, int64_t M, int64_t N, dpma_dtype dtype, int K);
/*
 * Host only: the directions (alpha[j], beta[j]), j = 0..n, and the exact
 * solve of degree n of the discrete Radon step:
 *   T_{n-b,b} = (sum_j E[b*(n+1) + j] * mu_j) / D[b],   mu_j = sum_t t^n P_j(t).
 * Any pointer may be NULL.  0 <= n <= DPMA_MAX_K.
 */
dpma_status dpma_drt_plan(int n, int* alpha, int* beta, int64_t* E, int64_t* D);

/*
 * Step 3 alone (Eqs. 10-16 generalised): 3-D moments from the 2-D moments
 * of dpma_image_moments (device buffers), enqueued on `stream`.  Integer
 * combines are exact (256-bit accumulation, exact division); a division
 * that leaves a remainder sets DPMA_ERR_INTERNAL in `status` (a device int,
 * may be NULL).
 */
dpma_status dpma_combine(const void* moments2d, dpma_dtype dtype, int K, void* out, void* stream,
                         int* status);

/*
 * 3-D moments from given projection images (the tomographic use of the
 * method, Sec. 3.2: a few chosen projections stand in for a reconstructed
 * volume).  `images` (device) holds the first max(3, K+1) images of the
 * table above for an L x M x N volume, back to back in that order and
 * layout: uint32 pixels for DPMA_U8 / DPMA_U16 (any integer line sums),
 * IEEE doubles for DPMA_F32.  `dtype` only selects the pixel type and the
 * magnitude bound (the largest voxel value 255 / 65535 bounds the int128
 * range check).  Runs steps 2 and 3 on `stream` with the library's own
 * workspace and waits for them.  DPMA_ERR_INTERNAL: an exact integer
 * division left a remainder, i.e. the integer images are not the
 * projections of any integer volume.
 */
dpma_status dpma_moments_from_projections(const void* images, int64_t L, int64_t M, int64_t N,
                                          dpma_dtype dtype, int K, void* out, void* stream);

/*
 * Features derived from the moments (the post-step of Sec. 4), on the
 * device: `moments` holds dpma_num_moments(K) raw moments as the other entry
 * points return them (int128 for DPMA_U8 / DPMA_U16, double for DPMA_F32).
 * `out` (device) receives 3 + 3 * dpma_num_moments(K) doubles:
 *   out[0..2]              centroid (M100, M010, M001) / M000 in voxel units;
 *   out[3 .. 3+nm)         central moments mu_pqr (graded order);
 *   out[3+nm .. 3+2nm)     eta_pqr = mu_pqr / mu_000^((p+q+r)/3 + 1)  (Eq. 17);
 *   out[3+2nm .. 3+3nm)    mu'_pqr = a^(1+p) b^(1+q) c^(1+r) mu_pqr for the
 *                          voxel spacings spacing = {a, b, c} (host array;
 *                          NULL: unit spacing).
 * The binomial expansion about the centroid runs in double-double arithmetic
 * from the exact moments; only the results are rounded.  M000 = 0 gives NaN
 * everywhere; K = 0 gives a NaN centroid (no first-degree moments).  Enqueued on `stream`.  Errors: DPMA_ERR_INVALID_ARG (null
 * pointer, K or dtype out of range, a non-positive spacing), DPMA_ERR_CUDA.
 */
dpma_status dpma_derived_moments(const void* moments, dpma_dtype dtype, int K,
                                 const double* spacing, double* out, void* stream);

/* ---------------- batches of volumes ---------------- */

/*
 * One volume of a batch.  `volume` is a device pointer laid out like every
 * volume of this library; `out_offset` is the byte offset of this volume's
 * dpma_num_moments(K) moments inside the batch's output buffer (a multiple of
 * 16; int128 moments for integer volumes, doubles for float32 ones).  Sizes,
 * element types and orders may differ between the volumes of one batch.
 */
typedef struct dpma_volume_desc {
  const void* volume;
  int64_t L, M, N;
  int32_t dtype; /* dpma_dtype */
  int32_t K;
  int64_t out_offset;
} dpma_volume_desc;

/* Opaque batch plan: the task table, its device buffers and the tuned launch. */
typedef struct dpma_batch dpma_batch;

#define DPMA_BATCH_AUTOTUNE 1 /* time the candidate CTA sizes at creation */

/*
 * Plans the moments of `count` volumes (the method of Sec. 3 applied to each
 * volume): validates every descriptor on the host, uploads the task table
 * and allocates the plan's device buffers (synchronous).  Volumes whose
 * images fit on chip (integer element types, a z-slice of at most 24 KB,
 * images within shared memory) run in persistent fused launches: projection
 * and 2-D moments per volume in shared memory, then one batched combine
 * launch.  The fused volumes whose footprint lets two 256-thread CTAs share
 * an SM run in a second launch after the larger ones (one launch when all
 * are alike).  The others (float32 or larger volumes) run through the
 * single-volume pipeline, one after another on the same stream.  With
 * DPMA_BATCH_AUTOTUNE the volumes must already hold their data: the split
 * and a single launch are timed at 256 and 512 threads per CTA and the
 * fastest is kept.
 * The descriptors' pointers are kept by the plan until dpma_batch_destroy.
 * Errors: DPMA_ERR_INVALID_ARG (null pointers, bad descriptor, unknown
 * flag), DPMA_ERR_OVERFLOW (a volume's moments could leave int128),
 * DPMA_ERR_OOM, DPMA_ERR_CUDA.
 */
dpma_status dpma_batch_create(const dpma_volume_desc* descs, int count, int flags,
                              dpma_batch** plan);

/*
 * Enqueues the whole batch on `stream` and returns: device memsets and
 * kernel launches only (no host synchronisation, no allocation), so the call
 * can be captured into a CUDA graph and replayed.  `out` is a device buffer
 * holding every descriptor's out_offset range.  The device status of the run
 * is read back by dpma_batch_status.  Runs of one plan must not overlap.
 */
dpma_status dpma_batch_run(dpma_batch* plan, void* out, void* stream);

/*
 * Waits for `stream` and returns the status of the plan's last run:
 * DPMA_OK, DPMA_ERR_INTERNAL (an exact combine left a remainder) or
 * DPMA_ERR_TIMEOUT (a bounded device wait gave up).
 */
dpma_status dpma_batch_status(dpma_batch* plan, void* stream);

/*
 * Plan facts for tests and tuning: what = 0 volumes in the fused launches,
 * 1 volumes on the single-volume path, 2 threads per CTA, 3 CTAs and 4
 * dynamic shared memory in bytes of the first fused launch, 5 fused
 * launches (0, 1 or 2), 6 volumes, 7 threads per CTA and 8 CTAs of the
 * second; -1 for a bad query.
 */
int dpma_batch_info(const dpma_batch* plan, int what);

/* Frees the plan and its device buffers (NULL is accepted). */
dpma_status dpma_batch_destroy(dpma_batch* plan);

/*
 * One-shot batch: dpma_batch_create (no autotuning), dpma_batch_run on
 * `stream`, dpma_batch_status and dpma_batch_destroy.  Synchronous.
 */
dpma_status dpma_moments_batched(const dpma_volume_desc* descs, int count, void* out,
                                 void* stream);

/* ---------------- serving ---------------- */

/*
 * Continuous-batching server for a stream of moment requests (each request:
 * the method of Sec. 3 on one volume).  Zero fields take the defaults.
 *   device_bytes  device memory the server holds for requests in flight
 *                 (default: a quarter of the free memory at creation);
 *   max_inflight  requests on the device at once (default 64);
 *   streams       CUDA streams the launches are spread over (default 4);
 *   max_group     most small volumes fused into one launch (default 256);
 *   max_pending   queued requests before submit refuses (default 4096).
 */
typedef struct dpma_server_config {
  int64_t device_bytes;
  int32_t max_inflight;
  int32_t streams;
  int32_t max_group;
  int32_t max_pending;
} dpma_server_config;

/* Counters since creation (or the last reset).  Latencies run from the entry
 * to dpma_server_submit (before the volume is copied into pinned memory) to
 * the moment the result is complete on the host. */
typedef struct dpma_server_counters {
  int64_t submitted, completed, failed, rejected, pending, inflight, launches;
  int64_t device_bytes_peak;
  double p50_ms, p99_ms, mean_ms, max_ms;
  double volumes_per_s, voxels_per_s; /* completed / (last done - first submit) */
  int64_t cache_hits;       /* keyed requests served from resident images */
  int64_t resident_volumes; /* keyed volumes whose images are resident now */
} dpma_server_counters;

typedef struct dpma_server dpma_server;

/*
 * Creates a server on the current device: allocates its device arena,
 * control blocks and streams, makes every combine plan resident and starts
 * its scheduler thread.  A scheduler admits queued requests in arrival order
 * whenever a slot and enough arena memory are free and launches them at once
 * (small integer volumes fused into one launch, the rest through the
 * single-volume pipeline), so requests that arrive while others run are
 * admitted as resources free up and their work overlaps on the device.
 * Errors: DPMA_ERR_INVALID_ARG, DPMA_ERR_OOM, DPMA_ERR_CUDA.
 */
dpma_status dpma_server_create(const dpma_server_config* cfg, dpma_server** server);

/*
 * Queues one request.  desc->volume is a HOST pointer; the volume is copied
 * before the call returns (desc->out_offset is ignored).  *ticket identifies
 * the request for dpma_server_wait / dpma_server_poll.  Thread-safe.
 * Errors: DPMA_ERR_INVALID_ARG / DPMA_ERR_OVERFLOW (descriptor), 
 * DPMA_ERR_REJECTED (queue full, or more device memory than the server
 * holds), DPMA_ERR_OOM (pinned host memory).
 */
dpma_status dpma_server_submit(dpma_server* server, const dpma_volume_desc* desc,
                               uint64_t* ticket);

/*
 * As dpma_server_submit, for a volume named by `key` (0: no key).  The
 * caller promises that one key always names the same volume (dimensions,
 * element type and voxels).  A keyed integer volume that runs through the
 * single-volume pipeline leaves its projection images resident in the
 * server's arena; a later request with the same key at an order K no higher
 * than theirs skips the upload and the projection and only takes the image
 * moments and the combine (the image set of order K is a prefix of the set
 * of every larger order, with the same geometry).  Resident images are
 * evicted, least recently used first, when admission needs the memory.
 * Float32 volumes keep no images: theirs are quantised on a grid of the
 * volume's own (or redone by the compensated fallback), so a keyed float32
 * request is computed in full.
 */
dpma_status dpma_server_submit_keyed(dpma_server* server, const dpma_volume_desc* desc,
                                     uint64_t key, uint64_t* ticket);

/*
 * Waits up to timeout_ms (< 0: no limit, 0: just check) for a request; on
 * success copies its dpma_num_moments(K) moments to host_out (int128 or
 * double; may be NULL) and releases the ticket.  DPMA_ERR_TIMEOUT: not
 * finished yet (the ticket stays valid); any other error releases the ticket
 * and reports the request's failure.  Thread-safe.
 */
dpma_status dpma_server_wait(dpma_server* server, uint64_t ticket, int64_t timeout_ms,
                             void* host_out);

/* 1: finished, 0: queued or running, -1: unknown ticket. */
int dpma_server_poll(dpma_server* server, uint64_t ticket);

/* Copies the counters; reset != 0 starts new ones. */
dpma_status dpma_server_stats(dpma_server* server, dpma_server_counters* out, int reset);

/*
 * Stops admitting, waits for the requests in flight, fails the queued ones
 * (DPMA_ERR_REJECTED) and frees the server.  No thread may use the server
 * during or after the call.  NULL is accepted.
 */
dpma_status dpma_server_destroy(dpma_server* server);

/* ---------------- no device allocation ---------------- */

/*
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc -- for example an application whose own memory
 * pool already holds the device memory it may use, or a latency-critical
 * loop that cannot accept cudaMalloc's device-wide synchronisation or its
 * possible failure.
 *
 * Same result as dpma_moments_async (device `volume` and `out`, enqueued on
 * `stream`, returns once enqueued), but the workspace -- projection images,
 * partial sums, status word -- lives in one static device array of 32 MiB,
 * and the combine tables of every order in a second one of 128 KiB; every
 * GPU which loads the library holds both until the process exits.  The call
 * allocates no device memory.  Volumes needing more workspace than 32 MiB
 * (dpma_workspace_size) are refused with DPMA_ERR_REJECTED; 512^3 float32 at
 * K = 6 fits.
 *
 * The first call on a device (with that device current) looks up the arrays'
 * device addresses and copies the combine tables into the second array
 * (synchronously); make that first call before any stream capture.  Later
 * calls only launch kernels.  Every call reuses the same workspace array and
 * clears what must start at zero; calls whose work overlaps on the GPU race
 * on it and must be serialised by the caller.
 *
 * A failure on the device (a bounded wait that gave up, DPMA_ERR_TIMEOUT; a
 * combine division that left a remainder, DPMA_ERR_INTERNAL) cannot be
 * returned by this asynchronous call; instead every one of the
 * dpma_num_moments(K) output moments is overwritten with a sentinel: a quiet
 * NaN for float32 volumes, the most negative int128 (-2^127) for integer
 * volumes, a value no integer volume's moment can take.
 */
dpma_status dpma_moments_noalloc(const void* volume, int64_t L, int64_t M, int64_t N,
                                 dpma_dtype dtype, int K, void* out, void* stream);

/* ---------------- profiling aid ---------------- */

/*
 * Per-stage device timing, off by default.  While enabled, the hot-path
 * calls record CUDA events on their launching stream around each stage:
 * 0 = clearing the image buffer, 1 = projection (Sec. 3.1), 2 = image
 * moments, 3 = combine.  The events add no device work.
 */
dpma_status dpma_stage_timing(int enable);
/*
 * Waits for the recorded events and returns, per stage, the summed device
 * milliseconds (`ms[4]`) and the number of library kernels launched
 * (`launches[4]`) since the last reset; `reset` != 0 clears the totals.
 * Either array may be NULL.
 */
dpma_status dpma_stage_times(double* ms, int64_t* launches, int reset);

#ifdef __cplusplus
}
#endif

#endif /* DPMA_H */
