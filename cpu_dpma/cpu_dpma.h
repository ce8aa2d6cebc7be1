// Multithreaded CPU implementation of the Discrete Projection Moment method
// (Sec. 3): the timed CPU baseline.  It shares no code with the CUDA library
// or with the oracle.
//
// Volumes are V[z][y][x] with x fastest (L columns, M rows, N slices),
// element type 0 = uint8, 1 = uint16, 2 = float32.  Moments M_pqr with
// p + q + r <= K come in graded order: degree ascending, then p descending,
// then q descending ((K+1)(K+2)(K+3)/6 of them).
#pragma once
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

// Largest supported order.
int cpu_dpma_max_order(void);

// Number of projection images the method uses at order K (0 if K is out of
// range or no image set of full rank exists).
int cpu_dpma_num_images(int K);

// All raw moments of the volume `vol` (host memory, not modified).
//   threads: worker threads (<= 0: all hardware threads).
//   out:     integer volumes: two int64 words (low, then high, two's
//            complement) per moment, i.e. an int128; float32 volumes: one
//            double per moment.
//   threads_used (may be null): receives the thread count actually used.
// Returns 0 on success; 1 invalid argument, 2 non-finite float voxel,
// 3 a result outside the int128 range, 4 no image set of full rank at this
// order, 5 out of memory.  On error `out` is left unspecified.
int cpu_dpma_moments(const void* vol, int64_t L, int64_t M, int64_t N, int dtype, int K,
                     int threads, void* out, int* threads_used);

// The quantisation exponent e used for the last float32 call on this thread:
// every voxel was rounded to the nearest multiple of 2^-e before the exact
// integer pipeline (so |error of M_pqr| <= 2^(-e-1) * sum x^p y^q z^r).
int cpu_dpma_last_float_exponent(void);

#ifdef __cplusplus
}
#endif
