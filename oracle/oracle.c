/*
 * CPU oracle for the Discrete Projection Moment method (Diggin & Diggin,
 * "Fast 3D Image Moments", 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * Every function is a plain restatement of a definition from the paper:
 *
 *   oracle_moments_*        Sec. 1, Eq. 2: M_pqr = sum V(x,y,z) x^p y^q z^r,
 *                           0 <= x < L, 0 <= y < M, 0 <= z < N, for all
 *                           p+q+r <= K.  Integer volumes accumulate in
 *                           __int128 with overflow detection; float volumes
 *                           in FP64 with Neumaier-compensated summation.
 *   oracle_project_*        Sec. 3.1, Eq. 4 (general line sum) with the
 *                           image set of Eqs. 5-9 and the +-pi/4 families
 *                           named after Eq. 9: every voxel is added to the
 *                           pixel its two linear forms select.
 *   oracle_image_moments_*  Sec. 1, Eq. 1: M_pq = sum I(i,j) i^p j^q over a
 *                           stored image, with signed coordinates.
 *
 * Coordinates are 0-based with the origin at voxel (0,0,0) and 0^0 = 1.
 *
 * Moment order ("graded"): degree n = p+q+r ascending, then p descending,
 * then q descending: 000, 100, 010, 001, 200, 110, 101, 020, 011, 002, ...
 *
 * Image storage contract (image k is a row-major array [S_k][F_k]; a voxel
 * (x,y,z) lands on row s = slow(x,y,z) and column f = fast(x,y,z)):
 *
 *   k  line direction   slow s            fast f            S_k      F_k
 *   0  z                y                 x                 M        L
 *   1  x                z                 y                 N        M
 *   2  y                z                 x                 N        L
 *   3  (1,0,-1)         y                 x+z               M        L+N-1
 *   4  (1,0,1)          y                 x-z+(N-1)         M        L+N-1
 *   5  (0,1,-1)         y+z               x                 M+N-1    L
 *   6  (0,1,1)          y-z+(N-1)         x                 M+N-1    L
 *   7  (1,-1,0)         z                 x+y               N        L+M-1
 *   8  (1,1,0)          z                 x-y+(M-1)         N        L+M-1
 *   9  (2,0,-1)         y                 x+2z              M        L+2N-2
 *  10  (1,-1,-1)        x+z               2y+x-z+(N-1)      L+N-1    L+2M+N-3
 *
 * Images 0-2 are Eqs. 5-7, images 3-4 are Eqs. 8-9 and images 5-8 are the
 * remaining +-pi/4 projections about the x and z axes (Sec. 3.1).  Orders
 * K = 9 and 10 take one more image each from the further families Sec. 3.1
 * names after Eq. 9: image 9 is the arctan(1/2) rotation about y (line
 * direction (2,0,-1)), image 10 the isometric projection whose coordinates
 * (x+z, 2y+x-z) and zero-padded size (L+N-1) x (L+2M+N-3) the paper states.  The signed
 * coordinate of an offset column or row is the stored index minus the
 * offset (the origin shift described in Sec. 5).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef __int128 i128;

/* Largest order K the oracle takes, and the image count it needs. */
#define ORACLE_MAX_K 10
#define ORACLE_MAX_IMAGES 11

/* ------------------------------------------------------------------ */
/* moment bookkeeping                                                  */
/* ------------------------------------------------------------------ */

int oracle_num_moments(int K) { return (K + 1) * (K + 2) * (K + 3) / 6; }

/* List the exponent triples in graded order. */
static int graded_triples(int K, int* pq_r /* 3*count */) {
    int m = 0;
    for (int n = 0; n <= K; ++n)
        for (int p = n; p >= 0; --p)
            for (int q = n - p; q >= 0; --q) {
                pq_r[3 * m + 0] = p;
                pq_r[3 * m + 1] = q;
                pq_r[3 * m + 2] = n - p - q;
                ++m;
            }
    return m;
}

/* ------------------------------------------------------------------ */
/* Eq. 2 for integer volumes                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    const void* vol;
    int elem_bytes;
    int64_t L, M, N;
    int K, nmom;
    const int* trip;
    int64_t z0, z1;
    i128* acc;    /* nmom partial sums */
    int overflow; /* set if any product or sum left the int128 range */
} int_job;

/* pw[e] = c^e for e = 0..K; returns 1 if one of them leaves the int128 range. */
static int checked_powers(i128* pw, int64_t c, int K) {
    pw[0] = 1;
    for (int e = 1; e <= K; ++e)
        if (__builtin_mul_overflow(pw[e - 1], (i128)c, &pw[e])) return 1;
    return 0;
}

static uint32_t load_int(const void* vol, int elem_bytes, int64_t idx) {
    if (elem_bytes == 1) return ((const uint8_t*)vol)[idx];
    return ((const uint16_t*)vol)[idx];
}

static void* int_worker(void* arg) {
    int_job* J = (int_job*)arg;
    const int K = J->K;
    i128 xp[ORACLE_MAX_K + 1], yp[ORACLE_MAX_K + 1], zp[ORACLE_MAX_K + 1];
    for (int m = 0; m < J->nmom; ++m) J->acc[m] = 0;
    for (int64_t z = J->z0; z < J->z1; ++z) {
        int zov = checked_powers(zp, z, K);
        for (int64_t y = 0; y < J->M; ++y) {
            int yov = checked_powers(yp, y, K);
            for (int64_t x = 0; x < J->L; ++x) {
                uint32_t v = load_int(J->vol, J->elem_bytes, (z * J->M + y) * J->L + x);
                if (v == 0) continue; /* a zero voxel adds nothing to Eq. 2 */
                /* Coordinates are non-negative, so every term is too and a power
                 * c^e past the int128 range makes the moment with that single
                 * exponent (e, 0, 0), (0, e, 0) or (0, 0, e) overflow as well. */
                if (checked_powers(xp, x, K) || yov || zov) {
                    J->overflow = 1;
                    return NULL;
                }
                for (int m = 0; m < J->nmom; ++m) {
                    const int* t = J->trip + 3 * m;
                    i128 term, a, b;
                    /* V * x^p * y^q * z^r with every step checked */
                    if (__builtin_mul_overflow((i128)v, xp[t[0]], &a) ||
                        __builtin_mul_overflow(a, yp[t[1]], &b) ||
                        __builtin_mul_overflow(b, zp[t[2]], &term) ||
                        __builtin_add_overflow(J->acc[m], term, &J->acc[m])) {
                        J->overflow = 1;
                        return NULL;
                    }
                }
            }
        }
    }
    return NULL;
}

/*
 * out: nmom little-endian int128 values as (lo, hi) int64 pairs.
 * Returns 0 on success, 1 on bad arguments, 2 if a value overflowed int128.
 * Every product and sum is checked, so a volume whose moments leave the
 * int128 range (large volumes at K = 9, 10) is reported, never wrapped.
 */
int oracle_moments_int(const void* vol, int elem_bytes, int64_t L, int64_t M, int64_t N, int K,
                       int nthreads, int64_t* out) {
    if (!vol || !out || L < 1 || M < 1 || N < 1 || K < 0 || K > ORACLE_MAX_K) return 1;
    if (elem_bytes != 1 && elem_bytes != 2) return 1;
    if (L > 65536 || M > 65536 || N > 65536) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N) nthreads = (int)N;
    int nmom = oracle_num_moments(K);
    int* trip = (int*)malloc(sizeof(int) * 3 * nmom);
    graded_triples(K, trip);
    int_job* jobs = (int_job*)calloc(nthreads, sizeof(int_job));
    i128* acc = (i128*)calloc((size_t)nthreads * nmom, sizeof(i128));
    pthread_t* th = (pthread_t*)calloc(nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (int_job){vol, elem_bytes, L, M, N, K, nmom, trip,
                            N * t / nthreads, N * (t + 1) / nthreads, acc + (size_t)t * nmom, 0};
        if (nthreads > 1) pthread_create(&th[t], NULL, int_worker, &jobs[t]);
        else int_worker(&jobs[t]);
    }
    int overflow = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (nthreads > 1) pthread_join(th[t], NULL);
        overflow |= jobs[t].overflow;
    }
    for (int m = 0; m < nmom && !overflow; ++m) {
        i128 s = 0;
        for (int t = 0; t < nthreads; ++t)
            if (__builtin_add_overflow(s, acc[(size_t)t * nmom + m], &s)) overflow = 1;
        uint64_t lo = (uint64_t)s;
        uint64_t hi = (uint64_t)(s >> 64);
        out[2 * m] = (int64_t)lo;
        out[2 * m + 1] = (int64_t)hi;
    }
    free(trip); free(jobs); free(acc); free(th);
    return overflow ? 2 : 0;
}

/* ------------------------------------------------------------------ */
/* Eq. 2 for float32 volumes (FP64, Neumaier compensated)              */
/* ------------------------------------------------------------------ */

typedef struct { double s, c; } nsum; /* running sum and its compensation */

static void nsum_add(nsum* a, double v) {
    double t = a->s + v;
    if ((a->s < 0 ? -a->s : a->s) >= (v < 0 ? -v : v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

typedef struct {
    const float* vol;
    int64_t L, M, N;
    int K, nmom;
    const int* trip;
    int64_t z0, z1;
    nsum* acc;
} f_job;

static void* f_worker(void* arg) {
    f_job* J = (f_job*)arg;
    const int K = J->K;
    double xp[ORACLE_MAX_K + 1], yp[ORACLE_MAX_K + 1], zp[ORACLE_MAX_K + 1];
    for (int m = 0; m < J->nmom; ++m) J->acc[m] = (nsum){0.0, 0.0};
    for (int64_t z = J->z0; z < J->z1; ++z) {
        zp[0] = 1.0;
        for (int e = 1; e <= K; ++e) zp[e] = zp[e - 1] * (double)z;
        for (int64_t y = 0; y < J->M; ++y) {
            yp[0] = 1.0;
            for (int e = 1; e <= K; ++e) yp[e] = yp[e - 1] * (double)y;
            for (int64_t x = 0; x < J->L; ++x) {
                double v = (double)J->vol[(z * J->M + y) * J->L + x];
                if (v == 0.0) continue;
                xp[0] = 1.0;
                for (int e = 1; e <= K; ++e) xp[e] = xp[e - 1] * (double)x;
                for (int m = 0; m < J->nmom; ++m) {
                    const int* t = J->trip + 3 * m;
                    nsum_add(&J->acc[m], v * xp[t[0]] * yp[t[1]] * zp[t[2]]);
                }
            }
        }
    }
    return NULL;
}

/*
 * out: nmom doubles.  With abs_values != 0 the oracle sums |V| instead of V
 * (the reference magnitude M_pqr(|V|) used by the float tolerance).
 */
static int moments_f32_impl(const float* vol, int64_t L, int64_t M, int64_t N, int K,
                            int nthreads, double* out, int abs_values) {
    if (!vol || !out || L < 1 || M < 1 || N < 1 || K < 0 || K > ORACLE_MAX_K) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > N) nthreads = (int)N;
    int nmom = oracle_num_moments(K);
    int* trip = (int*)malloc(sizeof(int) * 3 * nmom);
    graded_triples(K, trip);
    const float* src = vol;
    float* absbuf = NULL;
    if (abs_values) {
        size_t n = (size_t)L * M * N;
        absbuf = (float*)malloc(n * sizeof(float));
        for (size_t i = 0; i < n; ++i) absbuf[i] = vol[i] < 0 ? -vol[i] : vol[i];
        src = absbuf;
    }
    f_job* jobs = (f_job*)calloc(nthreads, sizeof(f_job));
    nsum* acc = (nsum*)calloc((size_t)nthreads * nmom, sizeof(nsum));
    pthread_t* th = (pthread_t*)calloc(nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (f_job){src, L, M, N, K, nmom, trip, N * t / nthreads, N * (t + 1) / nthreads,
                          acc + (size_t)t * nmom};
        if (nthreads > 1) pthread_create(&th[t], NULL, f_worker, &jobs[t]);
        else f_worker(&jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t)
        if (nthreads > 1) pthread_join(th[t], NULL);
    for (int m = 0; m < nmom; ++m) {
        nsum s = {0.0, 0.0};
        for (int t = 0; t < nthreads; ++t) {
            nsum_add(&s, acc[(size_t)t * nmom + m].s);
            nsum_add(&s, acc[(size_t)t * nmom + m].c);
        }
        out[m] = s.s + s.c;
    }
    free(trip); free(jobs); free(acc); free(th); free(absbuf);
    return 0;
}

int oracle_moments_f32(const float* vol, int64_t L, int64_t M, int64_t N, int K, int nthreads,
                       double* out) {
    return moments_f32_impl(vol, L, M, N, K, nthreads, out, 0);
}

int oracle_moments_f32_abs(const float* vol, int64_t L, int64_t M, int64_t N, int K,
                           int nthreads, double* out) {
    return moments_f32_impl(vol, L, M, N, K, nthreads, out, 1);
}

/* ------------------------------------------------------------------ */
/* Projection images (Eq. 4 with the image set of the table above)     */
/* ------------------------------------------------------------------ */

int oracle_num_images(int K) { return K + 1 < 3 ? 3 : K + 1; }

/* Image geometry from the table in the header comment. */
int oracle_image_geometry(int k, int64_t L, int64_t M, int64_t N, int64_t* S, int64_t* F,
                          int64_t* off_s, int64_t* off_f) {
    int64_t s = 0, f = 0, os = 0, of = 0;
    switch (k) {
        case 0: s = M; f = L; break;
        case 1: s = N; f = M; break;
        case 2: s = N; f = L; break;
        case 3: s = M; f = L + N - 1; break;
        case 4: s = M; f = L + N - 1; of = N - 1; break;
        case 5: s = M + N - 1; f = L; break;
        case 6: s = M + N - 1; f = L; os = N - 1; break;
        case 7: s = N; f = L + M - 1; break;
        case 8: s = N; f = L + M - 1; of = M - 1; break;
        case 9: s = M; f = L + 2 * (N - 1); break;
        case 10: s = L + N - 1; f = L + 2 * M + N - 3; of = N - 1; break;
        default: return 1;
    }
    *S = s; *F = f; *off_s = os; *off_f = of;
    return 0;
}

/* Signed (slow, fast) coordinates of voxel (x,y,z) in image k. */
static void image_coords(int k, int64_t x, int64_t y, int64_t z, int64_t* s, int64_t* f) {
    switch (k) {
        case 0: *s = y;     *f = x;     break;
        case 1: *s = z;     *f = y;     break;
        case 2: *s = z;     *f = x;     break;
        case 3: *s = y;     *f = x + z; break;
        case 4: *s = y;     *f = x - z; break;
        case 5: *s = y + z; *f = x;     break;
        case 6: *s = y - z; *f = x;     break;
        case 7: *s = z;     *f = x + y; break;
        case 8: *s = z;     *f = x - y; break;
        case 9: *s = y;     *f = x + 2 * z; break;
        default: *s = x + z; *f = 2 * y + x - z; break;
    }
}

/*
 * Images 0..P-1 are written back to back into out (uint64 pixels), each in
 * its [S_k][F_k] layout.  Returns 0, or 1 on bad arguments.
 */
int oracle_project_int(const void* vol, int elem_bytes, int64_t L, int64_t M, int64_t N, int P,
                       uint64_t* out) {
    if (!vol || !out || L < 1 || M < 1 || N < 1 || P < 1 || P > ORACLE_MAX_IMAGES) return 1;
    if (elem_bytes != 1 && elem_bytes != 2) return 1;
    int64_t base[ORACLE_MAX_IMAGES], S[ORACLE_MAX_IMAGES], F[ORACLE_MAX_IMAGES];
    int64_t os[ORACLE_MAX_IMAGES], of[ORACLE_MAX_IMAGES], tot = 0;
    for (int k = 0; k < P; ++k) {
        oracle_image_geometry(k, L, M, N, &S[k], &F[k], &os[k], &of[k]);
        base[k] = tot;
        tot += S[k] * F[k];
    }
    memset(out, 0, sizeof(uint64_t) * (size_t)tot);
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < M; ++y)
            for (int64_t x = 0; x < L; ++x) {
                uint64_t v = load_int(vol, elem_bytes, (z * M + y) * L + x);
                for (int k = 0; k < P; ++k) {
                    int64_t s, f;
                    image_coords(k, x, y, z, &s, &f);
                    out[base[k] + (s + os[k]) * F[k] + (f + of[k])] += v;
                }
            }
    return 0;
}

/* Same for float32 volumes; each pixel is an FP64 sum. */
int oracle_project_f32(const float* vol, int64_t L, int64_t M, int64_t N, int P, double* out) {
    if (!vol || !out || L < 1 || M < 1 || N < 1 || P < 1 || P > ORACLE_MAX_IMAGES) return 1;
    int64_t base[ORACLE_MAX_IMAGES], S[ORACLE_MAX_IMAGES], F[ORACLE_MAX_IMAGES];
    int64_t os[ORACLE_MAX_IMAGES], of[ORACLE_MAX_IMAGES], tot = 0;
    for (int k = 0; k < P; ++k) {
        oracle_image_geometry(k, L, M, N, &S[k], &F[k], &os[k], &of[k]);
        base[k] = tot;
        tot += S[k] * F[k];
    }
    memset(out, 0, sizeof(double) * (size_t)tot);
    for (int64_t z = 0; z < N; ++z)
        for (int64_t y = 0; y < M; ++y)
            for (int64_t x = 0; x < L; ++x) {
                double v = (double)vol[(z * M + y) * L + x];
                for (int k = 0; k < P; ++k) {
                    int64_t s, f;
                    image_coords(k, x, y, z, &s, &f);
                    out[base[k] + (s + os[k]) * F[k] + (f + of[k])] += v;
                }
            }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Eq. 1 on a stored image, signed coordinates                         */
/* ------------------------------------------------------------------ */

/*
 * T_ab = sum_{s,f} I[s][f] (s - off_s)^a (f - off_f)^b for a+b <= K, in the
 * order (0,0), (1,0), (0,1), (2,0), (1,1), (0,2), ... (degree ascending,
 * slow exponent a descending).  Output int128 as (lo, hi) pairs.
 * Returns 0, 1 on bad arguments, 2 on int128 overflow.
 */
int oracle_image_moments_int(const uint64_t* img, int64_t S, int64_t F, int64_t off_s,
                             int64_t off_f, int K, int64_t* out) {
    if (!img || !out || S < 1 || F < 1 || K < 0 || K > ORACLE_MAX_K) return 1;
    int nm = (K + 1) * (K + 2) / 2;
    i128 acc[(ORACLE_MAX_K + 1) * (ORACLE_MAX_K + 2) / 2];
    for (int m = 0; m < nm; ++m) acc[m] = 0;
    for (int64_t s = 0; s < S; ++s)
        for (int64_t f = 0; f < F; ++f) {
            i128 v = (i128)img[s * F + f];
            if (v == 0) continue;
            i128 cs = s - off_s, cf = f - off_f;
            int m = 0;
            for (int n = 0; n <= K; ++n)
                for (int a = n; a >= 0; --a, ++m) {
                    i128 t = v, r;
                    for (int e = 0; e < a; ++e)
                        if (__builtin_mul_overflow(t, cs, &t)) return 2;
                    for (int e = 0; e < n - a; ++e)
                        if (__builtin_mul_overflow(t, cf, &t)) return 2;
                    if (__builtin_add_overflow(acc[m], t, &r)) return 2;
                    acc[m] = r;
                }
        }
    for (int m = 0; m < nm; ++m) {
        out[2 * m] = (int64_t)(uint64_t)acc[m];
        out[2 * m + 1] = (int64_t)(uint64_t)(acc[m] >> 64);
    }
    return 0;
}

/* FP64 version for float images (Neumaier-compensated). */
int oracle_image_moments_f64(const double* img, int64_t S, int64_t F, int64_t off_s,
                             int64_t off_f, int K, double* out) {
    if (!img || !out || S < 1 || F < 1 || K < 0 || K > ORACLE_MAX_K) return 1;
    int nm = (K + 1) * (K + 2) / 2;
    nsum acc[(ORACLE_MAX_K + 1) * (ORACLE_MAX_K + 2) / 2];
    for (int m = 0; m < nm; ++m) acc[m] = (nsum){0.0, 0.0};
    for (int64_t s = 0; s < S; ++s)
        for (int64_t f = 0; f < F; ++f) {
            double v = img[s * F + f];
            if (v == 0.0) continue;
            double cs = (double)(s - off_s), cf = (double)(f - off_f);
            int m = 0;
            for (int n = 0; n <= K; ++n)
                for (int a = n; a >= 0; --a, ++m) {
                    double t = v;
                    for (int e = 0; e < a; ++e) t *= cs;
                    for (int e = 0; e < n - a; ++e) t *= cf;
                    nsum_add(&acc[m], t);
                }
        }
    for (int m = 0; m < nm; ++m) out[m] = acc[m].s + acc[m].c;
    return 0;
}

/* ------------------------------------------------------------------ */
/* central moments (Sec. 4): centroid, mu_pqr and the scale |mu|_pqr   */
/* ------------------------------------------------------------------ */

/*
 * Straight from the definitions of Sec. 4: the centroid
 * (M100/M000, M010/M000, M001/M000) from exact sums (int128 for integer
 * volumes, Neumaier-compensated FP64 for float32), then
 *     mu_pqr     = sum V (x-xbar)^p (y-ybar)^q (z-zbar)^r
 *     muabs_pqr  = sum |V| |x-xbar|^p |y-ybar|^q |z-zbar|^r
 * as compensated FP64 sums over the voxels.  elem_bytes: 1 (uint8),
 * 2 (uint16) or 4 (float32).  centroid: 3 doubles (NaN when M000 = 0).
 * Returns 0, or 1 on bad arguments.
 */
int oracle_central_moments(const void* vol, int elem_bytes, int64_t L, int64_t M, int64_t N,
                           int K, double* centroid, double* mu, double* muabs) {
    if (!vol || !centroid || !mu || !muabs || L < 1 || M < 1 || N < 1 || K < 0 || K > ORACLE_MAX_K) return 1;
    if (elem_bytes != 1 && elem_bytes != 2 && elem_bytes != 4) return 1;
    const int nmom = oracle_num_moments(K);
    int trip[3 * 165];
    graded_triples(K, trip);
    double c[3];
    if (elem_bytes == 4) {
        const float* f = (const float*)vol;
        nsum s0 = {0, 0}, sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
        for (int64_t z = 0; z < N; ++z)
            for (int64_t y = 0; y < M; ++y)
                for (int64_t x = 0; x < L; ++x) {
                    const double v = f[(z * M + y) * L + x];
                    nsum_add(&s0, v);
                    nsum_add(&sx, v * (double)x);
                    nsum_add(&sy, v * (double)y);
                    nsum_add(&sz, v * (double)z);
                }
        const double m0 = s0.s + s0.c;
        c[0] = (sx.s + sx.c) / m0;
        c[1] = (sy.s + sy.c) / m0;
        c[2] = (sz.s + sz.c) / m0;
    } else {
        i128 s0 = 0, sx = 0, sy = 0, sz = 0;
        for (int64_t z = 0; z < N; ++z)
            for (int64_t y = 0; y < M; ++y)
                for (int64_t x = 0; x < L; ++x) {
                    const i128 v = load_int(vol, elem_bytes, (z * M + y) * L + x);
                    s0 += v;
                    sx += v * x;
                    sy += v * y;
                    sz += v * z;
                }
        const long double m0 = (long double)s0;
        c[0] = (double)((long double)sx / m0);
        c[1] = (double)((long double)sy / m0);
        c[2] = (double)((long double)sz / m0);
    }
    for (int i = 0; i < 3; ++i) centroid[i] = c[i];
    nsum* acc = (nsum*)calloc((size_t)nmom, sizeof(nsum));
    nsum* aab = (nsum*)calloc((size_t)nmom, sizeof(nsum));
    if (!acc || !aab) { free(acc); free(aab); return 1; }
    double xp[ORACLE_MAX_K + 1], yp[ORACLE_MAX_K + 1], zp[ORACLE_MAX_K + 1];
    for (int64_t z = 0; z < N; ++z) {
        zp[0] = 1.0;
        for (int e = 1; e <= K; ++e) zp[e] = zp[e - 1] * ((double)z - c[2]);
        for (int64_t y = 0; y < M; ++y) {
            yp[0] = 1.0;
            for (int e = 1; e <= K; ++e) yp[e] = yp[e - 1] * ((double)y - c[1]);
            for (int64_t x = 0; x < L; ++x) {
                const int64_t idx = (z * M + y) * L + x;
                const double v = elem_bytes == 4 ? (double)((const float*)vol)[idx]
                                                 : (double)load_int(vol, elem_bytes, idx);
                if (v == 0.0) continue;
                xp[0] = 1.0;
                for (int e = 1; e <= K; ++e) xp[e] = xp[e - 1] * ((double)x - c[0]);
                for (int m = 0; m < nmom; ++m) {
                    const int* t = trip + 3 * m;
                    const double w = xp[t[0]] * yp[t[1]] * zp[t[2]];
                    nsum_add(&acc[m], v * w);
                    nsum_add(&aab[m], (v < 0 ? -v : v) * (w < 0 ? -w : w));
                }
            }
        }
    }
    for (int m = 0; m < nmom; ++m) {
        mu[m] = acc[m].s + acc[m].c;
        muabs[m] = aab[m].s + aab[m].c;
    }
    free(acc);
    free(aab);
    return 0;
}
