/*
 * Oracle GEMM in plain C, FP64.  TEST INFRASTRUCTURE ONLY.
 *
 * This file is the correctness reference for the Stream-K GEMM library.  It is
 * deliberately slow and obviously correct: a plain loop nest with no blocking,
 * no fusion and no reordering of the summation.  Only tests/, the smoke check in
 * __graft_entry__.py and the cpu_baseline / reference legs of bench.py may load
 * it.  It shares no code with the CUDA path.
 *
 * What it computes (paper, Section 2 "Background"): the GEMM product
 *
 *     C = alpha * A * B + beta * C
 *
 * for an m x k matrix A and a k x n matrix B.  For every output element the
 * sum over the accumulation index l = 0 .. k-1 is taken in increasing order of
 * l, exactly the innermost "kkk" loop of the sequential cache-blocked GEMM
 * (Algorithm 1) once the blocking is removed.  Inputs are given as doubles that
 * already hold the rounded FP16 / BF16 / FP8 input values (each of those widens
 * to FP64 exactly, and every product of two of them is exact in FP64), so the
 * only rounding here is FP64 summation, about 2^-53 relative.
 *
 * Besides C64 it returns (|A| |B|)_ij = sum_l |A_il| |B_lj|, the magnitude term
 * of the error bound the tests apply to the GPU results.
 *
 * Matrices are addressed through element strides, so one routine serves every
 * storage order: X(i, j) = X[i * rs + j * cs].
 */
#include <stdint.h>
#include <stddef.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Number of threads the OpenMP runtime will use for the next parallel region. */
int oracle_max_threads(int nthreads) {
#ifdef _OPENMP
    set_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* One output element: alpha * sum_l A(i,l) B(l,j) + beta * Cin(i,j). */
static void one_entry(int64_t i, int64_t j, int64_t k, double alpha,
                      const double* A, int64_t a_rs, int64_t a_cs,
                      const double* B, int64_t b_rs, int64_t b_cs,
                      double beta, const double* Cin, int64_t c_rs, int64_t c_cs,
                      double* out, double* abs_out) {
    double s = 0.0, s_abs = 0.0;
    for (int64_t l = 0; l < k; ++l) {
        double a = A[i * a_rs + l * a_cs];
        double b = B[l * b_rs + j * b_cs];
        s += a * b;
        s_abs += fabs(a) * fabs(b);
    }
    double c = alpha * s;
    if (beta != 0.0) c += beta * Cin[i * c_rs + j * c_cs];
    *out = c;
    if (abs_out) *abs_out = s_abs;
}

/*
 * Full product.  C64 and absAB (may be NULL) are m x n, row-major, dense.
 * Cin may be NULL only when beta == 0.
 */
int oracle_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t a_rs, int64_t a_cs,
                    const double* B, int64_t b_rs, int64_t b_cs,
                    double beta, const double* Cin, int64_t c_rs, int64_t c_cs,
                    double* C64, double* absAB, int nthreads) {
    if (m < 0 || n < 0 || k < 0 || C64 == NULL) return ORACLE_EINVAL;
    if (k > 0 && (A == NULL || B == NULL)) return ORACLE_EINVAL;
    if (beta != 0.0 && Cin == NULL) return ORACLE_EINVAL;
    set_threads(nthreads);
    int64_t total = m * n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t e = 0; e < total; ++e) {
        int64_t i = e / n, j = e % n;
        one_entry(i, j, k, alpha, A, a_rs, a_cs, B, b_rs, b_cs, beta, Cin, c_rs, c_cs,
                  &C64[e], absAB ? &absAB[e] : NULL);
    }
    return ORACLE_OK;
}

/*
 * Selected entries only: out[e] = C64(rows[e], cols[e]).  Used where the full
 * product is too large for the CPU (a seeded sample of a big GEMM) and by the
 * CPU timing leg.  Same arithmetic as oracle_gemm_f64 entry by entry.
 */
int oracle_gemm_entries_f64(int64_t count, const int64_t* rows, const int64_t* cols,
                            int64_t k, double alpha,
                            const double* A, int64_t a_rs, int64_t a_cs,
                            const double* B, int64_t b_rs, int64_t b_cs,
                            double beta, const double* Cin, int64_t c_rs, int64_t c_cs,
                            double* out, double* abs_out, int nthreads) {
    if (count < 0 || k < 0 || out == NULL || rows == NULL || cols == NULL) return ORACLE_EINVAL;
    if (beta != 0.0 && Cin == NULL) return ORACLE_EINVAL;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t e = 0; e < count; ++e) {
        one_entry(rows[e], cols[e], k, alpha, A, a_rs, a_cs, B, b_rs, b_cs, beta, Cin,
                  c_rs, c_cs, &out[e], abs_out ? &abs_out[e] : NULL);
    }
    return ORACLE_OK;
}
