/*
 * power_omp.c -- TEST INFRASTRUCTURE ONLY: a timed CPU baseline, built apart from
 * the oracle library.  Only the test suite and the benchmark's CPU-baseline leg
 * load it; the product path never does, and it shares no code with the CUDA
 * library.
 *
 * MAT-ITER of Section 4 on the uncompleted P, run on all host cores with OpenMP:
 *   X_0 = 0,  X_{k+1} = dPX_k + (1-d)V,
 *   stop when |X_{k+1} - X_k|_1 * d/(1-d) < tol  or after max_iter products.
 * It is the iteration of orc_power in oracle.c written as a pull over in-links,
 * X_{k+1}[j] = (1-d)V[j] + sum over in-links i -> j of d X_k[i] / #out_i, so that
 * every row is computed by one thread and no two threads write the same entry.
 * The row sums run in the in-link order of the lists, so the result differs from
 * orc_power's only by the order of additions; tests/test_oracle_pins.py checks
 * both against each other.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef int32_t i32;
typedef int64_t i64;

/* threads actually used by a parallel region (1 when compiled without OpenMP) */
int pomp_threads(int want) {
#ifdef _OPENMP
    if (want > 0) omp_set_num_threads(want);
    int got = 1;
#pragma omp parallel
    {
#pragma omp single
        got = omp_get_num_threads();
    }
    return got;
#else
    (void)want;
    return 1;
#endif
}

/*
 * in_ptr[n+1], in_src[L]: the in-link lists (row j lists every i with i -> j);
 * outdeg[n]: #out_i.  X[n] receives the last iterate.  Returns 0 when the stop
 * rule was met, 1 when max_iter products ran first.
 */
int pomp_power(i32 n, const i32 *in_ptr, const i32 *in_src, const i32 *outdeg, double d, const double *V,
               double tol, i64 max_iter, double *X, i64 *iters, double *last_delta) {
    double *Y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *Z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (i32 i = 0; i < n; ++i) X[i] = 0.0;
    i64 it = 0;
    double delta = INFINITY;
    int ok = 0;
    while (it < max_iter) {
        /* z_i = d X_i / #out_i (zero for a dangling node: its column of P is empty) */
#pragma omp parallel for schedule(static)
        for (i32 i = 0; i < n; ++i) Z[i] = outdeg[i] ? d * X[i] / (double)outdeg[i] : 0.0;
        delta = 0.0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : delta)
        for (i32 j = 0; j < n; ++j) {
            double acc = 0.0;
            for (i32 e = in_ptr[j]; e < in_ptr[j + 1]; ++e) acc += Z[in_src[e]];
            Y[j] = (1.0 - d) * V[j] + acc;
            delta += fabs(Y[j] - X[j]);
        }
#pragma omp parallel for schedule(static)
        for (i32 j = 0; j < n; ++j) X[j] = Y[j];
        ++it;
        if (delta * d / (1.0 - d) < tol) {
            ok = 1;
            break;
        }
    }
    free(Y);
    free(Z);
    *iters = it;
    *last_delta = delta;
    return ok ? 0 : 1;
}
