/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY: the reference computation that the CUDA
 * path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does.  It shares no code with the CUDA library.
 *
 * Everything is plain, sequential FP64 and follows the paper's statement:
 *
 *   D. Hong, "Optimized on-line computation of PageRank algorithm".
 *   Section 2.1   : X = dPX + (1-d)V, P_ij = p(i,j) = probability of j -> i,
 *                   so column j of P holds 1/outdeg(j) on each child of j.
 *   Section 2.2   : fluid F_0 = (1-d)V, F_n = (I - J_in + dPJ_in) F_{n-1},
 *                   history H_n = sum_k J_ik F_{k-1}, and ALGO-REF.
 *   Section 3.3   : "About dangling nodes": a node with no child loses its
 *                   fluid (R -= sent) and P is never completed.
 *   Section 4     : the sequence choices ALGO-PER, ALGO-RAND, ALGO-MAX, the
 *                   threshold sweeps that replace argmax, MAT-ITER and its
 *                   stopping rule |X_n - X_{n-1}| d/(1-d) < Target.
 *
 * Readings of points the paper leaves open (threshold schedule, snapshot sweep,
 * tie-breaks) are stated beside the code that takes them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef int32_t i32;
typedef int64_t i64;
typedef uint64_t u64;

/* ------------------------------------------------------------- graph views */

/* out-degree #out_i = number of listed out-links (multi-edges counted) */
void orc_outdeg(i32 n, const i32 *row_ptr, i32 *outdeg) {
    for (i32 i = 0; i < n; ++i) outdeg[i] = row_ptr[i + 1] - row_ptr[i];
}

/*
 * In-link lists (the "collection" view of the introduction): in_ptr[n+1],
 * in_src[L].  Row j lists every i with an edge i -> j, in ascending i
 * (a counting sort that walks the out-lists in order).
 */
void orc_transpose(i32 n, const i32 *row_ptr, const i32 *col_idx, i32 *in_ptr, i32 *in_src) {
    i64 L = row_ptr[n];
    for (i32 j = 0; j <= n; ++j) in_ptr[j] = 0;
    for (i64 e = 0; e < L; ++e) in_ptr[col_idx[e] + 1] += 1;
    for (i32 j = 0; j < n; ++j) in_ptr[j + 1] += in_ptr[j];
    i32 *fill = (i32 *)malloc(sizeof(i32) * (size_t)(n > 0 ? n : 1));
    for (i32 j = 0; j < n; ++j) fill[j] = in_ptr[j];
    for (i32 i = 0; i < n; ++i)
        for (i32 e = row_ptr[i]; e < row_ptr[i + 1]; ++e) in_src[fill[col_idx[e]]++] = i;
    free(fill);
}

/*
 * Degree bins: node i belongs to bin b = the number of cut values c with
 * outdeg_i > c (cuts ascending).  bin_ptr[nb+1] delimits, in bin_ids[n], each
 * bin's node list in ascending id.
 */
void orc_bins(i32 n, const i32 *row_ptr, i32 ncut, const i32 *cuts, i32 *bin_of, i32 *bin_ptr, i32 *bin_ids) {
    i32 nb = ncut + 1;
    for (i32 b = 0; b <= nb; ++b) bin_ptr[b] = 0;
    for (i32 i = 0; i < n; ++i) {
        i32 deg = row_ptr[i + 1] - row_ptr[i], b = 0;
        for (i32 c = 0; c < ncut; ++c) if (deg > cuts[c]) b = c + 1;
        bin_of[i] = b;
        bin_ptr[b + 1] += 1;
    }
    for (i32 b = 0; b < nb; ++b) bin_ptr[b + 1] += bin_ptr[b];
    i32 pos[64];
    for (i32 b = 0; b < nb && b < 64; ++b) pos[b] = bin_ptr[b];
    for (i32 i = 0; i < n; ++i) bin_ids[pos[bin_of[i]]++] = i;
}

/* ------------------------------------------------------ random sequence I */

/* SplitMix64 (Steele, Lea & Flood 2014), used here only for ALGO-RAND picks */
static u64 orc_splitmix(u64 z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------ D-iteration */

enum { ORC_PER = 0, ORC_RAND = 1, ORC_MAX = 2, ORC_THRESH = 3, ORC_SWEEP = 4 };

typedef struct {
    double R;          /* the residual R of ALGO-REF at exit */
    double l1F;        /* |F|_1 recomputed by a plain sum at exit */
    i64 pushes;        /* diffusions that moved non-zero fluid */
    i64 edges;         /* elementary steps: out-links used by those diffusions */
    i64 picks;         /* entries of the sequence I drawn, zero-fluid ones included */
    i64 sweeps;        /* threshold sweeps (THRESH / SWEEP orders) */
    i32 converged;     /* 1 if R/(1-d) <= tol at exit */
} orc_stats;

/* Initialization of ALGO-REF: H = 0, F = (1-d)V, R = 1-d (V is normalized). */
double orc_init(i32 n, double d, const double *V, double *F, double *H) {
    for (i32 i = 0; i < n; ++i) { H[i] = 0.0; F[i] = (1.0 - d) * V[i]; }
    return 1.0 - d;
}

/*
 * One diffusion of node i (the loop body of ALGO-REF with the dangling-node
 * condition of Section 3.3):
 *   sent := F[i]; H[i] += sent; F[i] := 0;
 *   no child:  R -= |sent|
 *   otherwise: F[j] += sent * p(j,i) * d for every child j;  R -= |sent|*(1-d)
 * p(j,i) = 1/outdeg(i) per listed out-link.  The fluid is non-negative except
 * after a graph update, whose injected fluid d(P'-P)H may hold negative terms
 * (Section 3.2, "Updating equation"); the diffusion is linear, so signed fluid
 * moves the same way, and since |F_j + x| <= |F_j| + |x| the decrement by |sent|
 * keeps R an upper bound on |F|_1.
 */
static void diffuse(i32 i, const i32 *row_ptr, const i32 *col_idx, double d, double *F, double *H,
                    double *R, orc_stats *st) {
    double sent = F[i];
    H[i] += sent;
    F[i] = 0.0;
    i32 beg = row_ptr[i], end = row_ptr[i + 1];
    if (end == beg) {
        *R -= fabs(sent);
    } else {
        double p = 1.0 / (double)(end - beg);
        for (i32 e = beg; e < end; ++e) F[col_idx[e]] += sent * p * d;
        *R -= fabs(sent) * (1.0 - d);
    }
    st->pushes += 1;
    st->edges += end - beg;
}

/* plain sum of |F_i|: the L1 norm that R stands for (Theorem 2) */
static double l1_norm(i32 n, const double *F) {
    double s = 0.0;
    for (i32 i = 0; i < n; ++i) s += fabs(F[i]);
    return s;
}

/*
 * Selection weights (Section 4.3, ALGO-OP and ALGO-OP2).  ALGO-OP replaces the
 * argmax of F by the argmax of F_i / ((#in_i + 1)(#out_i + 1)) and ALGO-OP2 by
 * the argmax of F_i / (#out_i + 1); wsel[i] holds 1/((#in_i+1)(#out_i+1)) or
 * 1/(#out_i+1), or wsel is NULL for the plain choice.  The argmax compares
 * |F_i| * wsel[i] in FP64.  A threshold sweep with weights selects i when
 * (float)|F_i| * wsel[i] > (float)(T * wscale), the product and the compare
 * made in FP32 (a selection rule only decides which diffusions happen, and any
 * choice converges, Section 2.2); wscale is the power of two nearest below the
 * mean weight, which keeps the weighted threshold on the scale of F * w.
 * With weights the threshold is only ever lowered (the paper: the threshold is
 * scaled down progressively): after a sweep that diffused something,
 * T = min(T, beta R / N); after an empty one, T / 2.  Raising it again after the
 * halvings (the plain rule) would oscillate when the weights span many orders.
 */
static double pick_key(const double *F, const float *wsel, i32 i) {
    return wsel ? fabs(F[i]) * (double)wsel[i] : fabs(F[i]);
}

static int above(double f, const float *wsel, i32 i, double T, double wscale) {
    if (!wsel) return fabs(f) > T;
    float a = (float)fabs(f) * wsel[i];
    float t = (float)(T * wscale);
    return a > t;
}

/*
 * Run D-iteration on the state (F, H, R) until R/(1-d) <= tol or max_pushes
 * diffusions have been made.  F and H are updated in place, so a second call
 * resumes where the first stopped.  Orders of the sequence I (Section 4):
 *
 *   ORC_PER    i_n = n mod N.
 *   ORC_RAND   i_n uniform on {0..N-1} (SplitMix64 of seed + n).
 *   ORC_MAX    i_n = argmax |F| (lowest index on ties).
 *   ORC_THRESH threshold sweeps: visit i = 0..N-1 and diffuse every i whose
 *              current |F_i| > T (F_i read at its turn, Gauss-Seidel style).
 *   ORC_SWEEP  threshold sweeps on a snapshot: S = {i : |F_i| > T} is fixed at
 *              the start of the sweep, all of S hands its fluid to H, then all
 *              of S pushes.  This is the diffusion of the set S at once,
 *              F' = (I - J_S + dPJ_S)F, H' = H + J_S F with J_S = sum_{i in S} J_i,
 *              for which Theorem 1 holds by the same induction.
 *
 * Threshold schedule (the paper only says the threshold is scaled down
 * progressively): T = beta * R / N before each sweep; a sweep that diffuses
 * nothing halves T for the next one.  With beta < 1 the largest entry
 * (>= |F|/N) always qualifies, which is the condition under which the Lemma of
 * Section 3.1 gives the contraction factor 1 - (1-d)/N.
 *
 * The residual R.  ALGO-REF keeps R by decrement; in exact arithmetic R equals
 * |F|_1 at every step (F only loses what R loses), and Theorem 2 is stated for
 * |F|_1.  In floating point the decrement drifts by rounding, which at tight
 * targets can hold R above the target after F has in fact met it.  The oracle
 * therefore keeps the decrement of ALGO-REF between re-synchronisations with
 * the plain sum of F: at the start of every sweep (THRESH, SWEEP), after every
 * N picks (PER, RAND, MAX), and before it accepts a stop.  A run cut short by
 * max_pushes reports the decremented R as it stands.
 *
 * Zero-fluid picks of PER / RAND are skipped without counting (Section 4.2).
 * The sequential orders test the stop rule after every diffusion, like the
 * while-loop of ALGO-REF; ORC_SWEEP tests it between sweeps.
 * ORC_SWEEP can record (T, R at the sweep start, nodes selected) per sweep in
 * trace[3 * trace_cap] (NULL: no record).
 * Returns 0 if converged, 1 if max_pushes was reached first.
 */
int orc_diter(i32 n, const i32 *row_ptr, const i32 *col_idx, double d, double *F, double *H, double R,
              double tol, int mode, double beta, u64 seed, i64 max_pushes, const float *wsel, double wscale,
              double *trace, i64 trace_cap, orc_stats *st) {
    memset(st, 0, sizeof(*st));
    if (mode < ORC_PER || mode > ORC_SWEEP) return -1;
    const int sweeping = (mode == ORC_THRESH || mode == ORC_SWEEP);
    i64 zero_run = 0;
    double T = beta * R / (double)n;
    int first = 1, last_empty = 0;
    i32 *S = NULL;
    double *sent = NULL;
    if (mode == ORC_SWEEP) {
        S = (i32 *)malloc(sizeof(i32) * (size_t)n);
        sent = (double *)malloc(sizeof(double) * (size_t)n);
    }
    for (;;) {
        if (st->pushes >= max_pushes) break;
        if (sweeping) {
            if (!first) {
                R = l1_norm(n, F);
                if (last_empty) T = T / 2.0;
                else if (wsel) T = fmin(T, beta * R / (double)n);   /* weighted: never raised */
                else T = beta * R / (double)n;
            }
            first = 0;
        }
        if (!isfinite(R)) break;             /* F overflowed: report, never loop */
        if (R / (1.0 - d) <= tol) {
            R = l1_norm(n, F);               /* accept a stop only on the exact norm */
            if (R / (1.0 - d) <= tol) break;
            if (sweeping) T = beta * R / (double)n;
        }
        if (mode == ORC_PER || mode == ORC_RAND || mode == ORC_MAX) {
            i32 i;
            if (mode == ORC_MAX) {
                i = 0;
                for (i32 k = 1; k < n; ++k) if (pick_key(F, wsel, k) > pick_key(F, wsel, i)) i = k;
            } else {
                i = (mode == ORC_PER) ? (i32)(st->picks % n) : (i32)(orc_splitmix(seed + (u64)st->picks) % (u64)n);
            }
            st->picks += 1;
            if (st->picks % n == 0) R = l1_norm(n, F);
            if (F[i] == 0.0) {
                /* every entry zero: nothing is left to diffuse */
                if (mode == ORC_MAX || ++zero_run > 64 * (i64)n) { R = l1_norm(n, F); break; }
                continue;
            }
            zero_run = 0;
            diffuse(i, row_ptr, col_idx, d, F, H, &R, st);
        } else if (mode == ORC_THRESH) {
            i64 before = st->pushes;
            for (i32 i = 0; i < n; ++i) {
                if (above(F[i], wsel, i, T, wscale)) {
                    st->picks += 1;
                    diffuse(i, row_ptr, col_idx, d, F, H, &R, st);
                    if (R / (1.0 - d) <= tol || st->pushes >= max_pushes) break;
                }
            }
            st->sweeps += 1;
            last_empty = (st->pushes == before);
            if (last_empty && T == 0.0) break;   /* F is identically zero */
        } else {
            i32 ns = 0;
            for (i32 i = 0; i < n; ++i) if (above(F[i], wsel, i, T, wscale)) S[ns++] = i;
            if (trace && st->sweeps < trace_cap) {    /* (T, R at the sweep start, nodes selected) */
                trace[3 * st->sweeps] = T;
                trace[3 * st->sweeps + 1] = R;
                trace[3 * st->sweeps + 2] = (double)ns;
            }
            for (i32 k = 0; k < ns; ++k) {
                i32 i = S[k];
                sent[k] = F[i];
                H[i] += sent[k];
                F[i] = 0.0;
            }
            for (i32 k = 0; k < ns; ++k) {
                i32 i = S[k];
                i32 beg = row_ptr[i], end = row_ptr[i + 1];
                if (end == beg) {
                    R -= fabs(sent[k]);
                } else {
                    double p = 1.0 / (double)(end - beg);
                    for (i32 e = beg; e < end; ++e) F[col_idx[e]] += sent[k] * p * d;
                    R -= fabs(sent[k]) * (1.0 - d);
                }
                st->edges += end - beg;
            }
            st->pushes += ns;
            st->picks += ns;
            st->sweeps += 1;
            last_empty = (ns == 0);
            if (last_empty && T == 0.0) break;
        }
    }
    free(S); free(sent);
    st->R = R;
    st->l1F = l1_norm(n, F);
    st->converged = (st->l1F / (1.0 - d) <= tol) ? 1 : 0;
    return st->converged ? 0 : 1;
}

/* ---------------------------------------------------------- graph update */

/*
 * The updating equation (Section 3.2).  A run on P stopped at (F_n0, H_n0);
 * the graph becomes P'.  Continuing with P' from the fluid
 *   F_0' = F_n0 + d(P' - P) H_n0
 * and the history H_n0 reaches H_n0 + H'_inf, the solution of X = dP'X + F_0
 * (the theorem after the updating equation).  This writes F_0' into F:
 * every node i takes back d*H_i/#out_i from each child under P and hands it to
 * each child under P' (a dangling node passes nothing in either graph).
 */
void orc_update_inject(i32 n, const i32 *rp_old, const i32 *ci_old, const i32 *rp_new, const i32 *ci_new,
                       double d, const double *H, double *F) {
    for (i32 i = 0; i < n; ++i) {
        i32 beg = rp_old[i], end = rp_old[i + 1];
        if (end == beg) continue;
        double p = 1.0 / (double)(end - beg);
        for (i32 e = beg; e < end; ++e) F[ci_old[e]] -= H[i] * p * d;
    }
    for (i32 i = 0; i < n; ++i) {
        i32 beg = rp_new[i], end = rp_new[i + 1];
        if (end == beg) continue;
        double p = 1.0 / (double)(end - beg);
        for (i32 e = beg; e < end; ++e) F[ci_new[e]] += H[i] * p * d;
    }
}

/* ------------------------------------------------------ power iteration */

/*
 * MAT-ITER on the uncompleted P (Section 4, with the stop rule of Section 4):
 *   X_0 = 0,  X_{n+1} = dPX_n + (1-d)V,
 *   stop when |X_{n+1} - X_n|_1 * d/(1-d) < tol  or after max_iter products.
 * From X_0 = 0 the iterate X_n equals the partial series S_{n-1} of
 * Section 2.2.  Each product uses every listed out-link once (L elementary
 * steps).  Returns 0 if the stop rule was met.
 */
int orc_power(i32 n, const i32 *row_ptr, const i32 *col_idx, double d, const double *V, double tol,
              i64 max_iter, double *X, i64 *iters, double *last_delta) {
    double *Y = (double *)malloc(sizeof(double) * (size_t)n);
    for (i32 i = 0; i < n; ++i) X[i] = 0.0;
    i64 it = 0;
    double delta = INFINITY;
    int ok = 0;
    while (it < max_iter) {
        for (i32 j = 0; j < n; ++j) Y[j] = (1.0 - d) * V[j];
        for (i32 i = 0; i < n; ++i) {
            i32 beg = row_ptr[i], end = row_ptr[i + 1];
            if (end == beg) continue;
            double p = 1.0 / (double)(end - beg);
            for (i32 e = beg; e < end; ++e) Y[col_idx[e]] += d * p * X[i];
        }
        delta = 0.0;
        for (i32 j = 0; j < n; ++j) { delta += fabs(Y[j] - X[j]); X[j] = Y[j]; }
        ++it;
        if (delta * d / (1.0 - d) < tol) { ok = 1; break; }
    }
    free(Y);
    *iters = it;
    *last_delta = delta;
    return ok ? 0 : 1;
}
