/*
 * Subspace acceleration of the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Algorithm 2: pick a basis V of a subspace of span of past solutions, solve
 *   z* = argmin_z || A V z - b ||_2   (by a QR factorisation, Sec. 4),
 * and start the iterative solver from x0 = V z*.
 * Algorithm 4 (EWMA): V = Y with Y = sum over past solutions of
 *   r^(age) x omega^T, updated after every solve as Y <- r Y + x omega^T
 *   (the rank-1 form printed below Algorithm 4).  omega ~ N(0, I_k).
 * The age is counted in solves (one decay factor r per solve); see the
 * reading recorded with the decay parameter.
 * Algorithm 3 (randomized range finder): Y = X Omega with X the K newest
 * solutions and a fresh Gaussian Omega (K x k) for every solve.
 * Both sketches are used as V = Y, or, with the parameter orthonormalize, as
 * V = Q from the QR factorisation Y = Q R (the optional step of both
 * algorithms): the same span, so the same x0 in exact arithmetic, but a
 * well-conditioned basis when the columns of Y are nearly dependent.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "internal.h"

/* SplitMix64 (Steele, Lea & Flood 2014): i-th output (i >= 1) of the stream with
 * the given seed is the finaliser applied to seed + i * golden-gamma. */
uint64_t or_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + i * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* omega_c for solve s: Box-Muller on outputs 2(s k + c) + 1 and 2(s k + c) + 2. */
void or_draw_omega(uint64_t seed, long solve_index, int k, double *omega)
{
    const double two53 = 1.0 / 9007199254740992.0;
    const double two_pi = 6.283185307179586476925286766559;
    for (int c = 0; c < k; ++c) {
        uint64_t i1 = 2 * ((uint64_t)solve_index * (uint64_t)k + (uint64_t)c) + 1;
        double u1 = ((double)(or_splitmix64(seed, i1) >> 11) + 1.0) * two53;   /* (0, 1] */
        double u2 = (double)(or_splitmix64(seed, i1 + 1) >> 11) * two53;       /* [0, 1) */
        double rr = sqrt(-2.0 * log(u1));
        double th = two_pi * u2;
        omega[c] = rr * cos(th);
    }
}

/* Householder QR of W (m x k, column-major), then z = R^-1 (Q^T b)[0:k].
 * Columns whose |R_jj| falls below 1e-12 |R_00| are treated as dependent
 * and get z_j = 0.  Returns the numerical rank. */
int or_lstsq_qr(int m, int k, const double *W, const double *b, double *z)
{
    double *R = malloc((size_t)m * k * sizeof(double));
    double *qb = malloc(m * sizeof(double));
    double *v = malloc(m * sizeof(double));
    double *diag = malloc(k * sizeof(double));
    memcpy(R, W, (size_t)m * k * sizeof(double));
    memcpy(qb, b, m * sizeof(double));
    for (int j = 0; j < k && j < m; ++j) {
        double *cj = R + (size_t)j * m;
        double nx = 0;
        for (int i = j; i < m; ++i) nx += cj[i] * cj[i];
        nx = sqrt(nx);
        if (nx == 0.0) { diag[j] = 0.0; continue; }
        double alpha = cj[j] > 0 ? -nx : nx;
        for (int i = j; i < m; ++i) v[i] = cj[i];
        v[j] -= alpha;
        double vn = 0;
        for (int i = j; i < m; ++i) vn += v[i] * v[i];
        diag[j] = alpha;
        if (vn == 0.0) continue;
        /* H = I - 2 v v^T / (v^T v) on the remaining columns and on b */
        for (int l = j; l < k; ++l) {
            double *cl = R + (size_t)l * m;
            double s = 0;
            for (int i = j; i < m; ++i) s += v[i] * cl[i];
            s = 2.0 * s / vn;
            for (int i = j; i < m; ++i) cl[i] -= s * v[i];
        }
        double s = 0;
        for (int i = j; i < m; ++i) s += v[i] * qb[i];
        s = 2.0 * s / vn;
        for (int i = j; i < m; ++i) qb[i] -= s * v[i];
    }
    int rank = 0;
    double r00 = k > 0 ? fabs(diag[0]) : 0.0;
    for (int j = k - 1; j >= 0; --j) {
        double rjj = R[(size_t)j * m + j];
        if (!(fabs(rjj) > 1e-12 * r00) ) { z[j] = 0.0; continue; }
        double s = qb[j];
        for (int l = j + 1; l < k; ++l) s -= R[(size_t)l * m + j] * z[l];
        z[j] = s / rjj;
        rank++;
    }
    free(R); free(qb); free(v); free(diag);
    return rank;
}

int or_orth_basis(int m, int k, const double *Y, double *Q)
{
    double ymax = 0.0;
    for (int c = 0; c < k; ++c) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += Y[(size_t)c * m + i] * Y[(size_t)c * m + i];
        if (sqrt(s) > ymax) ymax = sqrt(s);
    }
    int r = 0;
    for (int c = 0; c < k; ++c) {
        double *q = Q + (size_t)r * m;
        memcpy(q, Y + (size_t)c * m, m * sizeof(double));
        for (int pass = 0; pass < 2; ++pass) {          /* q <- q - Q_r (Q_r^T q), twice */
            double proj[64];
            for (int l = 0; l < r; ++l) {
                double s = 0.0;
                for (int i = 0; i < m; ++i) s += Q[(size_t)l * m + i] * q[i];
                proj[l] = s;
            }
            for (int l = 0; l < r; ++l)
                for (int i = 0; i < m; ++i) q[i] -= proj[l] * Q[(size_t)l * m + i];
        }
        double nq = 0.0;
        for (int i = 0; i < m; ++i) nq += q[i] * q[i];
        nq = sqrt(nq);
        if (!(nq > 1e-12 * ymax)) continue;             /* dependent on the kept columns */
        for (int i = 0; i < m; ++i) q[i] /= nq;
        r++;
    }
    return r;
}

/* Algorithm 2 on a basis V (m x kv): z* = argmin ||A V z - b||, x0 = V z*. */
static int guess_from_basis(or_problem *P, const double *V, int kv, const double *b, double *x0)
{
    int m = P->m;
    double *W = malloc((size_t)m * (kv > 0 ? kv : 1) * sizeof(double));
    double z[64];
    for (int c = 0; c < kv; ++c) or_matvec(P, V + (size_t)c * m, W + (size_t)c * m);
    int rank = kv > 0 ? or_lstsq_qr(m, kv, W, b, z) : 0;
    for (int i = 0; i < m; ++i) {
        double s = 0;
        for (int c = 0; c < kv; ++c) s += V[(size_t)c * m + i] * z[c];
        x0[i] = s;
    }
    free(W);
    return rank;
}

/* V = Y, or V = Q of Y = Q R when the problem asks for the orthonormalisation. */
static int guess_from_sketch(or_problem *P, const double *Y, int kc, const double *b, double *x0)
{
    if (!P->p.orthonormalize) return guess_from_basis(P, Y, kc, b, x0);
    double *Q = malloc((size_t)P->m * (kc > 0 ? kc : 1) * sizeof(double));
    int r = or_orth_basis(P->m, kc, Y, Q);
    int rank = guess_from_basis(P, Q, r, b, x0);
    free(Q);
    return rank;
}

int or_ewma_guess(or_problem *P, const double *b, double *x0)
{
    return guess_from_sketch(P, P->Y, P->p.k, b, x0);
}

void or_ewma_update(or_problem *P, const double *x, long solve_index)
{
    int m = P->m, k = P->p.k;
    double om[64];
    or_draw_omega(P->p.seed, solve_index, k, om);
    for (int c = 0; c < k; ++c) {
        double *yc = P->Y + (size_t)c * m;
        for (int i = 0; i < m; ++i) yc[i] = P->p.decay * yc[i] + x[i] * om[c];
    }
}

void or_get_sketch(const or_problem *P, double *Y)
{
    memcpy(Y, P->Y, (size_t)P->m * P->p.k * sizeof(double));
}

void or_set_sketch(or_problem *P, const double *Y)
{
    memcpy(P->Y, Y, (size_t)P->m * P->p.k * sizeof(double));
}

int or_rrf_sketch(const or_problem *P, double *Y)
{
    int m = P->m, k = P->p.k, K = P->p.history;
    long s = P->n_solves;
    int Ke = s < K ? (int)s : K;
    int ke = k < Ke ? k : Ke;
    double *om = malloc((size_t)K * k * sizeof(double));
    or_draw_omega(P->p.seed, s, K * k, om);
    for (int c = 0; c < ke; ++c) {
        double *yc = Y + (size_t)c * m;
        for (int i = 0; i < m; ++i) yc[i] = 0.0;
        for (int r = 0; r < Ke; ++r) {
            const double *xr = P->X + (size_t)((s - 1 - r) % K) * m;   /* r-th newest solution */
            const double w = om[r * k + c];
            for (int i = 0; i < m; ++i) yc[i] += xr[i] * w;
        }
    }
    free(om);
    return ke;
}

int or_rrf_guess(or_problem *P, const double *b, double *x0)
{
    double *Y = malloc((size_t)P->m * P->p.k * sizeof(double));
    int ke = or_rrf_sketch(P, Y);
    int rank = guess_from_sketch(P, Y, ke, b, x0);
    free(Y);
    return rank;
}

int or_solve(or_problem *P, const double *eta_prev, const double *eta_cur, const double *b,
             double *x_out, or_stats *st)
{
    int m = P->m;
    or_assemble(P, eta_prev, eta_cur);
    long s = P->n_solves;
    int mode = P->p.guess;
    if ((mode == OR_GUESS_EWMA || mode == OR_GUESS_RRF) && (s < P->p.n_init_solves || P->p.k == 0))
        mode = OR_GUESS_PREV;
    if (mode == OR_GUESS_RRF && s == 0) mode = OR_GUESS_PREV;
    if (mode == OR_GUESS_COLD) for (int i = 0; i < m; ++i) x_out[i] = 0.0;
    else if (mode == OR_GUESS_PREV) memcpy(x_out, P->x_prev, m * sizeof(double));
    else if (mode == OR_GUESS_RRF) or_rrf_guess(P, b, x_out);
    else or_ewma_guess(P, b, x_out);
    int status = or_gmres(P, b, x_out, st);
    memcpy(P->x_prev, x_out, m * sizeof(double));
    if (P->p.guess == OR_GUESS_EWMA && P->p.k > 0) or_ewma_update(P, x_out, s);
    if (P->p.guess == OR_GUESS_RRF && P->p.history > 0)
        memcpy(P->X + (size_t)(s % P->p.history) * m, x_out, m * sizeof(double));
    P->n_solves++;
    return status;
}
