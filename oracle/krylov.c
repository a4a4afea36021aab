/*
 * Preconditioner and Krylov solver of the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * Sec. 3: the mixed-stage systems are non-symmetric, so they are solved with
 * GMRES (Saad & Schultz), left-preconditioned with one fixed incomplete LU
 * factorisation of the operator assembled at still water, eta = 0 (the value
 * "eta = 1" printed in Sec. 5 is read as a slip for the still-water state of
 * Sec. 3 and Sec. 5.2).  The variant is ILU(0): no fill outside the sparsity
 * pattern of the still-water matrix, no pivoting, in a given unknown ordering.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "internal.h"

/* ---------- ILU(0), IKJ form (Saad, Iterative Methods, Alg. 10.4) ---------- */

int or_build_ilu(or_problem *P, const int *order)
{
    int n = P->m;
    or_csr *A0 = &P->A0;
    free(P->order); free(P->rank); free(P->diag);
    or_csr_free(&P->LU);
    P->order = malloc(n * sizeof(int));
    P->rank = malloc(n * sizeof(int));
    P->diag = malloc(n * sizeof(int));
    for (int i = 0; i < n; ++i) P->order[i] = order ? order[i] : i;
    for (int i = 0; i < n; ++i) P->rank[P->order[i]] = i;
    /* B = A0 with rows and columns renumbered: B[i][j] = A0[order[i]][order[j]] */
    int nnz = A0->rowptr[n];
    or_csr *B = &P->LU;
    B->n = n;
    B->rowptr = malloc((n + 1) * sizeof(int));
    B->col = malloc(nnz * sizeof(int));
    B->val = malloc(nnz * sizeof(double));
    B->rowptr[0] = 0;
    for (int i = 0; i < n; ++i) {
        int r = P->order[i];
        int q0 = B->rowptr[i], len = A0->rowptr[r + 1] - A0->rowptr[r];
        /* insertion sort of the renumbered columns */
        for (int q = 0; q < len; ++q) {
            int cj = P->rank[A0->col[A0->rowptr[r] + q]];
            double v = A0->val[A0->rowptr[r] + q];
            int t = q0 + q;
            while (t > q0 && B->col[t - 1] > cj) { B->col[t] = B->col[t - 1]; B->val[t] = B->val[t - 1]; --t; }
            B->col[t] = cj; B->val[t] = v;
        }
        B->rowptr[i + 1] = q0 + len;
    }
    /* factorisation in place */
    int *pos = malloc(n * sizeof(int));
    for (int j = 0; j < n; ++j) pos[j] = -1;
    int status = OR_OK;
    for (int i = 0; i < n && status == OR_OK; ++i) {
        for (int q = B->rowptr[i]; q < B->rowptr[i + 1]; ++q) pos[B->col[q]] = q;
        P->diag[i] = pos[i];
        if (pos[i] < 0) status = OR_SINGULAR;
        for (int q = B->rowptr[i]; q < B->rowptr[i + 1] && status == OR_OK; ++q) {
            int k = B->col[q];
            if (k >= i) break;
            double ukk = B->val[P->diag[k]];
            if (ukk == 0.0) { status = OR_SINGULAR; break; }
            B->val[q] /= ukk;                     /* l_ik */
            double lik = B->val[q];
            for (int r = P->diag[k] + 1; r < B->rowptr[k + 1]; ++r) {
                int jj = B->col[r];               /* jj > k */
                if (pos[jj] >= 0) B->val[pos[jj]] -= lik * B->val[r];
            }
        }
        for (int q = B->rowptr[i]; q < B->rowptr[i + 1]; ++q) pos[B->col[q]] = -1;
        if (status == OR_OK && B->val[P->diag[i]] == 0.0) status = OR_SINGULAR;
    }
    free(pos);
    return status;
}

int or_ilu_nnz(const or_problem *P) { return P->LU.rowptr[P->LU.n]; }

void or_export_ilu(const or_problem *P, int *rowptr, int *col, double *val)
{
    int nnz = P->LU.rowptr[P->LU.n];
    memcpy(rowptr, P->LU.rowptr, (P->LU.n + 1) * sizeof(int));
    memcpy(col, P->LU.col, nnz * sizeof(int));
    memcpy(val, P->LU.val, nnz * sizeof(double));
}

/* out = U^-1 L^-1 v (v and out in natural numbering). */
void or_ilu_apply(const or_problem *P, const double *v, double *out)
{
    int n = P->m;
    const or_csr *B = &P->LU;
    double *y = malloc(n * sizeof(double));
    for (int i = 0; i < n; ++i) y[i] = v[P->order[i]];
    for (int i = 0; i < n; ++i) {                 /* forward, unit lower L */
        double s = y[i];
        for (int q = B->rowptr[i]; q < P->diag[i]; ++q) s -= B->val[q] * y[B->col[q]];
        y[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {            /* backward, U */
        double s = y[i];
        for (int q = P->diag[i] + 1; q < B->rowptr[i + 1]; ++q) s -= B->val[q] * y[B->col[q]];
        y[i] = s / B->val[P->diag[i]];
    }
    for (int i = 0; i < n; ++i) out[P->order[i]] = y[i];
    free(y);
}

/* ---------- left-preconditioned restarted GMRES(m) ---------- */

static double dot(int n, const double *a, const double *b)
{
    double s = 0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* r = M^-1 (b - A x) */
static void precond_residual(const or_problem *P, const double *b, const double *x, double *t, double *r)
{
    or_matvec(P, x, t);
    for (int i = 0; i < P->m; ++i) t[i] = b[i] - t[i];
    or_ilu_apply(P, t, r);
}

int or_gmres_trace(or_problem *P, const double *b, double *x, or_stats *st, double *trace, int trace_len)
{
    int n = P->m, mr = P->p.restart;
    double tol = P->p.tol;
    double *V = malloc((size_t)(mr + 1) * n * sizeof(double));
    double *w = malloc(n * sizeof(double));
    double *t = malloc(n * sizeof(double));
    double *H = calloc((size_t)(mr + 1) * mr, sizeof(double));   /* H[i*mr + j] */
    double *cs = malloc(mr * sizeof(double)), *sn = malloc(mr * sizeof(double));
    double *gv = malloc((mr + 1) * sizeof(double)), *yv = malloc(mr * sizeof(double));
    double hcol[512];
    memset(st, 0, sizeof(*st));
    /* reference norms */
    or_ilu_apply(P, b, t);
    double bnorm = sqrt(dot(n, t, t));
    double braw = sqrt(dot(n, b, b));
    or_matvec(P, x, t);
    double g0 = 0;
    for (int i = 0; i < n; ++i) g0 += (b[i] - t[i]) * (b[i] - t[i]);
    st->guess_res = braw > 0 ? sqrt(g0) / braw : sqrt(g0);
    int status = OR_NOT_CONVERGED;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        st->converged = 1; status = OR_OK;
        goto done;
    }
    for (int cycle = 0; cycle <= P->p.max_restarts + 1; ++cycle) {
        precond_residual(P, b, x, t, V);
        double beta = sqrt(dot(n, V, V));
        if (cycle == 0) st->res0 = beta / bnorm;
        st->res_final = beta / bnorm;
        if (!(beta == beta)) { status = OR_NAN; break; }
        if (beta <= tol * bnorm) { st->converged = 1; status = OR_OK; break; }
        if (cycle == P->p.max_restarts + 1) break;
        if (cycle > 0) st->restarts++;
        for (int i = 0; i < n; ++i) V[i] /= beta;
        for (int i = 0; i <= mr; ++i) gv[i] = 0;
        gv[0] = beta;
        int jend = 0;
        for (int j = 0; j < mr; ++j) {
            double *vj = V + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            or_matvec(P, vj, t);
            or_ilu_apply(P, t, w);
            /* classical Gram-Schmidt, applied twice */
            for (int i = 0; i <= j; ++i) H[i * mr + j] = 0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = 0; i <= j; ++i) hcol[i] = dot(n, V + (size_t)i * n, w);
                for (int i = 0; i <= j; ++i) {
                    const double *vi = V + (size_t)i * n;
                    for (int q = 0; q < n; ++q) w[q] -= hcol[i] * vi[q];
                    H[i * mr + j] += hcol[i];
                }
            }
            double hn = sqrt(dot(n, w, w));
            H[(j + 1) * mr + j] = hn;
            int breakdown = hn == 0.0;
            if (!breakdown) for (int q = 0; q < n; ++q) vn[q] = w[q] / hn;
            /* previous rotations on the new column */
            for (int i = 0; i < j; ++i) {
                double a = H[i * mr + j], bb = H[(i + 1) * mr + j];
                H[i * mr + j] = cs[i] * a + sn[i] * bb;
                H[(i + 1) * mr + j] = -sn[i] * a + cs[i] * bb;
            }
            /* new rotation zeroing H[j+1][j] */
            double a = H[j * mr + j], bb = H[(j + 1) * mr + j];
            double den = hypot(a, bb);
            cs[j] = a / den; sn[j] = bb / den;
            H[j * mr + j] = den; H[(j + 1) * mr + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            st->iterations++;
            if (trace && st->iterations <= trace_len) trace[st->iterations - 1] = fabs(gv[j + 1]) / bnorm;
            jend = j + 1;
            if (fabs(gv[j + 1]) <= tol * bnorm || breakdown) break;
        }
        /* back substitution R y = g and update x += V y */
        for (int i = jend - 1; i >= 0; --i) {
            double s = gv[i];
            for (int l = i + 1; l < jend; ++l) s -= H[i * mr + l] * yv[l];
            yv[i] = s / H[i * mr + i];
        }
        for (int i = 0; i < jend; ++i) {
            const double *vi = V + (size_t)i * n;
            for (int q = 0; q < n; ++q) x[q] += yv[i] * vi[q];
        }
    }
done:
    or_matvec(P, x, t);
    {
        double s = 0;
        for (int i = 0; i < n; ++i) s += (b[i] - t[i]) * (b[i] - t[i]);
        st->true_res = braw > 0 ? sqrt(s) / braw : sqrt(s);
    }
    free(V); free(w); free(t); free(H); free(cs); free(sn); free(gv); free(yv);
    return status;
}

int or_gmres(or_problem *P, const double *b, double *x, or_stats *st)
{
    return or_gmres_trace(P, b, x, st, NULL, 0);
}
