/*
 * The discrete mixed-stage Poisson operator, assembled row by row.
 * TEST INFRASTRUCTURE ONLY.
 *
 * Grid (Sec. 3, Sec. 5.1): nx x ny columns, periodic in x and y, with
 * sigma levels sigma_j = j/(nz-1), j = 0..nz-1, plus one ghost level j = -1
 * below the bed.  Node (ix, iy, j) has index ((j+1)*ny + iy)*nx + ix.
 *
 * Walls (2-D; ghost nodes of Sec. 3, the flume of Sec. 5.2): the impermeable walls at
 * x = 0 and x = lx carry the Neumann condition n . grad p = n . G through one
 * ghost column outside each wall (columns 0 and nx-1).  The row of ghost node
 * (0, j) is the wall condition n . grad^(i-1) p = n . G evaluated at the wall
 * node (1, j), for j = -1..nz-2 (at j = -1 the condition is continued to the
 * ghost level below the bed, which closes the corner); the surface node of a
 * ghost column is a Dirichlet row like every surface node.  Next to a wall the
 * 7-point x stencils are shifted inside [0, nx-1] (off-centred, as next to bed
 * and surface in sigma).
 *
 * Rows (Eq. 16-18):
 *   j = nz-1  free surface, homogeneous Dirichlet p = 0: the row is the identity;
 *   0 <= j <= nz-2  the mixed-stage operator grad^(i) . grad^(i-1) p, with the
 *             push-forward of Eq. (9b) and the sigma derivatives of Eq. (13b-13d);
 *   j = -1    ghost row: the Neumann condition n . grad^(i-1) p of Eq. (17),
 *             evaluated at the bed node, so that the PDE and the boundary
 *             condition both hold at the bed (Sec. 3, ghost-node treatment).
 *
 * Expansion used for the interior rows.  Write a = sigma_x^(i-1),
 * b = sigma_x^(i), a' = sigma_y^(i-1), b' = sigma_y^(i), f = 1/d^(i-1),
 * e = 1/d^(i).  Applying grad^(i) . (grad^(i-1) p) with the chain rule, and
 * using that f, e do not depend on sigma, gives
 *   p_xx + p_yy + (a+b) p_xs + (a'+b') p_ys + (a b + a' b' + e f) p_ss
 *        + (a_x + b a_s + a'_y + b' a'_s) p_s,
 * where a_s = d(a)/d(sigma) = -d_x/d and a_x = d(a)/d(chi) at fixed sigma
 * = (h_xx - sigma d_xx - a d_x)/d (all at stage i-1).  Each derivative is then
 * replaced by its 7-point sixth-order formula; the mixed derivative is the
 * tensor product D_chi D_sigma.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "internal.h"

long or_index(const or_grid *g, int ix, int iy, int j)
{
    return ((long)(j + 1) * g->ny + iy) * g->nx + ix;
}

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

double or_sigma(const or_problem *P, int j) { return (double)j / (double)(P->g.nz - 1); }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int or_is_wall_ghost(const or_problem *P, int ix)
{
    return P->g.walls && (ix == 0 || ix == P->g.nx - 1);
}

double or_xcoord(const or_problem *P, int ix)
{
    return P->g.walls ? (ix - 1) * P->dx : ix * P->dx;
}

void or_xwin(const or_problem *P, int ix, int field, int *cols, const double **w1, const double **w2)
{
    int nx = P->g.nx;
    if (!P->g.walls) {
        for (int t = 0; t < OR_W; ++t) cols[t] = wrap(ix + t - OR_HALF, nx);
        *w1 = P->wx1;
        *w2 = P->wx2;
        return;
    }
    int s;
    if (field) {
        s = clampi(ix - OR_HALF, 0, nx - OR_W);
    } else {
        ix = clampi(ix, 1, nx - 2);
        s = clampi(ix - OR_HALF, 1, nx - 1 - OR_W);
    }
    for (int t = 0; t < OR_W; ++t) cols[t] = s + t;
    *w1 = P->wxo1[ix - s];
    *w2 = P->wxo2[ix - s];
}

void or_csr_free(or_csr *A)
{
    free(A->rowptr); free(A->col); free(A->val);
    A->rowptr = NULL; A->col = NULL; A->val = NULL; A->n = 0;
}

/* ---------- surface-grid and field derivatives ---------- */

void or_surface_derivs(const or_problem *P, const double *f, double *fx, double *fy,
                       double *fxx, double *fyy)
{
    const or_grid *g = &P->g;
    for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
            double s1 = 0, s2 = 0, t1 = 0, t2 = 0;
            int cols[OR_W];
            const double *w1, *w2;
            or_xwin(P, ix, 0, cols, &w1, &w2);
            for (int t = -OR_HALF; t <= OR_HALF; ++t) {
                double vx = f[iy * g->nx + cols[t + OR_HALF]];
                s1 += w1[t + OR_HALF] * vx;
                s2 += w2[t + OR_HALF] * vx;
                if (g->ny > 1) {
                    double vy = f[wrap(iy + t, g->ny) * g->nx + ix];
                    t1 += P->wy1[t + OR_HALF] * vy;
                    t2 += P->wy2[t + OR_HALF] * vy;
                }
            }
            int c = iy * g->nx + ix;
            if (fx) fx[c] = s1;
            if (fxx) fxx[c] = s2;
            if (fy) fy[c] = t1;
            if (fyy) fyy[c] = t2;
        }
}

void or_field_dx(const or_problem *P, const double *f, double *out, int field)
{
    const or_grid *g = &P->g;
    for (int j = -1; j < g->nz; ++j)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                int cols[OR_W];
                const double *w1, *w2;
                or_xwin(P, ix, field, cols, &w1, &w2);
                double s = 0;
                for (int t = 0; t < OR_W; ++t) s += w1[t] * f[or_index(g, cols[t], iy, j)];
                out[or_index(g, ix, iy, j)] = s;
            }
}

void or_field_dy(const or_problem *P, const double *f, double *out)
{
    const or_grid *g = &P->g;
    for (int j = -1; j < g->nz; ++j)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                double s = 0;
                if (g->ny > 1)
                    for (int t = -OR_HALF; t <= OR_HALF; ++t)
                        s += P->wy1[t + OR_HALF] * f[or_index(g, ix, wrap(iy + t, g->ny), j)];
                out[or_index(g, ix, iy, j)] = s;
            }
}

void or_field_dsigma(const or_problem *P, const double *f, double *out)
{
    const or_grid *g = &P->g;
    for (int j = -1; j < g->nz; ++j) {
        int s0 = P->win[j + 1];
        const double *w = P->ws1 + (j + 1) * OR_W;
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                double s = 0;
                for (int k = 0; k < OR_W; ++k) s += w[k] * f[or_index(g, ix, iy, s0 + k)];
                out[or_index(g, ix, iy, j)] = s;
            }
    }
}

/* ---------- column geometry, Eq. (13b-13d) ---------- */

void or_colgeom_alloc(const or_problem *P, or_colgeom *G)
{
    int n = P->ncol;
    G->d = calloc(n, sizeof(double)); G->dx = calloc(n, sizeof(double));
    G->dy = calloc(n, sizeof(double)); G->dxx = calloc(n, sizeof(double));
    G->dyy = calloc(n, sizeof(double));
}

void or_colgeom_free(or_colgeom *G)
{
    free(G->d); free(G->dx); free(G->dy); free(G->dxx); free(G->dyy);
}

/* d = h + eta and its surface derivatives (d_x = D_chi d etc., Sec. 3). */
void or_colgeom_eval(const or_problem *P, const double *eta, or_colgeom *G)
{
    for (int c = 0; c < P->ncol; ++c) G->d[c] = P->h[c] + (eta ? eta[c] : 0.0);
    or_surface_derivs(P, G->d, G->dx, G->dy, G->dxx, G->dyy);
}

/* ---------- row assembly ---------- */

typedef struct { int col; double val; } entry;
typedef struct { entry e[512]; int n; } rowbuf;

static void add(rowbuf *r, long col, double v)
{
    r->e[r->n].col = (int)col;
    r->e[r->n].val = v;
    r->n++;
}

static int cmp_entry(const void *a, const void *b)
{
    int ca = ((const entry *)a)->col, cb = ((const entry *)b)->col;
    return (ca > cb) - (ca < cb);
}

/* Sort by column and merge repeated columns (they occur when a stencil wraps
 * onto itself on very small periodic grids). */
static void finish_row(rowbuf *r)
{
    qsort(r->e, r->n, sizeof(entry), cmp_entry);
    int o = 0;
    for (int i = 0; i < r->n; ++i) {
        if (o > 0 && r->e[o - 1].col == r->e[i].col) r->e[o - 1].val += r->e[i].val;
        else r->e[o++] = r->e[i];
    }
    r->n = o;
}

/*
 * One row of A(eta_prev, eta_cur).  When box == 0 the sigma-cross terms and
 * the horizontal terms of the ghost row are left out of the sparsity pattern;
 * this is allowed only where their coefficients vanish (flat bed, still water).
 */
static void build_row(const or_problem *P, const or_colgeom *Gp, const or_colgeom *Gc,
                      int box, int ix, int iy, int j, rowbuf *r)
{
    const or_grid *g = &P->g;
    int c = iy * g->nx + ix;
    int three_d = g->ny > 1;
    r->n = 0;
    if (j == g->nz - 1) {                 /* free surface: p = 0 */
        add(r, or_index(g, ix, iy, j), 1.0);
        return;
    }
    int xc[OR_W];
    const double *wx1, *wx2;
    if (or_is_wall_ghost(P, ix)) {        /* wall row: n . grad^(i-1) p at the wall node (iw, j) */
        int iw = ix == 0 ? 1 : g->nx - 2;
        double nxs = ix == 0 ? -1.0 : 1.0;   /* outward normal (-1, 0) at x = 0, (1, 0) at x = lx */
        int cw = iy * g->nx + iw;
        or_xwin(P, iw, 1, xc, &wx1, &wx2);
        for (int t = 0; t < OR_W; ++t) add(r, or_index(g, xc[t], iy, j), nxs * wx1[t]);
        if (box) {
            double a = (P->hx[cw] - or_sigma(P, j) * Gp->dx[cw]) / Gp->d[cw];   /* sigma_x^(i-1) */
            int s0 = P->win[j + 1];
            const double *w1s = P->ws1 + (j + 1) * OR_W;
            for (int k = 0; k < OR_W; ++k) add(r, or_index(g, iw, iy, s0 + k), nxs * a * w1s[k]);
        }
        return;
    }
    or_xwin(P, ix, 1, xc, &wx1, &wx2);
    double hx = P->hx[c], hy = P->hy[c];
    if (j == -1) {                        /* ghost row: n . grad^(i-1) p at the bed */
        int jb = 0, s0 = P->win[jb + 1];
        const double *w1s = P->ws1 + (jb + 1) * OR_W;
        double dp = Gp->d[c];
        double f = 1.0 / dp;
        double a0 = hx / dp, a0y = hy / dp;          /* sigma_x, sigma_y at sigma = 0 */
        double nrm = 1.0 / sqrt(1.0 + hx * hx + hy * hy);
        /* outward normal at the bed z = -h is -(h_x, h_y, 1)/|.| */
        double cs = -nrm * (hx * a0 + hy * a0y + f);
        for (int k = 0; k < OR_W; ++k) add(r, or_index(g, ix, iy, s0 + k), cs * w1s[k]);
        if (box) {
            for (int t = -OR_HALF; t <= OR_HALF; ++t) {
                add(r, or_index(g, xc[t + OR_HALF], iy, jb), -nrm * hx * wx1[t + OR_HALF]);
                if (three_d)
                    add(r, or_index(g, ix, wrap(iy + t, g->ny), jb), -nrm * hy * P->wy1[t + OR_HALF]);
            }
        }
        return;
    }
    /* interior row, Eq. (16) left-hand side */
    double sg = or_sigma(P, j);
    int s0 = P->win[j + 1];
    const double *w1s = P->ws1 + (j + 1) * OR_W;
    const double *w2s = P->ws2 + (j + 1) * OR_W;
    double dp = Gp->d[c], dc = Gc->d[c];
    double f = 1.0 / dp, e = 1.0 / dc;
    double a = (hx - sg * Gp->dx[c]) / dp;               /* sigma_x at stage i-1 */
    double b = (hx - sg * Gc->dx[c]) / dc;               /* sigma_x at stage i   */
    double as = -Gp->dx[c] / dp;                         /* d a / d sigma */
    double ax = (P->hxx[c] - sg * Gp->dxx[c] - a * Gp->dx[c]) / dp;  /* d a / d chi */
    double ay_ = 0, by_ = 0, ays = 0, ayy = 0;
    if (three_d) {
        ay_ = (hy - sg * Gp->dy[c]) / dp;
        by_ = (hy - sg * Gc->dy[c]) / dc;
        ays = -Gp->dy[c] / dp;
        ayy = (P->hyy[c] - sg * Gp->dyy[c] - ay_ * Gp->dy[c]) / dp;
    }
    double c_ss = a * b + ay_ * by_ + e * f;
    double c_s = ax + b * as + ayy + by_ * ays;
    double c_xs = a + b, c_ys = ay_ + by_;
    for (int t = -OR_HALF; t <= OR_HALF; ++t) {
        add(r, or_index(g, xc[t + OR_HALF], iy, j), wx2[t + OR_HALF]);
        if (three_d) add(r, or_index(g, ix, wrap(iy + t, g->ny), j), P->wy2[t + OR_HALF]);
    }
    for (int k = 0; k < OR_W; ++k)
        add(r, or_index(g, ix, iy, s0 + k), c_ss * w2s[k] + c_s * w1s[k]);
    if (box) {
        for (int t = -OR_HALF; t <= OR_HALF; ++t)
            for (int k = 0; k < OR_W; ++k) {
                add(r, or_index(g, xc[t + OR_HALF], iy, s0 + k),
                    c_xs * wx1[t + OR_HALF] * w1s[k]);
                if (three_d)
                    add(r, or_index(g, ix, wrap(iy + t, g->ny), s0 + k),
                        c_ys * P->wy1[t + OR_HALF] * w1s[k]);
            }
    }
}

static int assemble_into(const or_problem *P, const or_colgeom *Gp, const or_colgeom *Gc,
                         int box, or_csr *A)
{
    const or_grid *g = &P->g;
    or_csr_free(A);
    int m = P->m;
    int cap = m * (box ? (g->ny > 1 ? 100 : 56) : (g->ny > 1 ? 20 : 14));
    A->n = m;
    A->rowptr = malloc((m + 1) * sizeof(int));
    A->col = malloc((size_t)cap * sizeof(int));
    A->val = malloc((size_t)cap * sizeof(double));
    rowbuf *r = malloc(sizeof(rowbuf));
    int nnz = 0;
    A->rowptr[0] = 0;
    for (int j = -1; j < g->nz; ++j)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                build_row(P, Gp, Gc, box, ix, iy, j, r);
                finish_row(r);
                for (int q = 0; q < r->n; ++q) {
                    A->col[nnz] = r->e[q].col;
                    A->val[nnz] = r->e[q].val;
                    nnz++;
                }
                A->rowptr[or_index(g, ix, iy, j) + 1] = nnz;
            }
    free(r);
    return nnz;
}

int or_assemble(or_problem *P, const double *eta_prev, const double *eta_cur)
{
    or_colgeom Gp, Gc;
    or_colgeom_alloc(P, &Gp); or_colgeom_alloc(P, &Gc);
    or_colgeom_eval(P, eta_prev, &Gp);
    or_colgeom_eval(P, eta_cur, &Gc);
    int nnz = assemble_into(P, &Gp, &Gc, 1, &P->A);
    or_colgeom_free(&Gp); or_colgeom_free(&Gc);
    return nnz;
}

void or_export_matrix(const or_problem *P, int *rowptr, int *col, double *val)
{
    int nnz = P->A.rowptr[P->A.n];
    memcpy(rowptr, P->A.rowptr, (P->A.n + 1) * sizeof(int));
    memcpy(col, P->A.col, nnz * sizeof(int));
    memcpy(val, P->A.val, nnz * sizeof(double));
}

void or_matvec(const or_problem *P, const double *x, double *y)
{
    const or_csr *A = &P->A;
    for (int i = 0; i < A->n; ++i) {
        double s = 0;
        for (int q = A->rowptr[i]; q < A->rowptr[i + 1]; ++q) s += A->val[q] * x[A->col[q]];
        y[i] = s;
    }
}

int or_size(const or_problem *P) { return P->m; }
int or_is_box_pattern(const or_problem *P) { return P->box; }
long or_solve_count(const or_problem *P) { return P->n_solves; }

/* ---------- problem set-up ---------- */

or_problem *or_create(const or_grid *g, const or_params *p, const double *h, int *status)
{
    *status = OR_BAD_ARG;
    if (g->nx < 1 || g->ny < 1 || g->nz < OR_W || !(g->lx > 0) || (g->ny > 1 && !(g->ly > 0)))
        return NULL;
    if (g->walls && (g->ny != 1 || g->nx < 16)) return NULL;
    if (p->restart < 1 || p->k < 0 || p->max_restarts < 0 || p->history < 0 || p->k > 64) return NULL;
    if (p->guess == OR_GUESS_RRF && (p->history < 1 || p->k > p->history)) return NULL;
    if (p->orthonormalize != 0 && p->orthonormalize != 1) return NULL;
    or_problem *P = calloc(1, sizeof(or_problem));
    P->g = *g;
    P->p = *p;
    P->ncol = g->nx * g->ny;
    P->m = P->ncol * (g->nz + 1);
    P->dx = g->walls ? g->lx / (g->nx - 3) : g->lx / g->nx;
    P->dy = g->ny > 1 ? g->ly / g->ny : 1.0;
    /* centred periodic weights on offsets -3..3 */
    double xs[OR_W], cw[3 * OR_W];
    for (int t = 0; t < OR_W; ++t) xs[t] = (t - OR_HALF) * P->dx;
    or_fornberg(0.0, xs, OR_W, 2, cw);
    for (int t = 0; t < OR_W; ++t) { P->wx1[t] = cw[OR_W + t]; P->wx2[t] = cw[2 * OR_W + t]; }
    /* walls: the 7 evaluation points of a window of 7 equispaced nodes */
    for (int t = 0; t < OR_W; ++t) xs[t] = t * P->dx;
    for (int o = 0; o < OR_W; ++o) {
        or_fornberg(o * P->dx, xs, OR_W, 2, cw);
        for (int t = 0; t < OR_W; ++t) { P->wxo1[o][t] = cw[OR_W + t]; P->wxo2[o][t] = cw[2 * OR_W + t]; }
    }
    for (int t = 0; t < OR_W; ++t) xs[t] = (t - OR_HALF) * P->dy;
    or_fornberg(0.0, xs, OR_W, 2, cw);
    for (int t = 0; t < OR_W; ++t) { P->wy1[t] = cw[OR_W + t]; P->wy2[t] = cw[2 * OR_W + t]; }
    /* sigma weights per level */
    int L = g->nz + 1;
    P->ws1 = malloc(L * OR_W * sizeof(double));
    P->ws2 = malloc(L * OR_W * sizeof(double));
    P->win = malloc(L * sizeof(int));
    for (int j = -1; j < g->nz; ++j) {
        int s0 = or_sigma_window(g->nz, j);
        P->win[j + 1] = s0;
        for (int k = 0; k < OR_W; ++k) xs[k] = or_sigma(P, s0 + k);
        or_fornberg(or_sigma(P, j), xs, OR_W, 2, cw);
        for (int k = 0; k < OR_W; ++k) {
            P->ws1[(j + 1) * OR_W + k] = cw[OR_W + k];
            P->ws2[(j + 1) * OR_W + k] = cw[2 * OR_W + k];
        }
    }
    int n = P->ncol;
    P->h = malloc(n * sizeof(double)); P->hx = calloc(n, sizeof(double));
    P->hy = calloc(n, sizeof(double)); P->hxx = calloc(n, sizeof(double));
    P->hyy = calloc(n, sizeof(double));
    memcpy(P->h, h, n * sizeof(double));
    for (int c = 0; c < n; ++c)
        if (!(h[c] > 0)) { or_destroy(P); return NULL; }
    or_surface_derivs(P, P->h, P->hx, P->hy, P->hxx, P->hyy);
    /* Preconditioner pattern: the sigma-cross terms of the still-water
     * operator vanish identically on a flat bed, so the pattern is the
     * 7-point cross there and the full box otherwise. */
    P->box = 0;
    for (int c = 1; c < n; ++c) if (h[c] != h[0]) P->box = 1;
    or_colgeom G0;
    or_colgeom_alloc(P, &G0);
    or_colgeom_eval(P, NULL, &G0);
    assemble_into(P, &G0, &G0, P->box, &P->A0);
    or_colgeom_free(&G0);
    P->Y = calloc((size_t)P->m * (p->k > 0 ? p->k : 1), sizeof(double));
    P->x_prev = calloc(P->m, sizeof(double));
    P->X = calloc((size_t)P->m * (p->history > 0 ? p->history : 1), sizeof(double));
    P->work = malloc((size_t)P->m * 8 * sizeof(double));
    /* Unknown ordering of the factorisation (not fixed by the paper): columns
     * are split into four colours, colour = (ix + iy) mod 4; colour 0
     * columns come first, then colours 1, 2, 3; inside a colour, columns go x
     * fastest then y, and each column lists its levels from the ghost level
     * up.  Columns of one colour are at least four apart along x and y, so a
     * 7-point stencil never couples two of them when nx and ny are multiples
     * of four. */
    int *order = malloc(P->m * sizeof(int));
    int q = 0;
    if (!g->walls) {
        for (int col = 0; col < 4; ++col)
            for (int iy = 0; iy < g->ny; ++iy)
                for (int ix = 0; ix < g->nx; ++ix) {
                    if ((ix + iy) % 4 != col) continue;
                    for (int j = -1; j < g->nz; ++j) order[q++] = (int)or_index(g, ix, iy, j);
                }
    } else {
        /* With walls the rows of columns 0-2 (and nx-3..nx-1) reach 7 columns
         * inwards, so those six columns get three groups of their own after the
         * four colours of columns 3..nx-4: {0, nx-1}, {1, nx-2}, {2, nx-3}. */
        for (int col = 0; col < 4; ++col)
            for (int ix = 3; ix <= g->nx - 4; ++ix) {
                if (ix % 4 != col) continue;
                for (int j = -1; j < g->nz; ++j) order[q++] = (int)or_index(g, ix, 0, j);
            }
        for (int e = 0; e < 3; ++e) {
            int pair[2] = {e, g->nx - 1 - e};
            for (int u = 0; u < 2; ++u)
                for (int j = -1; j < g->nz; ++j) order[q++] = (int)or_index(g, pair[u], 0, j);
        }
    }
    int st = or_build_ilu(P, order);
    free(order);
    if (st != OR_OK) { or_destroy(P); *status = st; return NULL; }
    *status = OR_OK;
    return P;
}

void or_destroy(or_problem *P)
{
    if (!P) return;
    or_csr_free(&P->A); or_csr_free(&P->A0); or_csr_free(&P->LU);
    free(P->ws1); free(P->ws2); free(P->win);
    free(P->h); free(P->hx); free(P->hy); free(P->hxx); free(P->hyy);
    free(P->order); free(P->rank); free(P->diag);
    free(P->Y); free(P->x_prev); free(P->X); free(P->work);
    free(P);
}
