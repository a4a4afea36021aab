/* Internal state of the oracle problem.  TEST INFRASTRUCTURE ONLY. */
#ifndef SAWAVE_ORACLE_INTERNAL_H
#define SAWAVE_ORACLE_INTERNAL_H
#include "oracle.h"

struct or_problem {
    or_grid g;
    or_params p;
    int ncol;            /* nx * ny */
    int m;               /* ncol * (nz + 1) */
    int box;             /* structural pattern includes the sigma-cross terms */
    double dx, dy;
    double wx1[OR_W], wx2[OR_W], wy1[OR_W], wy2[OR_W];  /* centred periodic weights */
    double wxo1[OR_W][OR_W], wxo2[OR_W][OR_W];          /* walls: weights at node o of a 7-node window */
    double *ws1, *ws2;   /* (nz+1) x 7 sigma weights, row j+1 */
    int *win;            /* (nz+1) first window level, row j+1 */
    double *h, *hx, *hy, *hxx, *hyy;  /* bathymetry and its surface-grid derivatives */
    or_csr A;            /* last assembled operator */
    or_csr A0;           /* still-water operator on the preconditioner pattern */
    or_csr LU;           /* ILU(0) factors in the permuted ordering (L unit lower + U) */
    int *order, *rank;   /* order[new] = old, rank[old] = new */
    int *diag;           /* position of the diagonal in each row of LU */
    double *Y;           /* EWMA sketch, k columns of length m, column-major */
    double *x_prev;      /* last solution */
    double *X;           /* range finder: ring of the K newest solutions, slot = solve index mod K */
    long n_solves;
    double *work;        /* scratch */
};

/* Column-geometry of one free surface, Sec. 2.1 (13b-13d). */
typedef struct {
    double *d, *dx, *dy, *dxx, *dyy;
} or_colgeom;

void or_colgeom_alloc(const or_problem *P, or_colgeom *G);
void or_colgeom_free(or_colgeom *G);
void or_colgeom_eval(const or_problem *P, const double *eta, or_colgeom *G);
/* Periodic surface-grid derivatives D_chi, D_chichi, D_gamma, D_gammagamma (Sec. 3). */
void or_surface_derivs(const or_problem *P, const double *f, double *fx, double *fy,
                       double *fxx, double *fyy);
/* The 7 columns and weights of the x derivatives at column ix.  Periodic: the
 * centred window.  Walls: field != 0 selects the window of an unknown of the
 * linear system (ghost columns included, start clamp(ix-3, 0, nx-7));
 * field == 0 the window of surface data and velocities (physical columns
 * only, start clamp(ix'-3, 1, nx-8) with ix' = ix moved off a ghost column). */
void or_xwin(const or_problem *P, int ix, int field, int *cols, const double **w1, const double **w2);
/* 1 for the ghost columns outside the walls. */
int or_is_wall_ghost(const or_problem *P, int ix);
/* 3-D field derivatives at all nodes (field: as in or_xwin). */
void or_field_dx(const or_problem *P, const double *f, double *out, int field);
void or_field_dy(const or_problem *P, const double *f, double *out);
void or_field_dsigma(const or_problem *P, const double *f, double *out);
void or_csr_free(or_csr *A);
double or_sigma(const or_problem *P, int j);
#endif
