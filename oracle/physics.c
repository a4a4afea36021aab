/*
 * Stage driver of the oracle: the sequence of systems A(tau) x = b(tau).
 * TEST INFRASTRUCTURE ONLY.
 *
 * Algorithm 1 with the low-storage update of Eq. (15a-15c) (Williamson 2N
 * form, alpha_i = A_i, beta_i = B_i) and the LSERK45 scheme of Carpenter &
 * Kennedy (1994) named in Sec. 5.  Inviscid (mu = 0), F = (0, 0, -rho g),
 * total pressure with p = 0 on the free surface (Sec. 2).
 *
 * Right-hand sides, Eq. (16)-(17): with
 *   G = rho/(beta_i dt) u + rho alpha_i/dt K_u + F - rho (u . grad^(i-1)) u
 *       + rho (sigma/d^(i-1)) (D_tau eta^(i-1)) D_sigma u
 * the interior rows take grad^(i) . G, the ghost rows n . G at the bed node,
 * and the surface rows 0.  D_tau eta^(i-1) is f_eta of Eq. (14b) at stage i-1.
 *
 * Walls: the ghost-column rows take n . G at the wall node; x derivatives of
 * the velocities and of G use the physical columns only, those of p the
 * ghost columns too.  The ghost columns carry no flow: f_eta and f_u are zero
 * there, so their state never changes.
 *
 * Generation and absorption zones (Sec. 5.2): after each stage the surface
 * and the velocities inside a zone are blended towards a target,
 * phi <- Gamma phi + (1 - Gamma) phi_target, with the relaxation weight of
 * Engsig-Karup, Bingham & Lindberg (J. Comput. Phys. 228, 2009),
 * Gamma(xi) = 1 - (exp(xi^3.5) - 1)/(e - 1), xi = 0 at the inner end of the
 * zone and 1 at the wall.  The generation target is the incident linear
 * (Airy) wave of height H and period T, its amplitude ramped in time by
 * (1 - cos(pi t / t_ramp))/2; the absorption target is still water.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "internal.h"

void or_lserk45(double *alpha, double *beta, double *c)
{
    static const double A[5] = {
        0.0,
        -567301805773.0 / 1357537059087.0,
        -2404267990393.0 / 2016746695238.0,
        -3550918686646.0 / 2091501179385.0,
        -1275806237668.0 / 842570457699.0};
    static const double B[5] = {
        1432997174477.0 / 9575080441755.0,
        5161836677717.0 / 13612068292357.0,
        1720146321549.0 / 2090206949498.0,
        3134564353537.0 / 4481467310338.0,
        2277821191437.0 / 14882151754819.0};
    static const double C[5] = {
        0.0,
        1432997174477.0 / 9575080441755.0,
        2526269341429.0 / 6820363962896.0,
        2006345519317.0 / 3224310063776.0,
        2802321613138.0 / 2924317926251.0};
    for (int i = 0; i < 5; ++i) { alpha[i] = A[i]; beta[i] = B[i]; c[i] = C[i]; }
}

/* Eq. (14b): f_eta = w - u D_chi eta - v D_gamma eta at sigma = 1. */
void or_f_eta(const or_problem *P, const double *u, const double *v, const double *w,
              const double *eta, double *out)
{
    const or_grid *g = &P->g;
    int n = P->ncol;
    double *ex = calloc(n, sizeof(double)), *ey = calloc(n, sizeof(double));
    or_surface_derivs(P, eta, ex, ey, NULL, NULL);
    for (int iy = 0; iy < g->ny; ++iy)
        for (int ix = 0; ix < g->nx; ++ix) {
            int c = iy * g->nx + ix;
            long s = or_index(g, ix, iy, g->nz - 1);
            out[c] = or_is_wall_ghost(P, ix) ? 0.0 : w[s] - u[s] * ex[c] - (v ? v[s] * ey[c] : 0.0);
        }
    free(ex); free(ey);
}

/* Per-node transform coefficients of one surface: sigma_x, sigma_y, 1/d. */
static void node_coefs(const or_problem *P, const or_colgeom *G, long node, int c, int j,
                       double *sx, double *sy, double *inv_d)
{
    double sg = or_sigma(P, j);
    *inv_d = 1.0 / G->d[c];
    *sx = (P->hx[c] - sg * G->dx[c]) * *inv_d;
    *sy = P->g.ny > 1 ? (P->hy[c] - sg * G->dy[c]) * *inv_d : 0.0;
    (void)node;
}

/* (u . grad^(i-1)) phi and D_sigma phi at every node. */
static void advect(const or_problem *P, const or_colgeom *Gp, const double *u, const double *v,
                   const double *w, const double *phi, double *adv, double *dphis)
{
    const or_grid *g = &P->g;
    int m = P->m;
    double *px = malloc(m * sizeof(double)), *py = malloc(m * sizeof(double));
    or_field_dx(P, phi, px, 0);
    or_field_dy(P, phi, py);
    or_field_dsigma(P, phi, dphis);
    for (int j = -1; j < g->nz; ++j)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                long q = or_index(g, ix, iy, j);
                int c = iy * g->nx + ix;
                double sx, sy, f;
                node_coefs(P, Gp, q, c, j, &sx, &sy, &f);
                double gx = px[q] + sx * dphis[q];
                double gy = py[q] + sy * dphis[q];
                double gz = f * dphis[q];
                adv[q] = u[q] * gx + (v ? v[q] * gy : 0.0) + w[q] * gz;
            }
    free(px); free(py);
}

void or_rhs(const or_problem *P, const or_physics *ph, int stage,
            const double *u, const double *v, const double *w,
            const double *Ku, const double *Kv, const double *Kw,
            const double *eta_prev, const double *eta_cur, const double *deta_dt, double *b)
{
    const or_grid *g = &P->g;
    int m = P->m;
    double al[5], be[5], cc[5];
    or_lserk45(al, be, cc);
    double a_i = al[stage - 1], b_i = be[stage - 1], dt = ph->dt, rho = ph->rho;
    or_colgeom Gp, Gc;
    or_colgeom_alloc(P, &Gp); or_colgeom_alloc(P, &Gc);
    or_colgeom_eval(P, eta_prev, &Gp);
    or_colgeom_eval(P, eta_cur, &Gc);
    const double *comp[3] = {u, v, w};
    const double *Kc[3] = {Ku, Kv, Kw};
    double *G[3], *adv = malloc(m * sizeof(double)), *ds = malloc(m * sizeof(double));
    for (int d = 0; d < 3; ++d) {
        G[d] = calloc(m, sizeof(double));
        if (!comp[d]) continue;
        advect(P, &Gp, u, v, w, comp[d], adv, ds);
        for (int j = -1; j < g->nz; ++j)
            for (int iy = 0; iy < g->ny; ++iy)
                for (int ix = 0; ix < g->nx; ++ix) {
                    long q = or_index(g, ix, iy, j);
                    int c = iy * g->nx + ix;
                    double sg = or_sigma(P, j);
                    double Fd = d == 2 ? -rho * ph->g : 0.0;
                    G[d][q] = rho / (b_i * dt) * comp[d][q] + rho * a_i / dt * Kc[d][q] + Fd
                              - rho * adv[q] + rho * (sg / Gp.d[c]) * deta_dt[c] * ds[q];
                }
    }
    /* divergence grad^(i) . G on the interior rows */
    double *gxu = malloc(m * sizeof(double)), *gsu = malloc(m * sizeof(double));
    double *gyv = malloc(m * sizeof(double)), *gsv = malloc(m * sizeof(double));
    double *gsw = malloc(m * sizeof(double));
    or_field_dx(P, G[0], gxu, 0); or_field_dsigma(P, G[0], gsu);
    or_field_dy(P, G[1], gyv); or_field_dsigma(P, G[1], gsv);
    or_field_dsigma(P, G[2], gsw);
    for (int j = -1; j < g->nz; ++j)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                long q = or_index(g, ix, iy, j);
                int c = iy * g->nx + ix;
                if (j == g->nz - 1) { b[q] = 0.0; continue; }
                if (or_is_wall_ghost(P, ix)) {          /* n . G at the wall node */
                    int iw = ix == 0 ? 1 : g->nx - 2;
                    double nxs = ix == 0 ? -1.0 : 1.0;
                    b[q] = nxs * G[0][or_index(g, iw, iy, j)];
                    continue;
                }
                if (j == -1) {
                    long qb = or_index(g, ix, iy, 0);
                    double hx = P->hx[c], hy = P->hy[c];
                    double nrm = 1.0 / sqrt(1.0 + hx * hx + hy * hy);
                    b[q] = -nrm * (hx * G[0][qb] + hy * G[1][qb] + G[2][qb]);
                    continue;
                }
                double sx, sy, e;
                node_coefs(P, &Gc, q, c, j, &sx, &sy, &e);
                b[q] = gxu[q] + sx * gsu[q] + gyv[q] + sy * gsv[q] + e * gsw[q];
            }
    for (int d = 0; d < 3; ++d) free(G[d]);
    free(adv); free(ds); free(gxu); free(gsu); free(gyv); free(gsv); free(gsw);
    or_colgeom_free(&Gp); or_colgeom_free(&Gc);
}

int or_stage(or_problem *P, const or_physics *ph, int stage,
             double *u, double *v, double *w, double *eta,
             double *Ku, double *Kv, double *Kw, double *Keta, double *p, or_stats *st)
{
    const or_grid *g = &P->g;
    int m = P->m, n = P->ncol;
    double al[5], be[5], cc[5];
    or_lserk45(al, be, cc);
    double a_i = al[stage - 1], b_i = be[stage - 1], dt = ph->dt;
    /* K_eta and eta^(i) (Algorithm 1, first two updates) */
    double *feta = malloc(n * sizeof(double)), *eta_new = malloc(n * sizeof(double));
    or_f_eta(P, u, v, w, eta, feta);
    for (int c = 0; c < n; ++c) {
        Keta[c] = a_i * Keta[c] + dt * feta[c];
        eta_new[c] = eta[c] + b_i * Keta[c];
    }
    /* pressure p^(i-1) from A(eta^(i-1), eta^(i)) p = b */
    double *b = malloc(m * sizeof(double));
    or_rhs(P, ph, stage, u, v, w, Ku, Kv, Kw, eta, eta_new, feta, b);
    int status = or_solve(P, eta, eta_new, b, p, st);
    /* f_u of Eq. (14a) with the stage i-1 geometry, then K_u and u */
    or_colgeom Gp;
    or_colgeom_alloc(P, &Gp);
    or_colgeom_eval(P, eta, &Gp);
    double *px = malloc(m * sizeof(double)), *py = malloc(m * sizeof(double));
    double *ps = malloc(m * sizeof(double));
    or_field_dx(P, p, px, 1); or_field_dy(P, p, py); or_field_dsigma(P, p, ps);
    double *comp[3] = {u, v, w};
    double *Kc[3] = {Ku, Kv, Kw};
    double *adv[3], *ds[3];
    for (int d = 0; d < 3; ++d) {
        adv[d] = malloc(m * sizeof(double)); ds[d] = malloc(m * sizeof(double));
        if (comp[d]) advect(P, &Gp, u, v, w, comp[d], adv[d], ds[d]);
    }
    for (int j = -1; j < g->nz; ++j)
        for (int iy = 0; iy < g->ny; ++iy)
            for (int ix = 0; ix < g->nx; ++ix) {
                long q = or_index(g, ix, iy, j);
                int c = iy * g->nx + ix;
                double sx, sy, f;
                node_coefs(P, &Gp, q, c, j, &sx, &sy, &f);
                double sg = or_sigma(P, j);
                double gradp[3] = {px[q] + sx * ps[q], py[q] + sy * ps[q], f * ps[q]};
                for (int d = 0; d < 3; ++d) {
                    if (!comp[d]) continue;
                    double Fd = d == 2 ? -ph->g : 0.0;
                    double fu = -gradp[d] / ph->rho + Fd - adv[d][q]
                                + (sg / Gp.d[c]) * feta[c] * ds[d][q];
                    if (or_is_wall_ghost(P, ix)) fu = 0.0;
                    Kc[d][q] = a_i * Kc[d][q] + dt * fu;
                }
            }
    for (int d = 0; d < 3; ++d) {
        if (comp[d]) for (int q = 0; q < m; ++q) comp[d][q] += b_i * Kc[d][q];
        free(adv[d]); free(ds[d]);
    }
    memcpy(eta, eta_new, n * sizeof(double));
    or_colgeom_free(&Gp);
    free(feta); free(eta_new); free(b); free(px); free(py); free(ps);
    return status;
}

/* ---------- generation and absorption zones ---------- */

double or_relax_weight(double xi)
{
    if (xi <= 0.0) return 1.0;
    if (xi >= 1.0) return 0.0;
    return 1.0 - (exp(pow(xi, 3.5)) - 1.0) / (exp(1.0) - 1.0);
}

double or_wavenumber(double omega, double depth, double g)
{
    double k = omega * omega / g;            /* deep-water start; F is increasing and concave */
    for (int it = 0; it < 100; ++it) {
        double th = tanh(k * depth);
        double F = g * k * th - omega * omega;
        double dF = g * th + g * k * depth * (1.0 - th * th);
        double dk = F / dF;
        k -= dk;
        if (fabs(dk) <= 1e-15 * k) break;
    }
    return k;
}

void or_relax(const or_problem *P, const or_relaxation *rl, double t, double *u, double *w, double *eta)
{
    const or_grid *g = &P->g;
    const double pi = 3.14159265358979323846;
    double omega = 2.0 * pi / rl->period;
    double k = or_wavenumber(omega, rl->depth, rl->g);
    double ramp = 1.0;
    if (rl->ramp_time > 0.0 && t < rl->ramp_time) ramp = 0.5 * (1.0 - cos(pi * t / rl->ramp_time));
    double amp = 0.5 * rl->height * ramp;
    for (int ix = 0; ix < g->nx; ++ix) {
        if (or_is_wall_ghost(P, ix)) continue;
        double x = or_xcoord(P, ix);
        double gam, th = k * x - omega * t;
        int gen;
        if (rl->gen_x1 > rl->gen_x0 && x >= rl->gen_x0 && x <= rl->gen_x1) {
            gam = or_relax_weight((rl->gen_x1 - x) / (rl->gen_x1 - rl->gen_x0));
            gen = 1;
        } else if (rl->abs_x1 > rl->abs_x0 && x >= rl->abs_x0 && x <= rl->abs_x1) {
            gam = or_relax_weight((x - rl->abs_x0) / (rl->abs_x1 - rl->abs_x0));
            gen = 0;
        } else {
            continue;
        }
        double eta_t = gen ? amp * cos(th) : 0.0;
        eta[ix] = gam * eta[ix] + (1.0 - gam) * eta_t;
        double d = P->h[ix] + eta[ix];
        for (int j = -1; j < g->nz; ++j) {
            long q = or_index(g, ix, 0, j);
            double z = or_sigma(P, j) * d - P->h[ix];
            double ut = 0.0, wt = 0.0;
            if (gen) {
                double sh = sinh(k * rl->depth);
                ut = amp * omega * cosh(k * (z + rl->depth)) / sh * cos(th);
                wt = amp * omega * sinh(k * (z + rl->depth)) / sh * sin(th);
            }
            u[q] = gam * u[q] + (1.0 - gam) * ut;
            w[q] = gam * w[q] + (1.0 - gam) * wt;
        }
    }
}
