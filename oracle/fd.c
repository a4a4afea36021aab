/*
 * Finite-difference weights for the oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * The paper discretises every spatial derivative with sixth-order
 * finite differences (Sec. 5.2); with 7 nodes per stencil this is the
 * highest order a 7-point formula reaches for first derivatives.  Weights are
 * obtained with Fornberg's recursion (B. Fornberg, Math. Comp. 51, 1988), which
 * builds the derivatives of the Lagrange interpolant through the nodes one
 * node at a time.
 */
#include "oracle.h"

/* c[d*n + i]: weight of node i for the d-th derivative at z, d = 0..mmax. */
void or_fornberg(double z, const double *x, int n, int mmax, double *c)
{
    for (int i = 0; i < (mmax + 1) * n; ++i) c[i] = 0.0;
    double c1 = 1.0;
    double c4 = x[0] - z;
    c[0] = 1.0;
    for (int i = 1; i < n; ++i) {
        int mn = i < mmax ? i : mmax;
        double c2 = 1.0;
        double c5 = c4;
        c4 = x[i] - z;
        for (int j = 0; j < i; ++j) {
            double c3 = x[i] - x[j];
            c2 *= c3;
            if (j == i - 1) {
                /* new node i: weights from those of node i-1 */
                for (int k = mn; k >= 1; --k)
                    c[k * n + i] = c1 * (k * c[(k - 1) * n + i - 1] - c5 * c[k * n + i - 1]) / c2;
                c[i] = -c1 * c5 * c[i - 1] / c2;
            }
            /* old nodes j: rescale for the added factor (x - x_i) */
            for (int k = mn; k >= 1; --k)
                c[k * n + j] = (c4 * c[k * n + j] - k * c[(k - 1) * n + j]) / c3;
            c[j] = c4 * c[j] / c3;
        }
        c1 = c2;
    }
}

/*
 * The sigma direction has nz levels plus one ghost level below the bed
 * (Sec. 5.1: "one additional ghost node just below the sea bed").  A
 * centred 7-node window is used where it fits; next to the bed and the free
 * surface the window is shifted inside the grid (off-centred formula).
 */
int or_sigma_window(int nz, int j)
{
    int s = j - OR_HALF;
    if (s < -1) s = -1;
    if (s > nz - OR_W) s = nz - OR_W;
    return s;
}
