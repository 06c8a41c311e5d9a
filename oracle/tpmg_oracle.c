/*
 * CPU oracle for the tensor-product multigrid of the paper (Section 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference the CUDA
 * library is checked against.  Only the tests, the package's smoke check and
 * the CPU-baseline leg of the benchmark may load it; the library never does.
 * It shares no code with the CUDA path.
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-adds), OpenMP over
 * independent rows of columns only.  Every routine exists twice through the
 * REAL template below: in double (the FP64 method) and in float (the FP32
 * inner V-cycle of the mixed-precision form, Section 1's single-precision
 * remark).
 *
 * Layout: [nz][nlat][nlon], index (k, j, i) -> (k*nlat + j)*nlon + i.
 *   tx[k,j,i]: face (i, i+1 mod nlon)   ty[k,j,i]: face (j, j+1), 0 on j = nlat-1
 *   tz[k,j,i]: face (k, k+1), 0 on k = nz-1   h[k,j,i]: Helmholtz term
 *
 * Operator (Section 2, H u = b, of Laplacian type), flux form:
 *   (H u)_c = h_c u_c + sum_faces T_f (u_c - u_nb(f))
 * Split H = H_z + dH (Section 2.1): H_z holds the diagonal of H and the
 * couplings inside a column (-tz); dH the horizontal couplings.
 * Smoother, Eq. (1) with the sign that makes it converge:
 *   u <- u + omega H_z^{-1} (b - H u)
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stddef.h>

#define IX(k, j, i) ((((size_t)(k)) * (size_t)nlat + (size_t)(j)) * (size_t)nlon + (size_t)(i))

/* ---------------------------------------------------------------- REAL = double */
#define REAL double
#define SFX(name) name##_d
#include "tpmg_oracle_real.h"
#undef REAL
#undef SFX

/* ---------------------------------------------------------------- REAL = float */
#define REAL float
#define SFX(name) name##_f
#include "tpmg_oracle_real.h"
#undef REAL
#undef SFX

/* Plain serial dot product in index order (deterministic). */
double orc_dot(size_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (size_t c = 0; c < n; ++c) s += x[c] * y[c];
    return s;
}

double orc_maxabs(size_t n, const double *x)
{
    double m = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double a = fabs(x[c]);
        if (a > m) m = a;
    }
    return m;
}

/*
 * Coarse-level coefficients (setup of level l+1 from level l), Sections 2.1
 * and 2.2: the grid is coarsened in the horizontal only; every coarse cell is
 * the union of 2 longitudes x cnt (1 or 2) latitude rows of the same layer.
 *   h, tz : sums over the children (the vertical is never coarsened).
 *   tx    : sum of the fine east faces that form the coarse east face,
 *           times sx = (fine lon spacing)/(coarse lon spacing) = 1/2.
 *   ty    : sum of the fine north faces of the top child row, times sy[J] =
 *           (fine centre distance across that face)/(coarse centre distance).
 * sx = 1 and sy = 1 give the Galerkin product P^T H P of piecewise-constant
 * prolongation.  row_of[j] = coarse row of fine row j; top_row[J] = the
 * northern-most fine row of coarse row J.
 */
void orc_coarsen_coeffs(int nlon, int nlat, int nz, int nlat_c,
                        const int *row_of, const int *top_row,
                        double sx, const double *sy,
                        const double *tx, const double *ty, const double *tz,
                        const double *h,
                        double *txc, double *tyc, double *tzc, double *hc)
{
    const int nlon_c = nlon / 2;
    const size_t nc = (size_t)nz * nlat_c * nlon_c;
    memset(hc, 0, nc * sizeof(double));
    memset(tzc, 0, nc * sizeof(double));
    memset(txc, 0, nc * sizeof(double));
    memset(tyc, 0, nc * sizeof(double));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j) {
            int J = row_of[j];
            for (int i = 0; i < nlon; ++i) {
                int I = i / 2;
                size_t f = IX(k, j, i);
                size_t c = (((size_t)k) * nlat_c + J) * nlon_c + I;
                hc[c] += h[f];
                tzc[c] += tz[f];
                if (i % 2 == 1) txc[c] += tx[f];            /* east face of coarse cell */
                if (j == top_row[J]) tyc[c] += ty[f];         /* north face of coarse row */
            }
        }
    for (int k = 0; k < nz; ++k)
        for (int J = 0; J < nlat_c; ++J)
            for (int I = 0; I < nlon_c; ++I) {
                size_t c = (((size_t)k) * nlat_c + J) * nlon_c + I;
                txc[c] *= sx;
                tyc[c] = (J == nlat_c - 1) ? 0.0 : tyc[c] * sy[J];
            }
}

/*
 * Coefficient gradient of L(x(b, H)) (differentiable solve): with
 * lambda = H^{-T} dL/dx and H x = b,
 *   dL/dh_c = -lambda_c x_c,   dL/dT_f = -(lambda_c1 - lambda_c2)(x_c1 - x_c2)
 * for the two cells c1, c2 of face f.
 */
void orc_coeff_grad(int nlon, int nlat, int nz, const double *lam, const double *x,
                    double *gh, double *gtx, double *gty, double *gtz)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                size_t c = IX(k, j, i);
                gh[c] = -lam[c] * x[c];
                size_t e = IX(k, j, (i + 1) % nlon);
                gtx[c] = -(lam[c] - lam[e]) * (x[c] - x[e]);
                if (j + 1 < nlat) {
                    size_t n = IX(k, j + 1, i);
                    gty[c] = -(lam[c] - lam[n]) * (x[c] - x[n]);
                } else {
                    gty[c] = 0.0;
                }
                if (k + 1 < nz) {
                    size_t u = IX(k + 1, j, i);
                    gtz[c] = -(lam[c] - lam[u]) * (x[c] - x[u]);
                } else {
                    gtz[c] = 0.0;
                }
            }
}

void orc_to_float(size_t n, const double *x, float *y)
{
    for (size_t c = 0; c < n; ++c) y[c] = (float)x[c];
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
