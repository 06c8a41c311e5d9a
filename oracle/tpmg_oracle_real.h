/*
 * Precision-generic body of the CPU oracle (TEST INFRASTRUCTURE ONLY),
 * included twice by tpmg_oracle.c with REAL = double and REAL = float.
 * SFX(name) appends _d / _f.  IX(k, j, i) is defined by the includer.
 */

/* (H u)_c in flux form: h_c u_c + sum over the six faces of T_f (u_c - u_nb).
 * Longitude is periodic; the pole, surface and top faces carry T = 0 and have
 * no neighbour, so their terms are skipped. */
static REAL SFX(hu_cell)(int nlon, int nlat, int nz,
                         const REAL *tx, const REAL *ty, const REAL *tz, const REAL *h,
                         const REAL *u, int k, int j, int i)
{
    size_t c = IX(k, j, i);
    int ie = (i + 1) % nlon;
    int iw = (i + nlon - 1) % nlon;
    REAL uc = u[c];
    REAL acc = h[c] * uc;
    acc += tx[c] * (uc - u[IX(k, j, ie)]);
    acc += tx[IX(k, j, iw)] * (uc - u[IX(k, j, iw)]);
    if (j + 1 < nlat) acc += ty[c] * (uc - u[IX(k, j + 1, i)]);
    if (j > 0) acc += ty[IX(k, j - 1, i)] * (uc - u[IX(k, j - 1, i)]);
    if (k + 1 < nz) acc += tz[c] * (uc - u[IX(k + 1, j, i)]);
    if (k > 0) acc += tz[IX(k - 1, j, i)] * (uc - u[IX(k - 1, j, i)]);
    return acc;
}

/* y = H u (Section 2: the operator of H u = b). */
void SFX(orc_apply)(int nlon, int nlat, int nz,
                    const REAL *tx, const REAL *ty, const REAL *tz, const REAL *h,
                    const REAL *u, REAL *y)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i)
                y[IX(k, j, i)] = SFX(hu_cell)(nlon, nlat, nz, tx, ty, tz, h, u, k, j, i);
}

/* r = b - H u (the residual whose norm the paper's iteration reduces). */
void SFX(orc_residual)(int nlon, int nlat, int nz,
                       const REAL *tx, const REAL *ty, const REAL *tz, const REAL *h,
                       const REAL *b, const REAL *u, REAL *r)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                size_t c = IX(k, j, i);
                r[c] = b[c] - SFX(hu_cell)(nlon, nlat, nz, tx, ty, tz, h, u, k, j, i);
            }
}

/* r = b - H u for u = omega H_z^{-1} b (the sweep of Eq. (1) from zero):
 * H_z u = omega b leaves (1 - omega) b plus the four horizontal couplings
 * of u, added east, west, north, south (om1 = 1 - omega). */
void SFX(orc_presmooth_residual)(int nlon, int nlat, int nz, const REAL *tx, const REAL *ty,
                                 const REAL *b, const REAL *u, REAL om1, REAL *r)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                size_t c = IX(k, j, i);
                int ie = (i + 1) % nlon;
                int iw = (i + nlon - 1) % nlon;
                REAL v = om1 * b[c];
                v += tx[c] * u[IX(k, j, ie)];
                v += tx[IX(k, j, iw)] * u[IX(k, j, iw)];
                if (j + 1 < nlat) v += ty[IX(k, j, i)] * u[IX(k, j + 1, i)];  /* north */
                if (j > 0) v += ty[IX(k, j - 1, i)] * u[IX(k, j - 1, i)];     /* south */
                r[c] = v;
            }
}

/*
 * x = H_z^{-1} r for the column (j, i) (Section 2.1: H_z holds the diagonal of
 * H and the couplings within a vertical column).
 *
 * Row k of H_z: diagonal s_k + t_{k-1} + t_k, off-diagonals -t_{k-1}, -t_k,
 * where t_k = tz(k) couples layers k and k+1 and s_k = h + the four horizontal
 * couplings of the cell (the part of the diagonal that does not cancel
 * against the column's own off-diagonals).  Gaussian elimination without
 * pivoting, with each pivot written as p_k = q_k + t_k:
 *   q_0 = s_0,  q_k = s_k + t_{k-1} q_{k-1} / p_{k-1}
 *   y_k = (r_k + t_{k-1} y_{k-1}) / p_k                 (forward)
 *   x_k = x_{k+1} + (y_k - (q_k / p_k) x_{k+1})          (backward)
 * This equals the textbook Thomas recursion (backward: x_k = y_k +
 * (t_k / p_k) x_{k+1}) and keeps the small quantities q_k and q_k / p_k to
 * full relative accuracy although t_k exceeds s_k by up to ~1e6-1e8.
 */
static void SFX(column_solve)(int nlon, int nlat, int nz,
                              const REAL *tx, const REAL *ty, const REAL *tz, const REAL *h,
                              const REAL *r, int j, int i,
                              REAL *q, REAL *p, REAL *y, REAL *x)
{
    int iw = (i + nlon - 1) % nlon;
    for (int k = 0; k < nz; ++k) {
        size_t c = IX(k, j, i);
        REAL s = h[c] + tx[c] + tx[IX(k, j, iw)] + ty[c];
        if (j > 0) s += ty[IX(k, j - 1, i)];
        REAL tup = tz[c];
        if (k == 0) {
            q[0] = s;
            p[0] = q[0] + tup;
            y[0] = r[c] / p[0];
        } else {
            REAL tdn = tz[IX(k - 1, j, i)];
            q[k] = s + tdn * q[k - 1] / p[k - 1];
            p[k] = q[k] + tup;
            y[k] = (r[c] + tdn * y[k - 1]) / p[k];
        }
    }
    x[nz - 1] = y[nz - 1];
    for (int k = nz - 2; k >= 0; --k)
        x[k] = x[k + 1] + (y[k] - (q[k] / p[k]) * x[k + 1]);
}

/*
 * One block-Jacobi (vertical line relaxation) sweep, Eq. (1):
 *   u <- u + omega H_z^{-1} (b - H u).
 * With H = H_z + dH this equals (1 - omega) u + omega H_z^{-1} (b - dH u),
 * and that is how it is evaluated: b - dH u = b + sum over the four
 * horizontal faces of T_f u_nb(f) has no vertical fluxes, so the
 * cancellation of the large vertical terms inside b - H u (couplings ~1e6
 * times the row sums) never happens.  rhs is caller-provided work space of
 * the field's size; every column reads the old u.
 */
void SFX(orc_smooth)(int nlon, int nlat, int nz,
                     const REAL *tx, const REAL *ty, const REAL *tz, const REAL *h,
                     const REAL *b, REAL *u, REAL omega, REAL *rhs)
{
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                size_t c = IX(k, j, i);
                int ie = (i + 1) % nlon;
                int iw = (i + nlon - 1) % nlon;
                REAL v = b[c];
                v += tx[c] * u[IX(k, j, ie)];
                v += tx[IX(k, j, iw)] * u[IX(k, j, iw)];
                if (j + 1 < nlat) v += ty[c] * u[IX(k, j + 1, i)];
                if (j > 0) v += ty[IX(k, j - 1, i)] * u[IX(k, j - 1, i)];
                rhs[c] = v;
            }
    const REAL one = (REAL)1;
#pragma omp parallel
    {
        REAL *q = (REAL *)malloc(4 * (size_t)nz * sizeof(REAL));
        REAL *p = q + nz, *y = p + nz, *x = y + nz;
#pragma omp for schedule(static)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                SFX(column_solve)(nlon, nlat, nz, tx, ty, tz, h, rhs, j, i, q, p, y, x);
                for (int k = 0; k < nz; ++k) {
                    size_t c = IX(k, j, i);
                    u[c] = (one - omega) * u[c] + omega * x[k];
                }
            }
        free(q);
    }
}

/* x = H_z^{-1} r for every column (used by tests and the coarse solve). */
void SFX(orc_column_solve_all)(int nlon, int nlat, int nz,
                               const REAL *tx, const REAL *ty, const REAL *tz, const REAL *h,
                               const REAL *r, REAL *xout)
{
#pragma omp parallel
    {
        REAL *q = (REAL *)malloc(4 * (size_t)nz * sizeof(REAL));
        REAL *p = q + nz, *y = p + nz, *x = y + nz;
#pragma omp for schedule(static)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                SFX(column_solve)(nlon, nlat, nz, tx, ty, tz, h, r, j, i, q, p, y, x);
                for (int k = 0; k < nz; ++k) xout[IX(k, j, i)] = x[k];
            }
        free(q);
    }
}

/*
 * Prolongation P (horizontal only; the vertical is never coarsened): bilinear
 * interpolation of the coarse correction to the fine cell centres.
 *   lon: fine cell i lies a quarter coarse spacing west (i even) or east
 *        (i odd) of its parent I = i/2: weights 3/4 on I, 1/4 on I-1 or I+1
 *        (periodic).
 *   lat: fine row j takes w0[j] of coarse row j0[j] and w1[j] of row j1[j]
 *        (j1 = -1 when the row centre coincides with its parent's or no
 *        neighbour exists towards the pole); weights come from the row
 *        centres (see the Python hierarchy builder).
 * Restriction R = P^T: every fine residual is scattered back with the same
 * weights.  u += P e adds the correction.
 */
static void SFX(lon_parents)(int i, int nlon_c, int *I, int *Inb)
{
    *I = i / 2;
    *Inb = (i % 2 == 0) ? (*I + nlon_c - 1) % nlon_c : (*I + 1) % nlon_c;
}

void SFX(orc_restrict)(int nlon, int nlat, int nz, int nlat_c,
                       const int *j0, const double *w0, const int *j1, const double *w1,
                       const REAL *r, REAL *bc)
{
    const int nlon_c = nlon / 2;
    const REAL three4 = (REAL)0.75, one4 = (REAL)0.25;
    memset(bc, 0, (size_t)nz * nlat_c * nlon_c * sizeof(REAL));
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                int I, Inb;
                SFX(lon_parents)(i, nlon_c, &I, &Inb);
                REAL rv = r[IX(k, j, i)];
                for (int a = 0; a < 2; ++a) {
                    int J = a == 0 ? j0[j] : j1[j];
                    if (J < 0) continue;
                    REAL w = (REAL)(a == 0 ? w0[j] : w1[j]);
                    size_t base = (((size_t)k) * nlat_c + J) * nlon_c;
                    bc[base + I] += w * three4 * rv;
                    bc[base + Inb] += w * one4 * rv;
                }
            }
}

void SFX(orc_prolong_add)(int nlon, int nlat, int nz, int nlat_c,
                          const int *j0, const double *w0, const int *j1, const double *w1,
                          const REAL *ec, REAL *u)
{
    const int nlon_c = nlon / 2;
    const REAL three4 = (REAL)0.75, one4 = (REAL)0.25;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nlat; ++j)
            for (int i = 0; i < nlon; ++i) {
                int I, Inb;
                SFX(lon_parents)(i, nlon_c, &I, &Inb);
                REAL add = 0;
                for (int a = 0; a < 2; ++a) {
                    int J = a == 0 ? j0[j] : j1[j];
                    if (J < 0) continue;
                    REAL w = (REAL)(a == 0 ? w0[j] : w1[j]);
                    size_t base = (((size_t)k) * nlat_c + J) * nlon_c;
                    add += w * (three4 * ec[base + I] + one4 * ec[base + Inb]);
                }
                u[IX(k, j, i)] += add;
            }
}
