/*
 * sl_oracle.c -- plain FP64 CPU oracle of the multi-stage semi-Lagrangian
 * schemes of Cameron, Raynaud & Dormy, "Multi-stage high order
 * semi-Lagrangian schemes for incompressible flows in Cartesian geometries"
 * (arXiv 1606.06117).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * library: the two are independent implementations of the same paper.
 *
 * Conventions (all arithmetic in double, compiled with -ffp-contract=off):
 *   - Grid: periodic, n[0] x n[1] x n[2] cells stored [z][y][x], x fastest.
 *     ndim = 1, 2 or 3; unused axes have n = 1.
 *   - c: ndim planes of prod(n) doubles, plane d holds the Courant number
 *     C_d = u_d dt / dx_d of the velocity at that (arrival) cell.
 *   - Indices are in cell units: cell i sits at x_i = (i + 1/2) dx.
 *
 * Every function cites the passage of the paper it follows.  Readings of
 * passages that are silent or garbled are stated where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_CIR = 0, ORC_FEC = 1, ORC_BEC = 2, ORC_CEC = 3, ORC_CEC_DEF = 4, ORC_CEC_SL = 5, ORC_CEC_SL_LIT = 6 };

static int64_t wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static int64_t ncells(const int64_t n[3]) { return n[0] * n[1] * n[2]; }

static int64_t at(const int64_t n[3], int64_t x, int64_t y, int64_t z)
{
    return (wrap(z, n[2]) * n[1] + wrap(y, n[1])) * n[0] + wrap(x, n[0]);
}

/*
 * Interpolation operator L_U (Sec. 2: L_U[Phi](x) = interpolated Phi at the
 * departure point x - U dt), with multilinear interpolation, i.e. the CIR
 * scheme (Sec. 3 in 1D, eq. CIR2D in 2D, the same tensor product in 3D).
 *
 * The departure point of cell i is X_d = i_d - dir * C_d(i): a straight-line
 * backtrace with the velocity taken at the arrival cell.  dir = +1 gives L_U,
 * dir = -1 gives L_{-U} (the reversed flow of eq. intro:FEC), which uses -u at
 * its own arrival cell.  X_d is split as floor(X_d) + f_d, f_d in [0,1), and the
 * 2^ndim corners floor(X) + b, b in {0,1}^ndim, are weighted by
 * prod_d (b_d ? f_d : 1 - f_d).  For |C| <= 1 this is the paper's
 * (1 - U) Phi[i] + U Phi[i - s] form.
 */
int orc_interp(double *out, const double *phi, const double *c,
               const int64_t n[3], int ndim, int dir)
{
    if (!out || !phi || !c || ndim < 1 || ndim > 3 || out == phi) return -1;
    const int64_t N = ncells(n);
    for (int64_t z = 0; z < n[2]; ++z)
        for (int64_t y = 0; y < n[1]; ++y)
            for (int64_t x = 0; x < n[0]; ++x) {
                const int64_t cell = (z * n[1] + y) * n[0] + x;
                const int64_t pos[3] = {x, y, z};
                int64_t base[3];
                double f[3];
                for (int d = 0; d < 3; ++d) {
                    if (d < ndim) {
                        const double X = (double)pos[d] - (double)dir * c[d * N + cell];
                        const double fl = floor(X);
                        base[d] = (int64_t)fl;
                        f[d] = X - fl;
                    } else {
                        base[d] = pos[d];
                        f[d] = 0.0;
                    }
                }
                double sum = 0.0;
                for (int b = 0; b < (1 << ndim); ++b) {
                    double w = 1.0;
                    int64_t q[3] = {base[0], base[1], base[2]};
                    for (int d = 0; d < ndim; ++d) {
                        const int bit = (b >> d) & 1;
                        w *= bit ? f[d] : 1.0 - f[d];
                        q[d] += bit;
                    }
                    sum += w * phi[at(n, q[0], q[1], q[2])];
                }
                out[cell] = sum;
            }
    return 0;
}

/*
 * One-dimensional interpolation along a single axis (the directional sweep of
 * eqs. split:1 and split:2): the departure point moves along `axis` only,
 * X = i_axis - dir * ca(i), and the value is the linear interpolation between
 * the two bracketing cells of that grid line.
 */
int orc_interp_axis(double *out, const double *phi, const double *ca,
                    const int64_t n[3], int axis, int dir)
{
    if (!out || !phi || !ca || axis < 0 || axis > 2 || out == phi) return -1;
    for (int64_t z = 0; z < n[2]; ++z)
        for (int64_t y = 0; y < n[1]; ++y)
            for (int64_t x = 0; x < n[0]; ++x) {
                const int64_t cell = (z * n[1] + y) * n[0] + x;
                const int64_t pos[3] = {x, y, z};
                const double X = (double)pos[axis] - (double)dir * ca[cell];
                const double fl = floor(X);
                const double f = X - fl;
                int64_t p0[3] = {x, y, z}, p1[3] = {x, y, z};
                p0[axis] = (int64_t)fl;
                p1[axis] = (int64_t)fl + 1;
                out[cell] = (1.0 - f) * phi[at(n, p0[0], p0[1], p0[2])] +
                            f * phi[at(n, p1[0], p1[1], p1[2])];
            }
    return 0;
}

/* A generic interpolation call: axis < 0 means the multilinear operator on all
 * ndim axes, otherwise the 1D operator along that axis. */
static int interp(double *out, const double *phi, const double *c,
                  const int64_t n[3], int ndim, int axis, int dir)
{
    if (axis < 0) return orc_interp(out, phi, c, n, ndim, dir);
    return orc_interp_axis(out, phi, c + (int64_t)axis * ncells(n), n, axis, dir);
}

/*
 * FEC, BEC and CEC built from calls of the interpolation operator.
 *   Phi_bar = L_{-U}[L_U[Phi]]                         (Sec. 2, eq. intro:FEC)
 *   FEC     = L_U[Phi] + (Phi - Phi_bar) / 2            (eq. intro:FEC)
 *   BEC     = L_U[Phi + (Phi - Phi_bar) / 2]            (eq. intro:BEC)
 *   CEC     = a FEC + b BEC, 3a = 2 - dx/(|u| dt),
 *             b = 1 - a                                 (eqs. intro:CEC, intro:CECcoef)
 * CEC has coefficients only in one dimension (Sec. 5), so it is only defined
 * for a single-axis sweep here (axis >= 0).  The per-cell coefficients use the
 * reduced velocity U_i = |C(i)| of the output cell.
 *
 * ORC_CEC_DEF evaluates a FEC + b BEC literally.  It is singular at U = 0 and
 * loses accuracy as U -> 0 (a and b grow like 1/U), so it only serves to pin
 * ORC_CEC.  ORC_CEC evaluates the same combination with the 1/U divided out:
 * with L the 1D CIR operator, BEC - FEC = (L[delta] - delta)/2 (linearity of
 * L) and L[delta]_i - delta_i = U_i (delta_{i-s_i} - delta_i) (Sec. 3 CIR form),
 * so CEC_i = FEC_i + b_i (BEC_i - FEC_i) = FEC_i + (1 + U_i)/6 (delta_{i-s_i}
 * - delta_i), s_i = sgn C(i).  At U_i = 0, FEC_i = BEC_i and the combination
 * equals that common value for any a + b = 1 (s_i = 0 gives exactly that).
 *
 * Large Courant numbers (Sec. 4, eq. intro:CECcoefSL).  L_U above is already
 * non-local: its corners bracket the departure point however far it is.  The
 * CEC weights then come from the fractional part of U: 3a = 2 - 1/(U % 1),
 * b = 1 - a.  Where the correction terms are taken is not stated; two readings
 * (1D sweeps only, like ORC_CEC):
 *   ORC_CEC_SL_LIT  the operator definitions unchanged, a FEC + b BEC with
 *                   FEC = L_U[Phi] + delta/2 and BEC = L_U[Phi + delta/2],
 *                   delta at the arrival cell.  Where U % 1 = 0 it takes FEC
 *                   (L_U is then an exact shift, delta = 0 and FEC = BEC).
 *   ORC_CEC_SL      the local scheme's correction taken at the departure cell:
 *                   with m = trunc(C) and r = C - m, j = i - m, s = sgn r,
 *                   CEC_i = L_U[Phi]_i + delta_j/2 + (1 + |r|)/6 (delta_{j-s} - delta_j).
 *                   For constant velocity this is the local CEC at Courant
 *                   number r shifted by m cells, so the scheme stays third
 *                   order (the literal reading falls to second order); for
 *                   |C| < 1 (m = 0) it is ORC_CEC term for term.
 */
int orc_scheme_on(double *out, const double *phi, const double *c,
                  const int64_t n[3], int ndim, int axis, int scheme)
{
    const int64_t N = ncells(n);
    if (!out || !phi || !c || out == phi) return -1;
    if (scheme == ORC_CIR) return interp(out, phi, c, n, ndim, axis, +1);
    if (scheme >= ORC_CEC && axis < 0) return -1;
    if (scheme < 0 || scheme > ORC_CEC_SL_LIT) return -1;

    double *lphi = malloc(sizeof(double) * N);   /* L_U[Phi]           */
    double *bar = malloc(sizeof(double) * N);    /* Phi_bar            */
    double *tmp = malloc(sizeof(double) * N);
    double *tmp2 = malloc(sizeof(double) * N);
    if (!lphi || !bar || !tmp || !tmp2) {
        free(lphi); free(bar); free(tmp); free(tmp2);
        return -2;
    }
    interp(lphi, phi, c, n, ndim, axis, +1);
    interp(bar, lphi, c, n, ndim, axis, -1);

    if (scheme == ORC_FEC) {
        for (int64_t i = 0; i < N; ++i) out[i] = lphi[i] + (phi[i] - bar[i]) / 2.0;
    } else if (scheme == ORC_BEC) {
        for (int64_t i = 0; i < N; ++i) tmp[i] = phi[i] + (phi[i] - bar[i]) / 2.0;
        interp(out, tmp, c, n, ndim, axis, +1);
    } else if (scheme == ORC_CEC_DEF) {
        const double *ca = c + (int64_t)axis * N;
        for (int64_t i = 0; i < N; ++i) tmp[i] = phi[i] + (phi[i] - bar[i]) / 2.0;
        interp(tmp2, tmp, c, n, ndim, axis, +1);              /* BEC */
        for (int64_t i = 0; i < N; ++i) {
            const double fec = lphi[i] + (phi[i] - bar[i]) / 2.0;
            const double U = fabs(ca[i]);
            const double a = (2.0 - 1.0 / U) / 3.0;
            const double b = 1.0 - a;
            out[i] = a * fec + b * tmp2[i];
        }
    } else if (scheme == ORC_CEC_SL_LIT) {
        const double *ca = c + (int64_t)axis * N;
        for (int64_t i = 0; i < N; ++i) tmp[i] = phi[i] + (phi[i] - bar[i]) / 2.0;
        interp(tmp2, tmp, c, n, ndim, axis, +1);              /* BEC */
        for (int64_t i = 0; i < N; ++i) {
            const double fec = lphi[i] + (phi[i] - bar[i]) / 2.0;
            const double f = fmod(fabs(ca[i]), 1.0);
            if (f == 0.0) {
                out[i] = fec;
            } else {
                const double a = (2.0 - 1.0 / f) / 3.0;
                out[i] = a * fec + (1.0 - a) * tmp2[i];
            }
        }
    } else if (scheme == ORC_CEC_SL) {
        const double *ca = c + (int64_t)axis * N;
        for (int64_t i = 0; i < N; ++i) tmp[i] = phi[i] - bar[i];   /* delta */
        for (int64_t z = 0; z < n[2]; ++z)
            for (int64_t y = 0; y < n[1]; ++y)
                for (int64_t x = 0; x < n[0]; ++x) {
                    const int64_t i = (z * n[1] + y) * n[0] + x;
                    const double C = ca[i];
                    const double m = trunc(C), r = C - m;
                    const int s = (r > 0.0) - (r < 0.0);
                    int64_t qj[3] = {x, y, z}, qu[3] = {x, y, z};
                    qj[axis] -= (int64_t)m;
                    qu[axis] -= (int64_t)m + s;
                    const double dj = tmp[at(n, qj[0], qj[1], qj[2])];
                    const double du = tmp[at(n, qu[0], qu[1], qu[2])];
                    out[i] = lphi[i] + dj / 2.0 + (1.0 + fabs(r)) / 6.0 * (du - dj);
                }
    } else { /* ORC_CEC */
        const double *ca = c + (int64_t)axis * N;
        for (int64_t i = 0; i < N; ++i) tmp[i] = phi[i] - bar[i];   /* delta */
        for (int64_t z = 0; z < n[2]; ++z)
            for (int64_t y = 0; y < n[1]; ++y)
                for (int64_t x = 0; x < n[0]; ++x) {
                    const int64_t i = (z * n[1] + y) * n[0] + x;
                    const double C = ca[i];
                    const double U = fabs(C);
                    const int s = (C > 0.0) - (C < 0.0);
                    int64_t q[3] = {x, y, z};
                    q[axis] -= s;
                    const double d_up = tmp[at(n, q[0], q[1], q[2])];
                    const double fec = lphi[i] + tmp[i] / 2.0;
                    out[i] = fec + (1.0 + U) / 6.0 * (d_up - tmp[i]);
                }
    }
    free(lphi); free(bar); free(tmp); free(tmp2);
    return 0;
}

/*
 * One time step of a scheme on the whole grid.
 *   CIR, FEC, BEC: the unsplit multilinear operator on all ndim axes
 *                  (Sec. 5, eq. CIR2D, composed as in Sec. 2).
 *   CEC:           directionally split (Sec. 2 last paragraph, Sec. 5
 *                  eqs. split:1-2): one 1D CEC sweep per axis, each on the
 *                  result of the previous sweep.  Reading of Sec. 5 (a simple
 *                  split is only first order; a symmetric splitting is
 *                  needed): the sweep order alternates between steps,
 *                  x, y, z when parity is even and z, y, x when it is odd.
 */
int orc_step(double *out, const double *phi, const double *c,
             const int64_t n[3], int ndim, int scheme, int parity)
{
    const int64_t N = ncells(n);
    if (!out || !phi || !c || out == phi || ndim < 1 || ndim > 3) return -1;
    if (scheme != ORC_CEC && scheme != ORC_CEC_SL && scheme != ORC_CEC_SL_LIT)
        return orc_scheme_on(out, phi, c, n, ndim, -1, scheme);

    double *a = malloc(sizeof(double) * N);
    double *b = malloc(sizeof(double) * N);
    if (!a || !b) { free(a); free(b); return -2; }
    memcpy(a, phi, sizeof(double) * N);
    for (int k = 0; k < ndim; ++k) {
        const int axis = (parity & 1) ? ndim - 1 - k : k;
        orc_scheme_on(b, a, c, n, ndim, axis, scheme);
        double *t = a; a = b; b = t;
    }
    memcpy(out, a, sizeof(double) * N);
    free(a); free(b);
    return 0;
}

/*
 * The result of orc_step at a list of cells, without computing the whole
 * grid.  For |C| <= 1 every scheme here reads Phi at most 3 cells and the
 * velocity at most 2 cells away from the output cell along each axis, so the
 * result at a cell equals the result, at the centre, of the same step on the
 * 7^ndim window around it treated as a periodic grid: the wrap-around inside
 * the window only changes intermediate values that the centre never reads.
 * cells holds ns (x, y, z) triples.  Returns -3, computing nothing, if any
 * |C| > 1 (the window would be too narrow).
 */
int orc_sample(double *out, const double *phi, const double *c,
               const int64_t n[3], int ndim, int scheme, int parity,
               const int64_t *cells, int64_t ns)
{
    enum { R = 3, W = 2 * R + 1 };
    if (!out || !phi || !c || !cells || ndim < 1 || ndim > 3) return -1;
    const int64_t N = ncells(n);
    for (int64_t i = 0; i < N * ndim; ++i)
        if (fabs(c[i]) > 1.0) return -3;
    int64_t wn[3] = {1, 1, 1};
    for (int d = 0; d < ndim; ++d) wn[d] = W;
    const int64_t WN = wn[0] * wn[1] * wn[2];
    double *wp = malloc(sizeof(double) * WN);
    double *wc = malloc(sizeof(double) * WN * ndim);
    double *wo = malloc(sizeof(double) * WN);
    if (!wp || !wc || !wo) { free(wp); free(wc); free(wo); return -2; }
    int rc = 0;
    for (int64_t s = 0; s < ns && rc == 0; ++s) {
        const int64_t cx = cells[3 * s], cy = cells[3 * s + 1], cz = cells[3 * s + 2];
        for (int64_t k = 0; k < wn[2]; ++k)
            for (int64_t j = 0; j < wn[1]; ++j)
                for (int64_t i = 0; i < wn[0]; ++i) {
                    const int64_t gx = ndim > 0 ? cx + i - R : cx;
                    const int64_t gy = ndim > 1 ? cy + j - R : cy;
                    const int64_t gz = ndim > 2 ? cz + k - R : cz;
                    const int64_t g = at(n, gx, gy, gz);
                    const int64_t w = (k * wn[1] + j) * wn[0] + i;
                    wp[w] = phi[g];
                    for (int d = 0; d < ndim; ++d) wc[d * WN + w] = c[d * N + g];
                }
        rc = orc_step(wo, wp, wc, wn, ndim, scheme, parity);
        const int64_t ci = ndim > 0 ? R : 0, cj = ndim > 1 ? R : 0, ck = ndim > 2 ? R : 0;
        out[s] = wo[(ck * wn[1] + cj) * wn[0] + ci];
    }
    free(wp); free(wc); free(wo);
    return rc;
}

/* Discrete error norms (FP64 accumulation): out[0] = RMS of a - b,
 * out[1] = max |a - b|, out[2] = ||a - b||_2 / ||b||_2. */
int orc_norms(double out[3], const double *a, const double *b, int64_t n)
{
    if (!out || !a || !b || n <= 0) return -1;
    double s2 = 0.0, m = 0.0, r2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double d = a[i] - b[i];
        s2 += d * d;
        r2 += b[i] * b[i];
        if (fabs(d) > m) m = fabs(d);
    }
    out[0] = sqrt(s2 / (double)n);
    out[1] = m;
    out[2] = r2 > 0.0 ? sqrt(s2 / r2) : sqrt(s2);
    return 0;
}
