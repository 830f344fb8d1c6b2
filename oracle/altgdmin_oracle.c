/*
 * altgdmin_oracle.c -- plain FP64 CPU oracle for the altGDmin hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the package smoke check
 * and the benchmark's CPU-baseline leg, never by the product path.  It shares
 * no code with the CUDA library.
 *
 * Every routine follows the paper's definitions directly, in the paper's order:
 *   - measurement model y_k = A_k z_k, A_k = [H_k F D_j]_j       (Sec. II-A)
 *   - auto-altGDmin initialisation and iterations                 (Alg. 2)
 *   - subspace distance SD(U1, U2) = ||(I - U1 U1^H) U2||_F       (Sec. II-A)
 * The only liberties taken are exact ones: a naive DFT that skips rows known
 * to be zero (adding zero terms changes nothing) and computes only the output
 * rows that are sampled, and A_k U assembled from F(d_j o u_l) computed once
 * per call (the same numbers as recomputing them per frame).
 *
 * Readings of points the paper leaves open (stated in the design notes):
 *   - DFT is unitary, exp(-2 pi i k x / N) forward, DC at index 0;
 *   - "^T" is the conjugate transpose;
 *   - gamma's denominator "mq" is the number of measured entries nc * sum m_k;
 *   - truncation keeps |y|^2 <= gamma (inclusive, complex modulus);
 *   - ||grad|| in the step size is the spectral norm;
 *   - the rank cap min(n, q, nc min_k m_k)/10 is floored and at least 1;
 *   - QR factors have real positive diag(R), which makes Q unique.
 */
#include "altgdmin_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846264338327950288

static orc_cx *cx_alloc(size_t n) { return (orc_cx *)calloc(n ? n : 1, sizeof(orc_cx)); }
static int64_t frame_m(const orc_problem *P, int k) { return P->fp[k + 1] - P->fp[k]; }
static int frame_n(const orc_problem *P) { return P->ny * P->nx; }
static double cabs2(orc_cx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* ------------------------------------------------------------------------ */
/* Naive DFT                                                                 */
/* ------------------------------------------------------------------------ */

/* w[t] = exp(sign * 2 pi i t / N) for t in [0, N). */
static void twiddle_table(int N, int sign, orc_cx *w)
{
    for (int t = 0; t < N; ++t) {
        double a = 2.0 * ORC_PI * (double)t / (double)N;
        w[t] = cos(a) + I * ((double)sign * sin(a));
    }
}

/*
 * out = F2 in (unitary 2D DFT, sign -1) or F2^H in (sign +1), computed as the
 * 1D DFT along x of every row and then the 1D DFT along y of every column:
 *     out[ky, kx] = 1/sqrt(ny nx) sum_y sum_x in[y, x] w_y^(ky y) w_x^(kx x).
 * in_rows (may be NULL): rows of `in` that can be non-zero; other rows are
 * skipped, which only drops zero terms.  out_rows (may be NULL): output rows
 * wanted; the others are set to zero.
 */
static void dft2_rows(const orc_cx *in, orc_cx *out, int ny, int nx, int sign,
                      const unsigned char *in_rows, const unsigned char *out_rows)
{
    orc_cx *wx = cx_alloc(nx), *wy = cx_alloc(ny);
    orc_cx *tmp = cx_alloc((size_t)ny * nx);
    twiddle_table(nx, sign, wx);
    twiddle_table(ny, sign, wy);
    const double sx = 1.0 / sqrt((double)nx), sy = 1.0 / sqrt((double)ny);
    for (int y = 0; y < ny; ++y) {
        if (in_rows && !in_rows[y]) continue;
        const orc_cx *a = in + (size_t)y * nx;
        orc_cx *b = tmp + (size_t)y * nx;
        for (int kx = 0; kx < nx; ++kx) {
            orc_cx acc = 0;
            for (int x = 0; x < nx; ++x) acc += a[x] * wx[(int)(((int64_t)kx * x) % nx)];
            b[kx] = acc * sx;
        }
    }
    orc_cx *col = cx_alloc(ny);
    for (int kx = 0; kx < nx; ++kx) {
        for (int y = 0; y < ny; ++y) col[y] = tmp[(size_t)y * nx + kx];
        for (int ky = 0; ky < ny; ++ky) {
            orc_cx acc = 0;
            if (!out_rows || out_rows[ky]) {
                for (int y = 0; y < ny; ++y) {
                    if (in_rows && !in_rows[y]) continue;
                    acc += col[y] * wy[(int)(((int64_t)ky * y) % ny)];
                }
            }
            out[(size_t)ky * nx + kx] = acc * sy;
        }
    }
    free(col);
    free(tmp);
    free(wy);
    free(wx);
}

void orc_dft2(const orc_cx *in, orc_cx *out, int ny, int nx, int sign)
{
    dft2_rows(in, out, ny, nx, sign, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* Measurement operator A_k and its adjoint (Sec. II-A)                     */
/* ------------------------------------------------------------------------ */

static unsigned char *frame_rows(const orc_problem *P, int k)
{
    unsigned char *rows = (unsigned char *)calloc((size_t)P->ny, 1);
    const int32_t *id = P->idx + P->fp[k];
    for (int64_t s = 0; s < frame_m(P, k); ++s) rows[id[s] / P->nx] = 1;
    return rows;
}

/* y_k = [H_k F (d_j o x)]_j, coil j's m_k samples at y_k + j * m_k. */
void orc_forward(const orc_problem *P, int k, const orc_cx *x, orc_cx *yk)
{
    const int n = frame_n(P);
    const int64_t mk = frame_m(P, k);
    if (P->kind == ORC_KIND_DENSE) {
        const orc_cx *A = P->dense + (size_t)n * P->fp[k];
        for (int64_t s = 0; s < mk; ++s) {
            orc_cx acc = 0;
            for (int i = 0; i < n; ++i) acc += A[(size_t)s * n + i] * x[i];
            yk[s] = acc;
        }
        return;
    }
    const int32_t *id = P->idx + P->fp[k];
    unsigned char *rows = frame_rows(P, k);
    orc_cx *t = cx_alloc(n), *f = cx_alloc(n);
    for (int j = 0; j < P->nc; ++j) {
        const orc_cx *d = P->smaps + (size_t)j * n;
        for (int i = 0; i < n; ++i) t[i] = d[i] * x[i];
        dft2_rows(t, f, P->ny, P->nx, -1, NULL, rows);
        for (int64_t s = 0; s < mk; ++s) yk[j * mk + s] = f[id[s]];
    }
    free(f);
    free(t);
    free(rows);
}

/* x = A_k^H y_k = sum_j conj(d_j) o F^H (H_k^T y_kj). */
void orc_adjoint(const orc_problem *P, int k, const orc_cx *yk, orc_cx *x)
{
    const int n = frame_n(P);
    const int64_t mk = frame_m(P, k);
    if (P->kind == ORC_KIND_DENSE) {
        const orc_cx *A = P->dense + (size_t)n * P->fp[k];
        for (int i = 0; i < n; ++i) x[i] = 0;
        for (int64_t s = 0; s < mk; ++s)
            for (int i = 0; i < n; ++i) x[i] += conj(A[(size_t)s * n + i]) * yk[s];
        return;
    }
    const int32_t *id = P->idx + P->fp[k];
    unsigned char *rows = frame_rows(P, k);
    orc_cx *z = cx_alloc(n), *f = cx_alloc(n);
    for (int i = 0; i < n; ++i) x[i] = 0;
    for (int j = 0; j < P->nc; ++j) {
        for (int i = 0; i < n; ++i) z[i] = 0;
        for (int64_t s = 0; s < mk; ++s) z[id[s]] = yk[j * mk + s];
        dft2_rows(z, f, P->ny, P->nx, +1, rows, NULL);
        const orc_cx *d = P->smaps + (size_t)j * n;
        for (int i = 0; i < n; ++i) x[i] += conj(d[i]) * f[i];
    }
    free(f);
    free(z);
    free(rows);
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra: Hermitian Jacobi, Householder QR and least squares */
/* ------------------------------------------------------------------------ */

/*
 * Cyclic Jacobi for a Hermitian matrix.  Each rotation first removes the phase
 * of a_pq with diag(1, e^{-i phi}) and then applies the real symmetric 2x2
 * Jacobi rotation [[c, s], [-s, c]] (t = sgn(tau)/(|tau| + sqrt(1 + tau^2)),
 * tau = (a_qq - a_pp) / (2 |a_pq|)), i.e. G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]],
 * A <- G^H A G, V <- V G.
 */
int orc_eigh(const orc_cx *A0, int q, double *w, orc_cx *V)
{
    orc_cx *A = cx_alloc((size_t)q * q);
    memcpy(A, A0, sizeof(orc_cx) * (size_t)q * q);
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) V[(size_t)i * q + j] = (i == j) ? 1.0 : 0.0;
    int sweep;
    for (sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < q; ++i)
            for (int j = 0; j < q; ++j) {
                double a2 = cabs2(A[(size_t)i * q + j]);
                tot += a2;
                if (i != j) off += a2;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < q - 1; ++p) {
            for (int r = p + 1; r < q; ++r) {
                orc_cx apr = A[(size_t)p * q + r];
                double b = cabs(apr);
                if (b < 1e-300) continue;
                orc_cx e = apr / b;          /* e^{i phi} */
                orc_cx eh = conj(e);         /* e^{-i phi} */
                double alpha = creal(A[(size_t)p * q + p]);
                double gam = creal(A[(size_t)r * q + r]);
                double tau = (gam - alpha) / (2.0 * b);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                for (int m = 0; m < q; ++m) {          /* rows: A <- G^H A */
                    orc_cx ap = A[(size_t)p * q + m], ar = A[(size_t)r * q + m];
                    A[(size_t)p * q + m] = c * ap - s * e * ar;
                    A[(size_t)r * q + m] = s * ap + c * e * ar;
                }
                for (int m = 0; m < q; ++m) {          /* columns: A <- A G */
                    orc_cx ap = A[(size_t)m * q + p], ar = A[(size_t)m * q + r];
                    A[(size_t)m * q + p] = c * ap - s * eh * ar;
                    A[(size_t)m * q + r] = s * ap + c * eh * ar;
                }
                A[(size_t)p * q + r] = 0;
                A[(size_t)r * q + p] = 0;
                A[(size_t)p * q + p] = creal(A[(size_t)p * q + p]);
                A[(size_t)r * q + r] = creal(A[(size_t)r * q + r]);
                for (int m = 0; m < q; ++m) {          /* V <- V G */
                    orc_cx vp = V[(size_t)m * q + p], vr = V[(size_t)m * q + r];
                    V[(size_t)m * q + p] = c * vp - s * eh * vr;
                    V[(size_t)m * q + r] = s * vp + c * eh * vr;
                }
            }
        }
    }
    for (int i = 0; i < q; ++i) w[i] = creal(A[(size_t)i * q + i]);
    /* sort descending, carrying the eigenvectors */
    for (int i = 0; i < q; ++i) {
        int best = i;
        for (int j = i + 1; j < q; ++j)
            if (w[j] > w[best]) best = j;
        if (best != i) {
            double tw = w[i];
            w[i] = w[best];
            w[best] = tw;
            for (int m = 0; m < q; ++m) {
                orc_cx tv = V[(size_t)m * q + i];
                V[(size_t)m * q + i] = V[(size_t)m * q + best];
                V[(size_t)m * q + best] = tv;
            }
        }
    }
    free(A);
    return sweep;
}

/*
 * Householder reduction of W (m x r, row-major) in place; the reflector of
 * column c is H_c = I - beta_c v_c v_c^H with v_c stored in Vh[:, c] (rows
 * c..m-1), chosen so that H_c W[c:, c] = alpha e_1, alpha = -e^{i arg w_cc} ||W[c:, c]||.
 * The same reflectors are applied to z (length m) when z != NULL.
 * Returns -1 if a column is (numerically) zero.
 */
static int householder(orc_cx *W, int m, int r, orc_cx *Vh, double *beta, orc_cx *z)
{
    for (int c = 0; c < r; ++c) {
        double nrm2 = 0.0;
        for (int i = c; i < m; ++i) nrm2 += cabs2(W[(size_t)i * r + c]);
        double nrm = sqrt(nrm2);
        if (!(nrm > 0.0)) return -1;
        orc_cx x0 = W[(size_t)c * r + c];
        double ax0 = cabs(x0);
        orc_cx ph = ax0 > 0.0 ? x0 / ax0 : 1.0;
        orc_cx alpha = -ph * nrm;
        double vn2 = 0.0;
        for (int i = c; i < m; ++i) {
            orc_cx v = W[(size_t)i * r + c] - (i == c ? alpha : 0.0);
            Vh[(size_t)i * r + c] = v;
            vn2 += cabs2(v);
        }
        beta[c] = vn2 > 0.0 ? 2.0 / vn2 : 0.0;
        for (int cc = c; cc < r; ++cc) {
            orc_cx s = 0;
            for (int i = c; i < m; ++i) s += conj(Vh[(size_t)i * r + c]) * W[(size_t)i * r + cc];
            s *= beta[c];
            for (int i = c; i < m; ++i) W[(size_t)i * r + cc] -= s * Vh[(size_t)i * r + c];
        }
        if (z) {
            orc_cx s = 0;
            for (int i = c; i < m; ++i) s += conj(Vh[(size_t)i * r + c]) * z[i];
            s *= beta[c];
            for (int i = c; i < m; ++i) z[i] -= s * Vh[(size_t)i * r + c];
        }
    }
    return 0;
}

int orc_qr(const orc_cx *A, int m, int r, orc_cx *Q, orc_cx *R)
{
    if (m < r || r <= 0) return -1;
    orc_cx *W = cx_alloc((size_t)m * r), *Vh = cx_alloc((size_t)m * r);
    double *beta = (double *)calloc((size_t)r, sizeof(double));
    memcpy(W, A, sizeof(orc_cx) * (size_t)m * r);
    int rc = householder(W, m, r, Vh, beta, NULL);
    if (rc == 0) {
        /* Q = H_0 H_1 ... H_{r-1} [I_r; 0] */
        for (int i = 0; i < m; ++i)
            for (int c = 0; c < r; ++c) Q[(size_t)i * r + c] = (i == c) ? 1.0 : 0.0;
        for (int c = r - 1; c >= 0; --c) {
            for (int cc = 0; cc < r; ++cc) {
                orc_cx s = 0;
                for (int i = c; i < m; ++i) s += conj(Vh[(size_t)i * r + c]) * Q[(size_t)i * r + cc];
                s *= beta[c];
                for (int i = c; i < m; ++i) Q[(size_t)i * r + cc] -= s * Vh[(size_t)i * r + c];
            }
        }
        for (int a = 0; a < r; ++a)
            for (int b = 0; b < r; ++b) R[(size_t)a * r + b] = (b >= a) ? W[(size_t)a * r + b] : 0.0;
        /* Q <- Q D, R <- D^H R with D = diag(e^{i arg r_cc}): diag(R) real positive */
        for (int c = 0; c < r; ++c) {
            orc_cx d = R[(size_t)c * r + c];
            double ad = cabs(d);
            if (!(ad > 0.0)) { rc = -1; break; }
            orc_cx ph = d / ad;
            for (int i = 0; i < m; ++i) Q[(size_t)i * r + c] *= ph;
            for (int b = 0; b < r; ++b) R[(size_t)c * r + b] *= conj(ph);
            R[(size_t)c * r + c] = ad;
        }
    }
    free(beta);
    free(Vh);
    free(W);
    return rc;
}

int orc_lstsq(const orc_cx *M, int m, int r, const orc_cx *y, orc_cx *b)
{
    if (m < r || r <= 0) return -1;
    orc_cx *W = cx_alloc((size_t)m * r), *Vh = cx_alloc((size_t)m * r), *z = cx_alloc(m);
    double *beta = (double *)calloc((size_t)r, sizeof(double));
    memcpy(W, M, sizeof(orc_cx) * (size_t)m * r);
    memcpy(z, y, sizeof(orc_cx) * (size_t)m);
    int rc = householder(W, m, r, Vh, beta, z);
    if (rc == 0) {
        for (int c = r - 1; c >= 0; --c) {     /* R b = (Q^H y)[0:r] */
            orc_cx acc = z[c];
            for (int cc = c + 1; cc < r; ++cc) acc -= W[(size_t)c * r + cc] * b[cc];
            b[c] = acc / W[(size_t)c * r + c];
        }
    }
    free(beta);
    free(z);
    free(Vh);
    free(W);
    return rc;
}

double orc_sd(const orc_cx *U1, const orc_cx *U2, int n, int r)
{
    /* D = U2 - U1 (U1^H U2), SD = ||D||_F */
    orc_cx *C = cx_alloc((size_t)r * r);
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            orc_cx acc = 0;
            for (int i = 0; i < n; ++i) acc += conj(U1[(size_t)i * r + a]) * U2[(size_t)i * r + b];
            C[(size_t)a * r + b] = acc;
        }
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int b = 0; b < r; ++b) {
            orc_cx d = U2[(size_t)i * r + b];
            for (int a = 0; a < r; ++a) d -= U1[(size_t)i * r + a] * C[(size_t)a * r + b];
            s += cabs2(d);
        }
    free(C);
    return sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* A_k U for all k                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_cx *Fc;              /* MRI: F(d_j o u_l) at (j * r + l) * n, sampled rows only */
} au_cache;

static void au_build(const orc_problem *P, const orc_cx *U, int r, au_cache *c)
{
    c->Fc = NULL;
    if (P->kind != ORC_KIND_MRI) return;
    const int n = frame_n(P);
    unsigned char *rows = (unsigned char *)calloc((size_t)P->ny, 1);
    for (int64_t s = 0; s < P->fp[P->q]; ++s) rows[P->idx[s] / P->nx] = 1;
    c->Fc = cx_alloc((size_t)P->nc * r * n);
#pragma omp parallel for schedule(dynamic)
    for (int jl = 0; jl < P->nc * r; ++jl) {
        int j = jl / r, l = jl % r;
        orc_cx *t = cx_alloc(n);
        const orc_cx *d = P->smaps + (size_t)j * n;
        for (int i = 0; i < n; ++i) t[i] = d[i] * U[(size_t)i * r + l];
        dft2_rows(t, c->Fc + (size_t)jl * n, P->ny, P->nx, -1, NULL, rows);
        free(t);
    }
    free(rows);
}

static void au_free(au_cache *c) { free(c->Fc); }

/* M = A_k U, (nc * m_k) x r row-major. */
static void au_frame(const orc_problem *P, const au_cache *c, const orc_cx *U, int r, int k, orc_cx *M)
{
    const int n = frame_n(P);
    const int64_t mk = frame_m(P, k);
    if (P->kind == ORC_KIND_DENSE) {
        const orc_cx *A = P->dense + (size_t)n * P->fp[k];
        for (int64_t s = 0; s < mk; ++s)
            for (int l = 0; l < r; ++l) {
                orc_cx acc = 0;
                for (int i = 0; i < n; ++i) acc += A[(size_t)s * n + i] * U[(size_t)i * r + l];
                M[(size_t)s * r + l] = acc;
            }
        return;
    }
    const int32_t *id = P->idx + P->fp[k];
    for (int j = 0; j < P->nc; ++j)
        for (int64_t s = 0; s < mk; ++s)
            for (int l = 0; l < r; ++l)
                M[((size_t)j * mk + s) * r + l] = c->Fc[((size_t)j * r + l) * n + id[s]];
}

static int bstep_cached(const orc_problem *P, const orc_cx *y, const au_cache *c,
                        const orc_cx *U, int r, orc_cx *B)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
    for (int k = 0; k < P->q; ++k) {
        const int64_t rows = (int64_t)P->nc * frame_m(P, k);
        orc_cx *M = cx_alloc((size_t)rows * r);
        au_frame(P, c, U, r, k, M);
        if (orc_lstsq(M, (int)rows, r, y + (size_t)P->nc * P->fp[k], B + (size_t)k * r) != 0) bad = 1;
        free(M);
    }
    return bad ? -1 : 0;
}

int orc_bstep(const orc_problem *P, const orc_cx *y, const orc_cx *U, int r, orc_cx *B)
{
    au_cache c;
    au_build(P, U, r, &c);
    int rc = bstep_cached(P, y, &c, U, r, B);
    au_free(&c);
    return rc;
}

/*
 * Gradient sum_k A_k^H (A_k U b_k - y_k) b_k^H (Alg. 2, gradient step).
 * mode 0: literally, one adjoint per frame, then the sum over k in order.
 * mode 1 (MRI only): the same sum rearranged by linearity,
 *     sum_j conj(d_j) o F^H [ (F(d_j o U))[i, :] W_i ]  -  sum_k (A_k^H y_k) b_k^H,
 *     W_i = sum_{k : i in Omega_k} b_k b_k^H,
 * used to cross-check the rearrangement the GPU relies on.
 */
static void grad_cached(const orc_problem *P, const orc_cx *y, const au_cache *c,
                        const orc_cx *U, const orc_cx *B, int r, int mode, orc_cx *G)
{
    const int n = frame_n(P), q = P->q;
    for (size_t i = 0; i < (size_t)n * r; ++i) G[i] = 0;
    if (mode == 0 || P->kind != ORC_KIND_MRI) {
        orc_cx *gk = cx_alloc((size_t)q * n);
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < q; ++k) {
            const int64_t rows = (int64_t)P->nc * frame_m(P, k);
            orc_cx *M = cx_alloc((size_t)rows * r), *res = cx_alloc(rows);
            au_frame(P, c, U, r, k, M);
            const orc_cx *yk = y + (size_t)P->nc * P->fp[k];
            const orc_cx *bk = B + (size_t)k * r;
            for (int64_t s = 0; s < rows; ++s) {
                orc_cx acc = 0;
                for (int l = 0; l < r; ++l) acc += M[(size_t)s * r + l] * bk[l];
                res[s] = acc - yk[s];
            }
            orc_adjoint(P, k, res, gk + (size_t)k * n);
            free(res);
            free(M);
        }
        for (int k = 0; k < q; ++k)
            for (int i = 0; i < n; ++i)
                for (int l = 0; l < r; ++l)
                    G[(size_t)i * r + l] += gk[(size_t)k * n + i] * conj(B[(size_t)k * r + l]);
        free(gk);
        return;
    }
    /* mode 1 */
    orc_cx *W = cx_alloc((size_t)n * r * r);
    for (int k = 0; k < q; ++k) {
        const int32_t *id = P->idx + P->fp[k];
        const orc_cx *bk = B + (size_t)k * r;
        for (int64_t s = 0; s < frame_m(P, k); ++s)
            for (int a = 0; a < r; ++a)
                for (int b = 0; b < r; ++b) W[((size_t)id[s] * r + a) * r + b] += bk[a] * conj(bk[b]);
    }
    unsigned char *rows = (unsigned char *)calloc((size_t)P->ny, 1);
    for (int64_t s = 0; s < P->fp[q]; ++s) rows[P->idx[s] / P->nx] = 1;
    orc_cx *part = cx_alloc((size_t)P->nc * n * r);
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < P->nc; ++j) {
        orc_cx *K = cx_alloc(n), *f = cx_alloc(n);
        const orc_cx *d = P->smaps + (size_t)j * n;
        for (int l = 0; l < r; ++l) {
            for (int i = 0; i < n; ++i) {
                orc_cx acc = 0;
                for (int a = 0; a < r; ++a)
                    acc += c->Fc[((size_t)j * r + a) * n + i] * W[((size_t)i * r + a) * r + l];
                K[i] = acc;
            }
            dft2_rows(K, f, P->ny, P->nx, +1, rows, NULL);
            for (int i = 0; i < n; ++i) part[((size_t)j * n + i) * r + l] = conj(d[i]) * f[i];
        }
        free(f);
        free(K);
    }
    for (int j = 0; j < P->nc; ++j)
        for (size_t i = 0; i < (size_t)n * r; ++i) G[i] += part[(size_t)j * n * r + i];
    orc_cx *zk = cx_alloc(n);
    for (int k = 0; k < q; ++k) {
        orc_adjoint(P, k, y + (size_t)P->nc * P->fp[k], zk);
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < r; ++l)
                G[(size_t)i * r + l] -= zk[i] * conj(B[(size_t)k * r + l]);
    }
    free(zk);
    free(part);
    free(rows);
    free(W);
}

void orc_grad(const orc_problem *P, const orc_cx *y, const orc_cx *U,
              const orc_cx *B, int r, int mode, orc_cx *G)
{
    au_cache c;
    au_build(P, U, r, &c);
    grad_cached(P, y, &c, U, B, r, mode, G);
    au_free(&c);
}

double orc_cost(const orc_problem *P, const orc_cx *y, const orc_cx *U,
                const orc_cx *B, int r)
{
    au_cache c;
    au_build(P, U, r, &c);
    double f = 0.0;
    for (int k = 0; k < P->q; ++k) {
        const int64_t rows = (int64_t)P->nc * frame_m(P, k);
        orc_cx *M = cx_alloc((size_t)rows * r);
        au_frame(P, &c, U, r, k, M);
        const orc_cx *yk = y + (size_t)P->nc * P->fp[k];
        for (int64_t s = 0; s < rows; ++s) {
            orc_cx acc = 0;
            for (int l = 0; l < r; ++l) acc += M[(size_t)s * r + l] * B[(size_t)k * r + l];
            f += cabs2(yk[s] - acc);
        }
        free(M);
    }
    au_free(&c);
    return f;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: initialisation                                                   */
/* ------------------------------------------------------------------------ */

int orc_init(const orc_problem *P, const orc_cx *y, const orc_params *prm,
             int rank_in, int rmax, orc_cx *U0, double *sigma, orc_cx *X0_out,
             double *gamma_out)
{
    const int n = frame_n(P), q = P->q, nc = P->nc;
    const int64_t total = (int64_t)nc * P->fp[q];
    int64_t mmin = frame_m(P, 0), mmax = frame_m(P, 0);
    for (int k = 1; k < q; ++k) {
        if (frame_m(P, k) < mmin) mmin = frame_m(P, k);
        if (frame_m(P, k) > mmax) mmax = frame_m(P, k);
    }
    /* gamma = 36 * sum |y|^2 / (number of measured entries) */
    double e = 0.0;
    for (int64_t s = 0; s < total; ++s) e += cabs2(y[s]);
    const double gamma = prm->trunc_factor * e / (double)total;
    if (gamma_out) *gamma_out = gamma;
    const double mbar = (double)P->fp[q] / (double)q;

    orc_cx *X0 = cx_alloc((size_t)n * q);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < q; ++k) {
        const int64_t rows = (int64_t)nc * frame_m(P, k);
        const orc_cx *yk = y + (size_t)nc * P->fp[k];
        orc_cx *yt = cx_alloc(rows), *x = cx_alloc(n);
        double scale;
        if (prm->init_kind == 1) {          /* basic: X0 = [A_k^H y_k / m] */
            for (int64_t s = 0; s < rows; ++s) yt[s] = yk[s];
            scale = 1.0 / (double)mmax;
        } else {                            /* truncated, 1/sqrt(m_k mbar) */
            for (int64_t s = 0; s < rows; ++s) yt[s] = (cabs2(yk[s]) <= gamma) ? yk[s] : 0.0;
            scale = 1.0 / sqrt((double)frame_m(P, k) * mbar);
        }
        orc_adjoint(P, k, yt, x);
        for (int i = 0; i < n; ++i) X0[(size_t)i * q + k] = scale * x[i];
        free(x);
        free(yt);
    }
    if (X0_out) memcpy(X0_out, X0, sizeof(orc_cx) * (size_t)n * q);

    /* sigma_j^2 and right singular vectors from the q x q Gram X0^H X0 */
    orc_cx *Gm = cx_alloc((size_t)q * q), *V = cx_alloc((size_t)q * q);
    double *lam = (double *)calloc((size_t)q, sizeof(double));
    for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) {
            orc_cx acc = 0;
            for (int i = 0; i < n; ++i) acc += conj(X0[(size_t)i * q + a]) * X0[(size_t)i * q + b];
            Gm[(size_t)a * q + b] = acc;
        }
    orc_eigh(Gm, q, lam, V);
    for (int j = 0; j < q; ++j) sigma[j] = sqrt(lam[j] > 0.0 ? lam[j] : 0.0);

    int r = rank_in;
    if (r <= 0) {
        int64_t capn = n < q ? n : q;
        if (nc * mmin < capn) capn = nc * mmin;
        int cap = (int)(capn / 10);
        if (cap < 1) cap = 1;
        double tot = 0.0, acc = 0.0;
        for (int j = 0; j < cap; ++j) tot += lam[j];
        r = cap;
        for (int j = 0; j < cap; ++j) {
            acc += lam[j];
            if (acc >= prm->energy_pct / 100.0 * tot) { r = j + 1; break; }
        }
    }
    int rc = r;
    if (r > rmax || r > q || r > n || !(sigma[r - 1] > 0.0)) {
        rc = -1;
    } else {
        /* U0 = X0 V_r Sigma_r^{-1}: the top-r left singular vectors of X0 */
        orc_cx *Ut = cx_alloc((size_t)n * r), *R = cx_alloc((size_t)r * r);
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < r; ++l) {
                orc_cx acc = 0;
                for (int k = 0; k < q; ++k) acc += X0[(size_t)i * q + k] * V[(size_t)k * q + l];
                Ut[(size_t)i * r + l] = acc / sigma[l];
            }
        if (orc_qr(Ut, n, r, U0, R) != 0) rc = -1;
        free(R);
        free(Ut);
    }
    free(lam);
    free(V);
    free(Gm);
    free(X0);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: GDmin iterations                                                 */
/* ------------------------------------------------------------------------ */

static double spectral_norm(const orc_cx *G, int n, int r)
{
    orc_cx *H = cx_alloc((size_t)r * r), *V = cx_alloc((size_t)r * r);
    double *w = (double *)calloc((size_t)r, sizeof(double));
    for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) {
            orc_cx acc = 0;
            for (int i = 0; i < n; ++i) acc += conj(G[(size_t)i * r + a]) * G[(size_t)i * r + b];
            H[(size_t)a * r + b] = acc;
        }
    orc_eigh(H, r, w, V);
    double s = sqrt(w[0] > 0.0 ? w[0] : 0.0);
    free(w);
    free(V);
    free(H);
    return s;
}

int orc_iterate(const orc_problem *P, const orc_cx *y, const orc_params *prm,
                orc_cx *U, int r, int n_iter, double *eta, orc_cx *B,
                orc_cx *Uprev, orc_cx *X_hist, double *sd, double *gnorm)
{
    const int n = frame_n(P), q = P->q;
    orc_cx *Uold = cx_alloc((size_t)n * r), *G = cx_alloc((size_t)n * r);
    orc_cx *Up = cx_alloc((size_t)n * r), *R = cx_alloc((size_t)r * r);
    int t, rc = 0, passed = 0;
    for (t = 0; t < n_iter; ++t) {
        memcpy(Uold, U, sizeof(orc_cx) * (size_t)n * r);
        au_cache c;
        au_build(P, Uold, r, &c);
        if (bstep_cached(P, y, &c, Uold, r, B) != 0) { au_free(&c); rc = -2; break; }
        if (X_hist) {
            orc_cx *X = X_hist + (size_t)t * n * q;
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < q; ++k) {
                    orc_cx acc = 0;
                    for (int l = 0; l < r; ++l) acc += Uold[(size_t)i * r + l] * B[(size_t)k * r + l];
                    X[(size_t)i * q + k] = acc;
                }
        }
        grad_cached(P, y, &c, Uold, B, r, prm->grad_mode, G);
        au_free(&c);
        double gn;
        if (prm->frob_eta) {
            double s = 0.0;
            for (size_t i = 0; i < (size_t)n * r; ++i) s += cabs2(G[i]);
            gn = sqrt(s);
        } else {
            gn = spectral_norm(G, n, r);
        }
        if (gnorm) gnorm[t] = gn;
        if (*eta <= 0.0) *eta = prm->eta_c / gn;
        /* the step of this iteration: eta, or the variable step size
           eta * scale0 * decay^(t_offset + t) of the tuning notes */
        const double s0 = prm->eta_scale0 > 0.0 ? prm->eta_scale0 : 1.0;
        const double dk = prm->eta_decay > 0.0 ? prm->eta_decay : 1.0;
        const double eta_t = (*eta) * s0 * pow(dk, (double)(prm->t_offset + t));
        for (size_t i = 0; i < (size_t)n * r; ++i) Up[i] = Uold[i] - eta_t * G[i];
        if (orc_qr(Up, n, r, U, R) != 0) { rc = -3; break; }
        double d = orc_sd(Uold, U, n, r);
        if (sd) sd[t] = d;
        if (Uprev) memcpy(Uprev, Uold, sizeof(orc_cx) * (size_t)n * r);
        if (prm->exit_enabled) {
            /* Alg. 2's exit test; with exit_patience > 1 it must pass that many
               consecutive iterations (the robust exit of the tuning notes) */
            passed = d / sqrt((double)r) < prm->eps_exit ? passed + 1 : 0;
            if (passed >= (prm->exit_patience > 1 ? prm->exit_patience : 1)) { ++t; break; }
        }
    }
    free(R);
    free(Up);
    free(G);
    free(Uold);
    return rc < 0 ? rc : t;
}
