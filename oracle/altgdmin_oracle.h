/*
 * altgdmin_oracle.h -- FP64 CPU oracle for the altGDmin hot path
 * (Babu, Lingala, Vaswani, "Fast Low Rank column-wise Compressive Sensing for
 * Accelerated Dynamic MRI", Alg. 2 with the measurement model of Sec. II-A).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two agree only through
 * their outputs on the same inputs.
 *
 * Conventions
 *   complex numbers  : C99 double complex
 *   DFT              : unitary, forward kernel exp(-2 pi i k x / N), DC at index 0
 *   k-space index    : i = ky * nx + kx; pixel index i = y * nx + x
 *   U (n x r)        : row-major, element (i, l) at U[i * r + l]
 *   B (r x q)        : column-major, b_k contiguous, element (l, k) at B[k * r + l]
 *   X (n x q)        : row-major, element (i, k) at X[i * q + k]
 *   y (ragged)       : frame k, coil j, sample s at y[nc * fp[k] + j * m_k + s],
 *                      m_k = fp[k+1] - fp[k]
 */
#ifndef ALTGDMIN_ORACLE_H
#define ALTGDMIN_ORACLE_H

#include <complex.h>
#include <stdint.h>

typedef double _Complex orc_cx;

enum { ORC_KIND_MRI = 0, ORC_KIND_DENSE = 1 };

typedef struct orc_problem {
    int32_t kind;           /* ORC_KIND_MRI or ORC_KIND_DENSE */
    int32_t ny, nx, q, nc;  /* image ny x nx, q frames, nc coils (DENSE: nc = 1) */
    const orc_cx *smaps;    /* MRI: nc * n coil sensitivities d_j */
    const int32_t *idx;     /* MRI: sorted sample indices, frame k at idx[fp[k] .. fp[k+1]) */
    const int64_t *fp;      /* q + 1 per-coil sample offsets */
    const orc_cx *dense;    /* DENSE: A_k (m_k x n, row-major) at dense + n * fp[k] */
} orc_problem;

typedef struct orc_params {
    double trunc_factor;    /* 36      (Alg. 2, line 5: gamma = 36 sum |y|^2 / (m q)) */
    double energy_pct;      /* 85      (Alg. 2, rank rule, b = 85) */
    double eta_c;           /* 0.14    (Alg. 2, eta = 0.14 / ||grad||) */
    double eps_exit;        /* 0.01    (Alg. 2, exit test) */
    int32_t init_kind;      /* 0 = auto-altGDmin init (Alg. 2), 1 = basic init X0 = [A_k^H y_k / m] */
    int32_t exit_enabled;   /* 1 = stop when SD(U, U+)/sqrt(r) < eps_exit */
    int32_t frob_eta;       /* 0 = spectral norm in eta (default), 1 = Frobenius */
    int32_t grad_mode;      /* 0 = per-frame literal adjoint, 1 = summed over frames in k-space */
    /* tuning variants of the discussion section (defaults give Alg. 2 as printed) */
    int32_t exit_patience;  /* exit only after this many consecutive iterations pass the exit
                               test (robust exit); <= 1 = the first one (Alg. 2) */
    double eta_scale0;      /* variable step size: eta_t = eta * eta_scale0 * eta_decay^(t_offset + t - 1), */
    double eta_decay;       /*   t = 1, 2, ... within a call; 1 and 1 = the constant eta of Alg. 2 */
    int32_t t_offset;       /* iterations run before this call (for the step-size schedule) */
} orc_params;

#ifdef __cplusplus
extern "C" {
#endif

/* 2D unitary DFT of an ny x nx array (sign -1 forward, +1 inverse). */
void orc_dft2(const orc_cx *in, orc_cx *out, int ny, int nx, int sign);

/* y_k = A_k x (length nc * m_k) and x = A_k^H y_k (length n). */
void orc_forward(const orc_problem *P, int k, const orc_cx *x, orc_cx *yk);
void orc_adjoint(const orc_problem *P, int k, const orc_cx *yk, orc_cx *x);

/* Hermitian eigendecomposition (cyclic Jacobi): eigenvalues descending in w,
 * eigenvectors in the columns of V (row-major q x q).  Returns sweeps used. */
int orc_eigh(const orc_cx *A, int q, double *w, orc_cx *V);

/* Householder QR of an m x r matrix (row-major) with real positive diag(R).
 * Q is m x r (row-major), R is r x r (row-major). Returns 0, or -1 if rank deficient. */
int orc_qr(const orc_cx *A, int m, int r, orc_cx *Q, orc_cx *R);

/* Least squares min ||y - M b|| by Householder QR; M is m x r row-major. */
int orc_lstsq(const orc_cx *M, int m, int r, const orc_cx *y, orc_cx *b);

/* Spectral initialisation (Alg. 2, init).  rank_in > 0 fixes r, 0 selects it
 * by the energy rule.  U0 has room for n * rmax entries; sigma for q values.
 * X0 (n x q) and gamma may be NULL.  Returns the rank used, or < 0 on error. */
int orc_init(const orc_problem *P, const orc_cx *y, const orc_params *prm,
             int rank_in, int rmax, orc_cx *U0, double *sigma, orc_cx *X0,
             double *gamma);

/* B-update only: b_k = (A_k U)^dagger y_k for every k (B is r x q col-major). */
int orc_bstep(const orc_problem *P, const orc_cx *y, const orc_cx *U, int r, orc_cx *B);

/* Gradient sum_k A_k^H (A_k U b_k - y_k) b_k^H (n x r, row-major). */
void orc_grad(const orc_problem *P, const orc_cx *y, const orc_cx *U,
              const orc_cx *B, int r, int mode, orc_cx *G);

/* Cost f(U, B) = sum_k ||y_k - A_k U b_k||^2. */
double orc_cost(const orc_problem *P, const orc_cx *y, const orc_cx *U,
                const orc_cx *B, int r);

/* Run up to n_iter iterations of Alg. 2 from U (in/out, n x r).
 *   *eta      : in  <= 0 -> set from the first gradient (eta = eta_c/||grad||);
 *               out the step size used.
 *   B         : out B_t of the last iteration run (r x q)
 *   Uprev     : out U_{t-1} of the last iteration run (n x r); X = Uprev B
 *   X_hist    : optional, n_iter * n * q: X_t = U_{t-1} B_t after every iteration
 *   sd, gnorm : optional, per iteration SD(U_{t-1}, U_t) and ||grad||_2
 * Returns the number of iterations run, < 0 on error. */
int orc_iterate(const orc_problem *P, const orc_cx *y, const orc_params *prm,
                orc_cx *U, int r, int n_iter, double *eta, orc_cx *B,
                orc_cx *Uprev, orc_cx *X_hist, double *sd, double *gnorm);

/* Subspace distance ||(I - U1 U1^H) U2||_F for n x r orthonormal U1, U2. */
double orc_sd(const orc_cx *U1, const orc_cx *U2, int n, int r);

#ifdef __cplusplus
}
#endif

#endif
