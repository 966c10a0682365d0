/*
 * Oblique-projection FEAST (Yin, Chan & Yeung, "A FEAST algorithm with oblique
 * projection for generalized eigenvalue problems") -- plain FP64 CPU ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the GPU path is checked against.  Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is complex double, column-major, leading dimension given.
 * Each routine names the passage of the paper it follows.  No blocking,
 * fusion or reordering beyond what the plain definition states; OpenMP is
 * used only across independent quadrature nodes and right-hand sides
 * (the independence the paper points out at the end of Section 4.3).
 *
 * Parity status of each routine is stated in its comment: every routine here
 * is pinned by a CPU test against a closed form, a brute-force result or a
 * value printed in the paper, except the stopping-test bookkeeping, whose
 * exact iteration count is implementation-defined ("parity unpinned" for the
 * iteration index at which the stop fires; the flag logic itself is pinned
 * by scripted sequences).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ESINGULAR = -4, OR_ENOCONV = -7 };

/* ------------------------------------------------------------------------ */
/* Quadrature (Section 4.3, eq. 4.1)                                          */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes t_j and weights omega_j on [-1, 1], ascending.
 * Textbook construction: Newton's method on the Legendre polynomial P_q
 * evaluated by its three-term recurrence; omega = 2 / ((1 - t^2) P_q'(t)^2).
 * P_q(x) and P_q'(x) by the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static void legendre_eval(int q, double x, double *pq, double *dpq)
{
    double p0 = 1.0, p1 = x;
    for (int k = 1; k < q; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pq = p1;                                   /* P_q     */
    *dpq = q * (x * p1 - p0) / (x * x - 1.0);   /* P_q'    */
}

int or_gauss_legendre(int q, double *t, double *omega)
{
    if (q < 1) return OR_EINVAL;
    for (int j = 0; j < q; ++j) {
        double x = cos(M_PI * (j + 0.75) / (q + 0.5)); /* j-th largest root, initial guess */
        double pq, dp;
        for (int it = 0; it < 100; ++it) {
            legendre_eval(q, x, &pq, &dp);
            double dx = pq / dp;
            x -= dx;
            if (fabs(dx) < 1e-15) break;
        }
        legendre_eval(q, x, &pq, &dp);
        t[q - 1 - j] = x;
        omega[q - 1 - j] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return OR_OK;
}

/* Contour nodes z_j and weights w_j such that
 *   (1/(2 pi i)) \oint f(z) dz  ~=  sum_j w_j f(z_j).
 * Circle (centre gamma, radius rho = a = b), Gauss-Legendre: eq. 4.1,
 *   theta_j = (1 + t_j) pi, z_j = gamma + rho e^{i theta_j},
 *   w_j = (1/2) omega_j (z_j - gamma).
 * Trapezoid: theta_j = 2 pi (j - 1/2) / q (j = 1..q), weight 2 pi / q in theta.
 * Ellipse (semi-axes a along Re, b along Im): z(theta) = gamma + a cos + i b sin,
 * w_j = (dtheta weight) z'(theta_j) / (2 pi i); reduces to eq. 4.1 when a = b.
 * ckind: 0 circle, 1 ellipse.  rule: 0 trapezoid, 1 Gauss-Legendre.
 * z, w: 2q doubles each (interleaved complex). */
int or_contour(int ckind, int rule, int q, double cre, double cim, double a, double b,
               double *z, double *w)
{
    if (q < 1 || a <= 0.0 || (ckind == 1 && b <= 0.0)) return OR_EINVAL;
    if (ckind == 0) b = a;
    double *t = malloc(sizeof(double) * q), *om = malloc(sizeof(double) * q);
    if (!t || !om) { free(t); free(om); return OR_ENOMEM; }
    if (rule == 1) or_gauss_legendre(q, t, om);
    for (int j = 0; j < q; ++j) {
        double theta, dth; /* node angle and its quadrature weight in theta */
        if (rule == 1) { theta = (1.0 + t[j]) * M_PI; dth = M_PI * om[j]; }
        else           { theta = 2.0 * M_PI * (j + 0.5) / q; dth = 2.0 * M_PI / q; }
        zc zj = cre + I * cim + a * cos(theta) + I * b * sin(theta);
        zc dz = -a * sin(theta) + I * b * cos(theta); /* z'(theta) */
        zc wj = dth * dz / (2.0 * M_PI * I);
        z[2 * j] = creal(zj); z[2 * j + 1] = cimag(zj);
        w[2 * j] = creal(wj); w[2 * j + 1] = cimag(wj);
    }
    free(t); free(om);
    return OR_OK;
}

/* Strictly inside the contour (circle: |lambda - gamma| < rho; ellipse:
 * ((x - gr)/a)^2 + ((y - gi)/b)^2 < 1).  Section 4.3, lines 10 of GFEAST. */
int or_inside(int ckind, double cre, double cim, double a, double b, double lr, double li)
{
    if (ckind == 0) b = a;
    double x = (lr - cre) / a, y = (li - cim) / b;
    return x * x + y * y < 1.0;
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting and triangular substitution                */
/* (the direct solver of eq. 4.2; Section 5 uses LU + substitution)          */
/* ------------------------------------------------------------------------ */

/* Right-looking Gaussian elimination, P A = L U, unit-lower L stored below
 * the diagonal.  piv[k] = row swapped with row k at step k (0-based).
 * Returns 0, or k+1 if U(k,k) is exactly zero (factorisation completed). */
int or_zgetrf(int n, zc *a, int lda, int *piv)
{
    int info = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = cabs(a[IDX(k, k, lda)]);
        for (int i = k + 1; i < n; ++i) {
            double v = cabs(a[IDX(i, k, lda)]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (p != k)
            for (int j = 0; j < n; ++j) {
                zc tmp = a[IDX(k, j, lda)];
                a[IDX(k, j, lda)] = a[IDX(p, j, lda)];
                a[IDX(p, j, lda)] = tmp;
            }
        zc d = a[IDX(k, k, lda)];
        if (d == 0.0) { if (!info) info = k + 1; continue; }
        for (int i = k + 1; i < n; ++i) a[IDX(i, k, lda)] /= d;
        for (int j = k + 1; j < n; ++j) {
            zc u = a[IDX(k, j, lda)];
            if (u == 0.0) continue;
            for (int i = k + 1; i < n; ++i) a[IDX(i, j, lda)] -= a[IDX(i, k, lda)] * u;
        }
    }
    return info;
}

/* Solve A X = B from the factors of or_zgetrf: apply P, then L y = P b
 * (forward, unit diagonal), then U x = y (backward). */
void or_zgetrs(int n, int nrhs, const zc *lu, int lda, const int *piv, zc *b, int ldb)
{
    for (int c = 0; c < nrhs; ++c) {
        zc *x = b + (size_t)c * ldb;
        for (int k = 0; k < n; ++k)
            if (piv[k] != k) { zc t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
        for (int k = 0; k < n; ++k) {
            zc v = x[k];
            for (int i = k + 1; i < n; ++i) x[i] -= lu[IDX(i, k, lda)] * v;
        }
        for (int k = n - 1; k >= 0; --k) {
            x[k] /= lu[IDX(k, k, lda)];
            zc v = x[k];
            for (int i = 0; i < k; ++i) x[i] -= lu[IDX(i, k, lda)] * v;
        }
    }
}

/* The same substitution for nrhs independent right-hand sides, in parallel
 * over the columns (used by the CPU-baseline timing of the solve step). */
void or_zgetrs_cols(int n, int nrhs, const zc *lu, int lda, const int *piv, zc *b, int ldb)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < nrhs; ++c) or_zgetrs(n, 1, lu, lda, piv, b + (size_t)c * ldb, ldb);
}

/* ------------------------------------------------------------------------ */
/* Banded LU with partial pivoting (LAPACK general-band storage):            */
/* entry (i, j) of the matrix lives at ab[(kl + ku + i - j) + j * ldab] for   */
/* max(0, j - ku) <= i <= min(n - 1, j + kl); rows 0..kl-1 of ab hold the    */
/* fill created by pivoting, so ldab >= 2 kl + ku + 1.                        */
/* ------------------------------------------------------------------------ */

static inline zc *band_at(zc *ab, int ldab, int kv, int i, int j)
{
    return ab + (size_t)(kv + i - j) + (size_t)j * ldab;
}

/* Unblocked band Gaussian elimination with partial pivoting.  The upper
 * factor has bandwidth kl + ku after row interchanges.  Returns 0 or k+1. */
int or_zgbtrf(int n, int kl, int ku, zc *ab, int ldab, int *piv)
{
    int kv = kl + ku, info = 0;
    if (ldab < 2 * kl + ku + 1) return OR_EINVAL;
    /* zero the fill rows */
    for (int j = 0; j < n; ++j)
        for (int r = 0; r < kl; ++r) ab[(size_t)r + (size_t)j * ldab] = 0.0;
    for (int k = 0; k < n; ++k) {
        int last = k + kl < n - 1 ? k + kl : n - 1;
        int p = k;
        double best = cabs(*band_at(ab, ldab, kv, k, k));
        for (int i = k + 1; i <= last; ++i) {
            double v = cabs(*band_at(ab, ldab, kv, i, k));
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        int jlast = k + kv < n - 1 ? k + kv : n - 1;
        if (p != k)
            for (int j = k; j <= jlast; ++j) {
                zc t = *band_at(ab, ldab, kv, k, j);
                *band_at(ab, ldab, kv, k, j) = *band_at(ab, ldab, kv, p, j);
                *band_at(ab, ldab, kv, p, j) = t;
            }
        zc d = *band_at(ab, ldab, kv, k, k);
        if (d == 0.0) { if (!info) info = k + 1; continue; }
        for (int i = k + 1; i <= last; ++i) *band_at(ab, ldab, kv, i, k) /= d;
        for (int j = k + 1; j <= jlast; ++j) {
            zc u = *band_at(ab, ldab, kv, k, j);
            if (u == 0.0) continue;
            for (int i = k + 1; i <= last; ++i)
                *band_at(ab, ldab, kv, i, j) -= *band_at(ab, ldab, kv, i, k) * u;
        }
    }
    return info;
}

void or_zgbtrs(int n, int kl, int ku, int nrhs, const zc *ab, int ldab, const int *piv,
               zc *b, int ldb)
{
    int kv = kl + ku;
    for (int c = 0; c < nrhs; ++c) {
        zc *x = b + (size_t)c * ldb;
        for (int k = 0; k < n; ++k) {
            if (piv[k] != k) { zc t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
            zc v = x[k];
            int last = k + kl < n - 1 ? k + kl : n - 1;
            for (int i = k + 1; i <= last; ++i) x[i] -= ab[(size_t)(kv + i - k) + (size_t)k * ldab] * v;
        }
        for (int k = n - 1; k >= 0; --k) {
            x[k] /= ab[(size_t)kv + (size_t)k * ldab];
            zc v = x[k];
            int first = k - kv > 0 ? k - kv : 0;
            for (int i = first; i < k; ++i) x[i] -= ab[(size_t)(kv + i - k) + (size_t)k * ldab] * v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Matrix products (plain triple loops)                                      */
/* ------------------------------------------------------------------------ */

/* C = op(A) * B, op = identity (conj_a = 0) or conjugate transpose (1).
 * op(A) is m x k, B is k x n, C is m x n. */
void or_zgemm(int conj_a, int m, int n, int k, const zc *a, int lda, const zc *b, int ldb,
              zc *c, int ldc)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) {
            zc s = 0.0;
            for (int p = 0; p < k; ++p) {
                zc av = conj_a ? conj(a[IDX(p, i, lda)]) : a[IDX(i, p, lda)];
                s += av * b[IDX(p, j, ldb)];
            }
            c[IDX(i, j, ldc)] = s;
        }
}

/* Y = Op * X for a pencil operand given densely (ld) or in band storage
 * (band: entry (i,j) at ab[(ku + i - j) + j*ldab], ldab >= kl + ku + 1). */
static void apply_dense(int n, const zc *A, int ld, int m, const zc *X, int ldx, zc *Y, int ldy)
{
    or_zgemm(0, n, m, n, A, ld, X, ldx, Y, ldy);
}

void or_band_matmul(int n, int kl, int ku, const zc *ab, int ldab, int m, const zc *X, int ldx,
                    zc *Y, int ldy)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < m; ++c) {
        for (int i = 0; i < n; ++i) Y[IDX(i, c, ldy)] = 0.0;
        for (int j = 0; j < n; ++j) {
            zc xv = X[IDX(j, c, ldx)];
            int i0 = j - ku > 0 ? j - ku : 0, i1 = j + kl < n - 1 ? j + kl : n - 1;
            for (int i = i0; i <= i1; ++i) Y[IDX(i, c, ldy)] += ab[(size_t)(ku + i - j) + (size_t)j * ldab] * xv;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Householder QR (GFEAST lines 2 and 17: U = U1 R1, B U1 = U2 R2)           */
/* ------------------------------------------------------------------------ */

/* Thin QR of the m x k matrix a (m >= k) by Householder reflections
 * H = I - 2 v v^H.  The returned R has a real non-negative diagonal (each
 * column of Q is rescaled by the phase of R(j,j)), which makes Q unique for
 * full-rank input.  q: m x k, r: k x k (upper triangular). */
int or_zqr(int m, int k, const zc *a, int lda, zc *q, int ldq, zc *r, int ldr)
{
    if (k > m) return OR_EINVAL;
    zc *w = malloc(sizeof(zc) * (size_t)m * k);
    zc *v = malloc(sizeof(zc) * (size_t)m * k);
    if (!w || !v) { free(w); free(v); return OR_ENOMEM; }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < m; ++i) w[IDX(i, j, m)] = a[IDX(i, j, lda)];
    memset(v, 0, sizeof(zc) * (size_t)m * k);
    for (int j = 0; j < k; ++j) {
        double nrm = 0.0;
        for (int i = j; i < m; ++i) nrm += creal(w[IDX(i, j, m)] * conj(w[IDX(i, j, m)]));
        nrm = sqrt(nrm);
        zc x0 = w[IDX(j, j, m)];
        zc ph = (cabs(x0) > 0.0) ? x0 / cabs(x0) : 1.0;
        zc alpha = -ph * nrm; /* reflect x onto alpha e_1 */
        zc *vj = v + (size_t)j * m;
        for (int i = j; i < m; ++i) vj[i] = w[IDX(i, j, m)];
        vj[j] -= alpha;
        double vn = 0.0;
        for (int i = j; i < m; ++i) vn += creal(vj[i] * conj(vj[i]));
        vn = sqrt(vn);
        if (vn > 0.0) {
            for (int i = j; i < m; ++i) vj[i] /= vn;
            for (int c = j; c < k; ++c) {
                zc s = 0.0;
                for (int i = j; i < m; ++i) s += conj(vj[i]) * w[IDX(i, c, m)];
                for (int i = j; i < m; ++i) w[IDX(i, c, m)] -= 2.0 * vj[i] * s;
            }
        }
    }
    /* R = upper triangle of w; Q = H_0 H_1 ... H_{k-1} [I_k; 0] */
    for (int c = 0; c < k; ++c) {
        zc *qc = q + (size_t)c * ldq;
        for (int i = 0; i < m; ++i) qc[i] = (i == c) ? 1.0 : 0.0;
        for (int j = k - 1; j >= 0; --j) {
            zc *vj = v + (size_t)j * m;
            zc s = 0.0;
            for (int i = j; i < m; ++i) s += conj(vj[i]) * qc[i];
            for (int i = j; i < m; ++i) qc[i] -= 2.0 * vj[i] * s;
        }
    }
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) r[IDX(i, j, ldr)] = (i <= j) ? w[IDX(i, j, m)] : 0.0;
    for (int j = 0; j < k; ++j) {
        zc d = w[IDX(j, j, m)];
        zc ph = (cabs(d) > 0.0) ? d / cabs(d) : 1.0;
        /* row j of R scaled by conj(ph), column j of Q by ph */
        for (int c = j; c < k; ++c) r[IDX(j, c, ldr)] *= conj(ph);
        for (int i = 0; i < m; ++i) q[IDX(i, j, ldq)] *= ph;
    }
    free(w); free(v);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Complex QZ for the projected pencil (GFEAST line 6; the paper points to   */
/* the LAPACK drivers xGGES / xGGEV).  Hessenberg-triangular reduction by    */
/* Givens rotations, single-shift complex QZ iteration with deflation,       */
/* right eigenvectors by back-substitution on the generalized Schur form.    */
/* ------------------------------------------------------------------------ */

/* Left rotation G = [c s; -conj(s) c] (c real) with G [x; y] = [r; 0]. */
static void giv_left(zc x, zc y, double *c, zc *s)
{
    double ax = cabs(x), ay = cabs(y);
    if (ay == 0.0) { *c = 1.0; *s = 0.0; return; }
    if (ax == 0.0) { *c = 0.0; *s = 1.0; return; }
    double r = hypot(ax, ay);
    *c = ax / r;
    *s = (x / ax) * conj(y) / r;
}
static void rot_rows(zc *M, int ld, int i, int j, int c0, int c1, double c, zc s)
{
    for (int col = c0; col <= c1; ++col) {
        zc a = M[IDX(i, col, ld)], b = M[IDX(j, col, ld)];
        M[IDX(i, col, ld)] = c * a + s * b;
        M[IDX(j, col, ld)] = -conj(s) * a + c * b;
    }
}
/* Right rotation R = [c -conj(s); s c] on columns (i, j) chosen so that the
 * row vector [t0 t1] * R = [0 r]. */
static void giv_right(zc t0, zc t1, double *c, zc *s)
{
    double a0 = cabs(t0), a1 = cabs(t1);
    if (a0 == 0.0) { *c = 1.0; *s = 0.0; return; }
    if (a1 == 0.0) { *c = 0.0; *s = 1.0; return; }
    double r = hypot(a0, a1);
    *c = a1 / r;
    *s = -t0 * conj(t1) / (a1 * r);
}
static void rot_cols(zc *M, int ld, int i, int j, int r0, int r1, double c, zc s)
{
    for (int row = r0; row <= r1; ++row) {
        zc a = M[IDX(row, i, ld)], b = M[IDX(row, j, ld)];
        M[IDX(row, i, ld)] = a * c + b * s;
        M[IDX(row, j, ld)] = -a * conj(s) + b * c;
    }
}

/* Generalized eigenvalues alpha_i / beta_i and right eigenvectors v_i of the
 * m x m pencil (a, b):  beta_i a v_i = alpha_i b v_i, ||v_i||_2 = 1.
 * Returns 0, or OR_ENOCONV if the QZ iteration does not converge. */
int or_zggev(int m, const zc *a, int lda, const zc *b, int ldb, zc *alpha, zc *beta, zc *v,
             int ldv)
{
    if (m <= 0) return m == 0 ? OR_OK : OR_EINVAL;
    zc *H = malloc(sizeof(zc) * (size_t)m * m), *T = malloc(sizeof(zc) * (size_t)m * m);
    zc *Z = malloc(sizeof(zc) * (size_t)m * m);
    if (!H || !T || !Z) { free(H); free(T); free(Z); return OR_ENOMEM; }
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) {
            H[IDX(i, j, m)] = a[IDX(i, j, lda)];
            T[IDX(i, j, m)] = b[IDX(i, j, ldb)];
            Z[IDX(i, j, m)] = (i == j) ? 1.0 : 0.0;
        }
    double c; zc s;
    /* 1. triangularise T from the left (Q^H applied to both) */
    for (int j = 0; j < m; ++j)
        for (int i = m - 1; i > j; --i) {
            giv_left(T[IDX(i - 1, j, m)], T[IDX(i, j, m)], &c, &s);
            rot_rows(T, m, i - 1, i, 0, m - 1, c, s);
            rot_rows(H, m, i - 1, i, 0, m - 1, c, s);
            T[IDX(i, j, m)] = 0.0;
        }
    /* 2. Hessenberg-triangular reduction */
    for (int j = 0; j + 2 < m; ++j)
        for (int i = m - 1; i >= j + 2; --i) {
            giv_left(H[IDX(i - 1, j, m)], H[IDX(i, j, m)], &c, &s);
            rot_rows(H, m, i - 1, i, j, m - 1, c, s);
            rot_rows(T, m, i - 1, i, i - 1, m - 1, c, s);
            H[IDX(i, j, m)] = 0.0;
            giv_right(T[IDX(i, i - 1, m)], T[IDX(i, i, m)], &c, &s);
            rot_cols(H, m, i - 1, i, 0, m - 1, c, s);
            rot_cols(T, m, i - 1, i, 0, i, c, s);
            rot_cols(Z, m, i - 1, i, 0, m - 1, c, s);
            T[IDX(i, i - 1, m)] = 0.0;
        }
    /* 3. QZ iteration */
    const double eps = 2.220446049250313e-16;
    double hn = 0.0, tn = 0.0;
    for (int j = 0; j < m; ++j)
        for (int i = 0; i < m; ++i) { hn = fmax(hn, cabs(H[IDX(i, j, m)])); tn = fmax(tn, cabs(T[IDX(i, j, m)])); }
    double htol = eps * fmax(hn, 1e-300);
    int ihi = m - 1, iter = 0, total = 0, status = OR_OK;
    while (ihi > 0) {
        int l = ihi;
        while (l > 0) {
            double sub = cabs(H[IDX(l, l - 1, m)]);
            double loc = cabs(H[IDX(l - 1, l - 1, m)]) + cabs(H[IDX(l, l, m)]);
            if (sub <= eps * loc || sub <= htol) { H[IDX(l, l - 1, m)] = 0.0; break; }
            --l;
        }
        if (l == ihi) { --ihi; iter = 0; continue; }
        if (++total > 60 * m) { status = OR_ENOCONV; break; }
        ++iter;
        /* shift: root of det(Hb - sigma Tb) (trailing 2x2 block, Tb upper
         * triangular) closest to H(ihi,ihi)/T(ihi,ihi) */
        zc sigma;
        zc h00 = H[IDX(ihi - 1, ihi - 1, m)], h01 = H[IDX(ihi - 1, ihi, m)];
        zc h10 = H[IDX(ihi, ihi - 1, m)], h11 = H[IDX(ihi, ihi, m)];
        zc t00 = T[IDX(ihi - 1, ihi - 1, m)], t01 = T[IDX(ihi - 1, ihi, m)], t11 = T[IDX(ihi, ihi, m)];
        if (iter % 11 == 10) {
            sigma = h11 / (t11 != 0.0 ? t11 : 1.0) + cabs(h10) * (1.0 + 0.5 * I);
        } else if (cabs(t00) > eps * tn && cabs(t11) > eps * tn) {
            zc qa = t00 * t11, qb = -(h00 * t11 + h11 * t00 - t01 * h10), qc = h00 * h11 - h01 * h10;
            zc disc = csqrt(qb * qb - 4.0 * qa * qc);
            zc r1 = (-qb + disc) / (2.0 * qa), r2 = (-qb - disc) / (2.0 * qa);
            zc ref = h11 / t11;
            sigma = (cabs(r1 - ref) < cabs(r2 - ref)) ? r1 : r2;
        } else {
            sigma = 0.0; /* a (near) infinite eigenvalue in the window: zero shift */
        }
        /* chase the bulge from l to ihi */
        for (int k = l; k < ihi; ++k) {
            zc x, y;
            if (k == l) { x = H[IDX(l, l, m)] - sigma * T[IDX(l, l, m)]; y = H[IDX(l + 1, l, m)]; }
            else        { x = H[IDX(k, k - 1, m)]; y = H[IDX(k + 1, k - 1, m)]; }
            giv_left(x, y, &c, &s);
            rot_rows(H, m, k, k + 1, (k > l) ? k - 1 : l, m - 1, c, s);
            rot_rows(T, m, k, k + 1, k, m - 1, c, s);
            if (k > l) H[IDX(k + 1, k - 1, m)] = 0.0;
            giv_right(T[IDX(k + 1, k, m)], T[IDX(k + 1, k + 1, m)], &c, &s);
            int rl = (k + 2 < ihi) ? k + 2 : ihi;
            rot_cols(H, m, k, k + 1, 0, rl, c, s);
            rot_cols(T, m, k, k + 1, 0, k + 1, c, s);
            rot_cols(Z, m, k, k + 1, 0, m - 1, c, s);
            T[IDX(k + 1, k, m)] = 0.0;
        }
    }
    /* 4. eigenvalues and right eigenvectors */
    for (int k = 0; k < m; ++k) { alpha[k] = H[IDX(k, k, m)]; beta[k] = T[IDX(k, k, m)]; }
    zc *yh = malloc(sizeof(zc) * (size_t)m);
    double small = eps * (hn + tn);
    for (int k = 0; k < m && yh; ++k) {
        zc al = alpha[k], be = beta[k];
        for (int i = 0; i < m; ++i) yh[i] = 0.0;
        yh[k] = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            zc sum = 0.0;
            for (int p = i + 1; p <= k; ++p) sum += (be * H[IDX(i, p, m)] - al * T[IDX(i, p, m)]) * yh[p];
            zc d = be * H[IDX(i, i, m)] - al * T[IDX(i, i, m)];
            if (cabs(d) < small * (cabs(al) + cabs(be))) d = small * (cabs(al) + cabs(be));
            if (d == 0.0) d = 1e-300;
            yh[i] = -sum / d;
        }
        double nrm = 0.0;
        zc *vk = v + (size_t)k * ldv;
        for (int i = 0; i < m; ++i) {
            zc sacc = 0.0;
            for (int p = 0; p <= k; ++p) sacc += Z[IDX(i, p, m)] * yh[p];
            vk[i] = sacc;
            nrm += creal(sacc * conj(sacc));
        }
        nrm = sqrt(nrm);
        if (nrm > 0.0) for (int i = 0; i < m; ++i) vk[i] /= nrm;
    }
    free(yh); free(H); free(T); free(Z);
    return status;
}

/* ------------------------------------------------------------------------ */
/* GFEAST driver (Algorithm "GFEAST", lines 2-17, with the start block Y in  */
/* place of SEARCH: the first subspace is U = Q Y by the quadrature, as in   */
/* line 2 of Algorithm "EIGENPAIRS").                                        */
/* ------------------------------------------------------------------------ */

typedef struct or_ctx {
    int kind, n, kl, ku, b_identity;     /* kind 0 dense, 1 banded            */
    zc *A, *B;                           /* dense n x n, or band (kl+ku+1) x n */
    int ckind, rule, q;
    double cre, cim, ca, cb;
    zc *z, *w;                           /* nodes and weights                  */
    zc *fac;                             /* q factors                          */
    int *piv;
    size_t fac_stride;                   /* elements per factor                */
    int ldf;                             /* leading dim of each factor         */
    int m0;
    int projection;                      /* 0: oblique (test space U2), 1: Rayleigh-Ritz (U1) */
    int search_literal;                  /* SEARCH line 10 read literally (U = U1 after a full-rank step) */
    zc *U1, *U2, *R2, *AU1, *BU1;        /* n x m0, n x m0, m0 x m0, n x m0 x2 */
    double eps, eta;
    int max_iter;
    /* state (line 3) */
    int k, c_prev, done, flag;
    double e_prev;
    /* current iterate: all t Ritz pairs */
    zc *At, *Bt, *lam, *Xr;
    double *res;
    int *sel;
    /* accepted sets Lambda^(k), X^(k) and the previous ones */
    int cnt_cur, cnt_prev;
    zc *lam_cur, *lam_prev, *X_cur, *X_prev;
    double *r_cur, *r_prev;
    double err_cur, err_prev;
    /* output (lines 13-15) */
    int out_count, out_k;
    double out_err;
    zc *out_lam, *out_X;
    double *out_res;
} or_ctx;

/* Y = A X (which = 0) or B X (which = 1) for the pencil held by ctx. */
static void pencil_apply(const or_ctx *c, int which, int m, const zc *X, zc *Y)
{
    int n = c->n;
    if (which == 1 && c->b_identity) {
        memcpy(Y, X, sizeof(zc) * (size_t)n * m);
        return;
    }
    const zc *M = which ? c->B : c->A;
    if (c->kind == 0) apply_dense(n, M, n, m, X, n, Y, n);
    else or_band_matmul(n, c->kl, c->ku, M, c->kl + c->ku + 1, m, X, n, Y, n);
}

/* U = sum_j w_j (z_j B - A)^{-1} B V : the quadrature of eq. 4.1 applied to
 * the n x m block V, with the shifted systems of eq. 4.2 solved by the
 * stored LU factors.  Solves in parallel over (node, column); the weighted
 * sum is taken in node order j = 1..q. */
void or_filter(const or_ctx *c, const zc *V, zc *U)
{
    int n = c->n, m = c->m0, q = c->q;
    zc *BV = malloc(sizeof(zc) * (size_t)n * m);
    zc *Xs = malloc(sizeof(zc) * (size_t)n * m * q);
    pencil_apply(c, 1, m, V, BV);
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int j = 0; j < q; ++j)
        for (int col = 0; col < m; ++col) {
            zc *x = Xs + ((size_t)j * m + col) * n;
            memcpy(x, BV + (size_t)col * n, sizeof(zc) * n);
            if (c->kind == 0)
                or_zgetrs(n, 1, c->fac + j * c->fac_stride, c->ldf, c->piv + (size_t)j * n, x, n);
            else
                or_zgbtrs(n, c->kl, c->ku, 1, c->fac + j * c->fac_stride, c->ldf, c->piv + (size_t)j * n, x, n);
        }
    for (size_t i = 0; i < (size_t)n * m; ++i) U[i] = 0.0;
    for (int j = 0; j < q; ++j)
        for (size_t i = 0; i < (size_t)n * m; ++i) U[i] += c->w[j] * Xs[(size_t)j * n * m + i];
    free(BV); free(Xs);
}

/* Lines 17 (and 2): U = U1 R1 and B U1 = U2 R2 (Householder QR). */
static int orthonormalise(or_ctx *c, const zc *U)
{
    int n = c->n, m = c->m0;
    zc *R1 = malloc(sizeof(zc) * (size_t)m * m);
    int st = or_zqr(n, m, U, n, c->U1, n, R1, m);
    free(R1);
    if (st) return st;
    pencil_apply(c, 1, m, c->U1, c->BU1);
    return or_zqr(n, m, c->BU1, n, c->U2, n, c->R2, m);
}

void or_free(or_ctx *c)
{
    if (!c) return;
    zc *zp[] = {c->A, c->B, c->z, c->w, c->fac, c->U1, c->U2, c->R2, c->AU1, c->BU1, c->At, c->Bt,
                c->lam, c->Xr, c->lam_cur, c->lam_prev, c->X_cur, c->X_prev, c->out_lam, c->out_X};
    for (size_t i = 0; i < sizeof(zp) / sizeof(zp[0]); ++i) free(zp[i]);
    free(c->piv); free(c->res); free(c->sel); free(c->r_cur); free(c->r_prev); free(c->out_res);
    free(c);
}

/* Lines 1-3 with a given start block.  kind 0: A, B dense n x n (ld);
 * kind 1: A, B in compact band storage ((kl+ku+1) x n, ld = kl+ku+1);
 * b_identity: B = I (B ignored).  Y: n x m0.  *status receives 0 or an error
 * (OR_ESINGULAR if a shifted matrix is exactly singular). */
or_ctx *or_setup(int kind, int n, const zc *A, const zc *B, int ld, int kl, int ku, int b_identity,
                 int ckind, int rule, int q, double cre, double cim, double ca, double cb,
                 int m0, const zc *Y, double eps, double eta, int max_iter, int *status)
{
    *status = OR_EINVAL;
    if (n < 1 || m0 < 1 || m0 > n || q < 1 || (kind == 1 && (kl < 0 || ku < 0))) return NULL;
    or_ctx *c = calloc(1, sizeof(or_ctx));
    if (!c) { *status = OR_ENOMEM; return NULL; }
    c->kind = kind; c->n = n; c->kl = kl; c->ku = ku; c->b_identity = b_identity;
    c->ckind = ckind; c->rule = rule; c->q = q; c->cre = cre; c->cim = cim; c->ca = ca;
    c->cb = (ckind == 0) ? ca : cb;
    c->m0 = m0; c->eps = eps; c->eta = eta; c->max_iter = max_iter;
    size_t nn = (kind == 0) ? (size_t)n * n : (size_t)(kl + ku + 1) * n;
    int ldin = (kind == 0) ? n : kl + ku + 1;
    c->A = malloc(sizeof(zc) * nn);
    c->B = malloc(sizeof(zc) * nn);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < ldin; ++i) {
            c->A[IDX(i, j, ldin)] = A[IDX(i, j, ld)];
            c->B[IDX(i, j, ldin)] = b_identity ? 0.0 : B[IDX(i, j, ld)];
        }
    c->z = malloc(sizeof(zc) * q);
    c->w = malloc(sizeof(zc) * q);
    int st = or_contour(ckind, rule, q, cre, cim, ca, c->cb, (double *)c->z, (double *)c->w);
    if (st) { or_free(c); *status = st; return NULL; }
    /* line 2 of EIGENPAIRS / eq. 4.2: form z_j B - A and factor it once */
    c->ldf = (kind == 0) ? n : 2 * kl + ku + 1;
    c->fac_stride = (size_t)c->ldf * n;
    c->fac = malloc(sizeof(zc) * c->fac_stride * q);
    c->piv = malloc(sizeof(int) * (size_t)n * q);
    if (!c->fac || !c->piv) { or_free(c); *status = OR_ENOMEM; return NULL; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < q; ++j) {
        zc *F = c->fac + j * c->fac_stride;
        zc zj = c->z[j];
        if (kind == 0) {
            for (int cc = 0; cc < n; ++cc)
                for (int i = 0; i < n; ++i) {
                    zc bij = b_identity ? (i == cc ? 1.0 : 0.0) : c->B[IDX(i, cc, n)];
                    F[IDX(i, cc, n)] = zj * bij - c->A[IDX(i, cc, n)];
                }
            if (or_zgetrf(n, F, n, c->piv + (size_t)j * n)) {
#pragma omp atomic write
                bad = j + 1;
            }
        } else {
            int kv = kl + ku;
            for (size_t e = 0; e < c->fac_stride; ++e) F[e] = 0.0;
            for (int cc = 0; cc < n; ++cc)
                for (int i = (cc - ku > 0 ? cc - ku : 0); i <= (cc + kl < n - 1 ? cc + kl : n - 1); ++i) {
                    zc bij = b_identity ? (i == cc ? 1.0 : 0.0) : c->B[(size_t)(ku + i - cc) + (size_t)cc * ldin];
                    F[(size_t)(kv + i - cc) + (size_t)cc * c->ldf] = zj * bij - c->A[(size_t)(ku + i - cc) + (size_t)cc * ldin];
                }
            if (or_zgbtrf(n, kl, ku, F, c->ldf, c->piv + (size_t)j * n)) {
#pragma omp atomic write
                bad = j + 1;
            }
        }
    }
    if (bad) { or_free(c); *status = OR_ESINGULAR; return NULL; }
    size_t nm = (size_t)n * m0, mm = (size_t)m0 * m0;
    c->U1 = malloc(sizeof(zc) * nm); c->U2 = malloc(sizeof(zc) * nm);
    c->AU1 = malloc(sizeof(zc) * nm); c->BU1 = malloc(sizeof(zc) * nm);
    c->R2 = malloc(sizeof(zc) * mm); c->At = malloc(sizeof(zc) * mm); c->Bt = malloc(sizeof(zc) * mm);
    c->lam = malloc(sizeof(zc) * m0); c->Xr = malloc(sizeof(zc) * nm);
    c->res = malloc(sizeof(double) * m0); c->sel = malloc(sizeof(int) * m0);
    c->lam_cur = malloc(sizeof(zc) * m0); c->lam_prev = malloc(sizeof(zc) * m0);
    c->X_cur = malloc(sizeof(zc) * nm); c->X_prev = malloc(sizeof(zc) * nm);
    c->r_cur = malloc(sizeof(double) * m0); c->r_prev = malloc(sizeof(double) * m0);
    c->out_lam = malloc(sizeof(zc) * m0); c->out_X = malloc(sizeof(zc) * nm);
    c->out_res = malloc(sizeof(double) * m0);
    zc *U = malloc(sizeof(zc) * nm);
    or_filter(c, Y, U);
    st = orthonormalise(c, U);
    free(U);
    if (st) { or_free(c); *status = st; return NULL; }
    c->k = 0; c->c_prev = 0; c->e_prev = 0.0; c->done = 0; c->flag = 2;
    c->cnt_cur = c->cnt_prev = 0; c->err_cur = c->err_prev = 0.0;
    *status = OR_OK;
    return c;
}

/* One pass of lines 5-17.  Returns 0, OR_ENOCONV if the projected QZ failed,
 * or 1 if the algorithm had already stopped.  *flag: 2 = continue,
 * 1 / 0 / -1 = the three stopping criteria of lines 13-15. */
int or_iterate(or_ctx *c, int *k_out, int *count, int *flag, double *err)
{
    if (c->done) return 1;
    int n = c->n, m = c->m0;
    size_t nm = (size_t)n * m;
    c->k += 1;
    /* line 5: A~ = U2^H A U1, B~ = U2^H B U1 (oblique, eq. 3.10); with the
     * Rayleigh-Ritz projection of Algorithm FEAST (Section 3) the test space
     * is the search space itself: A~ = U1^H A U1, B~ = U1^H B U1 */
    pencil_apply(c, 0, m, c->U1, c->AU1);
    pencil_apply(c, 1, m, c->U1, c->BU1);
    const zc *T = c->projection ? c->U1 : c->U2;
    or_zgemm(1, m, m, n, T, n, c->AU1, n, c->At, m);
    or_zgemm(1, m, m, n, T, n, c->BU1, n, c->Bt, m);
    /* line 6: projected eigenpairs, x_i = U1 y_i */
    zc *al = malloc(sizeof(zc) * m), *be = malloc(sizeof(zc) * m), *Yv = malloc(sizeof(zc) * (size_t)m * m);
    int st = or_zggev(m, c->At, m, c->Bt, m, al, be, Yv, m);
    or_zgemm(0, n, m, m, c->U1, n, Yv, m, c->Xr, n);
    /* lines 7-12: residuals r_i (eq. 5.1), selection, c(k), e(k) */
    zc *AX = malloc(sizeof(zc) * nm), *BX = malloc(sizeof(zc) * nm);
    pencil_apply(c, 0, m, c->Xr, AX);
    pencil_apply(c, 1, m, c->Xr, BX);
    int ck = 0;
    double ek = 0.0;
    for (int i = 0; i < m; ++i) {
        int finite = cabs(be[i]) > 0.0;
        c->lam[i] = finite ? al[i] / be[i] : INFINITY;
        double num = 0.0, na = 0.0, nb = 0.0;
        for (int p = 0; p < n; ++p) {
            zc ax = AX[IDX(p, i, n)], bx = BX[IDX(p, i, n)];
            zc d = ax - c->lam[i] * bx;
            num += creal(d * conj(d)); na += creal(ax * conj(ax)); nb += creal(bx * conj(bx));
        }
        c->res[i] = finite ? sqrt(num) / (sqrt(na) + sqrt(nb)) : INFINITY;
        c->sel[i] = finite && or_inside(c->ckind, c->cre, c->cim, c->ca, c->cb, creal(c->lam[i]), cimag(c->lam[i]))
                    && c->res[i] < c->eta;
        if (c->sel[i]) {
            c->lam_cur[ck] = c->lam[i];
            memcpy(c->X_cur + (size_t)ck * n, c->Xr + (size_t)i * n, sizeof(zc) * n);
            c->r_cur[ck] = c->res[i];
            if (c->res[i] > ek) ek = c->res[i];
            ++ck;
        }
    }
    free(AX); free(BX); free(al); free(be); free(Yv);
    c->cnt_cur = ck; c->err_cur = ek;
    /* Lines 13-15.  The count is taken as fixed only once it is non-zero
     * (Section 4.2 fixes s from "s' eigenvalues inside Gamma whose accuracy
     * is below eta" unchanged over two iterations); while no pair has yet
     * reached eta the iteration continues, so an empty contour ends at
     * max_iter with flag -1 and no pairs. */
    int f = 2;
    int fixed = (ck == c->c_prev) && ck > 0;
    if (fixed && ek < c->eps) f = 1;                            /* line 13 */
    else if (fixed && ek > c->e_prev) f = 0;                    /* line 14 */
    else if (c->k == c->max_iter) f = -1;                       /* line 15 */
    if (f != 2) {
        c->done = 1; c->flag = f;
        if (f == 0) {
            c->out_count = c->cnt_prev; c->out_err = c->err_prev; c->out_k = c->k - 1;
            memcpy(c->out_lam, c->lam_prev, sizeof(zc) * c->cnt_prev);
            memcpy(c->out_X, c->X_prev, sizeof(zc) * (size_t)n * c->cnt_prev);
            memcpy(c->out_res, c->r_prev, sizeof(double) * c->cnt_prev);
        } else {
            c->out_count = ck; c->out_err = ek; c->out_k = c->k;
            memcpy(c->out_lam, c->lam_cur, sizeof(zc) * ck);
            memcpy(c->out_X, c->X_cur, sizeof(zc) * (size_t)n * ck);
            memcpy(c->out_res, c->r_cur, sizeof(double) * ck);
        }
    } else {
        /* lines 16-17: U = Q U1 by quadrature, then U = U1 R1, B U1 = U2 R2 */
        zc *U = malloc(sizeof(zc) * nm);
        or_filter(c, c->U1, U);
        int s2 = orthonormalise(c, U);
        free(U);
        if (s2 && !st) st = s2;
    }
    /* keep this iterate as "previous" for line 14 of the next pass */
    c->cnt_prev = ck; c->err_prev = ek;
    memcpy(c->lam_prev, c->lam_cur, sizeof(zc) * ck);
    memcpy(c->X_prev, c->X_cur, sizeof(zc) * (size_t)n * ck);
    memcpy(c->r_prev, c->r_cur, sizeof(double) * ck);
    c->c_prev = ck; c->e_prev = ek;
    *k_out = c->k; *count = ck; *flag = f; *err = ek;
    return st;
}

/* Accessors for the test-suite. what: 0 U1, 1 U2, 2 R2, 3 A~, 4 B~, 5 Ritz
 * vectors x_i (n x m0), 6 Ritz values (m0), 7 AU1, 8 BU1, 9 nodes, 10 weights. */
void or_get(const or_ctx *c, int what, zc *out)
{
    size_t nm = (size_t)c->n * c->m0, mm = (size_t)c->m0 * c->m0;
    switch (what) {
    case 0: memcpy(out, c->U1, sizeof(zc) * nm); break;
    case 1: memcpy(out, c->U2, sizeof(zc) * nm); break;
    case 2: memcpy(out, c->R2, sizeof(zc) * mm); break;
    case 3: memcpy(out, c->At, sizeof(zc) * mm); break;
    case 4: memcpy(out, c->Bt, sizeof(zc) * mm); break;
    case 5: memcpy(out, c->Xr, sizeof(zc) * nm); break;
    case 6: memcpy(out, c->lam, sizeof(zc) * c->m0); break;
    case 7: memcpy(out, c->AU1, sizeof(zc) * nm); break;
    case 8: memcpy(out, c->BU1, sizeof(zc) * nm); break;
    case 9: memcpy(out, c->z, sizeof(zc) * c->q); break;
    case 10: memcpy(out, c->w, sizeof(zc) * c->q); break;
    default: break;
    }
}
void or_get_ritz_info(const or_ctx *c, double *res, int *sel)
{
    memcpy(res, c->res, sizeof(double) * c->m0);
    memcpy(sel, c->sel, sizeof(int) * c->m0);
}
/* 0: the oblique projection of GFEAST (the paper's method); 1: the
 * Rayleigh-Ritz projection of Algorithm FEAST (comparison system). */
int or_set_projection(or_ctx *c, int projection)
{
    if (projection != 0 && projection != 1) return OR_EINVAL;
    c->projection = projection;
    return OR_OK;
}
/* 1: SEARCH's line 10 read literally (U = U1, orthonormal, after a
 * full-rank step); 0 (default): the block is kept as filtered columns. */
int or_set_search_literal(or_ctx *c, int literal)
{
    c->search_literal = literal ? 1 : 0;
    return OR_OK;
}
/* Replace U1 (and recompute U2 = orth(B U1)) -- lets a test drive one
 * filter step from a chosen subspace. */
int or_set_U1(or_ctx *c, const zc *U1)
{
    memcpy(c->U1, U1, sizeof(zc) * (size_t)c->n * c->m0);
    pencil_apply(c, 1, c->m0, c->U1, c->BU1);
    return or_zqr(c->n, c->m0, c->BU1, c->n, c->U2, c->n, c->R2, c->m0);
}
/* Output of lines 13-15 (valid once a stop fired). */
int or_result(const or_ctx *c, int *count, zc *lam, zc *X, double *res, double *err, int *flag, int *k)
{
    if (!c->done) return 1;
    *count = c->out_count; *err = c->out_err; *flag = c->flag; *k = c->out_k;
    memcpy(lam, c->out_lam, sizeof(zc) * c->out_count);
    if (X) memcpy(X, c->out_X, sizeof(zc) * (size_t)c->n * c->out_count);
    memcpy(res, c->out_res, sizeof(double) * c->out_count);
    return 0;
}
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* SEARCH (Algorithm "SEARCH", Section 4.1): an upper bound t of the number  */
/* s of eigenvalues inside the contour and a basis of the filtered subspace. */
/* ------------------------------------------------------------------------ */

/* Householder QR with column pivoting (Businger-Golub): at step j the
 * remaining column of largest norm is brought to position j.  a (m x k) is
 * copied; on return jpvt holds the column order, rdiag |R_jj|, *rank the
 * number of j with |R_jj| > tol |R_00|, and q (m x k) the first *rank
 * columns of Q (the rest are left as computed). */
int or_zqrcp(int m, int k, const zc *a, int lda, double tol, int *jpvt, double *rdiag, int *rank, zc *q, int ldq)
{
    if (k > m || k < 1) return OR_EINVAL;
    zc *w = malloc(sizeof(zc) * (size_t)m * k);
    zc *v = malloc(sizeof(zc) * (size_t)m * k);
    if (!w || !v) { free(w); free(v); return OR_ENOMEM; }
    for (int j = 0; j < k; ++j) {
        jpvt[j] = j;
        for (int i = 0; i < m; ++i) w[IDX(i, j, m)] = a[IDX(i, j, lda)];
    }
    memset(v, 0, sizeof(zc) * (size_t)m * k);
    int r = k;
    for (int j = 0; j < k; ++j) {
        /* pivot: largest remaining norm of rows j..m-1 */
        int best = j;
        double bn = -1.0;
        for (int c = j; c < k; ++c) {
            double s = 0.0;
            for (int i = j; i < m; ++i) s += creal(w[IDX(i, c, m)] * conj(w[IDX(i, c, m)]));
            if (s > bn) { bn = s; best = c; }
        }
        if (best != j) {
            for (int i = 0; i < m; ++i) {
                zc t = w[IDX(i, j, m)];
                w[IDX(i, j, m)] = w[IDX(i, best, m)];
                w[IDX(i, best, m)] = t;
            }
            int tp = jpvt[j]; jpvt[j] = jpvt[best]; jpvt[best] = tp;
        }
        double nrm = sqrt(bn > 0.0 ? bn : 0.0);
        rdiag[j] = nrm;   /* |R_jj| = norm of the pivot column below row j */
        zc x0 = w[IDX(j, j, m)];
        zc ph = (cabs(x0) > 0.0) ? x0 / cabs(x0) : 1.0;
        zc alpha = -ph * nrm;
        zc *vj = v + (size_t)j * m;
        for (int i = j; i < m; ++i) vj[i] = w[IDX(i, j, m)];
        vj[j] -= alpha;
        double vn = 0.0;
        for (int i = j; i < m; ++i) vn += creal(vj[i] * conj(vj[i]));
        vn = sqrt(vn);
        if (vn > 0.0) {
            for (int i = j; i < m; ++i) vj[i] /= vn;
            for (int c = j; c < k; ++c) {
                zc s = 0.0;
                for (int i = j; i < m; ++i) s += conj(vj[i]) * w[IDX(i, c, m)];
                for (int i = j; i < m; ++i) w[IDX(i, c, m)] -= 2.0 * vj[i] * s;
            }
        }
    }
    for (int j = 0; j < k; ++j)
        if (!(rdiag[j] > tol * rdiag[0])) { r = j; break; }
    *rank = r;
    /* Q = H_0 ... H_{k-1} [I; 0], first r columns, phases fixed so that R_jj > 0 */
    for (int c = 0; c < r; ++c) {
        zc *qc = q + (size_t)c * ldq;
        for (int i = 0; i < m; ++i) qc[i] = (i == c) ? 1.0 : 0.0;
        for (int j = k - 1; j >= 0; --j) {
            zc *vj = v + (size_t)j * m;
            zc s = 0.0;
            for (int i = j; i < m; ++i) s += conj(vj[i]) * qc[i];
            for (int i = j; i < m; ++i) qc[i] -= 2.0 * vj[i] * s;
        }
        zc d = w[IDX(c, c, m)];
        zc ph = (cabs(d) > 0.0) ? d / cabs(d) : 1.0;
        for (int i = 0; i < m; ++i) qc[i] *= ph;
    }
    free(w); free(v);
    return OR_OK;
}

/* Filter w columns of Y (leading dim n) into U (leading dim n) with the
 * context's factors: the block is zero-padded to the context's width. */
static void filter_cols(const or_ctx *c, const zc *Y, int w, zc *U)
{
    int n = c->n, m = c->m0;
    zc *V = calloc((size_t)n * m, sizeof(zc));
    zc *F = malloc(sizeof(zc) * (size_t)n * m);
    memcpy(V, Y, sizeof(zc) * (size_t)n * w);
    or_filter(c, V, F);
    memcpy(U, F, sizeof(zc) * (size_t)n * w);
    free(V); free(F);
}

/* Algorithm SEARCH with the random columns supplied: Ypool (n x npool)
 * gives Y_0 (its first p columns) and every augmentation (the next columns
 * in order).  alpha > 1: growth factor; rank_tol: the numerical rank of
 * line 9 counts |R_jj| > rank_tol |R_00|.  The working width may not exceed
 * the context's m0.  Out: *t, *s0 (line 2's estimate), U1 (n x t,
 * orthonormal, leading dim n).  OR_EINVAL when the pool or the width runs
 * out before a rank deficiency shows. */
int or_search(const or_ctx *c, const zc *Ypool, int npool, double alpha, int p, double rank_tol, zc *U1, int *t,
              int *s0)
{
    int n = c->n, cap = c->m0;
    if (p < 1 || p > cap || p > npool || !(alpha > 1.0) || !(rank_tol > 0.0)) return OR_EINVAL;
    zc *U = malloc(sizeof(zc) * (size_t)n * cap);
    zc *Q = malloc(sizeof(zc) * (size_t)n * cap);
    int *jp = malloc(sizeof(int) * cap);
    double *rd = malloc(sizeof(double) * cap);
    int st = OR_OK;
    /* line 1: U = Q Y_0 */
    filter_cols(c, Ypool, p, U);
    int used = p, have = p;
    /* line 2: s0 = ceil(trace(Y_0^H U) / p), real part of the trace */
    double tr = 0.0;
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < n; ++i) tr += creal(conj(Ypool[IDX(i, j, n)]) * U[IDX(i, j, n)]);
    *s0 = (int)ceil(tr / p);
    int sd = *s0 > p ? *s0 : p;
    if (sd > n) sd = n;
    for (;;) {
        if (sd > cap) { st = OR_EINVAL; break; }
        if (sd > have) {   /* lines 3-5: augment with the next sd - have filtered columns */
            if (used + (sd - have) > npool) { st = OR_EINVAL; break; }
            filter_cols(c, Ypool + (size_t)used * n, sd - have, U + (size_t)have * n);
            used += sd - have;
            have = sd;
        }
        /* lines 9-10: rank-revealing QR.  On full rank the block is kept as
         * filtered columns (the span of U1, on the scale of the columns that
         * join it next), so that the relative rank test compares like with
         * like */
        int r = 0;
        st = or_zqrcp(n, sd, U, n, rank_tol, jp, rd, &r, Q, n);
        if (st) break;
        if (r < sd) {
            *t = r;
            memcpy(U1, Q, sizeof(zc) * (size_t)n * r);
            break;
        }
        if (c->search_literal) {
            /* line 10 as printed: U = U1, the orthonormal basis of the
             * full-rank block, before the next filtered columns join it */
            memcpy(U, Q, sizeof(zc) * (size_t)n * r);
        }
        have = sd;
        sd = (int)ceil(alpha * r);
        if (sd > n) sd = n;
        if (sd == r) { st = OR_EINVAL; break; }   /* the whole space is full rank */
    }
    free(U); free(Q); free(jp); free(rd);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Block CIRR (Section 2.1, Algorithm Block_CIRR) -- the comparison method   */
/* ------------------------------------------------------------------------ */

/* Singular value decomposition a = U Sigma V^H of the m x k matrix a
 * (m >= k) by one-sided Jacobi (Hestenes): rotate column pairs of a copy W
 * until every pair is orthogonal; then sigma_i = ||w_i|| and u_i = w_i /
 * sigma_i, sorted by decreasing sigma.  A pair (p, q) with Gram entries
 * alpha = ||w_p||^2, beta = ||w_q||^2, gamma = w_p^H w_q = |gamma| e^{i phi}
 * is made orthogonal by w_q <- e^{-i phi} w_q followed by the real rotation
 * [c s; -s c] with t = s/c the smaller root of t^2 + 2 zeta t - 1 = 0,
 * zeta = (beta - alpha) / (2 |gamma|).  A column with sigma = 0 gives a zero
 * u column.  Returns 0, or OR_ENOCONV after 60 sweeps. */
int or_zsvd_jacobi(int m, int k, const zc *a, int lda, zc *u, int ldu, double *sigma)
{
    if (m < k || k < 0) return OR_EINVAL;
    zc *w = malloc(sizeof(zc) * (size_t)m * k);
    for (int j = 0; j < k; ++j) memcpy(w + (size_t)j * m, a + (size_t)j * lda, sizeof(zc) * m);
    const double tol = 1e-15;
    int st = OR_ENOCONV;
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < k - 1; ++p)
            for (int q = p + 1; q < k; ++q) {
                zc *wp = w + (size_t)p * m, *wq = w + (size_t)q * m;
                double al = 0.0, be = 0.0;
                zc ga = 0.0;
                for (int i = 0; i < m; ++i) {
                    al += creal(wp[i] * conj(wp[i]));
                    be += creal(wq[i] * conj(wq[i]));
                    ga += conj(wp[i]) * wq[i];
                }
                double g = cabs(ga);
                if (g == 0.0 || g <= tol * sqrt(al * be)) continue;
                rotated = 1;
                zc ph = conj(ga) / g;               /* e^{-i phi} */
                double zeta = (be - al) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = 0; i < m; ++i) {
                    zc x = wp[i], y = ph * wq[i];
                    wp[i] = cs * x - sn * y;
                    wq[i] = sn * x + cs * y;
                }
            }
        if (!rotated) { st = OR_OK; break; }
    }
    /* sigma, u, sorted by decreasing sigma (selection sort on columns) */
    for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += creal(w[IDX(i, j, m)] * conj(w[IDX(i, j, m)]));
        sigma[j] = sqrt(s);
    }
    for (int j = 0; j < k; ++j) {
        int best = j;
        for (int l = j + 1; l < k; ++l)
            if (sigma[l] > sigma[best]) best = l;
        if (best != j) {
            double ts = sigma[j]; sigma[j] = sigma[best]; sigma[best] = ts;
            for (int i = 0; i < m; ++i) {
                zc tz = w[IDX(i, j, m)]; w[IDX(i, j, m)] = w[IDX(i, best, m)]; w[IDX(i, best, m)] = tz;
            }
        }
        double inv = sigma[j] > 0.0 ? 1.0 / sigma[j] : 0.0;
        for (int i = 0; i < m; ++i) u[IDX(i, j, ldu)] = w[IDX(i, j, m)] * inv;
    }
    free(w);
    return st;
}

/* Algorithm Block_CIRR with the context's pencil, contour and quadrature:
 *   1. R_i = F_i Y (i = 0..g-1), F_i the moment integrals of Section 2.1
 *      taken by the context's quadrature; the moments are the shifted and
 *      scaled ((z - centre) / a)^i (they span the same space as z^i,
 *      degree by degree);
 *   2. the SVD [R_0, ..., R_{g-1}] = U Sigma V^H (all t = h g columns of U);
 *   3. A^ = U^H A U, B^ = U^H B U;  4. its t eigenpairs;
 *   5. x_i = U y_i, and the selection GFEAST uses (inside the contour and
 *      eq. 5.1 residual below eta).
 * Y: n x h.  Outputs (each t long / n x t): lam, X, res of the selected
 * pairs, *count of them; sigma (t) the singular values of step 2.  Returns
 * 0, OR_EINVAL, or OR_ENOCONV (SVD or QZ). */
int or_cirr(const or_ctx *c, const zc *Y, int h, int g, int *count, zc *lam, zc *X, double *res, double *sigma)
{
    int n = c->n, q = c->q;
    *count = 0;
    if (h < 1 || g < 1 || (size_t)h * g > (size_t)n) return OR_EINVAL;
    int t = h * g;
    size_t nh = (size_t)n * h, nt = (size_t)n * t;
    zc *Xs = malloc(sizeof(zc) * nh * q), *R = calloc(nt, sizeof(zc)), *U = malloc(sizeof(zc) * nt);
    zc *AU = malloc(sizeof(zc) * nt), *BU = malloc(sizeof(zc) * nt);
    zc *Ah = malloc(sizeof(zc) * (size_t)t * t), *Bh = malloc(sizeof(zc) * (size_t)t * t);
    zc *al = malloc(sizeof(zc) * t), *be = malloc(sizeof(zc) * t), *Yv = malloc(sizeof(zc) * (size_t)t * t);
    zc *Xr = malloc(sizeof(zc) * nt), *AX = malloc(sizeof(zc) * nt), *BX = malloc(sizeof(zc) * nt);
    /* step 1: X_j = (z_j B - A)^{-1} Y, then the weighted moments */
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int j = 0; j < q; ++j)
        for (int col = 0; col < h; ++col) {
            zc *x = Xs + ((size_t)j * h + col) * n;
            memcpy(x, Y + (size_t)col * n, sizeof(zc) * n);
            if (c->kind == 0)
                or_zgetrs(n, 1, c->fac + j * c->fac_stride, c->ldf, c->piv + (size_t)j * n, x, n);
            else
                or_zgbtrs(n, c->kl, c->ku, 1, c->fac + j * c->fac_stride, c->ldf, c->piv + (size_t)j * n, x, n);
        }
    zc centre = c->cre + I * c->cim;
    for (int i = 0; i < g; ++i)
        for (int j = 0; j < q; ++j) {
            zc wz = c->w[j] * cpow((c->z[j] - centre) / c->ca, (double)i);
            for (size_t e = 0; e < nh; ++e) R[(size_t)i * nh + e] += wz * Xs[(size_t)j * nh + e];
        }
    /* step 2 */
    int st = or_zsvd_jacobi(n, t, R, n, U, n, sigma);
    if (!st) {
        /* step 3 */
        pencil_apply(c, 0, t, U, AU);
        pencil_apply(c, 1, t, U, BU);
        or_zgemm(1, t, t, n, U, n, AU, n, Ah, t);
        or_zgemm(1, t, t, n, U, n, BU, n, Bh, t);
        /* step 4 */
        st = or_zggev(t, Ah, t, Bh, t, al, be, Yv, t);
    }
    if (!st) {
        /* step 5 */
        or_zgemm(0, n, t, t, U, n, Yv, t, Xr, n);
        pencil_apply(c, 0, t, Xr, AX);
        pencil_apply(c, 1, t, Xr, BX);
        for (int i = 0; i < t; ++i) {
            if (!(cabs(be[i]) > 0.0)) continue;
            zc l = al[i] / be[i];
            double num = 0.0, na = 0.0, nb = 0.0;
            for (int p = 0; p < n; ++p) {
                zc ax = AX[IDX(p, i, n)], bx = BX[IDX(p, i, n)], d = ax - l * bx;
                num += creal(d * conj(d)); na += creal(ax * conj(ax)); nb += creal(bx * conj(bx));
            }
            double r = sqrt(num) / (sqrt(na) + sqrt(nb));
            if (or_inside(c->ckind, c->cre, c->cim, c->ca, c->cb, creal(l), cimag(l)) && r < c->eta) {
                lam[*count] = l;
                res[*count] = r;
                memcpy(X + (size_t)(*count) * n, Xr + (size_t)i * n, sizeof(zc) * n);
                ++*count;
            }
        }
    }
    free(Xs); free(R); free(U); free(AU); free(BU); free(Ah); free(Bh);
    free(al); free(be); free(Yv); free(Xr); free(AX); free(BX);
    return st;
}
