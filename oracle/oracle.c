/*
 * oracle.c — plain, slow, obviously correct CPU FP64 oracle for the
 * matrix-valued biquaternion product  C <- alpha * op(A) * op(B) + beta * C.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline arm use it.  It shares no code, table or helper with the CUDA
 * library under paper_2609_02081_gb300/.
 *
 * What it computes (arXiv 2609.02081, "Biquaternion Algebra with Bilinear
 * Multiplication"):
 *   - Storage (Sec. III, Eq. biquat-repres): an m x n biquaternion matrix is
 *     eight real m x n matrices [M1..M8] = [E_R, E_I, F_R, F_I, G_I, -G_R,
 *     H_I, -H_R]; here laid out component-major, each component row-major.
 *   - Complex coefficients (Sec. III, Eq. main-biquat-eqn): the coefficient of
 *     the basis element 1, i, j, k is q_e = M_e + i*M_{e+4}, e = 1..4.
 *   - Scalar-vector form (Sec. II A, Eq. defQ): q = s + v . qv with the
 *     reversed vector qv = (k, j, i), so s = q_1, v_z = q_2, v_y = q_3,
 *     v_x = q_4.
 *   - Product (Sec. II A, Eq. MatrixQMultiplication): for matrix-valued
 *     biquaternions Q1 Q2 = (S1 S2 - V1 . V2) + (S1 V2 + V1 S2 - V1 x V2) . qv,
 *     dot and cross products taken component-wise with the order of the
 *     matrix factors preserved.  Every one of the 16 complex matrix products
 *     is formed with four real matrix products (the component-wise 64-product
 *     algorithm the paper calls HMAT-standard, Sec. III B), sums over the
 *     inner index in ascending order.
 *   - op(X) (Sec. III, the transposition, complex-conjugation and Hermitian-
 *     conjugation equations): a sign per component plus, for T and dagger, a
 *     transposition of every component.  Quaternion conjugation (vector part
 *     negated, no transposition) is added as a fifth op.
 *   - Complex scaling and addition (Sec. III, the scaling and addition
 *     equations): (alpha M)_c = aR M_c - aI M_{c+4},
 *     (alpha M)_{c+4} = aR M_{c+4} + aI M_c, c = 1..4; addition per component.
 *     With beta == 0 the incoming C is not read (BLAS convention).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC oracle.c
 * (fp-contract off keeps x86 and Arm rounding identical: no fused multiply-add).
 * The only parallelism is independent output rows handed to OpenMP threads;
 * the arithmetic of every output element is the sequential definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OP_N = 0, ORC_OP_T = 1, ORC_OP_C = 2, ORC_OP_H = 3, ORC_OP_QC = 4 };

/* Sign of stored component c (0-based) under op; Sec. III op equations. */
static int orc_sign(int op, int c)
{
    static const int t_mask[8]  = {+1, +1, -1, +1, +1, +1, -1, +1}; /* X^T      */
    static const int c_mask[8]  = {+1, -1, +1, -1, -1, +1, -1, +1}; /* X^*      */
    static const int h_mask[8]  = {+1, -1, -1, -1, -1, +1, +1, +1}; /* X^dagger */
    static const int qc_mask[8] = {+1, -1, -1, -1, +1, -1, -1, -1}; /* q-bar    */
    switch (op) {
    case ORC_OP_N: return +1;
    case ORC_OP_T: return t_mask[c];
    case ORC_OP_C: return c_mask[c];
    case ORC_OP_H: return h_mask[c];
    case ORC_OP_QC: return qc_mask[c];
    default: return 0;
    }
}

static int orc_transposes(int op) { return op == ORC_OP_T || op == ORC_OP_H; }

/*
 * op(X) materialised.  X is 8 x rows x cols (contiguous); Y receives
 * 8 x rows' x cols' where (rows', cols') = (cols, rows) for T and dagger.
 * Returns 0, or -1 for an unknown op.
 */
int oracle_apply_op(int op, int64_t rows, int64_t cols, const double *X, double *Y)
{
    if (op < ORC_OP_N || op > ORC_OP_QC) return -1;
    const int tr = orc_transposes(op);
    for (int c = 0; c < 8; ++c) {
        const double s = (double)orc_sign(op, c);
        const double *x = X + (int64_t)c * rows * cols;
        double *y = Y + (int64_t)c * rows * cols;
        for (int64_t r = 0; r < rows; ++r)
            for (int64_t q = 0; q < cols; ++q) {
                const double v = s * x[r * cols + q];
                if (tr) y[q * rows + r] = v;
                else y[r * cols + q] = v;
            }
    }
    return 0;
}

/* A complex matrix held as two real planes (re, im), row-major, ld = cols. */
typedef struct { const double *re, *im; } orc_cmat;

/*
 * Row i of the complex product X*Y (X is m x k, Y is k x n) written to
 * (out_re, out_im), n entries: four real products, inner index ascending.
 *   Re = sum_k (Xr Yr) - sum_k (Xi Yi),   Im = sum_k (Xr Yi) + sum_k (Xi Yr)
 * Each of the four real sums is accumulated on its own, as four separate
 * real matrix products would be.
 */
static void orc_cmul_row(int64_t i, int64_t n, int64_t k, orc_cmat X, orc_cmat Y,
                         double *out_re, double *out_im, double *t_rr,
                         double *t_ii, double *t_ri, double *t_ir)
{
    for (int64_t j = 0; j < n; ++j) t_rr[j] = t_ii[j] = t_ri[j] = t_ir[j] = 0.0;
    for (int64_t p = 0; p < k; ++p) {
        const double xr = X.re[i * k + p], xi = X.im[i * k + p];
        const double *yr = Y.re + p * n, *yi = Y.im + p * n;
        for (int64_t j = 0; j < n; ++j) {
            t_rr[j] += xr * yr[j];
            t_ii[j] += xi * yi[j];
            t_ri[j] += xr * yi[j];
            t_ir[j] += xi * yr[j];
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        out_re[j] = t_rr[j] - t_ii[j];
        out_im[j] = t_ri[j] + t_ir[j];
    }
}

/* acc += sign * term (complex rows). */
static void orc_acc(int64_t n, double sign, const double *tre, const double *tim,
                    double *are, double *aim)
{
    for (int64_t j = 0; j < n; ++j) {
        are[j] += sign * tre[j];
        aim[j] += sign * tim[j];
    }
}

/*
 * Selected output rows of  C = alpha * Aop * Bop + beta * C_in  where Aop
 * (8 x m x k) and Bop (8 x k x n) already have op applied.
 *   rows[r] (r < nrows) are the output row indices; C_in and C_out hold
 *   those rows only: 8 x nrows x n each.  C_in may be NULL when beta == 0.
 *   threads <= 0 means the OpenMP default.
 * Returns 0 on success, -1 on a bad argument, -2 if out of memory.
 */
int oracle_bq_gemm_rows(int64_t m, int64_t n, int64_t k, double alpha_re,
                        double alpha_im, const double *Aop, const double *Bop,
                        double beta_re, double beta_im, const double *C_in,
                        const int64_t *rows, int64_t nrows, double *C_out,
                        int threads)
{
    if (m < 0 || n < 0 || k < 0 || nrows < 0) return -1;
    if (beta_re != 0.0 || beta_im != 0.0) {
        if (!C_in) return -1;
    }
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= m) return -1;

    const int64_t ca = m * k, cb = k * n, cc = nrows * n;
    /* Complex coefficients (Eq. main-biquat-eqn): q_e = M_e + i M_{e+4}.
     * Scalar-vector names (Eq. defQ): S = q1, Vz = q2, Vy = q3, Vx = q4. */
    const orc_cmat S1 = {Aop + 0 * ca, Aop + 4 * ca}, Vz1 = {Aop + 1 * ca, Aop + 5 * ca},
                   Vy1 = {Aop + 2 * ca, Aop + 6 * ca}, Vx1 = {Aop + 3 * ca, Aop + 7 * ca};
    const orc_cmat S2 = {Bop + 0 * cb, Bop + 4 * cb}, Vz2 = {Bop + 1 * cb, Bop + 5 * cb},
                   Vy2 = {Bop + 2 * cb, Bop + 6 * cb}, Vx2 = {Bop + 3 * cb, Bop + 7 * cb};
    int err = 0;

#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
    {
        /* per-thread rows: 8 accumulators (S, Vx, Vy, Vz; re and im),
         * one complex term, four real partial sums */
        double *buf = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 14);
        if (!buf) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = -2;
        } else {
            double *Sre = buf, *Sim = buf + n, *Xre = buf + 2 * n, *Xim = buf + 3 * n;
            double *Yre = buf + 4 * n, *Yim = buf + 5 * n, *Zre = buf + 6 * n, *Zim = buf + 7 * n;
            double *Tre = buf + 8 * n, *Tim = buf + 9 * n;
            double *t0 = buf + 10 * n, *t1 = buf + 11 * n, *t2 = buf + 12 * n, *t3 = buf + 13 * n;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (int64_t r = 0; r < nrows; ++r) {
                const int64_t i = rows[r];
                for (int64_t j = 0; j < 8 * n; ++j) buf[j] = 0.0;
#define ORC_TERM(XM, YM, SIGN, ACCRE, ACCIM)                                  \
    do {                                                                      \
        orc_cmul_row(i, n, k, XM, YM, Tre, Tim, t0, t1, t2, t3);              \
        orc_acc(n, SIGN, Tre, Tim, ACCRE, ACCIM);                             \
    } while (0)
                /* scalar part: S1 S2 - V1 . V2 */
                ORC_TERM(S1, S2, +1.0, Sre, Sim);
                ORC_TERM(Vx1, Vx2, -1.0, Sre, Sim);
                ORC_TERM(Vy1, Vy2, -1.0, Sre, Sim);
                ORC_TERM(Vz1, Vz2, -1.0, Sre, Sim);
                /* vector part: S1 V2 + V1 S2 - V1 x V2, with
                 * (a x b)_x = a_y b_z - a_z b_y, (a x b)_y = a_z b_x - a_x b_z,
                 * (a x b)_z = a_x b_y - a_y b_x */
                ORC_TERM(S1, Vx2, +1.0, Xre, Xim);
                ORC_TERM(Vx1, S2, +1.0, Xre, Xim);
                ORC_TERM(Vy1, Vz2, -1.0, Xre, Xim);
                ORC_TERM(Vz1, Vy2, +1.0, Xre, Xim);

                ORC_TERM(S1, Vy2, +1.0, Yre, Yim);
                ORC_TERM(Vy1, S2, +1.0, Yre, Yim);
                ORC_TERM(Vz1, Vx2, -1.0, Yre, Yim);
                ORC_TERM(Vx1, Vz2, +1.0, Yre, Yim);

                ORC_TERM(S1, Vz2, +1.0, Zre, Zim);
                ORC_TERM(Vz1, S2, +1.0, Zre, Zim);
                ORC_TERM(Vx1, Vy2, -1.0, Zre, Zim);
                ORC_TERM(Vy1, Vx2, +1.0, Zre, Zim);
#undef ORC_TERM
                /* product components back in storage order:
                 * q1 = S, q2 = Vz, q3 = Vy, q4 = Vx; M_e = Re q_e, M_{e+4} = Im q_e */
                const double *Qre[4] = {Sre, Zre, Yre, Xre};
                const double *Qim[4] = {Sim, Zim, Yim, Xim};
                for (int e = 0; e < 4; ++e) {
                    double *ore = C_out + (int64_t)e * cc + r * n;
                    double *oim = C_out + (int64_t)(e + 4) * cc + r * n;
                    const double *cre = C_in ? C_in + (int64_t)e * cc + r * n : NULL;
                    const double *cim = C_in ? C_in + (int64_t)(e + 4) * cc + r * n : NULL;
                    const int use_beta = (beta_re != 0.0 || beta_im != 0.0);
                    for (int64_t j = 0; j < n; ++j) {
                        /* alpha * Q (complex scaling equation) */
                        double vre = alpha_re * Qre[e][j] - alpha_im * Qim[e][j];
                        double vim = alpha_re * Qim[e][j] + alpha_im * Qre[e][j];
                        if (use_beta) {
                            /* + beta * C (scaling, then the addition equation) */
                            vre += beta_re * cre[j] - beta_im * cim[j];
                            vim += beta_re * cim[j] + beta_im * cre[j];
                        }
                        ore[j] = vre;
                        oim[j] = vim;
                    }
                }
            }
            free(buf);
        }
    }
    return err;
}

/* Number of threads OpenMP would use (for reporting the CPU baseline). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
