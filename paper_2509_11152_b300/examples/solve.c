/* Plain-C use of the h2rs C-ABI on the GPU: factorise and solve a hand-built H^2
 * matrix.  The structure is that of plan_query.c (n = 8, depth 2, leaves of 2 points,
 * rank-1 bases; leaf pairs (0,2), (0,3), (1,3) and transposes admissible).  Values:
 * the kernel exp(-|x - y| / 0.5) at x_i = (i + 1/2) / 8 with 1.1 on the diagonal;
 * orthonormal bases U_i = [1, 1] / sqrt 2 and transfers 1 / sqrt 2 (so every basis is
 * the normalised constant), couplings S_st = U_s^T K_st U_t, exact near-field blocks.
 *
 * Steps: ||A|| by power iteration with h2_matvec; a float64 factor and solve
 * (Alg. 1, Alg. 3) checked by its residual; a float32 factor refined in float64 to a
 * backward error of 1e-10.  Host pointers throughout (the library copies).
 *
 * Build: cc solve.c -I<repo>/include -L<dir of libh2rs.so> -lh2rs -lm -o solve
 * Without a GPU every call returns a status code (H2_ERR_CUDA) and the program exits 2.
 */
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "h2rs.h"

enum { N = 8, NN = 7, NLEAF = 4, NADM = 6, NNEAR = 10 };

static double kernel(int i, int j) {
    const double xi = (i + 0.5) / N, xj = (j + 0.5) / N;
    return i == j ? 1.1 : exp(-fabs(xi - xj) / 0.5);
}

static double norm2(const double* v, int n) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += v[i] * v[i];
    return sqrt(s);
}

static int fail(const char* what, int rc) {
    fprintf(stderr, "%s failed (%d): %s\n", what, rc, h2_last_error());
    return 2;
}

int main(void) {
    /* heap numbering: 0 root; 1, 2 level 1; 3..6 leaves of 2 points */
    int64_t node_start[NN] = {0, 0, 4, 0, 2, 4, 6};
    int64_t node_size[NN] = {8, 4, 4, 2, 2, 2, 2};
    int64_t rank[NN] = {1, 1, 1, 1, 1, 1, 1};
    int64_t U_off[NLEAF + 1] = {0, 2, 4, 6, 8};
    int64_t E_off[NN + 1] = {0, 0, 1, 2, 3, 4, 5, 6};
    int64_t adm_ptr[NN + 1] = {0, 0, 0, 0, 2, 3, 4, 6};
    int64_t adm_col[NADM] = {5, 6, 6, 3, 3, 4};
    int64_t S_off[NADM + 1] = {0, 1, 2, 3, 4, 5, 6};
    int64_t inad_ptr[NN + 1] = {0, 1, 3, 5, 7, 10, 13, 15};
    int64_t inad_col[15] = {0, 1, 2, 1, 2, 3, 4, 3, 4, 5, 4, 5, 6, 5, 6};
    int64_t D_off[NNEAR + 1] = {0, 4, 8, 12, 16, 20, 24, 28, 32, 36, 40};
    double U[8], E[6], S[NADM], D[40];
    const double r2 = 1.0 / sqrt(2.0);
    for (int i = 0; i < 8; ++i) U[i] = r2;
    for (int g = 0; g < 6; ++g) E[g] = r2;
    /* couplings: U_s^T K_st U_t = (sum of the 2 x 2 kernel block) / 2 */
    for (int s = 3; s < NN; ++s)
        for (int64_t e = adm_ptr[s]; e < adm_ptr[s + 1]; ++e) {
            const int t = (int)adm_col[e];
            double sum = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) sum += kernel((int)node_start[s] + a, (int)node_start[t] + b);
            S[e] = 0.5 * sum;
        }
    /* near field: the j-th inadmissible entry of a leaf row, 2 x 2 column-major */
    for (int s = 3, j = 0; s < NN; ++s)
        for (int64_t e = inad_ptr[s]; e < inad_ptr[s + 1]; ++e, ++j) {
            const int t = (int)inad_col[e];
            for (int c = 0; c < 2; ++c)
                for (int r = 0; r < 2; ++r)
                    D[D_off[j] + r + 2 * c] = kernel((int)node_start[s] + r, (int)node_start[t] + c);
        }

    h2_matrix_desc d;
    memset(&d, 0, sizeof d);
    d.n = N;
    d.depth = 2;
    d.values_on_device = 0;
    d.node_start = node_start;
    d.node_size = node_size;
    d.rank = rank;
    d.U_off = U_off;
    d.U = U;
    d.E_off = E_off;
    d.E = E;
    d.adm_ptr = adm_ptr;
    d.adm_col = adm_col;
    d.S_off = S_off;
    d.S = S;
    d.inad_ptr = inad_ptr;
    d.inad_col = inad_col;
    d.D_off = D_off;
    d.D = D;

    h2_matrix* A = NULL;
    int rc = h2_matrix_create(&d, &A);
    if (rc != H2_OK) return fail("h2_matrix_create", rc);

    /* ||A||_2 by power iteration (A is symmetric) */
    double v[N], w[N], norm_a = 0;
    for (int i = 0; i < N; ++i) v[i] = 1.0 + 0.1 * i;
    for (int it = 0; it < 50; ++it) {
        const double nv = norm2(v, N);
        for (int i = 0; i < N; ++i) v[i] /= nv;
        if ((rc = h2_matvec(A, 1, v, N, w, N, 0)) != H2_OK) return fail("h2_matvec", rc);
        norm_a = norm2(w, N);
        memcpy(v, w, sizeof v);
    }

    /* float64 factor and solve, in place on the host vector */
    h2_factor_opts o;
    memset(&o, 0, sizeof o);
    o.eps_lu = 1e-12;
    o.norm_a = norm_a;
    o.precision = H2_PREC_FP64;
    h2_factor* Z = NULL;
    if ((rc = h2_factor_create(A, &o, &Z)) != H2_OK) return fail("h2_factor_create", rc);
    double b[N], x[N], Ax[N];
    for (int i = 0; i < N; ++i) b[i] = 1.0;
    memcpy(x, b, sizeof x);
    if ((rc = h2_solve(Z, 1, x, N, 0)) != H2_OK) return fail("h2_solve", rc);
    if ((rc = h2_matvec(A, 1, x, N, Ax, N, 0)) != H2_OK) return fail("h2_matvec", rc);
    double res[N];
    for (int i = 0; i < N; ++i) res[i] = b[i] - Ax[i];
    const double berr64 = norm2(res, N) / (norm_a * norm2(x, N));
    printf("||A|| = %.6f; float64 factor + solve: backward error %.2e\n", norm_a, berr64);
    h2_factor_destroy(Z);

    /* float32 factor, float64 refinement */
    o.eps_lu = 1e-6;
    o.precision = H2_PREC_FP32;
    if ((rc = h2_factor_create(A, &o, &Z)) != H2_OK) return fail("h2_factor_create", rc);
    int32_t iters = 0;
    double berr = 0;
    memset(x, 0, sizeof x);
    rc = h2_refine_solve(Z, A, 1, b, N, x, N, 1e-10, 30, 0, &iters, &berr);
    printf("float32 factor + %d float64 corrections: backward error %.2e (status %d)\n", iters, berr, rc);
    h2_factor_destroy(Z);
    h2_matrix_destroy(A);
    return (rc == H2_OK && berr64 <= 1e-12 && berr <= 1e-10) ? 0 : 1;
}
