/* A plain C client of the C ABI (test infrastructure): it reads two 8 x m x k /
 * 8 x k x n biquaternion matrices as text from stdin, runs hmat_bq_gemm in both
 * modes and hmat_bq_add, and prints the results as text.  It uses only
 * include/hmat.h and the CUDA runtime for device memory, as a C caller would.
 *
 * stdin:  m n k, then A (8 m k values), then B (8 k n values), row-major per
 *         component.
 * stdout: C = A B in FP64 mode (8 m n values), C = A B in split mode with
 *         tol 1e-12, then D = A + (2 - i) A (8 m k values).
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "hmat.h"

static int check(hmat_status s, const char *what) {
    if (s != HMAT_STATUS_SUCCESS) {
        fprintf(stderr, "%s: %s (%s)\n", what, hmat_status_string(s), hmat_last_cuda_error());
        return 1;
    }
    return 0;
}

static int read_values(double *x, long count) {
    for (long i = 0; i < count; ++i)
        if (scanf("%lf", &x[i]) != 1) return 1;
    return 0;
}

static void print_values(const double *x, long count) {
    for (long i = 0; i < count; ++i) printf("%.17g\n", x[i]);
}

int main(void) {
    long m, n, k;
    if (scanf("%ld %ld %ld", &m, &n, &k) != 3) return 2;
    const long na = 8 * m * k, nb = 8 * k * n, nc = 8 * m * n;
    double *A = malloc(sizeof(double) * na), *B = malloc(sizeof(double) * nb);
    double *C = malloc(sizeof(double) * nc), *D = malloc(sizeof(double) * na);
    if (!A || !B || !C || !D || read_values(A, na) || read_values(B, nb)) return 2;

    double *dA, *dB, *dC, *dD;
    void *ws = NULL;
    if (cudaMalloc((void **)&dA, sizeof(double) * na) != cudaSuccess) return 3;
    if (cudaMalloc((void **)&dB, sizeof(double) * nb) != cudaSuccess) return 3;
    if (cudaMalloc((void **)&dC, sizeof(double) * nc) != cudaSuccess) return 3;
    if (cudaMalloc((void **)&dD, sizeof(double) * na) != cudaSuccess) return 3;
    cudaMemcpy(dA, A, sizeof(double) * na, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, B, sizeof(double) * nb, cudaMemcpyHostToDevice);

    hmat_handle h = NULL;
    if (check(hmat_create(&h), "hmat_create")) return 4;
    const double tol = 1e-12;
    hmat_gemm_desc d = {HMAT_OP_N, HMAT_OP_N, HMAT_BQ, HMAT_BQ, m, n, k, 1.0, 0.0, 0.0, 0.0,
                        dA, k, m * k, dB, n, k * n, dC, n, m * n};
    size_t bytes = 0;
    if (check(hmat_workspace_size(h, 1, &d, HMAT_MODE_SPLIT, tol, &bytes), "hmat_workspace_size")) return 4;
    if (bytes && cudaMalloc(&ws, bytes) != cudaSuccess) return 3;

    for (int mode = HMAT_MODE_FP64; mode <= HMAT_MODE_SPLIT; ++mode) {
        if (check(hmat_bq_gemm(h, HMAT_OP_N, HMAT_OP_N, HMAT_BQ, HMAT_BQ, m, n, k, 1.0, 0.0, dA, k, m * k, dB, n,
                               k * n, 0.0, 0.0, dC, n, m * n, mode, tol, ws, bytes, NULL),
                  "hmat_bq_gemm"))
            return 4;
        if (cudaMemcpy(C, dC, sizeof(double) * nc, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
        print_values(C, nc);
    }
    if (check(hmat_bq_add(h, HMAT_OP_N, HMAT_OP_N, HMAT_BQ, HMAT_BQ, m, k, 1.0, 0.0, dA, k, m * k, 2.0, -1.0, dA, k,
                          m * k, dD, k, m * k, NULL),
              "hmat_bq_add"))
        return 4;
    if (cudaMemcpy(D, dD, sizeof(double) * na, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    print_values(D, na);

    uint32_t err = 0;
    if (check(hmat_get_device_error(h, &err), "hmat_get_device_error") || err) return 5;
    hmat_destroy(h);
    cudaFree(ws);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dC);
    cudaFree(dD);
    free(A);
    free(B);
    free(C);
    free(D);
    return 0;
}
