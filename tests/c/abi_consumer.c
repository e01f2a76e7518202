/*
 * A plain C consumer of libsrmc: no Python, no torch.  Builds the cos-model
 * problem given on the command line, solves it on the current device, evaluates
 * y_i and z_i at every stratum centre for every step, and prints them, one
 * line per (i, k): "i k y z_1 .. z_d".  Used by tests/test_gpu_c_abi.py, which
 * compares the output with the oracle.
 *
 * usage: abi_consumer d N C a M s0 lam kap precision(32|64)
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "srmc.h"

#define CHECK(call)                                                              \
    do {                                                                         \
        srmc_status st_ = (call);                                                \
        if (st_ != SRMC_OK) {                                                    \
            fprintf(stderr, "%s failed: %d %s\n", #call, (int)st_, srmc_last_error()); \
            return 1;                                                            \
        }                                                                        \
    } while (0)

int main(int argc, char **argv)
{
    if (argc != 10) {
        fprintf(stderr, "usage: %s d N C a M s0 lam kap precision\n", argv[0]);
        return 2;
    }
    const int d = atoi(argv[1]), N = atoi(argv[2]), C = atoi(argv[3]);
    const double a = atof(argv[4]);
    const long long M = atoll(argv[5]);
    const double s0 = atof(argv[6]), lam = atof(argv[7]), kap = atof(argv[8]);
    const int prec = atoi(argv[9]) == 64 ? SRMC_FP64 : SRMC_FP32;
    if (d < 1 || d > SRMC_DMAX) return 2;

    double b[SRMC_DMAX] = {0}, sigma[SRMC_DMAX * SRMC_DMAX] = {0}, lo[SRMC_DMAX], hi[SRMC_DMAX];
    int cells[SRMC_DMAX];
    for (int l = 0; l < d; ++l) {
        sigma[l * d + l] = s0;
        lo[l] = -a;
        hi[l] = a;
        cells[l] = C;
    }
    const double params[4] = {lam, kap, 0.0, s0};
    srmc_problem pr = {0};
    pr.d = d; pr.q = d; pr.N = N; pr.T = 1.0; pr.b = b; pr.sigma = sigma;
    pr.model = SRMC_MODEL_COS; pr.params = params; pr.n_params = 4;
    srmc_strata sa = {0};
    sa.cells = cells; sa.lo = lo; sa.hi = hi; sa.mu = 1.0; sa.kind = SRMC_STRATA_EQUAL_SIZE;
    srmc_config cf = {0};
    cf.basis = SRMC_LP1; cf.prec = prec; cf.M = M; cf.seed = 1; cf.instance = 0;
    /* truncation (eq. TL): |u| <= e^{lam T}, so C_y = 2 e^{lam T} is inactive at the
     * solution; C_z = C_y / sqrt(dt) */
    cf.Cy = 2.0 * exp(lam * 1.0);
    cf.Cz = cf.Cy / sqrt(1.0 / N);

    srmc_solver *s = NULL;
    CHECK(srmc_create(&pr, &sa, &cf, &s));
    CHECK(srmc_solve(s, NULL));
    long long K = 0;
    CHECK(srmc_table(s, NULL, NULL, NULL, NULL, NULL, &K));

    double *dx = NULL, *dy = NULL, *dz = NULL;
    if (cudaMalloc((void **)&dx, sizeof(double) * K * d) != cudaSuccess ||
        cudaMalloc((void **)&dy, sizeof(double) * K) != cudaSuccess ||
        cudaMalloc((void **)&dz, sizeof(double) * K * d) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    double *hy = (double *)malloc(sizeof(double) * K), *hz = (double *)malloc(sizeof(double) * K * d);
    CHECK(srmc_centres(s, dx, NULL));
    for (int i = 0; i < N; ++i) {
        CHECK(srmc_eval(s, i, dx, K, dy, dz, NULL));
        if (cudaMemcpy(hy, dy, sizeof(double) * K, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(hz, dz, sizeof(double) * K * d, cudaMemcpyDeviceToHost) != cudaSuccess) {
            fprintf(stderr, "cudaMemcpy failed\n");
            return 1;
        }
        for (long long k = 0; k < K; ++k) {
            printf("%d %lld %.17g", i, k, hy[k]);
            for (int l = 0; l < d; ++l) printf(" %.17g", hz[k * d + l]);
            printf("\n");
        }
    }
    unsigned long long st[3];
    CHECK(srmc_stats(s, st));
    fprintf(stderr, "path-steps %llu, fallbacks %llu, non-finite %llu, version %d\n", st[2], st[0], st[1],
            srmc_version());
    free(hy); free(hz);
    cudaFree(dx); cudaFree(dy); cudaFree(dz);
    srmc_destroy(s);
    return 0;
}
