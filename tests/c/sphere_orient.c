/*
 * A plain C caller of the library (no Python, no torch): orients the normals
 * of a Fibonacci sphere with the iteration of Alg. 3 and checks the result
 * against the outward normals and the winding number at the points
 * (Thm. 1: F = 1/2 on the surface).  Exit status 0 when every check passes.
 *
 *   sphere_orient [n]      (default n = 20000)
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "wnnc.h"

#define CHECK(call)                                                            \
    do {                                                                       \
        wnnc_status st_ = (call);                                              \
        if (st_ != WNNC_OK) {                                                  \
            fprintf(stderr, "%s failed: %d %s\n", #call, (int)st_, wnnc_last_error()); \
            return 1;                                                          \
        }                                                                      \
    } while (0)
#define CUDA(call)                                                             \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_)); \
            return 1;                                                          \
        }                                                                      \
    } while (0)

int main(int argc, char** argv) {
    const int64_t n = argc > 1 ? atoll(argv[1]) : 20000;
    const double golden = 3.14159265358979323846 * (3.0 - sqrt(5.0));
    float* x = malloc(sizeof(float) * 3 * n);
    float* mu = malloc(sizeof(float) * 3 * n);
    float* F = malloc(sizeof(float) * n);
    if (!x || !mu || !F) return 1;
    for (int64_t i = 0; i < n; ++i) {      /* golden-angle spiral on the unit sphere */
        const double z = 1.0 - 2.0 * ((double)i + 0.5) / (double)n;
        const double r = sqrt(1.0 - z * z), a = golden * (double)i;
        x[3 * i] = (float)(r * cos(a));
        x[3 * i + 1] = (float)(r * sin(a));
        x[3 * i + 2] = (float)z;
    }
    float *dx, *dmu, *dF;
    CUDA(cudaMalloc((void**)&dx, sizeof(float) * 3 * n));
    CUDA(cudaMalloc((void**)&dmu, sizeof(float) * 3 * n));
    CUDA(cudaMalloc((void**)&dF, sizeof(float) * n));
    CUDA(cudaMemcpy(dx, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice));

    wnnc_tree_params tp;
    wnnc_iter_params ip;
    CHECK(wnnc_tree_params_default(&tp));
    CHECK(wnnc_iter_params_default(&ip));
    ip.n_iter = 10;
    wnnc_tree* tree = NULL;
    CHECK(wnnc_build_tree(dx, n, &tp, NULL, &tree));
    CHECK(wnnc_iterate(tree, dmu, NULL, &ip, NULL, NULL));
    CHECK(wnnc_eval_w(tree, dmu, ip.w1, dF, NULL));
    CHECK(wnnc_sync_status(tree, NULL));
    CUDA(cudaMemcpy(mu, dmu, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost));
    CUDA(cudaMemcpy(F, dF, sizeof(float) * n, cudaMemcpyDeviceToHost));
    int64_t far_pairs = 0, near_pairs = 0;
    CHECK(wnnc_get_stats(tree, &far_pairs, &near_pairs));
    CHECK(wnnc_tree_free(tree));

    /* every normal points outward (the sphere's outward normal is x itself) */
    int64_t outward = 0;
    double fmean = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double d = x[3 * i] * mu[3 * i] + x[3 * i + 1] * mu[3 * i + 1] + x[3 * i + 2] * mu[3 * i + 2];
        outward += d > 0.0;
        fmean += F[i];
    }
    fmean /= (double)n;
    printf("n %lld, outward %lld, mean F %.4f, pairs per operator %lld\n", (long long)n, (long long)outward,
           fmean, (long long)(far_pairs + near_pairs));
    cudaFree(dx);
    cudaFree(dmu);
    cudaFree(dF);
    free(x);
    free(mu);
    free(F);
    if (outward != n) return 2;
    if (fabs(fmean - 0.5) > 0.02) return 3;
    return 0;
}
