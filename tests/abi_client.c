/* A plain C client of libfif (no Python, no PyTorch): builds a small field on the GPU, queries it
 * through fif_query_host (host buffers, copies on a second stream) and through fif_query
 * (device buffers), and checks that the two agree bitwise, that in-lattice poses get finite
 * metrics and that no bounded device wait ran out.  Prints "abi client ok" and exits 0 on
 * success.  Built and run by tests/test_abi_cpu.py (compile and link) and
 * tests/test_gpu_query.py (run). */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "fif.h"

#define CHECK(x)                                                                     \
    do {                                                                             \
        int32_t rc_ = (int32_t)(x);                                                  \
        if (rc_ != 0) {                                                              \
            fprintf(stderr, "%s:%d: %s -> %d (%s)\n", __FILE__, __LINE__, #x, rc_,   \
                    rc_ < 0 ? fif_status_str(rc_) : "cuda");                         \
            return 1;                                                                \
        }                                                                            \
    } while (0)

static uint32_t lcg = 12345u;
static float uniform(float lo, float hi) {
    lcg = lcg * 1664525u + 1013904223u;
    return lo + (hi - lo) * (float)(lcg >> 8) * (1.0f / 16777216.0f);
}

int main(void) {
    enum { N = 600, M = 100, CHUNK = 32 };
    const fif_grid grid = {{0.f, 0.f, 0.f}, 0.5f, 9, 9, 4};
    fif_params prm;
    memset(&prm, 0, sizeof prm);
    prm.half_fov = 0.78539816339744831;
    prm.v_alpha = 0.8;
    prm.r_min = 0.1;
    prm.r_max = 5.0;
    prm.sigma = 1.0;

    static float lm[N][3], poses[M][7];
    for (int i = 0; i < N; ++i) {
        lm[i][0] = uniform(0.f, 4.f);
        lm[i][1] = uniform(0.f, 4.f);
        lm[i][2] = uniform(0.f, 1.5f);
    }
    for (int i = 0; i < M; ++i) {
        poses[i][0] = uniform(0.2f, 3.8f);
        poses[i][1] = uniform(0.2f, 3.8f);
        poses[i][2] = uniform(0.2f, 1.3f);
        float q[4], n = 0.f;
        for (int c = 0; c < 4; ++c) {
            q[c] = uniform(-1.f, 1.f);
            n += q[c] * q[c];
        }
        n = sqrtf(n);
        for (int c = 0; c < 4; ++c) poses[i][3 + c] = q[c] / n;
    }

    fif_field field;
    const size_t fbytes = fif_field_bytes(&grid, FIF_STORAGE_F32);
    void *d_coeffs = NULL, *d_ws = NULL, *d_staging = NULL;
    float *d_lm = NULL, *d_poses = NULL;
    double* d_met = NULL;
    CHECK(cudaMalloc(&d_coeffs, fbytes));
    CHECK(fif_field_init(&field, &grid, &prm, FIF_STORAGE_F32, d_coeffs, fbytes));
    const size_t wsb = fif_build_workspace_bytes(&field, N);
    CHECK(cudaMalloc(&d_ws, wsb));
    CHECK(cudaMalloc((void**)&d_lm, sizeof lm));
    CHECK(cudaMemcpy(d_lm, lm, sizeof lm, cudaMemcpyHostToDevice));
    cudaStream_t s, cs;
    CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CHECK(fif_build(&field, d_lm, N, d_ws, wsb, (fif_stream_t)s));

    /* host buffers through fif_query_host */
    double *h_met = NULL, *h_met2 = NULL;
    CHECK(cudaMallocHost((void**)&h_met, M * 3 * sizeof(double)));
    h_met2 = (double*)malloc(M * 3 * sizeof(double));
    int32_t h_st[M];
    const size_t sb = fif_query_host_staging_bytes(CHUNK);
    CHECK(cudaMalloc(&d_staging, sb));
    CHECK(fif_query_host(&field, &poses[0][0], M, FIF_Q_METRICS, NULL, h_met, NULL, h_st, CHUNK, d_staging, sb,
                         (fif_stream_t)s, (fif_stream_t)cs));
    /* device buffers through fif_query */
    CHECK(cudaMalloc((void**)&d_poses, sizeof poses));
    CHECK(cudaMalloc((void**)&d_met, M * 3 * sizeof(double)));
    CHECK(cudaMemcpyAsync(d_poses, poses, sizeof poses, cudaMemcpyHostToDevice, s));
    CHECK(fif_query(&field, d_poses, M, FIF_Q_METRICS, NULL, d_met, NULL, NULL, (fif_stream_t)s));
    CHECK(cudaMemcpyAsync(h_met2, d_met, M * 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CHECK(cudaStreamSynchronize(s));
    int32_t dev_err = 0;
    CHECK(fif_device_error(&dev_err, 0, (fif_stream_t)s));
    if (dev_err != 0) {
        fprintf(stderr, "device error %d\n", dev_err);
        return 1;
    }
    if (memcmp(h_met, h_met2, M * 3 * sizeof(double)) != 0) {
        fprintf(stderr, "host-buffer and device-buffer queries differ\n");
        return 1;
    }
    for (int i = 0; i < M; ++i) {
        if ((h_st[i] & FIF_POSE_OUTSIDE) == 0 && !(isfinite(h_met[3 * i]) && h_met[3 * i] > 0.0)) {
            fprintf(stderr, "pose %d: trace %g\n", i, h_met[3 * i]);
            return 1;
        }
    }
    printf("abi client ok: version %d, trace[0] %.6g, log|det|[0] %.6g\n", fif_version(), h_met[0], h_met[1]);
    cudaFree(d_coeffs);
    cudaFree(d_ws);
    cudaFree(d_staging);
    cudaFree(d_lm);
    cudaFree(d_poses);
    cudaFree(d_met);
    cudaFreeHost(h_met);
    free(h_met2);
    cudaStreamDestroy(s);
    cudaStreamDestroy(cs);
    return 0;
}
