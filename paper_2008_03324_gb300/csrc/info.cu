// info.cu -- information threshold and potential cost (Sec. VI-B of the paper; sm_103a).
//
// Threshold.  The paper turns a localisation specification (M landmarks in the field of view
// between d_min and d_max) into a threshold for any metric of any map representation: draw
// sets meeting the specification, compute the metric each representation gives for each set,
// and average.  For a field the value is what the field built from the set returns at the
// node the camera sits on, which by Eq. fim_separation is the point-cloud sum weighted by the
// field's visibility model; so every representation reduces to
//   I_s = sum_i v(u_i) I_i,   I_i = [[P/n^2, -[u]x/n], [[u]x/n, P]] / sigma^2,
// with v = 1 (point cloud: every landmark of a set is in the field of view), v_quad(cos theta)
// (quadratic field, Eq. quad_vis_approx) or v_gp(e3; u) = a(e3)^T v^s(u) (GP field, Eq.
// gp_vis_approx; a = (K^s + s_n^2 I)^-1 K_e3 computed once on the host in double precision).
//
// info_sets_kernel: a warp per set, lanes over the set's landmarks accumulate the 15 moments of
// bearing.cuh (fixed-order butterfly across lanes); once a warp has 32 sets, lane = set expands
// them to the FIM and computes trace / log|det| / lambda_min as the query does.
// info_mean_kernel: one CTA, fixed-order double-precision means over the sets (optionally only
// those with lambda_min > 1e-6 trace), so the result is bitwise reproducible.
// info_cost_kernel: the potential cost (Eq. info_pot_cost) and its derivative, elementwise.
#include "bearing.cuh"
#include "fif_common.cuh"
#include "fif_internal.h"

#include <cmath>

namespace fif {

namespace {

constexpr int kIWarps = 8;
constexpr int kIThreads = kIWarps * 32;

__global__ void __launch_bounds__(kIThreads, 1) info_sets_kernel(InfoArgs a) {
    __shared__ float mom[kIWarps][32][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t groups = (a.n + 31) / 32;
    const float ca = a.gp_cos_alpha, ks = a.gp_ks;
    for (int64_t g = (int64_t)blockIdx.x * kIWarps + warp; g < groups; g += (int64_t)gridDim.x * kIWarps) {
        const int64_t s0 = g * 32;
        const int cnt = (a.n - s0 < 32) ? (int)(a.n - s0) : 32;
        for (int k = 0; k < cnt; ++k) {
            const float* set = a.sets + (s0 + k) * (int64_t)a.m * 3;
            float mo[15];
#pragma unroll
            for (int q = 0; q < 15; ++q) mo[q] = 0.f;
            for (int i = lane; i < a.m; i += 32) {
                const float px = __ldg(set + 3 * i), py = __ldg(set + 3 * i + 1), pz = __ldg(set + 3 * i + 2);
                const float n2 = px * px + py * py + pz * pz;
                const float r = rsqrtf(n2);
                const float x = px * r, y = py * r, z = pz * r;
                float v = 1.f;
                if (a.model == FIF_MODEL_QUAD) {
                    v = fmaf(fmaf(a.k2, z, a.k1), z, a.k0);
                } else if (a.model == FIF_MODEL_GP) {
                    v = 0.f;
                    for (int s = 0; s < a.gp_ns; ++s) {
                        const float c = fmaf(a.gp_axes[s][0], x, fmaf(a.gp_axes[s][1], y, a.gp_axes[s][2] * z));
                        v = fmaf(a.gp_a[s], 1.f / (1.f + expf(-ks * (c - ca))), v);
                    }
                }
                const float w2 = r * r;
                const float t[15] = {x * x, y * y, z * z, x * y, x * z, y * z, x * x * w2, y * y * w2, z * z * w2,
                                     x * y * w2, x * z * w2, y * z * w2, x * r, y * r, z * r};
#pragma unroll
                for (int q = 0; q < 15; ++q) mo[q] = fmaf(v, t[q], mo[q]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 15; ++q) mo[q] += __shfl_xor_sync(0xffffffffu, mo[q], o);
            if (lane == 0)
#pragma unroll
                for (int q = 0; q < 15; ++q) mom[warp][k][q] = mo[q];
        }
        __syncwarp();
        if (lane < cnt) {
            const int64_t s = s0 + lane;
            float fim[21];
#pragma unroll
            for (int e = 0; e < 21; ++e) fim[e] = bearing_entry(e, mom[warp][lane]) * a.inv_sigma2;
            const double tr = (double)trace6(fim);
            double lad;
            int sg;
            logdet_f64(fim, lad, sg);
            const double lm = lambda_min_f64(fim);
            a.metrics[3 * s + 0] = tr;
            a.metrics[3 * s + 1] = lad;
            a.metrics[3 * s + 2] = lm;
            if (a.sign) a.sign[s] = (int8_t)sg;
        }
        __syncwarp();
    }
}

// fixed-order means of the three metric columns (count: sets with lambda_min > 1e-6 trace
// when a.exclude, else all)
__global__ void __launch_bounds__(1024) info_mean_kernel(const double* __restrict__ met, int64_t n, int exclude,
                                                         double* __restrict__ out) {
    __shared__ double part[4][1024];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, c = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        const double tr = met[3 * i], ld = met[3 * i + 1], lm = met[3 * i + 2];
        if (exclude && !(lm > 1e-6 * tr)) continue;
        s0 += tr;
        s1 += ld;
        s2 += lm;
        c += 1.0;
    }
    part[0][threadIdx.x] = s0;
    part[1][threadIdx.x] = s1;
    part[2][threadIdx.x] = s2;
    part[3][threadIdx.x] = c;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
#pragma unroll
            for (int q = 0; q < 4; ++q) part[q][threadIdx.x] += part[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double cnt = part[3][0];
        for (int q = 0; q < 3; ++q) out[q] = cnt > 0.0 ? part[q][0] / cnt : (double)NAN;
    }
}

__global__ void info_cost_kernel(const double* __restrict__ v, int64_t m, int64_t stride, double eps, double kq,
                                 double* __restrict__ cost, double* __restrict__ dcost) {
    const double kl = -2.0 * kq * eps, bl = kq * eps * eps;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = v[i * stride];
        double c, d;
        if (x != x) { c = x; d = x; }
        else if (x > eps) { c = 0.0; d = 0.0; }
        else if (x >= 0.0) { c = kq * (x - eps) * (x - eps); d = 2.0 * kq * (x - eps); }
        else { c = fma(kl, x, bl); d = kl; }
        if (cost) cost[i] = c;
        if (dcost) dcost[i] = d;
    }
}

}  // namespace

int launch_info_threshold(const InfoArgs& a, int exclude, double* d_threshold, cudaStream_t stream) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (a.n + 31) / 32;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((groups + kIWarps - 1) / kIWarps, 8 * (int64_t)sms));
    if (a.n > 0) info_sets_kernel<<<(unsigned)grid, kIThreads, 0, stream>>>(a);
    if (d_threshold) info_mean_kernel<<<1, 1024, 0, stream>>>(a.metrics, a.n, exclude, d_threshold);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

int launch_info_cost(const double* v, int64_t m, int64_t stride, double eps, double kq, double* cost, double* dcost,
                     cudaStream_t stream) {
    if (m == 0) return FIF_OK;
    const int T = 256;
    const int64_t blocks = std::min<int64_t>((m + T - 1) / T, 152 * 16);
    info_cost_kernel<<<(unsigned)blocks, T, 0, stream>>>(v, m, stride, eps, kq, cost, dcost);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

}  // namespace fif
