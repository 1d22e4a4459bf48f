// pointcloud.cu -- direct point-cloud FIM, the baseline the field replaces (sm_103a).
//
// Sec. IV / Eq. cost_info of the paper: for each pose T,
//   I_T = sum_{k in V} I_T(p_k),  V = landmarks in the range shell around t that project
//   inside the image (Eq. exact_vis_func),
// with I_T(p) the information of one bearing under the local (camera-frame) perturbation
// (second form of Eq. deriv_se3):
//   I = sigma^-2 [[P/n^2, -[u]x/n], [[u]x/n, P]],  u = p^c/n, P = I - u u^T.
//
// One thread = one pose (pose and accumulators in registers); all landmarks stream through
// a shared-memory tile that every thread of the CTA reads as a broadcast.  Per landmark the
// thread keeps 17 sums (u u^T/n^2, 1/n^2, u/n, u u^T, count) in compensated form (a block of
// 64 landmarks summed in registers, then Kahan-added).  The shell and visibility decisions
// round after every single-precision operation (no contraction) so that they are
// reproducible bit for bit.
#include "fif_common.cuh"
#include "fif_internal.h"

namespace fif {

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 512;    // landmarks per tile
constexpr int kBlock = 64;

// R_wc from a quaternion, normalised with one IEEE square root and four divisions, every
// product and sum rounded (the visibility decision depends on these exact values)
__device__ __forceinline__ void quat_to_rot_exact(const float q[4], float R[3][3], float& n2) {
    float s = __fadd_rn(__fmul_rn(q[0], q[0]), __fmul_rn(q[1], q[1]));
    s = __fadd_rn(s, __fmul_rn(q[2], q[2]));
    s = __fadd_rn(s, __fmul_rn(q[3], q[3]));
    n2 = s;
    const float r = __fsqrt_rn(s);
    const float w = __fdiv_rn(q[0], r), x = __fdiv_rn(q[1], r), y = __fdiv_rn(q[2], r), z = __fdiv_rn(q[3], r);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    R[0][0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(yy, zz)));
    R[0][1] = __fmul_rn(2.f, __fsub_rn(xy, wz));
    R[0][2] = __fmul_rn(2.f, __fadd_rn(xz, wy));
    R[1][0] = __fmul_rn(2.f, __fadd_rn(xy, wz));
    R[1][1] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, zz)));
    R[1][2] = __fmul_rn(2.f, __fsub_rn(yz, wx));
    R[2][0] = __fmul_rn(2.f, __fsub_rn(xz, wy));
    R[2][1] = __fmul_rn(2.f, __fadd_rn(yz, wx));
    R[2][2] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, yy)));
}

__global__ void __launch_bounds__(kThreads) pointcloud_kernel(PointCloudArgs a) {
    __shared__ float tile[kTile * 3];
    const int64_t pid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = pid < a.m;
    float t[3] = {0.f, 0.f, 0.f}, q[4] = {1.f, 0.f, 0.f, 0.f};
    if (active) {
#pragma unroll
        for (int i = 0; i < 3; ++i) t[i] = a.poses[pid * 7 + i];
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = a.poses[pid * 7 + 3 + i];
    }
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) finite &= isfinite(t[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) finite &= isfinite(q[i]);
    float R[3][3], n2q;
    quat_to_rot_exact(q, R, n2q);
    finite &= (n2q > 0.f) && isfinite(n2q);

    // sums: [0..5] u u^T / n^2, [6] 1/n^2, [7..9] u/n, [10..15] u u^T, [16] count
    constexpr int kN = 17;
    float hi[kN], lo[kN], acc[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) hi[i] = lo[i] = acc[i] = 0.f;

    const float rmin2 = a.rmin2, rmax2 = a.rmax2;
    for (int64_t base = 0; base < a.n; base += kTile) {
        const int cnt = (int)(a.n - base < kTile ? a.n - base : kTile);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt * 3; i += kThreads) tile[i] = __ldg(a.landmarks + base * 3 + i);
        __syncthreads();
        for (int b0 = 0; b0 < cnt; b0 += kBlock) {
            const int b1 = min(cnt, b0 + kBlock);
#pragma unroll 2
            for (int l = b0; l < b1; ++l) {
                const float px = tile[3 * l], py = tile[3 * l + 1], pz = tile[3 * l + 2];
                const float dx = __fsub_rn(px, t[0]), dy = __fsub_rn(py, t[1]), dz = __fsub_rn(pz, t[2]);
                const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                // p^c = R^T d
                const float cxv = __fadd_rn(__fadd_rn(__fmul_rn(R[0][0], dx), __fmul_rn(R[1][0], dy)), __fmul_rn(R[2][0], dz));
                const float cyv = __fadd_rn(__fadd_rn(__fmul_rn(R[0][1], dx), __fmul_rn(R[1][1], dy)), __fmul_rn(R[2][1], dz));
                const float czv = __fadd_rn(__fadd_rn(__fmul_rn(R[0][2], dx), __fmul_rn(R[1][2], dy)), __fmul_rn(R[2][2], dz));
                const float ux = __fadd_rn(__fmul_rn(a.fx, cxv), __fmul_rn(a.cx, czv));
                const float uy = __fadd_rn(__fmul_rn(a.fy, cyv), __fmul_rn(a.cy, czv));
                const float wz = __fmul_rn(a.W, czv), hz = __fmul_rn(a.H, czv);
                const bool vis = (n2 > rmin2) && (n2 <= rmax2) && (czv > 0.f) && (ux >= 0.f) && (ux < wz) &&
                                 (uy >= 0.f) && (uy < hz);
                const float r = rsqrtf(n2);
                const float inv_n = vis ? r : 0.f;
                const float x = cxv * inv_n, y = cyv * inv_n, z = czv * inv_n;
                const float w2 = inv_n * inv_n;
                const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
                acc[0] = fmaf(xx, w2, acc[0]);
                acc[1] = fmaf(xy, w2, acc[1]);
                acc[2] = fmaf(xz, w2, acc[2]);
                acc[3] = fmaf(yy, w2, acc[3]);
                acc[4] = fmaf(yz, w2, acc[4]);
                acc[5] = fmaf(zz, w2, acc[5]);
                acc[6] += w2;
                acc[7] = fmaf(x, inv_n, acc[7]);
                acc[8] = fmaf(y, inv_n, acc[8]);
                acc[9] = fmaf(z, inv_n, acc[9]);
                acc[10] += xx;
                acc[11] += xy;
                acc[12] += xz;
                acc[13] += yy;
                acc[14] += yz;
                acc[15] += zz;
                acc[16] += vis ? 1.f : 0.f;
            }
#pragma unroll
            for (int i = 0; i < kN; ++i) {
                const float y = acc[i] - lo[i];
                const float s = hi[i] + y;
                lo[i] = (s - hi[i]) - y;
                hi[i] = s;
                acc[i] = 0.f;
            }
        }
    }
    if (!active) return;
    float v[kN];
#pragma unroll
    for (int i = 0; i < kN; ++i) v[i] = (hi[i] - lo[i]) * a.inv_sigma2;
    // assemble the camera-frame FIM
    Blocks B;
    const float uu2[3][3] = {{v[0], v[1], v[2]}, {v[1], v[3], v[4]}, {v[2], v[4], v[5]}};
    const float uu0[3][3] = {{v[10], v[11], v[12]}, {v[11], v[13], v[14]}, {v[12], v[14], v[15]}};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            B.A[r][c] = (r == c ? v[6] : 0.f) - uu2[r][c];
            B.D[r][c] = (r == c ? v[16] : 0.f) - uu0[r][c];
        }
    // -[u]x / n summed: [[0, u3, -u2], [-u3, 0, u1], [u2, -u1, 0]] / n
    B.B[0][0] = 0.f;   B.B[0][1] = v[9];  B.B[0][2] = -v[8];
    B.B[1][0] = -v[9]; B.B[1][1] = 0.f;   B.B[1][2] = v[7];
    B.B[2][0] = v[8];  B.B[2][1] = -v[7]; B.B[2][2] = 0.f;
    if (a.flags & FIF_Q_WORLD) {
        // I_t = blkdiag(R, R) I_c blkdiag(R^T, R^T), then about the world origin: M_t^T I_t M_t
        float Rt[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Rt[r][c] = R[c][r];
        rotate_into(B, Rt);
        shift_ref(B, t);
    }
    float fim[21];
    pack(B, fim);
    uint32_t st = 0;
    if (!finite) {
        st |= FIF_POSE_NAN;
#pragma unroll
        for (int e = 0; e < 21; ++e) fim[e] = __int_as_float(0x7fc00000);
    }
    if (fabsf(n2q - 1.f) > 1e-3f) st |= FIF_POSE_QUAT;
    const bool nan = !finite;
    if (a.fim) {
#pragma unroll
        for (int e = 0; e < 21; ++e) a.fim[pid * 21 + e] = fim[e];
    }
    double* mo = a.metrics ? a.metrics + pid * 3 : nullptr;
    if (a.flags & FIF_Q_TRACE) {
        if (mo) mo[0] = nan ? (double)NAN : (double)trace6(fim);
    }
    if (a.flags & FIF_Q_LOGDET) {
        double lad;
        int sg;
        logdet_f64(fim, lad, sg);
        if (nan) { lad = NAN; sg = 0; }
        if (mo) mo[1] = lad;
        if (a.sign) a.sign[pid] = (int8_t)sg;
        if (sg <= 0 && !nan) st |= FIF_POSE_NOT_PD;
    }
    if (a.flags & FIF_Q_LMIN) {
        double lm = lambda_min_f64(fim);
        if (nan) lm = NAN;
        if (mo) mo[2] = lm;
        if (!(lm > 0.0) && !nan) st |= FIF_POSE_NOT_PD;
    }
    if (a.status) a.status[pid] = (int32_t)st;
}

}  // namespace

int launch_pointcloud(const PointCloudArgs& a, cudaStream_t stream) {
    const int64_t blocks = (a.m + kThreads - 1) / kThreads;
    if (blocks <= 0) return FIF_OK;
    if (blocks > (int64_t)INT32_MAX) return FIF_ERANGE;
    pointcloud_kernel<<<(unsigned)blocks, kThreads, 0, stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

}  // namespace fif
