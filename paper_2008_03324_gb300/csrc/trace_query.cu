// trace_query.cu -- query of the positional trace factor (sm_103a).
//
// Sec. VI-A-2 of the paper: with T-optimality as the metric, the field can store one N_v-vector
// per voxel, C_Tr = sum_i v_p,i Tr(I_i) (Eq. general_trace_pif), and the trace of a pose's FIM is
// v_r(R)^T C_Tr(t) (Eq. fim_trace_separation, general_trace_query) -- in the world frame, since
// the trace of the global-perturbation information is what the factor sums.
//
// One thread per pose: cell lookup as in the full query, 8 corners x 10 floats (three 16-B
// loads each; stride 12 floats = 48 B per node), trilinear blend, dot with v_r(z).
#include "fif_common.cuh"
#include "fif_internal.h"

namespace fif {

namespace {

__global__ void __launch_bounds__(256) trace_query_kernel(QueryArgs a) {
    const int64_t pid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pid >= a.m) return;
    const float* ps = a.poses + pid * 7;
    float t[3], qv[4];
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = __ldg(ps + i);
#pragma unroll
    for (int i = 0; i < 4; ++i) qv[i] = __ldg(ps + 3 + i);
    uint32_t st = 0;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) finite &= isfinite(t[i]);
#pragma unroll
    for (int i = 0; i < 4; ++i) finite &= isfinite(qv[i]);
    float R[3][3];
    const float n2 = quat_to_rot(qv[0], qv[1], qv[2], qv[3], R);
    finite &= (n2 > 0.f) && isfinite(n2);
    if (!finite) st |= FIF_POSE_NAN;
    if (fabsf(n2 - 1.f) > 1e-3f) st |= FIF_POSE_QUAT;
    const float org[3] = {a.ox, a.oy, a.oz};
    const int dims[3] = {a.nx, a.ny, a.nz};
    float w[3];
    int i0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float gg = __fdiv_rn(__fsub_rn(t[k], org[k]), a.res);
        if (finite) {
            if (gg < 0.f || gg > (float)(dims[k] - 1)) st |= FIF_POSE_OUTSIDE;
        } else {
            gg = 0.f;
        }
        if (a.flags & FIF_Q_NEAREST) {
            int ii = (int)floorf(__fadd_rn(gg, 0.5f));
            ii = max(0, min(ii, dims[k] - 1));
            const int b0 = min(ii, dims[k] - 2);
            i0[k] = b0;
            w[k] = (ii > b0) ? 1.f : 0.f;
        } else {
            int ii = (int)floorf(gg);
            ii = max(0, min(ii, dims[k] - 2));
            i0[k] = ii;
            w[k] = fminf(fmaxf(gg - (float)ii, 0.f), 1.f);
        }
    }
    const float z[3] = {R[0][2], R[1][2], R[2][2]};
    float vr[10];
    vis_vr(z, a.k0, a.k1, a.k2, vr);
    const int64_t nx = a.nx, nxy = (int64_t)a.nx * a.ny;
    const int64_t base = i0[0] + nx * i0[1] + nxy * i0[2];
    const float4* C = reinterpret_cast<const float4*>(a.coeffs);
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int bx = j & 1, by = (j >> 1) & 1, bz = (j >> 2) & 1;
        const float wj = (bx ? w[0] : 1.f - w[0]) * (by ? w[1] : 1.f - w[1]) * (bz ? w[2] : 1.f - w[2]);
        const int64_t node = base + bx + by * nx + bz * nxy;
        const float4* p = C + node * 3;
        const float4 c0 = __ldg(p), c1 = __ldg(p + 1), c2 = __ldg(p + 2);
        const float cv[12] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] = fmaf(wj, cv[k], acc[k]);
    }
    float tr = 0.f;
#pragma unroll
    for (int k = 0; k < 10; ++k) tr = fmaf(vr[k], acc[k], tr);
    if (a.metrics) a.metrics[pid * 3] = finite ? (double)tr : (double)NAN;
    if (a.status) a.status[pid] = (int32_t)st;
}

}  // namespace

int launch_trace_query(const QueryArgs& a, cudaStream_t stream) {
    const int64_t blocks = (a.m + 255) / 256;
    if (blocks <= 0) return FIF_OK;
    if (blocks > (int64_t)INT32_MAX) return FIF_ERANGE;
    trace_query_kernel<<<(unsigned)blocks, 256, 0, stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

}  // namespace fif
