// adjoint.cu -- hand-written adjoint of the pose query (sm_103a).
//
// For a metric m(I) of the queried FIM (trace, log|det|, lambda_min; Sec. IV) this computes
// dm/dt (world position) and dm/dphi (right so(3) perturbation R <- R exp(phi^)) of
//   I_c = B^T M_b^T T M_b B,   T = sum_j w_j(t) M_dj^T S_j(z) M_dj,   S_j = sum_k v_r(z)[k] C_jk,
// with B = blkdiag(R, R), b = c0 - t, d_j the lattice offset of corner j from the base node c0
// and z = R e3 (Eq. fim_separation, Eq. general_info_query).
//
//   G   = dm/dI_c  (trace: I; log|det|: I_c^-1; lambda_min: x x^T)
//   G_t = B G B^T,  G' = M_b G_t M_b^T,  G_j = M_dj G' M_dj^T
//   dm/dt_a   = sum_j dw_j/dt_a <G_j, S_j> + 2 <G_t, I_t E_a>,   E_a = [[0, [e_a]x], [0, 0]]
//   dm/dz_a   = sum_j w_j <G_j, dS_j/dz_a>
//   dm/dphi   = e3 x (R^T dm/dz)      (dz/dphi = -R [e3]x; the optical-axis component is 0)
// The metrics are invariant under the orthogonal B, so R enters only through z.  In the
// world frame (about the origin) I_w = M_c0^T T M_c0 and only the weights and z depend on
// the pose.
//
// Structure mirrors the query: a warp owns 32 poses; lane = pose computes G, G' and the
// per-pose tables (P); then per pose the warp gathers the 8 corners through shared memory
// and lane (j, q) forms the 10 partial products <G_j, C_jk> over its entries, weights them
// with v_r, dv_r/dz, w_j and dw_j/dt, and a warp reduction gives 6 numbers (G); lane = pose
// assembles the gradient (F).
#include "fif_common.cuh"
#include "fif_internal.h"
#include "gather.cuh"

namespace fif {

namespace {

using namespace gather;

struct AdjEntry {  // 320 B
    int32_t base_lo, base_hi;
    float w[3];
    float dw[3];     // d w_a / d t_a (1/res inside the lattice along that axis, else 0)
    float vr[10];
    float dvr[3][10];
    float G[21];     // G' (about the base node)
    float pad[10];
};

template <int kElem>
constexpr int adj_warp_bytes() {
    return ((kStages * Layout<kElem>::kPoseBytes + 32 * (int)sizeof(AdjEntry) + 32 * 8 * 4 + 64 + 127) / 128) * 128;
}

template <int kElem>
__global__ void __launch_bounds__(kWarps * 32) adjoint_kernel(AdjointArgs args) {
    using L = Layout<kElem>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    constexpr int kWarpBytes = adj_warp_bytes<kElem>();
    unsigned char* wbase = smem_raw + warp * kWarpBytes;
    unsigned char* stage = wbase;
    AdjEntry* ptab = reinterpret_cast<AdjEntry*>(wbase + kStages * L::kPoseBytes);
    float* gsum = reinterpret_cast<float*>(wbase + kStages * L::kPoseBytes + 32 * sizeof(AdjEntry));  // [32][8]
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + kStages * L::kPoseBytes + 32 * sizeof(AdjEntry) + 32 * 8 * 4);

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 4);
        fence_mbar_init();
    }
    __syncwarp();

    const int j = lane >> 2, q = lane & 3;
    const int bx = j & 1, by = (j >> 1) & 1, bz = (j >> 2) & 1;
    const int P = j >> 1;
    const int corner_off = L::slot(P) + bx * L::kNodeBytes;
    const bool world = (args.flags & FIF_Q_WORLD) != 0;

    const int64_t nx = args.nx, nxy = (int64_t)args.nx * args.ny;
    const char* coeffs = reinterpret_cast<const char*>(args.coeffs);
    uint32_t phase_bits = 0;

    const int64_t groups = (args.m + 31) / 32;
    const int64_t gwarp = (int64_t)blockIdx.x * kWarps + warp;
    const int64_t nwarps = (int64_t)gridDim.x * kWarps;

    auto pair_src = [&](int64_t base, int pp) -> const void* {
        const int64_t node = base + (pp & 1) * nx + (pp >> 1) * nxy;
        return coeffs + node * (int64_t)L::kNodeBytes;
    };

    for (int64_t g = gwarp; g < groups; g += nwarps) {
        const int64_t p0 = g * 32;
        const int cnt = (int)(int)(args.m - p0 < 32 ? args.m - p0 : 32);
        // ---------------- phase P: lane = pose ----------------
        float t[3] = {0.f, 0.f, 0.f};
        float R[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
        float Mterm[3] = {0.f, 0.f, 0.f};
        bool nan = false;
        if (lane < cnt) {
            const int64_t pid = p0 + lane;
            const float* ps = args.poses + pid * 7;
            float qv[4];
#pragma unroll
            for (int a = 0; a < 3; ++a) t[a] = __ldg(ps + a);
#pragma unroll
            for (int a = 0; a < 4; ++a) qv[a] = __ldg(ps + 3 + a);
            bool finite = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) finite &= isfinite(t[a]);
#pragma unroll
            for (int a = 0; a < 4; ++a) finite &= isfinite(qv[a]);
            const float n2 = quat_to_rot(qv[0], qv[1], qv[2], qv[3], R);
            finite &= (n2 > 0.f) && isfinite(n2);
            nan = !finite;
            const float org[3] = {args.ox, args.oy, args.oz};
            const int dims[3] = {args.nx, args.ny, args.nz};
            int i0[3];
            float w[3], dw[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float gg = __fdiv_rn(__fsub_rn(t[a], org[a]), args.res);
                if (nan) gg = 0.f;
                int ii = (int)floorf(gg);
                ii = max(0, min(ii, dims[a] - 2));
                i0[a] = ii;
                const float fr = gg - (float)ii;
                w[a] = fminf(fmaxf(fr, 0.f), 1.f);
                dw[a] = (fr >= 0.f && fr <= 1.f) ? 1.f / args.res : 0.f;
            }
            const float z[3] = {R[0][2], R[1][2], R[2][2]};
            AdjEntry& pe = ptab[lane];
            const int64_t base = i0[0] + nx * i0[1] + nxy * i0[2];
            pe.base_lo = (int32_t)(base & 0xffffffff);
            pe.base_hi = (int32_t)(base >> 32);
#pragma unroll
            for (int a = 0; a < 3; ++a) { pe.w[a] = w[a]; pe.dw[a] = dw[a]; }
            float vr[10];
            vis_vr(z, args.k0, args.k1, args.k2, vr);
#pragma unroll
            for (int k = 0; k < 10; ++k) pe.vr[k] = vr[k];
            {
                const float k1 = args.k1, k2 = args.k2;
                const float d0[10] = {2 * k2 * z[0], 0, 0, 2 * k2 * z[1], 2 * k2 * z[2], 0, k1, 0, 0, 0};
                const float d1[10] = {0, 2 * k2 * z[1], 0, 2 * k2 * z[0], 0, 2 * k2 * z[2], 0, k1, 0, 0};
                const float d2[10] = {0, 0, 2 * k2 * z[2], 0, 2 * k2 * z[0], 2 * k2 * z[1], 0, 0, k1, 0};
#pragma unroll
                for (int k = 0; k < 10; ++k) { pe.dvr[0][k] = d0[k]; pe.dvr[1][k] = d1[k]; pe.dvr[2][k] = d2[k]; }
            }
            // G = dm/dI in the output frame
            float I[21];
#pragma unroll
            for (int e = 0; e < 21; ++e) I[e] = args.fim[pid * 21 + e];
            const double gtr = args.gm[pid * 3 + 0], gld = args.gm[pid * 3 + 1], glm = args.gm[pid * 3 + 2];
            float G[21];
#pragma unroll
            for (int e = 0; e < 21; ++e) G[e] = (sym_row(e) == sym_col(e)) ? (float)gtr : 0.f;
            if (gld != 0.0) {
                double inv[21];
                inverse6_f64(I, inv);
#pragma unroll
                for (int e = 0; e < 21; ++e) G[e] += (float)(gld * inv[e]);
            }
            if (glm != 0.0) {
                float x[6];
                lambda_min_f64(I, x);
#pragma unroll
                for (int e = 0; e < 21; ++e) G[e] += (float)glm * x[sym_row(e)] * x[sym_col(e)];
            }
            Blocks Gb;
            unpack(G, Gb);
            const float c0[3] = {__fadd_rn(args.ox, __fmul_rn(args.res, (float)i0[0])),
                                 __fadd_rn(args.oy, __fmul_rn(args.res, (float)i0[1])),
                                 __fadd_rn(args.oz, __fmul_rn(args.res, (float)i0[2]))};
            if (world) {
                shift_dual(Gb, c0);  // G' = M_c0 G_w M_c0^T
            } else {
                // G_t = B G B^T and I_t = B I_c B^T (rotate_into with R^T computes R S R^T)
                float Rt[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) Rt[r][c] = R[c][r];
                rotate_into(Gb, Rt);
                Blocks It;
                unpack(I, It);
                rotate_into(It, Rt);
                // 2 <G_t, I_t E_a>: (I_t E_a)[i][3 + c] = sum_l I_t[i][l] [e_a]x[l][c]
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float acc = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
#pragma unroll
                        for (int l = 0; l < 3; ++l) {
                            const float ke = kx(a, l, c);
                            // rows 0..2: G_t[r][3+c] = Gb.B[r][c]; I_t[r][l] = It.A[r][l]
                            // rows 3..5: G_t[3+r][3+c] = Gb.D[r][c]; I_t[3+r][l] = It.B[l][r]
#pragma unroll
                            for (int r = 0; r < 3; ++r) acc += ke * (Gb.B[r][c] * It.A[r][l] + Gb.D[r][c] * It.B[l][r]);
                        }
                    Mterm[a] = 2.f * acc;
                }
                const float b[3] = {c0[0] - t[0], c0[1] - t[1], c0[2] - t[2]};
                shift_dual(Gb, b);  // G' = M_b G_t M_b^T
            }
            float Gp[21];
            pack(Gb, Gp);
#pragma unroll
            for (int e = 0; e < 21; ++e) pe.G[e] = nan ? 0.f : Gp[e];
        }
        __syncwarp();
        auto base_of = [&](int i) -> int64_t {
            return (int64_t)(uint32_t)ptab[i].base_lo | ((int64_t)ptab[i].base_hi << 32);
        };
        if (lane < 4) {
            for (int i = 0; i < min(cnt, kPrefetch + kStages - 1); ++i)
                bulk_prefetch_l2(pair_src(base_of(i), lane), L::kPairBytes);
            fence_proxy_async();
            for (int i = 0; i < min(cnt, kStages - 1); ++i) {
                uint64_t* bar = &bars[i % kStages];
                mbar_arrive_expect_tx(bar, L::kPairBytes);
                bulk_g2s(stage + (i % kStages) * L::kPoseBytes + L::slot(lane), pair_src(base_of(i), lane),
                         L::kPairBytes, bar);
            }
        }
        // ---------------- phase G: warp per pose ----------------
        for (int i = 0; i < cnt; ++i) {
            const int s = i % kStages;
            if (lane < 4) {
                const int inext = i + kStages - 1;
                if (inext < cnt) {
                    const int sn = inext % kStages;
                    fence_proxy_async();
                    mbar_arrive_expect_tx(&bars[sn], L::kPairBytes);
                    bulk_g2s(stage + sn * L::kPoseBytes + L::slot(lane), pair_src(base_of(inext), lane),
                             L::kPairBytes, &bars[sn]);
                }
                const int ipf = i + kStages - 1 + kPrefetch;
                if (ipf < cnt) bulk_prefetch_l2(pair_src(base_of(ipf), lane), L::kPairBytes);
            }
            const uint32_t par = (phase_bits >> s) & 1u;
            if (!mbar_wait_bounded(&bars[s], par)) set_error(args.err, FIF_ETIMEOUT);
            phase_bits ^= (1u << s);
            const AdjEntry& pe = ptab[i];
            // G_j = M_dj G' M_dj^T for my corner
            Blocks Gj;
            unpack(pe.G, Gj);
            const float d[3] = {bx * args.res, by * args.res, bz * args.res};
            shift_dual(Gj, d);
            float Gp[21];
            pack(Gj, Gp);
            const float* C = reinterpret_cast<const float*>(stage + s * L::kPoseBytes + corner_off);
            // my entries e = q + 4 ii, weighted 2 off the diagonal (symmetric inner product);
            // picked with selects so Gp stays in registers
            float gsel[6];
#pragma unroll
            for (int ii = 0; ii < 6; ++ii) {
                float v = 0.f;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    const int e = qq + 4 * ii;
                    if (e < 21) {
                        const float mult = (sym_row(e) == sym_col(e)) ? 1.f : 2.f;
                        v = (q == qq) ? mult * Gp[e] : v;
                    }
                }
                gsel[ii] = v;
            }
            const float* Cq = C + q;
            float r1 = 0.f, r2[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                float qk = 0.f;
#pragma unroll
                for (int ii = 0; ii < 6; ++ii) qk = fmaf(gsel[ii], Cq[k * 21 + 4 * ii], qk);
                r1 = fmaf(pe.vr[k], qk, r1);
#pragma unroll
                for (int a = 0; a < 3; ++a) r2[a] = fmaf(pe.dvr[a][k], qk, r2[a]);
            }
            const float wx = bx ? pe.w[0] : 1.f - pe.w[0];
            const float wy = by ? pe.w[1] : 1.f - pe.w[1];
            const float wz = bz ? pe.w[2] : 1.f - pe.w[2];
            const float wj = wx * wy * wz;
            const float dwx = (bx ? pe.dw[0] : -pe.dw[0]) * wy * wz;
            const float dwy = wx * (by ? pe.dw[1] : -pe.dw[1]) * wz;
            const float dwz = wx * wy * (bz ? pe.dw[2] : -pe.dw[2]);
            float out[6] = {dwx * r1, dwy * r1, dwz * r1, wj * r2[0], wj * r2[1], wj * r2[2]};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int c = 0; c < 6; ++c) out[c] += __shfl_xor_sync(0xffffffffu, out[c], o);
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < 6; ++c) gsum[i * 8 + c] = out[c];
            }
            __syncwarp();
        }
        // ---------------- phase F: lane = pose ----------------
        if (lane < cnt) {
            const int64_t pid = p0 + lane;
            float gt[3], gz[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gt[a] = gsum[lane * 8 + a] + Mterm[a];
                gz[a] = gsum[lane * 8 + 3 + a];
            }
            // w = R^T g_z ; dm/dphi = e3 x w = (-w_y, w_x, 0)
            const float wv0 = R[0][0] * gz[0] + R[1][0] * gz[1] + R[2][0] * gz[2];
            const float wv1 = R[0][1] * gz[0] + R[1][1] * gz[1] + R[2][1] * gz[2];
            float* go = args.grad + pid * 6;
            const float qnan = __int_as_float(0x7fc00000);
            go[0] = nan ? qnan : gt[0];
            go[1] = nan ? qnan : gt[1];
            go[2] = nan ? qnan : gt[2];
            go[3] = nan ? qnan : -wv1;
            go[4] = nan ? qnan : wv0;
            go[5] = nan ? qnan : 0.f;
        }
        __syncwarp();
    }
}

}  // namespace

int launch_adjoint(const AdjointArgs& a, cudaStream_t stream) {
    const int smem = kWarps * adj_warp_bytes<4>();
    if (cudaFuncSetAttribute(adjoint_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return FIF_ECUDA;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_kernel<4>, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t groups = (a.m + 31) / 32;
    const int64_t need = (groups + kWarps - 1) / kWarps;
    const int64_t grid = std::min<int64_t>(need, (int64_t)sms * per_sm);
    if (grid <= 0) return FIF_OK;
    adjoint_kernel<4><<<(unsigned)grid, kWarps * 32, smem, stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

}  // namespace fif
