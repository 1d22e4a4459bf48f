// query.cu -- constant-time pose query of the Fisher Information Field (sm_103a).
//
// Sec. VI-A-1 / Eq. fim_separation / Eq. general_info_query of the paper:
//   I(T) = V_I(R) C_I(t) = sum_k v_r(z)[k] C_k(t),  z = R e3,
// with C_k(t) interpolated over the 8 nodes around t (Sec. VII-A-1), rotated into the
// camera frame and reduced to trace / log|det| / lambda_min (Sec. IV).
//
// Design (one warp owns a group of 32 poses):
//  P  lane = pose: cell lookup, trilinear weights, v_r(z), status -> per-pose table (smem).
//  G  for each pose of the group the warp gathers the 8 corner coefficient sets
//     (4 x-adjacent node pairs, 4 bulk copies of 1728 B, triple-buffered through shared
//     memory, plus an L2 bulk prefetch a few poses ahead).  lane = (corner j, quarter q):
//     the lane contracts its corner over the 10 monomials for the entries e = q mod 4,
//     weights by w_j, and a 3-level shuffle butterfly over the corner bits turns the 8
//     corners into the superset sums sum_{j' >= m} w_j' S_j' that the exact change of the
//     rotational reference point needs (see finalize()).  No lane ever needs a whole
//     6x6, so there is no per-corner shift and no full reduction.
//  F  lane = pose: assemble T (about the base node), move it to the camera position,
//     rotate into the camera frame, write the FIM, then the metrics (FP32 trace, FP64 LU
//     log|det|, FP32 Jacobi + FP64 Rayleigh lambda_min).
#include "fif_common.cuh"
#include "fif_internal.h"
#include "gather.cuh"

namespace fif {

namespace {

using namespace gather;

struct PoseEntry {      // 64 B
    int32_t base_lo, base_hi;
    float w[3];
    float vr[10];
    uint32_t status;
};

// moment slot for entry e held by corner-lane j (-1 if that superset sum is not needed)
__device__ __forceinline__ int mom_slot(int e, int j) {
    // TT block entries: superset sums m in {0..6} (all but xyz)
    switch (e) {
        case 0: return j <= 6 ? j * 6 + 0 : -1;
        case 1: return j <= 6 ? j * 6 + 1 : -1;
        case 2: return j <= 6 ? j * 6 + 2 : -1;
        case 6: return j <= 6 ? j * 6 + 3 : -1;
        case 7: return j <= 6 ? j * 6 + 4 : -1;
        case 11: return j <= 6 ? j * 6 + 5 : -1;
        default: break;
    }
    int ms = (j == 0) ? 0 : (j == 1) ? 1 : (j == 2) ? 2 : (j == 4) ? 3 : -1;
    switch (e) {  // TR block: superset sums m in {0, x, y, z}
        case 3: return ms >= 0 ? 42 + ms * 9 + 0 : -1;
        case 4: return ms >= 0 ? 42 + ms * 9 + 1 : -1;
        case 5: return ms >= 0 ? 42 + ms * 9 + 2 : -1;
        case 8: return ms >= 0 ? 42 + ms * 9 + 3 : -1;
        case 9: return ms >= 0 ? 42 + ms * 9 + 4 : -1;
        case 10: return ms >= 0 ? 42 + ms * 9 + 5 : -1;
        case 12: return ms >= 0 ? 42 + ms * 9 + 6 : -1;
        case 13: return ms >= 0 ? 42 + ms * 9 + 7 : -1;
        case 14: return ms >= 0 ? 42 + ms * 9 + 8 : -1;
        default: break;
    }
    if (e >= 15 && e <= 20) return j == 0 ? 78 + (e - 15) : -1;  // RR block: total only
    return -1;
}

// Assemble T = sum_j w_j M_dj^T S_j M_dj (reference point: the base node c0) from the
// superset sums.  With X_j = -[d_j]x = -res sum_a b_a(j) K_a:
//   T_TT = A^0
//   T_TR = B^0 - res sum_a A^a K_a
//   T_RR = D^0 - res sum_a (K_a^T B^a + B^a^T K_a) + res^2 sum_{a,c} K_a^T A^{ac} K_c
// (A^{aa} = A^a since b_a^2 = b_a).
__device__ __forceinline__ void assemble_T(const float* mom, float res, Blocks& T) {
    // A^m packed as (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
    auto Am = [&](int m, int r, int c) { return mom[m * 6 + sym3_idx(r, c)]; };
    auto Bm = [&](int ms, int r, int c) { return mom[42 + ms * 9 + r * 3 + c]; };
    auto Dm = [&](int r, int c) { return mom[78 + sym3_idx(r, c)]; };
    const int jsingle[3] = {1, 2, 4};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T.A[r][c] = Am(0, r, c);
            // TR
            float v = Bm(0, r, c);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float acc = 0.f;
#pragma unroll
                for (int l = 0; l < 3; ++l) acc += Am(jsingle[a], r, l) * kx(a, l, c);
                v -= res * acc;
            }
            T.B[r][c] = v;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = Dm(r, c);
            float lin = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int ms = a + 1;  // B superset slot of the single bit a
#pragma unroll
                for (int l = 0; l < 3; ++l) lin += kx(a, l, r) * Bm(ms, l, c) + Bm(ms, l, r) * kx(a, l, c);
            }
            float quad = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int m = jsingle[a] | jsingle[b];
#pragma unroll
                    for (int l = 0; l < 3; ++l)
#pragma unroll
                        for (int n = 0; n < 3; ++n) quad += kx(a, l, r) * Am(m, l, n) * kx(b, n, c);
                }
            T.D[r][c] = v - res * lin + res * res * quad;
        }
}

template <int kElem>
constexpr int warp_bytes() {
    return ((kStages * Layout<kElem>::kPoseBytes + 32 * (int)sizeof(PoseEntry) + 32 * kMomStride * 4 + 64 + 127) / 128) * 128;
}

template <int kElem>
__global__ void __launch_bounds__(kWarps * 32) query_kernel(QueryArgs args) {
    using L = Layout<kElem>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // per-warp shared memory (each warp's region starts on a 128-B boundary)
    constexpr int kWarpBytes = warp_bytes<kElem>();
    unsigned char* wbase = smem_raw + warp * kWarpBytes;
    unsigned char* stage = wbase;
    PoseEntry* ptab = reinterpret_cast<PoseEntry*>(wbase + kStages * L::kPoseBytes);
    float* mom = reinterpret_cast<float*>(wbase + kStages * L::kPoseBytes + 32 * sizeof(PoseEntry));
    uint64_t* bars = reinterpret_cast<uint64_t*>(wbase + kStages * L::kPoseBytes + 32 * sizeof(PoseEntry) +
                                                 32 * kMomStride * 4);

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 4);
        fence_mbar_init();
    }
    __syncwarp();

    const int j = lane >> 2;  // corner: bits (x, y, z)
    const int q = lane & 3;   // entry quarter
    const int bx = j & 1, by = (j >> 1) & 1, bz = (j >> 2) & 1;
    const int P = j >> 1;     // node pair holding this corner
    int slot[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int e = q + 4 * i;
        slot[i] = (e < 21) ? mom_slot(e, j) : -1;
    }
    const int corner_off = L::slot(P) + bx * L::kNodeBytes;  // byte offset of my corner in a stage

    const int64_t nx = args.nx, nxy = (int64_t)args.nx * args.ny;
    const char* coeffs = reinterpret_cast<const char*>(args.coeffs);
    uint32_t phase_bits = 0;     // parity of the next wait, per stage
    bool ok = true;

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
        float t[3] = {0.f, 0.f, 0.f}, qv[4] = {1.f, 0.f, 0.f, 0.f};
        int i0[3] = {0, 0, 0};
        uint32_t st = 0;
        if (lane < cnt) {
            const float* ps = args.poses + (p0 + lane) * 7;
#pragma unroll
            for (int a = 0; a < 3; ++a) t[a] = __ldg(ps + a);
#pragma unroll
            for (int a = 0; a < 4; ++a) qv[a] = __ldg(ps + 3 + a);
            bool finite = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) finite &= isfinite(t[a]);
#pragma unroll
            for (int a = 0; a < 4; ++a) finite &= isfinite(qv[a]);
            float R[3][3];
            const float n2 = quat_to_rot(qv[0], qv[1], qv[2], qv[3], R);
            finite &= (n2 > 0.f) && isfinite(n2);
            if (!finite) st |= FIF_POSE_NAN;
            if (fabsf(n2 - 1.f) > 1e-3f) st |= FIF_POSE_QUAT;
            float w[3];
            const float org[3] = {args.ox, args.oy, args.oz};
            const int dims[3] = {args.nx, args.ny, args.nz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float gg = __fdiv_rn(__fsub_rn(t[a], org[a]), args.res);
                if (!(st & FIF_POSE_NAN)) {
                    if (gg < 0.f || gg > (float)(dims[a] - 1)) st |= FIF_POSE_OUTSIDE;
                } else {
                    gg = 0.f;
                }
                if (args.flags & FIF_Q_NEAREST) {
                    int ii = (int)floorf(__fadd_rn(gg, 0.5f));
                    ii = max(0, min(ii, dims[a] - 1));
                    const int b0 = min(ii, dims[a] - 2);
                    i0[a] = b0;
                    w[a] = (ii > b0) ? 1.f : 0.f;
                } else {
                    int ii = (int)floorf(gg);
                    ii = max(0, min(ii, dims[a] - 2));
                    i0[a] = ii;
                    w[a] = fminf(fmaxf(gg - (float)ii, 0.f), 1.f);
                }
            }
            const float z[3] = {R[0][2], R[1][2], R[2][2]};
            float vr[10];
            vis_vr(z, args.k0, args.k1, args.k2, vr);
            if (st & FIF_POSE_NAN) {
#pragma unroll
                for (int k = 0; k < 10; ++k) vr[k] = 0.f;
            }
            const int64_t base = i0[0] + nx * i0[1] + nxy * i0[2];
            PoseEntry& pe = ptab[lane];
            pe.base_lo = (int32_t)(base & 0xffffffff);
            pe.base_hi = (int32_t)(base >> 32);
            pe.w[0] = w[0]; pe.w[1] = w[1]; pe.w[2] = w[2];
#pragma unroll
            for (int k = 0; k < 10; ++k) pe.vr[k] = vr[k];
            pe.status = st;
        }
        __syncwarp();
        auto base_of = [&](int i) -> int64_t {
            return (int64_t)(uint32_t)ptab[i].base_lo | ((int64_t)ptab[i].base_hi << 32);
        };
        // prologue: L2 prefetch of the first poses, bulk copies of the first stages
        if (lane < 4) {
            for (int i = 0; i < min(cnt, kPrefetch + kStages - 1); ++i)
                bulk_prefetch_l2(pair_src(base_of(i), lane), L::kPairBytes);
            fence_proxy_async();
            for (int i = 0; i < min(cnt, kStages - 1); ++i) {
                uint64_t* bar = &bars[i % kStages];
                unsigned char* dst = stage + (i % kStages) * L::kPoseBytes + L::slot(lane);
                mbar_arrive_expect_tx(bar, L::kPairBytes);
                bulk_g2s(dst, pair_src(base_of(i), lane), L::kPairBytes, bar);
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
                    uint64_t* bar = &bars[sn];
                    mbar_arrive_expect_tx(bar, L::kPairBytes);
                    bulk_g2s(stage + sn * L::kPoseBytes + L::slot(lane), pair_src(base_of(inext), lane),
                             L::kPairBytes, bar);
                }
                const int ipf = i + kStages - 1 + kPrefetch;
                if (ipf < cnt) bulk_prefetch_l2(pair_src(base_of(ipf), lane), L::kPairBytes);
            }
            const uint32_t par = (phase_bits >> s) & 1u;
            if (!mbar_wait_bounded(&bars[s], par)) {
                ok = false;
                set_error(args.err, FIF_ETIMEOUT);
            }
            phase_bits ^= (1u << s);
            // corner weight and weighted v_r
            const PoseEntry& pe = ptab[i];
            const float wj = (bx ? pe.w[0] : 1.f - pe.w[0]) * (by ? pe.w[1] : 1.f - pe.w[1]) *
                             (bz ? pe.w[2] : 1.f - pe.w[2]);
            float vrj[10];
#pragma unroll
            for (int k = 0; k < 10; ++k) vrj[k] = wj * pe.vr[k];
            const float* C = reinterpret_cast<const float*>(stage + s * L::kPoseBytes + corner_off) + q;
            float v[6];
#pragma unroll
            for (int ii = 0; ii < 6; ++ii) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 10; ++k) acc = fmaf(vrj[k], C[k * 21 + 4 * ii], acc);
                v[ii] = acc;
            }
            // superset-sum butterfly over the corner bits x (lane bit 2), y (3), z (4)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int mask = 4 << a;
                const bool low = ((j >> a) & 1) == 0;
#pragma unroll
                for (int ii = 0; ii < 6; ++ii) {
                    const float o = __shfl_xor_sync(0xffffffffu, v[ii], mask);
                    v[ii] = low ? v[ii] + o : v[ii];
                }
            }
            float* mrow = mom + i * kMomStride;
#pragma unroll
            for (int ii = 0; ii < 6; ++ii)
                if (slot[ii] >= 0) mrow[slot[ii]] = v[ii];
            __syncwarp();
        }
        // ---------------- phase F: lane = pose ----------------
        if (lane < cnt) {
            const PoseEntry& pe = ptab[lane];
            st = pe.status;
            Blocks T;
            assemble_T(mom + lane * kMomStride, args.res, T);
            const float c0[3] = {__fadd_rn(args.ox, __fmul_rn(args.res, (float)i0[0])),
                                 __fadd_rn(args.oy, __fmul_rn(args.res, (float)i0[1])),
                                 __fadd_rn(args.oz, __fmul_rn(args.res, (float)i0[2]))};
            float fim[21];
            if (args.flags & FIF_Q_WORLD) {
                shift_ref(T, c0);
            } else {
                float R[3][3];
                quat_to_rot(qv[0], qv[1], qv[2], qv[3], R);
                // the coefficients were taken at the clamped cell; the FIM is expressed about t
                const float b[3] = {c0[0] - t[0], c0[1] - t[1], c0[2] - t[2]};
                shift_ref(T, b);
                rotate_into(T, R);
            }
            pack(T, fim);
            const bool nan = (st & FIF_POSE_NAN) != 0;
            if (nan) {
#pragma unroll
                for (int e = 0; e < 21; ++e) fim[e] = __int_as_float(0x7fc00000);
            }
            const int64_t pid = p0 + lane;
            if (args.fim) {
                float* out = args.fim + pid * 21;
#pragma unroll
                for (int e = 0; e < 21; ++e) out[e] = fim[e];
            }
            if (args.flags & FIF_Q_METRICS) {
                double* mo = args.metrics ? args.metrics + pid * 3 : nullptr;
                if (args.flags & FIF_Q_TRACE) {
                    if (mo) mo[0] = nan ? (double)NAN : (double)trace6(fim);
                }
                if (args.flags & FIF_Q_LOGDET) {
                    double lad;
                    int sg;
                    logdet_f64(fim, lad, sg);
                    if (nan) { lad = NAN; sg = 0; }
                    if (mo) mo[1] = lad;
                    if (args.sign) args.sign[pid] = (int8_t)sg;
                    if (sg <= 0 && !nan) st |= FIF_POSE_NOT_PD;
                }
                if (args.flags & FIF_Q_LMIN) {
                    double lm = lambda_min_f64(fim);
                    if (nan) lm = NAN;
                    if (mo) mo[2] = lm;
                    if (!(lm > 0.0) && !nan) st |= FIF_POSE_NOT_PD;
                }
            }
            if (args.status) args.status[pid] = (int32_t)st;
        }
        __syncwarp();
    }
    (void)ok;
}

}  // namespace

int launch_query(const QueryArgs& a, cudaStream_t stream) {
    const int smem = kWarps * warp_bytes<4>();
    if (cudaFuncSetAttribute(query_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return FIF_ECUDA;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, query_kernel<4>, kWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t groups = (a.m + 31) / 32;
    const int64_t need = (groups + kWarps - 1) / kWarps;
    const int64_t grid = std::min<int64_t>(need, (int64_t)sms * per_sm);
    if (grid <= 0) return FIF_OK;
    query_kernel<4><<<(unsigned)grid, kWarps * 32, smem, stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

}  // namespace fif
