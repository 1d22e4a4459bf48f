// query.cu -- constant-time pose query of the Fisher Information Field (sm_103a).
//
// Sec. VI-A-1 / Eq. fim_separation / Eq. general_info_query of the paper:
//   I(T) = V_I(R) C_I(t) = sum_k v_r(z)[k] C_k(t),  z = R e3,
// with C_k(t) interpolated over the 8 nodes around t (Sec. VII-A-1), rotated into the
// camera frame and reduced to trace / log|det| / lambda_min (Sec. IV).
//
// Design (one warp owns a group of 32 poses):
//  P  lane = pose: cell lookup, trilinear weights, v_r(z), status -> per-pose table (smem,
//     columns by pose so that the 32 lanes write distinct banks): the base node's address,
//     the 8 corner weights w_j and v_r(z) duplicated for the packed FMAs.
//  G  for each pose of the group the warp gathers the 8 corner coefficient sets
//     (4 x-adjacent node pairs, 4 bulk copies of 1728 B (896 B for bfloat16), double-
//     buffered through shared memory, plus an L2 bulk prefetch of the pose after the next;
//     float32: 8 gather and 4 metric warps per SM, bfloat16: 10 and 5, so that enough copies
//     are in flight).  lane = (corner j, quarter q):
//     the lane contracts its corner over the 10 monomials for the entries e = q mod 4
//     (bfloat16 storage: the entry pairs 2p, 2p + 1 with p = q mod 4, one 32-bit word per
//     pair and monomial, contracted with packed f32x2 FMAs),
//     weights by w_j, and a 3-level shuffle butterfly over the corner bits turns the 8
//     corners into the superset sums sum_{j' >= m} w_j' S_j' that the exact change of the
//     rotational reference point needs (see finalize()).  No lane ever needs a whole
//     6x6, so there is no per-corner shift and no full reduction.
//  F  lane = pose: assemble T (about the base node), move it to the camera position,
//     rotate into the camera frame, write the FIM, then the metrics (FP32 trace, FP64 LU
//     log|det|, lambda_min from a Sturm-bisection shift, inverse iteration and the FP64
//     Rayleigh quotient).
#include "fif_common.cuh"
#include "fif_internal.h"
#include "gather.cuh"

namespace fif {

namespace {

using namespace gather;

// per-pose table of a group of 32 poses, written by lane = pose (conflict-free rows) and read
// by the whole warp for one pose at a time
struct PoseTable {
    const char* src[32];     // the base node's record
    float2 vr2[10][32];      // v_r(z)[k] twice (the operand of a packed FMA)
    float wj[32][9];         // trilinear weight of corner j (bits x, y, z of j); odd row stride
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

// ---- warp-specialised kernel ----------------------------------------------------------
// kGather gather warps stream corners and assemble T; kMetric metric warps finish poses.
// Metric warp m serves gather warps m, m + kMetric, ... (kGather / kMetric of them; two
// slots each, double-buffered).  Every bounded wait that runs out sets a shared abort flag
// that all warps of the CTA see, so the CTA leaves as a whole (after draining its copies).
constexpr int kGather = 8;     // gather warps per CTA of the float32 configuration
constexpr int kMetric = 4;     // metric warps per CTA of the float32 configuration
constexpr int kRow = 33;              // floats per pose in a slot (odd stride: no bank conflicts)
// slot row: [0..20] T (about the base node, world axes), [21..23] t, [24..27] q,
//           [28..30] c0, [31] status bits
constexpr int kSlotFloats = 32 * kRow;

template <int kElem, int NS>
struct GatherSmem {
    unsigned char stage[NS][Layout<kElem>::kPoseBytes];
    PoseTable pt;
    float mom[kMomStride];
    float slot[2][kSlotFloats];
    uint64_t bars[NS];
    uint64_t full[2];
    uint64_t empty[2];
};

template <int kElem, int NS>
constexpr int gather_smem_bytes() {
    return (int)((sizeof(GatherSmem<kElem, NS>) + 127) / 128 * 128);
}

// Entry e of T as a linear combination of the 84 superset sums,
//   T[e] = sum_{u < 9} coef_u(res) * mom[idx_u]   (unused terms have coef 0),
// following the algebra of the reference-point change:
//   T_TT = A^0,  T_TR = B^0 - res sum_a A^a K_a,
//   T_RR = D^0 - res (L + L^T) + res^2 Q,  L = sum_a K_a^T B^a,  Q = sum_ab K_a^T A^{ab} K_b,
// K_a = [e_a]x, A^{ab} the superset sum of corners with bits a and b set (A^{aa} = A^a).
// The nonzero terms of entry e (at most 9) in a fixed enumeration order: term u adds
// sgn_u * res^pw_u * mom[idx_u].  Which terms are nonzero does not depend on res (> 0), so the
// shape is enumerated once on the host and each launch passes the table with res applied
// (computed on the device per lane, the enumeration's cold code cost ~15-100 us per launch).
struct TermShape {
    int16_t idx[21][9];
    int8_t sgn[21][9];
    int8_t pw[21][9];
};

struct TermTable {
    float coef[21][9];
    int16_t idx[21][9];
};

TermShape make_term_shape() {
    TermShape S{};
    for (int e = 0; e < 21; ++e) {
        int n = 0;
        auto add = [&](int idx, float sgn, int pw) {
            if (sgn == 0.f) return;
            if (n < 9) {
                S.idx[e][n] = (int16_t)idx;
                S.sgn[e][n] = (int8_t)(sgn > 0.f ? 1 : -1);
                S.pw[e][n] = (int8_t)pw;
            }
            ++n;
        };
        auto A = [](int m, int r, int c) { return m * 6 + sym3_idx(r, c); };
        auto B = [](int ms, int r, int c) { return 42 + ms * 9 + r * 3 + c; };
        auto D = [](int r, int c) { return 78 + sym3_idx(r, c); };
        const int R = sym_row(e), C = sym_col(e);
        if (R < 3 && C < 3) {
            add(A(0, R, C), 1.f, 0);
        } else if (R < 3) {
            const int r = R, c = C - 3;
            add(B(0, r, c), 1.f, 0);
            for (int a = 0; a < 3; ++a)
                for (int l = 0; l < 3; ++l) add(A(1 << a, r, l), -kx(a, l, c), 1);
        } else {
            const int r = R - 3, c = C - 3;
            add(D(r, c), 1.f, 0);
            for (int a = 0; a < 3; ++a)
                for (int l = 0; l < 3; ++l) {
                    add(B(a + 1, l, c), -kx(a, l, r), 1);
                    add(B(a + 1, l, r), -kx(a, l, c), 1);
                }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    for (int l = 0; l < 3; ++l)
                        for (int m = 0; m < 3; ++m) add(A((1 << a) | (1 << b), l, m), kx(a, l, r) * kx(b, m, c), 2);
        }
    }
    return S;
}

// coefficients for this res, rounded as the single-precision products res, res * res
TermTable term_table(float res) {
    static const TermShape S = make_term_shape();
    TermTable T{};
    const float p[3] = {1.f, res, res * res};
    for (int e = 0; e < 21; ++e)
        for (int u = 0; u < 9; ++u) {
            T.idx[e][u] = S.idx[e][u];
            T.coef[e][u] = S.sgn[e][u] == 0 ? 0.f : (S.sgn[e][u] > 0 ? p[S.pw[e][u]] : -p[S.pw[e][u]]);
        }
    return T;
}

// NG gather warps, NM metric warps (NG a multiple of NM), NS pose stages per gather warp,
// L2 prefetch NP poses beyond the stages
template <int kElem, int NG, int NM, int NS, int NP>
__global__ void __launch_bounds__((NG + NM) * 32, 1) query_kernel(QueryArgs args, TermTable tt) {
    using L = Layout<kElem>;
    using GS = GatherSmem<kElem, NS>;
    constexpr int kStages = NS;
    constexpr int kPrefetch = NP;
    constexpr int kGather = NG;
    constexpr int kMetric = NM;
    static_assert(NG % NM == 0, "each metric warp serves the same number of gather warps");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    constexpr int kGB = gather_smem_bytes<kElem, NS>();
    const int64_t groups = (args.m + 31) / 32;
    const int64_t ngather = (int64_t)gridDim.x * kGather;
    // set when a bounded wait runs out: every warp then leaves its loop (after waiting, with a
    // short bound, for its own bulk copies still in flight)
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem_raw + kGather * kGB);

    if (threadIdx.x == 0) *abort_flag = 0;
    if (threadIdx.x < kGather) {
        GS& G = *reinterpret_cast<GS*>(smem_raw + threadIdx.x * kGB);
        for (int s = 0; s < kStages; ++s) mbar_init(&G.bars[s], 4);
        for (int s = 0; s < 2; ++s) { mbar_init(&G.full[s], 1); mbar_init(&G.empty[s], 1); }
        fence_mbar_init();
    }
    __syncthreads();

    if (warp < kGather) {
        // =============================== gather warp ===============================
        GS& G = *reinterpret_cast<GS*>(smem_raw + warp * kGB);
        const int j = lane >> 2, q = lane & 3;
        const int bx = j & 1;
        int mslot[6];
#pragma unroll
        for (int ii = 0; ii < 6; ++ii) {
            const int e = (kElem == 2) ? 2 * (q + 4 * (ii >> 1)) + (ii & 1) : q + 4 * ii;
            mslot[ii] = (e < 21) ? mom_slot(e, j) : -1;
        }
        const int corner_off = L::slot(j >> 1) + bx * L::kNodeBytes;
        int t_idx[9];
        float t_coef[9];
        const int te = lane < 21 ? lane : 0;
#pragma unroll
        for (int u = 0; u < 9; ++u) {
            t_idx[u] = tt.idx[te][u];
            t_coef[u] = tt.coef[te][u];
        }
        const int64_t nx = args.nx, nxy = (int64_t)args.nx * args.ny;
        const char* coeffs = reinterpret_cast<const char*>(args.coeffs);
        // byte offset of my node pair (lanes 0..3: pairs (y, z) = (0, 0), (1, 0), (0, 1), (1, 1))
        const int64_t pair_off = ((lane & 1) * nx + ((lane >> 1) & 1) * nxy) * (int64_t)L::kNodeBytes;
        uint32_t phase_bits = 0;
        int k = 0;
        for (int64_t g = (int64_t)blockIdx.x * kGather + warp; g < groups; g += ngather, ++k) {
            const int sl = k & 1;
            const uint32_t use = (uint32_t)(k >> 1);
            if (__any_sync(0xffffffffu, *abort_flag != 0 || !mbar_wait_bounded(&G.empty[sl], (use & 1u) ^ 1u, args.wait_ns))) {
                set_error(args.err, FIF_ETIMEOUT);
                *abort_flag = 1;
                break;
            }
            float* slot = G.slot[sl];
            const int64_t p0 = g * 32;
            const int cnt = (int)(args.m - p0 < 32 ? args.m - p0 : 32);
            // ---- phase P: lane = pose ----
            if (lane < cnt) {
                const float* ps = args.poses + (p0 + lane) * 7;
                float t[3], qv[4];
#pragma unroll
                for (int a = 0; a < 3; ++a) t[a] = __ldg(ps + a);
#pragma unroll
                for (int a = 0; a < 4; ++a) qv[a] = __ldg(ps + 3 + a);
                uint32_t st = 0;
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
                const float org[3] = {args.ox, args.oy, args.oz};
                const int dims[3] = {args.nx, args.ny, args.nz};
                float w[3];
                int i0[3];
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
                    for (int kk = 0; kk < 10; ++kk) vr[kk] = 0.f;
                }
                const int64_t base = i0[0] + nx * i0[1] + nxy * i0[2];
                G.pt.src[lane] = coeffs + base * (int64_t)L::kNodeBytes;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                    G.pt.wj[lane][jj] = ((jj & 1) ? w[0] : 1.f - w[0]) * ((jj & 2) ? w[1] : 1.f - w[1]) *
                                        ((jj & 4) ? w[2] : 1.f - w[2]);
#pragma unroll
                for (int kk = 0; kk < 10; ++kk) G.pt.vr2[kk][lane] = make_float2(vr[kk], vr[kk]);
                float* row = slot + lane * kRow;
#pragma unroll
                for (int a = 0; a < 3; ++a) row[21 + a] = t[a];
#pragma unroll
                for (int a = 0; a < 4; ++a) row[24 + a] = qv[a];
                row[28] = __fadd_rn(args.ox, __fmul_rn(args.res, (float)i0[0]));
                row[29] = __fadd_rn(args.oy, __fmul_rn(args.res, (float)i0[1]));
                row[30] = __fadd_rn(args.oz, __fmul_rn(args.res, (float)i0[2]));
                row[31] = __uint_as_float(st);
            }
            __syncwarp();
            auto pair_src = [&](int i) -> const void* { return G.pt.src[i] + pair_off; };
            if (lane < 4) {
                for (int i = 0; i < min(cnt, kPrefetch + kStages - 1); ++i)
                    bulk_prefetch_l2(pair_src(i), L::kPairBytes);
                fence_proxy_async();
                for (int i = 0; i < min(cnt, kStages - 1); ++i) {
                    uint64_t* bar = &G.bars[i % kStages];
                    mbar_arrive_expect_tx(bar, L::kPairBytes);
                    bulk_g2s(G.stage[i % kStages] + L::slot(lane), pair_src(i), L::kPairBytes, bar);
                }
            }
            // ---- phase G: warp per pose ----
            bool dead = false;
            int s = 0;                          // stage of pose i
            int sn = kStages - 1;               // stage of pose i + kStages - 1
            for (int i = 0; i < cnt; ++i, s = (s == kStages - 1) ? 0 : s + 1, sn = (sn == kStages - 1) ? 0 : sn + 1) {
                if (lane < 4) {
                    const int inext = i + kStages - 1;
                    if (inext < cnt) {
                        fence_proxy_async();
                        mbar_arrive_expect_tx(&G.bars[sn], L::kPairBytes);
                        bulk_g2s(G.stage[sn] + L::slot(lane), pair_src(inext), L::kPairBytes, &G.bars[sn]);
                    }
                    const int ipf = i + kStages - 1 + kPrefetch;
                    if (ipf < cnt) bulk_prefetch_l2(pair_src(ipf), L::kPairBytes);
                }
                if (__any_sync(0xffffffffu, !mbar_wait_bounded(&G.bars[s], (phase_bits >> s) & 1u, args.wait_ns))) {
                    set_error(args.err, FIF_ETIMEOUT);
                    *abort_flag = 1;
                    // the copies of poses i .. i + kStages - 1 may still be in flight
                    if (lane == 0)
                        for (int r = i; r < min(cnt, i + kStages); ++r)
                            mbar_wait_bounded(&G.bars[r % kStages], ((phase_bits >> (r % kStages)) & 1u) ^
                                                                        (r - i >= kStages ? 1u : 0u),
                                              100000000ull);
                    dead = true;
                    break;
                }
                phase_bits ^= (1u << s);
                const float wj = G.pt.wj[i][j];
                const unsigned char* C = G.stage[s] + corner_off;
                float v[6];
                if constexpr (kElem == 2) {
                    // blocks of 22 bfloat16: word kk * 11 + p holds entries 2p (low half) and 2p + 1
                    const uint32_t* Cw = reinterpret_cast<const uint32_t*>(C) + q;
                    float2 acc[3];
#pragma unroll
                    for (int pp = 0; pp < 3; ++pp) acc[pp] = make_float2(0.f, 0.f);
#pragma unroll
                    for (int kk = 0; kk < 10; ++kk) {
                        const float2 vv = G.pt.vr2[kk][i];
#pragma unroll
                        for (int pp = 0; pp < 3; ++pp) {
                            const uint32_t u = Cw[kk * 11 + 4 * pp];
                            acc[pp] = fma2(vv, make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u)),
                                           acc[pp]);
                        }
                    }
#pragma unroll
                    for (int pp = 0; pp < 3; ++pp) {
                        const float2 r = mul2(acc[pp], make_float2(wj, wj));
                        v[2 * pp] = r.x;
                        v[2 * pp + 1] = r.y;
                    }
                } else {
                    float vrj[10];
#pragma unroll
                    for (int kk = 0; kk < 10; ++kk) vrj[kk] = wj * G.pt.vr2[kk][i].x;
#pragma unroll
                    for (int ii = 0; ii < 6; ++ii) {
                        float acc = 0.f;
#pragma unroll
                        for (int kk = 0; kk < 10; ++kk) acc = fmaf(vrj[kk], L::load(C, kk * 21 + 4 * ii + q), acc);
                        v[ii] = acc;
                    }
                }
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
#pragma unroll
                for (int ii = 0; ii < 6; ++ii)
                    if (mslot[ii] >= 0) G.mom[mslot[ii]] = v[ii];
                __syncwarp();
                if (lane < 21) {
                    float acc = 0.f;
#pragma unroll
                    for (int u = 0; u < 9; ++u) acc = fmaf(t_coef[u], G.mom[t_idx[u]], acc);
                    slot[i * kRow + lane] = acc;
                }
                __syncwarp();
            }
            if (dead) break;
            fence_proxy_async();
            if (lane == 0) mbar_arrive(&G.full[sl]);
        }
    } else {
        // =============================== metric warp ===============================
        const int mw = warp - kGather;
        int k = 0;
        bool dead = false;
        for (; !dead; ++k) {
            bool any = false;
#pragma unroll 1
            for (int h = 0; h < kGather / kMetric; ++h) {
                const int gw = mw + h * kMetric;
                const int64_t g = (int64_t)blockIdx.x * kGather + gw + (int64_t)k * ngather;
                if (g >= groups) continue;
                any = true;
                GS& G = *reinterpret_cast<GS*>(smem_raw + gw * kGB);
                const int sl = k & 1;
                const uint32_t use = (uint32_t)(k >> 1);
                if (__any_sync(0xffffffffu, *abort_flag != 0 || !mbar_wait_bounded(&G.full[sl], use & 1u, args.wait_ns))) {
                    set_error(args.err, FIF_ETIMEOUT);
                    *abort_flag = 1;
                    dead = true;
                    break;
                }
                const float* slot = G.slot[sl];
                const int64_t p0 = g * 32;
                const int cnt = (int)(args.m - p0 < 32 ? args.m - p0 : 32);
                if (lane < cnt) {
                    const float* row = slot + lane * kRow;
                    float Tp[21];
#pragma unroll
                    for (int e = 0; e < 21; ++e) Tp[e] = row[e];
                    const float t[3] = {row[21], row[22], row[23]};
                    const float c0[3] = {row[28], row[29], row[30]};
                    uint32_t st = __float_as_uint(row[31]);
                    Blocks T;
                    unpack(Tp, T);
                    if (args.flags & FIF_Q_WORLD) {
                        shift_ref(T, c0);
                    } else {
                        float R[3][3];
                        quat_to_rot(row[24], row[25], row[26], row[27], R);
                        const float b[3] = {c0[0] - t[0], c0[1] - t[1], c0[2] - t[2]};
                        shift_ref(T, b);
                        rotate_into(T, R);
                    }
                    float fim[21];
                    pack(T, fim);
                    const bool nan = (st & FIF_POSE_NAN) != 0;
                    if (nan) {
#pragma unroll
                        for (int e = 0; e < 21; ++e) fim[e] = __int_as_float(0x7fc00000);
                    }
                    const int64_t pid = p0 + lane;
                    // stage the outputs in this pose's slot row (T, t and q are consumed) so the
                    // warp can write them out with coalesced stores
                    float* wrow = const_cast<float*>(row);
#pragma unroll
                    for (int e = 0; e < 21; ++e) wrow[e] = fim[e];
                    double mv[3] = {0.0, 0.0, 0.0};
                    if (args.flags & FIF_Q_METRICS) {
                        if (args.flags & FIF_Q_TRACE) mv[0] = nan ? (double)NAN : (double)trace6(fim);
                        if (args.flags & FIF_Q_LOGDET) {
                            double lad;
                            int sg;
                            logdet_f64(fim, lad, sg);
                            if (nan) { lad = NAN; sg = 0; }
                            mv[1] = lad;
                            if (args.sign) args.sign[pid] = (int8_t)sg;
                            if (sg <= 0 && !nan) st |= FIF_POSE_NOT_PD;
                        }
                        if (args.flags & FIF_Q_LMIN) {
                            double lm = lambda_min_f64(fim);
                            if (nan) lm = NAN;
                            mv[2] = lm;
                            if (!(lm > 0.0) && !nan) st |= FIF_POSE_NOT_PD;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const unsigned long long b = (unsigned long long)__double_as_longlong(mv[c]);
                        wrow[21 + 2 * c] = __uint_as_float((uint32_t)(b & 0xffffffffu));
                        wrow[22 + 2 * c] = __uint_as_float((uint32_t)(b >> 32));
                    }
                    if (args.status) args.status[pid] = (int32_t)st;
                }
                __syncwarp();
                if (args.fim) {
                    float* out = args.fim + p0 * 21;
                    for (int idx = lane; idx < cnt * 21; idx += 32) out[idx] = slot[(idx / 21) * kRow + idx % 21];
                }
                if (args.metrics && (args.flags & FIF_Q_METRICS)) {
                    const int cols = args.flags & FIF_Q_METRICS;
                    double* out = args.metrics + p0 * 3;
                    for (int idx = lane; idx < cnt * 3; idx += 32) {
                        const int c = idx % 3;
                        if (!(cols & (FIF_Q_TRACE << c))) continue;   // unselected columns stay untouched
                        const float* r = slot + (idx / 3) * kRow + 21 + 2 * c;
                        const unsigned long long b =
                            (unsigned long long)__float_as_uint(r[0]) | ((unsigned long long)__float_as_uint(r[1]) << 32);
                        out[idx] = __longlong_as_double((long long)b);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&G.empty[sl]);
            }
            if (!any) break;
        }
    }
}

}  // namespace

template <int kElem, int NG, int NM, int NS, int NP>
int launch_query_cfg(const QueryArgs& a, cudaStream_t stream) {
    auto kern = query_kernel<kElem, NG, NM, NS, NP>;
    const int smem = NG * gather_smem_bytes<kElem, NS>() + 16;   // + the abort flag
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return FIF_ECUDA;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (a.m + 31) / 32;
    const int64_t need = (groups + NG - 1) / NG;
    const int64_t grid = std::min<int64_t>(need, (int64_t)sms);
    if (grid <= 0) return FIF_OK;
    kern<<<(unsigned)grid, (NG + NM) * 32, smem, stream>>>(a, term_table(a.res));
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

// A large batch is bound by the bytes in flight: more gather warps with two stages each.  A
// small batch (fewer than 4 groups of 32 poses per gather warp of that configuration) is bound
// by the latency of each warp's poses: fewer gather warps, three stages and a deeper L2 prefetch.
int launch_query(const QueryArgs& a, cudaStream_t stream) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t groups = (a.m + 31) / 32;
    if (a.storage == FIF_STORAGE_BF16) {
        if (groups < 4 * 10 * (int64_t)sms) return launch_query_cfg<2, 8, 8, 3, 2>(a, stream);
        return launch_query_cfg<2, 10, 5, 2, 1>(a, stream);
    }
    if (groups < 4 * kGather * (int64_t)sms) return launch_query_cfg<4, 6, 6, 3, 4>(a, stream);
    return launch_query_cfg<4, kGather, kMetric, 2, 1>(a, stream);
}

}  // namespace fif
