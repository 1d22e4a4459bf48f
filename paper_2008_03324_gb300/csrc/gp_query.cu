// gp_query.cu -- Fisher Information Field with GP visibility (Sec. V-B-2 of the paper): the
// pose query for sm_103a (the build is in gp_build.cu).
//
// The GP visibility of a landmark with bearing u seen along optical axis z is
//   v_gp(z) = K_z (K^s + s_n^2 I)^-1 v^s(u),   v^s_g(u) = 1 / (1 + exp(-k_s (z_g . u - cos a))),
// so the field is separable with N_v = N_s (Eq. gp_vis_approx, Eq. fim_separation).  The
// field stores, per node c and sample axis g, the 6x6
//   D_g(c) = sum_{i in shell(c)} v^s_g(u_i) I_i        (I_i about the node, as in build.cu)
// and the query contracts it with the kriging weights a(z) = (K^s + s_n^2 I)^-1 K_z^T:
//   I(T) = sum_g a_g(z) D_g(t),  which equals K_z C_I with the paper's C_I = (K^s)^-1 D.
// Storing D instead of C_I keeps every stored weight in (0, 1); the ill-conditioning of K^s
// then sits in a(z) alone, which the query evaluates with double-precision kernel values and
// compensated single-precision sums.
//
// Node record (float32): entry e (upper-triangular 6x6, row-major) of D_g at e * rs + g,
// rs = fif_gp_row_stride(N_s) (rs = 2 mod 4: a lane per entry e reading 8-byte pairs hits
// distinct banks), zero pads, stride = 21 rs rounded up to 4 floats.
//
// Query (gp_query_kernel): a persistent CTA walks groups of 32 poses with three warp roles:
//  contract (4 warps)  warp p streams the x-adjacent corner pair p of each pose (one bulk copy
//                      of both node records into its own ring), lane e < 21 forms
//                      w_j sum_g a_g D_g[e] for both corners (in single precision, or as a
//                      compensated dot product with FIF_Q_GP_COMPENSATED);
//  weights  (8 warps)  K_z in double-float arithmetic, a(z) = W K_z as compensated
//                      single-precision sums with W split into high and low parts
//                      (two-product / two-sum);
//  metric   (2 or 4)   one per buffer of the corner table (4 buffers up to N_s = 64, when
//                      they fit), lane = pose: moves the 8 corner
//                      matrices from their nodes to the camera position, sums, rotates into the
//                      camera frame, and reduces to trace / log|det| / lambda_min as the
//                      quadratic query does.
#include "fif_common.cuh"
#include "fif_internal.h"

#include <cmath>
#include <cstring>

namespace fif {

namespace {

// ------------------------------------------------------------------------------------
// query
// ------------------------------------------------------------------------------------
constexpr int kGqContract = 4;                 // one warp per x-adjacent corner pair
constexpr int kGqWeights = 8;                  // one block of kGqPB poses per group each
constexpr int kGqMaxNB = 4;                    // table buffers (= metric warps) at most
constexpr int kGqPB = 4;                       // poses per weights block
constexpr int kEbRow = 169;                    // floats per pose in the corner table (odd)
constexpr int kGqMaxStages = 4;

struct GqLayout {
    int ring, atab, eb, kbuf, ptab, wsm, tab, bars, flag, total, stages, nb;
    int w_smem;   // 1: W is staged in shared memory at wsm; 0: read from global memory
};

// shared-memory layout for S floats per node, row stride rs, N_s samples, `stages` ring slots per
// contract warp, W in shared memory or not, nb buffers of the weights and corner tables
__host__ __device__ inline GqLayout gq_layout(int S, int rs, int ns, int stages, int w_smem, int nb) {
    GqLayout L;
    int off = 0;
    L.stages = stages;
    L.w_smem = w_smem;
    L.nb = nb;
    L.ring = off;  off += kGqContract * stages * 2 * S * 4;
    L.atab = off;  off += nb * 32 * rs * 4;
    L.eb = off;    off += nb * 32 * kEbRow * 4;
    off = (off + 15) / 16 * 16;
    L.kbuf = off;  off += kGqWeights * (kGqPB / 2) * rs * 16;
    L.ptab = off;  off += kGqContract * 2 * 32 * 16;
    L.wsm = off;   off += w_smem ? ns * rs * 8 : 0;
    L.tab = off;   off += 18 * 16;
    L.bars = off;  off += (kGqContract * kGqMaxStages + 4 * kGqMaxNB) * 8;
    L.flag = off;  off += 16;
    L.total = (off + 127) / 128 * 128;
    return L;
}

struct GqBars {
    uint64_t full[kGqContract][kGqMaxStages];
    uint64_t aready[kGqMaxNB], afree[kGqMaxNB], efull[kGqMaxNB], eempty[kGqMaxNB];
};

// lattice cell and trilinear weights of a position (the same arithmetic as query.cu)
FIF_DEV void gq_cell(const QueryArgs& a, const float t[3], uint32_t& st, int i0[3], float w[3]) {
    const float org[3] = {a.ox, a.oy, a.oz};
    const int dims[3] = {a.nx, a.ny, a.nz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float gg = __fdiv_rn(__fsub_rn(t[c], org[c]), a.res);
        if (!(st & FIF_POSE_NAN)) {
            if (gg < 0.f || gg > (float)(dims[c] - 1)) st |= FIF_POSE_OUTSIDE;
        } else {
            gg = 0.f;
        }
        if (a.flags & FIF_Q_NEAREST) {
            int ii = (int)floorf(__fadd_rn(gg, 0.5f));
            ii = max(0, min(ii, dims[c] - 1));
            const int b0 = min(ii, dims[c] - 2);
            i0[c] = b0;
            w[c] = (ii > b0) ? 1.f : 0.f;
        } else {
            int ii = (int)floorf(gg);
            ii = max(0, min(ii, dims[c] - 2));
            i0[c] = ii;
            w[c] = fminf(fmaxf(gg - (float)ii, 0.f), 1.f);
        }
    }
}

FIF_DEV uint32_t gq_pose(const QueryArgs& a, int64_t p, float t[3], float q[4]) {
    const float* ps = a.poses + p * 7;
#pragma unroll
    for (int c = 0; c < 3; ++c) t[c] = __ldg(ps + c);
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = __ldg(ps + 3 + c);
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) finite &= isfinite(t[c]);
#pragma unroll
    for (int c = 0; c < 4; ++c) finite &= isfinite(q[c]);
    const float n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    finite &= (n2 > 0.f) && isfinite(n2);
    uint32_t st = 0;
    if (!finite) st |= FIF_POSE_NAN;
    if (fabsf(n2 - 1.f) > 1e-3f) st |= FIF_POSE_QUAT;
    return st;
}

// position `it` of this CTA's pose stream (its groups of 32, in order) -> pose index, or -1
FIF_DEV int64_t gq_stream(int64_t it, int64_t m) {
    const int64_t k = it >> 5;
    const int64_t p = ((int64_t)blockIdx.x + k * (int64_t)gridDim.x) * 32 + (it & 31);
    return p < m ? p : -1;
}

FIF_DEV bool gq_wait(uint64_t* bar, uint32_t parity, volatile int* flag, int* err) {
    if (mbar_wait_bounded(bar, parity)) return true;
    set_error(err, FIF_ETIMEOUT);
    *flag = 1;
    return false;
}

// error-free transformations (single precision, round to nearest)
FIF_DEV void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
FIF_DEV void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// exp(xh + xl) for xh + xl in [-87, 0] as a (high, low) pair of floats: Tang's table-driven
// method (ACM TOMS 15(2), 1989) carried out in double-float arithmetic.  x = N ln2/32 + r with
// ln2/32 = C1 + C2 + C3 (C1 has 12 significant bits, so N C1 is exact), exp(x) =
// 2^(N div 32) 2^((N mod 32)/32) (1 + expm1(r)), |r| <= ln2/64, expm1(r) = r + r^2/2 + r^3 q(r)
// with q the next four Taylor terms.  k = (C1, C2, C3, 32/ln2); tab[j] = 2^(j/32).
// Relative error below 2e-13 (checked against double-precision exp over [-87, 0]).
FIF_DEV float2 exp_df(float xh, float xl, float4 k, const float2* tab) {
    const float N = rintf(__fmul_rn(xh, k.w));
    const float r1 = fmaf(-N, k.x, xh);
    float pn, pe;
    two_prod(N, k.y, pn, pe);
    float rh0, re;
    two_sum(r1, -pn, rh0, re);
    const float rl0 = __fsub_rn(__fadd_rn(__fsub_rn(re, pe), xl), __fmul_rn(N, k.z));
    float rh, rl;
    two_sum(rh0, rl0, rh, rl);
    const float s = rh * fmaf(rh, fmaf(rh, fmaf(rh, 1.f / 720.f, 1.f / 120.f), 1.f / 24.f), 1.f / 6.f);
    float r2h, r2e;
    two_prod(rh, rh, r2h, r2e);
    const float small = rl + 0.5f * (r2e + 2.f * (rh * rl)) + r2h * s;
    float ph, pe2;
    two_sum(rh, 0.5f * r2h, ph, pe2);
    const float pl = pe2 + small;
    const int Ni = (int)N;
    const int j = Ni & 31;
    const int m = (Ni - j) >> 5;
    const float2 T = tab[j];
    float q, qe;
    two_prod(T.x, ph, q, qe);
    float sh, se;
    two_sum(T.x, q, sh, se);
    const float sl = ((se + T.y) + qe) + fmaf(T.x, pl, T.y * ph);
    const float scale = __int_as_float((m + 127) << 23);   // 2^m, m >= -126 on this range
    return make_float2(sh * scale, sl * scale);
}

// K_z[h] = exp(-|z - z_h|^2 / (2 l^2)) = exp((z.z_h - 1) / l^2) for unit z, z_h given as
// (high, low) float parts; 1/l^2 = cH + cL.  Relative error below 5e-13.
FIF_DEV float2 kz_df(const float* zH, const float* zL, float4 aH, float4 aL, float cH, float cL, float4 k,
                     const float2* tab) {
    float p0, e0, p1, e1, p2, e2;
    two_prod(zH[0], aH.x, p0, e0);
    two_prod(zH[1], aH.y, p1, e1);
    two_prod(zH[2], aH.z, p2, e2);
    e0 = fmaf(zH[0], aL.x, fmaf(zL[0], aH.x, e0));
    e1 = fmaf(zH[1], aL.y, fmaf(zL[1], aH.y, e1));
    e2 = fmaf(zH[2], aL.z, fmaf(zL[2], aH.z, e2));
    float s1, f1, s2, f2;
    two_sum(p0, p1, s1, f1);
    two_sum(s1, p2, s2, f2);
    const float tl = ((f1 + f2) + (e0 + e1)) + e2;
    float yh, ye;
    two_sum(1.f, -s2, yh, ye);
    const float yl = ye - tl;
    float xh, xe;
    two_prod(yh, cH, xh, xe);
    const float xl = xe + fmaf(yh, cL, yl * cH);
    if (!(xh <= 87.f)) return make_float2(0.f, 0.f);
    return exp_df(-xh, -xl, k, tab);
}

// (hi, lo) += W K for two poses at once, in double-float arithmetic on packed pairs:
// W = Wh + Wl (the same for both halves), K = Kh + Kl per pose.  The product of the high parts
// is split exactly with an fma (two-product), its sum into hi exactly with Knuth's two-sum, and
// the rounding errors plus the cross terms go to lo.  Only -W.hi is used to form -p, so no
// packed negation is needed.
FIF_DEV void df_fma2(float2 Wh, float2 Whn, float2 Wl, float2 Kh, float2 Kl, float2& hi, float2& lo) {
    const float2 pn = mul2(Whn, Kh);            // -p, exact negation of fl(W K)
    float2 e = fma2(Wh, Kh, pn);                // W K - p, exact
    e = fma2(Wh, Kl, e);
    e = fma2(Wl, Kh, e);
    const float2 s = sub2(hi, pn);              // hi + p
    const float2 bb = sub2(s, hi);
    const float2 err = sub2(sub2(hi, sub2(s, bb)), add2(pn, bb));   // (hi - (s - bb)) + (p - bb)
    hi = s;
    lo = add2(lo, add2(err, e));
}

// One step of the compensated dot product on packed pairs: (s, e) += a v, where an = -a.
// fl(a v) is formed negated (exact), its rounding error a v - fl(a v) exactly by an fma, the sum
// s + fl(a v) by Knuth's two-sum; both errors go to e.
FIF_DEV void dot2_step(float2 a, float2 an, float2 v, float2& s, float2& e) {
    const float2 pn = mul2(an, v);                      // -fl(a v)
    const float2 pe = fma2(a, v, pn);                   // a v - fl(a v)
    const float2 sn = sub2(s, pn);                      // fl(s + fl(a v))
    const float2 bb = sub2(sn, s);
    const float2 err = sub2(sub2(s, sub2(sn, bb)), add2(pn, bb));   // (s - (sn - bb)) + (p - bb)
    s = sn;
    e = add2(e, add2(err, pe));
}

// two compensated packed sums (s, e) and (t, f) combined into one float: the four partial sums
// by two-sums, then all rounding errors added
FIF_DEV float dot2_finish(float2 s, float2 e, float2 t, float2 f) {
    float h0, l0, h1, l1, h, l;
    two_sum(s.x, s.y, h0, l0);
    two_sum(t.x, t.y, h1, l1);
    two_sum(h0, h1, h, l);
    const float err = __fadd_rn(__fadd_rn(__fadd_rn(l0, l1), l), __fadd_rn(__fadd_rn(e.x, e.y), __fadd_rn(f.x, f.y)));
    return __fadd_rn(h, err);
}

// group k uses table buffer k mod NB
// NB table buffers and as many metric warps; kComp: compensated contraction (FIF_Q_GP_COMPENSATED)
template <int G, int NB, bool kComp>
__global__ void __launch_bounds__((kGqContract + kGqWeights + NB) * 32, 1) gp_query_kernel(QueryArgs a, GqLayout L) {
    constexpr int kThreads = (kGqContract + kGqWeights + NB) * 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw + L.ring);
    float* atab = reinterpret_cast<float*>(smem_raw + L.atab);
    float* eb = reinterpret_cast<float*>(smem_raw + L.eb);
    float4* kbuf = reinterpret_cast<float4*>(smem_raw + L.kbuf);
    int4* ptab = reinterpret_cast<int4*>(smem_raw + L.ptab);
    float2* wsm = reinterpret_cast<float2*>(smem_raw + L.wsm);
    float4* ctab = reinterpret_cast<float4*>(smem_raw + L.tab);   // exp constants and table
    const float2* wsrc = L.w_smem ? wsm : a.gp_wt;
    GqBars& B = *reinterpret_cast<GqBars*>(smem_raw + L.bars);
    volatile int* flag = reinterpret_cast<volatile int*>(smem_raw + L.flag);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NS = L.stages, rs = a.gp_rs, ns = a.gp_ns, S = a.stride;
    const int64_t m = a.m;
    const int64_t groups = (m + 31) / 32;

    if (threadIdx.x == 0) {
        for (int j = 0; j < kGqContract; ++j)
            for (int s = 0; s < kGqMaxStages; ++s) mbar_init(&B.full[j][s], 1);
        for (int b = 0; b < NB; ++b) {
            mbar_init(&B.aready[b], kGqWeights);
            mbar_init(&B.afree[b], kGqContract);
            mbar_init(&B.efull[b], kGqContract);
            mbar_init(&B.eempty[b], 1);
        }
        *flag = 0;
        fence_mbar_init();
    }
    for (int idx = threadIdx.x; idx < NB * 32 * rs; idx += kThreads) atab[idx] = 0.f;   // pads stay zero
    if (L.w_smem)
        for (int idx = threadIdx.x; idx < ns * rs; idx += kThreads) wsm[idx] = __ldg(a.gp_wt + idx);
    for (int idx = threadIdx.x; idx < 18; idx += kThreads) ctab[idx] = __ldg(a.gp_consts + idx);
    __syncthreads();

    if (warp < kGqContract) {
        // ================================ contract warp ================================
        // warp jp owns corners j = 2 jp + bx, bx = 0, 1: the two nodes adjacent along x, which
        // are contiguous in memory and arrive with one bulk copy
        const int jp = warp;
        const int by = jp & 1, bz = jp >> 1;
        const int S2 = 2 * S;
        float* myring = ring + (size_t)jp * NS * S2;
        int4* mytab = ptab + jp * 64;    // [2][32]: node of the pair (low, high word), w of bx = 0, 1
        const int64_t nx = a.nx, nxy = (int64_t)a.nx * a.ny;
        const float* coeffs = reinterpret_cast<const float*>(a.coeffs);
        // the pair's first node and the two trilinear weights for every pose of group k
        auto fill_table = [&](int64_t k) {
            const int64_t p = ((int64_t)blockIdx.x + k * (int64_t)gridDim.x) * 32 + lane;
            if (p < m) {
                float t[3], q[4];
                uint32_t st = gq_pose(a, p, t, q);
                int i0[3];
                float w[3];
                gq_cell(a, t, st, i0, w);
                const int64_t node = i0[0] + nx * (i0[1] + by) + nxy * (i0[2] + bz);
                const float wyz = (by ? w[1] : 1.f - w[1]) * (bz ? w[2] : 1.f - w[2]);
                mytab[(k & 1) * 32 + lane] = make_int4((int)(uint32_t)(node & 0xffffffffu), (int)(node >> 32),
                                                       __float_as_int((1.f - w[0]) * wyz), __float_as_int(w[0] * wyz));
            }
            __syncwarp();
        };
        auto node_of = [&](int64_t it) {   // the table of it's group is filled
            const int4 e = mytab[((it >> 5) & 1) * 32 + (it & 31)];
            return (int64_t)(uint32_t)e.x | ((int64_t)e.y << 32);
        };
        auto issue = [&](int64_t it) {   // lane 0 only
            if (gq_stream(it, m) < 0) return;
            const int64_t node = node_of(it);
            uint64_t* bar = &B.full[jp][it % NS];
            fence_proxy_async();
            mbar_arrive_expect_tx(bar, (uint32_t)S2 * 4u);
            bulk_g2s(myring + (it % NS) * S2, coeffs + node * S, (uint32_t)S2 * 4u, bar);
        };
        fill_table(0);
        if (lane == 0)
            for (int64_t it = 0; it < NS - 1; ++it) issue(it);
        int64_t it = 0;
        for (;; ++it) {
            const int64_t p = gq_stream(it, m);
            if (p < 0 || *flag) break;
            const int64_t k = it >> 5;
            const int i = (int)(it & 31);
            const int b = (int)(k % NB);
            const uint32_t use = (uint32_t)((k / NB) & 1);
            if (i == 0) {
                if ((int64_t)blockIdx.x + (k + 1) * (int64_t)gridDim.x < groups) fill_table(k + 1);
                if (!gq_wait(&B.aready[b], use, flag, a.err)) break;
                if (k >= NB && !gq_wait(&B.eempty[b], use ^ 1u, flag, a.err)) break;
            }
            if (lane == 0) issue(it + NS - 1);
            if (!gq_wait(&B.full[jp][it % NS], (uint32_t)((it / NS) & 1), flag, a.err)) break;
            const int4 te = mytab[b * 32 + i];
            if (lane < 21) {
                const float2* av = reinterpret_cast<const float2*>(atab + (b * 32 + i) * rs);
                const float2* r0 = reinterpret_cast<const float2*>(myring + (it % NS) * S2 + lane * rs);
                const float2* r1 = reinterpret_cast<const float2*>(myring + (it % NS) * S2 + S + lane * rs);
                const float2 zero = make_float2(0.f, 0.f);
                const int n2 = rs >> 1;
                float v0, v1;
                if constexpr (kComp) {
                    // entry e = lane of sum_g a_g D_g for both corners of the pair as a compensated
                    // dot product (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J.
                    // Sci. Comput. 26(6), 2005, Algorithm Dot2): each product split exactly with an
                    // fma, each addition with Knuth's two-sum, the rounding errors summed apart, so
                    // the result is as accurate as if carried in twice the precision although the
                    // weights a_g change sign and cancel.  Packed pairs run over (g, g + 1); two
                    // independent chains per corner (even and odd pairs of g).
                    const float2 neg1 = make_float2(-1.f, -1.f);
                    float2 s0 = zero, e0 = zero, s1 = zero, e1 = zero, t0 = zero, f0 = zero, t1 = zero, f1 = zero;
                    int g2 = 0;
                    for (; g2 + 1 < n2; g2 += 2) {
                        const float2 ag = av[g2], ah = av[g2 + 1];
                        const float2 an = mul2(ag, neg1), hn = mul2(ah, neg1);
                        dot2_step(ag, an, r0[g2], s0, e0);
                        dot2_step(ag, an, r1[g2], s1, e1);
                        dot2_step(ah, hn, r0[g2 + 1], t0, f0);
                        dot2_step(ah, hn, r1[g2 + 1], t1, f1);
                    }
                    if (g2 < n2) {
                        const float2 ag = av[g2];
                        const float2 an = mul2(ag, neg1);
                        dot2_step(ag, an, r0[g2], s0, e0);
                        dot2_step(ag, an, r1[g2], s1, e1);
                    }
                    v0 = dot2_finish(s0, e0, t0, f0);
                    v1 = dot2_finish(s1, e1, t1, f1);
                } else {
                    // both corners of the pair at once in single precision: each weight pair is
                    // loaded once, four independent accumulators keep several shared-memory loads
                    // in flight
                    float2 a0 = zero, a1 = zero, c0 = zero, c1 = zero;
                    int g2 = 0;
#pragma unroll 4
                    for (; g2 + 1 < n2; g2 += 2) {
                        const float2 w0 = av[g2], w1 = av[g2 + 1];
                        a0 = fma2(r0[g2], w0, a0);
                        a1 = fma2(r0[g2 + 1], w1, a1);
                        c0 = fma2(r1[g2], w0, c0);
                        c1 = fma2(r1[g2 + 1], w1, c1);
                    }
                    if (g2 < n2) {
                        const float2 w0 = av[g2];
                        a0 = fma2(r0[g2], w0, a0);
                        c0 = fma2(r1[g2], w0, c0);
                    }
                    v0 = (a0.x + a0.y) + (a1.x + a1.y);
                    v1 = (c0.x + c0.y) + (c1.x + c1.y);
                }
                float* er = eb + (b * 32 + i) * kEbRow + 2 * jp * 21 + lane;
                er[0] = __int_as_float(te.z) * v0;
                er[21] = __int_as_float(te.w) * v1;
            }
            __syncwarp();
            if (i == 31 || gq_stream(it + 1, m) < 0) {
                if (lane == 0) {
                    mbar_arrive(&B.efull[b]);
                    mbar_arrive(&B.afree[b]);
                }
            }
        }
        // after an early exit, wait (bounded) for this warp's copies that may still be in flight
        // (stream positions it .. it + NS - 1 at most)
        if (lane == 0 && *flag) {
            for (int64_t r = it; r < it + NS; ++r)
                if (gq_stream(r, m) >= 0) mbar_wait_bounded(&B.full[jp][r % NS], (uint32_t)((r / NS) & 1), 100000000ull);
        }
    } else if (warp < kGqContract + kGqWeights) {
        // ================================ weights warp ================================
        const int w = warp - kGqContract;
        float4* kb = kbuf + (size_t)w * (kGqPB / 2) * rs;   // [pose pair][h]: (Kh0, Kh1, Kl0, Kl1)
        float* kbf = reinterpret_cast<float*>(kb);
        for (int64_t k = 0;; ++k) {
            const int64_t g = (int64_t)blockIdx.x + k * gridDim.x;
            if (g >= groups || *flag) break;
            const int b = (int)(k % NB);
            if (k >= NB && !gq_wait(&B.afree[b], (uint32_t)((k / NB) & 1) ^ 1u, flag, a.err)) break;
            const int cnt = (m - g * 32 < 32) ? (int)(m - g * 32) : 32;
            for (int i0 = w * kGqPB; i0 < cnt; i0 += kGqWeights * kGqPB) {
                // optical axes of the block's poses: normalised in double precision (as the
                // oracle does), then kept as (high, low) float pairs
                float zl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                int okl = 0;
                if (lane < kGqPB && i0 + lane < cnt) {
                    const float* ps = a.poses + (g * 32 + i0 + lane) * 7 + 3;
                    const double qw = __ldg(ps), qx = __ldg(ps + 1), qy = __ldg(ps + 2), qz = __ldg(ps + 3);
                    const double nrm = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
                    if (nrm > 0.0 && isfinite(nrm)) {
                        const double W_ = qw / nrm, X_ = qx / nrm, Y_ = qy / nrm, Z_ = qz / nrm;
                        const double zd[3] = {2.0 * (X_ * Z_ + W_ * Y_), 2.0 * (Y_ * Z_ - W_ * X_),
                                              1.0 - 2.0 * (X_ * X_ + Y_ * Y_)};
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            zl[c] = (float)zd[c];
                            zl[3 + c] = (float)(zd[c] - (double)zl[c]);
                        }
                        okl = 1;
                    }
                }
                float zb[kGqPB][6];
                int okb[kGqPB];
#pragma unroll
                for (int qq = 0; qq < kGqPB; ++qq) {
#pragma unroll
                    for (int c = 0; c < 6; ++c) zb[qq][c] = __shfl_sync(0xffffffffu, zl[c], qq);
                    okb[qq] = __shfl_sync(0xffffffffu, okl, qq);
                }
                // K_z[h] as (high, low) float pairs, double-float arithmetic throughout
                const float4 kc = ctab[0];
                const float cH = ctab[1].x, cL = ctab[1].y;
                const float2* etab = reinterpret_cast<const float2*>(ctab + 2);
                for (int idx = lane; idx < kGqPB * ns; idx += 32) {
                    const int qq = idx / ns, h = idx - qq * ns;
                    float zq[6];
                    int okq = okb[0];
#pragma unroll
                    for (int c = 0; c < 6; ++c) zq[c] = zb[0][c];
#pragma unroll
                    for (int r = 1; r < kGqPB; ++r)
                        if (qq == r) {
#pragma unroll
                            for (int c = 0; c < 6; ++c) zq[c] = zb[r][c];
                            okq = okb[r];
                        }
                    const float2 K = okq ? kz_df(zq, zq + 3, __ldg(a.gp_axes + h), __ldg(a.gp_axes + ns + h), cH, cL,
                                                 kc, etab)
                                         : make_float2(0.f, 0.f);
                    float* slot = kbf + 4 * ((qq >> 1) * rs + h) + (qq & 1);
                    slot[0] = K.x;
                    slot[2] = K.y;
                }
                __syncwarp();
                // a = W K for the 4 poses (two packed pairs), lane g = lane + 32 kk
                float2 ahi[G][kGqPB / 2], alo[G][kGqPB / 2];
#pragma unroll
                for (int kk = 0; kk < G; ++kk)
#pragma unroll
                    for (int pp = 0; pp < kGqPB / 2; ++pp) ahi[kk][pp] = alo[kk][pp] = make_float2(0.f, 0.f);
                const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll 2
                for (int h = 0; h < ns; ++h) {
                    float4 Kq[kGqPB / 2];
#pragma unroll
                    for (int pp = 0; pp < kGqPB / 2; ++pp) Kq[pp] = kb[pp * rs + h];
#pragma unroll
                    for (int kk = 0; kk < G; ++kk) {
                        const int gi = lane + 32 * kk;
                        const float2 Wq = gi < ns ? wsrc[h * rs + gi] : make_float2(0.f, 0.f);
                        const float2 Wh = make_float2(Wq.x, Wq.x), Wl = make_float2(Wq.y, Wq.y);
                        const float2 Whn = mul2(Wh, neg1);
#pragma unroll
                        for (int pp = 0; pp < kGqPB / 2; ++pp)
                            df_fma2(Wh, Whn, Wl, make_float2(Kq[pp].x, Kq[pp].y), make_float2(Kq[pp].z, Kq[pp].w),
                                    ahi[kk][pp], alo[kk][pp]);
                    }
                }
#pragma unroll
                for (int pp = 0; pp < kGqPB / 2; ++pp)
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        const int qq = 2 * pp + half;
                        if (i0 + qq >= cnt) continue;
                        float* row = atab + (b * 32 + i0 + qq) * rs;
#pragma unroll
                        for (int kk = 0; kk < G; ++kk) {
                            const int gi = lane + 32 * kk;
                            if (gi < ns) row[gi] = half ? ahi[kk][pp].y + alo[kk][pp].y : ahi[kk][pp].x + alo[kk][pp].x;
                        }
                    }
                __syncwarp();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.aready[b]);
        }
    } else {
        // ================================ metric warp ================================
        const int mw = warp - kGqContract - kGqWeights;   // = the table buffer it serves
        for (int64_t k = mw;; k += NB) {
            const int64_t g = (int64_t)blockIdx.x + k * gridDim.x;
            if (g >= groups || *flag) break;
            const int b = (int)(k % NB);
            if (!gq_wait(&B.efull[b], (uint32_t)((k / NB) & 1), flag, a.err)) break;
            const int cnt = (m - g * 32 < 32) ? (int)(m - g * 32) : 32;
            if (lane < cnt) {
                const int64_t p = g * 32 + lane;
                float t[3], q[4];
                uint32_t st = gq_pose(a, p, t, q);
                int i0[3];
                float w[3];
                gq_cell(a, t, st, i0, w);
                const bool world = (a.flags & FIF_Q_WORLD) != 0;
                Blocks T;
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) T.A[r][c] = T.B[r][c] = T.D[r][c] = 0.f;
                const float* er = eb + (b * 32 + lane) * kEbRow;
#pragma unroll 1
                for (int jj = 0; jj < 8; ++jj) {
                    float Ep[21];
#pragma unroll
                    for (int e = 0; e < 21; ++e) Ep[e] = er[jj * 21 + e];
                    Blocks E;
                    unpack(Ep, E);
                    const float cj[3] = {__fadd_rn(a.ox, __fmul_rn(a.res, (float)(i0[0] + (jj & 1)))),
                                         __fadd_rn(a.oy, __fmul_rn(a.res, (float)(i0[1] + ((jj >> 1) & 1)))),
                                         __fadd_rn(a.oz, __fmul_rn(a.res, (float)(i0[2] + (jj >> 2))))};
                    const float d[3] = {world ? cj[0] : cj[0] - t[0], world ? cj[1] : cj[1] - t[1],
                                        world ? cj[2] : cj[2] - t[2]};
                    shift_ref(E, d);
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            T.A[r][c] += E.A[r][c];
                            T.B[r][c] += E.B[r][c];
                            T.D[r][c] += E.D[r][c];
                        }
                }
                if (!world) {
                    float R[3][3];
                    quat_to_rot(q[0], q[1], q[2], q[3], R);
                    rotate_into(T, R);
                }
                float fim[21];
                pack(T, fim);
                const bool nan = (st & FIF_POSE_NAN) != 0;
                if (nan) {
#pragma unroll
                    for (int e = 0; e < 21; ++e) fim[e] = __int_as_float(0x7fc00000);
                }
                if (a.fim) {
#pragma unroll
                    for (int e = 0; e < 21; ++e) a.fim[p * 21 + e] = fim[e];
                }
                if (a.flags & FIF_Q_METRICS) {
                    if (a.flags & FIF_Q_TRACE) {
                        const double tr = nan ? (double)NAN : (double)trace6(fim);
                        if (a.metrics) a.metrics[p * 3 + 0] = tr;
                    }
                    if (a.flags & FIF_Q_LOGDET) {
                        double lad;
                        int sg;
                        logdet_f64(fim, lad, sg);
                        if (nan) { lad = NAN; sg = 0; }
                        if (a.metrics) a.metrics[p * 3 + 1] = lad;
                        if (a.sign) a.sign[p] = (int8_t)sg;
                        if (sg <= 0 && !nan) st |= FIF_POSE_NOT_PD;
                    }
                    if (a.flags & FIF_Q_LMIN) {
                        double lm = lambda_min_f64(fim);
                        if (nan) lm = NAN;
                        if (a.metrics) a.metrics[p * 3 + 2] = lm;
                        if (!(lm > 0.0) && !nan) st |= FIF_POSE_NOT_PD;
                    }
                }
                if (a.status) a.status[p] = (int32_t)st;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.eempty[b]);
        }
    }
}

}  // namespace

template <int G, int NB, bool kComp>
static int launch_gp_query_kc(const QueryArgs& a, const GqLayout& L, int sms, cudaStream_t stream) {
    auto kern = gp_query_kernel<G, NB, kComp>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total) != cudaSuccess)
        return FIF_ECUDA;
    const int64_t groups = (a.m + 31) / 32;
    const int64_t grid = std::min<int64_t>(groups, (int64_t)sms);
    if (grid <= 0) return FIF_OK;
    kern<<<(unsigned)grid, (kGqContract + kGqWeights + NB) * 32, L.total, stream>>>(a, L);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

template <int G, int NB>
static int launch_gp_query_nb(const QueryArgs& a, const GqLayout& L, int sms, cudaStream_t stream) {
    return (a.flags & FIF_Q_GP_COMPENSATED) ? launch_gp_query_kc<G, NB, true>(a, L, sms, stream)
                                            : launch_gp_query_kc<G, NB, false>(a, L, sms, stream);
}

template <int G>
static int launch_gp_query_g(const QueryArgs& a, cudaStream_t stream) {
    int dev = 0, sms = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // Up to 64 samples the per-pose metric work outweighs the gather: four table buffers and
    // four metric warps, if W fits in shared memory beside at least 3 ring stages.  Otherwise two
    // buffers; prefer W in shared memory (its reads sit on the weights warps' critical path),
    // then as many ring stages as fit (at least 2); without room for W, read it from global memory.
    GqLayout L;
    if constexpr (G < 3) {
        for (int stages = kGqMaxStages; stages >= 3; --stages) {
            L = gq_layout(a.stride, a.gp_rs, a.gp_ns, stages, 1, 4);
            if (L.total <= max_smem) return launch_gp_query_nb<G, 4>(a, L, sms, stream);
        }
    }
    bool found = false;
    for (int w_smem = 1; w_smem >= 0 && !found; --w_smem)
        for (int stages = kGqMaxStages; stages >= 2 && !found; --stages) {
            L = gq_layout(a.stride, a.gp_rs, a.gp_ns, stages, w_smem, 2);
            found = L.total <= max_smem;
        }
    if (!found) return FIF_ERANGE;
    return launch_gp_query_nb<G, 2>(a, L, sms, stream);
}

int launch_gp_query(const QueryArgs& a, cudaStream_t stream) {
    if (a.gp_ns < 1 || a.gp_ns > FIF_GP_MAX_SAMPLES || !a.gp_axes || !a.gp_wt || !a.gp_consts) return FIF_EINVAL;
    const int G = (a.gp_ns + 31) / 32;
    if (G == 1) return launch_gp_query_g<1>(a, stream);
    if (G == 2) return launch_gp_query_g<2>(a, stream);
    return launch_gp_query_g<3>(a, stream);
}

GpAuxLayout gp_aux_layout(int ns, int rs) {
    GpAuxLayout L;
    size_t off = 0;
    L.axes_f = off;  off = align_up(off + 16 * (size_t)ns, 256);
    L.axes_df = off; off = align_up(off + 32 * (size_t)ns, 256);
    L.wt = off;      off = align_up(off + 8 * (size_t)ns * rs, 256);
    L.consts = off;  off = align_up(off + 16 * 18, 256);
    L.total = off;
    return L;
}

}  // namespace fif
