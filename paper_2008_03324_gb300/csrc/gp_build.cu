// gp_build.cu -- Fisher Information Field with GP visibility (Sec. V-B-2 of the paper): the
// field build for sm_103a (the query is in gp_query.cu).
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
// Build (gp_build_kernel): one CTA per 4 x 2 x 2 brick of nodes, one warp per node.  The
// brick's candidate landmarks stream through a ring of shared-memory tiles (landmark_stream),
// refilled by a 17th warp as soon as every node warp has released a slot;
// each warp takes the exact single-precision shell decision for its node 32 landmarks at a
// time, compacts the in-shell ones (u, 1/n) into a list, and every lane then accumulates, for
// its sample axes g = lane + 32 k, the 15 moments
//   sum v_g u_a u_b,  sum v_g u_a u_b / n^2,  sum v_g u_a / n
// from which all 21 entries of D_g follow (|u| = 1: 1 - u_a^2 = u_b^2 + u_c^2).  When the last
// slot of 32 axes holds r <= 16 samples, it takes q = 32 / r landmarks per pass instead of one
// (lane l: axis 32 k + l mod r, landmark l / r), and the epilogue adds the q partial sums of an
// axis in a fixed order; at N_s = 70 this removes the 26 idle lanes of the third slot.  Blocks
// of about 128 pairs are summed in registers and merged into Kahan pairs in shared memory.
//
#include "fif_common.cuh"
#include "fif_internal.h"
#include "landmark_stream.cuh"
#include "bearing.cuh"

#include <cmath>
#include <cstring>

namespace fif {

namespace {

// ------------------------------------------------------------------------------------
// build
// ------------------------------------------------------------------------------------
constexpr int kGbWarps = 16;                   // a 4 x 2 x 2 brick of nodes, one warp each
constexpr int kGbThreads = kGbWarps * 32;
constexpr int kGbTile = 256;
constexpr int kGbSlots = 3;
constexpr int kGbBlock = 128;                  // pairs per register block (Kahan granularity)
constexpr int kGbMaxRuns = 2048;
constexpr int kGbMom = 15;

// a compacted in-shell landmark: the bearing u, 1/n and the products the 15 moments weight
// (u_a u_b, u_a u_b / n^2, u_a / n), formed once by the lane that found it instead of by all 32
// lanes of the node's warp
struct GbPair {
    float4 m01;     // x^2, y^2, z^2, x y
    float4 m2w0;    // x z, y z, x^2 / n^2, y^2 / n^2
    float4 w12;     // z^2 / n^2, x y / n^2, x z / n^2, y z / n^2
    float4 un;      // x / n, y / n, z / n, unused
    float4 u;       // x, y, z, 1 / n
};

template <int G>
struct GpBuildSmem {
    float hi[kGbWarps][kGbMom * G][32];
    // the Kahan compensation in bfloat16: it is below half an ulp of the sum, so its 8
    // significant bits extend the sum to about 32 (and halve the space of a float32 term)
    __nv_bfloat16 lo[kGbWarps][kGbMom * G][32];
    float4 tile[kGbSlots][kGbTile];
    GbPair list[kGbWarps][32];
    int2 runs[kGbMaxRuns];
    int tile_count[kGbSlots];
    int nruns;
    uint64_t full[kGbSlots];    // tile landed (producer arrival + copy bytes)
    uint64_t empty[kGbSlots];   // every node warp is done with the tile
};

FIF_DEV float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
FIF_DEV float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int G>
__global__ void __launch_bounds__(kGbThreads + 32, 1) gp_build_kernel(BuildArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    GpBuildSmem<G>& S = *reinterpret_cast<GpBuildSmem<G>*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    static_assert(kGpBuildBrickZ == 2, "a GP brick is 4 x 2 x 2 nodes");
    const int nbx = (a.nx + 3) / 4, nby = (a.ny + 1) / 2;
    const int brick = blockIdx.x + (a.k_begin / 2) * nbx * nby;   // z-bricks meeting the slab
    const int i0 = 4 * (brick % nbx), j0 = 2 * ((brick / nbx) % nby), k0 = 2 * (brick / (nbx * nby));
    const int ni = i0 + (warp & 3), nj = j0 + ((warp >> 2) & 1), nk = k0 + (warp >> 3);
    const bool producer = warp == kGbWarps;   // the 17th warp streams the landmark tiles
    const bool valid = !producer && ni < a.nx && nj < a.ny && nk < a.nz && nk >= a.k_begin && nk < a.k_end;
    const float cx = __fadd_rn(a.ox, __fmul_rn(a.res, (float)ni));
    const float cy = __fadd_rn(a.oy, __fmul_rn(a.res, (float)nj));
    const float cz = __fadd_rn(a.oz, __fmul_rn(a.res, (float)nk));
    const float blo[3] = {a.ox + a.res * i0, a.oy + a.res * j0, a.oz + a.res * k0};
    const float bhi[3] = {a.ox + a.res * min(i0 + 3, a.nx - 1), a.oy + a.res * min(j0 + 1, a.ny - 1),
                          a.oz + a.res * min(k0 + 1, a.nz - 1)};

    float* hs = &S.hi[0][0][0];
    __nv_bfloat16* ls = &S.lo[0][0][0];
    for (int idx = tid; idx < kGbWarps * kGbMom * G * 32; idx += kGbThreads + 32) {
        hs[idx] = 0.f;
        ls[idx] = __float2bfloat16_rn(0.f);
    }
    const int* startp = reinterpret_cast<const int*>(a.ws + a.lay.start);
    const int nrows =
        enumerate_runs(a.bg, startp, blo, bhi, a.rcull, S.runs, kGbMaxRuns, tid, kGbThreads + 32, a.err);
    if (tid == 0) {
        S.nruns = nrows;
        for (int s = 0; s < kGbSlots; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kGbWarps);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // producer warp (lane 0): refills a slot as soon as every node warp is done with it
    if (producer) {
        if (lane == 0) {
            const float4* sorted = reinterpret_cast<const float4*>(a.ws + a.lay.sorted);
            TileProducer<kGbTile> prod;
            for (int it = 0;; ++it) {
                const int slot = it % kGbSlots;
                if (it >= kGbSlots && !mbar_wait_bounded(&S.empty[slot], (uint32_t)((it / kGbSlots - 1) & 1), a.wait_ns)) {
                    set_error(a.err, FIF_ETIMEOUT);
                    drain_fills<kGbSlots>(S.full, it - kGbSlots, it);
                    break;
                }
                fence_proxy_async();   // the node warps' reads of the slot precede the new copies
                const int cnt = prod.fill(S.tile[slot], S.runs, S.nruns, sorted, &S.full[slot]);
                S.tile_count[slot] = cnt;
                mbar_arrive(&S.full[slot]);
                if (cnt == 0) {       // the end marker
                    drain_fills<kGbSlots>(S.full, it - kGbSlots + 1, it);
                    break;
                }
            }
        }
        return;
    }

    // samples in the last slot of 32 axes, and landmarks it takes per pass (lane l of that slot:
    // axis 32 (G - 1) + l mod rr, landmark l / rr of the pass; lanes with l / rr >= qq idle)
    const int rr = a.gp_ns - 32 * (G - 1);
    const int qq = (rr <= 16) ? 32 / rr : 1;
    const int jq = lane / rr;
    const bool main_slots = G > 1 || qq == 1;   // some slot takes one landmark per pass
    // this lane's sample axes, scaled and negated so that v = 1 / (1 + 2^(shift + nz.u))
    float nzx[G], nzy[G], nzz[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int g = (k == G - 1 && qq > 1) ? 32 * k + lane % rr : lane + 32 * k;
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g < a.gp_ns) z = a.gp_axes[g];
        nzx[k] = -z.x * a.gp_scale;
        nzy[k] = -z.y * a.gp_scale;
        nzz[k] = -z.z * a.gp_scale;
    }
    const float shift = a.gp_shift;
    // moment sums of the current block, packed in pairs of moments: (xx, yy) (zz, xy) (xz, yz),
    // the same over n^2, (x, y) / n, and z / n alone
    float2 acc[G][7];
    float accz[G];
#pragma unroll
    for (int k = 0; k < G; ++k) {
#pragma unroll
        for (int q = 0; q < 7; ++q) acc[k][q] = make_float2(0.f, 0.f);
        accz[k] = 0.f;
    }
    float* hw = hs + warp * kGbMom * G * 32 + lane;
    __nv_bfloat16* lw = ls + warp * kGbMom * G * 32 + lane;
    // Kahan step of a block sum x into (hi, compensation)
    auto kmerge = [&](int idx, float x) {
        const float s0 = hw[idx], c = __bfloat162float(lw[idx]);
        const float y = x - c;
        const float t = s0 + y;
        lw[idx] = __float2bfloat16_rn((t - s0) - y);
        hw[idx] = t;
    };
    auto merge = [&]() {
#pragma unroll
        for (int k = 0; k < G; ++k) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                kmerge((k * kGbMom + 2 * q) * 32, acc[k][q].x);
                kmerge((k * kGbMom + 2 * q + 1) * 32, acc[k][q].y);
                acc[k][q] = make_float2(0.f, 0.f);
            }
            kmerge((k * kGbMom + 14) * 32, accz[k]);
            accz[k] = 0.f;
        }
    };
    // v_g of the bearing (x, y, z) for every owned sample axis, two axes per packed step
    // (the last slot's value is unused when that slot runs in its own loop)
    auto sigmoids = [&](float x, float y, float z, float* v) {
#pragma unroll
        for (int k = 0; k + 1 < G; k += 2) {
            float2 arg = fma2(make_float2(nzx[k], nzx[k + 1]), make_float2(x, x),
                              fma2(make_float2(nzy[k], nzy[k + 1]), make_float2(y, y),
                                   fma2(make_float2(nzz[k], nzz[k + 1]), make_float2(z, z), make_float2(shift, shift))));
            const float2 E = make_float2(ex2_approx(fminf(arg.x, 60.f)), ex2_approx(fminf(arg.y, 60.f)));
            const float2 d = add2(E, make_float2(1.f, 1.f));
            v[k] = rcp_approx(d.x);
            v[k + 1] = rcp_approx(d.y);
        }
        if ((G & 1) && qq == 1) {
            const int k = G - 1;
            const float arg = fmaf(nzx[k], x, fmaf(nzy[k], y, fmaf(nzz[k], z, shift)));
            v[k] = rcp_approx(1.f + ex2_approx(fminf(arg, 60.f)));
        }
    };

    const float rmin2 = a.rmin2, rmax2 = a.rmax2;
    int inblock = 0;
    unsigned long long in_pairs = 0, cand = 0;
    bool ok = true;
    GbPair* list = S.list[warp];
    for (int it = 0;; ++it) {
        const int slot = it % kGbSlots;
        const uint32_t par = (uint32_t)((it / kGbSlots) & 1);
        if (__any_sync(0xffffffffu, !mbar_wait_bounded(&S.full[slot], par, a.wait_ns))) {   // the warp exits together
            ok = false;
            if (lane == 0) set_error(a.err, FIF_ETIMEOUT);
            break;
        }
        const int cnt = S.tile_count[slot];
        if (cnt == 0) break;
        const float4* tile = S.tile[slot];
        if (valid) {
            cand += cnt;
            for (int base = 0; base < cnt; base += 32) {
                bool in = false;
                float dx = 0.f, dy = 0.f, dz = 0.f, n2 = 1.f;
                if (base + lane < cnt) {
                    const float4 P = tile[base + lane];
                    dx = __fsub_rn(P.x, cx);
                    dy = __fsub_rn(P.y, cy);
                    dz = __fsub_rn(P.z, cz);
                    n2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                    in = (n2 > rmin2) && (n2 <= rmax2);
                }
                const unsigned mask = __ballot_sync(0xffffffffu, in);
                if (in) {
                    const float r = rsqrtf(n2);
                    const float x = dx * r, y = dy * r, z = dz * r, w2 = r * r;
                    GbPair& P = list[__popc(mask & ((1u << lane) - 1u))];
                    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
                    P.m01 = make_float4(xx, yy, zz, xy);
                    P.m2w0 = make_float4(xz, yz, xx * w2, yy * w2);
                    P.w12 = make_float4(zz * w2, xy * w2, xz * w2, yz * w2);
                    P.un = make_float4(x * r, y * r, z * r, 0.f);
                    P.u = make_float4(x, y, z, r);
                }
                __syncwarp();
                const int nin = __popc(mask);
#pragma unroll 2
                for (int l = 0; l < (main_slots ? nin : 0); ++l) {
                    const GbPair& P = list[l];
                    const float4 A = P.m01, Bq = P.m2w0, Cq = P.w12, D = P.un, U = P.u;
                    const float x = U.x, y = U.y, z = U.z;
                    const float2 X[7] = {make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(Bq.x, Bq.y),
                                         make_float2(Bq.z, Bq.w), make_float2(Cq.x, Cq.y), make_float2(Cq.z, Cq.w),
                                         make_float2(D.x, D.y)};
                    const float zi = D.z;
                    float v[G];
                    sigmoids(x, y, z, v);
#pragma unroll
                    for (int k = 0; k < G; ++k) {
                        if (k == G - 1 && qq > 1) break;
                        const float2 vv = make_float2(v[k], v[k]);
#pragma unroll
                        for (int q = 0; q < 7; ++q) acc[k][q] = fma2(vv, X[q], acc[k][q]);
                        accz[k] = fmaf(v[k], zi, accz[k]);
                    }
                }
                // the last slot, qq landmarks per pass
                if (qq > 1) {
                    constexpr int k = G - 1;
#pragma unroll 2
                    for (int l0 = 0; l0 < nin; l0 += qq) {
                        const int li = l0 + jq;
                        const bool act = jq < qq && li < nin;   // idle lanes add zero weights
                        {
                            const GbPair& P = list[act ? li : 0];
                            const float4 A = P.m01, Bq = P.m2w0, Cq = P.w12, D = P.un, U = P.u;
                            const float x = U.x, y = U.y, z = U.z;
                            const float2 X[7] = {make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(Bq.x, Bq.y),
                                                 make_float2(Bq.z, Bq.w), make_float2(Cq.x, Cq.y), make_float2(Cq.z, Cq.w),
                                                 make_float2(D.x, D.y)};
                            const float arg = fmaf(nzx[k], x, fmaf(nzy[k], y, fmaf(nzz[k], z, shift)));
                            const float vk = act ? rcp_approx(1.f + ex2_approx(fminf(arg, 60.f))) : 0.f;
                            const float2 vv = make_float2(vk, vk);
#pragma unroll
                            for (int q = 0; q < 7; ++q) acc[k][q] = fma2(vv, X[q], acc[k][q]);
                            accz[k] = fmaf(vk, D.z, accz[k]);
                        }
                    }
                }
                __syncwarp();
                in_pairs += nin;
                inblock += nin;
                if (inblock >= kGbBlock) {
                    merge();
                    inblock = 0;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[slot]);   // this warp is done with the slot
    }
    if (valid && inblock > 0) merge();
    __syncwarp();
    {
        unsigned long long* stats = reinterpret_cast<unsigned long long*>(a.ws + a.lay.stats);
        if (valid && lane == 0) {
            if (in_pairs) atomicAdd(&stats[0], in_pairs);
            if (cand) atomicAdd(&stats[1], cand);
        }
    }
    if (!valid) return;
    if (a.accumulate != 0 && in_pairs == 0) return;   // an update leaves unreached nodes untouched
    const int64_t node = ni + (int64_t)a.nx * (nj + (int64_t)a.ny * nk);
    float* out = reinterpret_cast<float*>(a.out) + node * a.stride;
    const int rs = a.gp_rs;
#pragma unroll
    for (int k = 0; k < G; ++k) {
        const int g = lane + 32 * k;
        if (g >= rs) continue;
        float mo[kGbMom];
        if (k == G - 1 && qq > 1) {
            // the qq partial sums of axis g (lanes j rr + lane), in lane order
#pragma unroll
            for (int m = 0; m < kGbMom; ++m) {
                float t = 0.f;
                if (lane < rr)
                    for (int j = 0; j < qq; ++j)
                        t += hw[(k * kGbMom + m) * 32 + j * rr] - __bfloat162float(lw[(k * kGbMom + m) * 32 + j * rr]);
                mo[m] = t;
            }
        } else {
#pragma unroll
            for (int m = 0; m < kGbMom; ++m) mo[m] = hw[(k * kGbMom + m) * 32] - __bfloat162float(lw[(k * kGbMom + m) * 32]);
        }
        const bool live = ok && g < a.gp_ns;
#pragma unroll
        for (int e = 0; e < 21; ++e) {
            float v = live ? bearing_entry(e, mo) * a.inv_sigma2 : 0.f;
            if (a.accumulate != 0) v = fmaf((float)a.accumulate, v, out[e * rs + g]);
            out[e * rs + g] = v;
        }
    }
    if (a.accumulate == 0)
        for (int idx = 21 * rs + lane; idx < a.stride; idx += 32) out[idx] = 0.f;
}

}  // namespace

template <int G>
static int launch_gp_build_g(const BuildArgs& a, cudaStream_t stream) {
    const int smem = (int)sizeof(GpBuildSmem<G>);
    if (cudaFuncSetAttribute(gp_build_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return FIF_ECUDA;
    const int64_t bricks = (int64_t)((a.nx + 3) / 4) * ((a.ny + 1) / 2) * ((a.k_end + 1) / 2 - a.k_begin / 2);
    if (bricks <= 0) return FIF_OK;
    if (bricks > (int64_t)INT32_MAX) return FIF_ERANGE;
    gp_build_kernel<G><<<(unsigned)bricks, kGbThreads + 32, smem, stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

int launch_gp_build(const BuildArgs& a, cudaStream_t stream) {
    if (a.gp_ns < 1 || a.gp_ns > FIF_GP_MAX_SAMPLES || !a.gp_axes) return FIF_EINVAL;
    const int rc = launch_binning(a, stream);
    if (rc != FIF_OK) return rc;
    const int G = (a.gp_ns + 31) / 32;
    if (G == 1) return launch_gp_build_g<1>(a, stream);
    if (G == 2) return launch_gp_build_g<2>(a, stream);
    return launch_gp_build_g<3>(a, stream);
}

}  // namespace fif
