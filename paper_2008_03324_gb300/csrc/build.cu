// build.cu -- Fisher Information Field build (sm_103a).
//
// Sec. VI-A-1 / Eq. general_info_pif of the paper: for every voxel node c
//   C_k(c) = sum_{i : r_min < |p_i - c| <= r_max} v_p(u_i)[k] I_i,   k = 0..9,
// with u_i the unit bearing from c to landmark i, v_p the monomials of
// Eq. quad_vis_component and I_i the rotation-invariant information of one bearing
// (Eq. global_fim_eq) taken about the node itself:
//   I_i = sigma^-2 [[P/n^2, -[u]x/n], [[u]x/n, P]],  P = I - u u^T,  n = |p_i - c|.
//
// Kernels
//  bin_*      counting sort of the landmarks into cubic bins (deterministic order inside a
//             bin: by input index), so a brick of nodes reads only the landmarks whose bins
//             come within r_max of it, as contiguous runs.
//  build      one CTA = a brick of 8 x 4 x 4 nodes, one thread = one register-resident
//             node.  A fifth warp streams the brick's candidate landmarks through a 3-slot
//             ring of shared-memory tiles with bulk copies (cp.async.bulk + full/empty
//             mbarriers); each node warp copies the landmarks near its 4 x 4 x 2 sub-brick into
//             its own list and its 32 node threads read each as a shared-memory broadcast.
//
// Arithmetic per (node, landmark): every entry of v_p[k] * I_i is a polynomial in u of
// degree <= 4 times 1/n^2, 1/n or 1.  Because |u| = 1, multiplying by (u.u)^m raises any
// term to degree 3 or 4 (2 or 3 for 1/n), so all 210 entries are fixed integer combinations
// of 66 moments
//   sum u^a / n^2 (|a| = 4, 3),  sum u^a / n (|a| = 3, 2),  sum u^a (|a| = 4, 3),
// and the hot loop accumulates only those 66.  Its arithmetic runs on packed f32x2 pairs whose
// halves are the same monomial with x and y exchanged ((x^3, y^3), (x^2 z, y^2 z), ...), so every
// packed operand comes out of an earlier packed result without register moves; the landmarks sit
// in shared memory as (x, y, z, z) to give (z, z) the same way.  The degree-4 moments are formed
// inside their accumulating FMA (a degree-3 monomial times one coordinate), so a pair costs 26
// products and 66 accumulations (46 FMA, 20 FADD) after the shell test and the bearing.
// Accumulation is compensated: a block of 128 pairs (carried across tiles) is summed in
// registers, then the block sum is added to a Kahan (sum, compensation) pair held in shared
// memory.  The epilogue expands the 66 moments into the 210 stored coefficients through the
// integer map above, enumerated at compile time.
#include "fif_common.cuh"
#include "fif_internal.h"
#include "landmark_stream.cuh"

#include <cmath>
#include <cstring>
#include <utility>

namespace fif {

namespace {

constexpr int kBX = 8, kBY = 4, kBZ = kBuildBrickZ;
constexpr int kThreads = kBX * kBY * kBZ;  // 128
constexpr int kTile = 256;                  // landmarks per tile
constexpr int kSlots = 3;
constexpr int kBlock = 128;                 // pairs per register block (Kahan granularity)
constexpr int kMaxRuns = 1536;
constexpr int kMom = 66;

// monomial exponent tables (order fixed by the hot loop: x/y-exchanged pairs, then the rest)
constexpr int8_t kMon2[6][3] = {{2, 0, 0}, {0, 2, 0}, {1, 0, 1}, {0, 1, 1}, {0, 0, 2}, {1, 1, 0}};
constexpr int8_t kMon3[10][3] = {{3, 0, 0}, {0, 3, 0}, {2, 0, 1}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {0, 0, 3},
                                 {2, 1, 0}, {1, 2, 0}, {1, 1, 1}};
constexpr int8_t kMon4[15][3] = {{4, 0, 0}, {0, 4, 0}, {3, 0, 1}, {0, 3, 1}, {2, 0, 2}, {0, 2, 2}, {1, 0, 3},
                                 {0, 1, 3}, {0, 0, 4}, {3, 1, 0}, {1, 3, 0}, {2, 2, 0}, {2, 1, 1}, {1, 2, 1},
                                 {1, 1, 2}};
// v_p monomials of Eq. quad_vis_component
constexpr int8_t kVp[10][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1},
                                             {0, 1, 1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 0, 0}};
// moment blocks: base index of (power of 1/n, degree)
constexpr int kS4n2 = 0, kS3n2 = 15, kS3n1 = 25, kS2n1 = 35, kS4n0 = 41, kS3n0 = 56;

// ------------------------------------------------------------------------------------
// binning
// ------------------------------------------------------------------------------------
__global__ void fill_i32_kernel(int* p, int64_t n, int v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__device__ __forceinline__ int bin_of(const BinGrid& bg, float x, float y, float z) {
    const int ix = (int)floorf((x - bg.lo[0]) * bg.inv_size);
    const int iy = (int)floorf((y - bg.lo[1]) * bg.inv_size);
    const int iz = (int)floorf((z - bg.lo[2]) * bg.inv_size);
    if (!(ix >= 0 && ix < bg.n[0] && iy >= 0 && iy < bg.n[1] && iz >= 0 && iz < bg.n[2])) return -1;
    return ix + bg.n[0] * (iy + bg.n[1] * iz);
}

__global__ void bin_count_kernel(const float* __restrict__ lm, int64_t n, BinGrid bg, int* __restrict__ binof,
                                  int* __restrict__ count, unsigned long long* __restrict__ stats) {
    int dropped = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = lm[3 * i], y = lm[3 * i + 1], z = lm[3 * i + 2];
        int b = (isfinite(x) && isfinite(y) && isfinite(z)) ? bin_of(bg, x, y, z) : -1;
        binof[i] = b;
        if (b >= 0) atomicAdd(&count[b], 1);
        else ++dropped;
    }
    if (dropped) atomicAdd(&stats[2], (unsigned long long)dropped);
}

// exclusive scan of count[0..nb) into start[0..nb], then count <- 0 (reused as cursor)
__global__ void __launch_bounds__(1024) bin_scan_kernel(int* __restrict__ count, int* __restrict__ start, int nb) {
    __shared__ int warp_sums[32];
    const int tid = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
    int local = 0;
    for (int b = b0; b < b1; ++b) local += count[b];
    // block-wide exclusive scan of `local`
    int v = local;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    int run = v - local + (warp > 0 ? warp_sums[warp - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        start[b] = run;
        run += count[b];
        count[b] = 0;
    }
    if (tid == 1023) start[nb] = run;
}

__global__ void bin_scatter_kernel(const float* __restrict__ lm, int64_t n, const int* __restrict__ binof,
                                   const int* __restrict__ start, int* __restrict__ cursor, float4* __restrict__ sorted) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = binof[i];
        if (b < 0) continue;
        const int pos = start[b] + atomicAdd(&cursor[b], 1);
        sorted[pos] = make_float4(lm[3 * i], lm[3 * i + 1], lm[3 * i + 2], __int_as_float((int)i));
    }
}

// insertion sort of every bin by input index (makes the summation order deterministic)
__global__ void bin_sort_kernel(float4* __restrict__ sorted, const int* __restrict__ start, int nb) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const int s = start[b], e = start[b + 1];
        for (int i = s + 1; i < e; ++i) {
            const float4 v = sorted[i];
            const int key = __float_as_int(v.w);
            int j = i - 1;
            while (j >= s && __float_as_int(sorted[j].w) > key) {
                sorted[j + 1] = sorted[j];
                --j;
            }
            sorted[j + 1] = v;
        }
        for (int i = s; i < e; ++i) sorted[i].w = sorted[i].z;   // (x, y, z, z): packed (z, z) loads
    }
}

// ------------------------------------------------------------------------------------
// the brick kernel
// ------------------------------------------------------------------------------------
struct BuildSmem {
    float hi[kMom][kThreads];
    float lo[kMom][kThreads];
    float4 tile[kSlots][kTile];
    int2 runs[kMaxRuns];
    int tile_count[kSlots];
    float4 keep[kThreads / 32][kTile];   // per-warp copies of the tile's landmarks near its sub-brick
    int nruns;
    uint64_t full[kSlots];    // tile landed (producer arrival + copy bytes)
    uint64_t empty[kSlots];   // every consumer warp is done with the tile
};

// ---- moments -> coefficients -----------------------------------------------------------
// Entry e (upper-triangular 6x6) of the node-local C_k is a fixed integer combination of the 66
// moments (before 1/sigma^2):
//   TT: (delta_rc - u_r u_c)/n^2,  TR: (-[u]x)_{r b}/n = eps_{r b l} u_l / n,  RR: delta_ab - u_a u_b,
// each times the monomial v_p[k](u), with monomials below the stored degrees raised by u.u = 1
// (one or two levels).  The combination is enumerated at compile time, so the epilogue is a
// short sum of register moments per coefficient.
struct CoefTerm {
    int8_t idx, w;   // moment index, integer weight
};
struct CoefRow {
    CoefTerm t[12];
    int n;
};
struct CoefTable {
    CoefRow row[210];   // o = 21 k + e
};

constexpr void add_stored(CoefRow& r, int p, int ex, int ey, int ez, int w) {
    const int deg = ex + ey + ez;
    int base = kS2n1, cnt = 6, idx = -1;
    if (deg == 4) { base = (p == 2) ? kS4n2 : kS4n0; cnt = 15; }
    else if (deg == 3) { base = (p == 2) ? kS3n2 : (p == 1) ? kS3n1 : kS3n0; cnt = 10; }
    for (int i = 0; i < cnt; ++i) {
        const int8_t* m = deg == 4 ? kMon4[i] : deg == 3 ? kMon3[i] : kMon2[i];
        if (m[0] == ex && m[1] == ey && m[2] == ez) idx = base + i;
    }
    for (int i = 0; i < r.n; ++i)
        if (r.t[i].idx == idx) {
            r.t[i].w = (int8_t)(r.t[i].w + w);
            return;
        }
    r.t[r.n].idx = (int8_t)idx;
    r.t[r.n].w = (int8_t)w;
    ++r.n;
}

// w * sum u^a / n^p for any |a| <= 4 (stored degrees: 4 and 3 for p = 0, 2; 3 and 2 for p = 1)
constexpr void add_moment(CoefRow& r, int p, int ex, int ey, int ez, int w) {
    const int top = (p == 1) ? 3 : 4;
    if (ex + ey + ez >= top - 1) {
        add_stored(r, p, ex, ey, ez, w);
        return;
    }
    for (int c = 0; c < 3; ++c) {
        const int a0 = ex + (c == 0 ? 2 : 0), a1 = ey + (c == 1 ? 2 : 0), a2 = ez + (c == 2 ? 2 : 0);
        if (a0 + a1 + a2 >= top - 1) {
            add_stored(r, p, a0, a1, a2, w);
        } else {
            for (int d = 0; d < 3; ++d)
                add_stored(r, p, a0 + (d == 0 ? 2 : 0), a1 + (d == 1 ? 2 : 0), a2 + (d == 2 ? 2 : 0), w);
        }
    }
}

constexpr CoefTable make_coef_table() {
    CoefTable T{};
    for (int k = 0; k < 10; ++k)
        for (int e = 0; e < 21; ++e) {
            CoefRow& row = T.row[21 * k + e];
            const int r = sym_row(e), c = sym_col(e);
            const int mx = kVp[k][0], my = kVp[k][1], mz = kVp[k][2];
            if (r < 3 && c < 3) {
                add_moment(row, 2, mx + (r == 0) + (c == 0), my + (r == 1) + (c == 1), mz + (r == 2) + (c == 2), -1);
                if (r == c) add_moment(row, 2, mx, my, mz, 1);
            } else if (r < 3) {
                const int b = c - 3;
                if (r != b) {
                    const int l = 3 - r - b;
                    add_moment(row, 1, mx + (l == 0), my + (l == 1), mz + (l == 2), ((r + 1) % 3 == b) ? 1 : -1);
                }
            } else {
                const int ra = r - 3, cb = c - 3;
                add_moment(row, 0, mx + (ra == 0) + (cb == 0), my + (ra == 1) + (cb == 1), mz + (ra == 2) + (cb == 2), -1);
                if (ra == cb) add_moment(row, 0, mx, my, mz, 1);
            }
            // drop cancelled terms
            int n = 0;
            for (int i = 0; i < row.n; ++i)
                if (row.t[i].w != 0) row.t[n++] = row.t[i];
            row.n = n;
        }
    return T;
}

constexpr CoefTable kCoefTable = make_coef_table();

// coefficient o (o >= 210: a zero pad) from the node's moments
template <int O>
FIF_DEV float coef_of(const float (&m)[kMom]) {
    if constexpr (O >= 210) {
        return 0.f;
    } else {
        constexpr CoefRow R = kCoefTable.row[O];
        float v = 0.f;
#pragma unroll
        for (int t = 0; t < R.n; ++t) v = fmaf((float)R.t[t].w, m[R.t[t].idx], v);
        return v;
    }
}

// float32 storage: float4 group G of the node record (stride 216 = 54 groups)
template <int... G>
FIF_DEV void store_f32(float4* dst, const float (&m)[kMom], float scale, int acc, std::integer_sequence<int, G...>) {
    auto one = [&](float4* d, float4 v) {
        if (acc != 0) {
            const float sgn = (float)acc;
            const float4 old = *d;
            v = make_float4(fmaf(sgn, v.x, old.x), fmaf(sgn, v.y, old.y), fmaf(sgn, v.z, old.z), fmaf(sgn, v.w, old.w));
        }
        *d = v;
    };
    (one(dst + G, make_float4(coef_of<4 * G>(m) * scale, coef_of<4 * G + 1>(m) * scale, coef_of<4 * G + 2>(m) * scale,
                              coef_of<4 * G + 3>(m) * scale)),
     ...);
}

// bfloat16 storage: element O of the node record (stride 224; monomial blocks of 22 elements,
// entry 21 of each block and elements 220..223 zero)
template <int O>
FIF_DEV float coef_bf16(const float (&m)[kMom]) {
    if constexpr (O >= 220 || O % 22 == 21) return 0.f;
    else return coef_of<(O / 22) * 21 + O % 22>(m);
}
template <int... O>
FIF_DEV void store_bf16(__nv_bfloat16* dst, const float (&m)[kMom], float scale, int acc,
                        std::integer_sequence<int, O...>) {
    auto one = [&](__nv_bfloat16* d, float v) {
        if (acc != 0) v = fmaf((float)acc, v, __bfloat162float(*d));
        *d = __float2bfloat16_rn(v);
    };
    (one(dst + O, coef_bf16<O>(m) * scale), ...);
}

// the 21 entries of C_k (times scale)
template <int K, int... E>
FIF_DEV void coefs_k(const float (&m)[kMom], float scale, float (&C)[21], std::integer_sequence<int, E...>) {
    ((C[E] = coef_of<21 * K + E>(m) * scale), ...);
}

// the paper's positional trace factor (Sec. VI-A-2): tr of the world-frame C_k,
//   tr(M_c^T C M_c) = tr(A) + tr(D) + |c|^2 tr(A) - c^T A c + 2 tr([c]x B)
template <int K>
FIF_DEV float trace_k(const float (&m)[kMom], float scale, float cx, float cy, float cz) {
    float C[21];
    coefs_k<K>(m, scale, C, std::make_integer_sequence<int, 21>{});
    float A[3][3], Bm[3][3], trD = 0.f;
#pragma unroll
    for (int e = 0; e < 21; ++e) {
        const int r = sym_row(e), c = sym_col(e);
        if (r < 3 && c < 3) { A[r][c] = C[e]; A[c][r] = C[e]; }
        else if (r < 3) Bm[r][c - 3] = C[e];
        else if (r == c) trD += C[e];
    }
    const float c3[3] = {cx, cy, cz};
    const float cc = cx * cx + cy * cy + cz * cz;
    const float trA = A[0][0] + A[1][1] + A[2][2];
    float cAc = 0.f, cxB = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) cAc += c3[r] * A[r][c] * c3[c];
    // [c]x = [[0, -cz, cy], [cz, 0, -cx], [-cy, cx, 0]];  tr([c]x B) = sum_ij [c]x_ij B_ji
    const float S[3][3] = {{0.f, -cz, cy}, {cz, 0.f, -cx}, {-cy, cx, 0.f}};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) cxB += S[r][c] * Bm[c][r];
    return trA + trD + cc * trA - cAc + 2.f * cxB;
}

template <int... K>
FIF_DEV void traces(const float (&m)[kMom], float scale, float cx, float cy, float cz, float (&out)[10],
                    std::integer_sequence<int, K...>) {
    ((out[K] = trace_k<K>(m, scale, cx, cy, cz)), ...);
}

__global__ void __launch_bounds__(kThreads + 32, 2) build_kernel(BuildArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BuildSmem& S = *reinterpret_cast<BuildSmem*>(smem_raw);
    const int tid = threadIdx.x;

    // brick of nodes
    const int nbx = (a.nx + kBX - 1) / kBX, nby = (a.ny + kBY - 1) / kBY;
    // the launch covers the z-bricks that meet the slab [k_begin, k_end)
    const int brick = blockIdx.x + (a.k_begin / kBZ) * nbx * nby;
    const int bxi = brick % nbx, byi = (brick / nbx) % nby, bzi = brick / (nbx * nby);
    const int i0 = bxi * kBX, j0 = byi * kBY, k0 = bzi * kBZ;
    // consumer warp w < 4 owns the 4 x 4 x 2 sub-brick at x offset 4 (w & 1), z offset 2 (w >> 1);
    // warp 4 streams the landmark tiles
    const int warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == kThreads / 32;
    const int ti = 4 * (warp & 1) + (lane & 3), tj = (lane >> 2) & 3, tk = 2 * (warp >> 1) + (lane >> 4);
    const int ni = i0 + ti, nj = j0 + tj, nk = k0 + tk;
    // nodes of the brick outside the slab run along (their warp's culling box is the full
    // build's, so every node in the slab sees exactly the full build's arithmetic) but write nothing
    const bool valid = !producer && ni < a.nx && nj < a.ny && nk < a.nz && nk >= a.k_begin && nk < a.k_end;
    const float cx = __fadd_rn(a.ox, __fmul_rn(a.res, (float)ni));
    const float cy = __fadd_rn(a.oy, __fmul_rn(a.res, (float)nj));
    const float cz = __fadd_rn(a.oz, __fmul_rn(a.res, (float)nk));
    // brick box over its valid nodes
    const float blo[3] = {a.ox + a.res * i0, a.oy + a.res * j0, a.oz + a.res * k0};
    const float bhi[3] = {a.ox + a.res * min(i0 + kBX - 1, a.nx - 1), a.oy + a.res * min(j0 + kBY - 1, a.ny - 1),
                          a.oz + a.res * min(k0 + kBZ - 1, a.nz - 1)};

    // this warp's sub-brick box (its valid nodes); a landmark farther than r_cull from it is
    // outside every shell of the warp's nodes
    const int wi0 = i0 + 4 * (warp & 1), wk0 = k0 + 2 * (warp >> 1);
    const float wlo[3] = {a.ox + a.res * min(wi0, a.nx - 1), a.oy + a.res * j0, a.oz + a.res * min(wk0, a.nz - 1)};
    const float whi[3] = {a.ox + a.res * min(wi0 + 3, a.nx - 1), a.oy + a.res * min(j0 + kBY - 1, a.ny - 1),
                          a.oz + a.res * min(wk0 + 1, a.nz - 1)};

    for (int idx = tid; idx < kMom * kThreads; idx += kThreads + 32) {
        (&S.hi[0][0])[idx] = 0.f;
        (&S.lo[0][0])[idx] = 0.f;
    }

    // ---- enumerate candidate runs: one bin row (y, z) per entry ----
    const BinGrid& bg = a.bg;
    const float rc = a.rcull, rc2 = rc * rc;
    const int* startp = reinterpret_cast<const int*>(a.ws + a.lay.start);
    const int nrows = enumerate_runs(bg, startp, blo, bhi, rc, S.runs, kMaxRuns, tid, kThreads + 32, a.err);
    if (tid == 0) {
        S.nruns = nrows;
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], kThreads / 32);
        }
        fence_mbar_init();
    }
    __syncthreads();

    // ---- producer warp (lane 0): refills a slot as soon as every consumer warp is done with it,
    // so the consumer warps drift apart by up to kSlots tiles instead of meeting at a barrier ----
    if (producer) {
        if (lane == 0) {
            const float4* sorted = reinterpret_cast<const float4*>(a.ws + a.lay.sorted);
            TileProducer<kTile> prod;
            for (int it = 0;; ++it) {
                const int slot = it % kSlots;
                if (it >= kSlots && !mbar_wait_bounded(&S.empty[slot], (uint32_t)((it / kSlots - 1) & 1), a.wait_ns)) {
                    set_error(a.err, FIF_ETIMEOUT);
                    drain_fills<kSlots>(S.full, it - kSlots, it);
                    break;
                }
                fence_proxy_async();   // the consumers' reads of the slot precede the new copies
                const int cnt = prod.fill(S.tile[slot], S.runs, S.nruns, sorted, &S.full[slot]);
                S.tile_count[slot] = cnt;
                mbar_arrive(&S.full[slot]);
                if (cnt == 0) {       // the end marker
                    drain_fills<kSlots>(S.full, it - kSlots + 1, it);
                    break;
                }
            }
        }
        return;
    }

    // ---- consume ----
    const float rmin2 = a.rmin2, rmax2 = a.rmax2;
    const float2 cxy = make_float2(cx, cy), czz = make_float2(cz, cz);
    // register block of the 66 moment sums in the moment order of the tables above: per group the
    // packed pairs (x-half, y-half of a monomial pair) first, then the single moments
    float2 p4n2[4], p3n2[3], p3n1[3], p2n1[2], p4n0[4], p3n0[3];
    float s4n2[7], s3n2[4], s3n1[4], s2n1[2], s4n0[7], s3n0[4];
    auto zero_block = [&]() {
#pragma unroll
        for (int i = 0; i < 4; ++i) p4n2[i] = p4n0[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 3; ++i) p3n2[i] = p3n1[i] = p3n0[i] = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < 2; ++i) { p2n1[i] = make_float2(0.f, 0.f); s2n1[i] = 0.f; }
#pragma unroll
        for (int i = 0; i < 7; ++i) s4n2[i] = s4n0[i] = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) s3n2[i] = s3n1[i] = s3n0[i] = 0.f;
    };
    zero_block();
    float* hs = &S.hi[0][0];
    float* ls = &S.lo[0][0];
    // compensated merge of the register block into the shared Kahan pairs (moment order)
    auto merge_block = [&]() {
        auto merge = [&](int base, const float2* p, int np, const float* sv, int ns) {
#pragma unroll
            for (int i = 0; i < np; ++i) {
                kahan_merge(hs, ls, (base + 2 * i) * kThreads + tid, p[i].x);
                kahan_merge(hs, ls, (base + 2 * i + 1) * kThreads + tid, p[i].y);
            }
#pragma unroll
            for (int i = 0; i < ns; ++i) kahan_merge(hs, ls, (base + 2 * np + i) * kThreads + tid, sv[i]);
        };
        merge(kS4n2, p4n2, 4, s4n2, 7);
        merge(kS3n2, p3n2, 3, s3n2, 4);
        merge(kS3n1, p3n1, 3, s3n1, 4);
        merge(kS2n1, p2n1, 2, s2n1, 2);
        merge(kS4n0, p4n0, 4, s4n0, 7);
        merge(kS3n0, p3n0, 3, s3n0, 4);
        zero_block();
    };
    int blk = 0;   // pairs in the register block (warp-uniform); the block spans tiles
    unsigned int in_pairs = 0;
    unsigned long long cand = 0;
    bool ok = true;
    for (int it = 0;; ++it) {
        const int slot = it % kSlots;
        const uint32_t par = (uint32_t)((it / kSlots) & 1);
        if (__any_sync(0xffffffffu, !mbar_wait_bounded(&S.full[slot], par, a.wait_ns))) {  // the warp exits together
            ok = false;
            if (lane == 0) set_error(a.err, FIF_ETIMEOUT);
            break;
        }
        const int cnt = S.tile_count[slot];
        if (cnt == 0) break;
        const float4* tile = S.tile[slot];
        // exact culling against this warp's sub-brick, compacted in tile order
        float4* keep = S.keep[warp];
        int nkeep = 0;
        for (int base = 0; base < cnt; base += 32) {
            bool near = false;
            float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
            if (base + lane < cnt) {
                P = tile[base + lane];
                const float ex = fmaxf(0.f, fmaxf(wlo[0] - P.x, P.x - whi[0]));
                const float ey = fmaxf(0.f, fmaxf(wlo[1] - P.y, P.y - whi[1]));
                const float ez = fmaxf(0.f, fmaxf(wlo[2] - P.z, P.z - whi[2]));
                near = ex * ex + ey * ey + ez * ez <= rc2;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, near);
            if (near) keep[nkeep + __popc(mask & ((1u << lane) - 1u))] = P;
            nkeep += __popc(mask);
        }
        __syncwarp();
        cand += nkeep;
        for (int b0 = 0; b0 < nkeep;) {
            const int b1 = min(nkeep, b0 + (kBlock - blk));
            blk += b1 - b0;
#pragma unroll 4
            for (int l = b0; l < b1; ++l) {
                const float4 L = keep[l];   // (x, y, z, z)
                // the shell test in rounded single precision, one operation at a time
                const float2 dxy = sub2(make_float2(L.x, L.y), cxy);
                const float2 dzz = sub2(make_float2(L.z, L.w), czz);
                const float dx = dxy.x, dy = dxy.y, dz = dzz.x;
                const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
                const bool in = (n2 > rmin2) && (n2 <= rmax2);
                in_pairs += in ? 1u : 0u;
                const float r = rsqrtf(n2);
                const float inv_n = in ? r : 0.f;
                const float2 rr = make_float2(inv_n, inv_n);
                // bearing u = (x, y, z) and w = 1/n^2; the x and y halves of the packed pairs are
                // monomials that differ by exchanging x and y
                const float2 P1 = mul2(dxy, rr);            // (x, y)
                const float2 Z1 = mul2(dzz, rr);            // (z, z)
                const float2 W = mul2(rr, rr);              // (w, w)
                const float x = P1.x, y = P1.y, z = Z1.x, w = W.x;
                const float2 P2 = mul2(P1, P1);             // x^2, y^2
                const float2 PZ = mul2(P1, Z1);             // xz, yz
                const float2 P3 = mul2(P2, P1);             // x^3, y^3
                const float2 P2Z = mul2(P2, Z1);            // x^2 z, y^2 z
                const float2 PZ2 = mul2(PZ, Z1);            // x z^2, y z^2
                const float z2 = z * z, xy = x * y;
                const float z3 = z2 * z, x2y = P2.x * y, xy2 = x * P2.y, xyz = xy * z;
                // degree 3 over n^2 (the degree-4 moments over n^2 are these times one coordinate)
                const float2 V3 = mul2(P3, W), V2Z = mul2(P2Z, W), VZ2 = mul2(PZ2, W);
                const float z3w = z3 * w, x2yw = x2y * w, xy2w = xy2 * w, xyzw = xyz * w;
                // sum u^a / n^2, |a| = 4: x^4 y^4 | x^3z y^3z | x^2z^2 y^2z^2 | xz^3 yz^3 ; z^4 x^3y xy^3 x^2y^2 x^2yz xy^2z xyz^2
                p4n2[0] = fma2(V3, P1, p4n2[0]);
                p4n2[1] = fma2(V3, Z1, p4n2[1]);
                p4n2[2] = fma2(V2Z, Z1, p4n2[2]);
                p4n2[3] = fma2(VZ2, Z1, p4n2[3]);
                s4n2[0] = fmaf(z3w, z, s4n2[0]);
                s4n2[1] = fmaf(V3.x, y, s4n2[1]);
                s4n2[2] = fmaf(x, V3.y, s4n2[2]);
                s4n2[3] = fmaf(x2yw, y, s4n2[3]);
                s4n2[4] = fmaf(x2yw, z, s4n2[4]);
                s4n2[5] = fmaf(xy2w, z, s4n2[5]);
                s4n2[6] = fmaf(xyzw, z, s4n2[6]);
                // sum u^a / n^2, |a| = 3: x^3 y^3 | x^2z y^2z | xz^2 yz^2 ; z^3 x^2y xy^2 xyz
                p3n2[0] = add2(p3n2[0], V3);
                p3n2[1] = add2(p3n2[1], V2Z);
                p3n2[2] = add2(p3n2[2], VZ2);
                s3n2[0] += z3w;
                s3n2[1] += x2yw;
                s3n2[2] += xy2w;
                s3n2[3] += xyzw;
                // sum u^a / n, |a| = 3 (same order)
                p3n1[0] = fma2(P3, rr, p3n1[0]);
                p3n1[1] = fma2(P2Z, rr, p3n1[1]);
                p3n1[2] = fma2(PZ2, rr, p3n1[2]);
                s3n1[0] = fmaf(z3, inv_n, s3n1[0]);
                s3n1[1] = fmaf(x2y, inv_n, s3n1[1]);
                s3n1[2] = fmaf(xy2, inv_n, s3n1[2]);
                s3n1[3] = fmaf(xyz, inv_n, s3n1[3]);
                // sum u^a / n, |a| = 2: x^2 y^2 | xz yz ; z^2 xy
                p2n1[0] = fma2(P2, rr, p2n1[0]);
                p2n1[1] = fma2(PZ, rr, p2n1[1]);
                s2n1[0] = fmaf(z2, inv_n, s2n1[0]);
                s2n1[1] = fmaf(xy, inv_n, s2n1[1]);
                // sum u^a, |a| = 4 (order of the n^2 group)
                p4n0[0] = fma2(P3, P1, p4n0[0]);
                p4n0[1] = fma2(P3, Z1, p4n0[1]);
                p4n0[2] = fma2(P2Z, Z1, p4n0[2]);
                p4n0[3] = fma2(PZ2, Z1, p4n0[3]);
                s4n0[0] = fmaf(z3, z, s4n0[0]);
                s4n0[1] = fmaf(P3.x, y, s4n0[1]);
                s4n0[2] = fmaf(x, P3.y, s4n0[2]);
                s4n0[3] = fmaf(x2y, y, s4n0[3]);
                s4n0[4] = fmaf(x2y, z, s4n0[4]);
                s4n0[5] = fmaf(xy2, z, s4n0[5]);
                s4n0[6] = fmaf(xyz, z, s4n0[6]);
                // sum u^a, |a| = 3
                p3n0[0] = add2(p3n0[0], P3);
                p3n0[1] = add2(p3n0[1], P2Z);
                p3n0[2] = add2(p3n0[2], PZ2);
                s3n0[0] += z3;
                s3n0[1] += x2y;
                s3n0[2] += xy2;
                s3n0[3] += xyz;
            }
            b0 = b1;
            if (blk == kBlock) {
                merge_block();
                blk = 0;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.empty[slot]);   // this warp is done with the slot
    }
    if (blk > 0) merge_block();
    // statistics
    {
        unsigned long long* stats = reinterpret_cast<unsigned long long*>(a.ws + a.lay.stats);
        unsigned long long v = valid ? in_pairs : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0 && v) atomicAdd(&stats[0], v);
        const unsigned long long nv = __popc(__ballot_sync(0xffffffffu, valid));
        if (lane == 0) atomicAdd(&stats[1], cand * nv);
    }
    if (!valid) return;
    // an update leaves nodes that no landmark of the delta reaches untouched
    if (a.accumulate != 0 && cand == 0) return;
    // ---- epilogue: 66 moments -> 210 coefficients (times 1/sigma^2) ----
    const int64_t node = ni + (int64_t)a.nx * (nj + (int64_t)a.ny * nk);
    float m[kMom];
#pragma unroll
    for (int i = 0; i < kMom; ++i) m[i] = ok ? hs[i * kThreads + tid] - ls[i * kThreads + tid] : 0.f;
    if (a.storage == FIF_STORAGE_TRACE) {
        float* dst = reinterpret_cast<float*>(a.out) + node * a.stride;
        float tr[10];
        traces(m, a.inv_sigma2, cx, cy, cz, tr, std::make_integer_sequence<int, 10>{});
        for (int k = 0; k < 10; ++k) dst[k] = a.accumulate != 0 ? fmaf((float)a.accumulate, tr[k], dst[k]) : tr[k];
        for (int k = 10; k < a.stride; ++k) dst[k] = 0.f;
    } else if (a.storage == FIF_STORAGE_F32) {
        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(a.out) + node * a.stride);
        store_f32(dst, m, a.inv_sigma2, a.accumulate, std::make_integer_sequence<int, 216 / 4>{});
    } else {
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(a.out) + node * a.stride;
        store_bf16(dst, m, a.inv_sigma2, a.accumulate, std::make_integer_sequence<int, 224>{});
    }
}

}  // namespace

BinGrid make_bin_grid(const fif_field* f) {
    BinGrid bg;
    const double rmax = f->params.r_max;
    double size = f->params.bin_size > 0 ? f->params.bin_size : 1.0;
    const double res = f->grid.res;
    const int dims[3] = {f->grid.nx, f->grid.ny, f->grid.nz};
    // rows of bins a brick can touch must fit the run table
    const double ext = res * (std::max(kBY, kBZ) - 1) + 2.0 * (rmax + 0.02 + 1e-4 * rmax);
    const double min_size = ext / (std::sqrt((double)kMaxRuns) - 2.0);
    if (size < min_size) size = min_size;
    bg.size = (float)size;
    bg.inv_size = (float)(1.0 / size);
    for (int a = 0; a < 3; ++a) {
        const double lo = (double)f->grid.origin[a] - rmax - size;
        const double hi = (double)f->grid.origin[a] + res * (dims[a] - 1) + rmax + size;
        bg.lo[a] = (float)lo;
        bg.n[a] = (int)std::ceil((hi - lo) / size) + 1;
    }
    return bg;
}

BuildLayout build_layout(const BinGrid& bg, int64_t n) {
    BuildLayout L;
    const int64_t nb = (int64_t)bg.n[0] * bg.n[1] * bg.n[2];
    size_t off = 0;
    L.sorted = off; off = align_up(off + sizeof(float4) * (size_t)std::max<int64_t>(n, 1), 256);
    L.binof = off;  off = align_up(off + sizeof(int) * (size_t)std::max<int64_t>(n, 1), 256);
    L.count = off;  off = align_up(off + sizeof(int) * (size_t)nb, 256);
    L.start = off;  off = align_up(off + sizeof(int) * (size_t)(nb + 1), 256);
    L.stats = off;  off = align_up(off + 4 * sizeof(unsigned long long), 256);
    L.total = off;
    return L;
}

int launch_binning(const BuildArgs& a, cudaStream_t stream) {
    const int64_t nb = (int64_t)a.bg.n[0] * a.bg.n[1] * a.bg.n[2];
    if (nb > (int64_t)INT32_MAX - 1 || a.n > (int64_t)INT32_MAX) return FIF_ERANGE;
    int* count = reinterpret_cast<int*>(a.ws + a.lay.count);
    int* start = reinterpret_cast<int*>(a.ws + a.lay.start);
    int* binof = reinterpret_cast<int*>(a.ws + a.lay.binof);
    float4* sorted = reinterpret_cast<float4*>(a.ws + a.lay.sorted);
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(a.ws + a.lay.stats);
    const int T = 256;
    auto blocks = [&](int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + T - 1) / T, 152 * 32)); };
    fill_i32_kernel<<<blocks(nb), T, 0, stream>>>(count, nb, 0);
    fill_i32_kernel<<<1, 32, 0, stream>>>(reinterpret_cast<int*>(stats), 8, 0);
    if (a.n > 0) bin_count_kernel<<<blocks(a.n), T, 0, stream>>>(a.landmarks, a.n, a.bg, binof, count, stats);
    bin_scan_kernel<<<1, 1024, 0, stream>>>(count, start, (int)nb);
    if (a.n > 0) {
        bin_scatter_kernel<<<blocks(a.n), T, 0, stream>>>(a.landmarks, a.n, binof, start, count, sorted);
        bin_sort_kernel<<<blocks(nb), T, 0, stream>>>(sorted, start, (int)nb);
    }
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

int launch_build(const BuildArgs& a, cudaStream_t stream) {
    if (a.storage == FIF_STORAGE_GP) return launch_gp_build(a, stream);
    const int rc = launch_binning(a, stream);
    if (rc != FIF_OK) return rc;
    const int smem = (int)sizeof(BuildSmem);
    if (cudaFuncSetAttribute(build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return FIF_ECUDA;
    const int bz0 = a.k_begin / kBZ, bz1 = (a.k_end + kBZ - 1) / kBZ;
    const int64_t bricks = (int64_t)((a.nx + kBX - 1) / kBX) * ((a.ny + kBY - 1) / kBY) * (bz1 - bz0);
    if (bricks <= 0) return FIF_OK;
    if (bricks > (int64_t)INT32_MAX) return FIF_ERANGE;
    build_kernel<<<(unsigned)bricks, kThreads + 32, smem, stream>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}

}  // namespace fif
