// fif_common.cuh -- device helpers shared by the FIF kernels (sm_103a).
//
// Contents: inline-PTX wrappers for the bulk-copy engine (cp.async.bulk + mbarrier) with
// bounded waits, the packed symmetric 6x6 algebra, the quadratic-visibility monomials, and
// the information metrics (Sec. IV of the paper: trace, determinant, smallest eigenvalue).
#pragma once

#include <cstring>

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "../../include/fif.h"

#define FIF_DEV __device__ __forceinline__

namespace fif {

// ------------------------------------------------------------------------------------
// packed symmetric 6x6: 21 upper-triangular entries, row-major
// ------------------------------------------------------------------------------------
__host__ __device__ constexpr int sym_idx(int r, int c) {
    return (r <= c) ? (r * 6 - (r * (r - 1)) / 2 + (c - r)) : (c * 6 - (c * (c - 1)) / 2 + (r - c));
}
__host__ __device__ constexpr int sym_row(int e) {
    return e < 6 ? 0 : e < 11 ? 1 : e < 15 ? 2 : e < 18 ? 3 : e < 20 ? 4 : 5;
}
__host__ __device__ constexpr int sym_col(int e) {
    return e - sym_idx(sym_row(e), sym_row(e)) + sym_row(e);
}

// 3x3 blocks of a symmetric 6x6 S = [[A, B], [B^T, D]]
struct Blocks {
    float A[3][3];  // symmetric
    float B[3][3];
    float D[3][3];  // symmetric
};

FIF_DEV void unpack(const float* s, Blocks& b) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            b.A[r][c] = s[sym_idx(r, c)];
            b.B[r][c] = s[sym_idx(r, 3 + c)];
            b.D[r][c] = s[sym_idx(3 + r, 3 + c)];
        }
}

FIF_DEV void pack(const Blocks& b, float* s) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            s[sym_idx(r, c)] = b.A[r][c];
            s[sym_idx(3 + r, 3 + c)] = b.D[r][c];
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) s[sym_idx(r, 3 + c)] = b.B[r][c];
}

// X = -[a]x
FIF_DEV void neg_skew(const float a[3], float X[3][3]) {
    X[0][0] = 0.f;   X[0][1] = a[2];  X[0][2] = -a[1];
    X[1][0] = -a[2]; X[1][1] = 0.f;   X[1][2] = a[0];
    X[2][0] = a[1];  X[2][1] = -a[0]; X[2][2] = 0.f;
}

// S <- M_a^T S M_a with M_a = [[I, X], [0, I]], X = -[a]x:
//   A' = A, B' = A X + B, D' = X^T A X + X^T B + B^T X + D
// (moves the rotational reference point of a 6x6 information by a).
FIF_DEV void shift_ref(Blocks& s, const float a[3]) {
    float X[3][3];
    neg_skew(a, X);
    float AX[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) AX[r][c] = s.A[r][0] * X[0][c] + s.A[r][1] * X[1][c] + s.A[r][2] * X[2][c];
    float Bn[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) Bn[r][c] = AX[r][c] + s.B[r][c];
    // D' = X^T (A X + B) + B^T X + D = X^T Bn + B^T X + D
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = s.D[r][c];
#pragma unroll
            for (int l = 0; l < 3; ++l) v += X[l][r] * Bn[l][c] + s.B[l][r] * X[l][c];
            s.D[r][c] = v;
        }
    // symmetrise D exactly
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r + 1; c < 3; ++c) {
            float v = 0.5f * (s.D[r][c] + s.D[c][r]);
            s.D[r][c] = v;
            s.D[c][r] = v;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) s.B[r][c] = Bn[r][c];
}

// S <- blkdiag(R^T, R^T) S blkdiag(R, R)
FIF_DEV void rotate_into(Blocks& s, const float R[3][3]) {
    auto conj = [&](float M[3][3]) {
        float T[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) T[r][c] = M[r][0] * R[0][c] + M[r][1] * R[1][c] + M[r][2] * R[2][c];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) M[r][c] = R[0][r] * T[0][c] + R[1][r] * T[1][c] + R[2][r] * T[2][c];
    };
    conj(s.A);
    conj(s.B);
    conj(s.D);
}

// ------------------------------------------------------------------------------------
// rotation from a quaternion (w, x, y, z) -> R_wc; returns |q|^2
// ------------------------------------------------------------------------------------
FIF_DEV float quat_to_rot(float qw, float qx, float qy, float qz, float R[3][3]) {
    float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    float inv = rsqrtf(n2);
    float w = qw * inv, x = qx * inv, y = qy * inv, z = qz * inv;
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z);       R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z);       R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y);       R[2][1] = 2.f * (y * z + w * x);       R[2][2] = 1.f - 2.f * (x * x + y * y);
    return n2;
}

// v_r of Eq. quad_vis_component from the optical axis z = R e3
FIF_DEV void vis_vr(const float z[3], float k0, float k1, float k2, float vr[10]) {
    vr[0] = k2 * z[0] * z[0];
    vr[1] = k2 * z[1] * z[1];
    vr[2] = k2 * z[2] * z[2];
    vr[3] = 2.f * k2 * z[0] * z[1];
    vr[4] = 2.f * k2 * z[0] * z[2];
    vr[5] = 2.f * k2 * z[1] * z[2];
    vr[6] = k1 * z[0];
    vr[7] = k1 * z[1];
    vr[8] = k1 * z[2];
    vr[9] = k0;
}

// ------------------------------------------------------------------------------------
// metrics
// ------------------------------------------------------------------------------------

// log|det| and sign of a symmetric 6x6 (packed, float) by double-precision LU with partial
// pivoting; the row exchange is done with selects so the matrix stays in registers.
FIF_DEV void logdet_f64(const float* s, double& logabs, int& sign) {
    double a[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) a[r][c] = (double)s[sym_idx(r, c)];
    double prod = 1.0;
    int sg = 1;
    bool zero = false;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        // pivot search over rows c..5 (on single-precision magnitudes: the choice only
        // affects stability, and the comparisons stay off the slow double-precision pipe)
        int p = c;
        float best = fabsf((float)a[c][c]);
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (r <= c) continue;
            const float v = fabsf((float)a[r][c]);
            if (v > best) { best = v; p = r; }
        }
        // exchange rows c and p with selects
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (r <= c) continue;
            const bool sw = (r == p);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const double x = a[c][j], y = a[r][j];
                a[c][j] = sw ? y : x;
                a[r][j] = sw ? x : y;
            }
        }
        if (p != c) sg = -sg;
        const double piv = a[c][c];
        if (piv == 0.0) zero = true;
        const double inv = 1.0 / piv;
        prod *= piv;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (r <= c) continue;
            const double f = a[r][c] * inv;
#pragma unroll
            for (int j = 0; j < 6; ++j) a[r][j] = (j > c) ? fma(-f, a[c][j], a[r][j]) : a[r][j];
        }
    }
    if (zero || !(prod == prod)) {
        logabs = zero ? -INFINITY : (double)NAN;
        sign = 0;
        return;
    }
    if (prod < 0) { sg = -sg; prod = -prod; }
    logabs = log(prod);
    sign = sg;
}

// ---- smallest eigenvalue ------------------------------------------------------------
// Jacobi rotation (t = tan, c = cos, s = sin) that zeroes a_pq of a symmetric 2x2 block,
// with the convention a'_rp = c a_rp - s a_rq, a'_rq = s a_rp + c a_rq.  Fast intrinsics:
// the angle only has to reduce the off-diagonal mass, not be correctly rounded.
FIF_DEV void jacobi_angle(float app, float aqq, float apq, float& t, float& c, float& s) {
    const float theta = __fdividef(aqq - app, 2.f * apq);
    const float h = fmaf(theta, theta, 1.f);
    const float root = h * rsqrtf(h);
    float tt = copysignf(__fdividef(1.f, fabsf(theta) + root), theta);
    const bool skip = !(fabsf(apq) > 1e-30f * (fabsf(app) + fabsf(aqq))) || !isfinite(tt);
    tt = skip ? 0.f : tt;
    t = tt;
    c = rsqrtf(fmaf(tt, tt, 1.f));
    s = tt * c;
}

// One round of the parallel (Brent-Luk) ordering for n = 6: three rotations on disjoint index
// pairs, whose angles all come from the current matrix, applied together as A <- J^T A J,
// V <- V J.  Three independent dependency chains per round instead of one.
template <int p0, int q0, int p1, int q1, int p2, int q2>
FIF_DEV void jacobi_round(float (&a)[6][6], float (&V)[6][6]) {
    constexpr int P[3] = {p0, p1, p2}, Q[3] = {q0, q1, q2};
    float t[3], c[3], s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) jacobi_angle(a[P[k]][P[k]], a[Q[k]][Q[k]], a[P[k]][Q[k]], t[k], c[k], s[k]);
    // blocks between two different pairs: X' = J_k^T X J_l
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = k + 1; l < 3; ++l) {
            const int p = P[k], q = Q[k], u = P[l], v = Q[l];
            // columns (pair l)
            const float xpu = c[l] * a[p][u] - s[l] * a[p][v], xpv = s[l] * a[p][u] + c[l] * a[p][v];
            const float xqu = c[l] * a[q][u] - s[l] * a[q][v], xqv = s[l] * a[q][u] + c[l] * a[q][v];
            // rows (pair k)
            const float ypu = c[k] * xpu - s[k] * xqu, yqu = s[k] * xpu + c[k] * xqu;
            const float ypv = c[k] * xpv - s[k] * xqv, yqv = s[k] * xpv + c[k] * xqv;
            a[p][u] = a[u][p] = ypu;
            a[p][v] = a[v][p] = ypv;
            a[q][u] = a[u][q] = yqu;
            a[q][v] = a[v][q] = yqv;
        }
    // diagonal blocks
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int p = P[k], q = Q[k];
        const float apq = a[p][q];
        a[p][p] = a[p][p] - t[k] * apq;
        a[q][q] = a[q][q] + t[k] * apq;
        a[p][q] = a[q][p] = 0.f;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float vp = V[r][P[k]], vq = V[r][Q[k]];
            V[r][P[k]] = c[k] * vp - s[k] * vq;
            V[r][Q[k]] = s[k] * vp + c[k] * vq;
        }
}

// Smallest eigenvalue of a symmetric 6x6 (packed, float): parallel-ordered Jacobi in single
// precision gives the eigenvector x of the smallest diagonal; the eigenvalue is the Rayleigh
// quotient x^T S x / x^T x in double precision (its error is second order in the error of x).
// If xout is given, x (unit, float) is returned too.
template <int SWEEPS = 4>
FIF_DEV double lambda_min_f64(const float* s, float* xout = nullptr) {
    float a[6][6], V[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            a[r][c] = s[sym_idx(r, c)];
            V[r][c] = (r == c) ? 1.f : 0.f;
        }
#pragma unroll 1
    for (int sweep = 0; sweep < SWEEPS; ++sweep) {
        jacobi_round<0, 1, 2, 3, 4, 5>(a, V);
        jacobi_round<0, 2, 1, 4, 3, 5>(a, V);
        jacobi_round<0, 3, 1, 5, 2, 4>(a, V);
        jacobi_round<0, 4, 1, 3, 2, 5>(a, V);
        jacobi_round<0, 5, 1, 2, 3, 4>(a, V);
    }
    float best = a[0][0];
    float x[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) x[r] = V[r][0];
#pragma unroll
    for (int c = 1; c < 6; ++c) {
        const float d = a[c][c];
        const bool take = d < best;
        best = take ? d : best;
#pragma unroll
        for (int r = 0; r < 6; ++r) x[r] = take ? V[r][c] : x[r];
    }
    double xd[6], num = 0.0, den = 0.0;
#pragma unroll
    for (int r = 0; r < 6; ++r) xd[r] = (double)x[r];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        double y = 0.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) y = fma((double)s[sym_idx(r, c)], xd[c], y);
        num = fma(xd[r], y, num);
        den = fma(xd[r], xd[r], den);
    }
    if (xout) {
        const float inv = rsqrtf((float)den);
#pragma unroll
        for (int r = 0; r < 6; ++r) xout[r] = x[r] * inv;
    }
    return num / den;
}

FIF_DEV float trace6(const float* s) {
    return ((s[0] + s[6]) + (s[11] + s[15])) + (s[18] + s[20]);
}

// ------------------------------------------------------------------------------------
// bulk-copy engine and mbarrier (inline PTX)
// ------------------------------------------------------------------------------------
FIF_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

FIF_DEV void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
FIF_DEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
FIF_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

FIF_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
FIF_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
FIF_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier to complete, giving up after ~`limit_ns`
// nanoseconds of global-timer time.  Returns false on timeout.
FIF_DEV bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        uint64_t t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > limit_ns) return false;
    }
}

// global -> shared bulk copy completing on an mbarrier (bytes and both addresses multiples of 16)
FIF_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// bulk prefetch of global memory into L2 (address and size multiples of 16)
FIF_DEV void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// packed single-precision pairs (sm_100+ f32x2 instructions: one issue slot, two lanes' worth
// of FP32 work; each half rounds exactly like the scalar instruction)
FIF_DEV unsigned long long pk2(float2 v) {
    unsigned long long u;
    memcpy(&u, &v, 8);
    return u;
}
FIF_DEV float2 upk2(unsigned long long u) {
    float2 v;
    memcpy(&v, &u, 8);
    return v;
}
FIF_DEV float2 add2(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
FIF_DEV float2 sub2(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
FIF_DEV float2 mul2(float2 a, float2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(d);
}
FIF_DEV float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return upk2(d);
}

// record a device-side failure (first code wins)
FIF_DEV void set_error(int* err, int code) {
    if (err) atomicCAS(err, 0, code);
}

}  // namespace fif

namespace fif {

// Inverse of a symmetric 6x6 (packed, float) in double precision by Gauss-Jordan with
// partial pivoting (row exchanges by selects so the matrix stays in registers).  Returns
// false when a pivot is exactly zero.  Output packed (upper triangle of the inverse).
FIF_DEV bool inverse6_f64(const float* s, double* out) {
    double a[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) a[r][c] = (double)s[sym_idx(r, c)];
    int perm[6];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        int p = k;
        double best = fabs(a[k][k]);
#pragma unroll
        for (int r = k + 1; r < 6; ++r) {
            const double v = fabs(a[r][k]);
            if (v > best) { best = v; p = r; }
        }
        perm[k] = p;
#pragma unroll
        for (int r = k + 1; r < 6; ++r) {
            const bool sw = (r == p);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const double x = a[k][c], y = a[r][c];
                a[k][c] = sw ? y : x;
                a[r][c] = sw ? x : y;
            }
        }
        const double piv = a[k][k];
        ok &= (piv != 0.0);
        const double inv = 1.0 / piv;
        a[k][k] = 1.0;
#pragma unroll
        for (int c = 0; c < 6; ++c) a[k][c] *= inv;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (r == k) continue;
            const double f = a[r][k];
            a[r][k] = 0.0;
#pragma unroll
            for (int c = 0; c < 6; ++c) a[r][c] = fma(-f, a[k][c], a[r][c]);
        }
    }
    // undo the row exchanges as column exchanges, last first
#pragma unroll
    for (int k = 5; k >= 0; --k) {
#pragma unroll
        for (int c = k + 1; c < 6; ++c) {
            const bool sw = (perm[k] == c);
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                const double x = a[r][k], y = a[r][c];
                a[r][k] = sw ? y : x;
                a[r][c] = sw ? x : y;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) out[sym_idx(r, c)] = 0.5 * (a[r][c] + a[c][r]);
    return ok;
}

// S <- M_a S M_a^T with M_a = [[I, X], [0, I]], X = -[a]x (the dual of shift_ref: it moves a
// gradient with respect to the information from one reference point to another):
//   A' = A + X B^T + B X^T + X D X^T,  B' = B + X D,  D' = D
FIF_DEV void shift_dual(Blocks& s, const float a[3]) {
    float X[3][3];
    neg_skew(a, X);
    float XD[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) XD[r][c] = X[r][0] * s.D[0][c] + X[r][1] * s.D[1][c] + X[r][2] * s.D[2][c];
    float An[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float v = s.A[r][c];
#pragma unroll
            for (int l = 0; l < 3; ++l) v += X[r][l] * s.B[c][l] + s.B[r][l] * X[c][l] + XD[r][l] * X[c][l];
            An[r][c] = v;
        }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s.A[r][c] = 0.5f * (An[r][c] + An[c][r]);
            s.B[r][c] += XD[r][c];
        }
}

}  // namespace fif
