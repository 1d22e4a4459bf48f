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
        uint32_t best = (uint32_t)__double2hiint(a[c][c]) & 0x7fffffffu;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (r <= c) continue;
            const uint32_t v = (uint32_t)__double2hiint(a[r][c]) & 0x7fffffffu;
            if (v > best) { best = v; p = r; }
        }
        // exchange rows c and p with selects (the columns left of c are not read again)
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            if (r <= c) continue;
            const bool sw = (r == p);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                if (j < c) continue;
                const double x = a[c][j], y = a[r][j];
                a[c][j] = sw ? y : x;
                a[r][j] = sw ? x : y;
            }
        }
        if (p != c) sg = -sg;
        const double piv = a[c][c];
        if (piv == 0.0) zero = true;
        // 1 / piv: hardware approximation refined by two steps of Newton's iteration
        // x <- x + x (1 - piv x)
        double inv;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(inv) : "d"(piv));
        inv = fma(inv, fma(-piv, inv, 1.0), inv);
        inv = fma(inv, fma(-piv, inv, 1.0), inv);
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
// Smallest eigenvalue of a symmetric 6x6 (packed, float).  Householder reduction to tridiagonal
// form T in single precision (Golub and Van Loan, Sec. 8.3.1); bisection on Sturm counts of T (the
// number of negative pivots of the LDL^T factorisation of T - sigma I is the number of eigenvalues
// below sigma, Golub and Van Loan, Sec. 8.4.1) to single-precision resolution gives the shift mu;
// three steps of inverse iteration with S - mu I on the original matrix give the eigenvector x;
// the eigenvalue is the Rayleigh quotient x^T S x / x^T x in double precision on the original
// matrix, whose error is second order in the error of x.  If xout is given, x (unit, float) is
// returned too.
FIF_DEV double lambda_min_f64(const float* s, float* xout = nullptr) {
    float a[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) a[r][c] = s[sym_idx(r, c)];
    // reflections H_k = I - beta_k v_k v_k^T acting on rows / columns k+1..5, v_k kept in
    // a[k+1..5][k]; the lower triangle of the trailing block holds the reduced matrix
    float e[5], d[6];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float nrm2 = 0.f;
#pragma unroll
        for (int i = k + 1; i < 6; ++i) nrm2 = fmaf(a[i][k], a[i][k], nrm2);
        const float x0 = a[k + 1][k];
        const float nrm = sqrtf(nrm2);
        const float alpha = x0 >= 0.f ? -nrm : nrm;
        const float v0 = x0 - alpha;
        const float vv = fmaf(v0, v0, nrm2 - x0 * x0);
        const bool skip = !(vv > 0.f);
        const float beta = skip ? 0.f : 2.f / vv;
        a[k + 1][k] = v0;
        e[k] = skip ? x0 : alpha;
        // trailing block B (rows / columns k+1..5): B <- H B H
        float p[6], K = 0.f;
#pragma unroll
        for (int i = k + 1; i < 6; ++i) {
            float t = 0.f;
#pragma unroll
            for (int j = k + 1; j < 6; ++j) t = fmaf(a[i > j ? i : j][i > j ? j : i], a[j][k], t);
            p[i] = beta * t;
            K = fmaf(p[i], a[i][k], K);
        }
        K *= 0.5f * beta;
#pragma unroll
        for (int i = k + 1; i < 6; ++i) p[i] = fmaf(-K, a[i][k], p[i]);
#pragma unroll
        for (int i = k + 1; i < 6; ++i)
#pragma unroll
            for (int j = k + 1; j <= i; ++j) a[i][j] = a[i][j] - a[i][k] * p[j] - p[i] * a[j][k];
    }
    e[4] = a[5][4];
#pragma unroll
    for (int i = 0; i < 6; ++i) d[i] = a[i][i];
    float e2[5], lo = d[0], hi = d[0], scale = fabsf(d[0]);
#pragma unroll
    for (int i = 0; i < 5; ++i) e2[i] = e[i] * e[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float ri = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i < 5 ? fabsf(e[i]) : 0.f);
        lo = fminf(lo, d[i] - ri);
        hi = fminf(hi, d[i]);
        scale = fmaxf(scale, fabsf(d[i]) + ri);
    }
    // whether an eigenvalue lies below sigma: a negative pivot of T - sigma I = L D L^T.  A zero
    // pivot (flushed when subnormal) gives an infinite reciprocal and a next pivot of -inf, which
    // counts the same eigenvalue; e^2 is at least the smallest normal number, so that 0 * inf
    // never arises
#pragma unroll
    for (int i = 0; i < 5; ++i) e2[i] = fmaxf(e2[i], 1.17549435e-38f);
    auto any_below = [&](float sigma) {
        float q = d[0] - sigma;
        uint32_t sgn = __float_as_uint(q);
#pragma unroll
        for (int i = 1; i < 6; ++i) {
            float r;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
            q = fmaf(-e2[i - 1], r, d[i] - sigma);
            sgn |= __float_as_uint(q);
        }
        return (sgn >> 31) != 0u;
    };
    // lambda_min in [lo, hi]: lo is a Gershgorin bound, hi the smallest diagonal entry
#pragma unroll 2
    for (int it = 0; it < 26; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (any_below(mid)) hi = mid;
        else lo = mid;
    }
    const float mu = 0.5f * (lo + hi);
    // the eigenvector: three steps of inverse iteration with S - mu I on the original matrix
    // (single-precision LU with partial pivoting; a pivot below 2^-22 of the scale is raised to it)
    float b[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) b[r][c] = s[sym_idx(r, c)] - (r == c ? mu : 0.f);
    const float tiny = fmaxf(scale * 2.384185791015625e-7f, 1e-30f);
    int pv[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        int p = c;
        float best = fabsf(b[c][c]);
#pragma unroll
        for (int r = c + 1; r < 6; ++r) {
            const float v = fabsf(b[r][c]);
            if (v > best) { best = v; p = r; }
        }
        pv[c] = p;
#pragma unroll
        for (int r = c + 1; r < 6; ++r) {
            const bool sw = (r == p);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                const float u = b[c][j], w = b[r][j];
                b[c][j] = sw ? w : u;
                b[r][j] = sw ? u : w;
            }
        }
        float dd = b[c][c];
        dd = fabsf(dd) < tiny ? (dd < 0.f ? -tiny : tiny) : dd;
        b[c][c] = dd;
        const float inv = __frcp_rn(dd);
#pragma unroll
        for (int r = c + 1; r < 6; ++r) {
            const float f = b[r][c] * inv;
            b[r][c] = f;
#pragma unroll
            for (int j = c + 1; j < 6; ++j) b[r][j] = fmaf(-f, b[c][j], b[r][j]);
        }
    }
    float x[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) x[r] = 1.f;
#pragma unroll
    for (int step = 0; step < 3; ++step) {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int r = c + 1; r < 6; ++r) {
                const bool sw = (r == pv[c]);
                const float u = x[c], w = x[r];
                x[c] = sw ? w : u;
                x[r] = sw ? u : w;
            }
#pragma unroll
        for (int r = 1; r < 6; ++r)
#pragma unroll
            for (int c = 0; c < r; ++c) x[r] = fmaf(-b[r][c], x[c], x[r]);
#pragma unroll
        for (int r = 5; r >= 0; --r) {
            float v = x[r];
#pragma unroll
            for (int c = r + 1; c < 6; ++c) v = fmaf(-b[r][c], x[c], v);
            x[r] = __fdividef(v, b[r][r]);
        }
        float mx = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) mx = fmaxf(mx, fabsf(x[r]));
        const float inv = mx > 0.f ? __frcp_rn(mx) : 1.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) x[r] *= inv;
    }
    double xd[6], num = 0.0, den = 0.0;
#pragma unroll
    for (int r = 0; r < 6; ++r) xd[r] = (double)x[r];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        double y = (double)s[sym_idx(r, r)] * xd[r];
#pragma unroll
        for (int c = r + 1; c < 6; ++c) y = fma((double)s[sym_idx(r, c)], 2.0 * xd[c], y);
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
