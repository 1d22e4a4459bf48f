/*
 * fif_oracle.c -- plain FP64 CPU oracle for the Fisher Information Field hot path
 * (Zhang & Scaramuzza, "Fisher Information Field: an Efficient and Differentiable
 * Map for Perception-aware Planning", arXiv 2008.03324).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant with the CUDA path.
 *
 * Everything is written the slow, obvious way, in the order and notation of the
 * paper:
 *   - Observed FIM with Gaussian noise, I = sigma^-2 J^T J          (Sec. III-A, Eq. fim_gaussian)
 *   - Bearing measurement f = p^c/|p^c| and df/dp^c                 (Sec. V-A, Eq. jac_f)
 *   - Global-perturbation pose Jacobian  J = df/dp^c R_cw [-I, [p^w]x] (Eq. jac_pose_global)
 *   - Local (camera-frame) perturbation, second form of Eq. deriv_se3
 *   - Exact pinhole visibility (Eq. exact_vis_func), cone visibility (Eq. theta_vis_func)
 *   - Quadratic visibility v = k2 cos^2 + k1 cos + k0 (Eq. quad_vis_approx) with
 *     v_r, v_p monomials (Eq. quad_vis_component) and the three conditions of
 *     Eq. quadratic_conditions
 *   - Positional information factor C_I = sum_i diag6(v_p,i) I_i  (Eq. general_info_pif)
 *   - Query I = V_I(R) C_I = sum_k v_r[k] C_k                       (Eq. fim_separation,
 *     Eq. general_info_query), trilinear over the 8 surrounding voxels (Sec. VII-A-1)
 *   - Point-cloud FIM  I_T = sum_{k in V} I_T(p_k)                  (Sec. IV, Eq. cost_info)
 *   - Metrics: trace, determinant, smallest eigenvalue              (Sec. IV, Tab. sim_complexity)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - sigma is a parameter (default 1).
 *   - xi = (rho, phi): translation first, as in [-I, [p]x].
 *   - The landmark set V is a range shell r_min < |p - x| <= r_max, measured from the
 *     voxel node (field) or the camera position (point cloud).  The shell test and the
 *     pinhole bounds test are decisions taken in single precision with a fixed order
 *     of operations (the precision of the GPU kernels), so both sides agree on every
 *     landmark; all values are then computed in double precision.
 *   - Rotations are unit quaternions (w, x, y, z) giving R_wc.
 *   - Camera frame output is Ad^T I_w Ad with Ad = [[R, [t]x R], [0, R]].
 *
 * Parity is pinned in tests/test_oracle_*.py against closed forms, finite differences,
 * brute force and textbook routines; no function here is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <float.h>
/* The single-precision decisions below must round after every operation: the file is
 * compiled with -ffp-contract=off and without -ffast-math, and float expressions must
 * be evaluated in float (no excess precision). */
#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "float expressions must be evaluated in single precision"
#endif

/* ------------------------------------------------------------------------- */
/* parameter structs (mirrored field by field by the Python wrapper)          */
/* ------------------------------------------------------------------------- */
typedef struct {
    double origin[3];  /* node (i,j,k) sits at origin + res*(i,j,k)         */
    double res;
    int32_t nx, ny, nz;
    int32_t pad_;
} or_grid;

typedef struct {
    double half_fov;   /* alpha, half of the field of view (rad)             */
    double v_alpha;    /* value of the quadratic visibility at theta = alpha  */
    double r_min, r_max;
    double sigma;      /* bearing noise std                                   */
    double fx, fy, cx, cy;  /* pinhole for exact visibility                   */
    int32_t width, height;
} or_params;

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* small dense helpers                                                        */
/* ------------------------------------------------------------------------- */
static void skew(const double a[3], double S[9]) {
    /* [a]x such that [a]x b = a x b */
    S[0] = 0.0;   S[1] = -a[2]; S[2] = a[1];
    S[3] = a[2];  S[4] = 0.0;   S[5] = -a[0];
    S[6] = -a[1]; S[7] = a[0];  S[8] = 0.0;
}

static void matmul(const double* A, const double* B, double* C, int n, int k, int m) {
    /* C[n x m] = A[n x k] B[k x m], row-major */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
            C[i * m + j] = s;
        }
}

static void transpose(const double* A, double* T, int n, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) T[j * n + i] = A[i * m + j];
}

/* ------------------------------------------------------------------------- */
/* Rotation from a unit quaternion (w, x, y, z), R = R_wc, row-major.         */
/* ------------------------------------------------------------------------- */
void or_quat_to_rot(const double q_in[4], double R[9]) {
    double nrm = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / nrm, x = q_in[1] / nrm, y = q_in[2] / nrm, z = q_in[3] / nrm;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* ------------------------------------------------------------------------- */
/* Quadratic visibility (Sec. V-B-1)                                          */
/* ------------------------------------------------------------------------- */

/* Solve Eq. quadratic_conditions, v(0) = 1, v(pi) = 0, v(alpha) = v_alpha, for
 * v(theta) = k2 cos^2 + k1 cos + k0, by Gaussian elimination with partial pivoting
 * on the 3x3 system in the unknowns (k2, k1, k0).  Output k[0]=k0, k[1]=k1, k[2]=k2. */
void or_quad_coeffs(double alpha, double v_alpha, double k[3]) {
    double c0 = cos(0.0), cpi = cos(M_PI), ca = cos(alpha);
    double A[3][4] = {
        {c0 * c0, c0, 1.0, 1.0},
        {cpi * cpi, cpi, 1.0, 0.0},
        {ca * ca, ca, 1.0, v_alpha},
    };
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 4; ++c) { double tmp = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = tmp; }
        for (int r = col + 1; r < 3; ++r) {
            double f = A[r][col] / A[col][col];
            for (int c = col; c < 4; ++c) A[r][c] -= f * A[col][c];
        }
    }
    double x[3];
    for (int r = 2; r >= 0; --r) {
        double s = A[r][3];
        for (int c = r + 1; c < 3; ++c) s -= A[r][c] * x[c];
        x[r] = s / A[r][r];
    }
    k[2] = x[0]; k[1] = x[1]; k[0] = x[2];
}

/* v_r of Eq. quad_vis_component, from z = R_wc e3 */
void or_vr(const double z[3], const double k[3], double vr[10]) {
    double k0 = k[0], k1 = k[1], k2 = k[2];
    vr[0] = k2 * z[0] * z[0]; vr[1] = k2 * z[1] * z[1]; vr[2] = k2 * z[2] * z[2];
    vr[3] = 2 * k2 * z[0] * z[1]; vr[4] = 2 * k2 * z[0] * z[2]; vr[5] = 2 * k2 * z[1] * z[2];
    vr[6] = k1 * z[0]; vr[7] = k1 * z[1]; vr[8] = k1 * z[2];
    vr[9] = k0;
}

/* d v_r / d z_a, a = 0..2 : dvr[a][10] */
void or_vr_grad(const double z[3], const double k[3], double dvr[30]) {
    double k1 = k[1], k2 = k[2];
    memset(dvr, 0, 30 * sizeof(double));
    for (int a = 0; a < 3; ++a) {
        double* d = dvr + 10 * a;
        d[a] = 2 * k2 * z[a];
        /* 2 k2 z1 z2 */
        if (a == 0) { d[3] = 2 * k2 * z[1]; d[4] = 2 * k2 * z[2]; }
        if (a == 1) { d[3] = 2 * k2 * z[0]; d[5] = 2 * k2 * z[2]; }
        if (a == 2) { d[4] = 2 * k2 * z[0]; d[5] = 2 * k2 * z[1]; }
        d[6 + a] = k1;
    }
}

/* v_p of Eq. quad_vis_component, from the unit bearing p = (p^w - t)/|p^w - t| */
void or_vp(const double p[3], double vp[10]) {
    vp[0] = p[0] * p[0]; vp[1] = p[1] * p[1]; vp[2] = p[2] * p[2];
    vp[3] = p[0] * p[1]; vp[4] = p[0] * p[2]; vp[5] = p[1] * p[2];
    vp[6] = p[0]; vp[7] = p[1]; vp[8] = p[2];
    vp[9] = 1.0;
}

/* ------------------------------------------------------------------------- */
/* Bearing Jacobians (Sec. V-A)                                               */
/* ------------------------------------------------------------------------- */

/* d f / d p^c = I/n - p^c p^c^T / n^3  (Eq. jac_f) */
static void dbearing(const double pc[3], double D[9]) {
    double n = sqrt(pc[0] * pc[0] + pc[1] * pc[1] + pc[2] * pc[2]);
    double n3 = n * n * n;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            D[i * 3 + j] = (i == j ? 1.0 / n : 0.0) - pc[i] * pc[j] / n3;
}

/* Global perturbation (first form of Eq. deriv_se3), Eq. jac_pose_global:
 *   J = df/dp^c  R_cw  [-I3, [p^w - o]x]
 * o = 0 is the paper's world frame; a non-zero o expresses the rotational part of the
 * perturbation about the point o instead of the world origin.                  */
void or_jac_global(const double pw[3], const double R[9], const double t[3],
                   const double o[3], double J[18]) {
    double Rcw[9], d[3], pc[3], D[9], A[18], S[9], q[3], DR[9];
    transpose(R, Rcw, 3, 3);
    for (int i = 0; i < 3; ++i) d[i] = pw[i] - t[i];
    matmul(Rcw, d, pc, 3, 3, 1);
    dbearing(pc, D);
    for (int i = 0; i < 3; ++i) q[i] = pw[i] - o[i];
    skew(q, S);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i * 6 + j] = (i == j) ? -1.0 : 0.0;
            A[i * 6 + 3 + j] = S[i * 3 + j];
        }
    matmul(D, Rcw, DR, 3, 3, 3);
    matmul(DR, A, J, 3, 3, 6);
}

/* Local perturbation (second form of Eq. deriv_se3): p^c = (T_wc exp(xi))^-1 p^w, so
 *   J = df/dp^c  [-I3, [p^c]x]                                                 */
void or_jac_local(const double pw[3], const double R[9], const double t[3], double J[18]) {
    double Rcw[9], d[3], pc[3], D[9], A[18], S[9];
    transpose(R, Rcw, 3, 3);
    for (int i = 0; i < 3; ++i) d[i] = pw[i] - t[i];
    matmul(Rcw, d, pc, 3, 3, 1);
    dbearing(pc, D);
    skew(pc, S);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i * 6 + j] = (i == j) ? -1.0 : 0.0;
            A[i * 6 + 3 + j] = S[i * 3 + j];
        }
    matmul(D, A, J, 3, 3, 6);
}

/* Eq. fim_gaussian: I = sigma^-2 J^T J */
void or_fim_gauss(const double J[18], double sigma, double I[36]) {
    double Jt[18];
    transpose(J, Jt, 3, 6);
    matmul(Jt, J, I, 6, 3, 6);
    double s2 = 1.0 / (sigma * sigma);
    for (int i = 0; i < 36; ++i) I[i] *= s2;
}

/* ------------------------------------------------------------------------- */
/* Single-precision decisions (taken in the precision of the GPU kernels).    */
/* Every operation rounds to nearest single; no fused multiply-add.           */
/* ------------------------------------------------------------------------- */

/* landmark p within the shell r_min < |p - x| <= r_max (squared, single precision) */
int or_in_shell_f32(const float p[3], const float x[3], float rmin2, float rmax2) {
    float dx = p[0] - x[0], dy = p[1] - x[1], dz = p[2] - x[2];
    float a = dx * dx, b = dy * dy, c = dz * dz;
    float s = a + b;
    float n2 = s + c;
    return (n2 > rmin2) && (n2 <= rmax2);
}

/* Node coordinate origin + res*i in single precision */
static float node_coord_f32(float origin, float res, int i) {
    float t = res * (float)i;
    float c = origin + t;
    return c;
}

/* Rotation from quaternion in single precision, fixed order of operations */
static void quat_to_rot_f32(const float q[4], float R[9]) {
    float s2a = q[0] * q[0], s2b = q[1] * q[1], s2c = q[2] * q[2], s2d = q[3] * q[3];
    float s = s2a + s2b; s = s + s2c; s = s + s2d;
    float r = sqrtf(s);
    float w = q[0] / r, x = q[1] / r, y = q[2] / r, z = q[3] / r;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
    float t;
    t = yy + zz; R[0] = 1.0f - 2.0f * t;
    t = xy - wz; R[1] = 2.0f * t;
    t = xz + wy; R[2] = 2.0f * t;
    t = xy + wz; R[3] = 2.0f * t;
    t = xx + zz; R[4] = 1.0f - 2.0f * t;
    t = yz - wx; R[5] = 2.0f * t;
    t = xz - wy; R[6] = 2.0f * t;
    t = yz + wx; R[7] = 2.0f * t;
    t = xx + yy; R[8] = 1.0f - 2.0f * t;
}

/* Exact pinhole visibility, Eq. exact_vis_func: project and test the image bounds.
 * u = fx x/z + cx in [0, W) and v = fy y/z + cy in [0, H) with z > 0, tested in the
 * division-free form fx x + cx z in [0, W z) (z > 0), single precision.          */
int or_pinhole_visible_f32(const float p[3], const float pose[7], float fx, float fy,
                           float cx, float cy, float W, float H) {
    float R[9];
    quat_to_rot_f32(pose + 3, R);
    float dx = p[0] - pose[0], dy = p[1] - pose[1], dz = p[2] - pose[2];
    float a, b, c, s;
    /* p^c = R^T d */
    a = R[0] * dx; b = R[3] * dy; c = R[6] * dz; s = a + b; float pcx = s + c;
    a = R[1] * dx; b = R[4] * dy; c = R[7] * dz; s = a + b; float pcy = s + c;
    a = R[2] * dx; b = R[5] * dy; c = R[8] * dz; s = a + b; float pcz = s + c;
    if (!(pcz > 0.0f)) return 0;
    a = fx * pcx; b = cx * pcz; float ux = a + b;
    float wz = W * pcz;
    if (!(ux >= 0.0f && ux < wz)) return 0;
    a = fy * pcy; b = cy * pcz; float uy = a + b;
    float hz = H * pcz;
    if (!(uy >= 0.0f && uy < hz)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Point-cloud FIM (Sec. IV, Eq. cost_info; Sec. V Eq. vis_fim)               */
/* ------------------------------------------------------------------------- */
enum { OR_VIS_PINHOLE = 0, OR_VIS_CONE = 1, OR_VIS_QUAD = 2, OR_VIS_ONE = 3 };
enum { OR_FRAME_CAMERA = 0, OR_FRAME_WORLD = 1 };

/* I_T = sum over landmarks in the range shell of v(T, p) I(p).
 * vis: exact pinhole (Eq. exact_vis_func), cone theta <= alpha (Eq. theta_vis_func),
 *      quadratic weight v_quad(theta) (Eq. quad_vis_approx), or v = 1.
 * frame: camera = local perturbation, world = global perturbation about the origin. */
static void pc_fim_one(const float* lm, int64_t n, const float pose[7], const or_params* prm,
                       int vis, int frame, const double kq[3], double I[36]) {
    double q[4] = {pose[3], pose[4], pose[5], pose[6]}, R[9], t[3] = {pose[0], pose[1], pose[2]};
    double o[3] = {0, 0, 0};
    or_quat_to_rot(q, R);
    double z[3] = {R[2], R[5], R[8]};
    float rmin2 = (float)(prm->r_min * prm->r_min), rmax2 = (float)(prm->r_max * prm->r_max);
    float tf[3] = {pose[0], pose[1], pose[2]};
    double cos_alpha = cos(prm->half_fov);
    memset(I, 0, 36 * sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        const float* pf = lm + 3 * i;
        if (!or_in_shell_f32(pf, tf, rmin2, rmax2)) continue;
        double pw[3] = {pf[0], pf[1], pf[2]};
        double v = 1.0;
        if (vis == OR_VIS_PINHOLE) {
            v = or_pinhole_visible_f32(pf, pose, (float)prm->fx, (float)prm->fy, (float)prm->cx,
                                       (float)prm->cy, (float)prm->width, (float)prm->height) ? 1.0 : 0.0;
        } else if (vis == OR_VIS_CONE || vis == OR_VIS_QUAD) {
            double d[3] = {pw[0] - t[0], pw[1] - t[1], pw[2] - t[2]};
            double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double ct = (z[0] * d[0] + z[1] * d[1] + z[2] * d[2]) / nn;   /* cos theta */
            if (vis == OR_VIS_CONE) v = (ct >= cos_alpha) ? 1.0 : 0.0;
            else v = kq[2] * ct * ct + kq[1] * ct + kq[0];
        }
        if (v == 0.0) continue;
        double J[18], Ii[36];
        if (frame == OR_FRAME_CAMERA) or_jac_local(pw, R, t, J);
        else or_jac_global(pw, R, t, o, J);
        or_fim_gauss(J, prm->sigma, Ii);
        for (int e = 0; e < 36; ++e) I[e] += v * Ii[e];
    }
}

void or_pc_fim(const float* lm, int64_t n, const float* poses, int64_t m, const or_params* prm,
               int vis, int frame, double* out /* [m][36] */) {
    double kq[3];
    or_quad_coeffs(prm->half_fov, prm->v_alpha, kq);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) pc_fim_one(lm, n, poses + 7 * j, prm, vis, frame, kq, out + 36 * j);
}

/* number of landmarks in the shell and visible (pinhole) per pose, for statistics */
void or_pc_counts(const float* lm, int64_t n, const float* poses, int64_t m, const or_params* prm,
                  int64_t* in_shell, int64_t* visible) {
    float rmin2 = (float)(prm->r_min * prm->r_min), rmax2 = (float)(prm->r_max * prm->r_max);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < m; ++j) {
        const float* pose = poses + 7 * j;
        int64_t a = 0, b = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!or_in_shell_f32(lm + 3 * i, pose, rmin2, rmax2)) continue;
            ++a;
            b += or_pinhole_visible_f32(lm + 3 * i, pose, (float)prm->fx, (float)prm->fy, (float)prm->cx,
                                        (float)prm->cy, (float)prm->width, (float)prm->height);
        }
        in_shell[j] = a; visible[j] = b;
    }
}

/* ------------------------------------------------------------------------- */
/* Field build (Sec. VI-A-1, Eq. general_info_pif)                            */
/* ------------------------------------------------------------------------- */

/* For each requested node c: C_k = sum_{i in V_c} v_p(u_i)[k] I_i,  k = 0..9,
 * where V_c is the range shell around c, u_i = (p_i - c)/|p_i - c| is the bearing
 * that enters v_p (Eq. quad_vis_approx with t = c), and I_i is the rotation-invariant
 * FIM of Eq. global_fim_eq, evaluated with R = I (the value does not depend on R).
 * about_node = 0: the paper's world frame (rotation about the world origin);
 * about_node = 1: rotation about the node itself (o = c).
 * out: [cnt][10][36], full symmetric 6x6 per k.                                 */
void or_field_nodes(const float* lm, int64_t n, const or_grid* g, const or_params* prm,
                    const int64_t* nodes, int64_t cnt, int about_node, double* out) {
    float rmin2 = (float)(prm->r_min * prm->r_min), rmax2 = (float)(prm->r_max * prm->r_max);
    const double Rid[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < cnt; ++s) {
        int64_t node = nodes[s];
        int ix = (int)(node % g->nx), iy = (int)((node / g->nx) % g->ny), iz = (int)(node / ((int64_t)g->nx * g->ny));
        float cf[3] = {node_coord_f32((float)g->origin[0], (float)g->res, ix),
                       node_coord_f32((float)g->origin[1], (float)g->res, iy),
                       node_coord_f32((float)g->origin[2], (float)g->res, iz)};
        double c[3] = {cf[0], cf[1], cf[2]};
        double o[3] = {0, 0, 0};
        if (about_node) { o[0] = c[0]; o[1] = c[1]; o[2] = c[2]; }
        double* C = out + 360 * s;
        memset(C, 0, 360 * sizeof(double));
        for (int64_t i = 0; i < n; ++i) {
            const float* pf = lm + 3 * i;
            if (!or_in_shell_f32(pf, cf, rmin2, rmax2)) continue;
            double pw[3] = {pf[0], pf[1], pf[2]};
            double d[3] = {pw[0] - c[0], pw[1] - c[1], pw[2] - c[2]};
            double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double u[3] = {d[0] / nn, d[1] / nn, d[2] / nn};
            double vp[10], J[18], Ii[36];
            or_vp(u, vp);
            or_jac_global(pw, Rid, c, o, J);
            or_fim_gauss(J, prm->sigma, Ii);
            /* diag6(v_p,i) I_i : the 6N_v x 6 block column, block k = v_p[k] I_i */
            for (int k = 0; k < 10; ++k)
                for (int e = 0; e < 36; ++e) C[36 * k + e] += vp[k] * Ii[e];
        }
    }
}

/* number of (node, landmark) pairs in the shell for the requested nodes */
int64_t or_field_pairs(const float* lm, int64_t n, const or_grid* g, const or_params* prm,
                       const int64_t* nodes, int64_t cnt) {
    float rmin2 = (float)(prm->r_min * prm->r_min), rmax2 = (float)(prm->r_max * prm->r_max);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : total)
    for (int64_t s = 0; s < cnt; ++s) {
        int64_t node = nodes[s];
        int ix = (int)(node % g->nx), iy = (int)((node / g->nx) % g->ny), iz = (int)(node / ((int64_t)g->nx * g->ny));
        float cf[3] = {node_coord_f32((float)g->origin[0], (float)g->res, ix),
                       node_coord_f32((float)g->origin[1], (float)g->res, iy),
                       node_coord_f32((float)g->origin[2], (float)g->res, iz)};
        for (int64_t i = 0; i < n; ++i) total += or_in_shell_f32(lm + 3 * i, cf, rmin2, rmax2);
    }
    return total;
}

/* ------------------------------------------------------------------------- */
/* Query (Sec. VI-A-1, Eq. fim_separation / general_info_query)               */
/* ------------------------------------------------------------------------- */
enum { OR_INTERP_TRILINEAR = 0, OR_INTERP_NEAREST = 1 };

/* Cell lookup for one position.  Trilinear: the 8 nodes around t; the base index is
 * clamp(floor(g), 0, dim-2) with g = (t - origin)/res, and the weight clamp(g - i0, 0, 1).
 * Nearest: the node round-half-up(g), clamped.  status 1 when t lies outside the lattice
 * box.  Poses are double; the outside test and the nearest-node choice are decisions
 * taken on the single-precision position, g = (t - origin)/res rounded to single.
 * corner j = bx + 2 by + 4 bz  sits at i0 + (bx, by, bz).                         */
void or_query_cell(const or_grid* g, const double t[3], int interp, int64_t nodes[8], double w[8],
                   double dw[24] /* d w_j / d t_a, [8][3] */, int32_t* status) {
    int dims[3] = {g->nx, g->ny, g->nz};
    int i0[3]; double f[3]; double dfa[3];
    int outside = 0;
    for (int a = 0; a < 3; ++a) {
        float num = (float)t[a] - (float)g->origin[a];
        float gf = num / (float)g->res;
        if (gf < 0.0f || gf > (float)(dims[a] - 1)) outside = 1;
        if (interp == OR_INTERP_NEAREST) {
            float h = gf + 0.5f;
            int ii = (int)floorf(h);
            if (ii < 0) ii = 0;
            if (ii > dims[a] - 1) ii = dims[a] - 1;
            i0[a] = ii; f[a] = 0.0; dfa[a] = 0.0;
        } else {
            double gd = (t[a] - g->origin[a]) / g->res;
            int ii = (int)floor(gd);
            if (ii < 0) ii = 0;
            if (ii > dims[a] - 2) ii = dims[a] - 2;
            double fr = gd - ii;
            double d = 1.0 / g->res;
            if (fr < 0.0) { fr = 0.0; d = 0.0; }
            if (fr > 1.0) { fr = 1.0; d = 0.0; }
            i0[a] = ii; f[a] = fr; dfa[a] = d;
        }
    }
    for (int j = 0; j < 8; ++j) {
        int b[3] = {j & 1, (j >> 1) & 1, (j >> 2) & 1};
        if (interp == OR_INTERP_NEAREST) {
            nodes[j] = i0[0] + (int64_t)dims[0] * (i0[1] + (int64_t)dims[1] * i0[2]);
            w[j] = (j == 0) ? 1.0 : 0.0;
            for (int a = 0; a < 3; ++a) dw[3 * j + a] = 0.0;
            continue;
        }
        int ii[3];
        double wa[3], da[3];
        for (int a = 0; a < 3; ++a) {
            ii[a] = i0[a] + b[a];
            wa[a] = b[a] ? f[a] : 1.0 - f[a];
            da[a] = b[a] ? dfa[a] : -dfa[a];
        }
        nodes[j] = ii[0] + (int64_t)dims[0] * (ii[1] + (int64_t)dims[1] * ii[2]);
        w[j] = wa[0] * wa[1] * wa[2];
        dw[3 * j + 0] = da[0] * wa[1] * wa[2];
        dw[3 * j + 1] = wa[0] * da[1] * wa[2];
        dw[3 * j + 2] = wa[0] * wa[1] * da[2];
    }
    *status = outside;
}

void or_query_cells(const or_grid* g, const double* poses, int64_t m, int interp,
                    int64_t* nodes /*[m][8]*/, double* w /*[m][8]*/, double* dw /*[m][8][3]*/,
                    int32_t* status) {
    for (int64_t i = 0; i < m; ++i)
        or_query_cell(g, poses + 7 * i, interp, nodes + 8 * i, w + 8 * i, dw + 24 * i, status + i);
}

/* Ad = [[R, [t]x R], [0, R]]  (6x6, row-major) */
static void adjoint_se3(const double R[9], const double t[3], double Ad[36]) {
    double S[9], SR[9];
    skew(t, S);
    matmul(S, R, SR, 3, 3, 3);
    memset(Ad, 0, 36 * sizeof(double));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Ad[i * 6 + j] = R[i * 3 + j];
            Ad[i * 6 + 3 + j] = SR[i * 3 + j];
            Ad[(3 + i) * 6 + 3 + j] = R[i * 3 + j];
        }
}

/* One query from world-frame coefficient sets of the 8 surrounding nodes.
 * I_w = V_I(R) sum_j w_j C_j = sum_k v_r[k] sum_j w_j C_jk    (Eq. fim_separation)
 * camera frame: I_c = Ad^T I_w Ad (the local-perturbation FIM, Sec. V-A).        */
static void query_one(const double* corners /*[8][360]*/, const double w[8], const double pose[7],
                      const double k[3], int frame, double I[36]) {
    double q[4] = {pose[3], pose[4], pose[5], pose[6]}, R[9], t[3] = {pose[0], pose[1], pose[2]};
    or_quat_to_rot(q, R);
    double z[3] = {R[2], R[5], R[8]}, vr[10];
    or_vr(z, k, vr);
    double Iw[36];
    memset(Iw, 0, sizeof(Iw));
    for (int j = 0; j < 8; ++j) {
        if (w[j] == 0.0) continue;
        for (int kk = 0; kk < 10; ++kk)
            for (int e = 0; e < 36; ++e) Iw[e] += vr[kk] * w[j] * corners[360 * j + 36 * kk + e];
    }
    if (frame == OR_FRAME_WORLD) { memcpy(I, Iw, sizeof(Iw)); return; }
    double Ad[36], AdT[36], tmp[36];
    adjoint_se3(R, t, Ad);
    transpose(Ad, AdT, 6, 6);
    matmul(AdT, Iw, tmp, 6, 6, 6);
    matmul(tmp, Ad, I, 6, 6, 6);
}

void or_query_batch(const double* corners /*[m][8][360]*/, const double* w /*[m][8]*/,
                    const double* poses, int64_t m, const double k[3], int frame, double* out /*[m][36]*/) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) query_one(corners + 2880 * i, w + 8 * i, poses + 7 * i, k, frame, out + 36 * i);
}

/* ------------------------------------------------------------------------- */
/* Information metrics s(.) (Sec. IV)                                          */
/* ------------------------------------------------------------------------- */

/* log|det| and sign by LU with partial pivoting */
void or_logdet(const double A_in[36], double* logabsdet, double* sign) {
    double A[36];
    memcpy(A, A_in, sizeof(A));
    double sgn = 1.0, lad = 0.0;
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r * 6 + c]) > fabs(A[piv * 6 + c])) piv = r;
        if (A[piv * 6 + c] == 0.0) { *logabsdet = -INFINITY; *sign = 0.0; return; }
        if (piv != c) {
            for (int j = 0; j < 6; ++j) { double tmp = A[c * 6 + j]; A[c * 6 + j] = A[piv * 6 + j]; A[piv * 6 + j] = tmp; }
            sgn = -sgn;
        }
        double p = A[c * 6 + c];
        if (p < 0) sgn = -sgn;
        lad += log(fabs(p));
        for (int r = c + 1; r < 6; ++r) {
            double f = A[r * 6 + c] / p;
            for (int j = c; j < 6; ++j) A[r * 6 + j] -= f * A[c * 6 + j];
        }
    }
    *logabsdet = lad; *sign = sgn;
}

/* Inverse by Gauss-Jordan with partial pivoting (used for d log|det| = tr(A^-1 dA)) */
int or_inverse6(const double A_in[36], double Ainv[36]) {
    double A[72];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) A[i * 12 + j] = (j < 6) ? A_in[i * 6 + j] : ((j - 6) == i ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r * 12 + c]) > fabs(A[piv * 12 + c])) piv = r;
        if (A[piv * 12 + c] == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j < 12; ++j) { double tmp = A[c * 12 + j]; A[c * 12 + j] = A[piv * 12 + j]; A[piv * 12 + j] = tmp; }
        double p = A[c * 12 + c];
        for (int j = 0; j < 12; ++j) A[c * 12 + j] /= p;
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            double f = A[r * 12 + c];
            for (int j = 0; j < 12; ++j) A[r * 12 + j] -= f * A[c * 12 + j];
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Ainv[i * 6 + j] = A[i * 12 + 6 + j];
    return 0;
}

/* Cyclic Jacobi eigenvalue iteration for a symmetric 6x6 matrix, until the
 * off-diagonal Frobenius norm is below 1e-15 of the full norm (textbook form).
 * evals ascending; evecs columns (row-major [6][6], column j = eigenvector j). */
void or_jacobi6(const double A_in[36], double evals[6], double evecs[36]) {
    double A[36], V[36];
    memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < 36; ++i) V[i] = (i % 7 == 0) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < 36; ++i) fro += A[i] * A[i];
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 6; ++p)
            for (int q = p + 1; q < 6; ++q) off += 2.0 * A[p * 6 + q] * A[p * 6 + q];
        if (sqrt(off) <= 1e-15 * fro || off == 0.0) break;
        for (int p = 0; p < 6; ++p)
            for (int q = p + 1; q < 6; ++q) {
                double apq = A[p * 6 + q];
                if (apq == 0.0) continue;
                double theta = (A[q * 6 + q] - A[p * 6 + p]) / (2.0 * apq);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                /* A <- G^T A G with G the rotation in the (p,q) plane */
                for (int r = 0; r < 6; ++r) {
                    double arp = A[r * 6 + p], arq = A[r * 6 + q];
                    A[r * 6 + p] = c * arp - s * arq;
                    A[r * 6 + q] = s * arp + c * arq;
                }
                for (int r = 0; r < 6; ++r) {
                    double apr = A[p * 6 + r], aqr = A[q * 6 + r];
                    A[p * 6 + r] = c * apr - s * aqr;
                    A[q * 6 + r] = s * apr + c * aqr;
                }
                for (int r = 0; r < 6; ++r) {
                    double vrp = V[r * 6 + p], vrq = V[r * 6 + q];
                    V[r * 6 + p] = c * vrp - s * vrq;
                    V[r * 6 + q] = s * vrp + c * vrq;
                }
            }
    }
    /* sort ascending */
    int idx[6] = {0, 1, 2, 3, 4, 5};
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j)
            if (A[idx[j] * 7] < A[idx[i] * 7]) { int tmp = idx[i]; idx[i] = idx[j]; idx[j] = tmp; }
    for (int i = 0; i < 6; ++i) {
        evals[i] = A[idx[i] * 7];
        for (int r = 0; r < 6; ++r) evecs[r * 6 + i] = V[r * 6 + idx[i]];
    }
}

/* metrics: out = [trace, log|det|, sign(det), lambda_min] */
void or_metrics(const double* I, int64_t m, double* out /*[m][4]*/) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const double* A = I + 36 * i;
        double tr = 0.0;
        for (int d = 0; d < 6; ++d) tr += A[d * 7];
        double lad, sg, ev[6], V[36];
        or_logdet(A, &lad, &sg);
        or_jacobi6(A, ev, V);
        out[4 * i + 0] = tr; out[4 * i + 1] = lad; out[4 * i + 2] = sg; out[4 * i + 3] = ev[0];
    }
}

void or_eig_batch(const double* I, int64_t m, double* evals /*[m][6]*/, double* evecs /*[m][36]*/) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) or_jacobi6(I + 36 * i, evals + 6 * i, evecs + 36 * i);
}

/* ------------------------------------------------------------------------- */
/* Gradient of sum_m gm[m] * metric_m(I_c) with respect to the pose            */
/* (t in the world, phi a right perturbation R <- R exp(phi^)).                */
/*                                                                           */
/*   I_c = Ad^T I_w Ad,  I_w = sum_k v_r(z)[k] sum_j w_j(t) C_jk,  z = R e3     */
/*   dm = <G, dI_c>,  G = dm/dI_c  (trace: Id; log|det|: I_c^-1; lambda_min: x x^T) */
/*   <G, dI_c> = 2 <G, Ad^T I_w dAd> + <Ad G Ad^T, dI_w>                        */
/*   dt_a:   dAd = [[0, [e_a]x R], [0, 0]],  dI_w = sum_k v_r[k] sum_j dw_j/dt_a C_jk */
/*   dphi_a: dAd = Ad blkdiag([e_a]x, [e_a]x), dz = R (e_a x e3),                */
/*           dI_w = sum_k (grad_z v_r[k] . dz) sum_j w_j C_jk                     */
/* ------------------------------------------------------------------------- */
static void grad_one(const double* corners, const double w[8], const double dw[24], const double pose[7],
                     const double k[3], const double gm[3], double g[6]) {
    double q[4] = {pose[3], pose[4], pose[5], pose[6]}, R[9], t[3] = {pose[0], pose[1], pose[2]};
    or_quat_to_rot(q, R);
    double z[3] = {R[2], R[5], R[8]}, vr[10], dvr[30];
    or_vr(z, k, vr);
    or_vr_grad(z, k, dvr);
    /* sum_j w_j C_jk  and  sum_j dw_j/dt_a C_jk */
    double Cw[360], Cdt[3][360];
    memset(Cw, 0, sizeof(Cw)); memset(Cdt, 0, sizeof(Cdt));
    for (int j = 0; j < 8; ++j)
        for (int e = 0; e < 360; ++e) {
            double c = corners[360 * j + e];
            Cw[e] += w[j] * c;
            for (int a = 0; a < 3; ++a) Cdt[a][e] += dw[3 * j + a] * c;
        }
    double Iw[36];
    memset(Iw, 0, sizeof(Iw));
    for (int kk = 0; kk < 10; ++kk)
        for (int e = 0; e < 36; ++e) Iw[e] += vr[kk] * Cw[36 * kk + e];
    double Ad[36], AdT[36], tmp[36], Ic[36];
    adjoint_se3(R, t, Ad);
    transpose(Ad, AdT, 6, 6);
    matmul(AdT, Iw, tmp, 6, 6, 6);
    matmul(tmp, Ad, Ic, 6, 6, 6);
    /* G = dm/dI_c */
    double G[36];
    memset(G, 0, sizeof(G));
    for (int d = 0; d < 6; ++d) G[d * 7] += gm[0];
    if (gm[1] != 0.0) {
        double Ci[36];
        or_inverse6(Ic, Ci);
        for (int e = 0; e < 36; ++e) G[e] += gm[1] * Ci[e];
    }
    if (gm[2] != 0.0) {
        double ev[6], V[36];
        or_jacobi6(Ic, ev, V);
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c) G[r * 6 + c] += gm[2] * V[r * 6] * V[c * 6];
    }
    /* H = Ad G Ad^T ;  K = Ad^T I_w  (so <G, Ad^T I_w dAd> = <K^T G, dAd>) */
    double H[36], K[36], GK[36];
    matmul(Ad, G, tmp, 6, 6, 6);
    matmul(tmp, AdT, H, 6, 6, 6);
    matmul(AdT, Iw, K, 6, 6, 6);
    /* <G, K dAd> = <K^T G, dAd> */
    double KT[36];
    transpose(K, KT, 6, 6);
    matmul(KT, G, GK, 6, 6, 6);
    for (int a = 0; a < 3; ++a) {
        double e[3] = {0, 0, 0}; e[a] = 1.0;
        double S[9], SR[9], dAd[36];
        skew(e, S);
        matmul(S, R, SR, 3, 3, 3);
        memset(dAd, 0, sizeof(dAd));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dAd[i * 6 + 3 + j] = SR[i * 3 + j];
        double dIw[36];
        memset(dIw, 0, sizeof(dIw));
        for (int kk = 0; kk < 10; ++kk)
            for (int x = 0; x < 36; ++x) dIw[x] += vr[kk] * Cdt[a][36 * kk + x];
        double s = 0.0;
        for (int x = 0; x < 36; ++x) s += 2.0 * GK[x] * dAd[x] + H[x] * dIw[x];
        g[a] = s;
    }
    for (int a = 0; a < 3; ++a) {
        double e[3] = {0, 0, 0}; e[a] = 1.0;
        double S[9], B[36], dAd[36];
        skew(e, S);
        memset(B, 0, sizeof(B));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) { B[i * 6 + j] = S[i * 3 + j]; B[(3 + i) * 6 + 3 + j] = S[i * 3 + j]; }
        matmul(Ad, B, dAd, 6, 6, 6);
        /* dz = R (e_a x e3) */
        double e3[3] = {0, 0, 1}, cr[3] = {e[1] * e3[2] - e[2] * e3[1], e[2] * e3[0] - e[0] * e3[2], e[0] * e3[1] - e[1] * e3[0]};
        double dz[3];
        matmul(R, cr, dz, 3, 3, 1);
        double dIw[36];
        memset(dIw, 0, sizeof(dIw));
        for (int kk = 0; kk < 10; ++kk) {
            double dv = dvr[kk] * dz[0] + dvr[10 + kk] * dz[1] + dvr[20 + kk] * dz[2];
            for (int x = 0; x < 36; ++x) dIw[x] += dv * Cw[36 * kk + x];
        }
        double s = 0.0;
        for (int x = 0; x < 36; ++x) s += 2.0 * GK[x] * dAd[x] + H[x] * dIw[x];
        g[3 + a] = s;
    }
}

void or_query_grad_batch(const double* corners /*[m][8][360]*/, const double* w /*[m][8]*/,
                         const double* dw /*[m][8][3]*/, const double* poses, int64_t m, const double k[3],
                         const double* gm /*[m][3]*/, double* g /*[m][6]*/) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i)
        grad_one(corners + 2880 * i, w + 8 * i, dw + 24 * i, poses + 7 * i, k, gm + 3 * i, g + 6 * i);
}

/* ------------------------------------------------------------------------- */
/* GP visibility (Sec. V-B-2, Eq. sigmoid_vis_func, Eq. gp_vis_approx)         */
/*                                                                           */
/*   v_sig(theta) = 1 / (1 + exp(-k_s (cos theta - cos alpha)))                */
/*   v_gp(z) = K_z (K^s + s_n^2 I)^-1 v^s,  K_z[g] = k(z, z_g),                */
/*   K^s[g][h] = k(z_g, z_h),  k(a, b) = exp(-|a - b|^2 / (2 l^2))             */
/* so v_r = K_z and v_p = (K^s + s_n^2 I)^-1 v^s (N_v = N_s).  Readings: the    */
/* printed Eq. gp_vis_approx omits the inverse of K^s (taken as in Eq.          */
/* gp_regress); the "noise parameter" s_n^2 is added to the diagonal of K^s;    */
/* the signal variance of k is 1 (it cancels in the mean).                      */
/* ------------------------------------------------------------------------- */

static double se_kernel(const double* a, const double* b, double l) {
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return exp(-(d0 * d0 + d1 * d1 + d2 * d2) / (2.0 * l * l));
}

/* W = (K^s + noise I)^-1, [ns][ns], by Gauss-Jordan with partial pivoting */
int or_gp_weights(const double* axes, int ns, double l, double noise, double* W) {
    double* A = (double*)malloc(sizeof(double) * (size_t)ns * 2 * ns);
    if (!A) return -1;
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < 2 * ns; ++j)
            A[i * 2 * ns + j] = (j < ns) ? se_kernel(axes + 3 * i, axes + 3 * j, l) + (i == j ? noise : 0.0)
                                         : ((j - ns) == i ? 1.0 : 0.0);
    int rc = 0;
    for (int c = 0; c < ns; ++c) {
        int piv = c;
        for (int r = c + 1; r < ns; ++r)
            if (fabs(A[r * 2 * ns + c]) > fabs(A[piv * 2 * ns + c])) piv = r;
        if (A[piv * 2 * ns + c] == 0.0) { rc = -1; break; }
        if (piv != c)
            for (int j = 0; j < 2 * ns; ++j) {
                double t = A[c * 2 * ns + j]; A[c * 2 * ns + j] = A[piv * 2 * ns + j]; A[piv * 2 * ns + j] = t;
            }
        double p = A[c * 2 * ns + c];
        for (int j = 0; j < 2 * ns; ++j) A[c * 2 * ns + j] /= p;
        for (int r = 0; r < ns; ++r) {
            if (r == c) continue;
            double f = A[r * 2 * ns + c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * ns; ++j) A[r * 2 * ns + j] -= f * A[c * 2 * ns + j];
        }
    }
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) W[i * ns + j] = A[i * 2 * ns + ns + j];
    free(A);
    return rc;
}

/* v^s: sigmoid visibility of a landmark with unit bearing p at the sample axes */
static void gp_vs(const double* axes, int ns, double ks, double cos_alpha, const double p[3], double* vs) {
    for (int g = 0; g < ns; ++g) {
        double c = axes[3 * g] * p[0] + axes[3 * g + 1] * p[1] + axes[3 * g + 2] * p[2];
        vs[g] = 1.0 / (1.0 + exp(-ks * (c - cos_alpha)));
    }
}

/* v_p = W v^s(p) */
void or_gp_vp(const double* axes, int ns, const double* W, double ks, double cos_alpha, const double p[3], double* vp) {
    double vs[512];
    gp_vs(axes, ns, ks, cos_alpha, p, vs);
    for (int g = 0; g < ns; ++g) {
        double s = 0.0;
        for (int h = 0; h < ns; ++h) s += W[g * ns + h] * vs[h];
        vp[g] = s;
    }
}

/* v_r = K_z */
void or_gp_vr(const double* axes, int ns, double l, const double z[3], double* vr) {
    for (int g = 0; g < ns; ++g) vr[g] = se_kernel(z, axes + 3 * g, l);
}

/* v_gp(z) for a landmark of bearing p: K_z W v^s(p) */
double or_gp_visibility(const double* axes, int ns, const double* W, double l, double ks, double cos_alpha,
                        const double z[3], const double p[3]) {
    double vp[512], vr[512], s = 0.0;
    or_gp_vp(axes, ns, W, ks, cos_alpha, p, vp);
    or_gp_vr(axes, ns, l, z, vr);
    for (int g = 0; g < ns; ++g) s += vr[g] * vp[g];
    return s;
}

/* log marginal likelihood of M training vectors y_m over the sample axes (independent GP
 * draws on the same inputs): sum_m [-1/2 y_m^T K^-1 y_m] - M/2 log|K| - M ns/2 log(2 pi),
 * K = K^s + noise I (Rasmussen & Williams, Eq. 2.30) */
double or_gp_log_marginal(const double* axes, int ns, double l, double noise, const double* Y, int M) {
    double* W = (double*)malloc(sizeof(double) * (size_t)ns * ns);
    double* K = (double*)malloc(sizeof(double) * (size_t)ns * ns);
    for (int i = 0; i < ns; ++i)
        for (int j = 0; j < ns; ++j) K[i * ns + j] = se_kernel(axes + 3 * i, axes + 3 * j, l) + (i == j ? noise : 0.0);
    or_gp_weights(axes, ns, l, noise, W);
    /* log det by LU */
    double lad = 0.0;
    {
        double* A = (double*)malloc(sizeof(double) * (size_t)ns * ns);
        memcpy(A, K, sizeof(double) * (size_t)ns * ns);
        for (int c = 0; c < ns; ++c) {
            int piv = c;
            for (int r = c + 1; r < ns; ++r)
                if (fabs(A[r * ns + c]) > fabs(A[piv * ns + c])) piv = r;
            if (piv != c)
                for (int j = 0; j < ns; ++j) { double t = A[c * ns + j]; A[c * ns + j] = A[piv * ns + j]; A[piv * ns + j] = t; }
            double p = A[c * ns + c];
            lad += log(fabs(p));
            for (int r = c + 1; r < ns; ++r) {
                double f = A[r * ns + c] / p;
                for (int j = c; j < ns; ++j) A[r * ns + j] -= f * A[c * ns + j];
            }
        }
        free(A);
    }
    double quad = 0.0;
    for (int m = 0; m < M; ++m) {
        const double* y = Y + (size_t)m * ns;
        for (int i = 0; i < ns; ++i) {
            double s = 0.0;
            for (int j = 0; j < ns; ++j) s += W[i * ns + j] * y[j];
            quad += y[i] * s;
        }
    }
    free(W);
    free(K);
    return -0.5 * quad - 0.5 * M * lad - 0.5 * M * ns * log(2.0 * M_PI);
}

/* training vectors for the fit: the sigmoid visibility of landmarks with unit bearings P[m] */
void or_gp_training(const double* axes, int ns, double ks, double cos_alpha, const double* P, int M, double* Y) {
    for (int m = 0; m < M; ++m) gp_vs(axes, ns, ks, cos_alpha, P + 3 * m, Y + (size_t)m * ns);
}

typedef struct {
    const double* axes;
    const double* W;
    int32_t ns;
    int32_t pad_;
    double l, ks, cos_alpha;
} or_gp;

/* Field with GP visibility: C_g(c) = sum_{i in V_c} v_p,i[g] I_i (Eq. general_info_pif with
 * v_p = W v^s); out [cnt][ns][36] */
void or_field_nodes_gp(const float* lm, int64_t n, const or_grid* g, const or_params* prm, const or_gp* gp,
                       const int64_t* nodes, int64_t cnt, int about_node, double* out) {
    float rmin2 = (float)(prm->r_min * prm->r_min), rmax2 = (float)(prm->r_max * prm->r_max);
    const double Rid[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    const int ns = gp->ns;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < cnt; ++s) {
        int64_t node = nodes[s];
        int ix = (int)(node % g->nx), iy = (int)((node / g->nx) % g->ny), iz = (int)(node / ((int64_t)g->nx * g->ny));
        float cf[3] = {node_coord_f32((float)g->origin[0], (float)g->res, ix),
                       node_coord_f32((float)g->origin[1], (float)g->res, iy),
                       node_coord_f32((float)g->origin[2], (float)g->res, iz)};
        double c[3] = {cf[0], cf[1], cf[2]};
        double o[3] = {0, 0, 0};
        if (about_node) { o[0] = c[0]; o[1] = c[1]; o[2] = c[2]; }
        double* C = out + (size_t)36 * ns * s;
        memset(C, 0, sizeof(double) * 36 * ns);
        double vp[512];
        for (int64_t i = 0; i < n; ++i) {
            const float* pf = lm + 3 * i;
            if (!or_in_shell_f32(pf, cf, rmin2, rmax2)) continue;
            double pw[3] = {pf[0], pf[1], pf[2]};
            double d[3] = {pw[0] - c[0], pw[1] - c[1], pw[2] - c[2]};
            double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double u[3] = {d[0] / nn, d[1] / nn, d[2] / nn};
            double J[18], Ii[36];
            or_gp_vp(gp->axes, ns, gp->W, gp->ks, gp->cos_alpha, u, vp);
            or_jac_global(pw, Rid, c, o, J);
            or_fim_gauss(J, prm->sigma, Ii);
            for (int k = 0; k < ns; ++k)
                for (int e = 0; e < 36; ++e) C[36 * k + e] += vp[k] * Ii[e];
        }
    }
}

/* Query with GP visibility from world-frame corner sets [m][8][ns][36] */
void or_query_gp_batch(const double* corners, const double* w, const double* poses, int64_t m, const or_gp* gp,
                       int frame, double* out) {
    const int ns = gp->ns;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        const double* pose = poses + 7 * i;
        double q[4] = {pose[3], pose[4], pose[5], pose[6]}, R[9], t[3] = {pose[0], pose[1], pose[2]};
        or_quat_to_rot(q, R);
        double z[3] = {R[2], R[5], R[8]}, vr[512];
        or_gp_vr(gp->axes, ns, gp->l, z, vr);
        double Iw[36];
        memset(Iw, 0, sizeof(Iw));
        for (int j = 0; j < 8; ++j) {
            double wj = w[8 * i + j];
            if (wj == 0.0) continue;
            const double* Cj = corners + ((size_t)i * 8 + j) * 36 * ns;
            for (int k = 0; k < ns; ++k)
                for (int e = 0; e < 36; ++e) Iw[e] += vr[k] * wj * Cj[36 * k + e];
        }
        double* I = out + 36 * i;
        if (frame == OR_FRAME_WORLD) { memcpy(I, Iw, sizeof(Iw)); continue; }
        double Ad[36], AdT[36], tmp[36];
        adjoint_se3(R, t, Ad);
        transpose(Ad, AdT, 6, 6);
        matmul(AdT, Iw, tmp, 6, 6, 6);
        matmul(tmp, Ad, I, 6, 6, 6);
    }
}

/* Point-cloud FIM weighted by the GP visibility of each landmark (what the GP field reproduces
 * at a node): sum_i v_gp(z; u_i) I_i over the range shell around t */
void or_pc_fim_gp(const float* lm, int64_t n, const double* poses, int64_t m, const or_params* prm, const or_gp* gp,
                  int frame, double* out) {
    float rmin2 = (float)(prm->r_min * prm->r_min), rmax2 = (float)(prm->r_max * prm->r_max);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < m; ++j) {
        const double* pose = poses + 7 * j;
        double q[4] = {pose[3], pose[4], pose[5], pose[6]}, R[9], t[3] = {pose[0], pose[1], pose[2]};
        double o[3] = {0, 0, 0};
        or_quat_to_rot(q, R);
        double z[3] = {R[2], R[5], R[8]};
        float tf[3] = {(float)t[0], (float)t[1], (float)t[2]};
        double* I = out + 36 * j;
        memset(I, 0, 36 * sizeof(double));
        for (int64_t i = 0; i < n; ++i) {
            const float* pf = lm + 3 * i;
            if (!or_in_shell_f32(pf, tf, rmin2, rmax2)) continue;
            double pw[3] = {pf[0], pf[1], pf[2]};
            double d[3] = {pw[0] - t[0], pw[1] - t[1], pw[2] - t[2]};
            double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double u[3] = {d[0] / nn, d[1] / nn, d[2] / nn};
            double v = or_gp_visibility(gp->axes, gp->ns, gp->W, gp->l, gp->ks, gp->cos_alpha, z, u);
            double J[18], Ii[36];
            if (frame == OR_FRAME_CAMERA) or_jac_local(pw, R, t, J);
            else or_jac_global(pw, R, t, o, J);
            or_fim_gauss(J, prm->sigma, Ii);
            for (int e = 0; e < 36; ++e) I[e] += v * Ii[e];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Information threshold and potential cost (Sec. VI-B, Eq. info_pot_cost)     */
/* ------------------------------------------------------------------------- */

/* Information threshold (Sec. VI-B): n sets of M landmarks in the camera frame (camera at the
 * origin, optical axis +z), each satisfying the specification (in the FoV, d_min..d_max).  The
 * FIM a map representation gives for a set, at the camera:
 *   model 0, point cloud: every landmark counts (v = 1; all are in the FoV by construction);
 *   model 1, quadratic field: v = v_quad(cos theta) (Eq. quad_vis_approx) -- what a field built
 *            from the set returns when queried at the node the camera sits on (Eq. fim_separation);
 *   model 2, GP field: v = v_gp(e3; u) (Eq. gp_vis_approx), likewise;
 * I_s = sum_i v_i I_i with I_i the camera-frame information of one bearing (Eq. fim_gaussian,
 * local perturbation).  metrics[s] = (trace, log|det|, sign, lambda_min); the threshold of a
 * metric is its mean over the sets, over the well-conditioned ones only when
 * exclude_degenerate (the paper's remedy for degenerate configurations: det > 0 and
 * lambda_min > 1e-6 trace, a condition-number test above single-precision noise); NaN when
 * none count. */
void or_info_threshold(const float* sets, int64_t n, int M, const or_params* prm, int model, const or_gp* gp,
                       int exclude_degenerate, double* metrics /*[n][4]*/, double* thr /*[3]*/) {
    double kq[3];
    or_quad_coeffs(prm->half_fov, prm->v_alpha, kq);
    const double Rid[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, t0[3] = {0, 0, 0}, e3[3] = {0, 0, 1};
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t s = 0; s < n; ++s) {
        double I[36];
        memset(I, 0, sizeof(I));
        for (int i = 0; i < M; ++i) {
            const float* pf = sets + 3 * ((size_t)s * M + i);
            double p[3] = {pf[0], pf[1], pf[2]};
            double nn = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
            double u[3] = {p[0] / nn, p[1] / nn, p[2] / nn};
            double v = 1.0;
            if (model == 1) v = kq[2] * u[2] * u[2] + kq[1] * u[2] + kq[0];
            else if (model == 2) v = or_gp_visibility(gp->axes, gp->ns, gp->W, gp->l, gp->ks, gp->cos_alpha, e3, u);
            double J[18], Ii[36];
            or_jac_local(p, Rid, t0, J);
            or_fim_gauss(J, prm->sigma, Ii);
            for (int e = 0; e < 36; ++e) I[e] += v * Ii[e];
        }
        or_metrics(I, 1, metrics + 4 * s);
    }
    double sum[3] = {0, 0, 0};
    int64_t cnt = 0;
    for (int64_t s = 0; s < n; ++s) {
        const double* m4 = metrics + 4 * s;
        if (exclude_degenerate && !(m4[2] > 0.0 && m4[3] > 1e-6 * m4[0])) continue;
        sum[0] += m4[0]; sum[1] += m4[1]; sum[2] += m4[3];
        ++cnt;
    }
    for (int c = 0; c < 3; ++c) thr[c] = cnt ? sum[c] / (double)cnt : NAN;
}

/* Information potential cost (Eq. info_pot_cost) of metric values v with threshold eps > 0 and
 * k_q > 0:  c = 0 for v > eps;  k_q (v - eps)^2 for 0 <= v <= eps;  k_l v + b_l for v < 0, with
 * k_l, b_l making c and dc/dv continuous at v = 0: k_l = -2 k_q eps, b_l = k_q eps^2.  Readings:
 * the printed middle case's (v - c) is taken as (v - eps), and the continuity "at c = 0" as at
 * v = 0.  Also returns dc/dv.  NaN in, NaN out. */
void or_info_cost(const double* v, int64_t m, double eps, double kq, double* c, double* dc) {
    const double kl = -2.0 * kq * eps, bl = kq * eps * eps;
    for (int64_t i = 0; i < m; ++i) {
        const double x = v[i];
        if (x != x) { c[i] = x; dc[i] = x; }
        else if (x > eps) { c[i] = 0.0; dc[i] = 0.0; }
        else if (x >= 0.0) { c[i] = kq * (x - eps) * (x - eps); dc[i] = 2.0 * kq * (x - eps); }
        else { c[i] = kl * x + bl; dc[i] = kl; }
    }
}
