/*
 * fif.h -- C ABI of the GB300-native Fisher Information Field library (libfif.so).
 *
 * The method (Zhang & Scaramuzza, arXiv 2008.03324): precompute, once, a per-voxel
 * positional information factor from a sparse landmark map (Sec. VI-A-1,
 * Eq. general_info_pif), then recover the Fisher information of any camera pose in
 * constant time by contracting the factor with the camera's optical-axis monomials
 * (Eq. fim_separation, Eq. general_info_query) and reducing it to an information metric
 * (Sec. IV).  The direct point-cloud FIM (Eq. cost_info) is provided as the baseline.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Ownership: the caller allocates and frees every buffer, host or device, including the
 *   field storage and the build workspace.  The library never allocates device memory.
 * - Pointers named d_* are device pointers (cudaMalloc or torch tensors on the current
 *   device); all others are host pointers.  Device pointers must be 16-byte aligned.
 * - Asynchrony: compute entry points enqueue kernels on `stream` and return at once.
 *   Their return code reports argument and launch errors only; results are valid after
 *   the stream has been synchronised.  A NULL stream is the legacy default stream.
 * - Errors: every call returns FIF_OK (0) or a negative FIF_E* code; fif_status_str()
 *   names it.  Device-side failures never trap: per-pose problems go to the optional
 *   per-pose status array, and a bounded wait that runs out sets the library's device
 *   error word (fif_device_error()).
 * - Pose layout: float32[m][7] = (tx, ty, tz, qw, qx, qy, qz); the quaternion gives R_wc
 *   (camera to world), t = camera centre in the world.  Non-unit quaternions are
 *   renormalised.
 * - Perturbation order: xi = (rho, phi), translation first, as in [-I3, [p]x]
 *   (Eq. jac_pose_global).
 * - A symmetric 6x6 matrix is stored as its 21 upper-triangular entries in row-major
 *   order: (0,0) (0,1) .. (0,5) (1,1) .. (1,5) (2,2) .. (5,5).
 * - Thread safety: calls on different fields may run concurrently; concurrent builds
 *   into the same field race.
 */
#ifndef FIF_H_
#define FIF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FIF_API __attribute__((visibility("default")))
#else
#define FIF_API
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* fif_stream_t;

/* ---- return codes ------------------------------------------------------------------ */
#define FIF_OK 0
#define FIF_EINVAL (-1)    /* a NULL pointer, a non-positive size, an unknown flag       */
#define FIF_ESIZE (-2)     /* a caller buffer is smaller than the call needs             */
#define FIF_EALIGN (-3)    /* a device pointer is not 16-byte aligned                    */
#define FIF_ECUDA (-4)     /* a CUDA launch or runtime call failed                       */
#define FIF_ETIMEOUT (-5)  /* a bounded device wait ran out (see fif_device_error)       */
#define FIF_EIO (-6)       /* file could not be opened, read or written                  */
#define FIF_EFORMAT (-7)   /* file is not a field of this version / size / layout        */
#define FIF_ERANGE (-8)    /* a size exceeds a fixed maximum of the call                 */

/* ---- per-pose status bits (d_status) ------------------------------------------------ */
#define FIF_POSE_OUTSIDE 1   /* position outside the lattice box; clamped onto it        */
#define FIF_POSE_QUAT 2      /* |q|^2 differed from 1 by more than 1e-3; renormalised    */
#define FIF_POSE_NOT_PD 4    /* the FIM is not positive definite (sign <= 0 or l_min <= 0)*/
#define FIF_POSE_NAN 8       /* non-finite pose; outputs are NaN                         */

/* ---- storage of the field ------------------------------------------------------------ */
#define FIF_STORAGE_F32 0    /* float32, 216 elements (864 B) per node                  */
#define FIF_STORAGE_BF16 1   /* bfloat16 (round to nearest even), 224 elements (448 B),   */
                             /* monomial blocks of 22 elements (see fif_field)            */
#define FIF_STORAGE_GP 3     /* GP visibility (Sec. V-B-2): float32, per node the 21 x N_s  */
                             /* matrix of D_g (see fif_gp), entry e of D_g at e*rs + g with  */
                             /* rs = fif_gp_row_stride(N_s); fif_gp_stride(N_s) per node     */
#define FIF_STORAGE_TRACE 2  /* the positional trace factor of Sec. VI-A-2 (Eq.             */
                             /* general_trace_pif): float32 tr(C_k^world), k = 0..9, plus 2 */
                             /* zero pads = 12 elements (48 B) per node; fif_query then      */
                             /* returns only the world-frame trace (FIF_Q_TRACE | FIF_Q_WORLD)*/

/* ---- query flags ---------------------------------------------------------------------- */
#define FIF_Q_TRILINEAR 0x0  /* interpolate over the 8 surrounding nodes (default)        */
#define FIF_Q_NEAREST 0x1    /* nearest node only (the paper's "FIM from nearest voxel")  */
#define FIF_Q_CAMERA 0x0     /* FIM in the camera frame, local perturbation (default)     */
#define FIF_Q_WORLD 0x2      /* FIM in the world frame, global perturbation about origin  */
#define FIF_Q_GP_COMPENSATED 0x4 /* GP field only: compensated contraction (see fif_query)   */
#define FIF_Q_TRACE 0x10     /* compute trace            (metrics column 0)               */
#define FIF_Q_LOGDET 0x20    /* compute log|det| + sign  (metrics column 1, d_sign)       */
#define FIF_Q_LMIN 0x40      /* compute lambda_min       (metrics column 2)               */
#define FIF_Q_METRICS 0x70   /* all three                                                 */

/* Lattice of voxel nodes: node (i, j, k) sits at origin + res * (i, j, k), i < nx, j < ny,
 * k < nz, each count >= 2.  Node index n = i + nx * (j + ny * k). */
typedef struct fif_grid {
    float origin[3];
    float res;
    int32_t nx, ny, nz;
} fif_grid;

/* Parameters of the method.
 * half_fov, v_alpha: the quadratic visibility v(theta) = k2 cos^2 + k1 cos + k0 meets
 *   v(0) = 1, v(pi) = 0, v(half_fov) = v_alpha (Eq. quadratic_conditions, Sec. V-B-1).
 * r_min, r_max: the landmarks seen from a position x are those with
 *   r_min < |p - x| <= r_max (the set V_t of Sec. V; the paper leaves its choice to the
 *   map, this library uses a range shell).  The test is taken in single precision:
 *   dx = p - x per axis, n2 = (dx*dx + dy*dy) + dz*dz, each operation rounded, compared
 *   with (float)(r_min*r_min) and (float)(r_max*r_max).
 * sigma: bearing noise std (Eq. fim_gaussian); every FIM is scaled by 1/sigma^2.
 * bin_size: edge of the cubic cells used to cull landmarks during the build (metres,
 *   0 selects 1.0).  It changes speed only, never results. */
typedef struct fif_params {
    double half_fov;
    double v_alpha;
    double r_min;
    double r_max;
    double sigma;
    float bin_size;
    int32_t reserved;
} fif_params;

/* Pinhole camera for the exact visibility of the point-cloud baseline
 * (Eq. exact_vis_func): a landmark is visible iff its camera-frame depth z > 0 and
 * fx*x + cx*z lies in [0, width*z) and fy*y + cy*z lies in [0, height*z), all in single
 * precision with one rounding per operation, i.e. its pixel lies inside the image. */
typedef struct fif_pinhole {
    float fx, fy, cx, cy;
    int32_t width, height;
} fif_pinhole;

/* GP visibility model (Sec. V-B-2, Eq. sigmoid_vis_func, Eq. gp_vis_approx).  The visibility of
 * a landmark with unit bearing u seen along the optical axis z is the GP regression mean
 *   v_gp(z) = K_z (K^s + noise_var I)^-1 v^s(u),
 *   v^s_g(u) = 1 / (1 + exp(-k_s (z_g . u - cos alpha)))   (the sigmoid visibility at axis z_g),
 *   K_z[g] = exp(-|z - z_g|^2 / (2 l^2)),  K^s[g][h] = exp(-|z_g - z_h|^2 / (2 l^2)),
 * over N_s sample optical axes z_g (the printed Eq. gp_vis_approx omits the inverse of K^s; it
 * is read as in Eq. gp_regress).  alpha is params.half_fov.
 * Storage: a GP field keeps, per node, D_g = sum_i v^s_g(u_i) I_i (every weight in (0, 1); I_i
 * about the node as for the quadratic field) and the query applies the kriging weights
 *   a(z) = (K^s + noise_var I)^-1 K_z^T   (double-precision kernel values, compensated sums),
 *   I = sum_g a_g(z) D_g = K_z (K^s + noise_var I)^-1 D = V_I C_I of Eq. fim_separation.
 * The paper's C_I = (K^s)^-1 D is never stored: its entries grow with the condition number of
 * K^s, and single-precision storage of them loses up to four digits in the query. */
#define FIF_GP_MAX_SAMPLES 96
typedef struct fif_gp {
    int32_t n_samples;                      /* N_s, 1 .. FIF_GP_MAX_SAMPLES                  */
    int32_t reserved;
    double length_scale;                    /* l                                              */
    double noise_var;                       /* added to the diagonal of K^s (paper: 1e-10)    */
    double k_s;                             /* sigmoid sharpness (paper: 15)                  */
    double axes[FIF_GP_MAX_SAMPLES][3];     /* sample optical axes z_g (normalised on upload) */
    void* d_aux;                            /* device buffer filled by fif_gp_upload           */
} fif_gp;

/* A field: the lattice, the method's parameters and the caller-owned device storage.
 * Storage layout: node n occupies elements [n*stride, (n+1)*stride) of `coeffs`; element
 * n*stride + 21*k + e holds entry e (upper-triangular, row-major) of the 6x6 matrix
 * C_k = sum_i v_p(u_i)[k] I_i, k indexing the monomials of Eq. quad_vis_component,
 * v_p = [u1^2, u2^2, u3^2, u1 u2, u1 u3, u2 u3, u1, u2, u3, 1], u_i the unit bearing
 * from the node to landmark i, I_i its information (Eq. global_fim_eq) with the
 * rotational part of the perturbation taken about the node itself (the paper's world
 * frame moved to the node: C^world = M_c^T C M_c, M_c = [[I, -[c]x], [0, I]]).
 * Elements 210 .. stride-1 are zero.  FIF_STORAGE_BF16 spaces the blocks by 22 instead: entry e
 * of C_k at n*stride + 22*k + e, with zeros at 22*k + 21 and at 220 .. 223 (so that a 32-bit word
 * holds two entries of one block).  With FIF_STORAGE_TRACE, node n holds instead the 10 traces
 * tr(C_k^world) (world frame: rotation about the origin) at n*12 + k, then two zeros.
 * k[] = (k0, k1, k2) is filled by fif_field_init. */
typedef struct fif_field {
    fif_grid grid;
    fif_params params;
    int32_t storage;   /* FIF_STORAGE_*                                              */
    int32_t stride;    /* elements per node                                         */
    void* coeffs;      /* device storage, caller-owned                              */
    size_t bytes;      /* size of `coeffs` in bytes                                 */
    double k[3];       /* k0, k1, k2                                                */
    fif_gp gp;         /* GP model (FIF_STORAGE_GP only)                             */
} fif_field;

/* Library version (major*10000 + minor*100 + patch). */
FIF_API int32_t fif_version(void);

/* Static name of a return code. */
FIF_API const char* fif_status_str(int32_t code);

/* Bytes of field storage for `grid` with the given storage type (0 on a bad argument; for
 * FIF_STORAGE_GP use fif_gp_field_bytes). */
FIF_API size_t fif_field_bytes(const fif_grid* grid, int32_t storage);

/* Fill *field: validate grid and params, solve (k0, k1, k2) from Eq. quadratic_conditions
 * in double precision, and bind the caller's device storage d_coeffs of `bytes` bytes
 * (at least fif_field_bytes()).  Host only; does not touch the storage. */
FIF_API int32_t fif_field_init(fif_field* field, const fif_grid* grid, const fif_params* params,
                       int32_t storage, void* d_coeffs, size_t bytes);

/* Row stride rs of a GP node record: the smallest count >= n_samples that is 2 more than a
 * multiple of 4 (0 on a bad count).  Entry e of D_g sits at e*rs + g; pads are zero. */
FIF_API int32_t fif_gp_row_stride(int32_t n_samples);

/* Elements per node of a GP field: 21 rs rounded up to a multiple of 4 (16-byte records). */
FIF_API int32_t fif_gp_stride(int32_t n_samples);

/* Bytes of the GP model's device buffer d_aux. */
FIF_API size_t fif_gp_aux_bytes(int32_t n_samples);

/* Prepare the model for device use: normalise the axes, compute W = (K^s + noise_var I)^-1 on
 * the host in double precision (Cholesky factorisation, then the inverse from the factor),
 * and copy W (split into single-precision high and low parts) and the axes into the caller's
 * device buffer d_aux (bytes >= fif_gp_aux_bytes(n_samples)); sets gp->d_aux.  Synchronises
 * `stream`.  FIF_EINVAL on a bad count, axis, length scale, noise or k_s, or when
 * K^s + noise_var I is not positive definite in double precision. */
FIF_API int32_t fif_gp_upload(fif_gp* gp, void* d_aux, size_t bytes, fif_stream_t stream);

/* Length scale by maximum marginal likelihood (Sec. V-B-2; Rasmussen and Williams Eq. 2.30):
 * training vectors y_m = v^s(p_m) for m unit bearings p_m (host double [m][3]) at the N_s
 * axes of gp, independent draws, maximise over l in [l_lo, l_hi]
 *   L(l) = sum_m -1/2 y_m^T (K^s_l + noise_var I)^-1 y_m - m/2 log|K^s_l + noise_var I|
 * by a scan of 97 log-spaced points, then golden-section refinement of the best bracket to a
 * relative width of 1e-7.  Host only, double precision (Cholesky).  gp->length_scale is
 * ignored; the maximiser is written to *l_out. */
FIF_API int32_t fif_gp_fit_length_scale(const fif_gp* gp, double half_fov, const double* bearings, int32_t m,
                                        double l_lo, double l_hi, double* l_out);

/* Bytes of GP field storage for `grid` and n_samples axes (0 on a bad argument). */
FIF_API size_t fif_gp_field_bytes(const fif_grid* grid, int32_t n_samples);

/* fif_field_init for a GP field (storage FIF_STORAGE_GP): gp must have been uploaded
 * (fif_gp_upload); the field keeps a copy of the struct, and gp->d_aux must stay valid while
 * the field is used.  params.v_alpha is unused.  fif_build, fif_build_update and fif_query
 * accept the field; fif_query_backward, fif_field_save and fif_build_static return FIF_EINVAL. */
FIF_API int32_t fif_field_init_gp(fif_field* field, const fif_grid* grid, const fif_params* params,
                                  const fif_gp* gp, void* d_coeffs, size_t bytes);

/* Bytes of device workspace fif_build() needs for n landmarks (0 on a bad argument). */
FIF_API size_t fif_build_workspace_bytes(const fif_field* field, int64_t n_landmarks);

/* Build the field (Sec. VI-A-1, Eq. general_info_pif): for every node c,
 *   C_k(c) = sum over landmarks with r_min < |p_i - c| <= r_max of v_p(u_i)[k] * I_i.
 * d_landmarks: float32[n][3] world positions.  d_workspace: at least
 * fif_build_workspace_bytes(field, n) bytes, contents on entry ignored.  Sums are taken
 * in single precision with compensated (Kahan) accumulation over blocks of landmarks;
 * the summation order is fixed by the input order, so equal inputs give bitwise equal
 * fields.  Overwrites the whole storage.  n may be 0 (the field becomes zero).
 * GP field (FIF_STORAGE_GP): the same reduction with weights v^s_g(u_i) gives D_g for every
 * sample axis g (single-precision bearings and sigmoid: ex2 / rcp approximations, relative
 * error of each weight below 3e-6). */
FIF_API int32_t fif_build(fif_field* field, const float* d_landmarks, int64_t n, void* d_workspace,
                  size_t workspace_bytes, fif_stream_t stream);

/* Online update of a built field (Sec. VI-A-1: the positional factor is a sum of one term per
 * landmark, so adding or deleting a landmark adds or subtracts its term).  sign = +1 adds the
 * n landmarks' contributions to every node they reach, sign = -1 removes them; nodes farther than
 * r_max from all of them are not touched.  The same arithmetic as fif_build (the delta of the n
 * landmarks is summed with compensation, then added to each stored coefficient in single
 * precision, or rounded back to bfloat16 for that storage); moving a landmark is a removal
 * followed by an addition.  Workspace as for fif_build with n landmarks. */
FIF_API int32_t fif_build_update(fif_field* field, const float* d_landmarks, int64_t n, int32_t sign,
                                 void* d_workspace, size_t workspace_bytes, fif_stream_t stream);

/* Build only the nodes of one z-slab of the lattice, k_begin <= k < k_end (0 <= k_begin < k_end <=
 * nz).  Sec. VI-A-1: each node's factor is a sum over the landmarks in its own range shell and
 * depends on no other node, so the lattice splits into slabs that separate GPUs build apart (one
 * replica each then gathers the slabs).  Nodes outside the slab are not touched.  Every slab node
 * gets bitwise the coefficients fif_build gives it from the same landmark array; for the quadratic
 * and trace fields also from any sub-array, in the same relative order, that keeps every landmark
 * whose z lies in the band of fif_slab_landmark_band (a GP field only to rounding then).  Workspace
 * as for fif_build with n landmarks. */
FIF_API int32_t fif_build_slab(fif_field* field, int32_t k_begin, int32_t k_end, const float* d_landmarks,
                               int64_t n, void* d_workspace, size_t workspace_bytes, fif_stream_t stream);

/* The band z_lo <= z <= z_hi (world z, as float32) holding every landmark that the build of slab
 * [k_begin, k_end) can use: the node layers of the slab's bricks widened by the build's cull radius
 * (r_max + 0.01 + 1e-4 r_max) and a rounding margin.  Host only; FIF_EINVAL on a bad range. */
FIF_API int32_t fif_slab_landmark_band(const fif_field* field, int32_t k_begin, int32_t k_end, float* z_lo,
                                       float* z_hi);

/* Size of the fixed device scratch array that fif_build_static uses (16 MiB). */
#define FIF_BUILD_STATIC_SCRATCH_BYTES (16u << 20)

/* fif_build without a workspace argument, for callers that cannot allocate device memory
 * once they run (for example a planner loaded as a plug-in into an application whose own
 * allocator owns the GPU memory, or a real-time loop that forbids cudaMalloc after start-up
 * because it may synchronise the device and take unbounded time).  The paper has no
 * counterpart: this is a library convenience.
 * The build's scratch lives in one fixed array of FIF_BUILD_STATIC_SCRATCH_BYTES inside the
 * library, present on every GPU that loads the library until the process exits.  Results
 * are those of fif_build.  Returns FIF_ERANGE, without launching anything, when n landmarks
 * on this field need more scratch than that (fif_build_workspace_bytes(field, n) > the
 * maximum; about 768,000 landmarks for the 200 x 200 x 40 warehouse lattice).  The first call on a device
 * looks up the array's device address (once per device, with that device current); make that
 * first call before any stream capture.  All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and corrupt each other's fields;
 * serialise them.  Calls no allocator. */
FIF_API int32_t fif_build_static(fif_field* field, const float* d_landmarks, int64_t n, fif_stream_t stream);

/* Query m poses (Sec. VI-A-1, Eq. fim_separation, Eq. general_info_query):
 *   I(T) = sum_k v_r(z)[k] * C_k(t),  z = R_wc e3 (the optical axis),
 * v_r = [k2 z1^2, k2 z2^2, k2 z3^2, 2 k2 z1 z2, 2 k2 z1 z3, 2 k2 z2 z3, k1 z1, k1 z2, k1 z3, k0]
 * with C_k(t) interpolated trilinearly from the 8 nodes around t (or taken from the
 * nearest node), expressed in the camera frame (Ad^T I_world Ad, the local perturbation)
 * or the world frame, then reduced to the metrics selected in `flags`.
 * Outputs (each optional, NULL to skip):
 *   d_fim      float32[m][21]  the 6x6 FIM, upper triangle
 *   d_metrics  float64[m][3]   trace, log|det|, lambda_min (unselected columns untouched)
 *   d_sign     int8[m]         sign of det (+1, -1, 0)
 *   d_status   int32[m]        FIF_POSE_* bits
 * Trace is summed in single precision; log|det| comes from a double-precision LU with partial
 * pivoting of the FIM, and lambda_min is the double-precision Rayleigh quotient of the eigenvector
 * that single-precision inverse iteration finds (its shift from bisection on the Sturm counts of
 * a Householder tridiagonal form).
 * Positions outside the lattice are clamped onto it.  m = 0 returns FIF_OK and touches nothing
 * (every pointer may then be NULL).
 * GP field (FIF_STORAGE_GP): I(T) = sum_g a_g(z) D_g(t) with the kriging weights
 *   a(z) = (K^s + noise_var I)^-1 K_z^T (K_z in double precision, the product as compensated
 *   single-precision sums with W split into high and low parts), D_g interpolated as above.
 *   The weights change sign and cancel, so the single-precision contraction sum_g a_g D_g loses
 *   digits in proportion to kappa = sum_g |a_g| ||D_g|| / ||I|| (at most about 16 u kappa relative,
 *   u = 2^-24); with FIF_Q_GP_COMPENSATED it is a compensated dot product (Dot2) and the query's
 *   error stays within about 2 u kappa (the storage and weight roundings), at roughly half the
 *   throughput.  The flag is FIF_EINVAL for other storage. */
FIF_API int32_t fif_query(const fif_field* field, const float* d_poses, int64_t m, int32_t flags,
                  float* d_fim, double* d_metrics, int8_t* d_sign, int32_t* d_status,
                  fif_stream_t stream);

/* Bytes of device staging fif_query_host() needs for chunks of `chunk` poses: two buffers,
 * each holding a chunk's poses and every output (141 B per pose, each array 256-B aligned).
 * 0 when chunk <= 0. */
FIF_API size_t fif_query_host_staging_bytes(int64_t chunk);

/* fif_query over HOST buffers.  h_poses (float32[m][7]) and the outputs h_fim, h_metrics,
 * h_sign, h_status (layouts and NULL meaning as for fif_query) are host memory; page-locked
 * memory lets the copies run asynchronously and overlap the queries.  The poses go through
 * the device in pieces of at most `chunk` poses (a quarter chunk first and last, to shorten the
 * copies not overlapped by a query), double-buffered in d_staging (caller-owned, at least
 * fif_query_host_staging_bytes(chunk) bytes, 16-byte aligned): chunk c's host-to-device copy
 * and chunk c-1's device-to-host copy run on copy_stream while chunk c-1 or c is queried on
 * `stream`, ordered by events (created and released inside the call); the first copy waits for
 * the work already queued on `stream`.  Each pose's results are
 * those fif_query gives it.  Asynchronous: the host outputs are complete once `stream` has
 * completed (it waits for the last copy); h_poses and the outputs must stay valid until then.
 * copy_stream must differ from stream (FIF_EINVAL otherwise).  m = 0 returns FIF_OK and
 * touches nothing.
 * When h_poses and every non-NULL output are page-locked memory the device can address
 * (cudaHostAlloc / cudaMallocHost memory, mapped on every system with unified addressing), the
 * arguments are checked as above and then fif_query runs on those buffers in place: its kernels
 * read the poses from host memory and write the results there over the host link, with no
 * staging copies (d_staging and copy_stream are not used; the results are the same). */
FIF_API int32_t fif_query_host(const fif_field* field, const float* h_poses, int64_t m, int32_t flags,
                               float* h_fim, double* h_metrics, int8_t* h_sign, int32_t* h_status,
                               int64_t chunk, void* d_staging, size_t staging_bytes, fif_stream_t stream,
                               fif_stream_t copy_stream);

/* Adjoint of fif_query for the metrics (FIF_Q_CAMERA or FIF_Q_WORLD, trilinear):
 *   d_grad_pose[i] = sum_c d_grad_metrics[i][c] * d metric_c(T_i) / d(t, phi)
 * with t the world position and phi a right (camera-frame) so(3) perturbation
 * R <- R exp(phi^).  d_fim must hold the FIM that fif_query wrote for the same poses,
 * field and flags.  d_grad_metrics float64[m][3] (trace, log|det|, lambda_min weights; a
 * zero weight skips that metric), d_grad_pose float32[m][6] = (dt_x, dt_y, dt_z, dphi_x,
 * dphi_y, dphi_z).  lambda_min's derivative assumes a simple smallest eigenvalue.  Poses
 * clamped onto the lattice get a zero derivative along the clamped axes. */
FIF_API int32_t fif_query_backward(const fif_field* field, const float* d_poses, int64_t m, int32_t flags,
                           const float* d_fim, const double* d_grad_metrics, float* d_grad_pose,
                           fif_stream_t stream);

/* Direct point-cloud FIM (Sec. IV, Eq. cost_info) -- the baseline the field replaces:
 *   I(T) = sum over landmarks with r_min < |p - t| <= r_max and exact pinhole visibility
 *          (Eq. exact_vis_func) of I_T(p)
 * over all n landmarks for each of m poses, in the frame selected by `flags`
 * (FIF_Q_CAMERA / FIF_Q_WORLD), with the same optional outputs and metrics as fif_query
 * (the status bit FIF_POSE_OUTSIDE is never set).  params supplies r_min, r_max, sigma. */
FIF_API int32_t fif_pointcloud_fim(const float* d_landmarks, int64_t n, const fif_params* params,
                           const fif_pinhole* camera, const float* d_poses, int64_t m,
                           int32_t flags, float* d_fim, double* d_metrics, int8_t* d_sign,
                           int32_t* d_status, fif_stream_t stream);

/* ---- information threshold and potential cost (Sec. VI-B) ------------------------------ */
#define FIF_MODEL_POINTCLOUD 0   /* the point cloud: every landmark of a set counts (v = 1)     */
#define FIF_MODEL_QUAD 1         /* a quadratic-visibility field (v = v_quad(cos theta))        */
#define FIF_MODEL_GP 2           /* a GP-visibility field (v = v_gp(e3; u))                     */

/* Information threshold (Sec. VI-B): the metric a map representation gives, averaged over
 * sets of landmarks that meet a localisation specification (M landmarks in the field of view
 * at distances d_min..d_max; the caller draws them).  d_sets: float32 [n_sets][m][3], each
 * set in the camera frame (camera at the origin looking along +z).  For every set
 *   I_s = sum_i v(u_i) I_i / sigma^2,  I_i = [[P/n^2, -[u]x/n], [[u]x/n, P]]  (camera frame),
 * with v from `model` (for a field this is what the field built from the set returns at the
 * node the camera sits on, Eq. fim_separation), then d_metrics[s] = (trace, log|det|,
 * lambda_min) as fif_query computes them, d_sign[s] = sign of det (optional).  No range shell
 * is applied.  d_threshold (device float64[3], optional): the mean of each metric over the
 * sets, only over sets with lambda_min > 1e-6 trace when exclude_degenerate (the paper's
 * remedy for degenerate configurations), NaN when no set counts; summed in a fixed order
 * (bitwise reproducible).  params supplies half_fov, v_alpha and sigma; gp (host struct, axes,
 * length scale, noise, k_s; no upload needed) is required for FIF_MODEL_GP, ignored otherwise.
 * 1 <= m; n_sets may be 0 (thresholds NaN). */
FIF_API int32_t fif_info_threshold(const fif_params* params, int32_t model, const fif_gp* gp, const float* d_sets,
                                   int64_t n_sets, int32_t m, int32_t exclude_degenerate, double* d_metrics,
                                   int8_t* d_sign, double* d_threshold, fif_stream_t stream);

/* Information potential cost (Eq. info_pot_cost) of metric values v (d_values[i * stride],
 * float64, e.g. a column of fif_query's d_metrics with stride 3):
 *   c = 0 for v > eps;  k_q (v - eps)^2 for 0 <= v <= eps;  k_l v + b_l for v < 0,
 * with k_l = -2 k_q eps and b_l = k_q eps^2 so that c and dc/dv are continuous at v = 0
 * (readings of the garbled equation: the middle case is taken as (v - eps)^2 and the continuity
 * condition at v = 0).  d_cost, d_dcost: float64[m] (either may be NULL); NaN values give NaN.
 * eps > 0, k_q > 0. */
FIF_API int32_t fif_info_cost(const double* d_values, int64_t m, int64_t stride, double eps, double k_q,
                              double* d_cost, double* d_dcost, fif_stream_t stream);

/* Save the field to a file: a fixed header (magic, version, grid, params, storage,
 * stride, FNV-1a checksum of the payload) followed by the raw storage.  Synchronises
 * `stream` and copies through `host_staging` (at least field->bytes bytes, caller-owned;
 * NULL uses pageable copies). */
FIF_API int32_t fif_field_save(const fif_field* field, const char* path, void* host_staging,
                       fif_stream_t stream);

/* Load a field saved by fif_field_save into caller device storage d_coeffs (bytes at least
 * the saved size); fills *field.  Verifies magic, version, sizes and checksum.  Synchronises
 * `stream`. */
FIF_API int32_t fif_field_load(fif_field* field, const char* path, void* d_coeffs, size_t bytes,
                       void* host_staging, fif_stream_t stream);

/* Read (and if reset != 0 clear) the library's device error word on the current device:
 * 0 when no bounded device wait has run out since the last reset.  Synchronises `stream`. */
FIF_API int32_t fif_device_error(int32_t* out_code, int32_t reset, fif_stream_t stream);

/* Limit, in nanoseconds of the GPU's global timer, of every bounded device wait in the kernels
 * launched after this call by fif_query on FIF_STORAGE_F32 / FIF_STORAGE_BF16 fields (and so
 * fif_query_host), fif_build, fif_build_update and fif_build_static: a bulk copy's completion, a
 * hand-over between warps, a slot of the landmark ring.  0 restores the default, 2 s.  A wait that
 * runs out makes its block record FIF_ETIMEOUT in the device error word (fif_device_error), wait
 * (at most 0.1 s more) for the copies it has issued, and return, leaving that launch's results
 * incomplete; the context stays usable.  Process-wide (all devices and threads).  Callers keep the
 * default; a limit far below the time one copy or hand-over takes forces the failure path, which is
 * how that path is tested.  Always FIF_OK. */
FIF_API int32_t fif_set_wait_limit(uint64_t limit_ns);

#ifdef __cplusplus
}
#endif
#endif /* FIF_H_ */
