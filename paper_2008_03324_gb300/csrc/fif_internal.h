// fif_internal.h -- launch interfaces between the C ABI (fif_abi.cu) and the kernel files.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fif.h"

namespace fif {

// ---- query ---------------------------------------------------------------------------
struct QueryArgs {
    const void* coeffs;
    int storage;
    int stride;
    float ox, oy, oz, res;
    int nx, ny, nz;
    float k0, k1, k2;
    const float* poses;
    int64_t m;
    int flags;
    float* fim;
    double* metrics;
    int8_t* sign;
    int32_t* status;
    int* err;
    uint64_t wait_ns;          // limit of each bounded device wait (fif_set_wait_limit)
    // GP visibility field (storage FIF_STORAGE_GP)
    int gp_ns, gp_rs;
    const float4* gp_axes;     // [2][ns]: axes as (high, low) single-precision parts (x, y, z, 0)
    const float2* gp_wt;       // [ns][rs]: (high, low) single-precision parts of W[g][h] at h * rs + g
    const float4* gp_consts;   // [9]: exp constants and table (see gp_model.cu)
};
int launch_query(const QueryArgs& a, cudaStream_t stream);
int launch_gp_query(const QueryArgs& a, cudaStream_t stream);
int launch_trace_query(const QueryArgs& a, cudaStream_t stream);

// ---- query adjoint -------------------------------------------------------------------
struct AdjointArgs {
    const void* coeffs;
    int storage;
    int stride;
    float ox, oy, oz, res;
    int nx, ny, nz;
    float k0, k1, k2;
    const float* poses;
    int64_t m;
    int flags;
    const float* fim;
    const double* gm;
    float* grad;
    int* err;
};
int launch_adjoint(const AdjointArgs& a, cudaStream_t stream);

// ---- build ---------------------------------------------------------------------------
struct BinGrid {
    float lo[3];     // corner of bin (0,0,0)
    float size;      // bin edge
    float inv_size;
    int n[3];        // bins per axis
};

struct BuildLayout {
    size_t sorted;   // float4[n]  (x, y, z, input index bits) while sorting, then (x, y, z, z)
    size_t binof;    // int32[n]
    size_t count;    // int32[nbins]  (count, then cursor)
    size_t start;    // int32[nbins + 1]
    size_t stats;    // uint64[4]  (in-shell pairs, candidate pairs, dropped landmarks, -)
    size_t total;
};

// z-depth (node layers) of the bricks a CTA of the quadratic / trace build and of the GP build owns
constexpr int kBuildBrickZ = 4;
constexpr int kGpBuildBrickZ = 2;

BinGrid make_bin_grid(const fif_field* f);
BuildLayout build_layout(const BinGrid& bg, int64_t n);

struct BuildArgs {
    const float* landmarks;
    int64_t n;
    unsigned char* ws;
    BuildLayout lay;
    BinGrid bg;
    float ox, oy, oz, res;
    int nx, ny, nz;
    float rmin2, rmax2, rcull;
    float inv_sigma2;
    int storage;
    int stride;
    void* out;
    int* err;
    int accumulate;   // 0: overwrite the field; +1 / -1: add / subtract these landmarks' share
    uint64_t wait_ns; // limit of each bounded device wait (fif_set_wait_limit)
    int k_begin, k_end;   // only nodes with k_begin <= k < k_end are built (a z-slab; 0, nz: all)
    // GP visibility field (storage FIF_STORAGE_GP): v^s_g = 1 / (1 + 2^(gp_shift - gp_scale z_g.u))
    const float4* gp_axes;    // [ns] (x, y, z, 0)
    int gp_ns, gp_rs;
    float gp_scale;           // k_s log2(e)
    float gp_shift;           // k_s log2(e) cos(alpha)
};
int launch_build(const BuildArgs& a, cudaStream_t stream);
// counting sort of the landmarks into the bins of a.bg (fills the workspace layout a.lay)
int launch_binning(const BuildArgs& a, cudaStream_t stream);
int launch_gp_build(const BuildArgs& a, cudaStream_t stream);

// GP model buffer (fif_gp.d_aux): offsets in bytes
struct GpAuxLayout {
    size_t axes_f;   // float4[ns]
    size_t axes_df;  // float4[2][ns]: high parts, then low parts
    size_t wt;       // float2[ns][rs] (high, low)
    size_t consts;   // float4[9]: (C1, C2, C3, 32/ln2), (1/l^2 high, low, 0, 0), then 2^(j/32) for
                     // j = 0..31 as (high, low) pairs, two per float4
    size_t total;
};
GpAuxLayout gp_aux_layout(int ns, int rs);

// ---- point cloud ---------------------------------------------------------------------
struct PointCloudArgs {
    const float* landmarks;
    int64_t n;
    float rmin2, rmax2;
    float inv_sigma2;
    float fx, fy, cx, cy, W, H;
    const float* poses;
    int64_t m;
    int flags;
    float* fim;
    double* metrics;
    int8_t* sign;
    int32_t* status;
};
int launch_pointcloud(const PointCloudArgs& a, cudaStream_t stream);

// ---- information threshold and potential cost ---------------------------------------
struct InfoArgs {
    const float* sets;     // [n][m][3] camera frame
    int64_t n;
    int m;
    int model;             // FIF_MODEL_*
    float inv_sigma2;
    float k0, k1, k2;      // quadratic visibility
    // GP visibility at the optical axis e3: v = sum_s gp_a[s] / (1 + exp(-ks (axes[s] . u - cos_alpha)))
    int gp_ns;
    float gp_ks, gp_cos_alpha;
    float gp_a[FIF_GP_MAX_SAMPLES];
    float gp_axes[FIF_GP_MAX_SAMPLES][3];
    double* metrics;       // [n][3]
    int8_t* sign;          // [n] or null
};
int launch_info_threshold(const InfoArgs& a, int exclude, double* d_threshold, cudaStream_t stream);
int launch_info_cost(const double* v, int64_t m, int64_t stride, double eps, double kq, double* cost, double* dcost,
                     cudaStream_t stream);

// the kriging weights a(z) = (K^s + noise I)^-1 K_z of a GP model (host, double precision);
// FIF_EINVAL when the model is invalid or K^s + noise I is not positive definite
int gp_kriging_weights(const fif_gp* gp, const double z[3], double* a);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace fif
