// fif_abi.cu -- the extern "C" entry points declared in include/fif.h: argument checks,
// launch configuration, field files and the device error word.  No device allocation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "fif_internal.h"

namespace {

// first bounded-wait failure seen by any kernel on this device (per device copy)
__device__ int g_device_error = 0;

constexpr int32_t kVersion = 10100;  // 1.1.0: bfloat16 records in monomial blocks of 22
constexpr uint64_t kDefaultWaitNs = 2000000000ull;   // 2 s
// limit of every bounded device wait in the kernels launched from now on (fif_set_wait_limit)
std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};
constexpr int kMaxDevices = 64;
int* g_err_ptr[kMaxDevices] = {nullptr};
std::mutex g_err_mu;

int* device_error_ptr() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_err_mu);
    if (!g_err_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_error) != cudaSuccess) return nullptr;
        g_err_ptr[dev] = static_cast<int*>(p);
    }
    return g_err_ptr[dev];
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int stride_of(int32_t storage) {
    return storage == FIF_STORAGE_F32 ? 216 : storage == FIF_STORAGE_BF16 ? 224 : storage == FIF_STORAGE_TRACE ? 12 : 0;
}
size_t elem_of(int32_t storage) { return storage == FIF_STORAGE_BF16 ? 2 : 4; }

int check_grid(const fif_grid* g) {
    if (!g) return FIF_EINVAL;
    if (g->nx < 2 || g->ny < 2 || g->nz < 2) return FIF_EINVAL;
    if (!(g->res > 0.f) || !std::isfinite(g->res)) return FIF_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(g->origin[a])) return FIF_EINVAL;
    return FIF_OK;
}

int check_params(const fif_params* p) {
    if (!p) return FIF_EINVAL;
    if (!(p->half_fov > 0.0 && p->half_fov < M_PI)) return FIF_EINVAL;
    if (!std::isfinite(p->v_alpha)) return FIF_EINVAL;
    if (!(p->r_min >= 0.0) || !(p->r_max > p->r_min) || !std::isfinite(p->r_max)) return FIF_EINVAL;
    if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return FIF_EINVAL;
    if (p->bin_size < 0.f || !std::isfinite(p->bin_size)) return FIF_EINVAL;
    return FIF_OK;
}

int check_gp(const fif_gp* gp) {
    if (gp->n_samples < 1 || gp->n_samples > FIF_GP_MAX_SAMPLES || !gp->d_aux) return FIF_EINVAL;
    if (!(gp->length_scale > 0.0) || !std::isfinite(gp->length_scale)) return FIF_EINVAL;
    if (!(gp->k_s > 0.0) || !std::isfinite(gp->k_s)) return FIF_EINVAL;
    if (reinterpret_cast<uintptr_t>(gp->d_aux) & 255u) return FIF_EALIGN;
    return FIF_OK;
}

// storage bytes a field of this kind needs
size_t field_need(const fif_field* f) {
    return f->storage == FIF_STORAGE_GP ? fif_gp_field_bytes(&f->grid, f->gp.n_samples)
                                        : fif_field_bytes(&f->grid, f->storage);
}

int check_field(const fif_field* f) {
    if (!f) return FIF_EINVAL;
    int rc = check_grid(&f->grid);
    if (rc) return rc;
    if ((rc = check_params(&f->params))) return rc;
    if (f->storage == FIF_STORAGE_GP) {
        if ((rc = check_gp(&f->gp))) return rc;
        if (f->stride != fif_gp_stride(f->gp.n_samples)) return FIF_EINVAL;
    } else if (stride_of(f->storage) == 0 || f->stride != stride_of(f->storage)) {
        return FIF_EINVAL;
    }
    if (!f->coeffs) return FIF_EINVAL;
    if (!aligned16(f->coeffs)) return FIF_EALIGN;
    if (f->bytes < field_need(f)) return FIF_ESIZE;
    return FIF_OK;
}

// (k0, k1, k2) from v(0) = 1, v(pi) = 0, v(alpha) = v_alpha (Eq. quadratic_conditions):
// the first two give k1 = 1/2 and k0 + k2 = 1/2; the third then fixes k2.
void quad_coeffs(double alpha, double va, double k[3]) {
    const double c = std::cos(alpha);
    const double k2 = (va - 0.5 - 0.5 * c) / (c * c - 1.0);
    k[0] = 0.5 - k2;
    k[1] = 0.5;
    k[2] = k2;
}

fif::QueryArgs query_args(const fif_field* f, const float* poses, int64_t m, int32_t flags) {
    fif::QueryArgs a{};
    a.coeffs = f->coeffs;
    a.storage = f->storage;
    a.stride = f->stride;
    a.ox = f->grid.origin[0]; a.oy = f->grid.origin[1]; a.oz = f->grid.origin[2];
    a.res = f->grid.res;
    a.nx = f->grid.nx; a.ny = f->grid.ny; a.nz = f->grid.nz;
    a.k0 = (float)f->k[0]; a.k1 = (float)f->k[1]; a.k2 = (float)f->k[2];
    a.poses = poses;
    a.m = m;
    a.flags = flags;
    a.err = device_error_ptr();
    a.wait_ns = g_wait_ns.load(std::memory_order_relaxed);
    return a;
}

uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct FileHeader {
    char magic[8];        // "FIFFIELD"
    int32_t version;
    int32_t storage;
    int32_t stride;
    int32_t pad;
    fif_grid grid;
    fif_params params;
    uint64_t payload_bytes;
    uint64_t checksum;
};

}  // namespace

extern "C" {

int32_t fif_version(void) { return kVersion; }

const char* fif_status_str(int32_t code) {
    switch (code) {
        case FIF_OK: return "ok";
        case FIF_EINVAL: return "invalid argument";
        case FIF_ESIZE: return "buffer too small";
        case FIF_EALIGN: return "device pointer not 16-byte aligned";
        case FIF_ECUDA: return "CUDA error";
        case FIF_ETIMEOUT: return "bounded device wait ran out";
        case FIF_EIO: return "file I/O error";
        case FIF_EFORMAT: return "file format mismatch";
        case FIF_ERANGE: return "size exceeds a fixed maximum";
        default: return "unknown status";
    }
}

size_t fif_field_bytes(const fif_grid* grid, int32_t storage) {
    if (check_grid(grid) || stride_of(storage) == 0) return 0;
    const size_t nodes = (size_t)grid->nx * grid->ny * grid->nz;
    return nodes * stride_of(storage) * elem_of(storage);
}

int32_t fif_field_init(fif_field* field, const fif_grid* grid, const fif_params* params, int32_t storage,
                       void* d_coeffs, size_t bytes) {
    if (!field) return FIF_EINVAL;
    int rc = check_grid(grid);
    if (rc) return rc;
    if ((rc = check_params(params))) return rc;
    if (stride_of(storage) == 0) return FIF_EINVAL;
    if (!d_coeffs) return FIF_EINVAL;
    if (!aligned16(d_coeffs)) return FIF_EALIGN;
    if (bytes < fif_field_bytes(grid, storage)) return FIF_ESIZE;
    std::memset(field, 0, sizeof(*field));
    field->grid = *grid;
    field->params = *params;
    field->storage = storage;
    field->stride = stride_of(storage);
    field->coeffs = d_coeffs;
    field->bytes = bytes;
    quad_coeffs(params->half_fov, params->v_alpha, field->k);
    return FIF_OK;
}

int32_t fif_field_init_gp(fif_field* field, const fif_grid* grid, const fif_params* params, const fif_gp* gp,
                          void* d_coeffs, size_t bytes) {
    if (!field || !gp) return FIF_EINVAL;
    int rc = check_grid(grid);
    if (rc) return rc;
    if ((rc = check_params(params))) return rc;
    if ((rc = check_gp(gp))) return rc;
    if (!d_coeffs) return FIF_EINVAL;
    if (!aligned16(d_coeffs)) return FIF_EALIGN;
    if (bytes < fif_gp_field_bytes(grid, gp->n_samples)) return FIF_ESIZE;
    std::memset(field, 0, sizeof(*field));
    field->grid = *grid;
    field->params = *params;
    field->storage = FIF_STORAGE_GP;
    field->stride = fif_gp_stride(gp->n_samples);
    field->coeffs = d_coeffs;
    field->bytes = bytes;
    field->gp = *gp;
    return FIF_OK;
}

size_t fif_build_workspace_bytes(const fif_field* field, int64_t n) {
    if (check_field(field) || n < 0) return 0;
    const fif::BinGrid bg = fif::make_bin_grid(field);
    return fif::build_layout(bg, n).total;
}

static int32_t build_impl(fif_field* field, const float* d_landmarks, int64_t n, void* d_ws, size_t ws_bytes,
                          int accumulate, int k_begin, int k_end, fif_stream_t stream);

int32_t fif_build(fif_field* field, const float* d_landmarks, int64_t n, void* d_ws, size_t ws_bytes,
                  fif_stream_t stream) {
    if (!field) return FIF_EINVAL;
    return build_impl(field, d_landmarks, n, d_ws, ws_bytes, 0, 0, field->grid.nz, stream);
}

int32_t fif_build_update(fif_field* field, const float* d_landmarks, int64_t n, int32_t sign, void* d_ws,
                         size_t ws_bytes, fif_stream_t stream) {
    if (sign != 1 && sign != -1) return FIF_EINVAL;
    if (!field) return FIF_EINVAL;
    return build_impl(field, d_landmarks, n, d_ws, ws_bytes, sign, 0, field->grid.nz, stream);
}

int32_t fif_build_slab(fif_field* field, int32_t k_begin, int32_t k_end, const float* d_landmarks, int64_t n,
                       void* d_ws, size_t ws_bytes, fif_stream_t stream) {
    if (!field) return FIF_EINVAL;
    if (k_begin < 0 || k_end <= k_begin || k_end > field->grid.nz) return FIF_EINVAL;
    return build_impl(field, d_landmarks, n, d_ws, ws_bytes, 0, k_begin, k_end, stream);
}

int32_t fif_slab_landmark_band(const fif_field* field, int32_t k_begin, int32_t k_end, float* z_lo, float* z_hi) {
    int rc = check_field(field);
    if (rc) return rc;
    if (!z_lo || !z_hi || k_begin < 0 || k_end <= k_begin || k_end > field->grid.nz) return FIF_EINVAL;
    // the node layers of the bricks that hold the slab's nodes (a warp's culling box may span layers
    // just outside the slab), widened by the build's cull radius (a landmark farther than that from
    // every node of a box never enters the sums), plus 1e-3 relative and 1 mm for the
    // single-precision rounding of positions and of the culling test
    const int bz = field->storage == FIF_STORAGE_GP ? fif::kGpBuildBrickZ : fif::kBuildBrickZ;
    const int kb0 = k_begin / bz * bz, kb1 = std::min((k_end + bz - 1) / bz * bz, (int)field->grid.nz);
    const double z0 = (double)field->grid.origin[2] + (double)field->grid.res * kb0;
    const double z1 = (double)field->grid.origin[2] + (double)field->grid.res * (kb1 - 1);
    const double r_cull = field->params.r_max + 0.01 + 1e-4 * field->params.r_max;
    const double m = r_cull * 1.001 + 1e-3 + 1e-6 * std::max(std::fabs(z0), std::fabs(z1));
    *z_lo = (float)(z0 - m);
    *z_hi = (float)(z1 + m);
    return FIF_OK;
}

static int32_t build_impl(fif_field* field, const float* d_landmarks, int64_t n, void* d_ws, size_t ws_bytes,
                          int accumulate, int k_begin, int k_end, fif_stream_t stream) {
    int rc = check_field(field);
    if (rc) return rc;
    if (n < 0 || (n > 0 && !d_landmarks) || !d_ws) return FIF_EINVAL;
    if (!aligned16(d_ws) || (n > 0 && (reinterpret_cast<uintptr_t>(d_landmarks) & 3u))) return FIF_EALIGN;
    const fif::BinGrid bg = fif::make_bin_grid(field);
    const fif::BuildLayout lay = fif::build_layout(bg, n);
    if (ws_bytes < lay.total) return FIF_ESIZE;
    fif::BuildArgs a{};
    a.landmarks = d_landmarks;
    a.n = n;
    a.ws = static_cast<unsigned char*>(d_ws);
    a.lay = lay;
    a.bg = bg;
    a.ox = field->grid.origin[0]; a.oy = field->grid.origin[1]; a.oz = field->grid.origin[2];
    a.res = field->grid.res;
    a.nx = field->grid.nx; a.ny = field->grid.ny; a.nz = field->grid.nz;
    a.rmin2 = (float)(field->params.r_min * field->params.r_min);
    a.rmax2 = (float)(field->params.r_max * field->params.r_max);
    a.rcull = (float)(field->params.r_max + 0.01 + 1e-4 * field->params.r_max);
    a.inv_sigma2 = (float)(1.0 / (field->params.sigma * field->params.sigma));
    a.storage = field->storage;
    a.stride = field->stride;
    a.out = field->coeffs;
    a.err = device_error_ptr();
    a.accumulate = accumulate;
    a.wait_ns = g_wait_ns.load(std::memory_order_relaxed);
    a.k_begin = k_begin;
    a.k_end = k_end;
    if (field->storage == FIF_STORAGE_GP) {
        const fif_gp& gp = field->gp;
        const fif::GpAuxLayout L = fif::gp_aux_layout(gp.n_samples, fif_gp_row_stride(gp.n_samples));
        a.gp_axes = reinterpret_cast<const float4*>(static_cast<const unsigned char*>(gp.d_aux) + L.axes_f);
        a.gp_ns = gp.n_samples;
        a.gp_rs = fif_gp_row_stride(gp.n_samples);
        const double log2e = 1.4426950408889634;
        a.gp_scale = (float)(gp.k_s * log2e);
        a.gp_shift = (float)(gp.k_s * log2e * std::cos(field->params.half_fov));
    }
    return fif::launch_build(a, stream);
}

int32_t fif_query(const fif_field* field, const float* d_poses, int64_t m, int32_t flags, float* d_fim,
                  double* d_metrics, int8_t* d_sign, int32_t* d_status, fif_stream_t stream) {
    int rc = check_field(field);
    if (rc) return rc;
    if (m < 0 || (m > 0 && !d_poses)) return FIF_EINVAL;
    if (flags & ~(FIF_Q_NEAREST | FIF_Q_WORLD | FIF_Q_METRICS | FIF_Q_GP_COMPENSATED)) return FIF_EINVAL;
    if ((flags & FIF_Q_GP_COMPENSATED) && field->storage != FIF_STORAGE_GP) return FIF_EINVAL;
    if (m == 0) return FIF_OK;   // nothing to write (empty buffers may be NULL)
    if ((flags & FIF_Q_METRICS) && !d_metrics && !d_sign && !d_status) return FIF_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_poses) & 3u) return FIF_EALIGN;
    fif::QueryArgs a = query_args(field, d_poses, m, flags);
    a.fim = d_fim;
    a.metrics = d_metrics;
    a.sign = d_sign;
    a.status = d_status;
    if (field->storage == FIF_STORAGE_TRACE) {
        // the trace factor answers only the world-frame trace (Eq. general_trace_query)
        if ((flags & FIF_Q_METRICS) != FIF_Q_TRACE || !(flags & FIF_Q_WORLD) || d_fim || d_sign) return FIF_EINVAL;
        return fif::launch_trace_query(a, stream);
    }
    if (field->storage == FIF_STORAGE_GP) {
        const fif_gp& gp = field->gp;
        a.gp_ns = gp.n_samples;
        a.gp_rs = fif_gp_row_stride(gp.n_samples);
        const fif::GpAuxLayout L = fif::gp_aux_layout(a.gp_ns, a.gp_rs);
        const unsigned char* aux = static_cast<const unsigned char*>(gp.d_aux);
        a.gp_axes = reinterpret_cast<const float4*>(aux + L.axes_df);
        a.gp_wt = reinterpret_cast<const float2*>(aux + L.wt);
        a.gp_consts = reinterpret_cast<const float4*>(aux + L.consts);
        return fif::launch_gp_query(a, stream);
    }
    return fif::launch_query(a, stream);
}

namespace {

// staging of one buffer of fif_query_host: poses, fim, metrics, sign, status (256-B aligned)
struct HostStaging {
    size_t poses, fim, metrics, sign, status, total;
};

HostStaging host_staging(int64_t chunk) {
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    HostStaging L;
    size_t off = 0;
    const size_t c = (size_t)chunk;
    L.poses = off;   off += up(c * 7 * sizeof(float));
    L.fim = off;     off += up(c * 21 * sizeof(float));
    L.metrics = off; off += up(c * 3 * sizeof(double));
    L.sign = off;    off += up(c);
    L.status = off;  off += up(c * sizeof(int32_t));
    L.total = off;
    return L;
}

}  // namespace

size_t fif_query_host_staging_bytes(int64_t chunk) {
    if (chunk <= 0) return 0;
    return 2 * host_staging(chunk).total;
}

int32_t fif_query_host(const fif_field* field, const float* h_poses, int64_t m, int32_t flags, float* h_fim,
                       double* h_metrics, int8_t* h_sign, int32_t* h_status, int64_t chunk, void* d_staging,
                       size_t staging_bytes, fif_stream_t stream, fif_stream_t copy_stream) {
    int rc = check_field(field);
    if (rc) return rc;
    if (m < 0 || (m > 0 && !h_poses)) return FIF_EINVAL;
    if (m == 0) return FIF_OK;
    if (chunk <= 0 || !d_staging || stream == copy_stream) return FIF_EINVAL;
    if (staging_bytes < fif_query_host_staging_bytes(chunk)) return FIF_ESIZE;
    if (reinterpret_cast<uintptr_t>(d_staging) & 15u) return FIF_EALIGN;
    // page-locked host buffers that the device can address (cudaHostAlloc memory, mapped on any
    // system with unified addressing): the query reads the poses from and writes the outputs to
    // them in place over the host link, with no staging copies and no HBM traffic for the I/O
    {
        auto mapped = [](const void* p, void** dp) -> bool {
            *dp = nullptr;
            if (!p) return true;
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
            *dp = at.devicePointer;
            return true;
        };
        void *dp, *df, *dm, *ds, *dt;
        if (mapped(h_poses, &dp) && mapped(h_fim, &df) && mapped(h_metrics, &dm) && mapped(h_sign, &ds) &&
            mapped(h_status, &dt))
            return fif_query(field, static_cast<const float*>(dp), m, flags, static_cast<float*>(df),
                             static_cast<double*>(dm), static_cast<int8_t*>(ds), static_cast<int32_t*>(dt), stream);
    }
    const HostStaging L = host_staging(chunk);
    unsigned char* base[2] = {static_cast<unsigned char*>(d_staging),
                              static_cast<unsigned char*>(d_staging) + L.total};
    cudaStream_t sq = reinterpret_cast<cudaStream_t>(stream), sc = reinterpret_cast<cudaStream_t>(copy_stream);
    cudaEvent_t h2d[2] = {nullptr, nullptr}, qd[2] = {nullptr, nullptr}, done = nullptr, start = nullptr;
    bool ok = cudaEventCreateWithFlags(&start, cudaEventDisableTiming) == cudaSuccess;
    // the copies start after the work already queued on `stream`
    ok = ok && cudaEventRecord(start, sq) == cudaSuccess && cudaStreamWaitEvent(sc, start, 0) == cudaSuccess;
    for (int b = 0; b < 2; ++b) {
        ok = ok && cudaEventCreateWithFlags(&h2d[b], cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&qd[b], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess;
    // pieces of the batch: a quarter chunk first and last (less copy time before the first query
    // and after the last one), full chunks between; every piece fits a staging buffer
    std::vector<int64_t> piece{0};
    if (m > chunk) {
        const int64_t q = std::max<int64_t>(1, chunk / 4);
        int64_t pos = q;
        piece.push_back(pos);
        while (m - pos > chunk + q) {
            pos += chunk;
            piece.push_back(pos);
        }
        if (m - pos > q) piece.push_back(m - q);
    }
    piece.push_back(m);
    const int64_t nch = (int64_t)piece.size() - 1;
    auto count = [&](int64_t c) { return piece[c + 1] - piece[c]; };
    auto upload = [&](int64_t c) {
        const int b = (int)(c & 1);
        ok = ok && cudaMemcpyAsync(base[b] + L.poses, h_poses + piece[c] * 7, (size_t)count(c) * 7 * sizeof(float),
                                   cudaMemcpyHostToDevice, sc) == cudaSuccess;
        ok = ok && cudaEventRecord(h2d[b], sc) == cudaSuccess;
    };
    // copy stream: H2D(0), H2D(1), D2H(0), H2D(2), D2H(1), ...; a buffer's poses are overwritten
    // only after the query that read them (D2H of that chunk waited for it and precedes in order),
    // and its outputs only after their D2H (the next query of the buffer waits for its H2D)
    if (ok) upload(0);
    for (int64_t c = 0; c < nch && ok; ++c) {
        const int b = (int)(c & 1);
        const int64_t n = count(c), p0 = piece[c];
        unsigned char* B = base[b];
        ok = cudaStreamWaitEvent(sq, h2d[b], 0) == cudaSuccess;
        if (!ok) break;
        rc = fif_query(field, reinterpret_cast<const float*>(B + L.poses), n, flags,
                       h_fim ? reinterpret_cast<float*>(B + L.fim) : nullptr,
                       h_metrics ? reinterpret_cast<double*>(B + L.metrics) : nullptr,
                       h_sign ? reinterpret_cast<int8_t*>(B + L.sign) : nullptr,
                       h_status ? reinterpret_cast<int32_t*>(B + L.status) : nullptr, stream);
        if (rc != FIF_OK) break;
        ok = cudaEventRecord(qd[b], sq) == cudaSuccess;
        if (ok && c + 1 < nch) upload(c + 1);
        ok = ok && cudaStreamWaitEvent(sc, qd[b], 0) == cudaSuccess;
        auto down = [&](void* dst, size_t off, size_t bytes) {
            if (dst) ok = ok && cudaMemcpyAsync(dst, B + off, bytes, cudaMemcpyDeviceToHost, sc) == cudaSuccess;
        };
        down(h_fim ? h_fim + p0 * 21 : nullptr, L.fim, (size_t)n * 21 * sizeof(float));
        down(h_metrics ? h_metrics + p0 * 3 : nullptr, L.metrics, (size_t)n * 3 * sizeof(double));
        down(h_sign ? h_sign + p0 : nullptr, L.sign, (size_t)n);
        down(h_status ? h_status + p0 : nullptr, L.status, (size_t)n * sizeof(int32_t));
    }
    // the query stream completes after the last copy, also on an error after work was queued
    if (done && cudaEventRecord(done, sc) == cudaSuccess) cudaStreamWaitEvent(sq, done, 0);
    for (int b = 0; b < 2; ++b) {
        if (h2d[b]) cudaEventDestroy(h2d[b]);
        if (qd[b]) cudaEventDestroy(qd[b]);
    }
    if (done) cudaEventDestroy(done);
    if (start) cudaEventDestroy(start);
    if (rc != FIF_OK) return rc;
    return ok ? FIF_OK : FIF_ECUDA;
}

int32_t fif_query_backward(const fif_field* field, const float* d_poses, int64_t m, int32_t flags,
                           const float* d_fim, const double* d_grad_metrics, float* d_grad_pose,
                           fif_stream_t stream) {
    int rc = check_field(field);
    if (rc) return rc;
    if (m < 0 || (m > 0 && (!d_poses || !d_fim || !d_grad_metrics || !d_grad_pose))) return FIF_EINVAL;
    if (flags & ~(FIF_Q_WORLD | FIF_Q_METRICS)) return FIF_EINVAL;  // trilinear only
    if (field->storage != FIF_STORAGE_F32) return FIF_EINVAL;  // the adjoint reads float32 coefficients
    if (m == 0) return FIF_OK;
    fif::QueryArgs q = query_args(field, d_poses, m, flags);
    fif::AdjointArgs a{};
    a.coeffs = q.coeffs; a.storage = q.storage; a.stride = q.stride;
    a.ox = q.ox; a.oy = q.oy; a.oz = q.oz; a.res = q.res;
    a.nx = q.nx; a.ny = q.ny; a.nz = q.nz;
    a.k0 = q.k0; a.k1 = q.k1; a.k2 = q.k2;
    a.poses = d_poses;
    a.m = m;
    a.flags = flags;
    a.fim = d_fim;
    a.gm = d_grad_metrics;
    a.grad = d_grad_pose;
    a.err = q.err;
    return fif::launch_adjoint(a, stream);
}

int32_t fif_pointcloud_fim(const float* d_landmarks, int64_t n, const fif_params* params, const fif_pinhole* cam,
                           const float* d_poses, int64_t m, int32_t flags, float* d_fim, double* d_metrics,
                           int8_t* d_sign, int32_t* d_status, fif_stream_t stream) {
    int rc = check_params(params);
    if (rc) return rc;
    if (!cam || cam->width <= 0 || cam->height <= 0) return FIF_EINVAL;
    if (n < 0 || m < 0 || (n > 0 && !d_landmarks) || (m > 0 && !d_poses)) return FIF_EINVAL;
    if (flags & ~(FIF_Q_WORLD | FIF_Q_METRICS)) return FIF_EINVAL;
    if (m == 0) return FIF_OK;
    fif::PointCloudArgs a{};
    a.landmarks = d_landmarks;
    a.n = n;
    a.rmin2 = (float)(params->r_min * params->r_min);
    a.rmax2 = (float)(params->r_max * params->r_max);
    a.inv_sigma2 = (float)(1.0 / (params->sigma * params->sigma));
    a.fx = cam->fx; a.fy = cam->fy; a.cx = cam->cx; a.cy = cam->cy;
    a.W = (float)cam->width; a.H = (float)cam->height;
    a.poses = d_poses;
    a.m = m;
    a.flags = flags;
    a.fim = d_fim;
    a.metrics = d_metrics;
    a.sign = d_sign;
    a.status = d_status;
    return fif::launch_pointcloud(a, stream);
}

int32_t fif_info_threshold(const fif_params* params, int32_t model, const fif_gp* gp, const float* d_sets,
                           int64_t n_sets, int32_t m, int32_t exclude_degenerate, double* d_metrics, int8_t* d_sign,
                           double* d_threshold, fif_stream_t stream) {
    int rc = check_params(params);
    if (rc) return rc;
    if (model < FIF_MODEL_POINTCLOUD || model > FIF_MODEL_GP || m < 1 || n_sets < 0) return FIF_EINVAL;
    if (n_sets > 0 && (!d_sets || !d_metrics)) return FIF_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_sets) & 3u) return FIF_EALIGN;
    fif::InfoArgs a{};
    a.sets = d_sets;
    a.n = n_sets;
    a.m = m;
    a.model = model;
    a.inv_sigma2 = (float)(1.0 / (params->sigma * params->sigma));
    double k[3];
    quad_coeffs(params->half_fov, params->v_alpha, k);
    a.k0 = (float)k[0]; a.k1 = (float)k[1]; a.k2 = (float)k[2];
    if (model == FIF_MODEL_GP) {
        if (!gp || !(gp->k_s > 0.0) || !std::isfinite(gp->k_s)) return FIF_EINVAL;
        const double e3[3] = {0.0, 0.0, 1.0};
        double w[FIF_GP_MAX_SAMPLES];
        if ((rc = fif::gp_kriging_weights(gp, e3, w))) return rc;
        a.gp_ns = gp->n_samples;
        a.gp_ks = (float)gp->k_s;
        a.gp_cos_alpha = (float)std::cos(params->half_fov);
        for (int s = 0; s < gp->n_samples; ++s) {
            const double* z = gp->axes[s];
            const double nz = std::sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
            a.gp_a[s] = (float)w[s];
            for (int c = 0; c < 3; ++c) a.gp_axes[s][c] = (float)(z[c] / nz);
        }
    }
    a.metrics = d_metrics;
    a.sign = d_sign;
    return fif::launch_info_threshold(a, exclude_degenerate != 0, d_threshold, stream);
}

int32_t fif_info_cost(const double* d_values, int64_t m, int64_t stride, double eps, double k_q, double* d_cost,
                      double* d_dcost, fif_stream_t stream) {
    if (m < 0 || stride < 1 || (m > 0 && !d_values)) return FIF_EINVAL;
    if (!(eps > 0.0) || !std::isfinite(eps) || !(k_q > 0.0) || !std::isfinite(k_q)) return FIF_EINVAL;
    return fif::launch_info_cost(d_values, m, stride, eps, k_q, d_cost, d_dcost, stream);
}

int32_t fif_field_save(const fif_field* field, const char* path, void* host_staging, fif_stream_t stream) {
    int rc = check_field(field);
    if (rc) return rc;
    if (field->storage == FIF_STORAGE_GP) return FIF_EINVAL;   // the file format has no GP model
    if (!path) return FIF_EINVAL;
    const size_t bytes = fif_field_bytes(&field->grid, field->storage);
    unsigned char* buf = static_cast<unsigned char*>(host_staging);
    unsigned char* own = nullptr;
    if (!buf) {
        own = static_cast<unsigned char*>(std::malloc(bytes));
        if (!own) return FIF_ESIZE;
        buf = own;
    }
    int result = FIF_OK;
    if (cudaMemcpyAsync(buf, field->coeffs, bytes, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        result = FIF_ECUDA;
    } else {
        FileHeader h{};
        std::memcpy(h.magic, "FIFFIELD", 8);
        h.version = kVersion;
        h.storage = field->storage;
        h.stride = field->stride;
        h.grid = field->grid;
        h.params = field->params;
        h.payload_bytes = bytes;
        h.checksum = fnv1a(buf, bytes);
        FILE* fp = std::fopen(path, "wb");
        if (!fp) {
            result = FIF_EIO;
        } else {
            if (std::fwrite(&h, sizeof(h), 1, fp) != 1 || std::fwrite(buf, 1, bytes, fp) != bytes) result = FIF_EIO;
            if (std::fclose(fp) != 0) result = FIF_EIO;
        }
    }
    std::free(own);
    return result;
}

int32_t fif_field_load(fif_field* field, const char* path, void* d_coeffs, size_t bytes, void* host_staging,
                       fif_stream_t stream) {
    if (!field || !path || !d_coeffs) return FIF_EINVAL;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return FIF_EIO;
    FileHeader h{};
    if (std::fread(&h, sizeof(h), 1, fp) != 1) { std::fclose(fp); return FIF_EFORMAT; }
    if (std::memcmp(h.magic, "FIFFIELD", 8) != 0 || h.version != kVersion || stride_of(h.storage) == 0 ||
        h.stride != stride_of(h.storage) || check_grid(&h.grid) || check_params(&h.params) ||
        h.payload_bytes != fif_field_bytes(&h.grid, h.storage)) {
        std::fclose(fp);
        return FIF_EFORMAT;
    }
    if (bytes < h.payload_bytes) { std::fclose(fp); return FIF_ESIZE; }
    unsigned char* buf = static_cast<unsigned char*>(host_staging);
    unsigned char* own = nullptr;
    if (!buf) {
        own = static_cast<unsigned char*>(std::malloc(h.payload_bytes));
        if (!own) { std::fclose(fp); return FIF_ESIZE; }
        buf = own;
    }
    int result = FIF_OK;
    if (std::fread(buf, 1, h.payload_bytes, fp) != h.payload_bytes) result = FIF_EFORMAT;
    std::fclose(fp);
    if (result == FIF_OK && fnv1a(buf, h.payload_bytes) != h.checksum) result = FIF_EFORMAT;
    if (result == FIF_OK) {
        result = fif_field_init(field, &h.grid, &h.params, h.storage, d_coeffs, bytes);
        if (result == FIF_OK &&
            (cudaMemcpyAsync(d_coeffs, buf, h.payload_bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
             cudaStreamSynchronize(stream) != cudaSuccess))
            result = FIF_ECUDA;
    }
    std::free(own);
    return result;
}

int32_t fif_set_wait_limit(uint64_t limit_ns) {
    g_wait_ns.store(limit_ns == 0 ? kDefaultWaitNs : limit_ns, std::memory_order_relaxed);
    return FIF_OK;
}

int32_t fif_device_error(int32_t* out_code, int32_t reset, fif_stream_t stream) {
    if (!out_code) return FIF_EINVAL;
    int* p = device_error_ptr();
    if (!p) return FIF_ECUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FIF_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FIF_ECUDA;
    if (reset) {
        const int z = 0;
        if (cudaMemcpy(p, &z, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return FIF_ECUDA;
    }
    *out_code = v;
    return FIF_OK;
}

}  // extern "C"
