// gp_model.cu -- host side of the GP visibility model (Sec. V-B-2): record layout, the
// inverse kernel matrix W = (K^s + s_n^2 I)^-1, the maximum-marginal-likelihood length
// scale, and the device copy of the model.  Double precision, Cholesky factorisations.
#include <cmath>
#include <cstring>
#include <vector>

#include "fif_internal.h"

namespace {

bool valid_count(int32_t ns) { return ns >= 1 && ns <= FIF_GP_MAX_SAMPLES; }

// K[g][h] = exp(-|z_g - z_h|^2 / (2 l^2)) + noise * delta_gh
void kernel_matrix(const double (*axes)[3], int ns, double l, double noise, std::vector<double>& K) {
    K.assign((size_t)ns * ns, 0.0);
    const double s = 1.0 / (2.0 * l * l);
    for (int g = 0; g < ns; ++g)
        for (int h = 0; h < ns; ++h) {
            const double d0 = axes[g][0] - axes[h][0], d1 = axes[g][1] - axes[h][1], d2 = axes[g][2] - axes[h][2];
            K[(size_t)g * ns + h] = std::exp(-(d0 * d0 + d1 * d1 + d2 * d2) * s) + (g == h ? noise : 0.0);
        }
}

// in-place lower Cholesky factor of the symmetric positive definite A (row-major); false if a
// pivot is not positive
bool cholesky(std::vector<double>& A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = s / ljj;
        }
        for (int k = j + 1; k < n; ++k) A[(size_t)j * n + k] = 0.0;
    }
    return true;
}

// solve L x = b in place (L lower triangular)
void forward_solve(const std::vector<double>& Lf, int n, double* b) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= Lf[(size_t)i * n + k] * b[k];
        b[i] = s / Lf[(size_t)i * n + i];
    }
}

// W = (L L^T)^-1 = L^-T L^-1
void inverse_from_cholesky(const std::vector<double>& Lf, int n, std::vector<double>& W) {
    std::vector<double> Li((size_t)n * n, 0.0);   // L^-1, lower triangular, column by column
    std::vector<double> e(n);
    for (int c = 0; c < n; ++c) {
        std::fill(e.begin(), e.end(), 0.0);
        e[c] = 1.0;
        forward_solve(Lf, n, e.data());
        for (int r = 0; r < n; ++r) Li[(size_t)r * n + c] = e[r];
    }
    W.assign((size_t)n * n, 0.0);
    for (int g = 0; g < n; ++g)
        for (int h = g; h < n; ++h) {
            double s = 0.0;
            for (int k = std::max(g, h); k < n; ++k) s += Li[(size_t)k * n + g] * Li[(size_t)k * n + h];
            W[(size_t)g * n + h] = s;
            W[(size_t)h * n + g] = s;
        }
}

bool normalised_axes(const fif_gp* gp, double (*out)[3]) {
    for (int g = 0; g < gp->n_samples; ++g) {
        const double* a = gp->axes[g];
        const double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        if (!(n > 0.0) || !std::isfinite(n)) return false;
        for (int c = 0; c < 3; ++c) out[g][c] = a[c] / n;
    }
    return true;
}

// sum_m -1/2 y_m^T K^-1 y_m - M/2 log|K| (the constant -M N/2 log 2 pi omitted), or -inf when
// K is not positive definite
double log_marginal(const double (*axes)[3], int ns, double l, double noise, const std::vector<double>& Y, int M) {
    std::vector<double> K;
    kernel_matrix(axes, ns, l, noise, K);
    if (!cholesky(K, ns)) return -INFINITY;
    double logdet = 0.0;
    for (int i = 0; i < ns; ++i) logdet += 2.0 * std::log(K[(size_t)i * ns + i]);
    std::vector<double> y(ns);
    double quad = 0.0;
    for (int m = 0; m < M; ++m) {
        std::memcpy(y.data(), &Y[(size_t)m * ns], sizeof(double) * ns);
        forward_solve(K, ns, y.data());
        for (int i = 0; i < ns; ++i) quad += y[i] * y[i];
    }
    return -0.5 * quad - 0.5 * M * logdet;
}

}  // namespace

namespace fif {

int gp_kriging_weights(const fif_gp* gp, const double z[3], double* a) {
    if (!gp || !valid_count(gp->n_samples)) return FIF_EINVAL;
    if (!(gp->length_scale > 0.0) || !std::isfinite(gp->length_scale)) return FIF_EINVAL;
    if (!(gp->noise_var >= 0.0) || !std::isfinite(gp->noise_var)) return FIF_EINVAL;
    const int ns = gp->n_samples;
    double axes[FIF_GP_MAX_SAMPLES][3];
    if (!normalised_axes(gp, axes)) return FIF_EINVAL;
    std::vector<double> K;
    kernel_matrix(axes, ns, gp->length_scale, gp->noise_var, K);
    if (!cholesky(K, ns)) return FIF_EINVAL;
    // a = (L L^T)^-1 k_z: forward then backward substitution
    std::vector<double> y(ns);
    const double s = 1.0 / (2.0 * gp->length_scale * gp->length_scale);
    for (int g = 0; g < ns; ++g) {
        const double d0 = z[0] - axes[g][0], d1 = z[1] - axes[g][1], d2 = z[2] - axes[g][2];
        y[g] = std::exp(-(d0 * d0 + d1 * d1 + d2 * d2) * s);
    }
    forward_solve(K, ns, y.data());
    for (int i = ns - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < ns; ++k) v -= K[(size_t)k * ns + i] * a[k];
        a[i] = v / K[(size_t)i * ns + i];
    }
    return FIF_OK;
}

}  // namespace fif

extern "C" {

int32_t fif_gp_row_stride(int32_t ns) {
    if (!valid_count(ns)) return 0;
    int32_t rs = ns;
    while (rs % 4 != 2) ++rs;
    return rs;
}

int32_t fif_gp_stride(int32_t ns) {
    const int32_t rs = fif_gp_row_stride(ns);
    return rs ? (21 * rs + 3) / 4 * 4 : 0;
}

size_t fif_gp_aux_bytes(int32_t ns) {
    if (!valid_count(ns)) return 0;
    return fif::gp_aux_layout(ns, fif_gp_row_stride(ns)).total;
}

size_t fif_gp_field_bytes(const fif_grid* grid, int32_t ns) {
    if (!grid || grid->nx < 2 || grid->ny < 2 || grid->nz < 2 || !valid_count(ns)) return 0;
    return (size_t)grid->nx * grid->ny * grid->nz * (size_t)fif_gp_stride(ns) * 4;
}

int32_t fif_gp_upload(fif_gp* gp, void* d_aux, size_t bytes, fif_stream_t stream) {
    if (!gp || !d_aux || !valid_count(gp->n_samples)) return FIF_EINVAL;
    if (!(gp->length_scale > 0.0) || !std::isfinite(gp->length_scale)) return FIF_EINVAL;
    if (!(gp->noise_var >= 0.0) || !std::isfinite(gp->noise_var)) return FIF_EINVAL;
    if (!(gp->k_s > 0.0) || !std::isfinite(gp->k_s)) return FIF_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_aux) & 255u) return FIF_EALIGN;
    const int ns = gp->n_samples, rs = fif_gp_row_stride(ns);
    const fif::GpAuxLayout L = fif::gp_aux_layout(ns, rs);
    if (bytes < L.total) return FIF_ESIZE;
    double axes[FIF_GP_MAX_SAMPLES][3];
    if (!normalised_axes(gp, axes)) return FIF_EINVAL;
    std::vector<double> K, W;
    kernel_matrix(axes, ns, gp->length_scale, gp->noise_var, K);
    if (!cholesky(K, ns)) return FIF_EINVAL;
    inverse_from_cholesky(K, ns, W);
    std::vector<unsigned char> img(L.total, 0);
    float* af = reinterpret_cast<float*>(img.data() + L.axes_f);
    float* adf = reinterpret_cast<float*>(img.data() + L.axes_df);
    float* wt = reinterpret_cast<float*>(img.data() + L.wt);
    float* cst = reinterpret_cast<float*>(img.data() + L.consts);
    for (int g = 0; g < ns; ++g) {
        for (int c = 0; c < 3; ++c) {
            const float hi = (float)axes[g][c];
            af[4 * g + c] = hi;
            adf[4 * g + c] = hi;
            adf[4 * (ns + g) + c] = (float)(axes[g][c] - (double)hi);
        }
    }
    // constants of the double-float exponential (Tang's table-driven method): ln2/32 split as
    // C1 + C2 + C3 with C1 carrying 12 significant bits (so N * C1 is exact for |N| < 2^12),
    // 32/ln2 to pick N, 1/l^2 as a (high, low) pair, and the table 2^(j/32) as (high, low) pairs
    {
        const double ln2_32 = std::log(2.0) / 32.0;
        const double c1 = std::ldexp(std::nearbyint(std::ldexp(ln2_32, 17)), -17);
        const double rest = ln2_32 - c1;
        const float C1 = (float)c1, C2 = (float)rest, C3 = (float)(rest - (double)C2);
        const double inv_l2 = 1.0 / (gp->length_scale * gp->length_scale);
        const float cH = (float)inv_l2, cL = (float)(inv_l2 - (double)cH);
        const float v[8] = {C1, C2, C3, (float)(32.0 / std::log(2.0)), cH, cL, 0.f, 0.f};
        std::memcpy(cst, v, sizeof(v));
        for (int j = 0; j < 32; ++j) {
            const double t = std::exp2(j / 32.0);
            const float th = (float)t;
            cst[8 + 2 * j] = th;
            cst[8 + 2 * j + 1] = (float)(t - (double)th);
        }
    }
    for (int h = 0; h < ns; ++h)
        for (int g = 0; g < ns; ++g) {
            const double w = W[(size_t)g * ns + h];
            const float hi = (float)w;
            wt[2 * ((size_t)h * rs + g)] = hi;
            wt[2 * ((size_t)h * rs + g) + 1] = (float)(w - (double)hi);
        }
    for (int g = 0; g < ns; ++g)
        for (int c = 0; c < 3; ++c) gp->axes[g][c] = axes[g][c];
    if (cudaMemcpyAsync(d_aux, img.data(), L.total, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return FIF_ECUDA;
    gp->d_aux = d_aux;
    return FIF_OK;
}

int32_t fif_gp_fit_length_scale(const fif_gp* gp, double half_fov, const double* bearings, int32_t m, double l_lo,
                                double l_hi, double* l_out) {
    if (!gp || !bearings || !l_out || m < 1 || !valid_count(gp->n_samples)) return FIF_EINVAL;
    if (!(l_lo > 0.0) || !(l_hi > l_lo) || !std::isfinite(l_hi)) return FIF_EINVAL;
    if (!(half_fov > 0.0 && half_fov < M_PI) || !(gp->k_s > 0.0) || !(gp->noise_var >= 0.0)) return FIF_EINVAL;
    const int ns = gp->n_samples;
    double axes[FIF_GP_MAX_SAMPLES][3];
    if (!normalised_axes(gp, axes)) return FIF_EINVAL;
    // training vectors: the sigmoid visibility (Eq. sigmoid_vis_func) at every sample axis
    std::vector<double> Y((size_t)m * ns);
    const double ca = std::cos(half_fov);
    for (int i = 0; i < m; ++i) {
        const double* p = bearings + 3 * i;
        const double n = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        if (!(n > 0.0) || !std::isfinite(n)) return FIF_EINVAL;
        for (int g = 0; g < ns; ++g) {
            const double c = (axes[g][0] * p[0] + axes[g][1] * p[1] + axes[g][2] * p[2]) / n;
            Y[(size_t)i * ns + g] = 1.0 / (1.0 + std::exp(-gp->k_s * (c - ca)));
        }
    }
    auto f = [&](double l) { return log_marginal(axes, ns, l, gp->noise_var, Y, m); };
    constexpr int kScan = 97;
    const double a0 = std::log(l_lo), a1 = std::log(l_hi);
    int best = -1;
    double fb = -INFINITY;
    std::vector<double> ls(kScan);
    for (int i = 0; i < kScan; ++i) {
        ls[i] = std::exp(a0 + (a1 - a0) * i / (kScan - 1));
        const double v = f(ls[i]);
        if (v > fb) { fb = v; best = i; }
    }
    if (best < 0) return FIF_EINVAL;
    // golden-section search for the maximum on the bracket around the best scan point
    double lo = ls[std::max(0, best - 1)], hi = ls[std::min(kScan - 1, best + 1)];
    const double r = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = hi - r * (hi - lo), x2 = lo + r * (hi - lo);
    double f1 = f(x1), f2 = f(x2);
    while (hi - lo > 1e-7 * hi) {
        if (f1 < f2) {
            lo = x1; x1 = x2; f1 = f2;
            x2 = lo + r * (hi - lo); f2 = f(x2);
        } else {
            hi = x2; x2 = x1; f2 = f1;
            x1 = hi - r * (hi - lo); f1 = f(x1);
        }
    }
    const double lm = 0.5 * (lo + hi);
    *l_out = (f(lm) >= fb) ? lm : ls[best];
    return FIF_OK;
}

}  // extern "C"
