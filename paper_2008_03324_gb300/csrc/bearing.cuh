// bearing.cuh -- the information of a set of bearings from its moment sums (used by the GP
// build and the information-threshold kernels).
#pragma once

#include "fif_common.cuh"

namespace fif {

// Entry e (upper triangle, row-major) of a weighted sum of single-bearing informations
// sum_i v_i [[P_i/n_i^2, -[u_i]x/n_i], [[u_i]x/n_i, P_i]] (P = I - u u^T; Eq. global_fim_eq with
// the rotation taken about the observer), from its 15 moments: m[0..5] = sum v (xx yy zz xy xz
// yz), m[6..11] the same over n^2, m[12..14] = sum v (x y z) / n.  |u| = 1 makes the diagonal
// of P the sum of the other two squares.
__host__ __device__ inline float bearing_entry(int e, const float* m) {
    const int r = sym_row(e), c = sym_col(e);
    auto diag = [&](int base, int a) {
        return a == 0 ? m[base + 1] + m[base + 2] : a == 1 ? m[base + 0] + m[base + 2] : m[base + 0] + m[base + 1];
    };
    if (r < 3 && c < 3) return r == c ? diag(6, r) : -m[6 + 2 + r + c];
    if (r < 3) {
        const int b = c - 3;
        if (r == b) return 0.f;
        const int l = 3 - r - b;
        return ((r + 1) % 3 == b) ? m[12 + l] : -m[12 + l];
    }
    const int ra = r - 3, cb = c - 3;
    return ra == cb ? diag(0, ra) : -m[2 + ra + cb];
}

}  // namespace fif
