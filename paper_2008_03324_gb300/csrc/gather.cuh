// gather.cuh -- shared-memory image of the 8 corner coefficient sets of one pose, used by
// the query and its adjoint: 4 x-adjacent node pairs land in 4 slots whose offsets put the
// 8 corner bases on distinct 4-bank groups (residues 0, 16, 64, 80 modulo 128 B plus the
// 864-B node offset), so a warp whose lane (j, q) reads corner j, entries e = q (mod 4) of
// each monomial block, hits 32 distinct banks.
#pragma once

#include "fif_common.cuh"

namespace fif {
namespace gather {

constexpr int kWarps = 3;          // warps per CTA (independent)
constexpr int kStages = 3;         // pose stages in the shared-memory ring
constexpr int kPrefetch = 4;       // L2 prefetch distance (poses)
constexpr int kMomStride = 85;     // floats per pose in the moment table (odd: no bank conflicts)
constexpr int kNumMom = 84;

// per-pose shared-memory image: 4 pair slots (1728 B each for f32) at offsets chosen so the
// 8 corner bases fall on distinct 4-bank groups (residues 0, 16, 64, 80 modulo 128 B)
template <int kElem>
struct Layout;
template <>
struct Layout<4> {
    static constexpr int kStride = 216;                 // floats per node
    static constexpr int kBlock = 21;                   // elements per monomial block
    static constexpr int kNodeBytes = kStride * 4;      // 864
    static constexpr int kPairBytes = 2 * kNodeBytes;   // 1728
    static constexpr int kPoseBytes = 7296;             // 57 * 128
    __device__ static constexpr int slot(int P) { return P * 1792 + (P == 0 ? 0 : P == 1 ? 16 : P == 2 ? 64 : 80); }
    __device__ static float load(const unsigned char* p, int idx) { return reinterpret_cast<const float*>(p)[idx]; }
};
// bfloat16 storage: 224 elements (448 B) per node, pair 896 B; monomial block k holds its 21
// entries at 22 k + e and a zero at 22 k + 21 (elements 220..223 zero), so 32-bit word 11 k + p
// holds entries 2p and 2p + 1 of block k.  The corners of pair P start at residues 16 P and
// 16 P + 64 modulo 128 B, so the 8 corners occupy distinct 4-bank groups and the 4 lanes of a
// corner, reading 4 consecutive words, never collide with another corner
template <>
struct Layout<2> {
    static constexpr int kStride = 224;
    static constexpr int kBlock = 22;                   // elements per monomial block
    static constexpr int kNodeBytes = kStride * 2;      // 448
    static constexpr int kPairBytes = 2 * kNodeBytes;   // 896
    static constexpr int kPoseBytes = 4096;
    __device__ static constexpr int slot(int P) { return P * 1024 + 16 * P; }
    __device__ static float load(const unsigned char* p, int idx) {
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(p)[idx]);
    }
};


__host__ __device__ constexpr int sym3_idx(int r, int c) {
    return (r <= c) ? (r * 3 - (r * (r - 1)) / 2 + (c - r)) : (c * 3 - (c * (c - 1)) / 2 + (r - c));
}

// K_a = [e_a]x
__host__ __device__ inline float kx(int a, int r, int c) {
    const float e[3] = {a == 0 ? 1.f : 0.f, a == 1 ? 1.f : 0.f, a == 2 ? 1.f : 0.f};
    const float S[3][3] = {{0.f, -e[2], e[1]}, {e[2], 0.f, -e[0]}, {-e[1], e[0], 0.f}};
    return S[r][c];
}

}  // namespace gather
}  // namespace fif
