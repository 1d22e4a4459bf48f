// landmark_stream.cuh -- streaming the binned landmarks near a box of nodes through shared
// memory, for the field builds (quadratic and GP visibility).
//
// The landmarks are counting-sorted into cubic bins (build.cu); the bins whose cells come
// within the cull radius of a box of nodes form one contiguous run of the sorted array per bin
// row (fixed y, z).  One thread (lane 0 of a dedicated producer warp) fills shared-memory tiles
// from that run list with bulk copies (cp.async.bulk) completing on a slot's "full" mbarrier;
// the consumer warps read the tiles in order and release each slot on its "empty" mbarrier.
#pragma once

#include "fif_common.cuh"
#include "fif_internal.h"

namespace fif {

// Run list of the bin rows near the box [blo, bhi] (cull radius rc).  Threads tid of nthr
// share the rows; every thread returns the same count.  More rows than max_runs would drop
// landmarks, so that case records FIF_ERANGE instead of truncating silently.
FIF_DEV int enumerate_runs(const BinGrid& bg, const int* startp, const float blo[3], const float bhi[3], float rc,
                           int2* runs, int max_runs, int tid, int nthr, int* err) {
    const float rc2 = rc * rc;
    const int ry0 = max(0, (int)floorf((blo[1] - rc - bg.lo[1]) * bg.inv_size));
    const int ry1 = min(bg.n[1] - 1, (int)floorf((bhi[1] + rc - bg.lo[1]) * bg.inv_size));
    const int rz0 = max(0, (int)floorf((blo[2] - rc - bg.lo[2]) * bg.inv_size));
    const int rz1 = min(bg.n[2] - 1, (int)floorf((bhi[2] + rc - bg.lo[2]) * bg.inv_size));
    const int nry = max(0, ry1 - ry0 + 1), nrz = max(0, rz1 - rz0 + 1);
    if (nry * nrz > max_runs && tid == 0) set_error(err, FIF_ERANGE);
    const int nrows = min(nry * nrz, max_runs);
    for (int r = tid; r < nrows; r += nthr) {
        const int ry = ry0 + r % nry, rz = rz0 + r / nry;
        const float ylo = bg.lo[1] + ry * bg.size, yhi = ylo + bg.size;
        const float zlo = bg.lo[2] + rz * bg.size, zhi = zlo + bg.size;
        const float dy = fmaxf(0.f, fmaxf(ylo - bhi[1], blo[1] - yhi));
        const float dz = fmaxf(0.f, fmaxf(zlo - bhi[2], blo[2] - zhi));
        const float d2 = dy * dy + dz * dz;
        int2 run = make_int2(0, 0);
        if (d2 <= rc2) {
            const float rx = sqrtf(rc2 - d2);
            const int bx0 = max(0, (int)floorf((blo[0] - rx - bg.lo[0]) * bg.inv_size));
            const int bx1 = min(bg.n[0] - 1, (int)floorf((bhi[0] + rx - bg.lo[0]) * bg.inv_size));
            if (bx1 >= bx0) {
                const int rowb = bg.n[0] * (ry + bg.n[1] * rz);
                run = make_int2(startp[rowb + bx0], startp[rowb + bx1 + 1]);
            }
        }
        runs[r] = run;
    }
    return nrows;
}

// Producer state of one CTA (used by a single thread): position in the run list.
template <int kTile>
struct TileProducer {
    int run = 0, off = 0;

    // Fill `tile` with up to kTile landmarks from the runs (one bulk copy per run piece, each
    // announced to `bar`).  Returns the count (0 marks the end); the caller publishes it in
    // shared memory and then arrives on `bar`.
    FIF_DEV int fill(float4* tile, const int2* runs, int nruns, const float4* sorted, uint64_t* bar) {
        int cnt = 0;
        while (cnt < kTile && run < nruns) {
            const int2 r = runs[run];
            const int s0 = r.x + off;
            const int take = min(r.y - s0, kTile - cnt);
            if (take > 0) {
                asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                             "r"((uint32_t)take * 16u)
                             : "memory");
                bulk_g2s(&tile[cnt], sorted + s0, (uint32_t)take * 16u, bar);
                cnt += take;
                off += take;
            }
            if (r.x + off >= r.y) {
                ++run;
                off = 0;
            }
        }
        return cnt;
    }
};

// Wait, with a short bound, until the bulk copies of fills f0 .. f1 - 1 have landed (the "full"
// phase of a fill completes when its bytes have arrived), so the producer never lets its block
// exit while a copy still writes the block's shared memory.  Slot f % kSlots must not have been
// refilled since fill f (its phase parity would then alias): a producer that gave up waiting at
// iteration it drains it - kSlots .. it - 1; after the end marker of iteration it, it - kSlots + 1
// .. it - 1.
template <int kSlots>
FIF_DEV void drain_fills(uint64_t* full, int f0, int f1, uint64_t limit_ns = 100000000ull) {
    for (int f = max(0, f0); f < f1; ++f)
        mbar_wait_bounded(&full[f % kSlots], (uint32_t)((f / kSlots) & 1), limit_ns);
}

__device__ __forceinline__ void kahan_merge(float* hs, float* ls, int idx, float x) {
    const float s = hs[idx], c = ls[idx];
    const float y = x - c;
    const float t = s + y;
    ls[idx] = (t - s) - y;
    hs[idx] = t;
}

}  // namespace fif
