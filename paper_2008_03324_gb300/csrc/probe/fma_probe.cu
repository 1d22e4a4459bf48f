// fma_probe.cu -- FP32 FMA throughput probe (sm_103a), built as its own library
// (libfif_probe.so) for the benchmark and kept out of the product library and its header.
// Measurement infrastructure for the roofline of the ALU-bound kernels (the field builds), not
// part of the method: every thread
// runs `iters` rounds of eight independent FMA chains -- scalar fma.rn.f32, or four chains of
// packed fma.rn.f32x2 carrying the same eight lanes of work -- unrolled 8 rounds deep so that
// loop control takes few issue slots and the FMA pipe is the only limit.  Work per launch: 2 * 8 * iters flops per thread (both forms).
#include <cstdint>

#include "../fif_common.cuh"

namespace fif {

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float* sink, int iters, int packed, float a,
                                                                  float b) {
    const float s = (float)(blockIdx.x * kProbeThreads + threadIdx.x) * 1e-9f;
    float out;
    if (packed) {
        float2 x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = make_float2(s + (float)k, s - (float)k);
        const float2 va = make_float2(a, a), vb = make_float2(b, b);
#pragma unroll 8
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = fma2(x[k], va, vb);
        out = ((x[0].x + x[0].y) + (x[1].x + x[1].y)) + ((x[2].x + x[2].y) + (x[3].x + x[3].y));
    } else {
        float x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = s + (float)k;
#pragma unroll 8
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
        out = ((x[0] + x[1]) + (x[2] + x[3])) + ((x[4] + x[5]) + (x[6] + x[7]));
    }
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = out;
}

}  // namespace

}  // namespace fif

// d_sink: device float[blocks * 256]; FIF_OK, FIF_EINVAL (bad count or NULL), FIF_EALIGN or FIF_ECUDA
extern "C" __attribute__((visibility("default"))) int32_t fif_fma_probe(float* d_sink, int64_t blocks,
                                                                      int32_t iters, int32_t packed,
                                                                      cudaStream_t stream) {
    if (!d_sink || blocks <= 0 || blocks > (int64_t)INT32_MAX || iters <= 0) return FIF_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_sink) & 3u) return FIF_EALIGN;
    // a = 1 - 2^-20, b = 2^-24: the chains stay finite and bounded for any iteration count
    fif::fma_probe_kernel<<<(unsigned)blocks, fif::kProbeThreads, 0, stream>>>(
        d_sink, iters, packed ? 1 : 0, 1.f - 9.5367431640625e-7f, 5.9604644775390625e-8f);
    return cudaPeekAtLastError() == cudaSuccess ? FIF_OK : FIF_ECUDA;
}
