// A measurement aid with no paper counterpart: the integer issue rate of
// this GPU for the instruction mix of the filter's tap (the roofline that
// bounds the filter and the strength search is the integer pipes, whose
// ceiling is derived from the SM count and clock; this measures it).
//
// Per tap the filter issues 6 operations on the integer ALU pipe (two
// packed add-min, two packed max, the shift and its per-lane mask) and 2
// multiply-adds (the subtractions), which the compiler places on the FMA
// pipe.  The probe kernel runs that sequence in 8 independent chains per
// thread on 4 CTAs of 256 threads per SM, with every operand a runtime
// value, and the host times it with CUDA events.  mix 0: the tap sequence
// (6 ALU + 2 FMA per step); mix 1: five of the ALU operations alone.  Mixes
// 2-6 take the pipes apart, 4 instructions per step: 2 integer multiply-adds
// and 2 more, 4 multiplies-high, 2 packed maxima with 2 multiply-adds, 2
// logic operations with 2 multiply-adds, 4 fp32 FMAs.
#include "cdef_internal.h"

namespace cdefgb {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <int kMix>
__global__ void __launch_bounds__(kProbeThreads, 4)
int_mix_kernel(uint32_t seed, uint32_t m1, uint32_t sh, uint32_t mask, uint32_t floor_,
               int iters, uint32_t *sink)
{
    const uint32_t t = blockIdx.x * kProbeThreads + threadIdx.x;
    uint32_t a[kChains], b[kChains];
    float f[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) {
        a[k] = (seed ^ (t * 0x9e3779b9u)) + 0x01010101u * k;
        b[k] = (seed + t) * 0x85ebca6bu + k;
        f[k] = (float)(a[k] & 1023u);
    }
    const float fm = __uint_as_float(0x3f7fbe77u ^ (seed & 1u));   // ~0.999, a runtime value
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) {
            if (kMix == 0) {
                const uint32_t t1 = a[k] * m1 + b[k];                       // FMA pipe
                uint32_t m = __vmaxu2(__viaddmin_u16x2(a[k], b[k], t1), floor_);
                m = (m >> sh) & mask;                                      // ALU, ALU
                const uint32_t q = __vmaxu2(a[k], m * m1 + b[k]);          // FMA, ALU
                a[k] = __viaddmin_u16x2(m, b[k], q);
            } else if (kMix == 1) {   // the five ALU operations alone
                uint32_t m = __vmaxu2(__viaddmin_u16x2(a[k], b[k], sh), floor_);
                m &= mask;
                a[k] = __viaddmin_u16x2(m, b[k], __vmaxu2(a[k], m));
            } else if (kMix == 2) {   // 4 integer multiply-adds
                a[k] = a[k] * m1 + b[k];
                b[k] = b[k] * m1 + a[k];
                a[k] = a[k] * m1 + b[k];
                b[k] = b[k] * m1 + a[k];
            } else if (kMix == 3) {   // 4 multiplies-high
                a[k] = __umulhi(a[k], floor_);
                b[k] = __umulhi(b[k], a[k]);
                a[k] = __umulhi(a[k], m1);
                b[k] = __umulhi(b[k], mask);
            } else if (kMix == 4) {   // 2 packed maxima, 2 multiply-adds
                a[k] = __vmaxu2(a[k], b[k]);
                b[k] = b[k] * m1 + a[k];
                a[k] = __vmaxu2(a[k], b[k]);
                b[k] = b[k] * m1 + a[k];
            } else if (kMix == 5) {   // 2 logic operations, 2 multiply-adds
                a[k] = (a[k] & b[k]) ^ mask;
                b[k] = b[k] * m1 + a[k];
                a[k] = (a[k] ^ b[k]) & mask;
                b[k] = b[k] * m1 + a[k];
            } else {                  // 4 fp32 FMAs
                f[k] = f[k] * fm + 1.0f;
                f[k] = f[k] * fm + 0.5f;
                f[k] = f[k] * fm + 0.25f;
                f[k] = f[k] * fm + 0.125f;
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kChains; k++) x ^= a[k] ^ b[k] ^ __float_as_uint(f[k]);
    if (x == seed) sink[t & 1023] = x;   // keeps the chains live; practically never taken
}

}  // namespace

int probe_int_mix(int device, int mix, int iters, double *lane_instr_per_s, cudaStream_t s)
{
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return CDEF_ERR_CUDA;
    uint32_t *sink = nullptr;
    if (cudaMallocAsync(&sink, 1024 * sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_NOMEM;
    }
    const dim3 grid(sms * 4);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto launch = [&](int n) {
        switch (mix) {
#define CDEF_PROBE_LAUNCH(M)                                                                    \
    case M:                                                                                     \
        int_mix_kernel<M><<<grid, kProbeThreads, 0, s>>>(0x1234567u, 0xffffffffu, 2u, 0x3fff3fffu, \
                                                         0x08000800u, n, sink);                 \
        break;
            CDEF_PROBE_LAUNCH(0)
            CDEF_PROBE_LAUNCH(1)
            CDEF_PROBE_LAUNCH(2)
            CDEF_PROBE_LAUNCH(3)
            CDEF_PROBE_LAUNCH(4)
            CDEF_PROBE_LAUNCH(5)
            CDEF_PROBE_LAUNCH(6)
#undef CDEF_PROBE_LAUNCH
        }
    };
    if (e == cudaSuccess) {
        launch(iters / 8 + 1);   // warm-up
        e = cudaEventRecord(e0, s);
    }
    if (e == cudaSuccess) {
        launch(iters);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(sink, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    const double per_step = mix == 0 ? 8.0 : mix == 1 ? 5.0 : 4.0;   // warp instructions per chain step
    const double lanes = (double)grid.x * kProbeThreads * kChains * iters * per_step;
    *lane_instr_per_s = ms > 0.f ? lanes / (ms * 1e-3) : 0.0;
    return CDEF_OK;
}

}  // namespace cdefgb
