// Pieces of section 5's preset selection (eq. 15, the greedy search and the
// one-at-a-time re-optimisation) over a range of filter blocks, for a
// selection that the host drives step by step: a strength search sharded
// over devices, each holding the distortion tables of its own blocks, sums
// its per-preset totals with the others' through a collective before every
// argmin.  Integer arithmetic; the totals of a step over several block
// ranges add up to the totals over their union exactly.
#include <cuda_runtime.h>

#include <cstdint>

#include "cdef_internal.h"

namespace cdefgb {

namespace {

constexpr int kTotThreads = 256;     // presets per CTA row
constexpr int kTotBlocks = 32;       // filter blocks per CTA column
constexpr int kArgThreads = 1024;
constexpr int kAssignThreads = 256;

__device__ __forceinline__ unsigned long long dist(const long long *dl, const long long *dc,
                                                   int width, int b, int t)
{
    return (unsigned long long)(dl[(int64_t)b * width + t / width] +
                                dc[(int64_t)b * width + t % width]);
}

// totals[t] += sum over the CTA's blocks of min(best[b], D_b(t)); a warp
// reads one luma entry (broadcast) and 32 consecutive chroma entries per
// block.
__global__ void __launch_bounds__(kTotThreads)
preset_totals_kernel(int nblocks, int width, const long long *dl, const long long *dc,
                     const uint8_t *skipped, const unsigned long long *best, long long *totals)
{
    const int t = blockIdx.x * kTotThreads + threadIdx.x;
    const int b0 = blockIdx.y * kTotBlocks;
    const int b1 = min(nblocks, b0 + kTotBlocks);
    if (t >= width * width) return;
    unsigned long long acc = 0;
    for (int b = b0; b < b1; b++) {
        if (skipped && skipped[b]) continue;
        unsigned long long m = dist(dl, dc, width, b, t);
        if (best) m = min(m, best[b]);
        acc += m;
    }
    if (acc) atomicAdd(reinterpret_cast<unsigned long long *>(totals) + t, acc);
}

struct ArgMin {
    long long v;
    int t;
};

__device__ __forceinline__ ArgMin better(ArgMin a, ArgMin b)
{
    if (b.t < 0) return a;
    if (a.t < 0) return b;
    return (b.v < a.v || (b.v == a.v && b.t < a.t)) ? b : a;
}

// One CTA: the least total among the allowed presets, lowest index on ties;
// `keep` (the slot's current preset in a re-optimisation step) is kept when
// it attains the least total.
__global__ void __launch_bounds__(kArgThreads)
preset_argmin_kernel(int width, const long long *totals, unsigned long long luma_pairs,
                     unsigned long long chroma_pairs, int keep, long long *out)
{
    __shared__ ArgMin part[kArgThreads / 32];
    ArgMin m = {0, -1};
    for (int t = threadIdx.x; t < width * width; t += kArgThreads) {
        const int ql = (t / width) & 63, qc = (t % width) & 63;
        if (!((luma_pairs >> ql) & 1) || !((chroma_pairs >> qc) & 1)) continue;
        m = better(m, ArgMin{totals[t], t});
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        ArgMin n;
        n.v = __shfl_xor_sync(0xffffffffu, m.v, o);
        n.t = __shfl_xor_sync(0xffffffffu, m.t, o);
        m = better(m, n);
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        ArgMin r = part[0];
        for (int w = 1; w < kArgThreads / 32; w++) r = better(r, part[w]);
        if (keep >= 0 && r.t >= 0 && totals[keep] == r.v) r.t = keep;
        out[0] = r.t;
        out[1] = r.t >= 0 ? totals[r.t] : 0;
    }
}

// One thread per block: its least distortion over the set and the first
// preset of the set attaining it; warp sums of the least distortions and
// of the blocks counted.
__global__ void __launch_bounds__(kAssignThreads)
preset_assign_kernel(int nblocks, int width, const long long *dl, const long long *dc,
                     const uint8_t *skipped, PresetList set, unsigned long long *best, uint8_t *ids,
                     long long *sums)
{
    const int b = blockIdx.x * kAssignThreads + threadIdx.x;
    unsigned long long s = 0, counted = 0;
    if (b < nblocks) {
        int id = 0;
        unsigned long long m = 0;
        const bool skip = skipped && skipped[b];
        if (!skip && set.n == 0) {
            m = ~0ull;
        } else if (!skip) {
            m = dist(dl, dc, width, b, set.t[0]);
#pragma unroll 1
            for (int k = 1; k < set.n; k++) {
                const unsigned long long d = dist(dl, dc, width, b, set.t[k]);
                if (d < m) {
                    m = d;
                    id = k;
                }
            }
            s = m;
        }
        counted = skip ? 0 : 1;
        if (best) best[b] = m;
        if (ids) ids[b] = (uint8_t)id;
    }
    if (!sums) return;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        counted += __shfl_xor_sync(0xffffffffu, counted, o);
    }
    if ((threadIdx.x & 31) == 0 && (s || counted)) {
        atomicAdd(reinterpret_cast<unsigned long long *>(sums), s);
        atomicAdd(reinterpret_cast<unsigned long long *>(sums) + 1, counted);
    }
}

}  // namespace

cudaError_t launch_preset_totals(int nblocks, int width, const long long *dl, const long long *dc,
                                 const uint8_t *skipped, const unsigned long long *best,
                                 long long *totals, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    const dim3 grid((width * width + kTotThreads - 1) / kTotThreads,
                    (nblocks + kTotBlocks - 1) / kTotBlocks);
    preset_totals_kernel<<<grid, kTotThreads, 0, s>>>(nblocks, width, dl, dc, skipped, best, totals);
    return cudaGetLastError();
}

cudaError_t launch_preset_argmin(int width, const long long *totals, unsigned long long luma_pairs,
                                 unsigned long long chroma_pairs, int keep, long long *out,
                                 cudaStream_t s)
{
    preset_argmin_kernel<<<1, kArgThreads, 0, s>>>(width, totals, luma_pairs, chroma_pairs, keep,
                                                   out);
    return cudaGetLastError();
}

cudaError_t launch_preset_assign(int nblocks, int width, const long long *dl, const long long *dc,
                                 const uint8_t *skipped, PresetList set, unsigned long long *best,
                                 uint8_t *ids, long long *sums, cudaStream_t s)
{
    if (nblocks <= 0) return cudaSuccess;
    preset_assign_kernel<<<(nblocks + kAssignThreads - 1) / kAssignThreads, kAssignThreads, 0, s>>>(
        nblocks, width, dl, dc, skipped, set, best, ids, sums);
    return cudaGetLastError();
}

}  // namespace cdefgb
