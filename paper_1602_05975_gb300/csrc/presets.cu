// Preset selection of the strength search (section 5, eq. 15): the greedy
// search, the optional one-at-a-time re-optimisation of the presets, and
// the final choice of N and of each block's preset, as ONE persistent
// kernel whose phases are separated by grid-wide barriers.
//
// Phases of one step:
//   partial  every CTA takes chunks of 16 filter blocks of any frame and
//            adds, for all 4096 (luma pair, chroma pair) presets t, the
//            chunk's sum_b min(best_b, D_b(t)) to the frame's totals (u64
//            atomics); best_b is the block's least distortion over the
//            presets kept so far (greedy) or over all presets but the one
//            being re-chosen (re-optimisation);
//   select   one CTA per frame takes the least total (greedy: lowest index
//            on ties; re-optimisation: the current preset if it attains the
//            least total, else the lowest index), records it, lowers the
//            blocks' best distortion (greedy) and clears the totals.
// The kernel is launched cooperatively (every CTA resident), so the
// barriers complete; each barrier wait is bounded and sets the timeout
// status bit when it gives up.
#include <climits>

#include "cdef_internal.h"
#include "tma.cuh"

namespace cdefgb {
namespace {

constexpr int kChunk = 16;         // blocks per partial unit
constexpr int kThreads = 256;
constexpr int kMaxWidth = 128;     // combinations per plane group (64 or 128)
constexpr int kPerThread = 16;     // presets per thread and group of 4096
constexpr long long kBarrierCycles = 1ll << 30;

struct Ctl {                       // lives in device scratch
    unsigned arrive;               // CTAs arrived at the current barrier
    unsigned gen;                  // barrier generation
    unsigned done_frames[4];       // per set size: frames whose re-optimisation converged
                                   // (never reset inside a launch: every CTA reads the
                                   // count of its size after the pass's barrier)
    unsigned changed[kMaxBatch];   // the current pass changed a preset
    unsigned done[kMaxBatch];      // the frame's re-optimisation converged
};

static_assert(sizeof(Ctl) <= kPresetCtlBytes, "preset control block outgrew its scratch");

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier; false when the wait gave up (status set).
__device__ bool grid_sync(Ctl *ctl, int *status)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire(&ctl->gen);
        __threadfence();
        if (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1) {
            atomicExch(&ctl->arrive, 0u);
            __threadfence();
            st_release(&ctl->gen, g + 1);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(&ctl->gen) == g) {
                if (clock64() - t0 > kBarrierCycles) {
                    atomicOr(status, kStatusTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int frame_chunks(const SearchFrameDev &F)
{
    return (F.fb_cols * F.fb_rows + kChunk - 1) / kChunk;
}

__device__ __forceinline__ unsigned long long dist_of(const long long *dl, const long long *dc,
                                                      int width, int g, int t)
{
    return (unsigned long long)(dl[(int64_t)g * width + t / width] +
                                dc[(int64_t)g * width + t % width]);
}

struct Shared {
    unsigned long long dl[kChunk][kMaxWidth], dc[kChunk][kMaxWidth], cur[kChunk];
    unsigned long long red_v[kThreads / 32];
    int red_t[kThreads / 32];
    int best;
};

// partial phase.  refine_lg < 0: greedy (best_b from `cur`); otherwise the
// re-optimisation of slot k of the set of size n = 1 << refine_lg.
__device__ void partial_phase(const SearchBatch &batch, const long long *dl, const long long *dc,
                              const unsigned long long *cur, unsigned long long *tot,
                              const SearchResultDev *res, const Ctl *ctl, int refine_lg, int k,
                              int width, const uint8_t *skipped, Shared &sh)
{
    const int ntuples = width * width;
    const int tid = threadIdx.x;
    int units = 0;
    for (int f = 0; f < batch.n; f++) units += frame_chunks(batch.f[f]);
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        int fi = 0, c = u;
        while (c >= frame_chunks(batch.f[fi])) c -= frame_chunks(batch.f[fi++]);
        if (refine_lg >= 0 && __ldcg(&ctl->done[fi])) continue;
        const SearchFrameDev &F = batch.f[fi];
        const int B = F.fb_cols * F.fb_rows;
        const int b0 = c * kChunk, nb = min(kChunk, B - b0);
        const int g0 = F.block_start + b0;
        for (int i = tid; i < nb * width; i += kThreads) {
            const int b = i / width, q = i - b * width;
            sh.dl[b][q] = (unsigned long long)dl[(int64_t)(g0 + b) * width + q];
            sh.dc[b][q] = (unsigned long long)dc[(int64_t)(g0 + b) * width + q];
        }
        __syncthreads();
        if (tid < nb) {
            unsigned long long m;
            if (skipped && skipped[g0 + tid]) {
                m = 0;   // no preset id: the block adds nothing to any total
            } else if (refine_lg < 0) {
                m = __ldcg(&cur[g0 + tid]);
            } else {
                const int n = 1 << refine_lg;
                m = ULLONG_MAX;
                for (int j = 0; j < n; j++) {
                    if (j == k) continue;
                    const int t = __ldcg(&res[fi].refined[refine_lg][j]);
                    const unsigned long long v = sh.dl[tid][t / width] + sh.dc[tid][t % width];
                    m = v < m ? v : m;
                }
            }
            sh.cur[tid] = m;
        }
        __syncthreads();
        // thread tid, group g: presets t = g * 4096 + tid + 256 q, whose
        // chroma combination is always tid % width
        const int ci = tid % width, lstep = kThreads / width;
        unsigned long long *t = tot + (int64_t)fi * ntuples;
        for (int g = 0; g < ntuples / 4096; g++) {
            const int l0 = (g * 4096 + tid) / width;
            unsigned long long a[kPerThread];
#pragma unroll
            for (int q = 0; q < kPerThread; q++) a[q] = 0;
            for (int b = 0; b < nb; b++) {
                const unsigned long long cv = sh.cur[b], dcv = sh.dc[b][ci];
#pragma unroll
                for (int q = 0; q < kPerThread; q++) {
                    const unsigned long long v = sh.dl[b][l0 + lstep * q] + dcv;
                    a[q] += v < cv ? v : cv;
                }
            }
#pragma unroll
            for (int q = 0; q < kPerThread; q++)
                atomicAdd(&t[g * 4096 + tid + kThreads * q], a[q]);
        }
        __syncthreads();   // before the next unit overwrites the shared tables
    }
}

__device__ __forceinline__ bool better(unsigned long long a, int ta, unsigned long long b, int tb)
{
    return a < b || (a == b && ta < tb);
}

// The least of a frame's totals over the presets whose luma and chroma
// combinations are both allowed (section 5's low-complexity search; the
// mask of pair q covers q and 64 + q), and its lowest index (whole CTA).
__device__ void frame_argmin(unsigned long long *t, int width, const SearchFrameDev &F, Shared &sh,
                             unsigned long long *min_v, int *min_t)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntuples = width * width, lg = width == 128 ? 7 : 6;
    const unsigned long long lp = allowed_pairs(F, 0), cp = allowed_pairs(F, 1);
    unsigned long long bv = ULLONG_MAX;
    int bt = INT_MAX;
    if ((lp & cp) == ~0ull) {
        for (int i = tid; i < ntuples; i += kThreads) {
            const unsigned long long v = __ldcg(&t[i]);
            if (better(v, i, bv, bt)) { bv = v; bt = i; }
        }
    } else {
        for (int i = tid; i < ntuples; i += kThreads) {
            const int ql = (i >> lg) & 63, qc = i & 63;
            if (!((lp >> ql) & (cp >> qc) & 1)) continue;
            const unsigned long long v = __ldcg(&t[i]);
            if (better(v, i, bv, bt)) { bv = v; bt = i; }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
        if (better(ov, ot, bv, bt)) { bv = ov; bt = ot; }
    }
    if (lane == 0) { sh.red_v[warp] = bv; sh.red_t[warp] = bt; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kThreads / 32; w++)
            if (better(sh.red_v[w], sh.red_t[w], sh.red_v[0], sh.red_t[0])) {
                sh.red_v[0] = sh.red_v[w];
                sh.red_t[0] = sh.red_t[w];
            }
    }
    __syncthreads();
    *min_v = sh.red_v[0];
    *min_t = sh.red_t[0];
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
preset_kernel(const __grid_constant__ SearchBatch batch, const long long *__restrict__ dl,
              const long long *__restrict__ dc, unsigned long long *cur, unsigned long long *tot,
              SearchResultDev *res, uint8_t *block_ids, int *status, Ctl *ctl, int refine_passes,
              int width, const uint8_t *skipped)
{
    __shared__ Shared sh;
    const int tid = threadIdx.x;
    const int stride = gridDim.x * kThreads;
    const int n = batch.n;
    const int ntuples = width * width;

    for (int i = blockIdx.x * kThreads + tid; i < batch.total_blocks; i += stride) cur[i] = ULLONG_MAX;
    for (int i = blockIdx.x * kThreads + tid; i < n * ntuples; i += stride) tot[i] = 0;
    if (blockIdx.x == 0 && tid < n) {
        ctl->changed[tid] = 0;
        ctl->done[tid] = 0;
    }
    if (blockIdx.x == 0 && tid < 4) ctl->done_frames[tid] = 0;
    if (!grid_sync(ctl, status)) return;

    // ---- greedy: preset `step` is the best addition to presets 0..step-1
    for (int step = 0; step < 8; step++) {
        partial_phase(batch, dl, dc, cur, tot, res, ctl, -1, 0, width, skipped, sh);
        if (!grid_sync(ctl, status)) return;
        for (int f = blockIdx.x; f < n; f += gridDim.x) {
            unsigned long long *t = tot + (int64_t)f * ntuples;
            unsigned long long v;
            int best;
            frame_argmin(t, width, batch.f[f], sh, &v, &best);
            if (tid == 0) {
                res[f].greedy[step] = best;
                res[f].totals[step] = (long long)v;
            }
            const SearchFrameDev &F = batch.f[f];
            const int B = F.fb_cols * F.fb_rows;
            for (int b = tid; b < B; b += kThreads) {
                const int g = F.block_start + b;
                const unsigned long long d = dist_of(dl, dc, width, g, best);
                if (d < __ldcg(&cur[g])) cur[g] = d;
            }
            for (int i = tid; i < ntuples; i += kThreads) t[i] = 0;
            __syncthreads();
        }
        if (!grid_sync(ctl, status)) return;
    }

    // ---- sets of size 1, 2, 4, 8 from the greedy prefixes
    for (int f = blockIdx.x; f < n; f += gridDim.x) {
        if (tid < 4) {
            const int sz = 1 << tid;
            for (int j = 0; j < 8; j++) res[f].refined[tid][j] = j < sz ? res[f].greedy[j] : 0;
            res[f].ref_totals[tid] = res[f].totals[sz - 1];
        }
    }
    if (!grid_sync(ctl, status)) return;

    // ---- re-optimisation, one preset at a time (sizes 2, 4, 8; size 1 is
    // exhaustive already)
    for (int lg = 1; lg <= 3 && refine_passes > 0; lg++) {
        const int sz = 1 << lg;
        for (int pass = 0; pass < refine_passes; pass++) {
            for (int k = 0; k < sz; k++) {
                partial_phase(batch, dl, dc, cur, tot, res, ctl, lg, k, width, skipped, sh);
                if (!grid_sync(ctl, status)) return;
                for (int f = blockIdx.x; f < n; f += gridDim.x) {
                    if (__ldcg(&ctl->done[f])) continue;
                    unsigned long long *t = tot + (int64_t)f * ntuples;
                    const int old = __ldcg(&res[f].refined[lg][k]);
                    const unsigned long long old_v = __ldcg(&t[old]);
                    unsigned long long v;
                    int best;
                    frame_argmin(t, width, batch.f[f], sh, &v, &best);
                    if (tid == 0) {
                        if (old_v == v) best = old;        // keep the current preset on ties
                        if (best != old) {
                            res[f].refined[lg][k] = best;
                            ctl->changed[f] = 1;
                        }
                        res[f].ref_totals[lg] = (long long)v;
                    }
                    for (int i = tid; i < ntuples; i += kThreads) t[i] = 0;
                    __syncthreads();
                }
                if (!grid_sync(ctl, status)) return;
            }
            // end of the pass: a frame whose pass changed nothing is done
            for (int f = blockIdx.x; f < n; f += gridDim.x) {
                if (tid == 0 && !ctl->done[f]) {
                    if (!ctl->changed[f]) {
                        ctl->done[f] = 1;
                        atomicAdd(&ctl->done_frames[lg], 1u);
                    }
                    ctl->changed[f] = 0;
                }
            }
            if (!grid_sync(ctl, status)) return;
            if (ld_acquire(&ctl->done_frames[lg]) == (unsigned)n) break;
        }
        // next size: every frame starts again (each CTA resets only the
        // flags of its own frames, which no other CTA reads before the
        // barrier below)
        for (int f = blockIdx.x; f < n; f += gridDim.x)
            if (tid == 0) {
                ctl->done[f] = 0;
                ctl->changed[f] = 0;
            }
        if (!grid_sync(ctl, status)) return;
    }

    // ---- N in {1, 2, 4, 8} by J (ties to the smaller N), then each block's
    // least-distortion preset of that set (ties to the lower index)
    for (int f = blockIdx.x; f < n; f += gridDim.x) {
        const SearchFrameDev &F = batch.f[f];
        const int B = F.fb_cols * F.fb_rows;
        if (tid == 0) {
            int coded_blocks = B;   // blocks that signal a preset id
            if (skipped)
                for (int b = 0; b < B; b++) coded_blocks -= skipped[F.block_start + b] != 0;
            int bl = 0;
            long long bj = 0;
            for (int lg = 0; lg < 4; lg++) {
                const long long j = res[f].ref_totals[lg] + F.lambda * (long long)coded_blocks * lg;
                if (lg == 0 || j < bj) { bl = lg; bj = j; }
            }
            res[f].cost = bj;
            res[f].npresets = 1 << bl;
            // entries past N keep the greedy order (unspecified for callers)
            for (int j = 0; j < 8; j++)
                res[f].presets[j] = j < (1 << bl) ? res[f].refined[bl][j] : res[f].greedy[j];
            sh.best = 1 << bl;
        }
        __syncthreads();
        const int N = sh.best;
        for (int b = tid; b < B; b += kThreads) {
            const int g = F.block_start + b;
            int id = 0;
            if (!(skipped && skipped[g])) {
                long long bestd = LLONG_MAX;
                for (int j = 0; j < N; j++) {
                    const long long v = (long long)dist_of(dl, dc, width, g, res[f].presets[j]);
                    if (v < bestd) { bestd = v; id = j; }
                }
            }
            block_ids[g] = (uint8_t)id;
        }
        __syncthreads();
    }
}

// As many CTAs as the partial phases have chunks (and at least one per
// frame for the select phases), at most two per SM: fewer CTAs make the
// barriers of small searches cheaper.
int preset_grid(const SearchBatch &b)
{
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, preset_kernel, kThreads, 0);
        cached = sms * (occ < 2 ? (occ > 0 ? occ : 1) : 2);
        cached_dev = dev;
    }
    int units = 0;
    for (int i = 0; i < b.n; i++) units += (b.f[i].fb_cols * b.f[i].fb_rows + kChunk - 1) / kChunk;
    const int want = units > b.n ? units : b.n;
    return want < cached ? want : cached;
}

}  // namespace

size_t preset_ctl_bytes() { return sizeof(Ctl); }

cudaError_t launch_presets(const SearchBatch &b, const long long *dl, const long long *dc,
                           unsigned long long *cur, unsigned long long *tot, void *ctl,
                           SearchResultDev *results, uint8_t *block_ids, int *status,
                           int refine_passes, int width, const uint8_t *skipped, cudaStream_t s)
{
    if (width != 64 && width != kMaxWidth) return cudaErrorInvalidValue;
    // a barrier abandoned by an earlier timed-out launch must not leave
    // CTAs counted: the arrival count starts at zero
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(preset_grid(b));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Ctl *c = static_cast<Ctl *>(ctl);
    return cudaLaunchKernelEx(&cfg, preset_kernel, b, dl, dc, cur, tot, results, block_ids, status,
                              c, refine_passes, width, skipped);
}

}  // namespace cdefgb
