// The greedy preset search of section 5 (eq. 15) with one thread-block
// cluster per frame: no grid-wide barrier.  The eight CTAs of a cluster
// split the frame's filter blocks; each computes, for all 4096 (luma pair,
// chroma pair) presets t, its blocks' sum_b min(best_b, D_b(t)) into its
// own shared memory; after a cluster barrier CTA r adds the eight partial
// sums of presets [512 r, 512 r + 512) through distributed shared memory
// and finds their least total (lowest index on ties); after a second
// barrier every CTA takes the least of the eight slice minima, so all of
// them agree on the step's preset and lower their blocks' best distortion.
// Then N in {1, 2, 4, 8} by J and each block's preset id, as in
// presets.cu.  Used for the 64-combination search without re-optimisation
// (the other variants take the grid-wide kernel).
#include <climits>
#include <cooperative_groups.h>

#include "cdef_internal.h"

namespace cg = cooperative_groups;

namespace cdefgb {
namespace {

constexpr int kCS = 8;                   // CTAs per cluster (per frame)
constexpr int kCT = 512;                 // threads per CTA
constexpr int kTuples = 4096;            // presets of the 64-combination search
constexpr int kPer = kTuples / kCT;      // presets per thread
constexpr int kSlice = kTuples / kCS;    // presets reduced by one CTA
constexpr int kStage = 16;               // blocks staged in shared memory at a time
constexpr int kMaxOwn = 2048;            // blocks one CTA can hold (frames up to 16384 blocks)

struct ClusterSmem {
    unsigned long long part[kTuples];            // this CTA's partial totals
    unsigned long long dl[kStage][64], dc[kStage][64];
    unsigned dl32[kStage][64], dc32[kStage][64]; // the same below 2^32 (narrow tables)
    unsigned long long cur[kMaxOwn];             // best distortion of the CTA's blocks
    unsigned long long red_v[kCT / 32];
    int red_t[kCT / 32];
    unsigned long long slice_v;                  // this CTA's slice minimum
    int slice_t;
    int greedy[8];
    long long totals[8];
};

__device__ __forceinline__ bool better(unsigned long long a, int ta, unsigned long long b, int tb)
{
    return a < b || (a == b && ta < tb);
}

// kNarrow: every table entry of the call is below 2^32 (squared error of
// 8-bit frames): the per-block minima are taken in 32 bits.
template <bool kNarrow>
__global__ void __launch_bounds__(kCT)
preset_cluster_kernel(const __grid_constant__ SearchBatch batch, const long long *__restrict__ dl,
                      const long long *__restrict__ dc, SearchResultDev *res, uint8_t *block_ids)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    ClusterSmem &sm = *reinterpret_cast<ClusterSmem *>(smem_raw);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int f = blockIdx.x / kCS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SearchFrameDev &F = batch.f[f];
    const int B = F.fb_cols * F.fb_rows;
    const int b0 = (int)((long long)B * rank / kCS), b1 = (int)((long long)B * (rank + 1) / kCS);
    const int own = b1 - b0;
    const unsigned long long lp = allowed_pairs(F, 0), cp = allowed_pairs(F, 1);
    const bool full = (lp & cp) == ~0ull;

    for (int b = tid; b < own; b += kCT) sm.cur[b] = ULLONG_MAX;
    __syncthreads();

    for (int step = 0; step < 8; step++) {
        // partial totals of this CTA's blocks: thread tid, presets tid + kCT j
        // (chroma pair tid % 64 for every j, luma pair tid / 64 + (kCT / 64) j)
        unsigned long long a[kPer];
#pragma unroll
        for (int j = 0; j < kPer; j++) a[j] = 0;
        const int c = tid & 63, l0 = tid >> 6;
        for (int s0 = 0; s0 < own; s0 += kStage) {
            const int ns = min(kStage, own - s0);
            for (int i = tid; i < ns * 64; i += kCT) {
                const int bb = i >> 6, q = i & 63;
                const int64_t g = (int64_t)(F.block_start + b0 + s0 + bb) * 64 + q;
                if (kNarrow) {
                    sm.dl32[bb][q] = (unsigned)dl[g];
                    sm.dc32[bb][q] = (unsigned)dc[g];
                } else {
                    sm.dl[bb][q] = (unsigned long long)dl[g];
                    sm.dc[bb][q] = (unsigned long long)dc[g];
                }
            }
            __syncthreads();
            for (int bb = 0; bb < ns; bb++) {
                const unsigned long long cb = sm.cur[s0 + bb];
                if (kNarrow) {
                    // entries sum to below 2^32 (two tables of 8-bit squared
                    // errors); the block minimum clamps to 32 bits
                    const unsigned cb32 = cb > 0xffffffffull ? 0xffffffffu : (unsigned)cb;
                    const unsigned dcv = sm.dc32[bb][c];
#pragma unroll
                    for (int j = 0; j < kPer; j++) {
                        const unsigned v = sm.dl32[bb][l0 + (kCT / 64) * j] + dcv;
                        a[j] += v < cb32 ? v : cb32;
                    }
                } else {
                    const unsigned long long dcv = sm.dc[bb][c];
#pragma unroll
                    for (int j = 0; j < kPer; j++) {
                        const unsigned long long v = sm.dl[bb][l0 + (kCT / 64) * j] + dcv;
                        a[j] += v < cb ? v : cb;
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) sm.part[tid + kCT * j] = a[j];
        cluster.sync();

        // this CTA's slice: the eight partial sums, then its least total
        unsigned long long bv = ULLONG_MAX;
        int bt = INT_MAX;
        if (tid < kSlice) {   // one preset of the slice per thread
            const int t = rank * kSlice + tid;
            unsigned long long tot = 0;
#pragma unroll
            for (int r = 0; r < kCS; r++) tot += cluster.map_shared_rank(sm.part, r)[t];
            if (full || ((lp >> (t >> 6)) & (cp >> (t & 63)) & 1)) { bv = tot; bt = t; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (better(ov, ot, bv, bt)) { bv = ov; bt = ot; }
        }
        if (lane == 0) { sm.red_v[warp] = bv; sm.red_t[warp] = bt; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < kCT / 32; w++)
                if (better(sm.red_v[w], sm.red_t[w], sm.red_v[0], sm.red_t[0])) {
                    sm.red_v[0] = sm.red_v[w];
                    sm.red_t[0] = sm.red_t[w];
                }
            sm.slice_v = sm.red_v[0];
            sm.slice_t = sm.red_t[0];
        }
        cluster.sync();

        // every CTA: the least of the slice minima (the same in all of them)
        if (tid == 0) {
            unsigned long long v = ULLONG_MAX;
            int t = INT_MAX;
            for (int r = 0; r < kCS; r++) {
                const ClusterSmem *o = cluster.map_shared_rank(&sm, r);
                if (better(o->slice_v, o->slice_t, v, t)) { v = o->slice_v; t = o->slice_t; }
            }
            sm.greedy[step] = t;
            sm.totals[step] = (long long)v;
        }
        __syncthreads();
        const int best = sm.greedy[step];
        for (int b = tid; b < own; b += kCT) {
            const int64_t g = F.block_start + b0 + b;
            const unsigned long long d =
                (unsigned long long)(dl[g * 64 + (best >> 6)] + dc[g * 64 + (best & 63)]);
            if (d < sm.cur[b]) sm.cur[b] = d;
        }
        __syncthreads();
    }

    // N in {1, 2, 4, 8} by J (ties to the smaller N); block ids over the set
    int bl = 0;
    long long bj = 0;
    for (int lg = 0; lg < 4; lg++) {
        const long long j = sm.totals[(1 << lg) - 1] + F.lambda * (long long)B * lg;
        if (lg == 0 || j < bj) { bl = lg; bj = j; }
    }
    const int N = 1 << bl;
    if (rank == 0 && tid == 0) {
        SearchResultDev &r = res[f];
        for (int j = 0; j < 8; j++) {
            r.presets[j] = sm.greedy[j];
            r.greedy[j] = sm.greedy[j];
            r.totals[j] = sm.totals[j];
        }
        for (int lg = 0; lg < 4; lg++) {
            for (int j = 0; j < 8; j++) r.refined[lg][j] = j < (1 << lg) ? sm.greedy[j] : 0;
            r.ref_totals[lg] = sm.totals[(1 << lg) - 1];
        }
        r.cost = bj;
        r.npresets = N;
    }
    for (int b = tid; b < own; b += kCT) {
        const int64_t g = F.block_start + b0 + b;
        int id = 0;
        long long bestd = LLONG_MAX;
        for (int j = 0; j < N; j++) {
            const int t = sm.greedy[j];
            const long long v = dl[g * 64 + (t >> 6)] + dc[g * 64 + (t & 63)];
            if (v < bestd) { bestd = v; id = j; }
        }
        block_ids[g] = (uint8_t)id;
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

}  // namespace

bool preset_cluster_fits(const SearchBatch &b)
{
    for (int i = 0; i < b.n; i++)
        if ((b.f[i].fb_cols * b.f[i].fb_rows + kCS - 1) / kCS > kMaxOwn) return false;
    return true;
}

cudaError_t launch_presets_cluster(const SearchBatch &b, const long long *dl, const long long *dc,
                                   SearchResultDev *results, uint8_t *block_ids, bool narrow,
                                   cudaStream_t s)
{
    static_assert(kSlice <= kCT && kCT % 64 == 0 && kTuples % kCT == 0, "thread layout");
    constexpr size_t kSmem = sizeof(ClusterSmem);
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != configured_dev) {
        for (auto *k : {preset_cluster_kernel<true>, preset_cluster_kernel<false>}) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmem);
            if (e == cudaSuccess && kCS > 8)
                e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        configured_dev = dev;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.n * kCS);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = kSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kCS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return narrow ? cudaLaunchKernelEx(&cfg, preset_cluster_kernel<true>, b, dl, dc, results, block_ids)
                  : cudaLaunchKernelEx(&cfg, preset_cluster_kernel<false>, b, dl, dc, results, block_ids);
}

}  // namespace cdefgb
