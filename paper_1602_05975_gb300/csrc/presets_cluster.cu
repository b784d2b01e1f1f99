// The greedy preset search of section 5 (eq. 15) with one thread-block
// cluster per frame: no grid-wide barrier.  The eight CTAs of a cluster
// split the frame's filter blocks; each computes, for all 4096 (luma pair,
// chroma pair) presets t, its blocks' sum_b min(best_b, D_b(t)) into its
// own shared memory; after a cluster barrier CTA r adds the eight partial
// sums of presets [512 r, 512 r + 512) through distributed shared memory
// and finds their least total (lowest index on ties); after a second
// barrier every CTA takes the least of the eight slice minima, so all of
// them agree on the step's preset and lower their blocks' best distortion.
// The re-optimisation passes (section 5) re-choose one slot of a set at a
// time with the same step, each block's best distortion being its least
// over the set's other slots.  Then N in {1, 2, 4, 8} by J and each block's
// preset id, as in presets.cu.  Used for the 64-combination search (the
// 128-combination search takes the grid-wide kernel).
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
constexpr int kMaxOwn = 2048;            // blocks one CTA can hold (frames up to 16384 blocks)
constexpr int kTabBytes = 128 * 1024;    // the CTA's luma and chroma table rows

struct ClusterSmem {
    unsigned long long part[kTuples];            // this CTA's partial totals
    unsigned long long cur[kMaxOwn];             // best distortion of the CTA's blocks
    alignas(16) unsigned char tab[kTabBytes];    // table rows: luma [cap][64], chroma [cap][64]
    unsigned long long red_v[kCT / 32];
    int red_t[kCT / 32];
    unsigned long long slice_v;                  // this CTA's slice minimum
    int slice_t;
    unsigned long long slice_old;                // total of the step's current preset (its slice's CTA)
    int step_t;                                  // the step's chosen preset
    unsigned long long step_v;                   // and its total
    int greedy[8];
    long long totals[8];
    int refined[4][8];                           // sets of size 1, 2, 4, 8 (re-optimised)
    long long ref_totals[4];
};

__device__ __forceinline__ bool better(unsigned long long a, int ta, unsigned long long b, int tb)
{
    return a < b || (a == b && ta < tb);
}

// Eight consecutive entries of a shared-memory row (16-byte aligned).
template <typename T>
__device__ __forceinline__ void load8(const T *p, T (&v)[kPer])
{
    static_assert(kPer == 8, "eight presets per thread");
    if constexpr (sizeof(T) == 4) {
        const uint4 x = reinterpret_cast<const uint4 *>(p)[0];
        const uint4 y = reinterpret_cast<const uint4 *>(p)[1];
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
        v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const ulonglong2 x = reinterpret_cast<const ulonglong2 *>(p)[k];
            v[2 * k] = x.x;
            v[2 * k + 1] = x.y;
        }
    }
}

// a[j] += sum over n blocks of min(cur_b, L_b(lq + j) + C_b(c)).  With
// 32-bit entries (8-bit squared errors: a block's luma and chroma entries
// sum to at most 3 x 4096 x 255^2 < 2^30) four blocks' minima are summed
// in 32 bits before the 64-bit totals.
template <typename T>
__device__ __forceinline__ void sum_blocks(const T (*rl)[64], const T (*rc)[64], const T *cur,
                                           int n, int c, int lq, unsigned long long (&a)[kPer])
{
    constexpr int kChunk = sizeof(T) == 4 ? 4 : 1;
    for (int b0 = 0; b0 < n; b0 += kChunk) {
        T sum[kPer];
#pragma unroll
        for (int j = 0; j < kPer; j++) sum[j] = 0;
#pragma unroll
        for (int k = 0; k < kChunk; k++) {
            const int bb = b0 + k;
            if (kChunk > 1 && bb >= n) break;
            const T cb = cur[bb], dcv = rc[bb][c];
            T v[kPer];
            load8(rl[bb] + lq, v);
#pragma unroll
            for (int j = 0; j < kPer; j++) {
                const T x = v[j] + dcv;
                sum[j] += x < cb ? x : cb;
            }
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) a[j] += sum[j];
    }
}

// T: the width of the per-block minima; 32 bits when every table entry of
// the call is an 8-bit squared error (below 2^30).
template <typename T>
__global__ void __launch_bounds__(kCT, 1)
preset_cluster_kernel(const __grid_constant__ SearchBatch batch, const long long *__restrict__ dl,
                      const long long *__restrict__ dc, SearchResultDev *res, uint8_t *block_ids,
                      int refine_passes)
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
    // table rows of `cap` blocks fit; with own <= cap they stay for all steps
    constexpr int cap = kTabBytes / (2 * 64 * (int)sizeof(T));
    T (*rl)[64] = reinterpret_cast<T (*)[64]>(sm.tab);
    T (*rc)[64] = rl + cap;
    T *cur = reinterpret_cast<T *>(sm.cur);
    const bool resident = own <= cap;
    auto stage = [&](int s0, int n) {
        for (int i = tid; i < n * 64; i += kCT) {
            const int bb = i >> 6, q = i & 63;
            const int64_t g = (int64_t)(F.block_start + b0 + s0 + bb) * 64 + q;
            rl[bb][q] = (T)dl[g];
            rc[bb][q] = (T)dc[g];
        }
    };

    for (int b = tid; b < own; b += kCT) cur[b] = (T)~0ull;
    if (resident) stage(0, own);
    __syncthreads();

    // thread tid: chroma pair c, luma pairs lq .. lq + 7 (presets (lq + j) * 64 + c)
    const int c = tid & 63, lq = (tid >> 6) * kPer;
    // D_b(t) of the CTA's block b
    auto dist = [&](int b, int t) -> T {
        if (resident) return rl[b][t >> 6] + rc[b][t & 63];
        const int64_t g = F.block_start + b0 + b;
        return (T)(dl[g * 64 + (t >> 6)] + dc[g * 64 + (t & 63)]);
    };
    // One step: the cluster's least total sum_b min(cur_b, D_b(t)) over the
    // allowed presets t (lowest index on ties) into sm.step_t / sm.step_v,
    // identical in every CTA; with old >= 0 (re-optimisation of a slot
    // holding preset `old`) old is kept when its total attains the minimum.
    auto step = [&](int old) {
        unsigned long long a[kPer];
#pragma unroll
        for (int j = 0; j < kPer; j++) a[j] = 0;
        for (int s0 = 0; s0 < own; s0 += cap) {
            const int n = min(cap, own - s0);
            if (!resident) {
                stage(s0, n);
                __syncthreads();
            }
            sum_blocks<T>(rl, rc, cur + s0, n, c, lq, a);
            if (!resident) __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) sm.part[(lq + j) * 64 + c] = a[j];
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
            if (t == old) sm.slice_old = tot;
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

        // every CTA: the least of the slice minima (the same in all of them);
        // the slice values are rewritten only after the next step's first
        // cluster barrier
        if (tid == 0) {
            unsigned long long v = ULLONG_MAX;
            int t = INT_MAX;
            for (int r = 0; r < kCS; r++) {
                const ClusterSmem *o = cluster.map_shared_rank(&sm, r);
                if (better(o->slice_v, o->slice_t, v, t)) { v = o->slice_v; t = o->slice_t; }
            }
            if (old >= 0 && cluster.map_shared_rank(&sm, old / kSlice)->slice_old == v) t = old;
            sm.step_t = t;
            sm.step_v = v;
        }
        __syncthreads();
    };

    // ---- greedy: each step adds the preset of least total, then lowers
    // every block's best distortion
    for (int k = 0; k < 8; k++) {
        step(-1);
        const int best = sm.step_t;
        if (tid == 0) {
            sm.greedy[k] = best;
            sm.totals[k] = (long long)sm.step_v;
        }
        for (int b = tid; b < own; b += kCT) {
            const T d = dist(b, best);
            if (d < cur[b]) cur[b] = d;
        }
        __syncthreads();
    }
    if (tid < 4) {
        for (int j = 0; j < 8; j++) sm.refined[tid][j] = j < (1 << tid) ? sm.greedy[j] : 0;
        sm.ref_totals[tid] = sm.totals[(1 << tid) - 1];
    }
    __syncthreads();

    // ---- re-optimisation of the sets of size 2, 4, 8, one preset at a
    // time: slot k is re-chosen against every block's least distortion over
    // the other slots; passes end when one changes nothing (every CTA takes
    // the same decisions, so the cluster's barriers stay matched)
    for (int lg = 1; lg <= 3 && refine_passes > 0; lg++) {
        const int sz = 1 << lg;
        for (int pass = 0; pass < refine_passes; pass++) {
            bool changed = false;
            for (int k = 0; k < sz; k++) {
                for (int b = tid; b < own; b += kCT) {
                    T m = (T)~0ull;
                    for (int j = 0; j < sz; j++) {
                        if (j == k) continue;
                        const T d = dist(b, sm.refined[lg][j]);
                        m = d < m ? d : m;
                    }
                    cur[b] = m;
                }
                __syncthreads();
                const int old = sm.refined[lg][k];
                step(old);
                const int best = sm.step_t;
                changed = changed || best != old;
                __syncthreads();   // every thread has read the set before it changes
                if (tid == 0) {
                    sm.refined[lg][k] = best;
                    sm.ref_totals[lg] = (long long)sm.step_v;
                }
                __syncthreads();
            }
            if (!changed) break;
        }
    }

    // ---- N in {1, 2, 4, 8} by J (ties to the smaller N); block ids over the set
    int bl = 0;
    long long bj = 0;
    for (int lg = 0; lg < 4; lg++) {
        const long long j = sm.ref_totals[lg] + F.lambda * (long long)B * lg;
        if (lg == 0 || j < bj) { bl = lg; bj = j; }
    }
    const int N = 1 << bl;
    if (rank == 0 && tid == 0) {
        SearchResultDev &r = res[f];
        for (int j = 0; j < 8; j++) {
            // entries past N keep the greedy order
            r.presets[j] = j < N ? sm.refined[bl][j] : sm.greedy[j];
            r.greedy[j] = sm.greedy[j];
            r.totals[j] = sm.totals[j];
        }
        for (int lg = 0; lg < 4; lg++) {
            for (int j = 0; j < 8; j++) r.refined[lg][j] = sm.refined[lg][j];
            r.ref_totals[lg] = sm.ref_totals[lg];
        }
        r.cost = bj;
        r.npresets = N;
    }
    for (int b = tid; b < own; b += kCT) {
        const int64_t g = F.block_start + b0 + b;
        int id = 0;
        long long bestd = LLONG_MAX;
        for (int j = 0; j < N; j++) {
            const int t = sm.refined[bl][j];
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
                                   int refine_passes, cudaStream_t s)
{
    static_assert(kSlice <= kCT && kCT % 64 == 0 && kTuples % kCT == 0, "thread layout");
    constexpr size_t kSmem = sizeof(ClusterSmem);
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != configured_dev) {
        for (auto *k : {preset_cluster_kernel<unsigned>, preset_cluster_kernel<unsigned long long>}) {
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
    return narrow ? cudaLaunchKernelEx(&cfg, preset_cluster_kernel<unsigned>, b, dl, dc, results,
                                       block_ids, refine_passes)
                  : cudaLaunchKernelEx(&cfg, preset_cluster_kernel<unsigned long long>, b, dl, dc,
                                       results, block_ids, refine_passes);
}

}  // namespace cdefgb
