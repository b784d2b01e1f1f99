// The preset selection of section 5 (eq. 15) with one thread-block
// cluster per frame: no grid-wide barrier.  The eight CTAs of a cluster
// split the frame's filter blocks; in a greedy step each computes, for all
// W x W (luma combination, chroma combination) presets t (W = 64, or 128
// with the skip-condition bit), its blocks' sum_b min(best_b, D_b(t)) into
// its own shared memory; after a cluster barrier CTA r adds the eight
// partial sums of its eighth of the presets through distributed shared
// memory and finds their least total (lowest index on ties); after a
// second barrier every CTA takes the least of the eight slice minima, so
// all of them agree on the step's preset and lower their blocks' best
// distortion.  The re-optimisation passes (section 5) re-choose one slot
// of a set at a time with the same step, each block's best distortion
// being its least over the set's other slots.  Then N in {1, 2, 4, 8} by J
// and each block's preset id, as in presets.cu.  Filter blocks flagged
// skipped (section 4, 128-combination search) add nothing to any total,
// do not count in J's B and take id 0.
#include <climits>
#include <cooperative_groups.h>

#include "cdef_internal.h"

namespace cg = cooperative_groups;

namespace cdefgb {
namespace {

constexpr int kCS = 8;                   // CTAs per cluster (per frame)
constexpr int kCT = 512;                 // threads per CTA
constexpr int kPer = 8;                  // presets per thread and group
constexpr int kMaxOwn = 2048;            // blocks one CTA can hold (frames up to 16384 blocks)

// Per combination count W: W x W presets, in groups of kCT x kPer per
// thread pass; each CTA reduces an eighth of them; shared memory left for
// the table rows.
template <int kW>
struct Geo {
    static constexpr int kTuples = kW * kW;
    static constexpr int kGroups = kTuples / (kCT * kPer);
    static constexpr int kSlice = kTuples / kCS;
    static constexpr int kTabBytes = kW == 64 ? 128 * 1024 : 64 * 1024;
    static_assert(kTuples % (kCT * kPer) == 0 && kSlice % kCT == 0 && kCT % kW == 0, "layout");
};

template <int kW>
struct ClusterSmem {
    unsigned long long part[kW * kW];            // this CTA's partial totals
    unsigned long long cur[kMaxOwn];             // best distortion of the CTA's blocks
    alignas(16) unsigned char tab[Geo<kW>::kTabBytes];   // table rows: luma [cap][W], chroma [cap][W]
    unsigned long long red_v[kCT / 32];
    int red_t[kCT / 32];
    unsigned long long slice_v;                  // this CTA's slice minimum
    int slice_t;
    unsigned long long slice_old;                // total of the step's current preset (its slice's CTA)
    int step_t;                                  // the step's chosen preset
    unsigned long long step_v;                   // and its total
    int coded;                                   // blocks of the frame that signal a preset id
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
template <typename T, int kW>
__device__ __forceinline__ void sum_blocks(const T (*rl)[kW], const T (*rc)[kW], const T *cur,
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
// the call is an 8-bit squared error (below 2^30).  kW: combinations per
// plane group (64, or 128 with the skip-condition bit); `skipped` (W = 128
// only, may be null): one flag per filter block.
template <typename T, int kW>
__global__ void __launch_bounds__(kCT, 1)
preset_cluster_kernel(const __grid_constant__ SearchBatch batch, const long long *__restrict__ dl,
                      const long long *__restrict__ dc, SearchResultDev *res, uint8_t *block_ids,
                      const uint8_t *skipped, int refine_passes)
{
    using G = Geo<kW>;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    ClusterSmem<kW> &sm = *reinterpret_cast<ClusterSmem<kW> *>(smem_raw);
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
    constexpr int cap = G::kTabBytes / (2 * kW * (int)sizeof(T));
    T (*rl)[kW] = reinterpret_cast<T (*)[kW]>(sm.tab);
    T (*rc)[kW] = rl + cap;
    T *cur = reinterpret_cast<T *>(sm.cur);
    const bool resident = own <= cap;
    auto stage = [&](int s0, int n) {
        for (int i = tid; i < n * kW; i += kCT) {
            const int bb = i / kW, q = i % kW;
            const int64_t g = (int64_t)(F.block_start + b0 + s0 + bb) * kW + q;
            rl[bb][q] = (T)dl[g];
            rc[bb][q] = (T)dc[g];
        }
    };
    auto skip = [&](int b) { return skipped && skipped[F.block_start + b0 + b]; };

    // a skipped block's best distortion stays 0: it adds nothing to a total
    for (int b = tid; b < own; b += kCT) cur[b] = skip(b) ? (T)0 : (T)~0ull;
    if (tid == 0) sm.coded = 0;
    if (resident) stage(0, own);
    __syncthreads();
    if (skipped) {
        int n = 0;
        for (int b = tid; b < B; b += kCT) n += skipped[F.block_start + b] == 0;
        atomicAdd(&sm.coded, n);
    } else if (tid == 0) {
        sm.coded = B;
    }

    // D_b(t) of the CTA's block b
    auto dist = [&](int b, int t) -> T {
        if (resident) return rl[b][t / kW] + rc[b][t % kW];
        const int64_t g = F.block_start + b0 + b;
        return (T)(dl[g * kW + t / kW] + dc[g * kW + t % kW]);
    };
    // One step: the cluster's least total sum_b min(cur_b, D_b(t)) over the
    // allowed presets t (lowest index on ties) into sm.step_t / sm.step_v,
    // identical in every CTA; with old >= 0 (re-optimisation of a slot
    // holding preset `old`) old is kept when its total attains the minimum.
    auto step = [&](int old) {
        // thread tid, group g: chroma combination c, luma combinations lq .. lq + 7
        const int c = tid % kW;
#pragma unroll 1
        for (int g = 0; g < G::kGroups; g++) {
            const int lq = (tid / kW) * kPer + g * (kCT * kPer / kW);
            unsigned long long a[kPer];
#pragma unroll
            for (int j = 0; j < kPer; j++) a[j] = 0;
            for (int s0 = 0; s0 < own; s0 += cap) {
                const int n = min(cap, own - s0);
                if (!resident) {
                    stage(s0, n);
                    __syncthreads();
                }
                sum_blocks<T, kW>(rl, rc, cur + s0, n, c, lq, a);
                if (!resident) __syncthreads();
            }
#pragma unroll
            for (int j = 0; j < kPer; j++) sm.part[(lq + j) * kW + c] = a[j];
        }
        cluster.sync();

        // this CTA's slice: the eight partial sums, then its least total
        unsigned long long bv = ULLONG_MAX;
        int bt = INT_MAX;
#pragma unroll 1
        for (int i = 0; i < G::kSlice / kCT; i++) {
            const int t = rank * G::kSlice + i * kCT + tid;
            unsigned long long tot = 0;
#pragma unroll
            for (int r = 0; r < kCS; r++) tot += cluster.map_shared_rank(sm.part, r)[t];
            // pairs: the combination without its skip-condition bit
            if ((full || ((lp >> ((t / kW) & 63)) & (cp >> (t & 63)) & 1)) && better(tot, t, bv, bt)) {
                bv = tot;
                bt = t;
            }
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
                const ClusterSmem<kW> *o = cluster.map_shared_rank(&sm, r);
                if (better(o->slice_v, o->slice_t, v, t)) { v = o->slice_v; t = o->slice_t; }
            }
            if (old >= 0 && cluster.map_shared_rank(&sm, old / G::kSlice)->slice_old == v) t = old;
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
            if (d < cur[b]) cur[b] = d;   // never for a skipped block (0)
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
                    T m = skip(b) ? (T)0 : (T)~0ull;
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
        const long long j = sm.ref_totals[lg] + F.lambda * (long long)sm.coded * lg;
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
        if (!skip(b)) {
            long long bestd = LLONG_MAX;
            for (int j = 0; j < N; j++) {
                const int t = sm.refined[bl][j];
                const long long v = dl[g * kW + t / kW] + dc[g * kW + t % kW];
                if (v < bestd) { bestd = v; id = j; }
            }
        }
        block_ids[g] = (uint8_t)id;
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
}

template <typename T, int kW>
cudaError_t launch_one(const SearchBatch &b, const long long *dl, const long long *dc,
                       SearchResultDev *results, uint8_t *block_ids, const uint8_t *skipped,
                       int refine_passes, cudaStream_t s)
{
    constexpr size_t kSmem = sizeof(ClusterSmem<kW>);
    static_assert(kSmem <= 227 * 1024, "shared memory of one CTA");
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != configured_dev) {
        cudaError_t e = cudaFuncSetAttribute(preset_cluster_kernel<T, kW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess && kCS > 8)
            e = cudaFuncSetAttribute(preset_cluster_kernel<T, kW>,
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
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
    return cudaLaunchKernelEx(&cfg, preset_cluster_kernel<T, kW>, b, dl, dc, results, block_ids,
                              skipped, refine_passes);
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
                                   int refine_passes, int width, const uint8_t *skipped,
                                   cudaStream_t s)
{
    if (width == 128)
        return narrow ? launch_one<unsigned, 128>(b, dl, dc, results, block_ids, skipped,
                                                  refine_passes, s)
                      : launch_one<unsigned long long, 128>(b, dl, dc, results, block_ids, skipped,
                                                            refine_passes, s);
    return narrow ? launch_one<unsigned, 64>(b, dl, dc, results, block_ids, nullptr, refine_passes, s)
                  : launch_one<unsigned long long, 64>(b, dl, dc, results, block_ids, nullptr,
                                                       refine_passes, s);
}

}  // namespace cdefgb
