// Encoder strength search (section 5).
//
// dist_kernel: one CTA per 64x64 filter block of any frame of the batch.
//   The decoded tiles (plus the 2-pixel halo) are staged in shared memory,
//   the 64 luma directions found (section 2), and then every pixel is
//   filtered under all 64 (primary, secondary) strength pairs at once: the
//   constrained primary sum is formed once per primary strength (16) and the
//   secondary sum once per secondary strength (4), and the 64 pairs only
//   add, round, clip and accumulate (y - source)^2.  This factoring is
//   exact: eq. 8 is a sum of the two tap sets, each depending on one
//   strength only.  Each thread keeps 64 32-bit partial SSEs for the pixels
//   it owns; they are reduced into 64-bit block totals.
//
// greedy_kernel: one CTA per frame; the greedy preset search and the eq. 15
//   choice of N, with int64 totals.
#include <climits>

#include "cdef_device.cuh"
#include "cdef_internal.h"

namespace cdefgb {

namespace {

constexpr int kThreads = 256;
constexpr int kLumaRows = 64 + 4, kLumaPitch = 72;
constexpr int kChromaRows = 32 + 4, kChromaPitch = 40;
constexpr int kSentinel = 0x7fff;

struct SearchSmem {
    int16_t y[kLumaRows * kLumaPitch];
    int16_t u[kChromaRows * kChromaPitch];
    int16_t v[kChromaRows * kChromaPitch];
    uint8_t dir[64];
    int var[64];
    unsigned long long acc[64];
};

template <typename T>
__device__ __forceinline__ int load_sample(const uint8_t *plane, int64_t pitch, int y, int x)
{
    return (int)__ldg(reinterpret_cast<const T *>(plane + (int64_t)y * pitch) + x);
}

template <typename T>
__device__ void stage_tile(int16_t *tile, int pitch, int rows, int cols, const uint8_t *plane,
                           int64_t ppitch, int pw, int ph, int y0, int x0)
{
    for (int idx = threadIdx.x; idx < rows * cols; idx += kThreads) {
        const int r = idx / cols, c = idx - r * cols;
        const int y = y0 + r, x = x0 + c;
        int v = kSentinel;
        if (y >= 0 && y < ph && x >= 0 && x < pw) v = load_sample<T>(plane, ppitch, y, x);
        tile[r * pitch + c] = (int16_t)v;
    }
}

// The 12 tap values of the pixel at tile position (r, c): [0..3] primary
// (near +, near -, far +, far -), [4..11] secondary (d+2 then d-2, same
// order).  Out-of-frame taps read the sentinel.
__device__ __forceinline__ void gather_taps(const int16_t *tile, int pitch, int r, int c, int d,
                                            int p[12])
{
#pragma unroll
    for (int s = 0; s < 3; s++) {
        const int dd = s == 0 ? d : (d + (s == 1 ? 2 : 6)) & 7;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int dr = tap_dr(dd, k), dc = tap_dc(dd, k);
            p[s * 4 + k * 2 + 0] = tile[(r + dr) * pitch + c + dc];
            p[s * 4 + k * 2 + 1] = tile[(r - dr) * pitch + c - dc];
        }
    }
}

// Constrained, weighted primary sum for strength S / shift sh / weights.
__device__ __forceinline__ int pri_sum(const int p[12], int x, int S, int sh, int w0, int w1)
{
    int s = 0;
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const int f = p[t] == kSentinel ? 0 : constrain(p[t] - x, S, sh);
        s += (t < 2 ? w0 : w1) * f;
    }
    return s;
}

__device__ __forceinline__ int sec_sum(const int p[12], int x, int S, int sh)
{
    int s = 0;
#pragma unroll
    for (int t = 4; t < 12; t++) {
        const int f = p[t] == kSentinel ? 0 : constrain(p[t] - x, S, sh);
        s += (((t - 4) & 3) < 2 ? 2 : 1) * f;
    }
    return s;
}

// Accumulate the 64 strength pairs' squared errors of one pixel.
// chroma: the damping is D - 1 raised to floor(log2 S_p) (section 3.2),
// so the secondary shift may depend on the primary strength.
__device__ __forceinline__ void accumulate_pixel(const int16_t *tile, int pitch, int r, int c,
                                                 int d, int v, bool chroma, int damping,
                                                 int sh8, int src, unsigned acc[64])
{
    int p[12];
    gather_taps(tile, pitch, r, c, d, p);
    const int x = tile[r * pitch + c];
    int mn = x, mx = x;
#pragma unroll
    for (int t = 0; t < 12; t++) {
        if (p[t] != kSentinel) {
            mn = min(mn, p[t]);
            mx = max(mx, p[t]);
        }
    }
    const int Dp = chroma ? damping - 1 : damping;
    // secondary sums for the plane damping, and for the damping raised to 3
    // (only reachable when Dp < 3, i.e. chroma with D = 3)
    int Qa[4], Qb[4];
    const int svals[4] = {0, 1, 2, 4};
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const int S = svals[s];
        Qa[s] = S ? sec_sum(p, x, S << sh8, max(0, Dp - ilog2(S))) : 0;
        Qb[s] = S ? sec_sum(p, x, S << sh8, max(0, max(Dp, 3) - ilog2(S))) : 0;
    }
#pragma unroll
    for (int pi = 0; pi < 16; pi++) {
        const int Sp = chroma ? pi : adjust_strength(pi, v);
        const int lp = Sp ? ilog2(Sp) : 0;
        const int D = (Sp && Dp < lp) ? lp : Dp;
        const int P = Sp ? pri_sum(p, x, Sp << sh8, D - lp, (Sp & 1) ? 3 : 4, (Sp & 1) ? 3 : 2) : 0;
        const bool raised = D != Dp;
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int Q = raised ? Qb[s] : Qa[s];
            const int y = min(mx, max(mn, x + round16(P + Q)));
            const int e = y - src;
            acc[pi * 4 + s] += (unsigned)(e * e);
        }
    }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduce the 64 per-thread partial SSEs into sm.acc and write them out.
__device__ void reduce_store(unsigned acc[64], SearchSmem &sm, long long *out)
{
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 64) sm.acc[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 64; q++) {
        const unsigned long long s = warp_sum_u64(acc[q]);
        if (lane == 0) atomicAdd(&sm.acc[q], s);
    }
    __syncthreads();
    if (threadIdx.x < 64) out[threadIdx.x] = (long long)sm.acc[threadIdx.x];
    __syncthreads();
}

template <typename T>
__device__ void dist_block(const SearchFrameDev &F, int fby, int fbx, long long *dl,
                           long long *dc, SearchSmem &sm)
{
    const int sh8 = F.bitdepth - 8;
    const int ly0 = fby * 64, lx0 = fbx * 64, cy0 = fby * 32, cx0 = fbx * 32;
    const int cw = F.w >> 1, ch = F.h >> 1;
    stage_tile<T>(sm.y, kLumaPitch, kLumaRows, kLumaRows, F.rec[0], F.rec_pitch[0], F.w, F.h,
                  ly0 - 2, lx0 - 2);
    stage_tile<T>(sm.u, kChromaPitch, kChromaRows, kChromaRows, F.rec[1], F.rec_pitch[1], cw, ch,
                  cy0 - 2, cx0 - 2);
    stage_tile<T>(sm.v, kChromaPitch, kChromaRows, kChromaRows, F.rec[2], F.rec_pitch[2], cw, ch,
                  cy0 - 2, cx0 - 2);
    __syncthreads();
    if (threadIdx.x < 64) {
        const int by = threadIdx.x >> 3, bx = threadIdx.x & 7;
        int d = 0, v = 0;
        if (ly0 + by * 8 < F.h && lx0 + bx * 8 < F.w) {
            const int16_t *b = sm.y + (2 + by * 8) * kLumaPitch + 2 + bx * 8;
            d = find_dir_8x8([&](int i, int j) { return (int)b[i * kLumaPitch + j]; }, sh8, &v);
        }
        sm.dir[threadIdx.x] = (uint8_t)d;
        sm.var[threadIdx.x] = v;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned acc[64];
#pragma unroll
    for (int q = 0; q < 64; q++) acc[q] = 0;
    for (int k = warp; k < 64; k += kThreads / 32) {
        const int by = k >> 3, bx = k & 7;
        if (ly0 + by * 8 >= F.h || lx0 + bx * 8 >= F.w) continue;
        const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll 1
        for (int q = 0; q < 2; q++) {
            const int gy = ly0 + by * 8 + r, gx = lx0 + bx * 8 + c + q;
            const int src = load_sample<T>(F.src[0], F.src_pitch[0], gy, gx);
            accumulate_pixel(sm.y, kLumaPitch, 2 + by * 8 + r, 2 + bx * 8 + c + q, sm.dir[k],
                             sm.var[k], false, F.damping, sh8, src, acc);
        }
    }
    reduce_store(acc, sm, dl);

#pragma unroll
    for (int q = 0; q < 64; q++) acc[q] = 0;
    for (int k = warp; k < 64; k += kThreads / 32) {
        const int by = k >> 3, bx = k & 7;
        if (cy0 + by * 4 >= ch || cx0 + bx * 4 >= cw) continue;
        const int pl = lane >> 4, r = (lane & 15) >> 2, c = lane & 3;
        const int gy = cy0 + by * 4 + r, gx = cx0 + bx * 4 + c;
        const int src = load_sample<T>(F.src[1 + pl], F.src_pitch[1 + pl], gy, gx);
        accumulate_pixel(pl ? sm.v : sm.u, kChromaPitch, 2 + by * 4 + r, 2 + bx * 4 + c, sm.dir[k],
                         0, true, F.damping, sh8, src, acc);
    }
    reduce_store(acc, sm, dc);
}

__global__ void __launch_bounds__(kThreads)
dist_kernel(const __grid_constant__ SearchBatch batch, long long *dist_luma, long long *dist_chroma)
{
    __shared__ SearchSmem sm;
    const int blk = blockIdx.x;
    int fi = 0;
    while (fi + 1 < batch.n && blk >= batch.f[fi + 1].block_start) fi++;
    const SearchFrameDev &F = batch.f[fi];
    const int local = blk - F.block_start;
    const int fby = local / F.fb_cols, fbx = local - fby * F.fb_cols;
    long long *dl = dist_luma + (int64_t)blk * 64;
    long long *dc = dist_chroma + (int64_t)blk * 64;
    if (F.bitdepth == 8)
        dist_block<uint8_t>(F, fby, fbx, dl, dc, sm);
    else
        dist_block<uint16_t>(F, fby, fbx, dl, dc, sm);
}

// ---------------------------------------------------------------------------
// Greedy preset search, one CTA per frame (section 5, eq. 15).
constexpr int kGreedyThreads = 512;
constexpr int kTuplesPerThread = 4096 / kGreedyThreads;
constexpr int kChunk = 16;

__device__ __forceinline__ bool better(long long a, int ta, long long b, int tb)
{
    return a < b || (a == b && ta < tb);
}

__global__ void __launch_bounds__(kGreedyThreads)
greedy_kernel(const __grid_constant__ SearchBatch batch, const long long *__restrict__ dist_luma,
              const long long *__restrict__ dist_chroma, long long *cur, SearchResultDev *res,
              uint8_t *block_ids)
{
    __shared__ long long s_dl[kChunk][64], s_dc[kChunk][64], s_cur[kChunk];
    __shared__ long long s_best[kGreedyThreads / 32];
    __shared__ int s_bt[kGreedyThreads / 32];
    __shared__ int s_presets[8];
    __shared__ long long s_tot[8];

    const SearchFrameDev &F = batch.f[blockIdx.x];
    const int B = F.fb_cols * F.fb_rows;
    const long long *dl = dist_luma + (int64_t)F.block_start * 64;
    const long long *dc = dist_chroma + (int64_t)F.block_start * 64;
    long long *cb = cur + F.block_start;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int b = tid; b < B; b += kGreedyThreads) cb[b] = LLONG_MAX;
    __syncthreads();

    for (int n = 0; n < 8; n++) {
        long long tot[kTuplesPerThread];
#pragma unroll
        for (int k = 0; k < kTuplesPerThread; k++) tot[k] = 0;
        for (int c0 = 0; c0 < B; c0 += kChunk) {
            const int nb = min(kChunk, B - c0);
            for (int i = tid; i < nb * 64; i += kGreedyThreads) {
                s_dl[i >> 6][i & 63] = dl[(int64_t)(c0 + (i >> 6)) * 64 + (i & 63)];
                s_dc[i >> 6][i & 63] = dc[(int64_t)(c0 + (i >> 6)) * 64 + (i & 63)];
            }
            if (tid < nb) s_cur[tid] = cb[c0 + tid];
            __syncthreads();
            for (int bb = 0; bb < nb; bb++) {
                const long long cv = s_cur[bb];
                const long long cval = s_dc[bb][tid & 63];
#pragma unroll
                for (int k = 0; k < kTuplesPerThread; k++) {
                    const int l = (tid >> 6) + k * (kGreedyThreads >> 6);
                    tot[k] += min(cv, s_dl[bb][l] + cval);
                }
            }
            __syncthreads();
        }
        // arg-min over the 4096 tuples, lowest index on ties
        long long bv = tot[0];
        int bt = tid;
#pragma unroll
        for (int k = 1; k < kTuplesPerThread; k++) {
            const int t = tid + k * kGreedyThreads;
            if (better(tot[k], t, bv, bt)) { bv = tot[k]; bt = t; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (better(ov, ot, bv, bt)) { bv = ov; bt = ot; }
        }
        if (lane == 0) { s_best[warp] = bv; s_bt[warp] = bt; }
        __syncthreads();
        if (tid == 0) {
            long long v = s_best[0];
            int t = s_bt[0];
            for (int w = 1; w < kGreedyThreads / 32; w++)
                if (better(s_best[w], s_bt[w], v, t)) { v = s_best[w]; t = s_bt[w]; }
            s_presets[n] = t;
            s_tot[n] = v;
        }
        __syncthreads();
        const int t = s_presets[n];
        for (int b = tid; b < B; b += kGreedyThreads)
            cb[b] = min(cb[b], dl[(int64_t)b * 64 + (t >> 6)] + dc[(int64_t)b * 64 + (t & 63)]);
        __syncthreads();
    }

    __shared__ int s_n;
    if (tid == 0) {
        int bn = 0;
        long long bj = 0;
        for (int lg = 0; lg < 4; lg++) {
            const int n = 1 << lg;
            const long long j = s_tot[n - 1] + F.lambda * (long long)B * lg;
            if (bn == 0 || j < bj) { bn = n; bj = j; }
        }
        SearchResultDev &r = res[blockIdx.x];
        for (int k = 0; k < 8; k++) { r.presets[k] = s_presets[k]; r.totals[k] = s_tot[k]; }
        r.cost = bj;
        r.npresets = bn;
        s_n = bn;
    }
    __syncthreads();
    const int N = s_n;
    for (int b = tid; b < B; b += kGreedyThreads) {
        int id = 0;
        long long best = dl[(int64_t)b * 64 + (s_presets[0] >> 6)] + dc[(int64_t)b * 64 + (s_presets[0] & 63)];
        for (int k = 1; k < N; k++) {
            const long long v = dl[(int64_t)b * 64 + (s_presets[k] >> 6)] +
                                dc[(int64_t)b * 64 + (s_presets[k] & 63)];
            if (v < best) { best = v; id = k; }
        }
        block_ids[F.block_start + b] = (uint8_t)id;
    }
}

}  // namespace

cudaError_t launch_search(const SearchBatch &b, long long *dist_luma, long long *dist_chroma,
                          long long *cur, SearchResultDev *results, uint8_t *block_ids,
                          int *status, cudaStream_t s)
{
    (void)status;
    dist_kernel<<<b.total_blocks, kThreads, 0, s>>>(b, dist_luma, dist_chroma);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    greedy_kernel<<<b.n, kGreedyThreads, 0, s>>>(b, dist_luma, dist_chroma, cur, results, block_ids);
    return cudaGetLastError();
}

}  // namespace cdefgb
