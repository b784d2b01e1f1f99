// The CDEF filter (section 3, eq. 6-13) fused with the direction search
// (section 2): one CTA per 64x64 filter block (section 4).
//
// 1. The 64x64 luma tile and the two 32x32 chroma tiles, each with the
//    2-pixel halo the taps reach (max tap offset 2), are staged in shared
//    memory as int16.  Pixels outside the frame hold a sentinel; a tap on
//    the sentinel is ignored (section 3.1).
// 2. 64 threads run Algorithm 1 on the 64 luma 8x8 blocks of the tile (or
//    read caller-supplied maps).
// 3. Each warp filters whole 8x8 luma blocks (direction, strengths and
//    damping are uniform over an 8x8 block, section 3.1), two pixels per
//    lane, then pairs of co-located U/V 4x4 chroma blocks.
#include "cdef_device.cuh"
#include "cdef_internal.h"

namespace cdefgb {

namespace {

constexpr int kThreads = 256;
constexpr int kLumaRows = 64 + 4, kLumaPitch = 72;
constexpr int kChromaRows = 32 + 4, kChromaPitch = 40;
constexpr int kSentinel = 0x7fff;

template <typename T>
__device__ __forceinline__ int load_sample(const uint8_t *plane, int64_t pitch, int y, int x)
{
    return (int)__ldg(reinterpret_cast<const T *>(plane + (int64_t)y * pitch) + x);
}

template <typename T>
__device__ __forceinline__ void store_sample(uint8_t *plane, int64_t pitch, int y, int x, int v)
{
    reinterpret_cast<T *>(plane + (int64_t)y * pitch)[x] = (T)v;
}

// Stage a (rows x cols) window whose top-left is (y0, x0) in plane
// coordinates; out-of-frame pixels get the sentinel.
template <typename T>
__device__ void stage_tile(int16_t *tile, int pitch, int rows, int cols,
                           const PlaneDev &P, int y0, int x0)
{
    for (int idx = threadIdx.x; idx < rows * cols; idx += kThreads) {
        const int r = idx / cols, c = idx - r * cols;
        const int y = y0 + r, x = x0 + c;
        int v = kSentinel;
        if (y >= 0 && y < P.h && x >= 0 && x < P.w) v = load_sample<T>(P.in, P.in_pitch, y, x);
        tile[r * pitch + c] = (int16_t)v;
    }
}

// Eq. 8-12 for the pixel at tile position (r, c).
__device__ __forceinline__ int filter_px(const int16_t *tile, int pitch, int r, int c,
                                         int d, const Eff &e)
{
    const int x = tile[r * pitch + c];
    int sum = 0, mn = x, mx = x;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int dr = tap_dr(d, k), dc = tap_dc(d, k);
        const int w = k ? e.w1 : e.w0;
#pragma unroll
        for (int sg = -1; sg <= 1; sg += 2) {
            const int p = tile[(r + sg * dr) * pitch + c + sg * dc];
            if (p != kSentinel) {
                sum += w * constrain(p - x, e.pri, e.psh);
                mn = min(mn, p);
                mx = max(mx, p);
            }
        }
    }
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const int dd = (d + (side ? 6 : 2)) & 7;
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int dr = tap_dr(dd, k), dc = tap_dc(dd, k);
            const int w = k ? 1 : 2;
#pragma unroll
            for (int sg = -1; sg <= 1; sg += 2) {
                const int p = tile[(r + sg * dr) * pitch + c + sg * dc];
                if (p != kSentinel) {
                    sum += w * constrain(p - x, e.sec, e.ssh);
                    mn = min(mn, p);
                    mx = max(mx, p);
                }
            }
        }
    }
    return min(mx, max(mn, x + round16(sum)));
}

__device__ __forceinline__ bool valid_strengths(int pri, int sec)
{
    return (pri <= 15 || pri == 19) && (sec == 0 || sec == 1 || sec == 2 || sec == 4 || sec == 7);
}

struct FilterSmem {
    int16_t y[kLumaRows * kLumaPitch];
    int16_t u[kChromaRows * kChromaPitch];
    int16_t v[kChromaRows * kChromaPitch];
    uint8_t dir[64];
    int var[64];
};

template <typename T>
__device__ void filter_block(const FilterFrameDev &F, int fby, int fbx, int *status,
                             FilterSmem &sm)
{
    int16_t *sy = sm.y, *su = sm.u, *sv = sm.v;
    uint8_t *sdir = sm.dir;
    int *svar = sm.var;

    const int sh8 = F.bitdepth - 8;
    const int ly0 = fby * 64, lx0 = fbx * 64;
    const int cy0 = fby * 32, cx0 = fbx * 32;
    stage_tile<T>(sy, kLumaPitch, kLumaRows, kLumaRows, F.p[0], ly0 - 2, lx0 - 2);
    stage_tile<T>(su, kChromaPitch, kChromaRows, kChromaRows, F.p[1], cy0 - 2, cx0 - 2);
    stage_tile<T>(sv, kChromaPitch, kChromaRows, kChromaRows, F.p[2], cy0 - 2, cx0 - 2);

    cdef_fb_params prm = F.params[fby * F.fb_cols + fbx];
    if (!valid_strengths(prm.pri_y, prm.sec_y) || !valid_strengths(prm.pri_uv, prm.sec_uv) ||
        prm.damping < 3 || prm.damping > 6) {
        if (threadIdx.x == 0) atomicOr(status, kStatusBadParams);
        prm.pri_y = prm.sec_y = prm.pri_uv = prm.sec_uv = 0;  // identity, defined output
        prm.damping = 3;
    }
    __syncthreads();

    const int bw = F.p[0].w >> 3;
    if (threadIdx.x < 64) {
        const int by = threadIdx.x >> 3, bx = threadIdx.x & 7;
        const int gby = fby * 8 + by, gbx = fbx * 8 + bx;
        int d = 0, v = 0;
        if (gby * 8 < F.p[0].h && gbx * 8 < F.p[0].w) {
            if (F.dir) {
                d = F.dir[gby * bw + gbx];
                v = F.var[gby * bw + gbx];
            } else {
                const int16_t *b = sy + (2 + by * 8) * kLumaPitch + 2 + bx * 8;
                d = find_dir_8x8([&](int i, int j) { return (int)b[i * kLumaPitch + j]; }, sh8, &v);
            }
        }
        sdir[threadIdx.x] = (uint8_t)d;
        svar[threadIdx.x] = v;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Luma: warp-uniform 8x8 blocks, two pixels per lane.
    for (int k = warp; k < 64; k += kThreads / 32) {
        const int by = k >> 3, bx = k & 7;
        if (ly0 + by * 8 >= F.p[0].h || lx0 + bx * 8 >= F.p[0].w) continue;
        const Eff e = make_eff(prm.pri_y, prm.sec_y, prm.damping, false, svar[k], sh8);
        const int d = sdir[k];
        const int r = lane >> 2, c = (lane & 3) * 2;
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int y = filter_px(sy, kLumaPitch, 2 + by * 8 + r, 2 + bx * 8 + c + q, d, e);
            store_sample<T>(F.p[0].out, F.p[0].out_pitch, ly0 + by * 8 + r, lx0 + bx * 8 + c + q, y);
        }
    }
    // Chroma: co-located U and V 4x4 blocks share direction and strengths.
    for (int k = warp; k < 64; k += kThreads / 32) {
        const int by = k >> 3, bx = k & 7;
        if (cy0 + by * 4 >= F.p[1].h || cx0 + bx * 4 >= F.p[1].w) continue;
        const Eff e = make_eff(prm.pri_uv, prm.sec_uv, prm.damping, true, 0, sh8);
        const int d = sdir[k];
        const int pl = lane >> 4, r = (lane & 15) >> 2, c = lane & 3;
        const int16_t *tile = pl ? sv : su;
        const int y = filter_px(tile, kChromaPitch, 2 + by * 4 + r, 2 + bx * 4 + c, d, e);
        const PlaneDev &P = F.p[1 + pl];
        store_sample<T>(P.out, P.out_pitch, cy0 + by * 4 + r, cx0 + bx * 4 + c, y);
    }
}

template <int MAXF>
__global__ void __launch_bounds__(kThreads)
filter_kernel(const __grid_constant__ FilterBatch<MAXF> batch, int *status)
{
    const int blk = blockIdx.x;
    int fi = 0;
    if (MAXF > 1)
        while (fi + 1 < batch.n && blk >= batch.f[fi + 1].block_start) fi++;
    __shared__ FilterSmem sm;
    const FilterFrameDev &F = batch.f[fi];
    const int local = blk - F.block_start;
    const int fby = local / F.fb_cols, fbx = local - fby * F.fb_cols;
    if (F.bitdepth == 8)
        filter_block<uint8_t>(F, fby, fbx, status, sm);
    else
        filter_block<uint16_t>(F, fby, fbx, status, sm);
}

}  // namespace

cudaError_t launch_filter_single(const FilterBatch<1> &b, int *status, cudaStream_t s)
{
    filter_kernel<1><<<b.total_blocks, kThreads, 0, s>>>(b, status);
    return cudaGetLastError();
}

cudaError_t launch_filter_batch(const FilterBatch<kMaxBatch> &b, int *status, cudaStream_t s)
{
    filter_kernel<kMaxBatch><<<b.total_blocks, kThreads, 0, s>>>(b, status);
    return cudaGetLastError();
}

}  // namespace cdefgb
