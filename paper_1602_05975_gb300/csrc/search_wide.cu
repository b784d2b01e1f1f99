// Strength-search tables (section 5) for the frames the packed distortion
// kernel does not take: 4:2:2 frames (chroma not filtered, section 4 last
// paragraph), 4:4:4 frames (each chroma plane filtered in 8x8 blocks of the
// 64x64 filter block with the chroma strengths and the co-located luma
// direction) and 12-bit frames (whose sums leave 16-bit lanes).
//
// One CTA per (filter block, plane group).  The plane tiles of the block
// with their 2-sample halo are staged in shared memory as 32-bit samples
// (-1 outside the frame: such a tap adds nothing and is not in the clip
// range).  Four threads share an 8x8 (4:2:0 chroma: 4x4) block, so the
// direction and the strengths of a candidate are per thread.  Per sample the
// 64 (S_p, S_s) candidates come from 16 primary and 3 secondary constrained
// sums (eq. 8's sum splits into the two tap sets; chroma blocks whose damping
// is raised for S_p >= 8 take a second set of secondary sums), each rounded,
// clipped (eq. 9-12) and its squared error summed across the CTA.  The
// direction maps come from the direction-search kernel, launched first.
#include <type_traits>
#include "tile.cuh"

namespace cdefgb {
namespace {

using tile::tap_rc;

constexpr int kWThreads = 256;
constexpr int kTile = 69;   // 64 + 2 x 2 halo, plus one: an odd pitch spreads the rows over the banks

struct WideSmem {
    int tile[2][kTile * kTile];   // the group's planes (luma: one; chroma: U and V)
    unsigned long long acc[64];
};

// The group's plane k of frame F: pointers, size, and its geometry within
// the filter block.
struct PlaneView {
    const uint8_t *rec, *src;
    int64_t rec_pitch, src_pitch;
    int w, h;         // plane size
    int fw, fh;       // filter-block extent in this plane
    int bs;           // block size of one direction (8, or 4 for 4:2:0 chroma)
};

__device__ __forceinline__ PlaneView plane_view(const SearchFrameDev &F, int k)
{
    PlaneView v;
    v.rec = F.rec[k];
    v.src = F.src[k];
    v.rec_pitch = F.rec_pitch[k];
    v.src_pitch = F.src_pitch[k];
    if (k == 0 || F.chroma_format == 444) {
        v.w = F.w;
        v.h = F.h;
        v.fw = v.fh = 64;
        v.bs = 8;
    } else if (F.chroma_format == 422) {
        v.w = F.w >> 1;
        v.h = F.h;
        v.fw = 32;
        v.fh = 64;
        v.bs = 8;   // not filtered
    } else {
        v.w = F.w >> 1;
        v.h = F.h >> 1;
        v.fw = v.fh = 32;
        v.bs = 4;
    }
    return v;
}

__device__ __forceinline__ int sample_at(const uint8_t *row, int x, bool wide)
{
    return wide ? (int)reinterpret_cast<const uint16_t *>(row)[x] : (int)row[x];
}

// Per direction block and primary strength p: the scaled adjusted strength,
// the primary shift, whether the weights are 3/3 (odd strength), and
// whether the block's damping was raised to floor(log2 S_p) (section 3.2).
__device__ __forceinline__ int pack_primary(int pri, int psh, bool odd, bool raised)
{
    return pri | (psh << 12) | ((int)odd << 20) | ((int)raised << 21);
}

// kCoded: the 128-combination tables of section 5 with section 4's skip
// semantics: per candidate the error over every sample and over the samples
// of 8x8 blocks without coded residual (the threads of such a block), the
// unfiltered error likewise, and the (19, 7) preset's error; the entries
// with the skip bit clear leave the uncoded blocks unfiltered.
template <bool kCoded>
__global__ void __launch_bounds__(kWThreads, 2)
dist_wide_kernel(const __grid_constant__ SearchBatch batch, const uint8_t *__restrict__ dirs,
                 const int32_t *__restrict__ vars, long long *dist_luma, long long *dist_chroma,
                 uint8_t *skipped)
{
    __shared__ WideSmem sm;
    __shared__ unsigned long long acc_unc[64], base_sums[4];   // uncoded part; unfiltered, (19, 7)
    __shared__ int prim[64][16];
    // one copy of the body per plane group (0 luma, 1 chroma), the group's
    // plane count and strength rules fixed in each
    auto body = [&](auto group_c) {
    constexpr int group = decltype(group_c)::value;
    const int tid = threadIdx.x, lane = tid & 31;
    const int blk = blockIdx.x;
    int fi = 0;
    while (fi + 1 < batch.n && blk >= batch.f[fi + 1].block_start) fi++;
    const SearchFrameDev &F = batch.f[fi];
    const int local = blk - F.block_start;
    const int brow = local / F.fb_cols, fbx = local - brow * F.fb_cols;
    const int fby = brow + F.fb_row0;   // the frame's filter-block row
    const bool wide = F.bitdepth > 8;
    const int sh8 = F.bitdepth - 8;
    const bool filtered = group == 0 || F.chroma_format != 422;
    constexpr int nplanes = group == 0 ? 1 : 2;
    constexpr bool chroma = group != 0;
    const int bw = F.w >> 3;
    const int Dbase = chroma ? F.damping - 1 : F.damping;

    // stage the planes (rec) of the group with the halo
    for (int k = 0; k < nplanes; k++) {
        const PlaneView v = plane_view(F, group == 0 ? 0 : 1 + k);
        const int y0 = fby * v.fh - 2, x0 = fbx * v.fw - 2;
        for (int i = tid; i < (v.fh + 4) * (v.fw + 4); i += kWThreads) {
            const int r = i / (v.fw + 4), c = i - r * (v.fw + 4);
            const int gy = y0 + r, gx = x0 + c;
            sm.tile[k][r * kTile + c] = (gy >= 0 && gy < v.h && gx >= 0 && gx < v.w)
                                            ? sample_at(v.rec + gy * v.rec_pitch, gx, wide)
                                            : -1;
        }
    }
    // primary-strength constants per direction block (luma: after eq. 13)
    for (int i = tid; i < 64 * 16; i += kWThreads) {
        const int b = i >> 4, p = i & 15;
        const int gby = fby * 8 + (b >> 3), gbx = fbx * 8 + (b & 7);
        const int v = (gby * 8 < F.h && gbx * 8 < F.w) ? vars[F.map_start + gby * bw + gbx] : 0;
        const int pri = chroma ? p : adjust_strength(p, v);
        const int lp = pri ? ilog2(pri) : 0;
        const bool raised = pri && Dbase < lp;
        const int D = raised ? lp : Dbase;
        prim[b][p] = pack_primary(pri << sh8, pri ? D - lp : 0, pri & 1, raised);
    }
    if (tid < 64) {
        sm.acc[tid] = 0;
        acc_unc[tid] = 0;
    }
    if (tid < 4) base_sums[tid] = 0;
    __syncthreads();

    // four threads per direction block: 8x8 blocks (two rows each) or 4x4
    // blocks of 4:2:0 chroma (one row each)
    const int b8 = tid >> 2, part = tid & 3;
    const int by = b8 >> 3, bx = b8 & 7;
    const int gby = fby * 8 + by, gbx = fbx * 8 + bx;   // co-located luma 8x8 block
    const bool in_luma = gby * 8 < F.h && gbx * 8 < F.w;
    const int d = in_luma ? dirs[F.map_start + gby * bw + gbx] : 0;
    int o[12];
    for (int k = 0; k < 12; k++) {
        int dr, dc;
        tap_rc(d, k, dr, dc);
        o[k] = dr * kTile + dc;
    }
    // section 4: the coded-residual flag of the thread's (co-located luma)
    // 8x8 block, and whether the filter block has any
    const int cflag = kCoded ? (in_luma && F.coded[gby * bw + gbx] != 0) : 1;
    const bool any_coded = kCoded ? __syncthreads_or(cflag) != 0 : true;
    if (kCoded && group == 0 && tid == 0) skipped[blk] = (uint8_t)!any_coded;
    // the (19, 7) preset of the block (section 4), for the skip-bit-set (0, 0)
    // entry
    const Eff e19 = make_eff(19, 7, F.damping, chroma,
                             chroma ? 0 : (in_luma ? vars[F.map_start + gby * bw + gbx] : 0), sh8);
    const unsigned long long pairs = allowed_pairs(F, group);
    uint32_t pmask = 0;   // primaries with an allowed pair
    for (int p = 0; p < 16; p++) pmask |= (uint32_t)(((pairs >> (4 * p)) & 15ull) != 0) << p;
    // secondary shifts at the block's damping and at the raised one (3)
    const int Dhi = Dbase < 3 ? 3 : Dbase;

    // per candidate (p, s) the thread's squared error (at most 32 samples of
    // 12 bits: below 2^31)
    int acc[64], acc19 = 0, accu = 0;   // accu: the unfiltered error
#pragma unroll
    for (int q = 0; q < 64; q++) acc[q] = 0;
    for (int k = 0; k < nplanes; k++) {
        const PlaneView v = plane_view(F, group == 0 ? 0 : 1 + k);
        const int rows = v.bs == 8 ? 2 : 1, cols = v.bs;
        const int r0 = by * v.bs + part * rows, c0 = bx * v.bs;
        for (int i = 0; i < rows; i++) {
            const int gy = fby * v.fh + r0 + i;
            if (r0 + i >= v.fh || gy >= v.h) break;
            const uint8_t *srow = v.src + gy * v.src_pitch;
            for (int j = 0; j < cols; j++) {
                const int gx = fbx * v.fw + c0 + j;
                if (c0 + j >= v.fw || gx >= v.w) break;
                const int *t = &sm.tile[k][(r0 + i + 2) * kTile + c0 + j + 2];
                const int x = t[0], src = sample_at(srow, gx, wide);
                const int eu = x - src;
                accu += eu * eu;
                if (!filtered) {
#pragma unroll
                    for (int q = 0; q < 64; q++) acc[q] += eu * eu;
                    acc19 += eu * eu;
                    continue;
                }
                int pv[12], mn = x, mx = x;
#pragma unroll
                for (int m = 0; m < 12; m++) {
                    const int pm = t[o[m]];
                    pv[m] = pm < 0 ? x : pm;   // outside the frame: adds nothing
                    mn = min(mn, pv[m]);
                    mx = max(mx, pv[m]);
                }
                // secondary sums for S_s = 1, 2, 4 at both dampings (eq. 8's
                // sum splits into the two tap sets)
                int qlo[4] = {0, 0, 0, 0}, qhi[4] = {0, 0, 0, 0};
#pragma unroll
                for (int si = 1; si < 4; si++) {
                    const int ss = si == 3 ? 4 : si, S = ss << sh8, l2 = ss == 4 ? 2 : ss - 1;
                    const int shl = max(0, Dbase - l2), shh = max(0, Dhi - l2);
#pragma unroll
                    for (int m = 4; m < 12; m++) {
                        const int w = m < 8 ? 2 : 1;
                        qlo[si] += w * constrain(pv[m] - x, S, shl);
                        qhi[si] += w * constrain(pv[m] - x, S, shh);
                    }
                }
                if (kCoded) {   // the (19, 7) preset
                    int P = 0, Q = 0;
#pragma unroll
                    for (int m = 0; m < 4; m++)
                        P += (m < 2 ? e19.w0 : e19.w1) * constrain(pv[m] - x, e19.pri, e19.psh);
#pragma unroll
                    for (int m = 4; m < 12; m++)
                        Q += (m < 8 ? 2 : 1) * constrain(pv[m] - x, e19.sec, e19.ssh);
                    const int e = min(mx, max(mn, x + round16(P + Q))) - src;
                    acc19 += e * e;
                }
#pragma unroll
                for (int p = 0; p < 16; p++) {
                    if (!((pmask >> p) & 1)) continue;
                    const int pc = prim[b8][p];
                    const int S = pc & 0xfff, sh = (pc >> 12) & 0xff;
                    const int w0 = (pc >> 20) & 1 ? 3 : 4, w1 = 6 - w0;
                    const bool raised = (pc >> 21) & 1;
                    const int P = w0 * (constrain(pv[0] - x, S, sh) + constrain(pv[1] - x, S, sh)) +
                                  w1 * (constrain(pv[2] - x, S, sh) + constrain(pv[3] - x, S, sh));
#pragma unroll
                    for (int si = 0; si < 4; si++) {
                        const int y = min(mx, max(mn, x + round16(P + (raised ? qhi[si] : qlo[si]))));
                        const int e = y - src;
                        acc[p * 4 + si] += e * e;
                    }
                }
            }
        }
    }
    // CTA sums: warp shuffles, then one shared atomic per warp and candidate
    // (with the skip semantics also the uncoded blocks' part)
#pragma unroll
    for (int q = 0; q < 64; q++) {
        long long sum = acc[q], unc = kCoded && !cflag ? acc[q] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, off);
            if (kCoded) unc += __shfl_xor_sync(0xffffffffu, unc, off);
        }
        if (lane == 0) {
            atomicAdd(&sm.acc[q], (unsigned long long)sum);
            if (kCoded) atomicAdd(&acc_unc[q], (unsigned long long)unc);
        }
    }
    if (kCoded) {
        long long v[3] = {accu, cflag ? 0 : accu, acc19};
#pragma unroll
        for (int j = 0; j < 3; j++) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
            if (lane == 0) atomicAdd(&base_sums[j], (unsigned long long)v[j]);
        }
    }
    __syncthreads();
    if (!kCoded) {
        if (tid < 64) {
            long long *out = (group == 0 ? dist_luma : dist_chroma) + (int64_t)blk * 64;
            out[tid] = ((pairs >> tid) & 1) ? (long long)sm.acc[tid] : 0;
        }
    } else if (tid < 128) {
        // q = k * 64 + p * 4 + s
        const int q = tid & 63, k = tid >> 6;
        const long long base = (long long)base_sums[0], base_unc = (long long)base_sums[1];
        long long v;
        if (!any_coded) v = base;                                   // never filtered
        else if (k) v = q == 0 ? (long long)base_sums[2] : (long long)sm.acc[q];
        else v = q == 0 ? base : (long long)sm.acc[q] - (long long)acc_unc[q] + base_unc;
        long long *out = (group == 0 ? dist_luma : dist_chroma) + (int64_t)blk * 128;
        out[tid] = ((pairs >> q) & 1) ? v : 0;
    }
    };
    if (blockIdx.y == 0) body(std::integral_constant<int, 0>{});
    else body(std::integral_constant<int, 1>{});
}

}  // namespace

cudaError_t launch_search_wide(const SearchBatch &b, uint8_t *dirs, int32_t *vars,
                               long long *dist_luma, long long *dist_chroma, uint8_t *skipped,
                               cudaStream_t s)
{
    for (int i = 0; i < b.n; i++) {
        const SearchFrameDev &F = b.f[i];
        const cudaError_t e = launch_find_dir(F.rec[0], F.rec_pitch[0], F.w, F.h, F.bitdepth,
                                              dirs + F.map_start, vars + F.map_start, s);
        if (e != cudaSuccess) return e;
    }
    if (skipped)
        dist_wide_kernel<true><<<dim3(b.total_blocks, 2), kWThreads, 0, s>>>(
            b, dirs, vars, dist_luma, dist_chroma, skipped);
    else
        dist_wide_kernel<false><<<dim3(b.total_blocks, 2), kWThreads, 0, s>>>(
            b, dirs, vars, dist_luma, dist_chroma, nullptr);
    return cudaGetLastError();
}

}  // namespace cdefgb
