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
#include "eq14.cuh"
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
                 uint8_t *skipped, int *status)
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
                    const int pm = CDEF_IN_BOUNDS(t + o[m] - &sm.tile[k][0], kTile * kTile, status)
                                       ? t[o[m]] : -1;
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

// Section 5's eq. 14 tables for the same frames (12-bit, 4:2:2, 4:4:4): per
// filter block, plane group and candidate, the sum over the 8x8 blocks of
// each plane of the group of eq. 14's value (readings R22-R24: population
// variances of the source and the filtered samples, an 8x8 block cut by the
// frame edge taking its n in-frame samples, 1/256 units evaluated in single
// precision by eq14_value).  With d = x + r (r the filter's change of
// sample x) a candidate needs per 8x8 block the sums of r, r (2x + r) and
// r (2 (x - s) + r) besides the candidate-free sums n, s, s^2, x, x^2 and
// (x - s)^2.  One CTA per (filter block, plane group) as in
// dist_wide_kernel; the 64 candidates are taken in four groups of 16 (four
// primary strengths), the threads' sums reduced per 8x8 block in shared
// memory, then each block's value formed and summed per candidate.  4:2:2
// chroma is not filtered (section 4): every entry is the unfiltered value.
//
// kCoded: the 128 combinations with section 4's skip semantics.  A
// thread's samples belong to one direction block with one coded flag, so
// its sums also go to a second set restricted to coded blocks: the
// skip-bit-clear entry of a candidate takes each 8x8 block's value from
// those (uncoded samples unfiltered, r = 0), the skip-bit-set entry from
// the sums over all samples; the (0, 0) slot with the bit set evaluates the
// (19, 7) preset; a filter block without coded residual is never filtered.
struct WideEq14Smem {
    int tile[2][kTile * kTile];    // the group's planes (luma: one; chroma: U and V)
    int prim[64][16];
    int inv[64][6];                // per 8x8 block: n, sum s, s^2, x, x^2, (x - s)^2
    int gs[64][16][3];             // per 8x8 block and candidate of the group: r, r (2x + r),
                                   // r (2 (x - s) + r)
    int gc[64][16][3];             // kCoded: the same over the coded blocks' samples
    int g19[64][3];                // kCoded: the (19, 7) preset's sums
    unsigned long long acc[64];    // per candidate: the sum of the blocks' values
    unsigned long long acc_cod[64];  // kCoded: the same, skip bit clear
    unsigned long long acc19;      // kCoded: the (19, 7) preset
    unsigned long long base;       // unfiltered: 4:2:2 chroma, blocks without coded residual
};

template <int kGroup, bool kCoded>
__device__ __forceinline__ void wide_eq14_body(const SearchBatch &batch, const uint8_t *dirs,
                                               const int32_t *vars, long long *dist_luma,
                                               long long *dist_chroma, uint8_t *skipped,
                                               WideEq14Smem &sm, int *status)
{
    constexpr bool chroma = kGroup != 0;
    constexpr int nplanes = chroma ? 2 : 1;
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
    const bool filtered = !chroma || F.chroma_format != 422;
    const int bw = F.w >> 3;
    const int Dbase = chroma ? F.damping - 1 : F.damping;

    // stage the planes (rec) of the group with the halo
    for (int k = 0; k < nplanes; k++) {
        const PlaneView v = plane_view(F, kGroup == 0 ? 0 : 1 + k);
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
        sm.prim[b][p] = pack_primary(pri << sh8, pri ? D - lp : 0, pri & 1, raised);
    }
    if (tid < 64) sm.acc[tid] = sm.acc_cod[tid] = 0;
    if (tid == 0) sm.base = sm.acc19 = 0;
    __syncthreads();

    // four threads per direction block: 8x8 blocks (two rows each) or 4x4
    // blocks of 4:2:0 chroma (one row each)
    const int b8 = tid >> 2, part = tid & 3;
    const int by = b8 >> 3, bx = b8 & 7;
    const int gby = fby * 8 + by, gbx = fbx * 8 + bx;   // co-located luma 8x8 block
    const bool in_luma = gby * 8 < F.h && gbx * 8 < F.w;
    const int d = in_luma ? dirs[F.map_start + gby * bw + gbx] : 0;
    // section 4: the coded flag of the thread's (co-located luma) block, and
    // whether the filter block has any
    const bool cflag = kCoded ? (in_luma && F.coded[gby * bw + gbx] != 0) : true;
    const bool any_coded = kCoded ? __syncthreads_or(cflag) != 0 : true;
    if (kCoded && kGroup == 0 && tid == 0) skipped[blk] = (uint8_t)!any_coded;
    const Eff e19 = make_eff(19, 7, F.damping, chroma,
                             chroma ? 0 : (in_luma ? vars[F.map_start + gby * bw + gbx] : 0), sh8);
    int o[12];
    for (int k = 0; k < 12; k++) {
        int dr, dc;
        tap_rc(d, k, dr, dc);
        o[k] = dr * kTile + dc;
    }
    const unsigned long long pairs = allowed_pairs(F, kGroup);
    const int Dhi = Dbase < 3 ? 3 : Dbase;

    for (int k = 0; k < nplanes; k++) {
        const PlaneView v = plane_view(F, kGroup == 0 ? 0 : 1 + k);
        const int rows = v.bs == 8 ? 2 : 1, cols = v.bs;
        const int r0 = by * v.bs + part * rows, c0 = bx * v.bs;
        // the thread's 8x8 block of this plane (4:2:0 chroma: four
        // direction blocks share one) and the blocks per plane row
        const int eb = v.bs == 8 ? b8 : (by >> 1) * 4 + (bx >> 1);
        const int* const t0 = &sm.tile[k][(r0 + 2) * kTile + c0 + 2];
        // the thread's samples: rows r0 .. r0 + rows - 1, columns c0 .. of
        // the block, those inside the filter block and the frame
        const int gy0 = fby * v.fh + r0, gx0 = fbx * v.fw + c0;
        const int nr = max(0, min(rows, min(v.fh - r0, v.h - gy0)));
        const int nc = max(0, min(cols, min(v.fw - c0, v.w - gx0)));
        // candidate-free sums per 8x8 block
        for (int i = tid; i < 64 * 6; i += kWThreads) (&sm.inv[0][0])[i] = 0;
        __syncthreads();
        {
            int n = 0, ss = 0, ss2 = 0, sx = 0, sx2 = 0, se = 0;
            for (int i = 0; i < nr; i++) {
                const uint8_t *srow = v.src + (int64_t)(gy0 + i) * v.src_pitch;
                for (int j = 0; j < nc; j++) {
                    const int x = t0[i * kTile + j], sv = sample_at(srow, gx0 + j, wide);
                    n++;
                    ss += sv;
                    ss2 += sv * sv;
                    sx += x;
                    sx2 += x * x;
                    se += (x - sv) * (x - sv);
                }
            }
            if (n) {
                atomicAdd(&sm.inv[eb][0], n);
                atomicAdd(&sm.inv[eb][1], ss);
                atomicAdd(&sm.inv[eb][2], ss2);
                atomicAdd(&sm.inv[eb][3], sx);
                atomicAdd(&sm.inv[eb][4], sx2);
                atomicAdd(&sm.inv[eb][5], se);
            }
        }
        __syncthreads();
        if (!filtered || !any_coded) {
            // 4:2:2 chroma, or a filter block without coded residual: every
            // candidate gives the unfiltered samples
            if (tid < 64 && sm.inv[tid][0]) {
                const int *q = sm.inv[tid];
                atomicAdd(&sm.base, (unsigned long long)eq14_value(q[0], q[1], q[2], q[3], q[4], q[5],
                                                                   F.bitdepth));
            }
            __syncthreads();
            continue;
        }
        for (int cg = 0; cg < 4; cg++) {
            // the (19, 7) preset rides along with the first group
            const bool with19 = kCoded && cg == 0 && (pairs & 1);
            if (!((pairs >> (16 * cg)) & 0xffffull)) continue;   // no allowed pair in the group
            for (int i = tid; i < 64 * 16 * 3; i += kWThreads) {
                (&sm.gs[0][0][0])[i] = 0;
                if (kCoded) (&sm.gc[0][0][0])[i] = 0;
            }
            if (kCoded && tid < 64 * 3) (&sm.g19[0][0])[tid] = 0;
            __syncthreads();
            int a[16][3], a19[3] = {0, 0, 0};
#pragma unroll
            for (int c = 0; c < 16; c++) a[c][0] = a[c][1] = a[c][2] = 0;
            for (int i = 0; i < nr; i++) {
                const uint8_t *srow = v.src + (int64_t)(gy0 + i) * v.src_pitch;
                for (int j = 0; j < nc; j++) {
                    const int *t = t0 + i * kTile + j;
                    const int x = t[0], sv = sample_at(srow, gx0 + j, wide);
                    int pv[12], mn = x, mx = x;
#pragma unroll
                    for (int m = 0; m < 12; m++) {
                        const int pm = CDEF_IN_BOUNDS(t + o[m] - &sm.tile[k][0], kTile * kTile, status)
                                           ? t[o[m]] : -1;
                        pv[m] = pm < 0 ? x : pm;   // outside the frame: adds nothing
                        mn = min(mn, pv[m]);
                        mx = max(mx, pv[m]);
                    }
                    // secondary sums for S_s = 1, 2, 4 at both dampings
                    int qlo[4] = {0, 0, 0, 0}, qhi[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int si = 1; si < 4; si++) {
                        const int sS = si == 3 ? 4 : si, S = sS << sh8, l2 = sS == 4 ? 2 : sS - 1;
                        const int shl = max(0, Dbase - l2), shh = max(0, Dhi - l2);
#pragma unroll
                        for (int m = 4; m < 12; m++) {
                            const int w = m < 8 ? 2 : 1;
                            qlo[si] += w * constrain(pv[m] - x, S, shl);
                            qhi[si] += w * constrain(pv[m] - x, S, shh);
                        }
                    }
#pragma unroll
                    for (int pi = 0; pi < 4; pi++) {
                        const int pc = sm.prim[b8][cg * 4 + pi];
                        const int S = pc & 0xfff, sh = (pc >> 12) & 0xff;
                        const int w0 = (pc >> 20) & 1 ? 3 : 4, w1 = 6 - w0;
                        const bool raised = (pc >> 21) & 1;
                        const int Pp = w0 * (constrain(pv[0] - x, S, sh) + constrain(pv[1] - x, S, sh)) +
                                       w1 * (constrain(pv[2] - x, S, sh) + constrain(pv[3] - x, S, sh));
#pragma unroll
                        for (int si = 0; si < 4; si++) {
                            const int y = min(mx, max(mn, x + round16(Pp + (raised ? qhi[si] : qlo[si]))));
                            const int r = y - x;
                            a[pi * 4 + si][0] += r;
                            a[pi * 4 + si][1] += r * (2 * x + r);
                            a[pi * 4 + si][2] += r * (2 * (x - sv) + r);
                        }
                    }
                    if (with19) {   // the (19, 7) preset (section 4)
                        int P = 0, Q = 0;
#pragma unroll
                        for (int m = 0; m < 4; m++)
                            P += (m < 2 ? e19.w0 : e19.w1) * constrain(pv[m] - x, e19.pri, e19.psh);
#pragma unroll
                        for (int m = 4; m < 12; m++)
                            Q += (m < 8 ? 2 : 1) * constrain(pv[m] - x, e19.sec, e19.ssh);
                        const int r = min(mx, max(mn, x + round16(P + Q))) - x;
                        a19[0] += r;
                        a19[1] += r * (2 * x + r);
                        a19[2] += r * (2 * (x - sv) + r);
                    }
                }
            }
            // the four threads of a direction block, then the block's 8x8
            // block (four direction blocks in 4:2:0 chroma) in shared memory
#pragma unroll
            for (int c = 0; c < 16; c++) {
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    int w = a[c][j];
                    w += __shfl_xor_sync(0xffffffffu, w, 1);
                    w += __shfl_xor_sync(0xffffffffu, w, 2);
                    if (part == 0 && w) {
                        atomicAdd(&sm.gs[eb][c][j], w);
                        if (kCoded && cflag) atomicAdd(&sm.gc[eb][c][j], w);
                    }
                }
            }
            if (with19) {
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    int w = a19[j];
                    w += __shfl_xor_sync(0xffffffffu, w, 1);
                    w += __shfl_xor_sync(0xffffffffu, w, 2);
                    if (part == 0 && w) atomicAdd(&sm.g19[eb][j], w);
                }
            }
            __syncthreads();
            // each 8x8 block's value per candidate; thread: candidate tid % 16,
            // blocks tid / 16 + 16 m
            long long sum = 0, sum_cod = 0, sum19 = 0;
            for (int i = tid; i < 64 * 16; i += kWThreads) {
                const int e = i >> 4, c = i & 15;
                const int *q = sm.inv[e];
                if (!q[0]) continue;
                const int *g = sm.gs[e][c];
                sum += eq14_value(q[0], q[1], q[2], (long long)q[3] + g[0], (long long)q[4] + g[1],
                                  (long long)q[5] + g[2], F.bitdepth);
                if (kCoded) {
                    const int *h = sm.gc[e][c];
                    sum_cod += eq14_value(q[0], q[1], q[2], (long long)q[3] + h[0],
                                          (long long)q[4] + h[1], (long long)q[5] + h[2], F.bitdepth);
                }
                if (kCoded && with19 && c == 0) {
                    const int *h = sm.g19[e];
                    sum19 += eq14_value(q[0], q[1], q[2], (long long)q[3] + h[0],
                                        (long long)q[4] + h[1], (long long)q[5] + h[2], F.bitdepth);
                }
            }
            sum += __shfl_xor_sync(0xffffffffu, sum, 16);
            if (lane < 16) atomicAdd(&sm.acc[cg * 16 + lane], (unsigned long long)sum);
            if (kCoded) {
                sum_cod += __shfl_xor_sync(0xffffffffu, sum_cod, 16);
                if (lane < 16) atomicAdd(&sm.acc_cod[cg * 16 + lane], (unsigned long long)sum_cod);
                if (with19) {
                    sum19 += __shfl_xor_sync(0xffffffffu, sum19, 16);
                    if (lane == 0 && sum19) atomicAdd(&sm.acc19, (unsigned long long)sum19);
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    const bool plain = !filtered || !any_coded;   // every entry the unfiltered value
    if (!kCoded && tid < 64) {
        long long *out = (kGroup == 0 ? dist_luma : dist_chroma) + (int64_t)blk * 64;
        const long long v = plain ? (long long)sm.base : (long long)sm.acc[tid];
        out[tid] = ((pairs >> tid) & 1) ? v : 0;
    } else if (kCoded && tid < 128) {
        // q = k * 64 + p * 4 + s
        const int q = tid & 63, k = tid >> 6;
        const long long v = plain ? (long long)sm.base
                            : k ? (q == 0 ? (long long)sm.acc19 : (long long)sm.acc[q])
                                : (long long)sm.acc_cod[q];
        long long *out = (kGroup == 0 ? dist_luma : dist_chroma) + (int64_t)blk * 128;
        out[tid] = ((pairs >> q) & 1) ? v : 0;
    }
}

template <bool kCoded>
__global__ void __launch_bounds__(kWThreads, 2)
dist_wide_eq14_kernel(const __grid_constant__ SearchBatch batch, const uint8_t *__restrict__ dirs,
                      const int32_t *__restrict__ vars, long long *dist_luma, long long *dist_chroma,
                      uint8_t *skipped, int *status)
{
    extern __shared__ __align__(16) uint8_t wsm_bytes[];
    WideEq14Smem &sm = *reinterpret_cast<WideEq14Smem *>(wsm_bytes);
    if (blockIdx.y == 0)
        wide_eq14_body<0, kCoded>(batch, dirs, vars, dist_luma, dist_chroma, skipped, sm, status);
    else
        wide_eq14_body<1, kCoded>(batch, dirs, vars, dist_luma, dist_chroma, skipped, sm, status);
}

}  // namespace

cudaError_t launch_search_wide(const SearchBatch &b, uint8_t *dirs, int32_t *vars,
                               long long *dist_luma, long long *dist_chroma, uint8_t *skipped,
                               cudaStream_t s, bool eq14, int *status)
{
    for (int i = 0; i < b.n; i++) {
        const SearchFrameDev &F = b.f[i];
        const cudaError_t e = launch_find_dir(F.rec[0], F.rec_pitch[0], F.w, F.h, F.bitdepth,
                                              dirs + F.map_start, vars + F.map_start, s);
        if (e != cudaSuccess) return e;
    }
    if (eq14) {
        static int attr_dev = -1;
        int dev = 0;
        cudaGetDevice(&dev);
        if (dev != attr_dev) {
            cudaFuncSetAttribute(dist_wide_eq14_kernel<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WideEq14Smem));
            cudaFuncSetAttribute(dist_wide_eq14_kernel<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WideEq14Smem));
            attr_dev = dev;
        }
        if (skipped)
            dist_wide_eq14_kernel<true><<<dim3(b.total_blocks, 2), kWThreads, sizeof(WideEq14Smem), s>>>(
                b, dirs, vars, dist_luma, dist_chroma, skipped, status);
        else
            dist_wide_eq14_kernel<false><<<dim3(b.total_blocks, 2), kWThreads, sizeof(WideEq14Smem), s>>>(
                b, dirs, vars, dist_luma, dist_chroma, nullptr, status);
    } else if (skipped)
        dist_wide_kernel<true><<<dim3(b.total_blocks, 2), kWThreads, 0, s>>>(
            b, dirs, vars, dist_luma, dist_chroma, skipped, status);
    else
        dist_wide_kernel<false><<<dim3(b.total_blocks, 2), kWThreads, 0, s>>>(
            b, dirs, vars, dist_luma, dist_chroma, nullptr, status);
    return cudaGetLastError();
}

CDEF_FAULT_COUNTER(index_faults_search_wide)

}  // namespace cdefgb
