// The CDEF filter (section 3, eq. 6-13) fused with the direction search
// (section 2), one 64x64 filter block (section 4) at a time per CTA;
// persistent CTAs walk the blocks of all frames of a launch.
//
// 1. Stage.  One thread issues three 2-D TMA tile loads (luma 64x64 plus the
//    2-pixel halo the taps reach, both 32x32 chroma tiles plus halo) for the
//    CTA's NEXT block, then the CTA waits (bounded) on the mbarrier of its
//    current block's tiles (double buffering).  The raw tiles are re-laid as
//    16-bit values biased by +128, two per 32-bit word:
//      - luma twice, as pixel pairs starting at even columns and at odd
//        columns, so a tap at any column offset is one aligned word;
//      - chroma as (U, V) words: both planes take the luma direction
//        (section 2) and one chroma strength pair (section 3.2), so the two
//        samples of a word take identical steps.
//    Positions outside the frame hold 0, a value no biased sample takes.
// 2. Direction search.  Four threads per 8x8 luma block, each forming the
//    line sums of two directions (d, d+4) with compile-time line tables; then
//    one thread per block takes the first maximum and the contrast
//    (Algorithm 1) and derives the block's parameters (section 3.2, eq. 13).
// 3. Filter.  Warp w takes row w of the 8x8 luma blocks: lane = (block
//    column, pixel-pair column), and each lane walks the 8 rows of its block
//    (direction, strengths and damping are constant over an 8x8 block,
//    section 3.1); then row w of the 4x4 chroma blocks, one (U, V) word per
//    lane and row.  Both go through one code path; tap positions are
//    per-lane word offsets from a per-direction table.
//
// Packed arithmetic (two 16-bit lanes per word).  For a tap value p and the
// filtered pixel x, eq. 7 with strength S and shift sh = D - floor(log2 S)
// gives the clamped tap value c = x + f(p - x) = clamp(p, x - lim, x + lim)
// with lim = max(0, S - (|p - x| >> sh)).  With K = (S + 1) * 2^sh - 1,
//   lim = max(0, K - |p - x|) >> sh                       (exact)
//   K - |p - x| = min((x + K) - p, p - (x - K)),
// which maps onto the packed 16-bit min/max/add-min instructions, the shift
// being a multiply-high.  S = 0 gives lim = 0, c = x: a tap set with zero
// strength contributes nothing without a branch.  The weighted sum of the
// clamped values minus 24x is the eq. 8 sum (each tap set's weights sum to
// 12 sixteenths).  A tap outside the frame is ignored (section 3.1); it is
// replaced by the filtered pixel itself, which is exactly equivalent: f(0) =
// 0 and the pixel is already in the clip range.  12-bit frames, whose range
// the packed biases do not cover, take a scalar path.
#include "cdef_device.cuh"
#include "cdef_internal.h"
#include "tma.cuh"

namespace cdefgb {

namespace {

constexpr int kThreads = 256;
constexpr int kMinCtas = 3;                        // resident CTAs per SM the registers are sized for
constexpr int kLumaRows = kLumaBoxRows;            // 68
constexpr int kLumaPitch = 44;                     // words per row (16-byte multiple)
constexpr int kLumaWords = 40;                     // words with data: 80 columns
constexpr int kChromaRows = kChromaBoxRows;        // 36
constexpr int kChromaPitch = 36;                   // words per row
constexpr uint32_t kBias = 128;                    // sample bias in shared memory
constexpr uint32_t kB1 = 2048;                     // bias of the K - |p - x| lanes
constexpr uint32_t kLanes = 0x10001u;              // one in each 16-bit lane
constexpr long long kWaitCycles = 1ll << 28;       // ~0.13 s at 2 GHz

// Per-block constants of one tap set.
struct SetC {
    uint32_t mul;    // 2^(32 - sh); sh = 0: 0xffffffff (umulhi gives m - 1)
    uint32_t mask;   // per-lane mask after the packed shift
    uint32_t posb;   // (kB1 >> sh) in both lanes; sh = 0: the low lane one less
    uint32_t kb;     // K + kB1 in both lanes
};

struct alignas(16) BlockC {
    SetC p, s;
    uint32_t flags;  // bit0 primary on, bit1 secondary on, bit2 odd primary strength
    uint32_t pad[3];
};

// Raw TMA destinations, double-buffered: the next block's tiles land while
// the current block is filtered.
struct RawTiles {
    alignas(128) uint8_t y[kLumaRows * 80 * 2];
    alignas(128) uint8_t u[kChromaRows * 48 * 2];
    alignas(128) uint8_t v[kChromaRows * 48 * 2];
};

struct FilterSmem {
    RawTiles raw[2];
    alignas(16) uint32_t le[kLumaRows * kLumaPitch];   // pairs at even columns
    alignas(16) uint32_t lo[kLumaRows * kLumaPitch];   // pairs at odd columns (right after le)
    alignas(16) uint32_t cw[kChromaRows * kChromaPitch];  // (U, V)
    alignas(16) int off[2][8][12];                      // tap word offsets [luma/chroma][d][tap]
    int cost[64][8];
    BlockC lb[64];
    BlockC cb;
    uint8_t dir[64];
    int var[64];
    int blk[2];                                         // block id of each raw buffer
    alignas(8) uint64_t bar[2];
};

__device__ __forceinline__ SetC make_set(int S, int sh)
{
    SetC c;
    const uint32_t K = ((uint32_t)(S + 1) << sh) - 1;
    const uint32_t b = kB1 >> sh;
    if (sh) {
        c.mul = 1u << (32 - sh);
        c.mask = (0xffffu >> sh) * kLanes;
        c.posb = b * kLanes;
    } else {
        c.mul = 0xffffffffu;
        c.mask = 0xffffffffu;
        c.posb = (kB1 << 16) | (kB1 - 1);
    }
    c.kb = (K + kB1) * kLanes;
    return c;
}

__device__ __forceinline__ BlockC make_block_consts(const Eff &e)
{
    BlockC b;
    b.p = make_set(e.pri, e.psh);
    b.s = make_set(e.sec, e.ssh);
    b.flags = (e.pri ? 1u : 0u) | (e.sec ? 2u : 0u) | (e.w0 == 3 ? 4u : 0u);
    return b;
}

// One tap: clamp(p, x - lim, x + lim) on both lanes, xk1 = x + K + kB1,
// xk2 = K + kB1 - x.
//   m   = max(min(xk1 - p, p + xk2), kB1) = kB1 + max(0, K - |p - x|)
//   L   = m >> sh (multiply-high, masked per lane), lim = L - (kB1 >> sh)
__device__ __forceinline__ uint32_t tap(uint32_t p, uint32_t X, uint32_t xk1, uint32_t xk2,
                                        const SetC &s)
{
    const uint32_t t1 = xk1 - p;
    uint32_t m = __vmaxu2(__viaddmin_u16x2(p, xk2, t1), kB1 * kLanes);
    m = __umulhi(m, s.mul) & s.mask;
    const uint32_t lim = m - s.posb;
    const uint32_t lo = X - lim;
    return __viaddmin_u16x2(lim, X, __vmaxu2(p, lo));   // min(x + lim, max(p, x - lim))
}

// Lanes of p holding the out-of-frame marker 0 take the centre's value.
__device__ __forceinline__ uint32_t in_frame(uint32_t p, uint32_t X)
{
    const uint32_t keep = __vminu2(p, kLanes) * 0xffffu;   // 0xffff where p > 0
    return (p & keep) | (X & ~keep);
}

// Eq. 8 from the two weighted clamped-value sums P, Q (each = 12x when its
// strength is zero), then the clip of eq. 9-12 when both sets are on.
__device__ __forceinline__ uint32_t finish(uint32_t X, uint32_t P, uint32_t Q, bool clip,
                                           uint32_t mn, uint32_t mx)
{
    // u = s + 4096 per lane with s = P + Q - 24x (|s| <= 1248)
    const uint32_t u = P + Q + (4096u * kLanes - 24u * X);
    const uint32_t pos = (u >> 12) & kLanes;            // [s >= 0]
    const uint32_t w = u + pos + 7u * kLanes;           // s + 7 + [s >= 0] + 4096
    const uint32_t r = (w >> 4) & (0x0fffu * kLanes);   // round(s / 16) + 256, ties away from 0
    uint32_t y = X + r - 256u * kLanes;
    if (clip) y = __vminu2(__vmaxu2(y, mn), mx);
    return y;
}

// Word offset of the tap at (dr, dc) for the luma layout (odd column
// offsets read the odd-column copy that follows the even one).
__device__ __forceinline__ int luma_off(int dr, int dc)
{
    return (dc & 1) ? kLumaRows * kLumaPitch + dr * kLumaPitch + ((dc - 1) >> 1)
                    : dr * kLumaPitch + (dc >> 1);
}

// The 12 taps of direction d: primary near +/-, far +/-, then secondary
// near +/- (d+2), near +/- (d-2), far +/- (d+2), far +/- (d-2).
__device__ __forceinline__ void tap_rc(int d, int t, int &dr, int &dc)
{
    const int k = t < 4 ? (t >> 1) : ((t - 4) >> 2);
    const int dd = t < 4 ? d : (((t - 4) >> 1) & 1) ? (d + 6) & 7 : (d + 2) & 7;
    const int sg = (t & 1) ? -1 : 1;
    dr = sg * tap_dr(dd, k);
    dc = sg * tap_dc(dd, k);
}

// One filtered word from its centre X and the 12 tap values.
__device__ __forceinline__ uint32_t filter_word(uint32_t X, uint32_t v[12], const BlockC &bc,
                                                bool any_p, bool any_s, bool any_clip,
                                                bool any_edge)
{
    if (any_edge) {
#pragma unroll
        for (int k = 0; k < 12; k++) v[k] = in_frame(v[k], X);
    }
    uint32_t P = 12u * X, Q = 12u * X, mn = X, mx = X;
    if (any_p) {
        const uint32_t xk1 = X + bc.p.kb, xk2 = bc.p.kb - X;
        const uint32_t n = tap(v[0], X, xk1, xk2, bc.p) + tap(v[1], X, xk1, xk2, bc.p);
        const uint32_t f = tap(v[2], X, xk1, xk2, bc.p) + tap(v[3], X, xk1, xk2, bc.p);
        if (bc.flags & 4) {
            const uint32_t t = n + f;
            P = t + t + t;                 // weights 3, 3
        } else {
            const uint32_t t = n + n + f;  // weights 4, 2
            P = t + t;
        }
    }
    if (any_s) {
        const uint32_t xk1 = X + bc.s.kb, xk2 = bc.s.kb - X;
        const uint32_t n = tap(v[4], X, xk1, xk2, bc.s) + tap(v[5], X, xk1, xk2, bc.s) +
                           tap(v[6], X, xk1, xk2, bc.s) + tap(v[7], X, xk1, xk2, bc.s);
        const uint32_t f = tap(v[8], X, xk1, xk2, bc.s) + tap(v[9], X, xk1, xk2, bc.s) +
                           tap(v[10], X, xk1, xk2, bc.s) + tap(v[11], X, xk1, xk2, bc.s);
        Q = n + n + f;                     // weights 2, 1
    }
    if (any_clip) {
#pragma unroll
        for (int k = 0; k < 12; k += 2) {
            mn = __vimin3_u16x2(mn, v[k], v[k + 1]);
            mx = __vimax3_u16x2(mx, v[k], v[k + 1]);
        }
    }
    return finish(X, P, Q, (bc.flags & 3) == 3, mn, mx);
}

// ---------------------------------------------------------------------------
// Scalar path for 12-bit frames.  `px(r, c)` returns the sample at tile
// position (r, c), or -1 outside the frame.
template <typename PX>
__device__ __noinline__ int filter_scalar(PX px, int r, int c, int d, Eff e)
{
    const int x = px(r, c);
    int sum = 0, mn = x, mx = x;
    for (int t = 0; t < 12; t++) {
        int dr, dc;
        tap_rc(d, t, dr, dc);
        const int p = px(r + dr, c + dc);
        if (p < 0) continue;
        int w, f;
        if (t < 4) {
            w = (t >> 1) ? e.w1 : e.w0;
            f = constrain(p - x, e.pri, e.psh);
        } else {
            w = ((t - 4) >> 2) ? 1 : 2;
            f = constrain(p - x, e.sec, e.ssh);
        }
        sum += w * f;
        mn = min(mn, p);
        mx = max(mx, p);
    }
    return min(mx, max(mn, x + round16(sum)));
}

__device__ __forceinline__ bool valid_strengths(int pri, int sec)
{
    return (pri <= 15 || pri == 19) && (sec == 0 || sec == 1 || sec == 2 || sec == 4 || sec == 7);
}

// Direction search: line sums of directions Q and Q + 4 for block `blk`
// (Algorithm 1), from the biased luma pairs; costs into `cost`.
template <int Q>
__device__ __forceinline__ void dir_costs(const uint32_t *le, int blk, int sh8, int (*cost)[8])
{
    constexpr LineWeights LW = make_line_weights();
    int pa[15], pb[15];
#pragma unroll
    for (int k = 0; k < 15; k++) pa[k] = pb[k] = 0;
    const uint4 *b = reinterpret_cast<const uint4 *>(le + (2 + (blk >> 3) * 8) * kLumaPitch + 4 +
                                                     (blk & 7) * 4);
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint4 q = b[i * (kLumaPitch / 4)];
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const int x0 = (int)(((w4[m] & 0xffffu) - kBias) >> sh8) - 128;
            const int x1 = (int)(((w4[m] >> 16) - kBias) >> sh8) - 128;
            pa[line_of(Q, i, 2 * m)] += x0;
            pa[line_of(Q, i, 2 * m + 1)] += x1;
            pb[line_of(Q + 4, i, 2 * m)] += x0;
            pb[line_of(Q + 4, i, 2 * m + 1)] += x1;
        }
    }
    int sa = 0, sb = 0;
#pragma unroll
    for (int k = 0; k < 15; k++) {
        if (LW.w[Q][k]) sa += pa[k] * pa[k] * LW.w[Q][k];
        if (LW.w[Q + 4][k]) sb += pb[k] * pb[k] * LW.w[Q + 4][k];
    }
    cost[blk][Q] = sa;
    cost[blk][Q + 4] = sb;
}

// Biased word of two samples; each lane is 0 where its sample is outside
// [0, limit) (the out-of-frame marker).
__device__ __forceinline__ uint32_t mark(uint32_t w, bool lo_in, bool hi_in)
{
    return (lo_in ? (w & 0xffffu) + kBias : 0u) | (hi_in ? (w & 0xffff0000u) + (kBias << 16) : 0u);
}

// Raw tiles -> biased pair layouts, 4 words per step.  `border` is set when
// the filter block touches the frame edge; only then are positions checked.
template <typename T>
__device__ __forceinline__ void stage_relayout(FilterSmem &sm, const RawTiles &raw, bool border,
                                               int ly0, int lx0, int H, int W, int cy0, int cx0,
                                               int CH, int CW)
{
    constexpr int B = sizeof(T);
    constexpr uint32_t kb = kBias * kLanes;
    // luma: quads of even-column pairs and the matching odd-column pairs
    for (int i = threadIdx.x; i < kLumaRows * (kLumaWords / 4); i += kThreads) {
        const int r = i / (kLumaWords / 4), q = i - r * (kLumaWords / 4);
        uint32_t e[5];
        if (B == 2) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(raw.y + r * 160);
            const uint4 v = *reinterpret_cast<const uint4 *>(row + 4 * q);
            e[0] = v.x; e[1] = v.y; e[2] = v.z; e[3] = v.w;
            e[4] = q + 1 < kLumaWords / 4 ? row[4 * q + 4] : 0u;
        } else {
            // tile column c is raw byte c + 8: words 2 + 2q and 3 + 2q hold pairs 4q .. 4q + 3
            const uint32_t *row = reinterpret_cast<const uint32_t *>(raw.y + r * 96);
            const uint2 v = *reinterpret_cast<const uint2 *>(row + 2 + 2 * q);
            e[0] = __byte_perm(v.x, 0, 0x4140);
            e[1] = __byte_perm(v.x, 0, 0x4342);
            e[2] = __byte_perm(v.y, 0, 0x4140);
            e[3] = __byte_perm(v.y, 0, 0x4342);
            e[4] = q + 1 < kLumaWords / 4 ? __byte_perm(row[4 + 2 * q], 0, 0x4140) : 0u;
        }
        if (border) {
            const int y = ly0 - 2 + r, x = lx0 - 8 + 8 * q;   // frame row, column of e[0]'s low lane
            const bool yin = y >= 0 && y < H;
#pragma unroll
            for (int k = 0; k < 5; k++)
                e[k] = mark(e[k], yin && x + 2 * k >= 0 && x + 2 * k < W,
                            yin && x + 2 * k + 1 >= 0 && x + 2 * k + 1 < W);
        } else {
#pragma unroll
            for (int k = 0; k < 5; k++) e[k] += kb;
        }
        *reinterpret_cast<uint4 *>(sm.le + r * kLumaPitch + 4 * q) = make_uint4(e[0], e[1], e[2], e[3]);
        *reinterpret_cast<uint4 *>(sm.lo + r * kLumaPitch + 4 * q) =
            make_uint4(__byte_perm(e[0], e[1], 0x5432), __byte_perm(e[1], e[2], 0x5432),
                       __byte_perm(e[2], e[3], 0x5432), __byte_perm(e[3], e[4], 0x5432));
    }
    // chroma: (U, V) words, 4 per step; tile column c is raw column c + lead - 2
    constexpr int cc = chroma_box_cols(B), lead = box_lead(B);
    for (int i = threadIdx.x; i < kChromaRows * (kChromaPitch / 4); i += kThreads) {
        const int r = i / (kChromaPitch / 4), q = i - r * (kChromaPitch / 4);
        const T *ur = reinterpret_cast<const T *>(raw.u) + r * cc + 4 * q + lead - 2;
        const T *vr = reinterpret_cast<const T *>(raw.v) + r * cc + 4 * q + lead - 2;
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; k++) o[k] = ((uint32_t)ur[k] | ((uint32_t)vr[k] << 16)) + kb;
        if (border) {
            const int y = cy0 - 2 + r, x = cx0 - 2 + 4 * q;
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (!(y >= 0 && y < CH && x + k >= 0 && x + k < CW)) o[k] = 0u;
        }
        *reinterpret_cast<uint4 *>(sm.cw + r * kChromaPitch + 4 * q) = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Everything after the tiles have landed: re-layout, direction search,
// per-block parameters, filtering and stores of one 64x64 filter block.
template <typename T>
__device__ void process_block(const FilterFrameDev &F, int fby, int fbx, int *status,
                              FilterSmem &sm, const RawTiles &raw)
{
    const int sh8 = F.bitdepth - 8;
    const int W = F.p[0].w, H = F.p[0].h, CW = F.p[1].w, CH = F.p[1].h;
    const int ly0 = fby * 64, lx0 = fbx * 64;
    const int cy0 = fby * 32, cx0 = fbx * 32;
    const int tid = threadIdx.x;

    cdef_fb_params prm = F.params[fby * F.fb_cols + fbx];
    if (!valid_strengths(prm.pri_y, prm.sec_y) || !valid_strengths(prm.pri_uv, prm.sec_uv) ||
        prm.damping < 3 || prm.damping > 6) {
        if (tid == 0) atomicOr(status, kStatusBadParams);
        prm.pri_y = prm.sec_y = prm.pri_uv = prm.sec_uv = 0;  // identity, defined output
        prm.damping = 3;
    }

    // does the 2-pixel halo of this block reach outside the frame?
    const bool border = fby == 0 || fbx == 0 || ly0 + 66 > H || lx0 + 66 > W ||
                        cy0 + 34 > CH || cx0 + 34 > CW;
    stage_relayout<T>(sm, raw, border, ly0, lx0, H, W, cy0, cx0, CH, CW);
    __syncthreads();

    // ---- direction search
    const int bw = W >> 3;
    const bool fused = F.dir == nullptr;
    if (fused) {
        const int warp = tid >> 5, lane = tid & 31;
        const int blk = (warp >> 2) * 32 + lane;
        switch (warp & 3) {
        case 0: dir_costs<0>(sm.le, blk, sh8, sm.cost); break;
        case 1: dir_costs<1>(sm.le, blk, sh8, sm.cost); break;
        case 2: dir_costs<2>(sm.le, blk, sh8, sm.cost); break;
        default: dir_costs<3>(sm.le, blk, sh8, sm.cost); break;
        }
        __syncthreads();
    }
    if (tid < 64) {
        const int gby = fby * 8 + (tid >> 3), gbx = fbx * 8 + (tid & 7);
        int d = 0, v = 0;
        if (gby * 8 < H && gbx * 8 < W) {
            if (fused) {
                int best = 0, bc = sm.cost[tid][0];
#pragma unroll
                for (int k = 1; k < 8; k++) {
                    const int c = sm.cost[tid][k];
                    if (c > bc) { bc = c; best = k; }
                }
                d = best;
                v = bc - sm.cost[tid][(best + 4) & 7];
            } else {
                d = F.dir[gby * bw + gbx];
                v = F.var[gby * bw + gbx];
            }
        }
        sm.dir[tid] = (uint8_t)d;
        sm.var[tid] = v;
        sm.lb[tid] = make_block_consts(make_eff(prm.pri_y, prm.sec_y, prm.damping, false, v, sh8));
    }
    if (tid == 64)
        sm.cb = make_block_consts(make_eff(prm.pri_uv, prm.sec_uv, prm.damping, true, 0, sh8));
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    if (F.bitdepth > 10) {
        // 12-bit: scalar path over every sample
        for (int i = tid; i < 64 * 64 + 2 * 32 * 32; i += kThreads) {
            const int pl = i < 4096 ? 0 : (i < 5120 ? 1 : 2);
            const int j = pl == 0 ? i : (i - 4096 - (pl - 1) * 1024);
            const int w = pl ? 32 : 64, rr = j / w, cc = j - rr * w;
            const int gy = (pl ? cy0 : ly0) + rr, gx = (pl ? cx0 : lx0) + cc;
            if (gy >= F.p[pl].h || gx >= F.p[pl].w) continue;
            const int blk = pl ? (rr >> 2) * 8 + (cc >> 2) : (rr >> 3) * 8 + (cc >> 3);
            const Eff e = pl ? make_eff(prm.pri_uv, prm.sec_uv, prm.damping, true, 0, sh8)
                             : make_eff(prm.pri_y, prm.sec_y, prm.damping, false, sm.var[blk], sh8);
            auto px = [&](int r2, int c2) -> int {
                uint32_t w2;
                if (pl == 0) {
                    w2 = sm.le[r2 * kLumaPitch + (c2 >> 1)];
                    w2 = (c2 & 1) ? (w2 >> 16) : (w2 & 0xffff);
                } else {
                    w2 = sm.cw[r2 * kChromaPitch + c2];
                    w2 = pl == 2 ? (w2 >> 16) : (w2 & 0xffff);
                }
                return w2 ? (int)(w2 - kBias) : -1;
            };
            const int r = 2 + rr, c = pl ? 2 + cc : 8 + cc;
            reinterpret_cast<T *>(F.p[pl].out + (int64_t)gy * F.p[pl].out_pitch)[gx] =
                (T)filter_scalar(px, r, c, sm.dir[blk], e);
        }
        return;
    }

    // ---- filter: task 0 = row `warp` of 8x8 luma blocks (lane = block
    // column x pair column, 8 rows), task 1 = row `warp` of 4x4 chroma blocks
    // (lane = block column x column, 4 rows).  One code path for both.
#pragma unroll 1
    for (int task = 0; task < 2; task++) {
        const bool luma = task == 0;
        const int bx = lane >> 2, sub = lane & 3;
        const int blk = warp * 8 + bx;
        const int gby = fby * 8 + warp, gbx = fbx * 8 + bx;
        const bool inside = luma ? (gby * 8 < H && gbx * 8 < W) : (gby * 4 < CH && gbx * 4 < CW);
        // taps can leave the frame only in the outermost ring of 8x8 blocks
        const bool edge = gby == 0 || gbx == 0 || gby == (H >> 3) - 1 || gbx == bw - 1;
        const int rows = luma ? 8 : 4;
        const int pitch = luma ? kLumaPitch : kChromaPitch;
        const uint32_t *base = luma ? sm.le + (2 + warp * 8) * kLumaPitch + 4 + bx * 4 + sub
                                    : sm.cw + (2 + warp * 4) * kChromaPitch + 2 + bx * 4 + sub;
        const BlockC bc = luma ? sm.lb[blk] : sm.cb;
        const unsigned fl = inside ? bc.flags : 0u;
        const bool any_p = __any_sync(0xffffffffu, fl & 1), any_s = __any_sync(0xffffffffu, fl & 2);
        const bool any_clip = __any_sync(0xffffffffu, (fl & 3) == 3);
        const bool any_edge = __any_sync(0xffffffffu, inside && edge);
        if (!__any_sync(0xffffffffu, inside)) continue;
        const int4 *op = reinterpret_cast<const int4 *>(sm.off[task][sm.dir[blk]]);
        const int4 o0 = op[0], o1 = op[1], o2 = op[2];
        const int o[12] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w, o2.x, o2.y, o2.z, o2.w};
        // output: row 0 of this lane's column
        const int oy = luma ? fby * 64 + warp * 8 : fby * 32 + warp * 4;
        const int ox = luma ? fbx * 64 + bx * 8 + 2 * sub : fbx * 32 + bx * 4 + sub;
        uint8_t *o_a = (luma ? F.p[0].out : F.p[1].out) + (int64_t)oy * (luma ? F.p[0].out_pitch : F.p[1].out_pitch);
        uint8_t *o_b = F.p[2].out + (int64_t)oy * F.p[2].out_pitch;
        const int64_t pa = luma ? F.p[0].out_pitch : F.p[1].out_pitch, pb = F.p[2].out_pitch;
#pragma unroll 1  // a compact loop body: the hot code has to stay in the instruction cache
        for (int i = 0; i < rows; i++) {
            const uint32_t *b = base + i * pitch;
            const uint32_t X = b[0];
            uint32_t v[12];
#pragma unroll
            for (int k = 0; k < 12; k++) v[k] = b[o[k]];
            uint32_t y = filter_word(X, v, bc, any_p, any_s, any_clip, any_edge) - kBias * kLanes;
            if (inside) {
                if (luma) {
                    if (sizeof(T) == 2)
                        *reinterpret_cast<uint32_t *>(o_a + 2 * ox) = y;
                    else
                        *reinterpret_cast<uint16_t *>(o_a + ox) = (uint16_t)__byte_perm(y, 0, 0x0020);
                } else {
                    reinterpret_cast<T *>(o_a)[ox] = (T)(y & 0xffff);
                    reinterpret_cast<T *>(o_b)[ox] = (T)(y >> 16);
                }
            }
            o_a += pa;
            o_b += pb;
        }
    }
}

struct BlockRef {
    int fi, fby, fbx;
};

template <int MAXF>
__device__ __forceinline__ BlockRef locate(const FilterBatch<MAXF> &batch, int blk)
{
    int fi = 0;
    if (MAXF > 1)
        while (fi + 1 < batch.n && blk >= batch.f[fi + 1].block_start) fi++;
    const int local = blk - batch.f[fi].block_start;
    const int fby = local / batch.f[fi].fb_cols;
    return {fi, fby, local - fby * batch.f[fi].fb_cols};
}

// Issued by one thread: the three tile loads of block `blk` into `raw`.
template <int MAXF>
__device__ __forceinline__ void issue_loads(const FilterBatch<MAXF> &batch, int blk, RawTiles &raw,
                                            uint64_t *bar)
{
    const BlockRef r = locate(batch, blk);
    const FilterFrameDev &F = batch.f[r.fi];
    const int B = F.bitdepth == 8 ? 1 : 2;
    const int lead = box_lead(B);
    // order earlier generic-proxy reads of this buffer before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar, kLumaRows * luma_box_cols(B) * B + 2 * kChromaRows * chroma_box_cols(B) * B);
    tma_load_2d(raw.y, &F.tmap[0], r.fbx * 64 - lead, r.fby * 64 - 2, bar);
    tma_load_2d(raw.u, &F.tmap[1], r.fbx * 32 - lead, r.fby * 32 - 2, bar);
    tma_load_2d(raw.v, &F.tmap[2], r.fbx * 32 - lead, r.fby * 32 - 2, bar);
}

// Persistent: each CTA takes blocks from the launch's work counter
// (work[0], dynamic so that blocks of uneven cost balance out); the tiles of
// its next block are loaded while it filters the current one.  The last CTA
// to finish resets the counter pair (work[1] counts finished CTAs), so a
// counter slot is ready for its next launch.
template <int MAXF>
__global__ void __launch_bounds__(kThreads, kMinCtas)
filter_kernel(const __grid_constant__ FilterBatch<MAXF> batch, int *status, unsigned *work)
{
    // A direct cast keeps every access in the shared state space (LDS/STS).
    extern __shared__ __align__(128) uint8_t smem_bytes[];
    FilterSmem &sm = *reinterpret_cast<FilterSmem *>(smem_bytes);
    const int tid = threadIdx.x;
    const int total = batch.total_blocks;

    if (smem_u32(smem_bytes) & 127) {  // the tile loads need 128-byte aligned destinations
        if (tid == 0) atomicOr(status, kStatusMisaligned);
    } else {
        if (tid == 0) {
            mbar_init(&sm.bar[0], 1);
            mbar_init(&sm.bar[1], 1);
            const int b = (int)atomicAdd(&work[0], 1u);
            sm.blk[0] = b;
            if (b < total) issue_loads(batch, b, sm.raw[0], &sm.bar[0]);
        }
        if (tid < 192) {  // tap offset tables [luma/chroma][d][tap]
            const int pl = tid / 96, d = (tid / 12) & 7, t = tid % 12;
            int dr, dc;
            tap_rc(d, t, dr, dc);
            sm.off[pl][d][t] = pl == 0 ? luma_off(dr, dc) : dr * kChromaPitch + dc;
        }
        __syncthreads();

        for (int it = 0;; it++) {
            const int buf = it & 1;
            const int blk = sm.blk[buf];
            if (blk >= total) break;
            if (tid == 0) {
                const int nb = (int)atomicAdd(&work[0], 1u);
                sm.blk[buf ^ 1] = nb;
                if (nb < total) issue_loads(batch, nb, sm.raw[buf ^ 1], &sm.bar[buf ^ 1]);
            }
            const bool arrived = mbar_wait_bounded(&sm.bar[buf], (it >> 1) & 1, kWaitCycles);
            if (__syncthreads_or(!arrived)) {  // the whole CTA leaves together
                if (tid == 0) {
                    atomicOr(status, kStatusTimeout);
                    if (sm.blk[buf ^ 1] < total)  // let the prefetch in flight land first
                        mbar_wait_bounded(&sm.bar[buf ^ 1], ((it + 1) >> 1) & 1, kWaitCycles);
                }
                break;
            }
            const BlockRef r = locate(batch, blk);
            const FilterFrameDev &F = batch.f[r.fi];
            if (F.bitdepth == 8)
                process_block<uint8_t>(F, r.fby, r.fbx, status, sm, sm.raw[buf]);
            else
                process_block<uint16_t>(F, r.fby, r.fbx, status, sm, sm.raw[buf]);
            __syncthreads();  // shared tiles, tables and the next block id are settled
        }
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&work[1], 1u) == gridDim.x - 1) {  // last CTA: reset for the next launch
            work[0] = 0;
            work[1] = 0;
            __threadfence();
        }
    }
}

constexpr size_t kSmemBytes = sizeof(FilterSmem);

// Grid size: one wave of persistent CTAs (resident CTAs per SM x SMs),
// never more than the work.
template <int MAXF>
int persistent_grid(int total)
{
    static int cached_dev = -1, cached_ctas = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        cudaFuncSetAttribute(filter_kernel<MAXF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
        cudaFuncSetAttribute(filter_kernel<MAXF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, filter_kernel<MAXF>, kThreads, kSmemBytes);
        cached_ctas = sms * (occ > 0 ? occ : 1);
        cached_dev = dev;
    }
    return total < cached_ctas ? total : cached_ctas;
}

}  // namespace

cudaError_t launch_filter_single(const FilterBatch<1> &b, int *status, unsigned *work,
                                 cudaStream_t s)
{
    const int grid = persistent_grid<1>(b.total_blocks);
    filter_kernel<1><<<grid, kThreads, kSmemBytes, s>>>(b, status, work);
    return cudaGetLastError();
}

cudaError_t launch_filter_batch(const FilterBatch<kMaxFilterBatch> &b, int *status, unsigned *work,
                                cudaStream_t s)
{
    const int grid = persistent_grid<kMaxFilterBatch>(b.total_blocks);
    filter_kernel<kMaxFilterBatch><<<grid, kThreads, kSmemBytes, s>>>(b, status, work);
    return cudaGetLastError();
}

}  // namespace cdefgb
