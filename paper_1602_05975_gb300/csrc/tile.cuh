// Shared tile machinery of the CDEF kernels (filter and strength search):
// the staged tile layout, the packed 16-bit tap arithmetic of eq. 7, the
// eq. 8 rounding and eq. 9-12 clip, the per-block parameter words of
// section 3.2, and the direction-search line sums of Algorithm 1.
//
// Layout.  A 64x64 filter block's luma tile (plus the 2-pixel halo the taps
// reach) and both 32x32 chroma tiles are staged by 2-D TMA loads, then
// re-laid as 16-bit values biased by +128, two per 32-bit word: luma as
// pixel pairs at even and at odd column alignment (any tap column offset is
// one aligned word), chroma as (U, V) words.  Positions outside the frame
// hold 0, a value no biased sample takes.
//
// Packed arithmetic.  For a tap value p and the filtered pixel x, eq. 7 with
// strength S and shift sh = D - floor(log2 S) gives the clamped tap value
// c = x + f(p - x) = clamp(p, x - lim, x + lim), lim = max(0, S - (|p - x| >> sh)).
// With K = (S + 1) * 2^sh - 1:  lim = max(0, K - |p - x|) >> sh  (exact), and
// K - |p - x| = min((x + K) - p, p - (x - K)).  S = 0 gives lim = 0, c = x.
#pragma once

#include "cdef_device.cuh"
#include "cdef_internal.h"
#include "tma.cuh"

namespace cdefgb {
namespace tile {

constexpr int kLumaRows = kLumaBoxRows;            // 68
constexpr int kLumaPitch = 44;                     // words per row (16-byte multiple)
constexpr int kLumaWords = 40;                     // words with data: 80 columns
constexpr int kChromaRows = kChromaBoxRows;        // 36
constexpr int kChromaPitch = 36;                   // words per row
constexpr uint32_t kBias = 128;                    // sample bias in shared memory
constexpr uint32_t kB1 = 2048;                     // bias of the K - |p - x| lanes
constexpr uint32_t kLanes = 0x10001u;              // one in each 16-bit lane
constexpr long long kWaitCycles = kDefaultWaitCycles;

// Per-block constants of one tap set.
struct SetC {
    uint32_t sh;     // the damping shift of eq. 7 (0..15)
    uint32_t mask;   // per-lane mask after the packed shift: (0xffff >> sh) per lane
    uint32_t posb;   // (kB1 >> sh) in both lanes
    uint32_t kb;     // K + kB1 in both lanes
};

struct alignas(16) BlockC {
    SetC p, s;
    uint32_t flags;  // bit0 primary on, bit1 secondary on, bit2 odd primary strength
    uint32_t pneg;   // -posb of p per 16-bit lane (two's complement)
    uint32_t sneg;   // the same for s
    uint32_t pad;
};

// Per 16-bit lane a + b, the lanes read as signed and independent (no carry
// between them); every sum formed with it here stays within int16.
__device__ __forceinline__ uint32_t sadd16(uint32_t a, uint32_t b)
{
    return __viaddmax_s16x2(a, b, 0x80008000u);
}

// -v in each 16-bit lane (lanes 1..0xffff).
__host__ __device__ constexpr uint32_t lane_neg(uint32_t v)
{
    return ((0x10000u - (v & 0xffffu)) & 0xffffu) | (((0x10000u - (v >> 16)) & 0xffffu) << 16);
}

// Raw TMA destinations, double-buffered: the next block's tiles land while
// the current block is filtered.
struct RawTiles {
    alignas(128) uint8_t y[kLumaRows * 80 * 2];
    alignas(128) uint8_t u[kChromaRows * 48 * 2];
    alignas(128) uint8_t v[kChromaRows * 48 * 2];
};

// Re-laid tiles.
struct PairTiles {
    alignas(16) uint32_t le[kLumaRows * kLumaPitch];      // pairs at even columns
    alignas(16) uint32_t lo[kLumaRows * kLumaPitch];      // pairs at odd columns (right after le)
    alignas(16) uint32_t cw[kChromaRows * kChromaPitch];  // (U, V)
};

__device__ __forceinline__ SetC make_set(int S, int sh)
{
    SetC c;
    const uint32_t K = ((uint32_t)(S + 1) << sh) - 1;
    c.sh = (uint32_t)sh;
    c.mask = (0xffffu >> sh) * kLanes;
    c.posb = (kB1 >> sh) * kLanes;
    c.kb = (K + kB1) * kLanes;
    return c;
}

__device__ __forceinline__ BlockC make_block_consts(const Eff &e)
{
    BlockC b;
    b.p = make_set(e.pri, e.psh);
    b.s = make_set(e.sec, e.ssh);
    b.flags = (e.pri ? 1u : 0u) | (e.sec ? 2u : 0u) | (e.w0 == 3 ? 4u : 0u);
    b.pneg = lane_neg(b.p.posb);
    b.sneg = lane_neg(b.s.posb);
    b.pad = 0;
    return b;
}

// One tap: clamp(p, x - lim, x + lim) on both lanes, xk1 = x + K + kB1,
// xk2 = K + kB1 - x.
//   m   = max(min(xk1 - p, p + xk2), kB1) = kB1 + max(0, K - |p - x|)
//   L   = m >> sh (the word shifted, then masked per lane), lim = L - (kB1 >> sh)
// The shift is a funnel shift on the integer ALU; a multiply-high by
// 2^(32 - sh) does the same on the multiply-add pipe, where on this GPU it
// takes four times the issue slots of a multiply-add (the tap's two
// subtractions already run there): the filter's launches ran 3-5% slower
// with it.
__device__ __forceinline__ uint32_t tap(uint32_t p, uint32_t X, uint32_t xk1, uint32_t xk2,
                                        const SetC &s)
{
    const uint32_t t1 = xk1 - p;
    uint32_t m = __vmaxu2(__viaddmin_u16x2(p, xk2, t1), kB1 * kLanes);
    m = (m >> s.sh) & s.mask;
    const uint32_t lim = m - s.posb;
    const uint32_t lo = X - lim;
    return __viaddmin_u16x2(lim, X, __vmaxu2(p, lo));   // min(x + lim, max(p, x - lim))
}

// The same tap with the limit's offset folded into per-word constants:
// xp = x + posb and xm = x - posb (per lane), so that x - lim = xp - L and
// x + lim = L + xm with L the shifted value.  One operation fewer per tap.
__device__ __forceinline__ uint32_t tap_folded(uint32_t p, uint32_t xk1, uint32_t xk2, uint32_t xp,
                                               uint32_t xm, const SetC &s)
{
    const uint32_t t1 = xk1 - p;
    uint32_t m = __vmaxu2(__viaddmin_u16x2(p, xk2, t1), kB1 * kLanes);
    m = (m >> s.sh) & s.mask;
    return __viaddmin_u16x2(m, xm, __vmaxu2(p, xp - m));   // min(x + lim, max(p, x - lim))
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

__device__ __forceinline__ bool valid_strengths(int pri, int sec)
{
    return (pri <= 15 || pri == 19) && (sec == 0 || sec == 1 || sec == 2 || sec == 4 || sec == 7);
}

// Direction search: line sums of directions Q and Q + 4 for block `blk`
// (Algorithm 1), from the biased luma pairs; costs into `cost`.
//
// The two samples of a pair word lie on the same line of direction d
// (d = 1, 2, 3) or on neighbouring lines k and k + 1 (d = 0, 5, 6, 7) or k and
// k - 1 (d = 4), with k the low sample's line.  So each word is added whole
// into a packed accumulator indexed by k, and the line sums are recovered at
// the end: line k = low lane of acc[k] + high lane of acc[k - 1], acc[k + 1]
// or acc[k].  A lane holds at most 8 samples below 2^12 (no carry).  At bit
// depths above 8 each sample is first shifted per lane: (x + 128) >> sh8 =
// (x >> sh8) + (128 >> sh8) exactly.
__host__ __device__ constexpr int hi_step(int d) { return d == 4 ? -1 : (d >= 1 && d <= 3) ? 0 : 1; }

template <int D>
__device__ __forceinline__ int dir_cost_from(const uint32_t (&acc)[15], int bias)
{
    constexpr LineWeights LW = make_line_weights();
    constexpr int st = hi_step(D);
    int s = 0;
#pragma unroll
    for (int k = 0; k < 15; k++) {
        if (!LW.w[D][k]) continue;
        int raw = (int)(acc[k] & 0xffffu);
        if (st == 0) raw += (int)(acc[k] >> 16);
        else if (k - st >= 0 && k - st < 15) raw += (int)(acc[k - st] >> 16);
        const int part = raw - (840 / LW.w[D][k]) * bias;
        s += part * part * LW.w[D][k];
    }
    return s;
}

template <int Q>
__device__ __forceinline__ void dir_costs(const uint32_t *le, int blk, int sh8, int (*cost)[8])
{
    uint32_t pa[15], pb[15];
#pragma unroll
    for (int k = 0; k < 15; k++) pa[k] = pb[k] = 0;
    const uint4 *b = reinterpret_cast<const uint4 *>(le + (2 + (blk >> 3) * 8) * kLumaPitch + 4 +
                                                     (blk & 7) * 4);
    const uint32_t mask = (0xffffu >> sh8) * kLanes;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const uint4 q = b[i * (kLumaPitch / 4)];
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const uint32_t w = sh8 ? (w4[m] >> sh8) & mask : w4[m];
            pa[line_of(Q, i, 2 * m)] += w;
            pb[line_of(Q + 4, i, 2 * m)] += w;
        }
    }
    // each sample carries (x >> sh8) + (128 >> sh8); x' = (x >> sh8) - 128
    const int bias = (int)(kBias >> sh8) + 128;
    cost[blk][Q] = dir_cost_from<Q>(pa, bias);
    cost[blk][Q + 4] = dir_cost_from<Q + 4>(pb, bias);
}

// Biased word of two samples; each lane is 0 where its sample is outside
// [0, limit) (the out-of-frame marker).
__device__ __forceinline__ uint32_t mark(uint32_t w, bool lo_in, bool hi_in)
{
    return (lo_in ? (w & 0xffffu) + kBias : 0u) | (hi_in ? (w & 0xffff0000u) + (kBias << 16) : 0u);
}

// Raw tiles -> biased pair layouts, 4 words per step.  `border` is set when
// the filter block touches the frame edge; only then are positions checked.
template <typename T, int kThreads>
__device__ __forceinline__ void stage_relayout(PairTiles &sm, const RawTiles &raw, bool border,
                                               int ly0, int lx0, int H, int W, int cy0, int cx0,
                                               int CH, int CW, bool chroma = true)
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
    for (int i = threadIdx.x; chroma && i < kChromaRows * (kChromaPitch / 4); i += kThreads) {
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

// Issued by one thread: the three tile loads of filter block (fby, fbx)
// into `raw`, completing on `bar`.  `maps` are the y, u, v tile maps;
// `extra_tx` bytes no load delivers are added to the expected count (the
// test aid of WaitLimits).
__device__ __forceinline__ void issue_tile_loads(const CUtensorMap *maps, int bitdepth, int fby,
                                                 int fbx, RawTiles &raw, uint64_t *bar,
                                                 bool chroma = true, int extra_tx = 0)
{
    const int B = bitdepth == 8 ? 1 : 2;
    const int lead = box_lead(B);
    // order earlier generic-proxy reads of this buffer before the async writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar, kLumaRows * luma_box_cols(B) * B +
                                   (chroma ? 2 * kChromaRows * chroma_box_cols(B) * B : 0) +
                                   extra_tx);
    tma_load_2d(raw.y, &maps[0], fbx * 64 - lead, fby * 64 - 2, bar);
    if (chroma) {
        tma_load_2d(raw.u, &maps[1], fbx * 32 - lead, fby * 32 - 2, bar);
        tma_load_2d(raw.v, &maps[2], fbx * 32 - lead, fby * 32 - 2, bar);
    }
}

// After a wait on `bar` (phase `parity`) gave up: the calling thread takes
// back the `extra_tx` bytes no load will deliver, then waits (bounded) until
// the loads actually issued on the barrier have landed, so that no copy
// writes into this CTA's shared memory after it leaves.
__device__ __forceinline__ void drain_tile_loads(uint64_t *bar, uint32_t parity, int extra_tx)
{
    if (extra_tx) mbar_complete_tx(bar, (uint32_t)extra_tx);
    mbar_wait_bounded(bar, parity, kWaitCycles);
}

}  // namespace tile
}  // namespace cdefgb
