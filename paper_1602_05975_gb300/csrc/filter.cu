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
//    per-lane word offsets from a per-direction table.  (A warp's 32 lanes
//    read 32 consecutive words of a row: no shared-memory bank conflicts.)
// 4. Store.  The warp's output rows pass through a 512-byte staging area of
//    its own (the direction-cost array, idle while the block is filtered)
//    and leave as 16-byte stores of whole row segments: a warp store writes
//    full 128-byte lines.
//
// Packed arithmetic (two 16-bit lanes per word).  For a tap value p and the
// filtered pixel x, eq. 7 with strength S and shift sh = D - floor(log2 S)
// gives the clamped tap value c = x + f(p - x) = clamp(p, x - lim, x + lim)
// with lim = max(0, S - (|p - x| >> sh)).  With K = (S + 1) * 2^sh - 1,
//   lim = max(0, K - |p - x|) >> sh                       (exact)
//   K - |p - x| = min((x + K) - p, p - (x - K)),
// which maps onto the packed 16-bit min/max/add-min instructions, the shift
// being one shift of the word and a per-lane mask.  S = 0 gives lim = 0, c = x: a tap set with zero
// strength contributes nothing without a branch.  The weighted sum of the
// clamped values minus 24x is the eq. 8 sum (each tap set's weights sum to
// 12 sixteenths).  A tap outside the frame is ignored (section 3.1); it is
// replaced by the filtered pixel itself, which is exactly equivalent: f(0) =
// 0 and the pixel is already in the clip range.  12-bit frames, whose range
// the packed biases do not cover, take a scalar path.
#include <type_traits>

#include "tile.cuh"

namespace cdefgb {

namespace {

using namespace tile;

constexpr int kThreads = 256;
constexpr int kMinCtas = 4;                        // resident CTAs per SM the registers are sized for

struct FilterSmem {
    RawTiles raw;                                       // the next block's tiles land here
    PairTiles t;
    alignas(16) int off[2][8][12];                      // tap word offsets [luma/chroma][d][tap]
    // direction costs (direction search) and, while the block is filtered,
    // each warp's output rows on their way to 16-byte stores
    union {
        int cost[64][8];
        alignas(16) uint32_t stage[8][128];
    };
    BlockC lb[64];
    BlockC cb;
    BlockC bz;                                          // identity set (unfiltered blocks)
    uint8_t dir[64];
    uint8_t coded[64];                                  // 8x8 block has coded residual
    int var[64];
    int blk_next;                                       // block id of the tiles in `raw`
                                                        // (mode 3: plane << 28 | block)
    alignas(8) uint64_t bar;
};

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
        const uint32_t xp = X + bc.p.posb, xm = sadd16(X, bc.pneg);
        const uint32_t n = tap_folded(v[0], xk1, xk2, xp, xm, bc.p) +
                           tap_folded(v[1], xk1, xk2, xp, xm, bc.p);
        const uint32_t f = tap_folded(v[2], xk1, xk2, xp, xm, bc.p) +
                           tap_folded(v[3], xk1, xk2, xp, xm, bc.p);
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
        const uint32_t xp = X + bc.s.posb, xm = sadd16(X, bc.sneg);
        uint32_t n = 0, f = 0;
#pragma unroll
        for (int k = 4; k < 8; k++) n += tap_folded(v[k], xk1, xk2, xp, xm, bc.s);
#pragma unroll
        for (int k = 8; k < 12; k++) f += tap_folded(v[k], xk1, xk2, xp, xm, bc.s);
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

// Output of the filter loops.  Each lane hands its word of a row (two
// 16-bit lanes: a luma pixel pair, or a (U, V) pair) to its warp's 512-byte
// staging area (stage_put); once a group of whole rows is staged, the warp
// reads them back as 16-byte row segments and stores those (stage_flush),
// so that a warp store writes full 128-byte lines.  A segment cut by the
// frame's right edge stores only its blocks inside the frame.  The staging
// holds 4 rows of 16-bit luma, 8 rows of 8-bit luma, or the 4 rows of a
// chroma block row (U and V): kGroupRows.  kBytes: sample size in the frame.
template <bool kLuma, int kBytes>
struct StageOut {
    static constexpr int kGroupRows = (kLuma && kBytes == 1) ? 8 : 4;
    uint32_t off;        // byte offset in its plane of this lane's segment in its first row
    int n;               // blocks of the segment inside the frame (0: the lane stores nothing)
    int sp;              // luma layout: the plane written (0; 1, 2: a 4:4:4 chroma plane)

    // The plane in the luma layout a stage writes.
    __device__ __forceinline__ static const PlaneDev &lplane(const FilterFrameDev &F, int sp)
    {
        return sp == 0 ? F.p[0] : sp == 1 ? F.p[1] : F.p[2];
    }

    // The lane's segment: which staged row and 16 bytes it reads, where
    // they go.  fbx, fby: the filter block; warp: its block row.
    __device__ __forceinline__ StageOut(const FilterFrameDev &F, int lane, int fby, int fbx,
                                        int warp, bool row_in, int stage = 0)
        : sp(stage)
    {
        int plane = 0, r, c, nblk, blk_px, x_bytes, y0;
        if (kLuma && kBytes == 2) {          // lane L: row L / 8 of block L % 8
            r = lane >> 3, c = lane & 7, nblk = 1, blk_px = 8, x_bytes = (fbx * 64 + c * 8) * 2;
            y0 = fby * 64 + warp * 8;
        } else if (kLuma) {                  // row L / 4 of blocks 2 (L % 4), 2 (L % 4) + 1
            r = lane >> 2, c = lane & 3, nblk = 2, blk_px = 8, x_bytes = fbx * 64 + c * 16;
            y0 = fby * 64 + warp * 8;
        } else if (kBytes == 2) {            // lanes 0-15 U, 16-31 V: row (L % 16) / 4, two blocks
            plane = lane >> 4, r = (lane >> 2) & 3, c = lane & 3, nblk = 2, blk_px = 4;
            x_bytes = fbx * 64 + c * 16, y0 = fby * 32 + warp * 4;
        } else {                             // lanes 0-7 U, 8-15 V: row (L % 8) / 2, four blocks
            plane = (lane >> 3) & 1, r = (lane >> 1) & 3, c = lane & 1, nblk = 4, blk_px = 4;
            x_bytes = fbx * 32 + c * 16, y0 = fby * 32 + warp * 4;
        }
        const PlaneDev &P = kLuma ? lplane(F, sp) : plane ? F.p[2] : F.p[1];
        const int first = (fbx * 8 + c * nblk) * blk_px;
        int k = (P.w - first) / blk_px;
        k = k < 0 ? 0 : (k > nblk ? nblk : k);
        n = (row_in && (kLuma || kBytes == 2 || lane < 16)) ? k : 0;
        off = (uint32_t)((int64_t)(y0 + r) * P.out_pitch + x_bytes);
    }

    // the lane's word of row i (of the group) into the staging area
    __device__ __forceinline__ static void put(uint8_t *st8, int lane, int i, uint32_t y)
    {
        if (kLuma && kBytes == 2) {
            reinterpret_cast<uint32_t *>(st8)[i * 32 + lane] = y;
        } else if (kLuma) {
            reinterpret_cast<uint16_t *>(st8 + i * 64)[lane] = (uint16_t)__byte_perm(y, 0, 0x0020);
        } else if (kBytes == 2) {
            reinterpret_cast<uint16_t *>(st8 + i * 64)[lane] = (uint16_t)(y & 0xffff);
            reinterpret_cast<uint16_t *>(st8 + 256 + i * 64)[lane] = (uint16_t)(y >> 16);
        } else {
            st8[i * 32 + lane] = (uint8_t)(y & 0xff);
            st8[128 + i * 32 + lane] = (uint8_t)((y >> 16) & 0xff);
        }
    }

    // the staged group out to the frame; the staging is free again after it
    __device__ __forceinline__ void flush(const FilterFrameDev &F, const uint8_t *st8, int lane,
                                          int *status)
    {
        (void)status;   // used by the index-checking build
        constexpr int nblk = kLuma ? (kBytes == 2 ? 1 : 2) : (kBytes == 2 ? 2 : 4);
        __syncwarp();
        if (n) {
            int so;   // the segment in the staging area
            if (kLuma && kBytes == 2) so = (lane >> 3) * 128 + (lane & 7) * 16;
            else if (kLuma) so = (lane >> 2) * 64 + (lane & 3) * 16;
            else if (kBytes == 2) so = (lane >> 4) * 256 + ((lane >> 2) & 3) * 64 + (lane & 3) * 16;
            else so = ((lane >> 3) & 1) * 128 + ((lane >> 1) & 3) * 32 + (lane & 1) * 16;
            // the plane, selected without indexing the parameter block
            const bool v_plane = !kLuma && (kBytes == 2 ? lane >= 16 : ((lane >> 3) & 1));
            const PlaneDev &P = kLuma ? lplane(F, sp) : v_plane ? F.p[2] : F.p[1];
            uint8_t *dst = P.out + off;
            const int64_t pitch = P.out_pitch;
            // the segment's last byte inside the plane's rows
            const int ph = P.h;
            const bool ok = CDEF_IN_BOUNDS((int64_t)off + 15, pitch * ph, status) &&
                            CDEF_IN_BOUNDS(so + 15, 512, status);
            (void)ph;
            const uint4 q = ok ? *reinterpret_cast<const uint4 *>(st8 + so) : make_uint4(0, 0, 0, 0);
            if (!ok) {
                // (index-checking build) the access is skipped
            } else if (n == nblk) {
                *reinterpret_cast<uint4 *>(dst) = q;
            } else if (kBytes == 2 || kLuma) {   // one of two 8-byte blocks
                *reinterpret_cast<uint2 *>(dst) = make_uint2(q.x, q.y);
            } else {                             // 1..3 of four 4-byte blocks
                uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
                d32[0] = q.x;
                if (n > 1) d32[1] = q.y;
                if (n > 2) d32[2] = q.z;
            }
            // the next group: 4 rows down (16-bit luma; the other layouts
            // flush once per block row)
            off += 4 * (uint32_t)pitch;
        }
        __syncwarp();
    }
};

// ---------------------------------------------------------------------------
// 12-bit frames: sums of 12-bit differences leave the 16-bit lanes, so each
// sample of a word is filtered with 32-bit arithmetic (eq. 7-12 directly).
// `p` holds the 12 tap values (biased; 0 outside the frame: such a tap adds
// nothing and is not in the clip range).
__device__ __forceinline__ int filter_sample_wide(int x, const int p[12], const Eff &e)
{
    int sum = 0, mn = x, mx = x;
#pragma unroll
    for (int k = 0; k < 12; k++) {
        const int q = p[k] ? p[k] : x;
        const int f = k < 4 ? constrain(q - x, e.pri, e.psh) : constrain(q - x, e.sec, e.ssh);
        const int w = k < 2 ? e.w0 : k < 4 ? e.w1 : k < 8 ? 2 : 1;
        sum += w * f;
        mn = min(mn, q);
        mx = max(mx, q);
    }
    return min(mx, max(mn, x + round16(sum)));
}

// The 12-bit filter of one block's planes over the re-laid tiles: the
// warp/lane geometry of the packed path (task 0 luma rows of 8x8 blocks,
// task 1 chroma (U, V) rows of 4x4 blocks), both samples of a word in turn.
__device__ __noinline__ void filter_wide(const FilterFrameDev &F, int fby, int fbx,
                                         const cdef_fb_params &prm, bool any_coded, bool skip_l,
                                         bool skip_c, FilterSmem &sm, int *status)
{
    const int sh8 = F.bitdepth - 8;
    const int H = F.p[0].h, W = F.p[0].w, CH = F.p[1].h, CW = F.p[1].w;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool with_chroma = F.mode == 0;
#pragma unroll 1
    for (int task = 0; task < (with_chroma ? 2 : 1); task++) {
        const bool luma = task == 0;
        const int bx = lane >> 2, sub = lane & 3;
        const int blk = warp * 8 + bx;
        const int gby = fby * 8 + warp, gbx = fbx * 8 + bx;
        const bool inside = luma ? (gby * 8 < H && gbx * 8 < W) : (gby * 4 < CH && gbx * 4 < CW);
        if (!__any_sync(0xffffffffu, inside)) continue;   // lanes outside compute, store nothing
        const bool row_in = luma ? gby * 8 < H : gby * 4 < CH;
        const bool cpl = !luma || F.mode == 2;   // chroma parameters
        const bool on = any_coded && (sm.coded[blk] || (cpl ? skip_c : skip_l));
        Eff e = cpl ? make_eff(prm.pri_uv, prm.sec_uv, prm.damping, true, 0, sh8)
                    : make_eff(prm.pri_y, prm.sec_y, prm.damping, false, sm.var[blk], sh8);
        if (!on) e.pri = e.sec = 0;   // not filtered (section 4): every tap adds 0
        const int rows = luma ? 8 : 4;
        const int pitch = luma ? kLumaPitch : kChromaPitch;
        const uint32_t *base = luma ? sm.t.le + (2 + warp * 8) * kLumaPitch + 4 + bx * 4 + sub
                                    : sm.t.cw + (2 + warp * 4) * kChromaPitch + 2 + bx * 4 + sub;
        const int *o = sm.off[task][sm.dir[blk]];
        uint8_t *st8 = reinterpret_cast<uint8_t *>(sm.stage[warp]);
        // the re-laid tile the taps read (luma: even and odd copies)
        const uint32_t *tile0 = luma ? sm.t.le : sm.t.cw;
        const int tile_words = luma ? 2 * kLumaRows * kLumaPitch : kChromaRows * kChromaPitch;
        (void)tile0;
        (void)tile_words;
        auto run = [&](auto luma_c) {
            using Out = StageOut<decltype(luma_c)::value, 2>;
            Out out(F, lane, fby, fbx, warp, row_in);
            for (int g = 0; g < rows; g += Out::kGroupRows) {
                for (int i = 0; i < Out::kGroupRows; i++) {
                    const uint32_t *b = base + (g + i) * pitch;
                    const uint32_t X = b[0];
                    uint32_t v[12];
#pragma unroll
                    for (int k = 0; k < 12; k++)
                        v[k] = CDEF_IN_BOUNDS(b + o[k] - tile0, tile_words, status) ? b[o[k]] : X;
                    int y[2];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        int p[12];
#pragma unroll
                        for (int k = 0; k < 12; k++) p[k] = (int)((v[k] >> (16 * h)) & 0xffffu);
                        y[h] = filter_sample_wide((int)((X >> (16 * h)) & 0xffffu), p, e) - (int)kBias;
                    }
                    Out::put(st8, lane, i, (uint32_t)y[0] | ((uint32_t)y[1] << 16));
                }
                out.flush(F, st8, lane, status);
            }
        };
        if (luma) run(std::true_type{});
        else run(std::false_type{});
    }
}

// Everything after the tiles have landed: re-layout, direction search,
// per-block parameters, filtering and stores of one 64x64 filter block.
// `prefetch` runs (on every thread) once the raw tiles have been re-laid,
// so that the next block's tiles can land in the same buffer.
// kM3: frame mode 3 (the plane `stage` of an 8/10-bit 4:4:4 block); other
// modes are compiled with stage 0, so their code carries no stage logic.
template <typename T, bool kM3, typename Prefetch>
__device__ void process_block(const FilterFrameDev &F, int fby, int fbx, int *status,
                              FilterSmem &sm, const RawTiles &raw, Prefetch prefetch, int stage_in)
{
    const int stage = kM3 ? stage_in : 0;
    const int sh8 = F.bitdepth - 8;
    const int W = F.p[0].w, H = F.p[0].h, CW = F.p[1].w, CH = F.p[1].h;
    const int ly0 = fby * 64, lx0 = fbx * 64;
    const int cy0 = fby * 32, cx0 = fbx * 32;
    const int tid = threadIdx.x;

    cdef_fb_params prm = F.params[fby * F.fb_cols + fbx];
    if (!valid_strengths(prm.pri_y, prm.sec_y) || !valid_strengths(prm.pri_uv, prm.sec_uv) ||
        prm.damping < 3 || prm.damping > 6 || prm.skip > 3) {
        if (tid == 0) atomicOr(status, kStatusBadParams);
        prm.pri_y = prm.sec_y = prm.pri_uv = prm.sec_uv = 0;  // identity, defined output
        prm.damping = 3;
        prm.skip = 0;
    }
    // Section 4: strengths (0, 0) with the skip-condition bit set stand for
    // primary 19 and secondary 7.
    const bool skip_l = prm.skip & 1, skip_c = (prm.skip >> 1) & 1;
    if (skip_l && prm.pri_y == 0 && prm.sec_y == 0) {
        prm.pri_y = 19;
        prm.sec_y = 7;
    }
    if (skip_c && prm.pri_uv == 0 && prm.sec_uv == 0) {
        prm.pri_uv = 19;
        prm.sec_uv = 7;
    }

    // does the 2-pixel halo of this block reach outside the frame?
    const bool with_chroma = F.mode == 0;   // 4:2:0 chroma rides along
    const bool border = fby == 0 || fbx == 0 || ly0 + 66 > H || lx0 + 66 > W ||
                        (with_chroma && (cy0 + 34 > CH || cx0 + 34 > CW));
    stage_relayout<T, kThreads>(sm.t, raw, border, ly0, lx0, H, W, cy0, cx0, CH, CW, with_chroma);
    __syncthreads();
    prefetch();

    // ---- direction search
    const int bw = W >> 3;
    const bool fused = F.dir == nullptr;
    // mode 3 (8/10-bit 4:4:4, the three planes of a block in turn): stage 0
    // is luma; stages 1 and 2 (U, V) keep its directions, contrasts and
    // coded flags in shared memory and take the chroma parameters
    const bool chroma_stage = stage > 0;
    if (fused && !chroma_stage) {
        const int warp = tid >> 5, lane = tid & 31;
        const int blk = (warp >> 2) * 32 + lane;
        switch (warp & 3) {
        case 0: dir_costs<0>(sm.t.le, blk, sh8, sm.cost); break;
        case 1: dir_costs<1>(sm.t.le, blk, sh8, sm.cost); break;
        case 2: dir_costs<2>(sm.t.le, blk, sh8, sm.cost); break;
        default: dir_costs<3>(sm.t.le, blk, sh8, sm.cost); break;
        }
        __syncthreads();
    }
    int coded = 0;
    if (chroma_stage) {
        if (tid < 64) coded = sm.coded[tid];
    } else if (tid < 64) {
        const int gby = fby * 8 + (tid >> 3), gbx = fbx * 8 + (tid & 7);
        int d = 0, v = 0;
        if (gby * 8 < H && gbx * 8 < W) {
            coded = F.coded ? F.coded[gby * bw + gbx] != 0 : 1;
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
        sm.coded[tid] = (uint8_t)coded;
        // mode 2: the plane in the luma slot is a 4:4:4 chroma plane
        sm.lb[tid] = F.mode == 2
                         ? make_block_consts(make_eff(prm.pri_uv, prm.sec_uv, prm.damping, true, 0, sh8))
                         : make_block_consts(make_eff(prm.pri_y, prm.sec_y, prm.damping, false, v, sh8));
    }
    if (tid == 64)
        sm.cb = make_block_consts(make_eff(prm.pri_uv, prm.sec_uv, prm.damping, true, 0, sh8));
    if (tid == 65) sm.bz = make_block_consts(make_eff(0, 0, prm.damping, false, 0, sh8));
    // Section 4: a filter block without coded residual is not filtered; in
    // one that has some, an 8x8 block without it is filtered only when its
    // plane group's skip-condition bit is set (chroma: the co-located luma
    // block's flag).
    const bool any_coded = __syncthreads_or(coded);

    const int warp = tid >> 5, lane = tid & 31;
    if (F.bitdepth > 10) {
        filter_wide(F, fby, fbx, prm, any_coded, skip_l, skip_c, sm, status);
        return;
    }

    // ---- filter: task 0 = row `warp` of 8x8 luma blocks (lane = block
    // column x pair column, 8 rows), task 1 = row `warp` of 4x4 chroma blocks
    // (lane = block column x column, 4 rows).  One body, compiled once per
    // task so that the plane's geometry is fixed in each copy.
    auto task_body = [&](auto luma_c) {
        constexpr bool luma = decltype(luma_c)::value;
        constexpr int task = luma ? 0 : 1;
        const int bx = lane >> 2, sub = lane & 3;
        const int blk = warp * 8 + bx;
        const int gby = fby * 8 + warp, gbx = fbx * 8 + bx;
        const bool inside = luma ? (gby * 8 < H && gbx * 8 < W) : (gby * 4 < CH && gbx * 4 < CW);
        // taps can leave the frame only in the outermost ring of 8x8 blocks
        const bool edge = gby == 0 || gbx == 0 || gby == (H >> 3) - 1 || gbx == bw - 1;
        constexpr int rows = luma ? 8 : 4;
        constexpr int pitch = luma ? kLumaPitch : kChromaPitch;
        const uint32_t *base = luma ? sm.t.le + (2 + warp * 8) * kLumaPitch + 4 + bx * 4 + sub
                                    : sm.t.cw + (2 + warp * 4) * kChromaPitch + 2 + bx * 4 + sub;
        // a block that is not filtered (section 4) takes the identity set
        // (strengths 0: every tap clamps to x, no clip), so the loop below
        // needs no per-word test
        const bool lp = luma && F.mode != 2 && !chroma_stage;   // luma parameters
        const bool on = any_coded && (sm.coded[blk] || (lp ? skip_l : skip_c));
        const BlockC bc = !on ? sm.bz : (luma && !chroma_stage) ? sm.lb[blk] : sm.cb;
        const unsigned fl = inside ? bc.flags : 0u;
        const bool any_p = __any_sync(0xffffffffu, fl & 1), any_s = __any_sync(0xffffffffu, fl & 2);
        const bool any_clip = __any_sync(0xffffffffu, (fl & 3) == 3);
        const bool any_edge = __any_sync(0xffffffffu, inside && edge);
        if (!__any_sync(0xffffffffu, inside)) return;
        const int4 *op = reinterpret_cast<const int4 *>(sm.off[task][sm.dir[blk]]);
        const int4 o0 = op[0], o1 = op[1], o2 = op[2];
        const int o[12] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w, o2.x, o2.y, o2.z, o2.w};
        const bool row_in = luma ? gby * 8 < H : gby * 4 < CH;
        using Out = StageOut<luma, sizeof(T)>;
        Out out(F, lane, fby, fbx, warp, row_in, stage);
        // the re-laid tile the taps read (luma: even and odd copies)
        const uint32_t *tile0 = luma ? sm.t.le : sm.t.cw;
        constexpr int tile_words = luma ? 2 * kLumaRows * kLumaPitch : kChromaRows * kChromaPitch;
        (void)tile0;
        uint8_t *st8 = reinterpret_cast<uint8_t *>(sm.stage[warp]);
        const uint32_t *b = base;
#pragma unroll 1
        for (int g = 0; g < rows; g += Out::kGroupRows) {
#pragma unroll 1  // a compact loop body: the hot code has to stay in the instruction cache
            for (int i = 0; i < Out::kGroupRows; i++, b += pitch) {
                const uint32_t X = b[0];
                uint32_t v[12];
#pragma unroll
                for (int k = 0; k < 12; k++)
                    v[k] = CDEF_IN_BOUNDS(b + o[k] - tile0, tile_words, status) ? b[o[k]] : X;
                Out::put(st8, lane, i, filter_word(X, v, bc, any_p, any_s, any_clip, any_edge) -
                                           kBias * kLanes);
            }
            out.flush(F, st8, lane, status);
        }
    };
    task_body(std::true_type{});
    if (with_chroma) task_body(std::false_type{});
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

// Issued by one thread: the tile loads of block `blk` into `raw` (mode 3:
// the one plane of `stage`, whose map has the luma box).
template <int MAXF>
__device__ __forceinline__ void issue_loads(const FilterBatch<MAXF> &batch, int blk, RawTiles &raw,
                                            uint64_t *bar, int stage = 0)
{
    const BlockRef r = locate(batch, blk);
    const FilterFrameDev &F = batch.f[r.fi];
    issue_tile_loads(F.mode == 3 ? &F.tmap[stage] : F.tmap, F.bitdepth, r.fby, r.fbx, raw, bar,
                     F.mode == 0, batch.waits.extra_tx);
}

// Persistent: each CTA takes blocks from the launch's work counter
// (work[0], dynamic so that blocks of uneven cost balance out); the tiles of
// its next block are loaded while it filters the current one.  The last CTA
// to finish resets the counter pair (work[1] counts finished CTAs), so a
// counter slot is ready for its next launch.
// kM3: the launch of one mode-3 frame (8/10-bit 4:4:4, the three planes of
// a filter block in turn); other launches are compiled without the stages.
template <int MAXF, bool kM3 = false>
__global__ void __launch_bounds__(kThreads, kMinCtas)
filter_kernel(const __grid_constant__ FilterBatch<MAXF> batch, int *status, unsigned *work,
              int dep_wait)
{
    // The next launch on the stream may be scheduled as soon as every CTA of
    // this one is running (programmatic dependent launch); it fills the SMs
    // this grid's last CTAs leave idle.  Unless the caller declared
    // consecutive calls independent, each launch first waits here until the
    // previous grid on the stream has finished and its writes are visible.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (dep_wait) asm volatile("griddepcontrol.wait;" ::: "memory");
    // A direct cast keeps every access in the shared state space (LDS/STS).
    extern __shared__ __align__(128) uint8_t smem_bytes[];
    FilterSmem &sm = *reinterpret_cast<FilterSmem *>(smem_bytes);
    const int tid = threadIdx.x;
    const int total = batch.total_blocks;

    if (smem_u32(smem_bytes) & 127) {  // the tile loads need 128-byte aligned destinations
        if (tid == 0) atomicOr(status, kStatusMisaligned);
    } else {
        if (tid == 0) {
            mbar_init(&sm.bar, 1);
            const int b = (int)atomicAdd(&work[0], 1u);
            sm.blk_next = b;
            if (b < total) issue_loads(batch, b, sm.raw, &sm.bar);
        }
        if (tid < 192) {  // tap offset tables [luma/chroma][d][tap]
            const int pl = tid / 96, d = (tid / 12) & 7, t = tid % 12;
            int dr, dc;
            tap_rc(d, t, dr, dc);
            sm.off[pl][d][t] = pl == 0 ? luma_off(dr, dc) : dr * kChromaPitch + dc;
        }
        __syncthreads();

        // one tile buffer: block n's tiles are re-laid into the pair tiles,
        // then block n+1's loads are issued into the buffer while block n is
        // searched and filtered
        for (int it = 0;; it++) {
            const int bn = sm.blk_next;
            const int blk = kM3 ? (bn & 0x0fffffff) : bn, stage = kM3 ? (bn >> 28) : 0;
            if (blk >= total) break;
            const bool arrived = mbar_wait_bounded(&sm.bar, it & 1, batch.waits.wait_cycles);
            if (__syncthreads_or(!arrived)) {  // the whole CTA leaves together
                if (tid == 0) {
                    atomicOr(status, kStatusTimeout);
                    drain_tile_loads(&sm.bar, it & 1, batch.waits.extra_tx);
                }
                break;
            }
            auto prefetch = [&]() {
                if (tid == 0) {
                    if (kM3 && stage < 2) {   // the block's next plane
                        sm.blk_next = blk | ((stage + 1) << 28);
                        issue_loads(batch, blk, sm.raw, &sm.bar, stage + 1);
                    } else {
                        const int nb = (int)atomicAdd(&work[0], 1u);
                        sm.blk_next = nb;
                        if (nb < total) issue_loads(batch, nb, sm.raw, &sm.bar);
                    }
                }
            };
            const BlockRef r = locate(batch, blk);
            const FilterFrameDev &F = batch.f[r.fi];
            if (F.bitdepth == 8)
                process_block<uint8_t, kM3>(F, r.fby, r.fbx, status, sm, sm.raw, prefetch, stage);
            else
                process_block<uint16_t, kM3>(F, r.fby, r.fbx, status, sm, sm.raw, prefetch, stage);
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
template <int MAXF, bool kM3 = false>
int persistent_grid(int total)
{
    static int cached_dev = -1, cached_ctas = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        cudaFuncSetAttribute(filter_kernel<MAXF, kM3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes);
        cudaFuncSetAttribute(filter_kernel<MAXF, kM3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, filter_kernel<MAXF, kM3>, kThreads, kSmemBytes);
        cached_ctas = sms * (occ > 0 ? occ : 1);
        cached_dev = dev;
    }
    return total < cached_ctas ? total : cached_ctas;
}

template <int MAXF, bool kM3 = false>
cudaError_t launch_pdl(const FilterBatch<MAXF> &b, int *status, unsigned *work, bool overlap,
                       cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(persistent_grid<MAXF, kM3>(b.total_blocks));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int dep_wait = overlap ? 0 : 1;
    return cudaLaunchKernelEx(&cfg, filter_kernel<MAXF, kM3>, b, status, work, dep_wait);
}

}  // namespace

cudaError_t launch_filter_single(const FilterBatch<1> &b, int *status, unsigned *work,
                                 bool overlap, cudaStream_t s)
{
    return launch_pdl<1>(b, status, work, overlap, s);
}

cudaError_t launch_filter_batch(const FilterBatch<kMaxFilterBatch> &b, int *status, unsigned *work,
                                bool overlap, cudaStream_t s)
{
    return launch_pdl<kMaxFilterBatch>(b, status, work, overlap, s);
}

cudaError_t launch_filter_planes(const FilterBatch<3> &b, int *status, unsigned *work,
                                 bool overlap, cudaStream_t s)
{
    return launch_pdl<3>(b, status, work, overlap, s);
}

cudaError_t launch_filter_444(const FilterBatch<1> &b, int *status, unsigned *work, bool overlap,
                              cudaStream_t s)
{
    return launch_pdl<1, true>(b, status, work, overlap, s);
}

CDEF_FAULT_COUNTER(index_faults_filter)

}  // namespace cdefgb
