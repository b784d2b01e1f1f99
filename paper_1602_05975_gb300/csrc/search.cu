// Encoder strength search (section 5).
//
// dist_kernel: persistent CTAs take 64x64 filter blocks of any frame of the
//   batch from a work counter.  The decoded tiles are staged exactly as for
//   the filter (TMA, double buffering, biased 16-bit pair layout; see
//   tile.cuh), the 64 luma directions found (section 2), and every word of
//   two samples is then filtered under all 64 (primary, secondary) strength
//   pairs at once.  The clamped primary sum is formed once per primary
//   strength (16) and the secondary sum once per secondary strength (4):
//   exact, since eq. 8 is the sum of the two tap sets, each depending on one
//   strength only.  Each of the 64 pairs then only rounds, clips (eq. 9-12,
//   when both strengths are on) and accumulates (y - source)^2 into one of 64
//   per-lane registers.  Lanes cover the 8 columns of 8x8 blocks of a block
//   row, so their 64 sums are reduced across the warp by a butterfly that
//   leaves lane l with pairs 2l and 2l + 1, then across warps in shared
//   memory, into 64-bit block totals.
//
// The preset selection that follows (greedy search, optional
//   re-optimisation, N and block ids; eq. 15) is one persistent kernel in
//   presets.cu.
#include <climits>

#include <type_traits>

#include "eq14.cuh"
#include "tile.cuh"

namespace cdefgb {

namespace {

using namespace tile;

constexpr int kThreads = 256;
constexpr int kMinCtas = 2;

struct SearchSmem {
    RawTiles raw[2];
    PairTiles t;
    alignas(16) int off[2][8][12];    // tap word offsets [luma/chroma][d][tap]
    int cost[64][8];
    // luma primary sets per 8x8 block and signalled strength (entry 16: the
    // strength 19 of the (0,0)+skip preset); 17 entries per row also keep
    // the eight blocks a warp reads at once in different banks
    alignas(16) SetC pset[64][17];
    alignas(16) SetC cset[17];        // chroma primary sets per signalled strength (16: 19)
    alignas(16) SetC sset[3][4];      // secondary: luma; chroma at D - 1; chroma at D = 3
    alignas(16) SetC s7[64];          // secondary 7 of the (19, 7) preset, per luma block
    alignas(16) SetC s7c;             // and for chroma
    uint32_t pbits[64];               // luma: bit p set when the adjusted strength is odd
    uint32_t cbits;                   // chroma: the same per signalled strength
    uint32_t craised;                 // chroma: bit p, damping raised to floor(log2 p) = 3
    uint8_t dir[64];
    uint8_t coded[64];                // 8x8 block has coded residual (128-combination search)
    int var[64];
    unsigned long long acc[64];       // block totals of the current plane group
    unsigned long long accu[64];      // the part of them from blocks without coded residual
    unsigned long long acc14c[8];     // eq. 14: chroma block totals of the unit's candidates
    // eq. 14: sums over the 4-row halves of the 4:2:0 chroma 8x8 blocks,
    // [plane][block][half][value]: per candidate (r, r (s + 128), r (2 (x - s) + r)),
    // then n, x, x^2, s, s^2, (x - s)^2
    int e14h[2][16][2][30];
    // eq. 14: per luma 8x8 block the candidate-free sums n, x, x^2, s, s^2,
    // (x - s)^2, formed in the first candidate group and kept for the others
    int e14l[64][6];
    // eq. 14: secondary sums kept across the candidate groups (with the
    // block's idle tile buffer, see dist_block)
    uint32_t qc[12 * 256];
    unsigned long long base[2];       // sum of (x - s)^2 over the same pixels, per plane group
    int blk[2];
    alignas(8) uint64_t bar[2];
};

// two CTAs per SM (228 KB of shared memory, 1 KB reserved per CTA)
static_assert(sizeof(SearchSmem) <= 112 * 1024, "the search kernels run two CTAs per SM");

// The signalled secondary strengths {0, 1, 2, 4} by index.
__device__ __forceinline__ int sec_value(int i) { return i == 3 ? 4 : i; }

// Packed biased pair of source samples at (row, x), (row, x + 1) (luma) or
// the (U, V) word at (row, x) (chroma).
template <typename T>
__device__ __forceinline__ uint32_t load_src_pair(const uint8_t *row, int x)
{
    if (sizeof(T) == 2) return __ldg(reinterpret_cast<const uint32_t *>(row + 2 * x)) + kBias * kLanes;
    const uint32_t two = __ldg(reinterpret_cast<const uint16_t *>(row + x));
    return __byte_perm(two, 0, 0x4140) + kBias * kLanes;
}

template <typename T>
__device__ __forceinline__ uint32_t load_src_uv(const uint8_t *urow, const uint8_t *vrow, int x)
{
    const uint32_t u = __ldg(reinterpret_cast<const T *>(urow) + x);
    const uint32_t v = __ldg(reinterpret_cast<const T *>(vrow) + x);
    return (u | (v << 16)) + kBias * kLanes;
}

// Squared error of both lanes, added to acc.  8-bit errors fit a byte, so
// one dot-product instruction squares and adds both.
template <typename T>
__device__ __forceinline__ uint32_t add_sq(uint32_t acc, uint32_t y, uint32_t s)
{
    const uint32_t e = __vmaxu2(y, s) - __vminu2(y, s);   // |y - s| per lane
    if (sizeof(T) == 1) return __dp2a_lo(e, __byte_perm(e, 0, 0x0020), acc);
    const uint32_t lo = e & 0xffffu, hi = e >> 16;
    return acc + lo * lo + hi * hi;
}

// Weighted sum of the 4 primary clamped values for one set.
__device__ __forceinline__ uint32_t pri_sum(const uint32_t v[12], uint32_t X, const SetC &s, bool odd)
{
    const uint32_t xk1 = X + s.kb, xk2 = s.kb - X;
    const uint32_t n = tap(v[0], X, xk1, xk2, s) + tap(v[1], X, xk1, xk2, s);
    const uint32_t f = tap(v[2], X, xk1, xk2, s) + tap(v[3], X, xk1, xk2, s);
    const uint32_t t3 = n + f, t2 = n + n + f;
    return odd ? t3 + t3 + t3 : t2 + t2;   // weights 3,3 or 4,2
}

__device__ __forceinline__ uint32_t sec_sum(const uint32_t v[12], uint32_t X, const SetC &s)
{
    const uint32_t xk1 = X + s.kb, xk2 = s.kb - X;
    const uint32_t n = tap(v[4], X, xk1, xk2, s) + tap(v[5], X, xk1, xk2, s) +
                       tap(v[6], X, xk1, xk2, s) + tap(v[7], X, xk1, xk2, s);
    const uint32_t f = tap(v[8], X, xk1, xk2, s) + tap(v[9], X, xk1, xk2, s) +
                       tap(v[10], X, xk1, xk2, s) + tap(v[11], X, xk1, xk2, s);
    return n + n + f;   // weights 2, 1
}

// Sums N (16, 32 or 64) per-lane values across the warp.  Lane l ends with
// the totals of entries 2l, 2l + 1 in a[0], a[1] (N = 64), of entry l in
// a[0] (N = 32), or of entry l / 2 in a[0] (N = 16).
template <int N>
__device__ __forceinline__ void butterfly(uint32_t (&a)[N], int lane)
{
#pragma unroll
    for (int o = 16, n = N; o >= 1; o >>= 1, n >>= 1) {
        if (n > 1) {
            const bool upper = lane & o;
            const int half = n >> 1;
#pragma unroll
            for (int i = 0; i < N / 2; i++) {
                if (i < half) {
                    const uint32_t give = upper ? a[i] : a[i + half];
                    const uint32_t keep = upper ? a[i + half] : a[i];
                    a[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
                }
            }
        } else {
            a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
        }
    }
}

// One work unit: filter block (fby, fbx) of frame F, primary strengths
// grp * 16 / kG .. (grp + 1) * 16 / kG - 1 with all four secondary
// strengths, for both plane groups (64 / kG luma and 64 / kG chroma
// candidates).
// Levels LO..HI-1 of a warp reduction of N values (offsets 1 << level, in
// increasing order): after level l a lane keeps N >> (l + 1) entries, the
// upper half when its bit l is set.  `a` holds the N >> LO entries still
// live before level LO.
template <int N, int LO, int HI, int LEN>
__device__ __forceinline__ void wreduce(uint32_t (&a)[LEN], int lane)
{
#pragma unroll
    for (int lvl = LO; lvl < HI; lvl++) {
        const int o = 1 << lvl, n = N >> lvl;
        if (n > 1) {
            const bool upper = lane & o;
            const int half = n >> 1;
#pragma unroll
            for (int i = 0; i < LEN / 2; i++) {
                if (i < half) {
                    const uint32_t give = upper ? a[i] : a[i + half];
                    const uint32_t keep = upper ? a[i + half] : a[i];
                    a[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
                }
            }
        } else {
            a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
        }
    }
}

// The first entry a lane holds after all five levels of wreduce<N>.
__device__ __forceinline__ int wentry(int N, int lane)
{
    int e = 0;
#pragma unroll
    for (int lvl = 0; lvl < 5; lvl++) {
        const int n = N >> lvl;
        if (n > 1) e += (n >> 1) * ((lane >> lvl) & 1);
    }
    return e;
}

// kEq14: the tables hold section 5's eq. 14 instead of the squared error:
// per 8x8 block of each plane ((sigma_s^2 + sigma_d^2 + C1) /
// (2 sqrt(sigma_s^2 sigma_d^2 + C2))) * squared error, summed over the
// filter block.  With d = x + r, a candidate needs per 8x8 block the sums
// of r, r (2x + r) and r (2 (x - s) + r) besides sums that do not depend on
// it, kept per sample lane (the two samples of a word belong to U and V in
// the chroma task).
//
// kCoded: the 128-combination search of section 5 with section 4's skip
// semantics.  The (0, 0) slot, whose error is sum (x - s)^2 with no work,
// evaluates the (19, 7) preset instead; each candidate's sum is also kept
// for the 8x8 blocks without coded residual, so that the skip-bit-clear
// entries (those blocks unfiltered) follow as base + total - uncoded part.
// kSub: a subset of the pairs is allowed (section 5's low-complexity
// search): primaries without an allowed pair are skipped.
// kPl: 8/10-bit 4:4:4 frames, one plane per work unit (grp: 0 luma, 1 U,
// 2 V).  Each plane's tile is staged and filtered in the luma layout (a
// 4:4:4 chroma plane has the luma geometry and takes the chroma strengths,
// section 3.2, with the co-located luma direction, read from the direction
// map `mdir`, `mvar`); U's and V's entries are added into the chroma table,
// which the caller zeroes first.
template <typename T, int kG, bool kCoded, bool kEq14, bool kSub, bool kPl = false>
__device__ void dist_block(const SearchFrameDev &F, int fby, int fbx, int blk_global, int grp,
                           SearchSmem &sm, RawTiles &raw, long long *dist_luma,
                           long long *dist_chroma, uint8_t *skipped, const uint8_t *mdir,
                           const int32_t *mvar CDEF_DEBUG_PARAM(int *status))
{
    static_assert(!kPl || (kG == 1 && !kEq14) || (kG == 8 && kEq14 && !kCoded),
                  "plane units: squared-error tables, or eq. 14 over 64 pairs");
    const int plane = kPl ? grp : 0;
    const bool cparams = kPl && plane > 0;   // a 4:4:4 chroma plane in the luma layout
    constexpr int kPP = 16 / kG;           // primary strengths per unit
    constexpr int kN = 4 * kPP;            // candidates per plane group
    const int p0_unit = (kG == 1 || kPl) ? 0 : grp * kPP;
    const int sh8 = F.bitdepth - 8;
    const int W = F.w, H = F.h, CW = F.w >> 1, CH = F.h >> 1;
    const int ly0 = fby * 64, lx0 = fbx * 64, cy0 = fby * 32, cx0 = fbx * 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = F.damping;

    const bool border = fby == 0 || fbx == 0 || ly0 + 66 > H || lx0 + 66 > W ||
                        (!kPl && (cy0 + 34 > CH || cx0 + 34 > CW));
    stage_relayout<T, kThreads>(sm.t, raw, border, ly0, lx0, H, W, cy0, cx0, CH, CW, !kPl);
    __syncthreads();

    if (!kPl) {   // direction search: four threads per 8x8 block, two directions each
        const int b = (warp >> 2) * 32 + lane;
        switch (warp & 3) {
        case 0: dir_costs<0>(sm.t.le, b, sh8, sm.cost); break;
        case 1: dir_costs<1>(sm.t.le, b, sh8, sm.cost); break;
        case 2: dir_costs<2>(sm.t.le, b, sh8, sm.cost); break;
        default: dir_costs<3>(sm.t.le, b, sh8, sm.cost); break;
        }
        __syncthreads();
    }
    if (tid < 64) {
        if (kPl) {   // the luma direction and contrast from the map
            const int gby = fby * 8 + (tid >> 3), gbx = fbx * 8 + (tid & 7);
            const bool in = gby * 8 < H && gbx * 8 < W;
            const int m = F.map_start + gby * (W >> 3) + gbx;
            sm.dir[tid] = in ? mdir[m] : 0;
            sm.var[tid] = in ? mvar[m] : 0;
        } else {
            int best = 0, bc = sm.cost[tid][0];
#pragma unroll
            for (int k = 1; k < 8; k++)
                if (sm.cost[tid][k] > bc) { bc = sm.cost[tid][k]; best = k; }
            sm.dir[tid] = (uint8_t)best;
            sm.var[tid] = bc - sm.cost[tid][(best + 4) & 7];
        }
        sm.acc[tid] = 0;
        sm.accu[tid] = 0;
        if (tid < 8) sm.acc14c[tid] = 0;
        if (tid < 2) sm.base[tid] = 0;
    }
    __syncthreads();

    // ---- strength tables (section 3.2)
    for (int e = tid; e < 64 * 16; e += kThreads) {
        const int k = e >> 4, p = e & 15;
        const int S = adjust_strength(p, sm.var[k]);
        const int lp = S ? ilog2(S) : 0;
        const int Deff = (S && D < lp) ? lp : D;
        sm.pset[k][p] = make_set(S << sh8, S ? Deff - lp : 0);
    }
    int cflag = 0;
    if (tid < 64) {
        uint32_t bits = 0;
        for (int p = 0; p < 16; p++) {
            const int S = adjust_strength(p, sm.var[tid]);
            bits |= (uint32_t)(S & 1) << p;
        }
        if (kCoded) {   // the (19, 7) preset of this 8x8 block (section 4)
            const Eff e = make_eff(19, 7, D, false, sm.var[tid], sh8);
            sm.pset[tid][16] = make_set(e.pri, e.psh);
            sm.s7[tid] = make_set(e.sec, e.ssh);
            bits |= (uint32_t)(e.w0 == 3) << 16;
            const int gby = fby * 8 + (tid >> 3), gbx = fbx * 8 + (tid & 7);
            if (gby * 8 < H && gbx * 8 < W) cflag = F.coded[gby * (W >> 3) + gbx] != 0;
            sm.coded[tid] = (uint8_t)cflag;
        }
        sm.pbits[tid] = bits;
    } else if (tid < 80) {
        const int p = tid - 64, Dc = D - 1, lp = p ? ilog2(p) : 0;
        const int Deff = (p && Dc < lp) ? lp : Dc;
        sm.cset[p] = make_set(p << sh8, p ? Deff - lp : 0);
    } else if (tid < 92) {
        const int g = (tid - 80) >> 2, si = (tid - 80) & 3, s = sec_value(si);
        const int Dg = g == 0 ? D : g == 1 ? D - 1 : 3;
        sm.sset[g][si] = make_set(s << sh8, s ? Dg - ilog2(s) : 0);
    } else if (tid == 92) {
        uint32_t bits = 0, raised = 0;
        for (int p = 0; p < 16; p++) {
            bits |= (uint32_t)(p & 1) << p;
            if (p && ilog2(p) > D - 1) raised |= 1u << p;
        }
        if (kCoded) {
            const Eff e = make_eff(19, 7, D, true, 0, sh8);
            sm.cset[16] = make_set(e.pri, e.psh);
            sm.s7c = make_set(e.sec, e.ssh);
            bits |= (uint32_t)(e.w0 == 3) << 16;
        }
        sm.cbits = bits;
        sm.craised = raised;
    }
    // section 4: a filter block without coded residual is never filtered
    const bool any_coded = kCoded ? __syncthreads_or(cflag) != 0 : (__syncthreads(), true);
    if (kCoded && grp == 0 && tid == 0) skipped[blk_global] = (uint8_t)!any_coded;

    // ---- both plane groups through one code path: task 0 luma, task 1 chroma
    const int bw = W >> 3;
    // eq. 14: the unit is the whole block and its candidate groups are
    // evaluated in turn on the same staged tiles, directions and tables.
    // Luma keeps one sum of each kind per candidate (the two samples of a
    // word are in one 8x8 block), chroma one per candidate and plane, so a
    // luma group holds twice the candidates of a chroma group: the luma
    // groups' shared work (tap loads, clip range, secondary sums) is done
    // half as often.
    constexpr int kPPl = (kEq14 && 2 * kPP <= 16) ? 2 * kPP : kPP;   // luma primaries per group
    constexpr int kGl = 16 / kPPl;                                     // luma groups
    {
        // task 0 luma, task 1 chroma, a copy of the body each (the plane
        // group's choices fixed at compile time; eq. 14 sums the luma lanes
        // in one dot product); g: the candidate group (eq. 14)
        auto task_body = [&](auto luma_c, const int g) {
            constexpr bool kL = decltype(luma_c)::value;
            const bool luma = kL;
            const int task = luma ? 0 : 1;
            constexpr int kPPt = kL ? kPPl : kPP;   // primaries of this task's group
            constexpr int kNt = 4 * kPPt;           // candidates of this task's group
            const int p0 = kEq14 ? g * kPPt : p0_unit;
            const int bx = lane >> 2, sub = lane & 3;
            const int blk = warp * 8 + bx;
            const int gby = fby * 8 + warp, gbx = fbx * 8 + bx;
            const bool inside = luma ? (gby * 8 < H && gbx * 8 < W) : (gby * 4 < CH && gbx * 4 < CW);
            const bool edge = gby == 0 || gbx == 0 || gby == (H >> 3) - 1 || gbx == bw - 1;
            const bool any_edge = __any_sync(0xffffffffu, inside && edge);
            const int rows = luma ? 8 : 4;
            const int pitch = luma ? kLumaPitch : kChromaPitch;
            const uint32_t *base = luma ? sm.t.le + (2 + warp * 8) * kLumaPitch + 4 + bx * 4 + sub
                                        : sm.t.cw + (2 + warp * 4) * kChromaPitch + 2 + bx * 4 + sub;
            // the re-laid tile the taps read (luma: even and odd copies)
            const uint32_t *tile0 = luma ? sm.t.le : sm.t.cw;
            const int tile_words = luma ? 2 * kLumaRows * kLumaPitch : kChromaRows * kChromaPitch;
            (void)tile0;
            (void)tile_words;
            const int4 *op = reinterpret_cast<const int4 *>(sm.off[task][sm.dir[blk]]);
            const int4 o0 = op[0], o1 = op[1], o2 = op[2];
            const int o[12] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w, o2.x, o2.y, o2.z, o2.w};
            // the parameters: luma's, or the chroma planes' (4:2:0 chroma, or
            // a 4:4:4 chroma plane in the luma layout); ptask: the table
            const bool lp = luma && !cparams;
            const int ptask = lp ? 0 : 1;
            const SetC *ps = lp ? sm.pset[blk] : sm.cset;
            const uint32_t bits = lp ? sm.pbits[blk] : sm.cbits;
            const uint32_t raised = lp ? 0u : sm.craised;
            // eq. 14: the secondary sums of the thread's words are formed in
            // the task's first candidate group and kept for the others: luma
            // S_s = 1, 2 in the block's tile buffer (idle once the tiles are
            // re-laid, until the next block's loads are issued) and S_s = 4
            // in qc; chroma all three in qc and those at the raised damping
            // in the tile buffer
            static_assert(sizeof(RawTiles) >= 2 * 8 * kThreads * 4 && kThreads == 256, "cache size");
            uint32_t *const idle = reinterpret_cast<uint32_t *>(&raw);
            auto qslot = [&](int s, int i) -> uint32_t & {
                if (kL) return s < 3 ? idle[((s - 1) * 8 + i) * kThreads + tid] : sm.qc[i * kThreads + tid];
                return sm.qc[((s - 1) * 4 + i) * kThreads + tid];
            };
            // (4:2:0 chroma only: rows i < 4)
            auto rslot = [&](int s, int i) -> uint32_t & { return idle[((s - 1) * 4 + i) * kThreads + tid]; };
            const SetC *ss = lp ? sm.sset[0] : sm.sset[1];
            SetC s7 = {};
            if (kCoded) s7 = lp ? sm.s7[blk] : sm.s7c;
            const int oy = luma ? ly0 + warp * 8 : cy0 + warp * 4;
            const int ox = luma ? lx0 + bx * 8 + 2 * sub : cx0 + bx * 4 + sub;
            const uint8_t *sa = luma ? (kPl ? F.src[plane] : F.src[0]) : F.src[1];
            const int64_t spa = luma ? (kPl ? F.src_pitch[plane] : F.src_pitch[0]) : F.src_pitch[1];

            // section 5's low-complexity search: primaries with no allowed pair
            // are not evaluated, entries of pairs outside the subset are 0
            uint32_t pmask = 0xffffu;
            if (kSub) {
                const unsigned long long pairs = allowed_pairs(F, ptask);
                pmask = 0;
    #pragma unroll
                for (int p = 0; p < 16; p++) pmask |= (uint32_t)(((pairs >> (4 * p)) & 15ull) != 0) << p;
            }

            uint32_t acc[kEq14 ? 1 : kN], sse0 = 0;
    #pragma unroll
            for (int q = 0; q < (kEq14 ? 1 : kN); q++) acc[q] = 0;
            // eq. 14: per candidate and sample lane the sums of r, r (2x + r),
            // r (2 (x - s) + r); then per lane x, x^2, s, s^2, (x - s)^2
            constexpr int kE = kEq14 ? kNt : 1;
            int e6[kE][6], e0[10];
    #pragma unroll
            for (int q = 0; q < kE; q++)
    #pragma unroll
                for (int j = 0; j < 6; j++) e6[q][j] = 0;
    #pragma unroll
            for (int j = 0; j < 10; j++) e0[j] = 0;
            if (inside) {
    #pragma unroll 1
                for (int i = 0; i < rows; i++) {
                    const uint32_t *b = base + i * pitch;
                    const uint32_t X = b[0];
                    uint32_t v[12];
    #pragma unroll
                    for (int k = 0; k < 12; k++)
                        v[k] = CDEF_IN_BOUNDS(b + o[k] - tile0, tile_words, status) ? b[o[k]] : X;
                    if (any_edge) {
    #pragma unroll
                        for (int k = 0; k < 12; k++) v[k] = in_frame(v[k], X);
                    }
                    uint32_t mn = X, mx = X;
    #pragma unroll
                    for (int k = 0; k < 12; k += 2) {
                        mn = __vimin3_u16x2(mn, v[k], v[k + 1]);
                        mx = __vimax3_u16x2(mx, v[k], v[k + 1]);
                    }
                    const uint32_t S = luma ? load_src_pair<T>(sa + (int64_t)(oy + i) * spa, ox)
                                            : load_src_uv<T>(sa + (int64_t)(oy + i) * spa,
                                                             F.src[2] + (int64_t)(oy + i) * F.src_pitch[2], ox);
                    // Squared error of one candidate, with e = y - s = (x - s) + r:
                    // e^2 = (x - s)^2 + r (2 (x - s) + r).  The first term does not
                    // depend on the candidate and is summed once per pixel; the
                    // second is formed from the candidate's correction r, which
                    // at 8 and 10 bits stays within a signed byte (|r| <= 57).
                    sse0 = add_sq<T>(sse0, X, S);
                    const uint32_t two_xs = sadd16(2u * (X + 4096u * kLanes - S), 0xdf00u * kLanes);
                    if (kEq14 && g == 0) {
                        const int xl = (int)(X & 0xffffu) - (int)kBias, xh = (int)(X >> 16) - (int)kBias;
                        const int sl = (int)(S & 0xffffu) - (int)kBias, sh = (int)(S >> 16) - (int)kBias;
                        e0[0] += xl; e0[1] += xh;
                        e0[2] += xl * xl; e0[3] += xh * xh;
                        e0[4] += sl; e0[5] += sh;
                        e0[6] += sl * sl; e0[7] += sh * sh;
                        e0[8] += (xl - sl) * (xl - sl); e0[9] += (xh - sh) * (xh - sh);
                    }
                    const uint32_t rlo = __vmaxu2(mn - X + 2048u * kLanes, 1792u * kLanes) - 1792u * kLanes;
                    const uint32_t rhi = mx - X + 256u * kLanes;
                    uint32_t Q[4], Qr[4];
                    Q[0] = Qr[0] = 12u * X;
                    if (!kEq14 || g == 0) {
    #pragma unroll
                        for (int s = 1; s < 4; s++) Q[s] = sec_sum(v, X, ss[s]);
                        if (kEq14) {
    #pragma unroll
                            for (int s = 1; s < 4; s++) qslot(s, i) = Q[s];
                        }
                    } else {
    #pragma unroll
                        for (int s = 1; s < 4; s++) Q[s] = qslot(s, i);
                    }
                    if (raised) {
                        // kept for 4:2:0 chroma (4 rows); a 4:4:4 chroma plane in
                        // the luma layout (8 rows) forms them in every group
                        if (!kEq14 || g == 0 || kL) {
    #pragma unroll
                            for (int s = 1; s < 4; s++) Qr[s] = sec_sum(v, X, sm.sset[2][s]);
                            if (kEq14 && !kL) {
    #pragma unroll
                                for (int s = 1; s < 4; s++) rslot(s, i) = Qr[s];
                            }
                        } else {
    #pragma unroll
                            for (int s = 1; s < 4; s++) Qr[s] = rslot(s, i);
                        }
                    } else {
    #pragma unroll
                        for (int s = 1; s < 4; s++) Qr[s] = Q[s];
                    }
                    const uint32_t C = 4096u * kLanes - 24u * X;
    #pragma unroll
                    for (int pp = 0; pp < kPPt; pp++) {
                        const int p = p0 + pp;
                        if (kSub && !((pmask >> p) & 1)) continue;
                        const SetC sc = ps[p];
                        const uint32_t T0 = pri_sum(v, X, sc, (bits >> p) & 1) + C;
                        const bool rz = (raised >> p) & 1;
                        const bool slot19 = kCoded && p == 0;   // (0, 0) slot: the (19, 7) preset
                        uint32_t u19 = 0;
                        if (slot19)
                            u19 = pri_sum(v, X, ps[16], (bits >> 16) & 1) + C + sec_sum(v, X, s7);
    #pragma unroll
                        for (int s = 0; s < 4; s++) {
                            // eq. 8 rounding of (P + Q - 24x) / 16, ties away from zero
                            const uint32_t u = (slot19 && s == 0) ? u19 : T0 + (rz ? Qr[s] : Q[s]);
                            const uint32_t pos = (u >> 12) & kLanes;
                            const uint32_t w = u + pos + 7u * kLanes;
                            uint32_t rb = (w >> 4) & (0x0fffu * kLanes);   // r + 256 per lane
                            // eq. 9-12 on r: x + r is held in [min, max].  Where the
                            // adjusted primary strength is 0 only the secondary set
                            // contributes, its weights sum to 12/16 < 1, and the
                            // clip cannot bind: it is applied without a test.
                            if (s > 0 || slot19) rb = __vminu2(__vmaxu2(rb, rlo), rhi);
                            const uint32_t a = sadd16(rb, two_xs);           // 2 (x - s) + r
                            const uint32_t r8 = __byte_perm(rb, 0, 0x0020);  // r of both lanes, bytes 0, 1
                            if (kEq14) {
                                const int c = pp * 4 + s;
                                // sums of r, r (s + 128) (the source as staged) and
                                // r (2 (x - s) + r); r (2x + r) follows from the last
                                // two at the block (r (2 (x - s) + r) + 2 r s)
                                if (luma) {
                                    // both lanes in one 8x8 block: one sum
                                    e6[c][0] = __dp2a_lo((int)kLanes, (int)r8, e6[c][0]);
                                    e6[c][2] = __dp2a_lo((int)S, (int)r8, e6[c][2]);
                                    e6[c][4] = __dp2a_lo((int)a, (int)r8, e6[c][4]);
                                } else {
                                    // (U, V) lanes kept apart
                                    const int rl = (int)(r8 & 0xffu), rh = (int)(r8 & 0xff00u);
                                    e6[c][0] = __dp2a_lo((int)kLanes, rl, e6[c][0]);
                                    e6[c][1] = __dp2a_lo((int)kLanes, rh, e6[c][1]);
                                    e6[c][2] = __dp2a_lo((int)S, rl, e6[c][2]);
                                    e6[c][3] = __dp2a_lo((int)S, rh, e6[c][3]);
                                    e6[c][4] = __dp2a_lo((int)a, rl, e6[c][4]);
                                    e6[c][5] = __dp2a_lo((int)a, rh, e6[c][5]);
                                }
                            } else {
                                acc[pp * 4 + s] = (uint32_t)__dp2a_lo((int)a, (int)r8, (int)acc[pp * 4 + s]);
                            }
                        }
                    }
                }
            }
            if constexpr (kEq14) {
                if (luma) {
                    // the two samples of a word are neighbours in one 8x8 block:
                    // add the lanes, then the four lanes of the block
                    int n = inside ? 16 : 0, sx = e0[0] + e0[1], sx2 = e0[2] + e0[3];
                    int ssum = e0[4] + e0[5], ss2 = e0[6] + e0[7], sxs = e0[8] + e0[9];
                    int A[kNt], BX[kNt], BS[kNt];
    #pragma unroll
                    for (int c = 0; c < kNt; c++) {
                        A[c] = e6[c][0] + e6[c][1];
                        BX[c] = e6[c][2] + e6[c][3];
                        BS[c] = e6[c][4] + e6[c][5];
                    }
    #pragma unroll
                    for (int o = 1; o <= 2; o <<= 1) {
                        if (g == 0) {
                            n += __shfl_xor_sync(0xffffffffu, n, o);
                            sx += __shfl_xor_sync(0xffffffffu, sx, o);
                            sx2 += __shfl_xor_sync(0xffffffffu, sx2, o);
                            ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
                            ss2 += __shfl_xor_sync(0xffffffffu, ss2, o);
                            sxs += __shfl_xor_sync(0xffffffffu, sxs, o);
                        }
    #pragma unroll
                        for (int c = 0; c < kNt; c++) {
                            A[c] += __shfl_xor_sync(0xffffffffu, A[c], o);
                            BX[c] += __shfl_xor_sync(0xffffffffu, BX[c], o);
                            BS[c] += __shfl_xor_sync(0xffffffffu, BS[c], o);
                        }
                    }
                    // r (2x + r) = r (2 (x - s) + r) + 2 r s, from the sum of
                    // r (s + 128)
    #pragma unroll
                    for (int c = 0; c < kNt; c++) BX[c] = BS[c] + 2 * (BX[c] - (int)kBias * A[c]);
                    // the candidate-free sums of the block: formed in the first
                    // group (the four lanes agree after the butterfly), kept
                    if (g == 0) {
                        if (sub == 0) {
                            int *k6 = sm.e14l[blk];
                            k6[0] = n, k6[1] = sx, k6[2] = sx2, k6[3] = ssum, k6[4] = ss2, k6[5] = sxs;
                        }
                    } else {
                        const int *k6 = sm.e14l[blk];
                        n = k6[0], sx = k6[1], sx2 = k6[2], ssum = k6[3], ss2 = k6[4], sxs = k6[5];
                    }
                    // each of the block's four lanes evaluates a quarter of the
                    // candidates; the eight blocks' values are summed across
                    // the warp before one shared atomic per candidate
                    constexpr int kC = kNt / 4;
                    long long tv[kC];
    #pragma unroll
                    for (int j = 0; j < kC; j++) tv[j] = 0;
    #pragma unroll
                    for (int c = 0; c < kNt; c++) {
                        if (n > 0 && (c * 4) / kNt == sub)
                            tv[c % kC] = eq14_value(n, ssum, ss2, sx + A[c], (long long)sx2 + BX[c],
                                                    (long long)sxs + BS[c], F.bitdepth);
                    }
    #pragma unroll
                    for (int o = 4; o <= 16; o <<= 1)
    #pragma unroll
                        for (int j = 0; j < kC; j++) tv[j] += __shfl_xor_sync(0xffffffffu, tv[j], o);
                    if (bx == 0)
    #pragma unroll
                        for (int j = 0; j < kC; j++)
                            atomicAdd(&sm.acc[sub * kC + j], (unsigned long long)tv[j]);
                } else {
                    // (U, V) lanes: per plane, the 4-row half of a chroma 8x8
                    // block is eight lanes (two 4x4 blocks) of this warp; the
                    // other half is the next warp's
                    const int cb = (warp >> 1) * 4 + (bx >> 1), half = warp & 1;
    #pragma unroll
                    for (int k = 0; k < 2; k++) {
                        int vals[30];
    #pragma unroll
                        for (int c = 0; c < kNt; c++) {
                            vals[3 * c] = e6[c][k];
                            vals[3 * c + 1] = e6[c][2 + k];
                            vals[3 * c + 2] = e6[c][4 + k];
                        }
                        // the candidate-free sums: from the first group, kept
                        vals[24] = inside ? 4 : 0;
                        vals[25] = e0[k];
                        vals[26] = e0[2 + k];
                        vals[27] = e0[4 + k];
                        vals[28] = e0[6 + k];
                        vals[29] = e0[8 + k];
    #pragma unroll
                        for (int o = 1; o <= 4; o <<= 1)
    #pragma unroll
                            for (int j = 0; j < 30; j++)
                                if (j < 24 || g == 0) vals[j] += __shfl_xor_sync(0xffffffffu, vals[j], o);
                        if ((lane & 7) == 0)
    #pragma unroll
                            for (int j = 0; j < 30; j++)
                                if (j < 24 || g == 0) sm.e14h[k][cb][half][j] = vals[j];
                    }
                }
                __syncthreads();
            } else {
                // the warp totals of r (2 (x - s) + r) are signed and fit 32 bits
                if (!kCoded) {
                    butterfly<kN>(acc, lane);
                    if (kN == 64) {
                        atomicAdd(&sm.acc[2 * lane], (unsigned long long)(long long)(int)acc[0]);
                        atomicAdd(&sm.acc[2 * lane + 1], (unsigned long long)(long long)(int)acc[1]);
                    } else if (kN == 32) {
                        atomicAdd(&sm.acc[lane], (unsigned long long)(long long)(int)acc[0]);
                    } else if (!(lane & 1)) {
                        atomicAdd(&sm.acc[lane >> 1], (unsigned long long)(long long)(int)acc[0]);
                    }
                } else {
                    // the four lanes of one 8x8 block first, then the uncoded blocks'
                    // part is split off and both are summed across the warp
                    wreduce<kN, 0, 2>(acc, lane);
                    constexpr int kQ = kN / 4;
                    uint32_t un[kQ];
                    const bool unc = !sm.coded[blk];
        #pragma unroll
                    for (int i = 0; i < kQ; i++) un[i] = unc ? acc[i] : 0u;
                    wreduce<kN, 2, 5>(acc, lane);
                    wreduce<kN, 2, 5>(un, lane);
                    const int e = wentry(kN, lane);
                    if (kN >= 32 || !(lane & 16)) {
        #pragma unroll
                        for (int j = 0; j < (kN >= 64 ? 2 : 1); j++) {
                            atomicAdd(&sm.acc[e + j], (unsigned long long)(long long)(int)acc[j]);
                            atomicAdd(&sm.accu[e + j], (unsigned long long)(long long)(int)un[j]);
                        }
                    }
                }
        #pragma unroll
                for (int o = 16; o >= 1; o >>= 1) sse0 += __shfl_xor_sync(0xffffffffu, sse0, o);
                if (lane == 0) atomicAdd(&sm.base[task], (unsigned long long)sse0);
                __syncthreads();
                if (tid < kN) {
                    const long long base_sse = (long long)sm.base[task];
                    const bool on = (allowed_pairs(F, ptask) >> (4 * p0 + tid)) & 1;
                    // a 4:4:4 chroma plane's entries are added into the zeroed
                    // chroma table (U and V): every entry is linear in the
                    // plane's sums
                    auto put = [&](long long *p, long long v) {
                        if (kPl && cparams) {
                            if (v) atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
                        } else {
                            *p = v;
                        }
                    };
                    if (!kCoded) {
                        long long *out = (lp ? dist_luma : dist_chroma) + (int64_t)blk_global * 64 + 4 * p0;
                        put(&out[tid], on ? (long long)sm.acc[tid] + base_sse : 0);
                    } else {
                        // q = k * 64 + p * 4 + s; skip bit clear: blocks without coded
                        // residual unfiltered, (0, 0) the unfiltered error
                        long long *out = (lp ? dist_luma : dist_chroma) + (int64_t)blk_global * 128 +
                                         4 * p0 + tid;
                        const long long tot = (long long)sm.acc[tid], un = (long long)sm.accu[tid];
                        put(&out[0], !on ? 0 : (!any_coded || (p0 == 0 && tid == 0)) ? base_sse : base_sse + tot - un);
                        put(&out[64], !on ? 0 : !any_coded ? base_sse : base_sse + tot);
                    }
                    sm.acc[tid] = 0;
                    sm.accu[tid] = 0;
                }
                __syncthreads();
            }
        };
        if constexpr (!kEq14) {
            task_body(std::true_type{}, 0);
            if (!kPl) task_body(std::false_type{}, 0);
        } else {
            // eq. 14: the luma groups, then the chroma groups (each task's
            // secondary sums are formed in its first group and kept)
#pragma unroll 1
            for (int g = 0; g < kGl; g++) {
                task_body(std::true_type{}, g);
                if (tid < 4 * kPPl) {   // the group's luma-layout candidates
                    const int q = 4 * kPPl * g + tid;
                    const bool on = (allowed_pairs(F, cparams ? 1 : 0) >> q) & 1;
                    if (kPl && cparams) {   // a 4:4:4 chroma plane: into the zeroed chroma table
                        if (on)
                            atomicAdd(reinterpret_cast<unsigned long long *>(
                                          &dist_chroma[(int64_t)blk_global * 64 + q]), sm.acc[tid]);
                    } else {
                        dist_luma[(int64_t)blk_global * 64 + q] = on ? (long long)sm.acc[tid] : 0;
                    }
                    sm.acc[tid] = 0;
                }
                __syncthreads();
            }
#pragma unroll 1
            for (int g = 0; g < (kPl ? 0 : kG); g++) {
                task_body(std::false_type{}, g);
                // chroma 8x8 blocks: two planes x 16 blocks x the group's
                // candidates, one per thread; lanes 8 apart hold the same
                // candidate
                static_assert(2 * 16 * kN == kThreads, "one chroma evaluation per thread");
                {
                    const int k = tid / (16 * kN), cb = (tid / kN) % 16, c = tid % kN;
                    const int *h0 = sm.e14h[k][cb][0], *h1 = sm.e14h[k][cb][1];
                    const int n = h0[24] + h1[24];
                    long long t = 0;
                    if (n > 0) {
                        const long long sx = h0[25] + h1[25], sx2 = h0[26] + h1[26];
                        const long long ssum = h0[27] + h1[27], ss2 = h0[28] + h1[28], sxs = h0[29] + h1[29];
                        const long long ra = h0[3 * c] + h1[3 * c];
                        const long long rs = h0[3 * c + 1] + h1[3 * c + 1];   // r (s + 128)
                        const long long rq = h0[3 * c + 2] + h1[3 * c + 2];   // r (2 (x - s) + r)
                        t = eq14_value(n, ssum, ss2, sx + ra, sx2 + rq + 2 * (rs - (long long)kBias * ra),
                                       sxs + rq, F.bitdepth);
                    }
                    t += __shfl_xor_sync(0xffffffffu, t, 8);
                    t += __shfl_xor_sync(0xffffffffu, t, 16);
                    if (lane < kN) atomicAdd(&sm.acc14c[c], (unsigned long long)t);
                }
                __syncthreads();
                if (tid < kN) {
                    const int q = 4 * kPP * g + tid;
                    const bool on = (allowed_pairs(F, 1) >> q) & 1;
                    dist_chroma[(int64_t)blk_global * 64 + q] = on ? (long long)sm.acc14c[tid] : 0;
                    sm.acc14c[tid] = 0;
                }
                __syncthreads();
            }
        }
    }
}

struct SBlockRef {
    int fi, fby, fbx;
};

__device__ __forceinline__ SBlockRef slocate(const SearchBatch &batch, int blk)
{
    int fi = 0;
    while (fi + 1 < batch.n && blk >= batch.f[fi + 1].block_start) fi++;
    const int local = blk - batch.f[fi].block_start;
    const int fby = local / batch.f[fi].fb_cols;
    return {fi, fby + batch.f[fi].fb_row0, local - fby * batch.f[fi].fb_cols};
}

// The tile loads of filter block `blk` (plane < 0: its luma and 4:2:0 chroma
// tiles; else the one plane, whose map has the luma box).
__device__ __forceinline__ void sissue(const SearchBatch &batch, int blk, RawTiles &raw, uint64_t *bar,
                                       int plane = -1)
{
    const SBlockRef r = slocate(batch, blk);
    const SearchFrameDev &F = batch.f[r.fi];
    if (plane < 0)
        issue_tile_loads(F.tmap, F.bitdepth, r.fby, r.fbx, raw, bar, true, batch.waits.extra_tx);
    else
        issue_tile_loads(&F.tmap[plane], F.bitdepth, r.fby, r.fbx, raw, bar, false, batch.waits.extra_tx);
}

// Persistent distortion kernel (same work-counter scheme as the filter).
// Work unit u is filter block u / kG, primary-strength group u % kG.
template <int kG, bool kCoded, bool kEq14, bool kSub, bool kPl = false>
__global__ void __launch_bounds__(kThreads, kMinCtas)
dist_kernel(const __grid_constant__ SearchBatch batch, long long *dist_luma, long long *dist_chroma,
            uint8_t *skipped, int *status, unsigned *work, const uint8_t *mdir, const int32_t *mvar)
{
    extern __shared__ __align__(128) uint8_t smem_bytes[];
    SearchSmem &sm = *reinterpret_cast<SearchSmem *>(smem_bytes);
    const int tid = threadIdx.x;
    // work units per filter block: its primary-strength groups, or (kPl) its
    // three planes
    constexpr int kUnits = kPl ? 3 : kEq14 ? 1 : kG;
    const int total = batch.total_blocks * kUnits;

    if (smem_u32(smem_bytes) & 127) {
        if (tid == 0) atomicOr(status, kStatusMisaligned);
    } else {
        if (tid == 0) {
            mbar_init(&sm.bar[0], 1);
            mbar_init(&sm.bar[1], 1);
            const int b = (int)atomicAdd(&work[0], 1u);
            sm.blk[0] = b;
            if (b < total) sissue(batch, b / kUnits, sm.raw[0], &sm.bar[0], kPl ? b % kUnits : -1);
        }
        if (tid < 192) {
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
                if (nb < total)
                    sissue(batch, nb / kUnits, sm.raw[buf ^ 1], &sm.bar[buf ^ 1], kPl ? nb % kUnits : -1);
            }
            const bool arrived = mbar_wait_bounded(&sm.bar[buf], (it >> 1) & 1, batch.waits.wait_cycles);
            if (__syncthreads_or(!arrived)) {
                // leave once both buffers' loads in flight have landed
                if (tid == 0) {
                    atomicOr(status, kStatusTimeout);
                    drain_tile_loads(&sm.bar[buf], (it >> 1) & 1, batch.waits.extra_tx);
                    if (sm.blk[buf ^ 1] < total)
                        drain_tile_loads(&sm.bar[buf ^ 1], ((it + 1) >> 1) & 1, batch.waits.extra_tx);
                }
                break;
            }
            const int fb = blk / kUnits, grp = blk - fb * kUnits;
            const SBlockRef r = slocate(batch, fb);
            const SearchFrameDev &F = batch.f[r.fi];
            if (F.bitdepth == 8)
                dist_block<uint8_t, kG, kCoded, kEq14, kSub, kPl>(F, r.fby, r.fbx, fb, grp, sm,
                                                                  sm.raw[buf], dist_luma, dist_chroma,
                                                                  skipped, mdir, mvar CDEF_DEBUG_ARG(status));
            else
                dist_block<uint16_t, kG, kCoded, kEq14, kSub, kPl>(F, r.fby, r.fbx, fb, grp, sm,
                                                                   sm.raw[buf], dist_luma, dist_chroma,
                                                                   skipped, mdir, mvar CDEF_DEBUG_ARG(status));
            __syncthreads();
        }
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&work[1], 1u) == gridDim.x - 1) {
            work[0] = 0;
            work[1] = 0;
            __threadfence();
        }
    }
}

constexpr size_t kSmemBytes = sizeof(SearchSmem);

// Persistent grid: `per_sm` CTAs on every SM (at most what fits), never more
// CTAs than work units.
template <int kG, bool kCoded, bool kEq14, bool kSub, bool kPl = false>
int dist_grid(int units, int per_sm)
{
    static int cached_dev = -1, cached_sms = 0, cached_occ = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        auto *kern = dist_kernel<kG, kCoded, kEq14, kSub, kPl>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        int sms = 0, occ = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, kSmemBytes);
        cached_sms = sms;
        cached_occ = occ > 0 ? occ : 1;
        cached_dev = dev;
    }
    const int ctas = cached_sms * (per_sm < cached_occ ? per_sm : cached_occ);
    return units < ctas ? units : ctas;
}

template <int kG, bool kCoded, bool kEq14, bool kSub, bool kPl = false>
void launch_dist_kernel(const SearchBatch &b, long long *dl, long long *dc, uint8_t *skipped,
                        int *status, unsigned *work, int units, int per_sm, cudaStream_t s,
                        const uint8_t *mdir = nullptr, const int32_t *mvar = nullptr)
{
    dist_kernel<kG, kCoded, kEq14, kSub, kPl><<<dist_grid<kG, kCoded, kEq14, kSub, kPl>(units, per_sm),
                                                kThreads, kSmemBytes, s>>>(b, dl, dc, skipped, status,
                                                                           work, mdir, mvar);
}

// Whether the call searches a subset of the pairs (the same for every frame).
bool subset_search(const SearchBatch &b)
{
    return (allowed_pairs(b.f[0], 0) & allowed_pairs(b.f[0], 1)) != ~0ull;
}

template <int kG>
cudaError_t launch_dist(const SearchBatch &b, long long *dl, long long *dc, uint8_t *skipped,
                        int *status, unsigned *work, int per_sm, cudaStream_t s)
{
    const int units = b.total_blocks * kG;
    const bool sub = subset_search(b);
    if (skipped) {
        if (sub) launch_dist_kernel<kG, true, false, true>(b, dl, dc, skipped, status, work, units, per_sm, s);
        else launch_dist_kernel<kG, true, false, false>(b, dl, dc, skipped, status, work, units, per_sm, s);
    } else {
        if (sub) launch_dist_kernel<kG, false, false, true>(b, dl, dc, nullptr, status, work, units, per_sm, s);
        else launch_dist_kernel<kG, false, false, false>(b, dl, dc, nullptr, status, work, units, per_sm, s);
    }
    return cudaGetLastError();
}

// 8/10-bit 4:4:4 squared-error tables: one work unit per filter block and
// plane, the planes in the luma layout; the chroma table is zeroed first
// (U and V add into it) and the direction maps are formed first.
cudaError_t launch_dist_planes(const SearchBatch &b, uint8_t *dirs, int32_t *vars, long long *dl,
                               long long *dc, uint8_t *skipped, int *status, unsigned *work,
                               cudaStream_t s, bool eq14)
{
    for (int i = 0; i < b.n; i++) {
        const SearchFrameDev &F = b.f[i];
        const cudaError_t e = launch_find_dir(F.rec[0], F.rec_pitch[0], F.w, F.h, F.bitdepth,
                                              dirs + F.map_start, vars + F.map_start, s);
        if (e != cudaSuccess) return e;
    }
    const size_t width = skipped ? 128 : 64;
    cudaError_t e = cudaMemsetAsync(dc, 0, sizeof(long long) * width * (size_t)b.total_blocks, s);
    if (e != cudaSuccess) return e;
    const int units = b.total_blocks * 3;
    const bool sub = subset_search(b);
    if (eq14) {   // eq. 14 (64 pairs): the luma-layout groups of each plane
        if (sub) launch_dist_kernel<8, false, true, true, true>(b, dl, dc, nullptr, status, work, units, 2, s, dirs, vars);
        else launch_dist_kernel<8, false, true, false, true>(b, dl, dc, nullptr, status, work, units, 2, s, dirs, vars);
    } else if (skipped) {
        if (sub) launch_dist_kernel<1, true, false, true, true>(b, dl, dc, skipped, status, work, units, 2, s, dirs, vars);
        else launch_dist_kernel<1, true, false, false, true>(b, dl, dc, skipped, status, work, units, 2, s, dirs, vars);
    } else {
        if (sub) launch_dist_kernel<1, false, false, true, true>(b, dl, dc, nullptr, status, work, units, 2, s, dirs, vars);
        else launch_dist_kernel<1, false, false, false, true>(b, dl, dc, nullptr, status, work, units, 2, s, dirs, vars);
    }
    return cudaGetLastError();
}

// Eq. 14 tables: one work unit per filter block, its 64 candidates in eight
// groups of eight (two primary strengths).
cudaError_t launch_dist_eq14(const SearchBatch &b, long long *dl, long long *dc, int *status,
                             unsigned *work, cudaStream_t s)
{
    const int units = b.total_blocks;
    if (subset_search(b))
        launch_dist_kernel<8, false, true, true>(b, dl, dc, nullptr, status, work, units, 2, s);
    else
        launch_dist_kernel<8, false, true, false>(b, dl, dc, nullptr, status, work, units, 2, s);
    return cudaGetLastError();
}

}  // namespace

// The preset selection: the cluster-per-frame kernel when every frame's
// blocks fit its per-CTA state, else the grid-wide cooperative kernel.
// `sse`: the tables hold squared errors (not eq. 14).
static cudaError_t select_presets(const SearchBatch &b, const long long *dl, const long long *dc,
                                  unsigned long long *cur, unsigned long long *tot,
                                  SearchResultDev *results, uint8_t *block_ids, int *status,
                                  int refine_passes, int width, const uint8_t *skipped, bool sse,
                                  bool grid_presets, cudaStream_t s)
{
    if (!grid_presets && preset_cluster_fits(b)) {
        // 8-bit squared errors: a block's luma and chroma entries sum to at
        // most 3 x 4096 x 255^2 < 2^30
        bool narrow = sse;
        for (int i = 0; i < b.n; i++) narrow = narrow && b.f[i].bitdepth == 8;
        return launch_presets_cluster(b, dl, dc, results, block_ids, narrow, refine_passes, width,
                                      skipped, s);
    }
    void *ctl = tot + (size_t)b.n * width * width;
    return launch_presets(b, dl, dc, cur, tot, ctl, results, block_ids, status, refine_passes,
                          width, skipped, s);
}

// An event on the stream; inside a stream capture, an event record node of
// the graph.
static cudaError_t stage_mark(const cudaEvent_t *ev, int k, cudaStream_t s)
{
    if (!ev) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev[k], s, cudaEventRecordExternal)
                                                : cudaEventRecord(ev[k], s);
}

cudaError_t launch_search(const SearchBatch &b, long long *dist_luma, long long *dist_chroma,
                          unsigned long long *cur, unsigned long long *tot, SearchResultDev *results,
                          uint8_t *block_ids, int *status, unsigned *work, SearchTune tune,
                          int refine_passes, cudaStream_t s, uint8_t *skipped,
                          const cudaEvent_t *stage_events, uint8_t *wide_dirs,
                          int32_t *wide_vars, bool grid_presets, bool tables_only)
{
    cudaError_t e = stage_mark(stage_events, 0, s);
    if (e != cudaSuccess) return e;
    const int per_sm = tune.ctas_per_sm;
    if (wide_dirs && b.planes) {   // 8/10-bit 4:4:4 frames
        const bool eq14 = tune.groups == 8;   // the eq. 14 tables
        e = launch_dist_planes(b, wide_dirs, wide_vars, dist_luma, dist_chroma, skipped, status, work,
                               s, eq14);
        if (e == cudaSuccess) e = stage_mark(stage_events, 1, s);
        if (e != cudaSuccess || tables_only) return e;
        e = select_presets(b, dist_luma, dist_chroma, cur, tot, results, block_ids, status,
                           refine_passes, skipped ? 128 : 64, skipped, !eq14, grid_presets, s);
        return e == cudaSuccess ? stage_mark(stage_events, 2, s) : e;
    }
    if (wide_dirs) {   // 4:2:2, 4:4:4 or 12-bit frames
        const bool eq14 = tune.groups == 8;   // the eq. 14 tables
        e = launch_search_wide(b, wide_dirs, wide_vars, dist_luma, dist_chroma, skipped, s, eq14,
                               status);
        if (e == cudaSuccess) e = stage_mark(stage_events, 1, s);
        if (e != cudaSuccess || tables_only) return e;
        const int width = skipped ? 128 : 64;
        e = select_presets(b, dist_luma, dist_chroma, cur, tot, results, block_ids, status,
                           refine_passes, width, skipped, !eq14, grid_presets, s);
        return e == cudaSuccess ? stage_mark(stage_events, 2, s) : e;
    }
    if (tune.groups == 8) {   // eq. 14 tables
        e = launch_dist_eq14(b, dist_luma, dist_chroma, status, work, s);
        if (e == cudaSuccess) e = stage_mark(stage_events, 1, s);
        if (e != cudaSuccess || tables_only) return e;
        e = select_presets(b, dist_luma, dist_chroma, cur, tot, results, block_ids, status,
                           refine_passes, 64, nullptr, false, grid_presets, s);
        return e == cudaSuccess ? stage_mark(stage_events, 2, s) : e;
    }
    switch (tune.groups) {
    case 2: e = launch_dist<2>(b, dist_luma, dist_chroma, skipped, status, work, per_sm, s); break;
    case 4: e = launch_dist<4>(b, dist_luma, dist_chroma, skipped, status, work, per_sm, s); break;
    default: e = launch_dist<1>(b, dist_luma, dist_chroma, skipped, status, work, per_sm, s); break;
    }
    if (e == cudaSuccess) e = stage_mark(stage_events, 1, s);
    if (e != cudaSuccess || tables_only) return e;
    const int width = skipped ? 128 : 64;
    e = select_presets(b, dist_luma, dist_chroma, cur, tot, results, block_ids, status,
                       refine_passes, width, skipped, true, grid_presets, s);
    return e == cudaSuccess ? stage_mark(stage_events, 2, s) : e;
}

CDEF_FAULT_COUNTER(index_faults_search)

}  // namespace cdefgb
