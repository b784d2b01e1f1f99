/*
 * CPU oracle for the CDEF hot path (arXiv 1602.05975).
 *
 * TEST INFRASTRUCTURE ONLY -- see cdef_ref.h.  Plain C99, int64 arithmetic,
 * one loop per sum of the paper, no vectorisation, no factoring, no code
 * shared with the CUDA library.
 *
 * Where the paper is silent, garbled or at odds with itself, this file
 * follows one written reading, named R1..R16 at the point of use:
 *   R1  line geometry of Fig. 1 (figure missing)
 *   R2  bit-depth reduction for the search is an arithmetic right shift
 *   R3  eq. 13 with floor(log2 floor(v / 2^16)) read as 0 when v < 2^16
 *   R4  contrast adjustment and tap parity on the unscaled strength, then
 *       bit-depth scaling (section 3.2)
 *   R5  chroma damping D-1, raised to floor(log2 S_p) for the whole block
 *   R7  eq. 7, d < 0 branch read as the mirror of the d >= 0 branch
 *   R8  primary/secondary tap positions of Figs. 3/4 (figures missing)
 *   R9  weights in sixteenths: primary (near, far) = (4,2) even, (3,3) odd;
 *       secondary (near, far) = (2,1)
 *   R11 the clipping range includes the filtered pixel itself
 *   R12 taps outside the frame give f = 0 and are left out of the clip range
 *   R13 the secondary cross uses the found direction even when S_p = 0
 *   R15 one preset picks both the luma and the chroma pair of a block
 *   R16 greedy order and tie-breaks of the preset search
 *
 * Parity status: cdef_ref_line_number (R1) is pinned only through the counts
 * and cardinalities the paper prints and through geometric properties (the
 * angles, and the costs permuting under the block's symmetries); the
 * direction numbering beyond d = 0/1 is unpinned.  The tap positions (R8)
 * are pinned to R1's geometry and to the same symmetries by tests.  The
 * secondary weights and the sixteenths normalisation (R9) are pinned only
 * by section 3.2's statement that all the weights together exceed unity;
 * otherwise they are parity unpinned: their figure is missing.
 */
#include "cdef_ref.h"

#include <math.h>
#include <stdlib.h>

static int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

/* floor(log2 s) for s >= 1, by counting halvings. */
static int64_t floor_log2(int64_t s)
{
    int64_t l = 0;
    while (s > 1) {
        s /= 2;
        l++;
    }
    return l;
}

/* ------------------------------------------------------------------------ */
/* Section 2: direction search                                              */
/* ------------------------------------------------------------------------ */

/* R1.  Fig. 1 gives, for each of the 8 directions, the line number k of
 * every pixel of an 8x8 block; the figure is missing from the text.  The
 * reading: d = 0 is the 45-degree up-right diagonal and each next direction
 * turns clockwise by roughly 22.5 degrees, with the lines of the two
 * in-between slopes stepping one row every two columns (or one column every
 * two rows).  i is the row, j the column. */
int cdef_ref_line_number(int d, int i, int j)
{
    switch (d) {
    case 0: return i + j;              /*  45 deg, 15 lines */
    case 1: return i + j / 2;          /*  26.6 deg, 11 lines */
    case 2: return i;                  /*   0 deg (rows), 8 lines */
    case 3: return 3 + i - j / 2;      /* -26.6 deg, 11 lines */
    case 4: return 7 + i - j;          /* -45 deg, 15 lines */
    case 5: return 3 - i / 2 + j;      /* -63.4 deg, 11 lines */
    case 6: return j;                  /* -90 deg (columns), 8 lines */
    case 7: return i / 2 + j;          /*  63.4 deg, 11 lines */
    default: return -1;
    }
}

/* Algorithm 1, first half: line sums partial[d][L], their cardinalities
 * count[d][L], and s[d] = sum_L partial^2 * 840 / count (eq. 5 times 840,
 * section 2: 840 is the least common multiple of the cardinalities 1..8). */
void cdef_ref_direction_costs(const int32_t x[64], int64_t s[8])
{
    for (int d = 0; d < 8; d++) {
        int64_t partial[15] = {0};
        int64_t count[15] = {0};
        for (int i = 0; i < 8; i++) {
            for (int j = 0; j < 8; j++) {
                int L = cdef_ref_line_number(d, i, j);
                partial[L] += x[i * 8 + j];
                count[L] += 1;
            }
        }
        s[d] = 0;
        for (int L = 0; L < 15; L++) {
            if (count[L] > 0)
                s[d] += partial[L] * partial[L] * (840 / count[L]);
        }
    }
}

/* Algorithm 1 on raw samples.  Section 2: 8-bit values are centred by -128;
 * higher bit depths are downscaled to 8 bits first (R2: x >> (bd - 8)).
 * The best direction is the first strict maximum of s[d]; the contrast is
 * s[best] - s[(best + 4) mod 8]. */
int cdef_ref_find_dir_block(const uint16_t *p, ptrdiff_t stride, int bitdepth,
                            int64_t *contrast)
{
    int32_t x[64];
    int64_t s[8];
    for (int i = 0; i < 8; i++)
        for (int j = 0; j < 8; j++)
            x[i * 8 + j] = (int32_t)(p[i * stride + j] >> (bitdepth - 8)) - 128;
    cdef_ref_direction_costs(x, s);
    int best = 0;
    for (int d = 0; d < 8; d++)
        if (s[d] > s[best])
            best = d;
    if (contrast)
        *contrast = s[best] - s[(best + 4) % 8];
    return best;
}

int cdef_ref_find_dir(const uint16_t *luma, int w, int h, ptrdiff_t stride,
                      int bitdepth, uint8_t *dir, int32_t *var)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8)
        return -1;
    if (bitdepth < 8 || bitdepth > 12)
        return -1;
    int bw = w / 8, bh = h / 8;
    for (int by = 0; by < bh; by++) {
        for (int bx = 0; bx < bw; bx++) {
            int64_t v = 0;
            int d = cdef_ref_find_dir_block(luma + (ptrdiff_t)by * 8 * stride + bx * 8,
                                            stride, bitdepth, &v);
            dir[by * bw + bx] = (uint8_t)d;
            var[by * bw + bx] = (int32_t)v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 3: the constrained non-linear filter                             */
/* ------------------------------------------------------------------------ */

/* Eq. 7.  For d >= 0: min(d, max(0, S - floor(d / 2^(D - floor(log2 S))))).
 * R7: the printed d < 0 branch uses a ceiling, which would break the stated
 * anti-symmetry around d = 0; the reading is f(-d) = -f(d).  S = 0 gives 0
 * (the filter tap is switched off and log2 0 is never taken). */
int64_t cdef_ref_constrain(int64_t diff, int64_t strength, int64_t damping)
{
    if (strength == 0)
        return 0;
    int64_t shift = damping - floor_log2(strength);
    if (shift < 0)
        return 0; /* excluded by D >= floor(log2 S); never reached */
    int64_t scale = (int64_t)1 << shift;
    if (diff >= 0)
        return min64(diff, max64(0, strength - diff / scale));
    return -min64(-diff, max64(0, strength - (-diff) / scale));
}

/* Eq. 13.  R3: for 2^10 <= v < 2^16 the term floor(log2 floor(v/2^16)) is
 * log2 of zero; it is read as 0, so that the factor (4 + i) / 16 runs from
 * 4/16 up to 16/16 as the contrast grows. */
int cdef_ref_adjust_strength(int strength, int64_t contrast)
{
    if (contrast < 1024)
        return 0;
    int64_t q = contrast / 65536;
    int64_t i = q > 0 ? min64(floor_log2(q), 12) : 0;
    return (int)((strength * (4 + i) + 8) / 16);
}

/* Eq. 8: round(sum / 16) with ties away from zero (R9: the weights are in
 * sixteenths). */
int64_t cdef_ref_round16(int64_t sum)
{
    if (sum >= 0)
        return (sum + 8) / 16;
    return -((-sum + 8) / 16);
}

/* Section 3.2 per 8x8 block.
 *  - luma S_p is adjusted by eq. 13 (chroma S_p is not);
 *  - R4: the primary weights follow the parity of that unscaled value, and
 *    both strengths are then scaled by 2^(bd-8), the damping offset by bd-8;
 *  - R5: chroma damping is the luma damping minus one, and a damping below
 *    floor(log2 S_p) is raised to it (worked example: chroma S_p = 15 with
 *    luma D = 3 gives chroma D = 3). */
void cdef_ref_block_params(int pri_raw, int sec_raw, int damping_luma,
                           int is_chroma, int bitdepth, int64_t contrast,
                           cdef_ref_eff_params *out)
{
    int pri = is_chroma ? pri_raw : cdef_ref_adjust_strength(pri_raw, contrast);
    int64_t damping = is_chroma ? damping_luma - 1 : damping_luma;
    if (pri > 0 && damping < floor_log2(pri))
        damping = floor_log2(pri);
    int shift8 = bitdepth - 8;
    out->parity = pri & 1;
    out->pri = (int64_t)pri << shift8;
    out->sec = (int64_t)sec_raw << shift8;
    out->damping = damping + shift8;
}

/* R8.  Fig. 3 (missing): the primary taps of direction d sit at distance 1
 * and 2 along d, on both sides of the filtered pixel.  Offsets are
 * (row, column).  The reading takes the pixels on the filtered pixel's own
 * line of Fig. 1 at one and two steps along the line. */
static const int tap_offset[8][2][2] = {
    {{-1, 1}, {-2, 2}},
    {{0, 1}, {-1, 2}},
    {{0, 1}, {0, 2}},
    {{0, 1}, {1, 2}},
    {{1, 1}, {2, 2}},
    {{1, 0}, {2, 1}},
    {{1, 0}, {2, 0}},
    {{1, 0}, {2, -1}},
};

/* R9.  Fig. 3 caption: for even strengths a = 2, b = 4; for odd ones
 * a = b = 3; b is read as the near (distance 1) tap.  Fig. 4 (missing):
 * secondary near 2, far 1.  All in sixteenths. */
static const int pri_weight[2][2] = {{4, 2}, {3, 3}};
static const int sec_weight[2] = {2, 1};

/* Eq. 8-12 for one sample.  The primary taps follow d; the secondary taps
 * form the cross of directions d+2 and d-2 (45 degrees either side, section
 * 3.1; R13: d is used whatever S_p is).  R12: a tap outside the w x h frame
 * contributes f = 0 and is not in the clip range.  R11: the clip range
 * R of eq. 12 is every in-frame tap plus the filtered pixel. */
int64_t cdef_ref_filter_sample(const uint16_t *plane, int w, int h,
                               ptrdiff_t stride, int i, int j, int d,
                               const cdef_ref_eff_params *e)
{
    int64_t x = plane[(ptrdiff_t)i * stride + j];
    int64_t sum = 0;
    int64_t ymin = x, ymax = x;
    /* Primary taps: direction d, distances 1 and 2, both signs. */
    for (int k = 0; k < 2; k++) {
        for (int sign = -1; sign <= 1; sign += 2) {
            int m = i + sign * tap_offset[d][k][0];
            int n = j + sign * tap_offset[d][k][1];
            if (m < 0 || m >= h || n < 0 || n >= w)
                continue;
            int64_t p = plane[(ptrdiff_t)m * stride + n];
            sum += pri_weight[e->parity][k] * cdef_ref_constrain(p - x, e->pri, e->damping);
            ymin = min64(ymin, p);
            ymax = max64(ymax, p);
        }
    }
    /* Secondary taps: directions d + 2 and d - 2 (mod 8), distances 1 and 2,
     * both signs. */
    for (int c = 0; c < 2; c++) {
        int dd = c == 0 ? (d + 2) % 8 : (d + 6) % 8;
        for (int k = 0; k < 2; k++) {
            for (int sign = -1; sign <= 1; sign += 2) {
                int m = i + sign * tap_offset[dd][k][0];
                int n = j + sign * tap_offset[dd][k][1];
                if (m < 0 || m >= h || n < 0 || n >= w)
                    continue;
                int64_t p = plane[(ptrdiff_t)m * stride + n];
                sum += sec_weight[k] * cdef_ref_constrain(p - x, e->sec, e->damping);
                ymin = min64(ymin, p);
                ymax = max64(ymax, p);
            }
        }
    }
    /* Eq. 8 rounding, then the clip of eq. 9-12. */
    int64_t y = x + cdef_ref_round16(sum);
    return min64(ymax, max64(ymin, y));
}

/* Section 4, skip semantics (readings R18-R20).  Byte 5 of a filter
 * block's parameters holds the presets' skip-condition bits: bit 0 luma,
 * bit 1 chroma.  `coded` (NULL = every block coded) marks the 8x8 luma
 * blocks with coded residual; the 4:2:0 chroma 4x4 block follows its
 * co-located luma 8x8 block.
 *   - A filter block with no coded 8x8 block is not filtered at all.
 *   - Otherwise an 8x8 block without coded residual is filtered only when
 *     its plane group's skip-condition bit is set.
 *   - Strengths (0, 0) with the skip-condition bit set stand for primary 19
 *     and secondary 7 (the skip condition stays set). */
static int fb_has_coded(const uint8_t *coded, int bw, int bh, int fby, int fbx)
{
    if (!coded)
        return 1;
    for (int r = fby * 8; r < fby * 8 + 8 && r < bh; r++)
        for (int c = fbx * 8; c < fbx * 8 + 8 && c < bw; c++)
            if (coded[r * bw + c])
                return 1;
    return 0;
}

/* Filters one plane.  sub = 0 for luma (8x8 blocks, 64x64 filter blocks),
 * 1 for 4:2:0 chroma (4x4 blocks, 32x32 filter blocks; section 2: chroma
 * takes the co-located luma direction). */
static void filter_plane_g(const uint16_t *in, ptrdiff_t is, uint16_t *out,
                           ptrdiff_t os, int pw, int ph, int sub, int chroma, int bitdepth,
                           const uint8_t *params, int fb_cols,
                           const uint8_t *dir, const int32_t *var, int bw, int bh,
                           const uint8_t *coded)
{
    int bs = 8 >> sub, fbs = 64 >> sub;
    for (int i = 0; i < ph; i++) {
        for (int j = 0; j < pw; j++) {
            int b8 = (i / bs) * bw + (j / bs);
            int fby = i / fbs, fbx = j / fbs;
            const uint8_t *pp = params + (fby * fb_cols + fbx) * CDEF_REF_PARAM_BYTES;
            int skip_bit = (pp[5] >> chroma) & 1;
            int on = fb_has_coded(coded, bw, bh, fby, fbx) &&
                     (!coded || coded[b8] || skip_bit);
            if (!on) {
                out[(ptrdiff_t)i * os + j] = in[(ptrdiff_t)i * is + j];
                continue;
            }
            int pri = pp[2 * chroma], sec = pp[2 * chroma + 1];
            if (skip_bit && pri == 0 && sec == 0) {
                pri = 19;
                sec = 7;
            }
            cdef_ref_eff_params e;
            cdef_ref_block_params(pri, sec, pp[4], chroma, bitdepth, chroma ? 0 : var[b8], &e);
            out[(ptrdiff_t)i * os + j] =
                (uint16_t)cdef_ref_filter_sample(in, pw, ph, is, i, j, dir[b8], &e);
        }
    }
}

static void filter_plane(const uint16_t *in, ptrdiff_t is, uint16_t *out,
                         ptrdiff_t os, int pw, int ph, int sub, int bitdepth,
                         const uint8_t *params, int fb_cols,
                         const uint8_t *dir, const int32_t *var, int bw, int bh,
                         const uint8_t *coded)
{
    filter_plane_g(in, is, out, os, pw, ph, sub, sub, bitdepth, params, fb_cols, dir, var, bw,
                   bh, coded);
}

static int valid_params(const uint8_t *params, int nblocks)
{
    for (int b = 0; b < nblocks; b++) {
        const uint8_t *p = params + b * CDEF_REF_PARAM_BYTES;
        for (int pl = 0; pl < 2; pl++) {
            int pri = p[2 * pl], sec = p[2 * pl + 1];
            if (!(pri <= 15 || pri == 19))
                return 0;
            if (!(sec == 0 || sec == 1 || sec == 2 || sec == 4 || sec == 7))
                return 0;
        }
        if (p[4] < 3 || p[4] > 6 || p[5] > 3)
            return 0;
    }
    return 1;
}

int cdef_ref_filter_frame_coded(int w, int h, int bitdepth,
                                const uint16_t *y, ptrdiff_t ys,
                                const uint16_t *u, ptrdiff_t us,
                                const uint16_t *v, ptrdiff_t vs,
                                const uint8_t *params, const uint8_t *coded,
                                const uint8_t *dir, const int32_t *var,
                                uint16_t *oy, ptrdiff_t oys,
                                uint16_t *ou, ptrdiff_t ous,
                                uint16_t *ov, ptrdiff_t ovs)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    if (!valid_params(params, fb_cols * fb_rows))
        return -1;
    int bw = w / 8, bh = h / 8;
    filter_plane(y, ys, oy, oys, w, h, 0, bitdepth, params, fb_cols, dir, var, bw, bh, coded);
    filter_plane(u, us, ou, ous, w / 2, h / 2, 1, bitdepth, params, fb_cols, dir, var, bw, bh,
                 coded);
    filter_plane(v, vs, ov, ovs, w / 2, h / 2, 1, bitdepth, params, fb_cols, dir, var, bw, bh,
                 coded);
    return 0;
}

int cdef_ref_filter_frame(int w, int h, int bitdepth,
                          const uint16_t *y, ptrdiff_t ys,
                          const uint16_t *u, ptrdiff_t us,
                          const uint16_t *v, ptrdiff_t vs,
                          const uint8_t *params,
                          const uint8_t *dir, const int32_t *var,
                          uint16_t *oy, ptrdiff_t oys,
                          uint16_t *ou, ptrdiff_t ous,
                          uint16_t *ov, ptrdiff_t ovs)
{
    return cdef_ref_filter_frame_coded(w, h, bitdepth, y, ys, u, us, v, vs, params, NULL, dir,
                                       var, oy, oys, ou, ous, ov, ovs);
}

/* ------------------------------------------------------------------------ */
/* Section 5: encoder search                                                */
/* ------------------------------------------------------------------------ */

/* The 4 signalled secondary strengths, in index order (section 3.2). */
static const int sec_values[4] = {0, 1, 2, 4};

/* Sum over the pixels of filter block (fby, fbx) of one plane of the squared
 * error between the source and the decoded plane filtered with raw
 * strengths (pri, sec). */
static int64_t block_sse(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src,
                         ptrdiff_t ss, int pw, int ph, int sub, int bitdepth,
                         int fby, int fbx, int pri, int sec, int damping,
                         const uint8_t *dir, const int32_t *var, int bw)
{
    int bs = 8 >> sub, fbs = 64 >> sub;
    int64_t sse = 0;
    for (int i = fby * fbs; i < (fby + 1) * fbs && i < ph; i++) {
        for (int j = fbx * fbs; j < (fbx + 1) * fbs && j < pw; j++) {
            int b8 = (i / bs) * bw + (j / bs);
            cdef_ref_eff_params e;
            cdef_ref_block_params(pri, sec, damping, sub, bitdepth, var[b8], &e);
            int64_t yv = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
            int64_t err = yv - (int64_t)src[(ptrdiff_t)i * ss + j];
            sse += err * err;
        }
    }
    return sse;
}

int cdef_ref_distortion(int w, int h, int bitdepth, int damping,
                        const uint16_t *ry, ptrdiff_t rys,
                        const uint16_t *ru, ptrdiff_t rus,
                        const uint16_t *rv, ptrdiff_t rvs,
                        const uint16_t *sy, ptrdiff_t sys,
                        const uint16_t *su, ptrdiff_t sus,
                        const uint16_t *sv, ptrdiff_t svs,
                        int64_t *dist_luma, int64_t *dist_chroma)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6)
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            for (int p = 0; p < 16; p++) {
                for (int s = 0; s < 4; s++) {
                    int q = p * 4 + s;
                    dist_luma[b * 64 + q] =
                        block_sse(ry, rys, sy, sys, w, h, 0, bitdepth, fby, fbx,
                                  p, sec_values[s], damping, dir, var, bw);
                    dist_chroma[b * 64 + q] =
                        block_sse(ru, rus, su, sus, w / 2, h / 2, 1, bitdepth, fby, fbx,
                                  p, sec_values[s], damping, dir, var, bw) +
                        block_sse(rv, rvs, sv, svs, w / 2, h / 2, 1, bitdepth, fby, fbx,
                                  p, sec_values[s], damping, dir, var, bw);
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* Distortion of block b under preset t = luma_pair * 64 + chroma_pair (R15:
 * the block's preset id selects the luma and the chroma pair together). */
static int64_t preset_dist(const int64_t *dl, const int64_t *dc, int b, int t)
{
    return dl[b * 64 + t / 64] + dc[b * 64 + t % 64];
}

/* Eq. 15 with the greedy search of section 5 (R16): N = 1 takes the preset
 * with the least total distortion; each later step adds the preset that
 * lowers sum_b min_{q in P} D_b(q) the most, the earlier ones held fixed;
 * ties go to the lowest preset index.  Then N in {1, 2, 4, 8} (the signalled
 * counts) minimising J(N) = lambda * B * log2 N + sum_b min, ties to the
 * smaller N; a block's id is its least-distortion preset, ties to the lower
 * id. */
int cdef_ref_select_presets(int nblocks, const int64_t *dist_luma,
                            const int64_t *dist_chroma, int64_t lambda,
                            int32_t *presets, int32_t *npresets,
                            uint8_t *block_ids, int64_t *cost,
                            int64_t *costs)
{
    if (nblocks <= 0)
        return -1;
    int64_t total[8];
    for (int n = 1; n <= 8; n++) {
        int best_t = -1;
        int64_t best_total = 0;
        for (int t = 0; t < 4096; t++) {
            int64_t tot = 0;
            for (int b = 0; b < nblocks; b++) {
                int64_t m = preset_dist(dist_luma, dist_chroma, b, t);
                for (int k = 0; k < n - 1; k++)
                    m = min64(m, preset_dist(dist_luma, dist_chroma, b, presets[k]));
                tot += m;
            }
            if (best_t < 0 || tot < best_total) {
                best_t = t;
                best_total = tot;
            }
        }
        presets[n - 1] = best_t;
        total[n - 1] = best_total;
    }
    int best_n = 0;
    int64_t best_j = 0;
    for (int n = 1; n <= 8; n++) {
        int64_t j = total[n - 1];
        int log2n = n == 1 ? 0 : n == 2 ? 1 : n == 4 ? 2 : n == 8 ? 3 : -1;
        if (log2n >= 0)
            j += lambda * nblocks * log2n;
        if (costs)
            costs[n - 1] = j;
        if (log2n >= 0 && (best_n == 0 || j < best_j)) {
            best_n = n;
            best_j = j;
        }
    }
    *npresets = best_n;
    *cost = best_j;
    for (int b = 0; b < nblocks; b++) {
        int id = 0;
        for (int k = 1; k < best_n; k++)
            if (preset_dist(dist_luma, dist_chroma, b, presets[k]) <
                preset_dist(dist_luma, dist_chroma, b, presets[id]))
                id = k;
        block_ids[b] = (uint8_t)id;
    }
    return 0;
}

/* Section 5, last paragraphs: "iteratively re-optimizing one preset at a
 * time" after the greedy search.  Reading (R17): for a fixed set size N,
 * starting from the greedy presets, one pass visits slots k = 0..N-1 in
 * order and replaces preset k by the preset t in [0, 4096) that minimises
 * sum_b min(D_b(t), min_{j != k} D_b(presets[j])), keeping the current
 * preset when it attains that minimum and otherwise taking the lowest such
 * t; passes repeat until one changes nothing or max_passes have run.
 * Every change strictly lowers the total, so the loop terminates.  Writes
 * the refined presets in place, the set's total, and the passes run. */
static int64_t set_total(int nblocks, const int64_t *dl, const int64_t *dc,
                         const int32_t *presets, int n)
{
    int64_t tot = 0;
    for (int b = 0; b < nblocks; b++) {
        int64_t m = preset_dist(dl, dc, b, presets[0]);
        for (int k = 1; k < n; k++)
            m = min64(m, preset_dist(dl, dc, b, presets[k]));
        tot += m;
    }
    return tot;
}

int cdef_ref_refine_presets(int nblocks, const int64_t *dist_luma,
                            const int64_t *dist_chroma, int32_t *presets, int n,
                            int max_passes, int64_t *total, int *passes)
{
    if (nblocks <= 0 || n < 1 || n > 8 || max_passes < 0)
        return -1;
    int run = 0;
    for (int pass = 0; pass < max_passes; pass++) {
        int changed = 0;
        run++;
        for (int k = 0; k < n; k++) {
            int32_t trial[8];
            for (int j = 0; j < n; j++)
                trial[j] = presets[j];
            int64_t cur_total = set_total(nblocks, dist_luma, dist_chroma, trial, n);
            int best_t = presets[k];
            int64_t best_total = cur_total;
            for (int t = 0; t < 4096; t++) {
                trial[k] = t;
                int64_t tot = set_total(nblocks, dist_luma, dist_chroma, trial, n);
                if (tot < best_total || (tot == best_total && best_t != presets[k] && t < best_t)) {
                    best_t = t;
                    best_total = tot;
                }
            }
            if (best_t != presets[k]) {
                presets[k] = best_t;
                changed = 1;
            }
        }
        if (!changed)
            break;
    }
    *total = set_total(nblocks, dist_luma, dist_chroma, presets, n);
    if (passes)
        *passes = run;
    return 0;
}

/* Greedy search (cdef_ref_select_presets) followed by the refinement above
 * for each N in {1, 2, 4, 8} (each from the greedy prefix of that size),
 * then N by J (ties to the smaller N) and block ids over the refined set
 * of that N (ties to the lower index).  max_passes = 0 gives the greedy
 * result.  presets receives the chosen set (npresets entries). */
int cdef_ref_select_presets_refined(int nblocks, const int64_t *dist_luma,
                                    const int64_t *dist_chroma, int64_t lambda,
                                    int max_passes, int32_t *presets,
                                    int32_t *npresets, uint8_t *block_ids,
                                    int64_t *cost)
{
    int32_t greedy[8];
    int32_t np = 0;
    int64_t c = 0;
    int rc = cdef_ref_select_presets(nblocks, dist_luma, dist_chroma, lambda, greedy, &np,
                                     block_ids, &c, NULL);
    if (rc)
        return rc;
    int best_n = 0;
    int64_t best_j = 0;
    int32_t best_set[8] = {0};
    for (int lg = 0; lg < 4; lg++) {
        const int n = 1 << lg;
        int32_t set[8];
        for (int k = 0; k < n; k++)
            set[k] = greedy[k];
        int64_t tot = 0;
        if (cdef_ref_refine_presets(nblocks, dist_luma, dist_chroma, set, n, max_passes, &tot,
                                    NULL))
            return -1;
        const int64_t j = tot + lambda * nblocks * lg;
        if (best_n == 0 || j < best_j) {
            best_n = n;
            best_j = j;
            for (int k = 0; k < n; k++)
                best_set[k] = set[k];
        }
    }
    for (int k = 0; k < 8; k++)
        presets[k] = k < best_n ? best_set[k] : greedy[k];
    *npresets = best_n;
    *cost = best_j;
    for (int b = 0; b < nblocks; b++) {
        int id = 0;
        for (int k = 1; k < best_n; k++)
            if (preset_dist(dist_luma, dist_chroma, b, best_set[k]) <
                preset_dist(dist_luma, dist_chroma, b, best_set[id]))
                id = k;
        block_ids[b] = (uint8_t)id;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 5 with section 4's skip semantics                                */
/* ------------------------------------------------------------------------ */

/* Reading R21.  The search covers the 128 combinations of a plane group
 * that section 5 counts (16 primary x 4 secondary strengths x the skip-
 * condition bit), index q = k * 64 + p * 4 + s.  D_{b,q} is the squared
 * error of what the decoder outputs for filter block b with that preset
 * (cdef_ref_filter_frame_coded): a pixel of 8x8 block j is filtered when
 * the filter block has coded residual and (j is coded or k = 1); strengths
 * (0, 0) with k = 1 stand for (19, 7).  A filter block without coded
 * residual is never filtered: its entries are all the unfiltered SSE, and
 * skipped[b] = 1 (it signals no preset id). */
static int64_t block_sse_coded(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src,
                               ptrdiff_t ss, int pw, int ph, int sub, int bitdepth,
                               int fby, int fbx, int pri, int sec, int k, int damping,
                               const uint8_t *dir, const int32_t *var, int bw,
                               const uint8_t *coded, int fb_coded)
{
    int bs = 8 >> sub, fbs = 64 >> sub;
    int64_t sse = 0;
    for (int i = fby * fbs; i < (fby + 1) * fbs && i < ph; i++) {
        for (int j = fbx * fbs; j < (fbx + 1) * fbs && j < pw; j++) {
            int b8 = (i / bs) * bw + (j / bs);
            int on = fb_coded && (!coded || coded[b8] || k);
            int64_t yv = rec[(ptrdiff_t)i * rs + j];
            if (on) {
                cdef_ref_eff_params e;
                cdef_ref_block_params(pri, sec, damping, sub, bitdepth, sub ? 0 : var[b8], &e);
                yv = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
            }
            int64_t err = yv - (int64_t)src[(ptrdiff_t)i * ss + j];
            sse += err * err;
        }
    }
    return sse;
}

int cdef_ref_distortion_coded(int w, int h, int bitdepth, int damping,
                              const uint16_t *ry, ptrdiff_t rys,
                              const uint16_t *ru, ptrdiff_t rus,
                              const uint16_t *rv, ptrdiff_t rvs,
                              const uint16_t *sy, ptrdiff_t sys,
                              const uint16_t *su, ptrdiff_t sus,
                              const uint16_t *sv, ptrdiff_t svs,
                              const uint8_t *coded, int64_t *dist_luma,
                              int64_t *dist_chroma, uint8_t *skipped)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6)
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            int fb_coded = fb_has_coded(coded, bw, bh, fby, fbx);
            skipped[b] = (uint8_t)!fb_coded;
            for (int k = 0; k < 2; k++) {
                for (int p = 0; p < 16; p++) {
                    for (int s = 0; s < 4; s++) {
                        int q = k * 64 + p * 4 + s;
                        int pri = p, sec = sec_values[s];
                        if (k && p == 0 && s == 0) {
                            pri = 19;
                            sec = 7;
                        }
                        dist_luma[b * 128 + q] =
                            block_sse_coded(ry, rys, sy, sys, w, h, 0, bitdepth, fby, fbx, pri,
                                            sec, k, damping, dir, var, bw, coded, fb_coded);
                        dist_chroma[b * 128 + q] =
                            block_sse_coded(ru, rus, su, sus, w / 2, h / 2, 1, bitdepth, fby,
                                            fbx, pri, sec, k, damping, dir, var, bw, coded,
                                            fb_coded) +
                            block_sse_coded(rv, rvs, sv, svs, w / 2, h / 2, 1, bitdepth, fby,
                                            fbx, pri, sec, k, damping, dir, var, bw, coded,
                                            fb_coded);
                    }
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* Preset selection over tables of `width` combinations per plane group
 * (presets t = luma_q * width + chroma_q), blocks with skipped[b] set left
 * out of every sum and of B.  The same rules as cdef_ref_select_presets
 * (greedy, R16) and cdef_ref_refine_presets (R17), restated for any width. */
static int64_t gen_dist(const int64_t *dl, const int64_t *dc, int width, int b, int t)
{
    return dl[(int64_t)b * width + t / width] + dc[(int64_t)b * width + t % width];
}

static int64_t gen_total(int nblocks, const int64_t *dl, const int64_t *dc, int width,
                         const uint8_t *skipped, const int32_t *set, int n)
{
    int64_t tot = 0;
    for (int b = 0; b < nblocks; b++) {
        if (skipped && skipped[b])
            continue;
        int64_t m = gen_dist(dl, dc, width, b, set[0]);
        for (int k = 1; k < n; k++)
            m = min64(m, gen_dist(dl, dc, width, b, set[k]));
        tot += m;
    }
    return tot;
}

/* Section 5's low-complexity search considers only a subset of the
 * combinations.  Reading R26: the subset is the caller's choice of allowed
 * (S_p, S_s) pairs per plane group, bit p * 4 + s of luma_pairs /
 * chroma_pairs (the same pairs with either skip-condition bit in the
 * 128-combination search); a preset is a candidate of the greedy search and
 * of the re-optimisation when its luma and its chroma combination are both
 * allowed.  Everything else is as in cdef_ref_select_presets_general. */
static int allowed_preset(int t, int width, uint64_t luma_pairs, uint64_t chroma_pairs)
{
    int ql = (t / width) % 64, qc = (t % width) % 64;
    return (int)((luma_pairs >> ql) & 1) && (int)((chroma_pairs >> qc) & 1);
}

int cdef_ref_select_presets_subset(int nblocks, const int64_t *dist_luma,
                                   const int64_t *dist_chroma, int width,
                                   const uint8_t *skipped, uint64_t luma_pairs,
                                   uint64_t chroma_pairs, int64_t lambda, int max_passes,
                                   int32_t *presets, int32_t *npresets,
                                   uint8_t *block_ids, int64_t *cost)
{
    if (nblocks <= 0 || (width != 64 && width != 128) || max_passes < 0)
        return -1;
    if (luma_pairs == 0 || chroma_pairs == 0)
        return -1;
    const int ntuples = width * width;
    int coded_blocks = 0;
    for (int b = 0; b < nblocks; b++)
        coded_blocks += !(skipped && skipped[b]);
    /* greedy */
    int32_t greedy[8];
    int64_t totals[8];
    for (int n = 1; n <= 8; n++) {
        int best_t = -1;
        int64_t best_total = 0;
        for (int t = 0; t < ntuples; t++) {
            if (!allowed_preset(t, width, luma_pairs, chroma_pairs))
                continue;
            greedy[n - 1] = t;
            int64_t tot = gen_total(nblocks, dist_luma, dist_chroma, width, skipped, greedy, n);
            if (best_t < 0 || tot < best_total) {
                best_t = t;
                best_total = tot;
            }
        }
        greedy[n - 1] = best_t;
        totals[n - 1] = best_total;
    }
    /* re-optimisation per set size, then N by J */
    int best_n = 0;
    int64_t best_j = 0;
    int32_t best_set[8] = {0};
    for (int lg = 0; lg < 4; lg++) {
        const int n = 1 << lg;
        int32_t set[8];
        for (int k = 0; k < n; k++)
            set[k] = greedy[k];
        int64_t tot = totals[n - 1];
        for (int pass = 0; pass < max_passes; pass++) {
            int changed = 0;
            for (int k = 0; k < n; k++) {
                const int32_t old = set[k];
                int best_t = old;
                int64_t best_total = gen_total(nblocks, dist_luma, dist_chroma, width, skipped,
                                               set, n);
                for (int t = 0; t < ntuples; t++) {
                    if (!allowed_preset(t, width, luma_pairs, chroma_pairs))
                        continue;
                    set[k] = t;
                    int64_t v = gen_total(nblocks, dist_luma, dist_chroma, width, skipped, set, n);
                    if (v < best_total || (v == best_total && best_t != old && t < best_t)) {
                        best_t = t;
                        best_total = v;
                    }
                }
                set[k] = best_t;
                if (best_t != old)
                    changed = 1;
                tot = best_total;
            }
            if (!changed)
                break;
        }
        const int64_t j = tot + lambda * coded_blocks * lg;
        if (best_n == 0 || j < best_j) {
            best_n = n;
            best_j = j;
            for (int k = 0; k < n; k++)
                best_set[k] = set[k];
        }
    }
    for (int k = 0; k < 8; k++)
        presets[k] = k < best_n ? best_set[k] : greedy[k];
    *npresets = best_n;
    *cost = best_j;
    for (int b = 0; b < nblocks; b++) {
        int id = 0;
        if (!(skipped && skipped[b]))
            for (int k = 1; k < best_n; k++)
                if (gen_dist(dist_luma, dist_chroma, width, b, best_set[k]) <
                    gen_dist(dist_luma, dist_chroma, width, b, best_set[id]))
                    id = k;
        block_ids[b] = (uint8_t)id;
    }
    return 0;
}

int cdef_ref_select_presets_general(int nblocks, const int64_t *dist_luma,
                                    const int64_t *dist_chroma, int width,
                                    const uint8_t *skipped, int64_t lambda, int max_passes,
                                    int32_t *presets, int32_t *npresets,
                                    uint8_t *block_ids, int64_t *cost)
{
    return cdef_ref_select_presets_subset(nblocks, dist_luma, dist_chroma, width, skipped,
                                          ~(uint64_t)0, ~(uint64_t)0, lambda, max_passes,
                                          presets, npresets, block_ids, cost);
}

/* Section 5's tables for the other chroma formats (section 4, last
 * paragraph; reading R25), at any bit depth.  Luma as cdef_ref_distortion.
 * Chroma (U + V): format 420 as cdef_ref_distortion; format 422, whose
 * chroma is not filtered, the unfiltered squared error of the filter
 * block's chroma region (w/2 x h planes: 32 columns x 64 rows) for every
 * pair; format 444 the squared error of each plane filtered in 8x8 blocks
 * of the 64x64 filter block with the chroma strengths and damping and the
 * co-located luma block's direction. */
static int64_t block_sse_g(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src, ptrdiff_t ss,
                           int pw, int ph, int sub, int chroma, int filtered, int bitdepth,
                           int fby, int fbx, int pri, int sec, int damping, const uint8_t *dir,
                           const int32_t *var, int bw, int fbw, int fbh)
{
    int bs = 8 >> sub;
    int64_t sse = 0;
    for (int i = fby * fbh; i < (fby + 1) * fbh && i < ph; i++) {
        for (int j = fbx * fbw; j < (fbx + 1) * fbw && j < pw; j++) {
            int64_t yv = rec[(ptrdiff_t)i * rs + j];
            if (filtered) {
                int b8 = (i / bs) * bw + (j / bs);
                cdef_ref_eff_params e;
                cdef_ref_block_params(pri, sec, damping, chroma, bitdepth, chroma ? 0 : var[b8], &e);
                yv = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
            }
            int64_t err = yv - (int64_t)src[(ptrdiff_t)i * ss + j];
            sse += err * err;
        }
    }
    return sse;
}

int cdef_ref_distortion_format(int w, int h, int bitdepth, int damping, int format,
                               const uint16_t *ry, ptrdiff_t rys,
                               const uint16_t *ru, ptrdiff_t rus,
                               const uint16_t *rv, ptrdiff_t rvs,
                               const uint16_t *sy, ptrdiff_t sys,
                               const uint16_t *su, ptrdiff_t sus,
                               const uint16_t *sv, ptrdiff_t svs,
                               int64_t *dist_luma, int64_t *dist_chroma)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6 || (format != 420 && format != 422 && format != 444))
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    /* chroma plane geometry: size, 8x8-block subsampling, filter-block size */
    int cw = format == 444 ? w : w / 2, ch = format == 420 ? h / 2 : h;
    int csub = format == 444 ? 0 : 1;
    int cfw = format == 444 ? 64 : 32, cfh = format == 420 ? 32 : 64;
    int cfilt = format != 422;
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            for (int p = 0; p < 16; p++) {
                for (int s = 0; s < 4; s++) {
                    int q = p * 4 + s;
                    dist_luma[b * 64 + q] =
                        block_sse_g(ry, rys, sy, sys, w, h, 0, 0, 1, bitdepth, fby, fbx, p,
                                    sec_values[s], damping, dir, var, bw, 64, 64);
                    dist_chroma[b * 64 + q] =
                        block_sse_g(ru, rus, su, sus, cw, ch, csub, 1, cfilt, bitdepth, fby, fbx,
                                    p, sec_values[s], damping, dir, var, bw, cfw, cfh) +
                        block_sse_g(rv, rvs, sv, svs, cw, ch, csub, 1, cfilt, bitdepth, fby, fbx,
                                    p, sec_values[s], damping, dir, var, bw, cfw, cfh);
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* The 128-combination tables (reading R21) for chroma format 420, 422 or
 * 444 at any bit depth (reading R25): as cdef_ref_distortion_coded, with
 * the chroma geometry of cdef_ref_distortion_format (4:2:2 chroma is never
 * filtered, so all its entries are the unfiltered error).  A pixel of the
 * 8x8 (4:2:0 chroma: 4x4) block j is filtered when the filter block has
 * coded residual and (j's co-located luma block is coded or the skip bit k
 * is set); (0, 0) with k set stands for (19, 7). */
static int64_t block_sse_coded_g(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src,
                                 ptrdiff_t ss, int pw, int ph, int sub, int chroma, int filtered,
                                 int bitdepth, int fby, int fbx, int pri, int sec, int k,
                                 int damping, const uint8_t *dir, const int32_t *var, int bw,
                                 int fbw, int fbh, const uint8_t *coded, int fb_coded)
{
    int bs = 8 >> sub;
    int64_t sse = 0;
    for (int i = fby * fbh; i < (fby + 1) * fbh && i < ph; i++) {
        for (int j = fbx * fbw; j < (fbx + 1) * fbw && j < pw; j++) {
            int b8 = (i / bs) * bw + (j / bs);
            int on = filtered && fb_coded && (!coded || coded[b8] || k);
            int64_t yv = rec[(ptrdiff_t)i * rs + j];
            if (on) {
                cdef_ref_eff_params e;
                cdef_ref_block_params(pri, sec, damping, chroma, bitdepth, chroma ? 0 : var[b8], &e);
                yv = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
            }
            int64_t err = yv - (int64_t)src[(ptrdiff_t)i * ss + j];
            sse += err * err;
        }
    }
    return sse;
}

int cdef_ref_distortion_coded_format(int w, int h, int bitdepth, int damping, int format,
                                     const uint16_t *ry, ptrdiff_t rys,
                                     const uint16_t *ru, ptrdiff_t rus,
                                     const uint16_t *rv, ptrdiff_t rvs,
                                     const uint16_t *sy, ptrdiff_t sys,
                                     const uint16_t *su, ptrdiff_t sus,
                                     const uint16_t *sv, ptrdiff_t svs,
                                     const uint8_t *coded, int64_t *dist_luma,
                                     int64_t *dist_chroma, uint8_t *skipped)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6 || (format != 420 && format != 422 && format != 444))
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    int cw = format == 444 ? w : w / 2, ch = format == 420 ? h / 2 : h;
    int csub = format == 444 ? 0 : 1;
    int cfw = format == 444 ? 64 : 32, cfh = format == 420 ? 32 : 64;
    int cfilt = format != 422;
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            int fb_coded = fb_has_coded(coded, bw, bh, fby, fbx);
            skipped[b] = (uint8_t)!fb_coded;
            for (int k = 0; k < 2; k++) {
                for (int p = 0; p < 16; p++) {
                    for (int s = 0; s < 4; s++) {
                        int q = k * 64 + p * 4 + s;
                        int pri = p, sec = sec_values[s];
                        if (k && p == 0 && s == 0) {
                            pri = 19;
                            sec = 7;
                        }
                        dist_luma[b * 128 + q] = block_sse_coded_g(
                            ry, rys, sy, sys, w, h, 0, 0, 1, bitdepth, fby, fbx, pri, sec, k,
                            damping, dir, var, bw, 64, 64, coded, fb_coded);
                        dist_chroma[b * 128 + q] =
                            block_sse_coded_g(ru, rus, su, sus, cw, ch, csub, 1, cfilt, bitdepth,
                                              fby, fbx, pri, sec, k, damping, dir, var, bw, cfw,
                                              cfh, coded, fb_coded) +
                            block_sse_coded_g(rv, rvs, sv, svs, cw, ch, csub, 1, cfilt, bitdepth,
                                              fby, fbx, pri, sec, k, damping, dir, var, bw, cfw,
                                              cfh, coded, fb_coded);
                    }
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* Chroma formats other than 4:2:0 (section 4, last paragraph; reading R25):
 *   format 422: chroma planes are w/2 x h; their subsampling differs
 *               horizontally and vertically, so chroma is not filtered (the
 *               output planes equal the input planes);
 *   format 444: chroma planes are w x h; each is filtered like the luma
 *               plane (8x8 blocks, 64x64 filter blocks) with the chroma
 *               strengths and damping (no contrast adjustment) and the
 *               co-located luma block's direction.
 * Luma is filtered as for 4:2:0; skip semantics as cdef_ref_filter_frame_coded. */
int cdef_ref_filter_frame_format(int w, int h, int bitdepth, int format,
                                 const uint16_t *y, ptrdiff_t ys,
                                 const uint16_t *u, ptrdiff_t us,
                                 const uint16_t *v, ptrdiff_t vs,
                                 const uint8_t *params, const uint8_t *coded,
                                 const uint8_t *dir, const int32_t *var,
                                 uint16_t *oy, ptrdiff_t oys,
                                 uint16_t *ou, ptrdiff_t ous,
                                 uint16_t *ov, ptrdiff_t ovs)
{
    if (format == 420)
        return cdef_ref_filter_frame_coded(w, h, bitdepth, y, ys, u, us, v, vs, params, coded,
                                           dir, var, oy, oys, ou, ous, ov, ovs);
    if (format != 422 && format != 444)
        return -1;
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    if (!valid_params(params, fb_cols * fb_rows))
        return -1;
    int bw = w / 8, bh = h / 8;
    filter_plane(y, ys, oy, oys, w, h, 0, bitdepth, params, fb_cols, dir, var, bw, bh, coded);
    if (format == 422) {
        for (int i = 0; i < h; i++)
            for (int j = 0; j < w / 2; j++) {
                ou[(ptrdiff_t)i * ous + j] = u[(ptrdiff_t)i * us + j];
                ov[(ptrdiff_t)i * ovs + j] = v[(ptrdiff_t)i * vs + j];
            }
    } else {
        filter_plane_g(u, us, ou, ous, w, h, 0, 1, bitdepth, params, fb_cols, dir, var, bw, bh,
                       coded);
        filter_plane_g(v, vs, ov, ovs, w, h, 0, 1, bitdepth, params, fb_cols, dir, var, bw, bh,
                       coded);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Section 5, eq. 14: the SSIM-weighted distortion                          */
/* ------------------------------------------------------------------------ */

/* Readings R22-R24.  R22: the 8x8 distortion function of eq. 14 is taken
 * over the 8x8 blocks of each plane (luma 64, each 4:2:0 chroma plane 16 per
 * filter block), with sigma^2 the population variance of the 64 source
 * samples and of the 64 filtered decoded samples; chroma sums U and V.
 * An 8x8 block cut by the frame edge (4:2:0 chroma planes whose size is
 * not a multiple of 8) uses its n in-frame samples.  R23: C1 = 6.25 *
 * 4^(bd-8) and C2 = 312.5 * 16^(bd-8) (the constants scale with the units
 * of a variance and of its square).  R24: the table holds the sum over the
 * 8x8 blocks of round(256 * D_8x8) (ties away from zero), so that the
 * preset search works on exact integers.  The paper fixes no precision;
 * this oracle evaluates eq. 14 as written in IEEE double precision:
 *   vs = (n sum s^2 - (sum s)^2) / n^2, vd likewise (both exact here: the
 *        numerators stay below 2^53 and n is 16, 32 or 64),
 *   D  = (vs + vd + C1) / (2 sqrt(vs vd + C2)) * sse,
 * which is within a few units in the last place of the exact value, so the
 * rounded result equals round(256 * D) of the exact value except where
 * 256 * D lies within a few units in the last place of a half-integer. */
static int64_t eq14_term(int64_t n, int64_t s1s, int64_t s2s, int64_t s1d, int64_t s2d,
                         int64_t sse, int bitdepth)
{
    const double c1 = 6.25 * (double)((int64_t)1 << (2 * (bitdepth - 8)));
    const double c2 = 312.5 * (double)((int64_t)1 << (4 * (bitdepth - 8)));
    const double nn = (double)(n * n);
    const double vs = (double)(n * s2s - s1s * s1s) / nn;
    const double vd = (double)(n * s2d - s1d * s1d) / nn;
    const double d = (vs + vd + c1) / (2.0 * sqrt(vs * vd + c2)) * (double)sse;
    return (int64_t)llround(256.0 * d);
}

static int64_t block_eq14(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src, ptrdiff_t ss,
                          int pw, int ph, int sub, int bitdepth, int fby, int fbx, int pri,
                          int sec, int damping, const uint8_t *dir, const int32_t *var, int bw)
{
    int bs = 8 >> sub, fbs = 64 >> sub;
    int64_t total = 0;
    /* 8x8 blocks of this plane inside the filter block */
    for (int by = fby * fbs; by < (fby + 1) * fbs && by < ph; by += 8) {
        for (int bx = fbx * fbs; bx < (fbx + 1) * fbs && bx < pw; bx += 8) {
            int64_t n = 0, s1s = 0, s2s = 0, s1d = 0, s2d = 0, sse = 0;
            for (int i = by; i < by + 8 && i < ph; i++) {
                for (int j = bx; j < bx + 8 && j < pw; j++) {
                    n++;
                    int b8 = (i / bs) * bw + (j / bs);
                    cdef_ref_eff_params e;
                    cdef_ref_block_params(pri, sec, damping, sub, bitdepth, sub ? 0 : var[b8], &e);
                    int64_t d = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
                    int64_t sv = src[(ptrdiff_t)i * ss + j];
                    s1s += sv;
                    s2s += sv * sv;
                    s1d += d;
                    s2d += d * d;
                    sse += (d - sv) * (d - sv);
                }
            }
            total += eq14_term(n, s1s, s2s, s1d, s2d, sse, bitdepth);
        }
    }
    return total;
}

int cdef_ref_distortion_eq14(int w, int h, int bitdepth, int damping,
                             const uint16_t *ry, ptrdiff_t rys,
                             const uint16_t *ru, ptrdiff_t rus,
                             const uint16_t *rv, ptrdiff_t rvs,
                             const uint16_t *sy, ptrdiff_t sys,
                             const uint16_t *su, ptrdiff_t sus,
                             const uint16_t *sv, ptrdiff_t svs,
                             int64_t *dist_luma, int64_t *dist_chroma)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6)
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            for (int p = 0; p < 16; p++) {
                for (int s = 0; s < 4; s++) {
                    int q = p * 4 + s;
                    dist_luma[b * 64 + q] =
                        block_eq14(ry, rys, sy, sys, w, h, 0, bitdepth, fby, fbx, p,
                                   sec_values[s], damping, dir, var, bw);
                    dist_chroma[b * 64 + q] =
                        block_eq14(ru, rus, su, sus, w / 2, h / 2, 1, bitdepth, fby, fbx, p,
                                   sec_values[s], damping, dir, var, bw) +
                        block_eq14(rv, rvs, sv, svs, w / 2, h / 2, 1, bitdepth, fby, fbx, p,
                                   sec_values[s], damping, dir, var, bw);
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* Eq. 14 tables for chroma format 420, 422 or 444 at any bit depth
 * (readings R22-R25): the sum over the 8x8 blocks of each plane inside the
 * filter block of eq. 14's value, with the chroma geometry of
 * cdef_ref_distortion_format (4:2:2 chroma is never filtered: every pair
 * gives the unfiltered value).  The 8x8 blocks are those of the plane's own
 * grid; a block cut by the frame edge takes its in-frame samples. */
static int64_t block_eq14_g(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src, ptrdiff_t ss,
                            int pw, int ph, int sub, int chroma, int filtered, int bitdepth,
                            int fby, int fbx, int pri, int sec, int damping, const uint8_t *dir,
                            const int32_t *var, int bw, int fbw, int fbh)
{
    int bs = 8 >> sub;
    int64_t total = 0;
    for (int by = fby * fbh; by < (fby + 1) * fbh && by < ph; by += 8) {
        for (int bx = fbx * fbw; bx < (fbx + 1) * fbw && bx < pw; bx += 8) {
            int64_t n = 0, s1s = 0, s2s = 0, s1d = 0, s2d = 0, sse = 0;
            for (int i = by; i < by + 8 && i < ph; i++) {
                for (int j = bx; j < bx + 8 && j < pw; j++) {
                    int64_t d = rec[(ptrdiff_t)i * rs + j];
                    if (filtered) {
                        int b8 = (i / bs) * bw + (j / bs);
                        cdef_ref_eff_params e;
                        cdef_ref_block_params(pri, sec, damping, chroma, bitdepth,
                                              chroma ? 0 : var[b8], &e);
                        d = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
                    }
                    int64_t sv = src[(ptrdiff_t)i * ss + j];
                    n++;
                    s1s += sv;
                    s2s += sv * sv;
                    s1d += d;
                    s2d += d * d;
                    sse += (d - sv) * (d - sv);
                }
            }
            total += eq14_term(n, s1s, s2s, s1d, s2d, sse, bitdepth);
        }
    }
    return total;
}

int cdef_ref_distortion_eq14_format(int w, int h, int bitdepth, int damping, int format,
                                    const uint16_t *ry, ptrdiff_t rys,
                                    const uint16_t *ru, ptrdiff_t rus,
                                    const uint16_t *rv, ptrdiff_t rvs,
                                    const uint16_t *sy, ptrdiff_t sys,
                                    const uint16_t *su, ptrdiff_t sus,
                                    const uint16_t *sv, ptrdiff_t svs,
                                    int64_t *dist_luma, int64_t *dist_chroma)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6 || (format != 420 && format != 422 && format != 444))
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    int cw = format == 444 ? w : w / 2, ch = format == 420 ? h / 2 : h;
    int csub = format == 444 ? 0 : 1;
    int cfw = format == 444 ? 64 : 32, cfh = format == 420 ? 32 : 64;
    int cfilt = format != 422;
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            for (int p = 0; p < 16; p++) {
                for (int s = 0; s < 4; s++) {
                    int q = p * 4 + s;
                    dist_luma[b * 64 + q] =
                        block_eq14_g(ry, rys, sy, sys, w, h, 0, 0, 1, bitdepth, fby, fbx, p,
                                     sec_values[s], damping, dir, var, bw, 64, 64);
                    dist_chroma[b * 64 + q] =
                        block_eq14_g(ru, rus, su, sus, cw, ch, csub, 1, cfilt, bitdepth, fby, fbx,
                                     p, sec_values[s], damping, dir, var, bw, cfw, cfh) +
                        block_eq14_g(rv, rvs, sv, svs, cw, ch, csub, 1, cfilt, bitdepth, fby, fbx,
                                     p, sec_values[s], damping, dir, var, bw, cfw, cfh);
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* Eq. 14 tables of the 128 combinations (readings R21-R25): as
 * cdef_ref_distortion_coded_format with each entry the sum over the 8x8
 * blocks of each plane (the plane's own grid) of eq. 14's value of what the
 * decoder outputs for that preset: a sample of the 8x8 (4:2:0 chroma: 4x4)
 * direction block j is filtered when the filter block has coded residual
 * and (j's co-located luma block is coded or the skip bit k is set); (0, 0)
 * with k set stands for (19, 7); 4:2:2 chroma is never filtered. */
static int64_t block_eq14_coded_g(const uint16_t *rec, ptrdiff_t rs, const uint16_t *src,
                                  ptrdiff_t ss, int pw, int ph, int sub, int chroma, int filtered,
                                  int bitdepth, int fby, int fbx, int pri, int sec, int k,
                                  int damping, const uint8_t *dir, const int32_t *var, int bw,
                                  int fbw, int fbh, const uint8_t *coded, int fb_coded)
{
    int bs = 8 >> sub;
    int64_t total = 0;
    for (int by = fby * fbh; by < (fby + 1) * fbh && by < ph; by += 8) {
        for (int bx = fbx * fbw; bx < (fbx + 1) * fbw && bx < pw; bx += 8) {
            int64_t n = 0, s1s = 0, s2s = 0, s1d = 0, s2d = 0, sse = 0;
            for (int i = by; i < by + 8 && i < ph; i++) {
                for (int j = bx; j < bx + 8 && j < pw; j++) {
                    int b8 = (i / bs) * bw + (j / bs);
                    int on = filtered && fb_coded && (!coded || coded[b8] || k);
                    int64_t d = rec[(ptrdiff_t)i * rs + j];
                    if (on) {
                        cdef_ref_eff_params e;
                        cdef_ref_block_params(pri, sec, damping, chroma, bitdepth,
                                              chroma ? 0 : var[b8], &e);
                        d = cdef_ref_filter_sample(rec, pw, ph, rs, i, j, dir[b8], &e);
                    }
                    int64_t sv = src[(ptrdiff_t)i * ss + j];
                    n++;
                    s1s += sv;
                    s2s += sv * sv;
                    s1d += d;
                    s2d += d * d;
                    sse += (d - sv) * (d - sv);
                }
            }
            total += eq14_term(n, s1s, s2s, s1d, s2d, sse, bitdepth);
        }
    }
    return total;
}

int cdef_ref_distortion_eq14_coded_format(int w, int h, int bitdepth, int damping, int format,
                                          const uint16_t *ry, ptrdiff_t rys,
                                          const uint16_t *ru, ptrdiff_t rus,
                                          const uint16_t *rv, ptrdiff_t rvs,
                                          const uint16_t *sy, ptrdiff_t sys,
                                          const uint16_t *su, ptrdiff_t sus,
                                          const uint16_t *sv, ptrdiff_t svs,
                                          const uint8_t *coded, int64_t *dist_luma,
                                          int64_t *dist_chroma, uint8_t *skipped)
{
    if (w <= 0 || h <= 0 || w % 8 || h % 8 || bitdepth < 8 || bitdepth > 12)
        return -1;
    if (damping < 3 || damping > 6 || (format != 420 && format != 422 && format != 444))
        return -1;
    int bw = w / 8, bh = h / 8;
    uint8_t *dir = (uint8_t *)malloc((size_t)bw * bh);
    int32_t *var = (int32_t *)malloc((size_t)bw * bh * sizeof(int32_t));
    if (!dir || !var) {
        free(dir);
        free(var);
        return -1;
    }
    cdef_ref_find_dir(ry, w, h, rys, bitdepth, dir, var);
    int cw = format == 444 ? w : w / 2, ch = format == 420 ? h / 2 : h;
    int csub = format == 444 ? 0 : 1;
    int cfw = format == 444 ? 64 : 32, cfh = format == 420 ? 32 : 64;
    int cfilt = format != 422;
    int fb_cols = (w + 63) / 64, fb_rows = (h + 63) / 64;
    for (int fby = 0; fby < fb_rows; fby++) {
        for (int fbx = 0; fbx < fb_cols; fbx++) {
            int b = fby * fb_cols + fbx;
            int fb_coded = fb_has_coded(coded, bw, bh, fby, fbx);
            skipped[b] = (uint8_t)!fb_coded;
            for (int k = 0; k < 2; k++) {
                for (int p = 0; p < 16; p++) {
                    for (int s = 0; s < 4; s++) {
                        int q = k * 64 + p * 4 + s;
                        int pri = p, sec = sec_values[s];
                        if (k && p == 0 && s == 0) {
                            pri = 19;
                            sec = 7;
                        }
                        dist_luma[b * 128 + q] = block_eq14_coded_g(
                            ry, rys, sy, sys, w, h, 0, 0, 1, bitdepth, fby, fbx, pri, sec, k,
                            damping, dir, var, bw, 64, 64, coded, fb_coded);
                        dist_chroma[b * 128 + q] =
                            block_eq14_coded_g(ru, rus, su, sus, cw, ch, csub, 1, cfilt, bitdepth,
                                               fby, fbx, pri, sec, k, damping, dir, var, bw, cfw,
                                               cfh, coded, fb_coded) +
                            block_eq14_coded_g(rv, rvs, sv, svs, cw, ch, csub, 1, cfilt, bitdepth,
                                               fby, fbx, pri, sec, k, damping, dir, var, bw, cfw,
                                               cfh, coded, fb_coded);
                    }
                }
            }
        }
    }
    free(dir);
    free(var);
    return 0;
}

/* The eq. 14 value of one 8x8 block from its sums (R22-R24), exported for
 * the pins. */
int64_t cdef_ref_eq14_term(int64_t n, int64_t s1s, int64_t s2s, int64_t s1d, int64_t s2d,
                           int64_t sse, int bitdepth)
{
    return eq14_term(n, s1s, s2s, s1d, s2d, sse, bitdepth);
}
