/*
 * Every entry point of the CPU oracle (oracle/cdef_ref.c) on small frames of
 * every bit depth and chroma format, built with AddressSanitizer and
 * UndefinedBehaviorSanitizer by tests/test_oracle_sanitized.py.  Buffers are
 * allocated at their exact sizes (pitch = width), so a read or write past a
 * plane, a table or a map is reported; so are signed overflows and shifts
 * out of range.  Exit status 0 when every call succeeded and nothing was
 * reported (the sanitizers abort on the first report).
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cdef_ref.h"

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;

static uint32_t next_u32(void)
{
    /* xorshift64* */
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return (uint32_t)((rng_state * 0x2545f4914f6cdd1dull) >> 32);
}

static uint16_t *plane_alloc(int w, int h, int bitdepth)
{
    uint16_t *p = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)w * h);
    if (!p)
        exit(3);
    for (int i = 0; i < w * h; i++)
        p[i] = (uint16_t)(next_u32() & ((1u << bitdepth) - 1));
    return p;
}

static int fail(const char *what, int w, int h, int bd, int fmt)
{
    fprintf(stderr, "oracle call failed: %s %dx%d bd %d fmt %d\n", what, w, h, bd, fmt);
    return 1;
}

static int frame_case(int w, int h, int bd, int fmt, int tables)
{
    const int cw = fmt == 444 ? w : w / 2, ch = fmt == 420 ? h / 2 : h;
    const int bw = w / 8, bh = h / 8, fb = ((w + 63) / 64) * ((h + 63) / 64);
    uint16_t *y = plane_alloc(w, h, bd), *u = plane_alloc(cw, ch, bd), *v = plane_alloc(cw, ch, bd);
    uint16_t *sy = plane_alloc(w, h, bd), *su = plane_alloc(cw, ch, bd), *sv = plane_alloc(cw, ch, bd);
    uint16_t *oy = malloc(sizeof(uint16_t) * (size_t)w * h);
    uint16_t *ou = malloc(sizeof(uint16_t) * (size_t)cw * ch);
    uint16_t *ov = malloc(sizeof(uint16_t) * (size_t)cw * ch);
    uint8_t *dir = malloc((size_t)bw * bh), *coded = malloc((size_t)bw * bh);
    int32_t *var = malloc(sizeof(int32_t) * (size_t)bw * bh);
    uint8_t *params = malloc((size_t)fb * CDEF_REF_PARAM_BYTES);
    int64_t *dl = malloc(sizeof(int64_t) * (size_t)fb * 128), *dc = malloc(sizeof(int64_t) * (size_t)fb * 128);
    uint8_t *skipped = malloc((size_t)fb), *ids = malloc((size_t)fb);
    int rc = 0;
    if (!oy || !ou || !ov || !dir || !coded || !var || !params || !dl || !dc || !skipped || !ids)
        exit(3);
    static const uint8_t sec[5] = {0, 1, 2, 4, 7};
    for (int b = 0; b < fb; b++) {
        uint8_t *p = params + (size_t)b * CDEF_REF_PARAM_BYTES;
        p[0] = (uint8_t)(next_u32() % 16);
        p[1] = sec[next_u32() % 5];
        p[2] = (uint8_t)(next_u32() % 16);
        p[3] = sec[next_u32() % 5];
        p[4] = (uint8_t)(3 + next_u32() % 4);
        p[5] = (uint8_t)(next_u32() % 4);
        p[6] = p[7] = 0;
    }
    for (int i = 0; i < bw * bh; i++)
        coded[i] = (uint8_t)(next_u32() & 1);

    if (cdef_ref_find_dir(y, w, h, w, bd, dir, var))
        rc |= fail("find_dir", w, h, bd, fmt);
    if (fmt == 420 && cdef_ref_filter_frame(w, h, bd, y, w, u, cw, v, cw, params, dir, var, oy, w,
                                            ou, cw, ov, cw))
        rc |= fail("filter_frame", w, h, bd, fmt);
    if (fmt == 420 && cdef_ref_filter_frame_coded(w, h, bd, y, w, u, cw, v, cw, params, coded, dir,
                                                  var, oy, w, ou, cw, ov, cw))
        rc |= fail("filter_frame_coded", w, h, bd, fmt);
    for (int c = 0; c < 2; c++)
        if (cdef_ref_filter_frame_format(w, h, bd, fmt, y, w, u, cw, v, cw, params, c ? coded : NULL,
                                         dir, var, oy, w, ou, cw, ov, cw))
            rc |= fail("filter_frame_format", w, h, bd, fmt);
    if (tables) {
        const int damping = 3 + (int)(next_u32() % 4);
        if (fmt == 420 && cdef_ref_distortion(w, h, bd, damping, y, w, u, cw, v, cw, sy, w, su, cw,
                                              sv, cw, dl, dc))
            rc |= fail("distortion", w, h, bd, fmt);
        if (fmt == 420 && cdef_ref_distortion_coded(w, h, bd, damping, y, w, u, cw, v, cw, sy, w, su,
                                                    cw, sv, cw, coded, dl, dc, skipped))
            rc |= fail("distortion_coded", w, h, bd, fmt);
        if (fmt == 420 && cdef_ref_distortion_eq14(w, h, bd, damping, y, w, u, cw, v, cw, sy, w, su,
                                                   cw, sv, cw, dl, dc))
            rc |= fail("distortion_eq14", w, h, bd, fmt);
        if (cdef_ref_distortion_format(w, h, bd, damping, fmt, y, w, u, cw, v, cw, sy, w, su, cw, sv,
                                       cw, dl, dc))
            rc |= fail("distortion_format", w, h, bd, fmt);
        if (cdef_ref_distortion_eq14_format(w, h, bd, damping, fmt, y, w, u, cw, v, cw, sy, w, su,
                                            cw, sv, cw, dl, dc))
            rc |= fail("distortion_eq14_format", w, h, bd, fmt);
        if (cdef_ref_distortion_eq14_coded_format(w, h, bd, damping, fmt, y, w, u, cw, v, cw, sy, w,
                                                  su, cw, sv, cw, coded, dl, dc, skipped))
            rc |= fail("distortion_eq14_coded_format", w, h, bd, fmt);
        if (cdef_ref_distortion_coded_format(w, h, bd, damping, fmt, y, w, u, cw, v, cw, sy, w, su,
                                             cw, sv, cw, coded, dl, dc, skipped))
            rc |= fail("distortion_coded_format", w, h, bd, fmt);
    }
    free(y); free(u); free(v); free(sy); free(su); free(sv); free(oy); free(ou); free(ov);
    free(dir); free(coded); free(var); free(params); free(dl); free(dc); free(skipped); free(ids);
    return rc;
}

static int selection_case(int nblocks, int width)
{
    const size_t n = (size_t)nblocks * width;
    int64_t *dl = malloc(sizeof(int64_t) * n), *dc = malloc(sizeof(int64_t) * n);
    uint8_t *skipped = malloc((size_t)nblocks), *ids = malloc((size_t)nblocks);
    int32_t presets[8], np = 0;
    int64_t cost = 0, costs[8], total = 0;
    int passes = 0, rc = 0;
    if (!dl || !dc || !skipped || !ids)
        exit(3);
    for (size_t i = 0; i < n; i++) {
        dl[i] = (int64_t)(next_u32() % 100000);
        dc[i] = (int64_t)(next_u32() % 100000);
    }
    for (int b = 0; b < nblocks; b++)
        skipped[b] = (uint8_t)(next_u32() % 4 == 0);
    for (int mp = 0; mp < 3; mp++) {
        if (cdef_ref_select_presets_general(nblocks, dl, dc, width, skipped, 1000, mp, presets, &np,
                                            ids, &cost))
            rc |= fail("select_presets_general", nblocks, width, mp, 0);
        if (cdef_ref_select_presets_subset(nblocks, dl, dc, width, NULL, 0x8421842184218421ull,
                                           0x0f0f0f0f0f0f0f0full, 500, mp, presets, &np, ids, &cost))
            rc |= fail("select_presets_subset", nblocks, width, mp, 0);
    }
    if (width == 64) {
        if (cdef_ref_select_presets(nblocks, dl, dc, 700, presets, &np, ids, &cost, costs))
            rc |= fail("select_presets", nblocks, width, 0, 0);
        if (cdef_ref_refine_presets(nblocks, dl, dc, presets, 4, 3, &total, &passes))
            rc |= fail("refine_presets", nblocks, width, 0, 0);
        if (cdef_ref_select_presets_refined(nblocks, dl, dc, 700, 2, presets, &np, ids, &cost))
            rc |= fail("select_presets_refined", nblocks, width, 0, 0);
    }
    free(dl); free(dc); free(skipped); free(ids);
    return rc;
}

int main(void)
{
    int rc = 0;
    for (int d = -1023; d <= 1023; d += 7)
        for (int64_t s = 0; s <= 76; s += 3)
            for (int64_t dmp = 3; dmp <= 10; dmp++)
                if (s == 0 || dmp >= 63 - __builtin_clzll((unsigned long long)s))
                    (void)cdef_ref_constrain(d, s, dmp);
    for (int64_t s = -3000; s <= 3000; s++)
        (void)cdef_ref_round16(s);
    for (int s = 0; s < 20; s++)
        for (int64_t v = 0; v < (int64_t)1 << 31; v = v * 3 + 1)
            (void)cdef_ref_adjust_strength(s, v);
    static const int sizes[][2] = {{8, 8}, {24, 16}, {72, 40}};
    static const int fmts[] = {420, 422, 444};
    for (int k = 0; k < 3; k++)
        for (int bd = 8; bd <= 12; bd += 2)
            for (int f = 0; f < 3; f++)
                rc |= frame_case(sizes[k][0], sizes[k][1], bd, fmts[f], k < 2 || bd == 10);
    rc |= selection_case(5, 64);
    rc |= selection_case(3, 128);
    if (!rc)
        printf("oracle under ASan/UBSan: every call succeeded, nothing reported\n");
    return rc;
}
