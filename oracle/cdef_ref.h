/*
 * CPU oracle for the CDEF hot path (Midtskogen & Valin, "The AV1 Constrained
 * Directional Enhancement Filter (CDEF)", arXiv 1602.05975).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, literal restatement of
 * the paper's definitions in C99 with 64-bit integers.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library; the CUDA
 * path never calls it and must never fall back to it.
 *
 * Samples are passed as uint16_t for every bit depth (8-bit frames are
 * widened by the caller).  Strides are in samples.  Every output buffer is
 * owned by the caller.  Functions return 0 on success and -1 on an argument
 * the paper does not define (the oracle does not try to be forgiving).
 *
 * Parity status of each function is stated in cdef_ref.c.
 */
#ifndef CDEF_REF_H
#define CDEF_REF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Section 2, Fig. 1 (reading): line number k of pixel (row i, column j) of an
 * 8x8 block for direction d = 0..7. */
int cdef_ref_line_number(int d, int i, int j);

/* Algorithm 1 on one 8x8 block of centred 8-bit values x[i*8+j] in
 * [-128, 127]: writes s[d] = 840 * s_d (eq. 5 scaled by 840). */
void cdef_ref_direction_costs(const int32_t x[64], int64_t s[8]);

/* Algorithm 1 on one 8x8 block of raw samples at bit depth bd (section 2:
 * high bit depths are brought down to 8 bits first).  Returns the direction
 * and writes the directional contrast v. */
int cdef_ref_find_dir_block(const uint16_t *p, ptrdiff_t stride, int bitdepth,
                            int64_t *contrast);

/* Algorithm 1 over every 8x8 block of a luma plane (w, h multiples of 8).
 * dir and var are (h/8) x (w/8), row-major. */
int cdef_ref_find_dir(const uint16_t *luma, int w, int h, ptrdiff_t stride,
                      int bitdepth, uint8_t *dir, int32_t *var);

/* Eq. 7: the constraint function f(d, S, D), with the anti-symmetric reading
 * of its d < 0 branch.  S = 0 gives 0. */
int64_t cdef_ref_constrain(int64_t diff, int64_t strength, int64_t damping);

/* Eq. 13: luma primary strength adjusted by the directional contrast v. */
int cdef_ref_adjust_strength(int strength, int64_t contrast);

/* Eq. 8: round(sum / 16), ties away from zero. */
int64_t cdef_ref_round16(int64_t sum);

/* Per-8x8 effective parameters (section 3.2): the strengths after contrast
 * adjustment (luma) and bit-depth scaling, the damping after the chroma
 * offset, the raise to floor(log2 S_p) and the bit-depth offset, and the
 * parity that picks the primary weights.  Exposed for tests. */
typedef struct {
    int64_t pri, sec;   /* scaled strengths used by eq. 7 */
    int64_t damping;    /* D used by eq. 7 */
    int parity;         /* 0 even, 1 odd (before scaling) */
} cdef_ref_eff_params;
void cdef_ref_block_params(int pri_raw, int sec_raw, int damping_luma,
                           int is_chroma, int bitdepth, int64_t contrast,
                           cdef_ref_eff_params *out);

/* Eq. 8-12 for one output sample at (row i, col j) of a plane of size w x h,
 * for direction d and the effective parameters e. */
int64_t cdef_ref_filter_sample(const uint16_t *plane, int w, int h,
                               ptrdiff_t stride, int i, int j, int d,
                               const cdef_ref_eff_params *e);

/* Per 64x64 filter block parameters: 8 bytes each, row-major over the
 * ceil(H/64) x ceil(W/64) filter-block grid:
 *   byte 0 luma primary strength, 1 luma secondary strength,
 *   byte 2 chroma primary strength, 3 chroma secondary strength,
 *   byte 4 luma damping (8-bit scale),
 *   byte 5 skip-condition bits of the presets (section 4): bit 0 luma,
 *          bit 1 chroma; bytes 6..7 unused. */
#define CDEF_REF_PARAM_BYTES 8

/* Filters one 4:2:0 frame (section 3): luma w x h, chroma w/2 x h/2.
 * dir/var are the luma 8x8 maps from cdef_ref_find_dir. */
int cdef_ref_filter_frame(int w, int h, int bitdepth,
                          const uint16_t *y, ptrdiff_t ys,
                          const uint16_t *u, ptrdiff_t us,
                          const uint16_t *v, ptrdiff_t vs,
                          const uint8_t *params,
                          const uint8_t *dir, const int32_t *var,
                          uint16_t *oy, ptrdiff_t oys,
                          uint16_t *ou, ptrdiff_t ous,
                          uint16_t *ov, ptrdiff_t ovs);

/* The filter with the skip semantics of section 4 (readings R18-R20 in
 * cdef_ref.c): `coded` marks the 8x8 luma blocks with coded residual
 * ((h/8) x (w/8) bytes, nonzero = coded; NULL = all coded). */
int cdef_ref_filter_frame_coded(int w, int h, int bitdepth,
                                const uint16_t *y, ptrdiff_t ys,
                                const uint16_t *u, ptrdiff_t us,
                                const uint16_t *v, ptrdiff_t vs,
                                const uint8_t *params, const uint8_t *coded,
                                const uint8_t *dir, const int32_t *var,
                                uint16_t *oy, ptrdiff_t oys,
                                uint16_t *ou, ptrdiff_t ous,
                                uint16_t *ov, ptrdiff_t ovs);

/* Chroma formats (reading R25 in cdef_ref.c): format 420, 422 (chroma
 * planes w/2 x h, not filtered) or 444 (chroma planes w x h, filtered in
 * 8x8 blocks with the chroma strengths and the luma directions). */
int cdef_ref_filter_frame_format(int w, int h, int bitdepth, int format,
                                 const uint16_t *y, ptrdiff_t ys,
                                 const uint16_t *u, ptrdiff_t us,
                                 const uint16_t *v, ptrdiff_t vs,
                                 const uint8_t *params, const uint8_t *coded,
                                 const uint8_t *dir, const int32_t *var,
                                 uint16_t *oy, ptrdiff_t oys,
                                 uint16_t *ou, ptrdiff_t ous,
                                 uint16_t *ov, ptrdiff_t ovs);

/* Section 5, two-pass search, first pass: for each filter block b and each of
 * the 64 (primary 0..15) x (secondary {0,1,2,4}) pairs, the SSE between the
 * source and the decoded frame filtered with that pair at damping D.
 * dist_luma[b*64 + p*4 + s_idx], dist_chroma likewise (U + V). */
int cdef_ref_distortion(int w, int h, int bitdepth, int damping,
                        const uint16_t *ry, ptrdiff_t rys,
                        const uint16_t *ru, ptrdiff_t rus,
                        const uint16_t *rv, ptrdiff_t rvs,
                        const uint16_t *sy, ptrdiff_t sys,
                        const uint16_t *su, ptrdiff_t sus,
                        const uint16_t *sv, ptrdiff_t svs,
                        int64_t *dist_luma, int64_t *dist_chroma);

/* Section 5, eq. 15 and the greedy preset search over nblocks blocks.
 * presets[k] = luma_pair * 64 + chroma_pair, k < 8 (all 8 greedy steps are
 * written); *npresets is the chosen N in {1,2,4,8}; block_ids[b] the preset
 * index of block b; *cost = J(N); costs[n-1] = J(n) for n = 1..8 (log2 n is
 * only defined as an integer for n in {1,2,4,8}; other entries hold the
 * distortion term alone). */
int cdef_ref_select_presets(int nblocks, const int64_t *dist_luma,
                            const int64_t *dist_chroma, int64_t lambda,
                            int32_t *presets, int32_t *npresets,
                            uint8_t *block_ids, int64_t *cost,
                            int64_t *costs);

/* Section 5: iterative re-optimisation of one preset at a time (reading
 * R17 in cdef_ref.c), on n presets (in/out), at most max_passes passes. */
int cdef_ref_refine_presets(int nblocks, const int64_t *dist_luma,
                            const int64_t *dist_chroma, int32_t *presets, int n,
                            int max_passes, int64_t *total, int *passes);

/* Greedy search, then the refinement for each N in {1, 2, 4, 8}, then N
 * by J and the block ids (max_passes = 0: the greedy result). */
int cdef_ref_select_presets_refined(int nblocks, const int64_t *dist_luma,
                                    const int64_t *dist_chroma, int64_t lambda,
                                    int max_passes, int32_t *presets,
                                    int32_t *npresets, uint8_t *block_ids,
                                    int64_t *cost);

/* Section 5 with section 4's skip semantics (reading R21 in cdef_ref.c):
 * per filter block 128 luma and 128 chroma combinations q = k*64 + p*4 + s
 * (k the skip-condition bit; (0,0) with k = 1 is (19,7)), computed on the
 * decoder's output for `coded` ((h/8) x (w/8) bytes, nonzero = coded
 * residual; NULL = all coded).  skipped[b] = 1 for filter blocks without
 * coded residual (entries = unfiltered SSE). */
int cdef_ref_distortion_coded(int w, int h, int bitdepth, int damping,
                              const uint16_t *ry, ptrdiff_t rys,
                              const uint16_t *ru, ptrdiff_t rus,
                              const uint16_t *rv, ptrdiff_t rvs,
                              const uint16_t *sy, ptrdiff_t sys,
                              const uint16_t *su, ptrdiff_t sus,
                              const uint16_t *sv, ptrdiff_t svs,
                              const uint8_t *coded, int64_t *dist_luma,
                              int64_t *dist_chroma, uint8_t *skipped);

/* Greedy search, optional re-optimisation, N by J and block ids over tables
 * of `width` (64 or 128) combinations per plane group; blocks with
 * skipped[b] set (or none when NULL) are left out of every sum and of B. */
int cdef_ref_select_presets_general(int nblocks, const int64_t *dist_luma,
                                    const int64_t *dist_chroma, int width,
                                    const uint8_t *skipped, int64_t lambda, int max_passes,
                                    int32_t *presets, int32_t *npresets,
                                    uint8_t *block_ids, int64_t *cost);

/* The same over the presets whose luma and chroma combinations are both
 * allowed: bit p * 4 + s of luma_pairs / chroma_pairs (applied to both
 * skip-bit halves when width = 128); both masks non-zero (reading R26). */
int cdef_ref_select_presets_subset(int nblocks, const int64_t *dist_luma,
                                   const int64_t *dist_chroma, int width,
                                   const uint8_t *skipped, uint64_t luma_pairs,
                                   uint64_t chroma_pairs, int64_t lambda, int max_passes,
                                   int32_t *presets, int32_t *npresets,
                                   uint8_t *block_ids, int64_t *cost);

/* Section 5's 64-pair tables for chroma format 420, 422 (chroma not
 * filtered: its entries are the unfiltered error) or 444 (chroma planes
 * filtered in the luma geometry), at bit depths 8-12 (reading R25). */
int cdef_ref_distortion_format(int w, int h, int bitdepth, int damping, int format,
                               const uint16_t *ry, ptrdiff_t rys,
                               const uint16_t *ru, ptrdiff_t rus,
                               const uint16_t *rv, ptrdiff_t rvs,
                               const uint16_t *sy, ptrdiff_t sys,
                               const uint16_t *su, ptrdiff_t sus,
                               const uint16_t *sv, ptrdiff_t svs,
                               int64_t *dist_luma, int64_t *dist_chroma);

/* The 128-combination tables (reading R21) for chroma format 420, 422 or
 * 444 at bit depths 8-12 (reading R25); skipped[b] as
 * cdef_ref_distortion_coded. */
int cdef_ref_distortion_coded_format(int w, int h, int bitdepth, int damping, int format,
                                     const uint16_t *ry, ptrdiff_t rys,
                                     const uint16_t *ru, ptrdiff_t rus,
                                     const uint16_t *rv, ptrdiff_t rvs,
                                     const uint16_t *sy, ptrdiff_t sys,
                                     const uint16_t *su, ptrdiff_t sus,
                                     const uint16_t *sv, ptrdiff_t svs,
                                     const uint8_t *coded, int64_t *dist_luma,
                                     int64_t *dist_chroma, uint8_t *skipped);

/* Section 5, eq. 14 (readings R22-R24 in cdef_ref.c): per filter block, 64
 * luma and 64 chroma entries sum_8x8 round(256 * D_8x8). */
int cdef_ref_distortion_eq14(int w, int h, int bitdepth, int damping,
                             const uint16_t *ry, ptrdiff_t rys,
                             const uint16_t *ru, ptrdiff_t rus,
                             const uint16_t *rv, ptrdiff_t rvs,
                             const uint16_t *sy, ptrdiff_t sys,
                             const uint16_t *su, ptrdiff_t sus,
                             const uint16_t *sv, ptrdiff_t svs,
                             int64_t *dist_luma, int64_t *dist_chroma);

/* Eq. 14 tables for chroma format 420, 422 or 444 at any bit depth
 * (readings R22-R25); 4:2:2 chroma entries are the unfiltered value. */
int cdef_ref_distortion_eq14_format(int w, int h, int bitdepth, int damping, int format,
                                    const uint16_t *ry, ptrdiff_t rys,
                                    const uint16_t *ru, ptrdiff_t rus,
                                    const uint16_t *rv, ptrdiff_t rvs,
                                    const uint16_t *sy, ptrdiff_t sys,
                                    const uint16_t *su, ptrdiff_t sus,
                                    const uint16_t *sv, ptrdiff_t svs,
                                    int64_t *dist_luma, int64_t *dist_chroma);

/* Eq. 14 tables of the 128 combinations with section 4's skip semantics for
 * chroma format 420, 422 or 444 (readings R21-R25): layout and skipped flags
 * as cdef_ref_distortion_coded_format. */
int cdef_ref_distortion_eq14_coded_format(int w, int h, int bitdepth, int damping, int format,
                                          const uint16_t *ry, ptrdiff_t rys,
                                          const uint16_t *ru, ptrdiff_t rus,
                                          const uint16_t *rv, ptrdiff_t rvs,
                                          const uint16_t *sy, ptrdiff_t sys,
                                          const uint16_t *su, ptrdiff_t sus,
                                          const uint16_t *sv, ptrdiff_t svs,
                                          const uint8_t *coded, int64_t *dist_luma,
                                          int64_t *dist_chroma, uint8_t *skipped);

/* round(256 * D_8x8) of eq. 14 from one 8x8 block's sums over its n
 * in-frame samples: source sum and sum of squares, filtered sum and sum of
 * squares, squared error. */
int64_t cdef_ref_eq14_term(int64_t n, int64_t s1s, int64_t s2s, int64_t s1d, int64_t s2d,
                           int64_t sse, int bitdepth);

#ifdef __cplusplus
}
#endif
#endif
