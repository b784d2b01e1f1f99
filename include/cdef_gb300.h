/*
 * cdef_gb300 -- C ABI of a GB300 (sm_103a) implementation of the hot path of
 * the Constrained Directional Enhancement Filter (CDEF) of
 * Midtskogen & Valin, "The AV1 Constrained Directional Enhancement Filter
 * (CDEF)", arXiv 1602.05975.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Frames are 4:2:0: the luma plane is W x H, both multiples of 8
 *    (section 2 works on 8x8 blocks), the chroma planes W/2 x H/2.
 *    cdef_filter_frame and cdef_filter_frame_coded also take 4:2:2 frames
 *    (chroma W/2 x H: section 4 disables chroma filtering when the
 *    subsampling differs horizontally and vertically, so the chroma planes
 *    are copied) and 4:4:4 frames (chroma W x H: each chroma plane is
 *    filtered in 8x8 blocks with the chroma strengths and damping and the
 *    co-located luma direction).  The format follows from the plane sizes.
 *    An 8/10-bit 4:4:4 frame is one launch in which the three planes of
 *    each 64x64 filter block are filtered in turn (the luma directions
 *    searched first, or read from dir/var); consecutive such calls overlap
 *    under cdef_ctx_set_overlap as 4:2:0 calls do.  A 12-bit 4:4:4 frame
 *    filtered without caller maps (dir = var = NULL) uses the context's
 *    direction-map scratch: such calls on one context belong on one stream
 *    (their launches are then ordered).
 *  - Samples are unsigned integers stored planar and row-major: uint8_t for
 *    bit depth 8, uint16_t (value in the low bits) for bit depths 10 and 12.
 *  - Plane memory is DEVICE memory owned by the caller.  `data` must be
 *    16-byte aligned and `pitch_bytes` a multiple of 16 that is at least
 *    width * sample size (the tiles are moved by the tensor memory
 *    accelerator, which needs both).
 *  - Filter blocks are 64x64 luma (32x32 chroma) pixels (section 4); there
 *    are B = ceil(W/64) * ceil(H/64) of them, numbered row-major.
 *  - 8x8 direction maps are (H/8) x (W/8) arrays, row-major, no padding.
 *  - Every call is asynchronous on the given CUDA stream (cudaStream_t passed
 *    as void*; NULL = the legacy default stream) unless it says otherwise.
 *    Results are valid once the stream reaches the call.  No call aborts or
 *    traps: errors come back as a negative status (cdef_strerror() names
 *    it) and leave the outputs unspecified.
 *  - A context is bound to one device.  Calls on one context must not run
 *    concurrently from several host threads.
 */
#ifndef CDEF_GB300_H
#define CDEF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CDEF_OK 0
#define CDEF_ERR_ARG (-1)      /* NULL pointer, aliasing, bad pitch/alignment, value out of range */
#define CDEF_ERR_SIZE (-2)     /* W or H not a positive multiple of 8, or chroma size != W/2 x H/2 */
#define CDEF_ERR_BITDEPTH (-3) /* bit depth other than 8, 10 or 12, or a plane of the wrong sample size */
#define CDEF_ERR_NOMEM (-4)    /* over the context's device-memory budget, or allocation failed */
#define CDEF_ERR_CUDA (-5)     /* a CUDA runtime/driver call failed */
#define CDEF_ERR_TIMEOUT (-6)  /* a bounded device-side wait gave up */
#define CDEF_ERR_DEVICE (-7)   /* a kernel reported an internal consistency error */

/* One plane: device pointer, size in samples, row pitch in bytes. */
typedef struct {
    void *data;
    int32_t width;
    int32_t height;
    int64_t pitch_bytes;
} cdef_plane;

/* One 4:2:0 frame. */
typedef struct {
    cdef_plane y, u, v;
    int32_t bitdepth; /* 8, 10 or 12 */
} cdef_frame;

/* Parameters of one 64x64 filter block, as signalled (section 3.2, 4):
 *   pri_y, pri_uv : primary strength S^(p), 0..15 (19 accepted: the value
 *                   the (0,0) preset stands for, section 4)
 *   sec_y, sec_uv : secondary strength S^(s) in {0, 1, 2, 4} (7 accepted)
 *   damping       : luma damping D at the 8-bit scale, 3..6; chroma uses
 *                   D - 1 (section 3.2)
 *   skip          : the preset's skip-condition bits (section 4): bit 0
 *                   luma, bit 1 chroma; 0..3.  With a bit set, strengths
 *                   (0, 0) of that plane group stand for (19, 7), and (with
 *                   cdef_filter_frame_coded) 8x8 blocks without coded
 *                   residual are filtered too.
 * Strengths are the 8-bit values; they are scaled by 2^(bitdepth-8) inside
 * (section 3.2).  8 bytes, no padding surprises. */
typedef struct {
    uint8_t pri_y, sec_y, pri_uv, sec_uv;
    uint8_t damping;
    uint8_t skip;
    uint8_t reserved[2];
} cdef_fb_params;

/* One preset of the frame header (section 4), without the skip-condition
 * bits: the primary and secondary strengths for luma and chroma. */
typedef struct {
    uint8_t pri_y, sec_y, pri_uv, sec_uv;
} cdef_preset;

/* One preset with its skip-condition bits (section 4): the strengths as in
 * cdef_preset and skip = bit 0 luma, bit 1 chroma.  Strengths (0, 0) with
 * the plane group's bit set stand for (19, 7).  Converts to cdef_fb_params
 * field for field (pri/sec/skip). */
typedef struct {
    uint8_t pri_y, sec_y, pri_uv, sec_uv;
    uint8_t skip;
    uint8_t reserved[3];
} cdef_preset_coded;

typedef struct cdef_ctx cdef_ctx;

/* Creates a context on CUDA device `device`.  It owns the library's device
 * scratch memory (allocated lazily, never more than hbm_budget_bytes in
 * total; 0 = no limit).  Returns CDEF_OK and *ctx, or an error. */
int cdef_ctx_create(cdef_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Releases the context and its scratch memory.  NULL is accepted.
 * Synchronises the device first. */
int cdef_ctx_destroy(cdef_ctx *ctx);

/* Kernel-reported errors since the last clear.  Strength values out of the
 * ranges above are found on the device (the parameters live in device
 * memory): the block is then left unfiltered and the context's status word
 * is set.  A bounded device-side wait that gave up (tile loads that never
 * arrived) also sets it, leaving its block unwritten.  Waits for all work on
 * the device, then returns CDEF_OK, CDEF_ERR_TIMEOUT or CDEF_ERR_ARG;
 * clear != 0 resets the word. */
int cdef_ctx_status(cdef_ctx *ctx, int clear);

/* The same status word without waiting: enqueues on cuda_stream a copy of
 * it into *host_status (HOST memory; pinned, or the copy is not
 * asynchronous), which holds it once the stream has passed this point.  0
 * means no kernel-reported error; any other value is a nonzero status (read
 * cdef_ctx_status for the code and to clear it).  CDEF_ERR_ARG for NULL
 * arguments, CDEF_ERR_CUDA if the copy cannot be enqueued. */
int cdef_ctx_status_async(cdef_ctx *ctx, int32_t *host_status, void *cuda_stream);

/* Direction search, section 2, eq. 1-5 and Algorithm 1.
 * For every 8x8 block of the luma plane: the direction d in 0..7 that
 * maximises s_d (first maximum on ties) and the directional contrast
 * v = s_best - s_{(best+4) mod 8} >= 0, with s_d in the 840-scaled units of
 * Algorithm 1 (int32 always suffices, section 2).  Samples of bit depth > 8 are brought to 8 bits by an
 * arithmetic right shift first.
 *   luma     : host pointer to the plane descriptor (device samples)
 *   bitdepth : 8, 10 or 12 (must match the plane's sample size)
 *   dir      : device, (H/8)*(W/8) bytes, written
 *   var      : device, (H/8)*(W/8) int32, written
 */
int cdef_find_dir(cdef_ctx *ctx, const cdef_plane *luma, int32_t bitdepth,
                  uint8_t *dir, int32_t *var, void *cuda_stream);

/* The CDEF filter over a whole 4:2:0 frame, section 3 (eq. 6-13):
 * primary taps along the block direction, secondary taps on the cross at
 * +-45 degrees, each through the constraint f(d, S, D) of eq. 7, the
 * weighted sum rounded (ties away from zero) and the result clipped to the
 * range of the filtered pixel and its in-frame taps.  Luma primary
 * strengths are adjusted per 8x8 block by the contrast (eq. 13); chroma
 * 4x4 blocks take the co-located luma direction.  Taps outside the frame
 * are ignored; filter-block borders inside the frame are read across, and
 * only the unfiltered input is ever read.
 *   in      : host pointer to the input frame descriptor (device planes)
 *   params  : DEVICE array of B cdef_fb_params, row-major over filter blocks
 *   dir,var : DEVICE maps from cdef_find_dir, or both NULL: the direction
 *             search then runs inside the filter kernel (fused)
 *   out     : host pointer to the output frame descriptor; same sizes and
 *             bit depth as `in`; its planes must not overlap `in`'s
 */
int cdef_filter_frame(cdef_ctx *ctx, const cdef_frame *in,
                      const cdef_fb_params *params, const uint8_t *dir,
                      const int32_t *var, const cdef_frame *out,
                      void *cuda_stream);

/* The filter with the skip semantics of section 4 (fused direction search):
 *   coded : DEVICE (H/8) x (W/8) bytes, row-major, nonzero where the 8x8
 *           luma block has coded residual (the 4:2:0 chroma 4x4 block
 *           follows its co-located luma block); required.
 * A filter block without any coded 8x8 block is copied unfiltered; in the
 * others an 8x8 block without coded residual is copied unfiltered unless
 * its plane group's skip-condition bit (params.skip) is set.  Otherwise as
 * cdef_filter_frame (which treats every 8x8 block as coded). */
int cdef_filter_frame_coded(cdef_ctx *ctx, const cdef_frame *in,
                            const cdef_fb_params *params, const uint8_t *coded,
                            const cdef_frame *out, void *cuda_stream);

/* The same filter over n frames of possibly different sizes and bit depths
 * in one kernel launch (the fused direction search is always used).
 *   in, out : HOST arrays of n frame descriptors
 *   params  : HOST array of n DEVICE pointers, params[i] has B_i entries
 * n <= 48.  Equivalent to n calls of cdef_filter_frame with dir = NULL. */
int cdef_filter_frames(cdef_ctx *ctx, int32_t n, const cdef_frame *in,
                       const cdef_fb_params *const *params,
                       const cdef_frame *out, void *cuda_stream);

/* Encoder strength search, section 5, for n frames (sizes may differ).
 *
 * First pass: for every filter block b of every frame and each of the 64
 * strength pairs q = p*4 + s (primary p in 0..15, secondary index s for
 * S^(s) in {0,1,2,4}), the distortion D_{b,q} = sum of squared differences
 * between the source and the decoded frame filtered with that pair at the
 * frame's damping, over the block's in-frame pixels; luma and chroma
 * (U + V) separately.  Skip-condition bits are not modelled (every 8x8
 * block counts as coded).
 *
 * Second pass, per frame: presets are (luma pair, chroma pair) tuples,
 * index t = luma_q*64 + chroma_q.  Greedy search for N = 1..8: each step
 * adds the preset minimising sum_b min_{presets} (D^luma_{b,.} +
 * D^chroma_{b,.}), ties to the lowest t; then N in {1, 2, 4, 8}
 * minimising J = lambda*B*log2(N) + that sum (eq. 15; ties to the smaller
 * N), and each block's id = its least-distortion preset (ties to the lower
 * id).
 *
 *   rec, src     : HOST arrays of n frame descriptors (device planes); src
 *                  is the uncoded frame, same sizes and bit depth
 *   damping      : HOST, n luma dampings (3..6), one per frame (section 4)
 *   lambda       : HOST, n non-negative rate multipliers
 *   dist_luma,
 *   dist_chroma  : DEVICE, sum_i B_i * 64 int64 each (frame i's blocks after
 *                  frame i-1's), written; or both NULL (context scratch)
 *   presets      : HOST, n*8 entries; presets[i*8+k] for k < npresets[i]
 *   npresets     : HOST, n entries
 *   block_ids    : DEVICE, sum_i B_i bytes, written
 *   cost         : HOST, n entries: J of the chosen N
 * 1 <= n <= 48; bit depth 8, 10 or 12; chroma format 4:2:0, 4:2:2 or 4:4:4
 * (inferred from the chroma plane sizes as for cdef_filter_frame).  4:2:2
 * chroma is not filtered (section 4), so its entries are the unfiltered
 * error for every pair; 4:4:4 chroma planes are filtered in 8x8 blocks
 * with the chroma strengths and the co-located luma direction.  A call of
 * 8/10-bit 4:4:4 frames only takes the packed 16-bit path one plane per
 * work unit (its direction maps formed first); a call holding any 12-bit
 * or 4:2:2 frame, or mixing 4:4:4 with other formats, computes its tables
 * with 32-bit arithmetic per sample (slower).  Both need (W/8)(H/8) * 5
 * bytes of direction maps per frame in the context.
 * This call synchronises the stream before returning (host outputs).
 */
int cdef_search_strengths(cdef_ctx *ctx, int32_t n, const cdef_frame *rec,
                          const cdef_frame *src, const int32_t *damping,
                          const int64_t *lambda, int64_t *dist_luma,
                          int64_t *dist_chroma, cdef_preset *presets,
                          int32_t *npresets, uint8_t *block_ids, int64_t *cost,
                          void *cuda_stream);

/* The strength search with section 4's skip semantics (section 5 counts
 * 16 x 4 x 2 = 128 combinations per plane group: the skip-condition bit is
 * searched too).  For every filter block the 128 luma and 128 chroma
 * entries q = skip * 64 + p * 4 + s are the squared error, against the
 * source, of what cdef_filter_frame_coded outputs for that preset: with the
 * bit clear the frame's 8x8 blocks without coded residual stay unfiltered,
 * and (p, s) = (0, 0) with the bit set filters with (19, 7).  A filter
 * block without coded residual is never filtered and signals no preset: all
 * its entries are its unfiltered error, it is left out of the sums and of
 * B in J, and its id is 0.  Presets are (luma q, chroma q) pairs, index
 * luma_q * 128 + chroma_q; otherwise as cdef_search_strengths (greedy
 * search, optional re-optimisation, N by J, ids).
 *   coded        : HOST array of n DEVICE maps, (H/8) x (W/8) bytes each,
 *                  nonzero where the 8x8 luma block has coded residual
 *   dist_luma,
 *   dist_chroma  : DEVICE, sum_i B_i * 128 int64 each, or both NULL
 *   presets      : HOST, n*8 entries (first npresets[i] of frame i valid)
 * Frames: as cdef_search_strengths (calls of 8/10-bit 4:4:4 frames only
 * through the packed plane units, 4:2:2, 12-bit and mixed-format calls
 * through the 32-bit path; 4:2:2 chroma entries are the unfiltered error).
 * Synchronises the stream before returning. */
int cdef_search_strengths_coded(cdef_ctx *ctx, int32_t n, const cdef_frame *rec,
                                const cdef_frame *src, const uint8_t *const *coded,
                                const int32_t *damping, const int64_t *lambda,
                                int64_t *dist_luma, int64_t *dist_chroma,
                                cdef_preset_coded *presets, int32_t *npresets,
                                uint8_t *block_ids, int64_t *cost, void *cuda_stream);

/* Launch configuration of the strength search's distortion kernel (the
 * first pass of cdef_search_strengths).  No paper counterpart: it decides
 * how the work is cut, never what is computed -- every configuration gives
 * identical tables, presets, ids and J.
 *   search_groups      : 1, 2 or 4.  The 16 primary strengths of a filter
 *                        block are split into this many work units of
 *                        64/groups luma and 64/groups chroma candidate
 *                        pairs each, so that a small search (few blocks)
 *                        still occupies every SM.
 *   search_ctas_per_sm : 1 or 2 persistent CTAs per SM.
 * A field of 0 means "autotuned": the first search of a batch shape (frame
 * count, sizes and bit depths) on a context times every configuration on
 * that call's own inputs, on the call's stream, and keeps the fastest for
 * the later searches of that shape.
 *   preset_kernel      : the kernel of the preset selection (eq. 15 and the
 *                        re-optimisation); both give identical results.
 *                        0 (default): one thread-block cluster per frame for
 *                        frames of up to 16384 filter blocks, else one
 *                        grid-wide cooperative kernel; 1: always the
 *                        grid-wide kernel.  Not autotuned; set_tuning(NULL)
 *                        resets it to 0. */
typedef struct {
    int32_t search_groups;
    int32_t search_ctas_per_sm;
    int32_t preset_kernel;
    int32_t reserved;      /* 0 */
} cdef_tuning;

/* Fix the configuration (NULL or zero fields: autotune, the default).
 * CDEF_ERR_ARG for a value outside the lists above.  Host only. */
int cdef_ctx_set_tuning(cdef_ctx *ctx, const cdef_tuning *tuning);

/* The configuration the context's last search ran with (search fields
 * zero before the first search; preset_kernel as set).  Host only. */
int cdef_ctx_get_tuning(const cdef_ctx *ctx, cdef_tuning *last);

/* Distortion measure of cdef_search_strengths (section 5):
 *   CDEF_METRIC_SSE  (default) D = sum of squared errors over the block;
 *   CDEF_METRIC_EQ14 D = sum over the 8x8 blocks of each plane (4:2:0 chroma
 *                    8x8 blocks cut by the frame edge use their samples) of
 *                    eq. 14, ((s_var + d_var + C1) / (2 sqrt(s_var d_var +
 *                    C2))) * squared error, with population variances of the
 *                    source and filtered blocks, C1 = 6.25 * 4^(bd-8), C2 =
 *                    312.5 * 16^(bd-8); each 8x8 value in units of 1/256,
 *                    rounded half away from zero after an IEEE
 *                    single-precision evaluation in a fixed order, so that the
 *                    tables are exact integers (an entry of n 8x8 terms is
 *                    within n + 2^-20 (entry + n) of eq. 14 evaluated
 *                    exactly).  Every chroma format and bit depth (4:2:2
 *                    chroma: the unfiltered value for every pair), and the
 *                    128 combinations of cdef_search_strengths_coded (each
 *                    8x8 block's value from what the decoder outputs for
 *                    the preset; formed by the 32-bit path).  Calls of
 *                    8/10-bit 4:4:4 frames only take the packed plane
 *                    units (64 pairs).
 * Host only; applies to later searches on the context. */
#define CDEF_METRIC_SSE 0
#define CDEF_METRIC_EQ14 1
int cdef_ctx_set_search_metric(cdef_ctx *ctx, int metric);

/* Low-complexity strength search (section 5: considering only a subset of
 * the combinations).  Bit p * 4 + s of luma_pairs / chroma_pairs allows the
 * pair (S_p = p, S_s = the s-th of 0, 1, 2, 4) for that plane group; in the
 * 128-combination search it allows the pair with either skip-condition bit.
 * Later cdef_search_strengths / cdef_search_strengths_coded calls on the
 * context evaluate only primaries with an allowed pair, write 0 to the
 * table entries of pairs outside the subset, and choose presets (greedy,
 * re-optimisation) only among those whose luma and chroma pairs are both
 * allowed.  Default: every pair (~0 for both).  A zero mask is CDEF_ERR_ARG.
 * Host only; cdef_search_strengths_noalloc always searches every pair. */
int cdef_ctx_set_search_subset(cdef_ctx *ctx, uint64_t luma_pairs, uint64_t chroma_pairs);

/* Per-stage device times of the strength search (no paper counterpart: a
 * profiling aid).  With timing on, later searches on the context record
 * CUDA events before the distortion-table kernel, between it and the preset
 * selection (greedy search, re-optimisation, choice of N and ids), and after
 * it; cdef_ctx_get_stage_times returns the two stage durations of the last
 * search, in milliseconds.  Returns CDEF_ERR_ARG when no search has run
 * with timing on since it was last enabled; CDEF_ERR_CUDA if the events
 * cannot be created or read.  Host only; timing is off by default (it adds
 * two event records to each search). */
int cdef_ctx_set_stage_timing(cdef_ctx *ctx, int enable);
int cdef_ctx_get_stage_times(cdef_ctx *ctx, float *distortion_ms, float *presets_ms);

/* Preset re-optimisation of cdef_search_strengths (section 5: "iteratively
 * re-optimizing one preset at a time" after the greedy search).  For each
 * N in {2, 4, 8}, starting from the greedy presets 1..N, a pass re-chooses
 * preset k = 1..N in turn as the preset minimising the frame's total with
 * the others fixed (the current preset kept when it attains the minimum,
 * else the lowest index); passes repeat until one changes nothing or
 * max_passes have run.  N, J and the block ids then follow from the
 * re-optimised sets.  0 (the default) = the greedy search alone; at most 16.
 * Host only; applies to later searches on the context. */
int cdef_ctx_set_search_refine(cdef_ctx *ctx, int max_passes);

/* Overlap of consecutive filter calls on one stream.  No paper counterpart.
 * Every cdef_filter_frame / cdef_filter_frames launch lets the next kernel
 * on its stream be scheduled before it ends (programmatic dependent
 * launch).  By default (enable = 0) a filter launch still waits, before it
 * reads or writes any memory, until the previous kernel on the stream has
 * finished and its writes are visible: ordinary stream order.  With
 * enable = 1 the wait is dropped: the filter calls of a run of consecutive
 * filter calls on one stream (no other operation between them) may execute
 * concurrently, a frame's filtering running alongside the previous frame's
 * last CTAs.  The caller then promises that no call of such a run writes
 * memory that another call of the run reads or writes, and that the first
 * call of the run does not depend on a kernel enqueued just before it
 * (independent frames of a decoded sequence, each with its own output).
 * Host only; applies to later calls. */
int cdef_ctx_set_overlap(cdef_ctx *ctx, int enable);

/* The strength search without any memory allocation.  The paper has no
 * counterpart: this is a deployment variant of cdef_search_strengths.
 *
 * Some callers may not allocate device memory once they are running: a
 * codec embedded in a host application that hands it a fixed memory budget
 * up front, or a real-time encoder loop that cannot afford the implicit
 * device-wide synchronisation cudaMalloc/cudaFree may cause.  For them this
 * entry point takes no context and calls no allocating routine.  The only
 * device scratch it needs (one 64-bit running minimum per filter block and
 * 4096 64-bit preset totals per frame for the greedy search, one result
 * record per frame, a work counter) lives in a fixed array inside the
 * library, which every GPU that loads the library holds until the process
 * exits: about 1.63 MiB (CDEF_NOALLOC_MAX_BLOCKS blocks, 48 frames).
 *
 *   - The arguments and results of cdef_search_strengths for 8- and 10-bit
 *     4:2:0 frames, with the default search (squared error, 64 pairs, greedy
 *     presets, no subset), except that there is no context and dist_luma /
 *     dist_chroma are required (device, sum_i B_i * 64 int64 each): the
 *     tables are outputs the caller provides.  Runs on the current device;
 *     the stream must belong to it.
 *   - 12-bit frames return CDEF_ERR_BITDEPTH and 4:2:2 or 4:4:4 frames
 *     CDEF_ERR_SIZE (those take cdef_search_strengths' 32-bit path, which
 *     needs direction-map scratch this variant does not hold).
 *   - At most CDEF_NOALLOC_MAX_BLOCKS filter blocks in total over the n
 *     frames (e.g. 8 frames of 3840x2160); beyond that it returns
 *     CDEF_ERR_NOMEM before doing any work.
 *   - Kernel-reported errors come back as the call's status: CDEF_ERR_TIMEOUT
 *     when a bounded device-side wait gave up, CDEF_ERR_DEVICE for any other
 *     error bit; the outputs are then unspecified.
 *   - The first call on a device looks up the device address of the array
 *     (cudaGetSymbolAddress) with that device current.  No call may be made
 *     while its stream is being captured into a graph: every call waits for
 *     its stream to return its host outputs.
 *   - All calls on a device share the one array and it keeps the last
 *     call's contents (every word the kernels read is written or cleared
 *     earlier in the same call).  Calls whose work overlaps on the GPU -- on
 *     different streams, or from several host threads -- race on it:
 *     serialise them.
 *   - Synchronises the stream before returning (host outputs). */
#define CDEF_NOALLOC_MAX_BLOCKS 16384
int cdef_search_strengths_noalloc(int32_t n, const cdef_frame *rec,
                                  const cdef_frame *src, const int32_t *damping,
                                  const int64_t *lambda, int64_t *dist_luma,
                                  int64_t *dist_chroma, cdef_preset *presets,
                                  int32_t *npresets, uint8_t *block_ids,
                                  int64_t *cost, void *cuda_stream);

/* ------------------------------------------------------------------------
 * The strength search split over devices (section 5, eq. 15).
 *
 * Section 5's tables are per filter block, so a search can be sharded: each
 * device computes the tables of its own band of filter-block rows
 * (cdef_search_tables), and the greedy search, the one-at-a-time
 * re-optimisation, N by J and the block ids are then driven from the host,
 * step by step, with one exchange per step: every device forms the totals
 * over its blocks of all presets (cdef_preset_totals), the host sums them
 * over devices (a collective), and every device takes the same least total
 * (cdef_preset_argmin).  Per-block state stays on its device
 * (cdef_preset_assign).  The totals of a step over several block ranges add
 * up exactly to the totals over their union, so the sharded selection
 * equals cdef_search_strengths' (its host driver is the package's
 * shard.py).  All four are asynchronous on cuda_stream and allocate
 * nothing.
 * ------------------------------------------------------------------------ */

/* Section 5's distortion tables (the first pass of cdef_search_strengths /
 * cdef_search_strengths_coded) for a band of filter-block rows of each of n
 * frames: rows row_begin[i] .. row_begin[i] + row_count[i] - 1 of frame i
 * (HOST arrays; row_count 0 allowed), the blocks of frame i after those of
 * frame i - 1, row-major within the band.  Taps and direction search read
 * the whole frame, so a band's tables equal the same rows of the whole
 * frame's tables.  The context's metric (squared error or eq. 14) and
 * subset apply.
 *   coded, skipped : both NULL (64 pairs) or both set (the 128 combinations
 *                    of cdef_search_strengths_coded): coded = HOST array of
 *                    n DEVICE maps, skipped = DEVICE, one flag per band block
 *   dist_luma,
 *   dist_chroma    : DEVICE, (band blocks) * 64 (or 128) int64 each, written
 * Frames as cdef_search_strengths.  CDEF_ERR_ARG for a band outside the
 * frame. */
int cdef_search_tables(cdef_ctx *ctx, int32_t n, const cdef_frame *rec, const cdef_frame *src,
                       const uint8_t *const *coded, const int32_t *damping,
                       const int32_t *row_begin, const int32_t *row_count, int64_t *dist_luma,
                       int64_t *dist_chroma, uint8_t *skipped, void *cuda_stream);

/* One step's totals over nblocks blocks of tables with `width` (64 or 128)
 * combinations per plane group: for every preset t = luma_q * width +
 * chroma_q (width^2 of them),
 *   totals[t] = sum over blocks b with skipped[b] == 0 of
 *               min(best[b], dist_luma[b][luma_q] + dist_chroma[b][chroma_q])
 *   dist_luma, dist_chroma : DEVICE tables, nblocks * width int64 each
 *   skipped                : DEVICE, nblocks flags, or NULL (none skipped)
 *   best                   : DEVICE, nblocks uint64, or NULL (no bound: the
 *                            first greedy step)
 *   totals                 : DEVICE, width^2 int64, written
 * nblocks 0 gives zero totals. */
int cdef_preset_totals(cdef_ctx *ctx, int32_t nblocks, int32_t width, const int64_t *dist_luma,
                       const int64_t *dist_chroma, const uint8_t *skipped, const uint64_t *best,
                       int64_t *totals, void *cuda_stream);

/* The step's choice from (summed) totals: the least total over the presets
 * whose luma and chroma pairs are allowed (bit q mod 64 of luma_pairs /
 * chroma_pairs, as cdef_ctx_set_search_subset; ~0 for all), the lowest
 * index on ties; in a re-optimisation step `keep` is the slot's current
 * preset, kept when it attains the least total (-1: none).
 *   totals : DEVICE, width^2 int64
 *   result : DEVICE, 2 int64 written: the preset, its total */
int cdef_preset_argmin(cdef_ctx *ctx, int32_t width, const int64_t *totals, uint64_t luma_pairs,
                       uint64_t chroma_pairs, int32_t keep, int64_t *result, void *cuda_stream);

/* Per-block state for a preset set P of npresets (0..8) presets (HOST array
 * `presets`): for each block b,
 *   best[b]      = min over P of D_b (2^64 - 1 when P is empty; 0 when
 *                  skipped), the bound of the next totals;
 *   block_ids[b] = the position in P of the first preset attaining it (0
 *                  when skipped): the block's id once P is final;
 *   sums         = {sum of best[b] over blocks not skipped (0 when P is
 *                  empty), the number of blocks not skipped}: the set's
 *                  total and the B of J.
 * best, block_ids and sums are DEVICE outputs, each may be NULL. */
int cdef_preset_assign(cdef_ctx *ctx, int32_t nblocks, int32_t width, const int64_t *dist_luma,
                       const int64_t *dist_chroma, const uint8_t *skipped, const int32_t *presets,
                       int32_t npresets, uint64_t *best, uint8_t *block_ids, int64_t *sums,
                       void *cuda_stream);

/* Test aid (no paper counterpart): the limits of the kernels' bounded
 * tile-load waits, process-wide, for every launch made after the call.
 *   wait_cycles    : SM clock cycles a CTA waits for a block's tiles before
 *                    it gives up (0 = the default, about 2^28)
 *   extra_tx_bytes : bytes added to every tile load's expected transaction
 *                    count that no load delivers (0..65536; 0 = none), so
 *                    that every wait runs out after wait_cycles
 * A CTA whose wait gives up sets the timeout status (cdef_ctx_status ->
 * CDEF_ERR_TIMEOUT; cdef_search_strengths_noalloc returns it), takes back
 * the undelivered bytes, waits (bounded) for the loads it did issue and
 * leaves; its blocks stay unwritten.  Nothing faults and the context stays
 * usable.  Searches record their launches into a cached graph, which takes
 * the limits of the call that recorded it (a call with other limits is
 * recorded again).  CDEF_ERR_ARG for values out of range.  Host only; not
 * for concurrent use with launches from other host threads. */
int cdef_debug_set_waits(int64_t wait_cycles, int32_t extra_tx_bytes);

/* Test aid (no paper counterpart): the index checks of the library.  The
 * library built with CDEF_DEBUG (libcdef_gb300_debug.so) checks every
 * shared-memory tap load, output staging write and 16-byte row store of
 * the filter and search kernels against its buffer before it is made; an
 * access out of range is skipped (nothing faults), sets the context's
 * status word (cdef_ctx_status -> CDEF_ERR_DEVICE; a search returns it) and
 * is counted on the device.
 *   faults : HOST output, the accesses skipped on ctx's device since the
 *            last clear (always 0 in the release build)
 *   clear  : nonzero = reset the count after reading it
 * Waits for all work on the device first.  Returns 1 when the library was
 * built with the checks, 0 when not, CDEF_ERR_ARG for a NULL argument,
 * CDEF_ERR_CUDA when the device cannot be read. */
int cdef_debug_checks(cdef_ctx *ctx, int64_t *faults, int32_t clear);

/* Measurement aid (no paper counterpart): the integer issue rate of this
 * GPU for the filter's tap instruction mix, the ceiling of the integer-
 * pipe roofline the filter and the strength search are bound by (the
 * library's kernels are otherwise compared with a ceiling derived from the
 * SM count and clock).  A probe kernel runs `iters` steps of 8 independent
 * chains per thread on 4 CTAs of 256 threads per SM; a step is the tap's 6
 * ALU operations (four packed 16-bit min/max/add-min, the shift and its
 * per-lane mask) and 2 multiply-adds (mix 0), or five ALU operations alone
 * (mix 1).  Mixes 2-6 measure the pipes apart, 4 instructions a step: 4
 * integer multiply-adds (2), 4 multiplies-high (3), 2 packed 16-bit maxima
 * and 2 multiply-adds (4), 2 logic operations and 2 multiply-adds (5), 4
 * fp32 FMAs (6).
 *   lane_instr_per_s : HOST output, lane instructions per second (warp
 *                      instructions x 32), from CUDA events around the
 *                      launch after one warm-up launch
 * Synchronises `cuda_stream`.  CDEF_ERR_ARG for mix outside 0..6 or iters
 * outside 1..2^20; CDEF_ERR_CUDA, CDEF_ERR_NOMEM on a runtime failure. */
int cdef_probe_int_mix(cdef_ctx *ctx, int32_t mix, int32_t iters, double *lane_instr_per_s,
                       void *cuda_stream);

/* A static description of a status code. */
const char *cdef_strerror(int status);

/* Library version, e.g. "cdef_gb300 0.1 sm_103a". */
const char *cdef_version(void);

#ifdef __cplusplus
}
#endif
#endif
