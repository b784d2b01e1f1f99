// Internal (not exported) descriptors and launchers shared by the C-ABI
// layer and the kernels of cdef_gb300.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cdef_gb300.h"

namespace cdefgb {

constexpr int kMaxBatch = 48;        // frames per batched search launch (kernel-parameter space)
constexpr int kMaxFilterBatch = 48;  // frames per batched filter launch (kernel-parameter space)

// One plane as a kernel sees it.
struct PlaneDev {
    const uint8_t *in;   // input samples (device)
    uint8_t *out;        // output samples (device); unused by the search
    int64_t in_pitch;    // bytes
    int64_t out_pitch;   // bytes
    int w, h;            // samples
};

// One frame of a filter launch.
struct FilterFrameDev {  // aligned as CUtensorMap requires
    CUtensorMap tmap[3];             // 2-D tile maps of the y, u, v input planes
    PlaneDev p[3];                   // y, u, v
    const cdef_fb_params *params;    // B entries
    const uint8_t *dir;              // optional 8x8 maps (NULL: fused search)
    const int32_t *var;
    const uint8_t *coded;            // optional 8x8 coded-residual map (NULL: all coded)
    int mode;                        // 0: 4:2:0 luma + chroma; 1: the luma plane alone;
                                     // 2: a full-resolution (4:4:4) chroma plane in the
                                     //    luma slot, with maps (chroma parameters);
                                     // 3: an 8/10-bit 4:4:4 frame, its three planes
                                     //    (p[0..2], each map with the luma box) filtered
                                     //    in turn per filter block
    int bitdepth;
    int fb_cols, fb_rows;
    int block_start;                 // first CTA index of this frame
};

// Limits of the kernels' bounded tile-load waits.  `wait_cycles` is how long
// a CTA waits for a block's tiles before it gives up (sets the timeout
// status bit, waits for its own loads in flight and leaves); `extra_tx`
// bytes are added to every tile load's expected transaction count, bytes no
// load delivers, so that the wait runs out (a test aid: 0 outside tests).
struct WaitLimits {
    long long wait_cycles;
    int extra_tx;
    int pad;
};
constexpr long long kDefaultWaitCycles = 1ll << 28;   // ~0.13 s at 2 GHz
// The process-wide limits every launch takes (cdef_debug_set_waits).
WaitLimits wait_limits();

template <int MAXF>
struct FilterBatch {
    int n;
    int total_blocks;
    WaitLimits waits = {kDefaultWaitCycles, 0, 0};
    FilterFrameDev f[MAXF];
};

// One frame of a strength search launch.
struct SearchFrameDev {  // aligned as CUtensorMap requires
    CUtensorMap tmap[3];             // 2-D tile maps of the decoded y, u, v planes
    const uint8_t *rec[3];
    const uint8_t *src[3];
    int64_t rec_pitch[3], src_pitch[3];
    int w, h;                        // luma size
    int bitdepth;
    int damping;
    int fb_cols, fb_rows;            // fb_rows: rows of filter blocks searched (a band)
    int block_start;                 // first filter block of this frame in the tables
    int fb_row0 = 0;                 // first filter-block row of the band in the frame
    long long lambda;
    const uint8_t *coded;            // 8x8 coded-residual map (128-combination search only)
    int chroma_format = 420;         // 420, 422 or 444 (formats other than 4:2:0: wide tables)
    int map_start = 0;               // first 8x8 block of this frame in the direction maps
    // allowed (S_p, S_s) pairs of the luma and the chroma group, bit p * 4 + s
    // (section 5's low-complexity search; all ones: every pair)
    unsigned long long pairs[2] = {~0ull, ~0ull};
};

struct SearchBatch {
    int n;
    int total_blocks;
    // 8/10-bit 4:4:4 frames searched one plane per work unit in the packed
    // layout (squared error, 64 pairs); the direction maps are formed first
    int planes = 0;
    WaitLimits waits = {kDefaultWaitCycles, 0, 0};
    SearchFrameDev f[kMaxBatch];
};
static_assert(sizeof(SearchBatch) <= 32764, "a search batch must fit the kernel parameter space");

// The allowed pairs of plane group g (0 luma, 1 chroma); an empty set is
// read as every pair.
__host__ __device__ inline unsigned long long allowed_pairs(const SearchFrameDev &F, int g)
{
    const unsigned long long v = g ? F.pairs[1] : F.pairs[0];   // no indexed parameter access
    return v ? v : ~0ull;
}

// Per-frame result of the preset search (device).
struct SearchResultDev {
    int presets[8];          // the chosen set (first npresets entries)
    long long cost;          // J of the chosen N
    int npresets;
    int pad;
    int greedy[8];           // greedy order
    long long totals[8];     // greedy totals over the first 1..8 presets
    int refined[4][8];       // per N = 1, 2, 4, 8: the (re-optimised) set
    long long ref_totals[4];
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_find_dir(const uint8_t *luma, int64_t pitch, int w, int h,
                            int bitdepth, uint8_t *dir, int32_t *var,
                            cudaStream_t s);
// `work` is a pair of zeroed device counters owned by this launch until it
// completes (the kernel leaves them zeroed again).  Launches are
// programmatic dependents of the previous grid on the stream; with
// `overlap` false each waits for that grid's completion before touching
// memory, with `overlap` true (the caller's promise that consecutive calls
// are independent) it runs alongside the previous grid's last CTAs.
cudaError_t launch_filter_single(const FilterBatch<1> &b, int *status, unsigned *work,
                                 bool overlap, cudaStream_t s);
cudaError_t launch_filter_batch(const FilterBatch<kMaxFilterBatch> &b, int *status,
                                unsigned *work, bool overlap, cudaStream_t s);
// One 8/10-bit 4:4:4 frame in mode 3 (its own kernel instantiation).
cudaError_t launch_filter_444(const FilterBatch<1> &b, int *status, unsigned *work, bool overlap,
                              cudaStream_t s);
// The three planes of a 4:4:4 frame (entries in modes 1, 2, 2) in one launch.
cudaError_t launch_filter_planes(const FilterBatch<3> &b, int *status, unsigned *work,
                                 bool overlap, cudaStream_t s);
constexpr int kWorkSlots = 1024;  // counter pairs per context (launches in flight at once)

// Filter tile geometry shared by the host (tensor-map boxes) and the kernel.
// The luma box starts 8 (16-bit) or 16 (8-bit) columns left of the filter
// block so that its first column is 16-byte aligned, and 2 rows above.
constexpr int kLumaBoxRows = 68;
constexpr int kChromaBoxRows = 36;
__host__ __device__ constexpr int luma_box_cols(int bytes) { return bytes == 2 ? 80 : 96; }
__host__ __device__ constexpr int chroma_box_cols(int bytes) { return bytes == 2 ? 48 : 64; }
__host__ __device__ constexpr int box_lead(int bytes) { return bytes == 2 ? 8 : 16; }
// Launch configuration of the distortion kernel.  `groups` (1, 2 or 4):
// the 16 primary strengths of a filter block are split into this many work
// units (64 / groups luma and as many chroma candidates each), which gives
// small searches more units than there are SMs; `ctas_per_sm` (1 or 2):
// persistent CTAs per SM.  Every configuration computes the same tables.
struct SearchTune {
    int groups;
    int ctas_per_sm;
};
constexpr SearchTune kSearchTunes[] = {{1, 2}, {1, 1}, {2, 2}, {4, 2}};
constexpr int kNumSearchTunes = sizeof(kSearchTunes) / sizeof(kSearchTunes[0]);
// The configuration used without timing: enough work units to give every
// persistent CTA a few of them.
inline SearchTune default_search_tune(int total_blocks, int sms)
{
    if (total_blocks >= 4 * 2 * sms) return {1, 2};
    if (2 * total_blocks >= 4 * 2 * sms) return {2, 2};
    return {4, 2};
}

// Strength search: distortion tables, then the greedy preset search.
// Device scratch: `cur` one u64 per block, `tot` 4096 u64 per frame (zeroed
// by the call itself), `work` a zeroed counter pair (left zeroed).
// `refine_passes`: 0 = the greedy presets; > 0 = then re-optimise each set
// one preset at a time for at most that many passes (section 5).
// `wide_dirs` / `wide_vars` non-null: the tables come from
// launch_search_wide (4:2:2, 4:4:4 or 12-bit frames; 64 combinations), the
// direction maps written there.
// `stage_events` non-null: three events recorded before the distortion
// kernel, between it and the preset selection, and after it (event nodes
// when the stream is being captured into a graph).
// `grid_presets`: the preset selection in the grid-wide kernel even where
// the cluster-per-frame kernel applies.
// `skipped` non-null: the 128-combination search of section 5 with section
// 4's skip semantics (each frame's `coded` map; tables of 128 entries per
// block; `skipped` receives one flag per block); null: 64 combinations.
cudaError_t launch_search(const SearchBatch &b, long long *dist_luma,
                          long long *dist_chroma, unsigned long long *cur,
                          unsigned long long *tot, SearchResultDev *results,
                          uint8_t *block_ids, int *status, unsigned *work, SearchTune tune,
                          int refine_passes, cudaStream_t s, uint8_t *skipped = nullptr,
                          const cudaEvent_t *stage_events = nullptr,
                          uint8_t *wide_dirs = nullptr, int32_t *wide_vars = nullptr,
                          bool grid_presets = false, bool tables_only = false);
// Section 5's tables for 4:2:2, 4:4:4 and 12-bit frames (32-bit arithmetic
// per sample): the direction maps of every frame into `dirs` / `vars` (at
// each frame's map_start), then one CTA per filter block and plane group.
// `skipped` non-null: the 128-combination tables over each frame's coded
// map (one flag per filter block written); null: 64 combinations.  `eq14`:
// section 5's eq. 14 tables instead of the squared error (64 combinations).
// `status`: the search's status word (the index-checking build records
// out-of-range tap loads there).
cudaError_t launch_search_wide(const SearchBatch &b, uint8_t *dirs, int32_t *vars,
                               long long *dist_luma, long long *dist_chroma, uint8_t *skipped,
                               cudaStream_t s, bool eq14, int *status);
// The preset selection (greedy, then up to `refine_passes` re-optimisation
// passes), one cluster of 8 CTAs per frame (no grid-wide barrier);
// preset_cluster_fits: every frame's blocks fit the kernel's per-CTA state.
// `width` 64 or 128 and `skipped` as for launch_presets.
bool preset_cluster_fits(const SearchBatch &b);
// `narrow`: every table entry is below 2^32 (the squared error of 8-bit frames).
cudaError_t launch_presets_cluster(const SearchBatch &b, const long long *dl, const long long *dc,
                                   SearchResultDev *results, uint8_t *block_ids, bool narrow,
                                   int refine_passes, int width, const uint8_t *skipped,
                                   cudaStream_t s);
// The preset selection alone (one cooperative launch); `ctl` is the control
// block that follows `tot` in the scratch.
// `width`: combinations per plane group in the tables (64 or 128; presets
// are width * width); `skipped` (may be null): blocks left out of the sums.
cudaError_t launch_presets(const SearchBatch &b, const long long *dl, const long long *dc,
                           unsigned long long *cur, unsigned long long *tot, void *ctl,
                           SearchResultDev *results, uint8_t *block_ids, int *status,
                           int refine_passes, int width, const uint8_t *skipped,
                           cudaStream_t s);
size_t preset_ctl_bytes();
constexpr int kMaxRefinePasses = 16;
constexpr size_t kPresetCtlBytes = 512;   // barrier and per-frame flags of launch_presets
// Scratch of one search: `cur` one u64 per block, `tot` 4096 u64 per frame,
// then the preset kernel's control block.
constexpr size_t search_scratch_bytes(int nframes, int nblocks, int width = 64)
{
    return sizeof(unsigned long long) * ((size_t)nblocks + (size_t)nframes * width * width) +
           kPresetCtlBytes + (width == 128 ? ((size_t)nblocks + 15) / 16 * 16 : 0);
}

// Pieces of the preset selection (eq. 15 and its re-optimisation) over a
// block range of distortion tables, for a selection driven from the host
// (a search sharded over devices, whose per-step totals are summed by a
// collective).  `width` 64 or 128; presets t = luma_q * width + chroma_q.
// totals[t] += sum over blocks b not skipped of min(best[b], D_b(t)), for
// all width^2 presets (best null: no bound).
cudaError_t launch_preset_totals(int nblocks, int width, const long long *dl, const long long *dc,
                                 const uint8_t *skipped, const unsigned long long *best,
                                 long long *totals, cudaStream_t s);
// out[0] = the least allowed preset (lowest index on ties; `keep` >= 0 is
// kept when it attains the least total), out[1] = its total.
cudaError_t launch_preset_argmin(int width, const long long *totals, unsigned long long luma_pairs,
                                 unsigned long long chroma_pairs, int keep, long long *out,
                                 cudaStream_t s);
// Per block: best[b] = min over the n presets of D_b (no preset: 2^64 - 1;
// skipped: 0), ids[b] = the first preset attaining it (skipped: 0);
// sums[0] += sum of best over blocks not skipped, sums[1] += their count.
struct PresetList {
    int t[8];
    int n;
};
cudaError_t launch_preset_assign(int nblocks, int width, const long long *dl, const long long *dc,
                                 const uint8_t *skipped, PresetList set, unsigned long long *best,
                                 uint8_t *ids, long long *sums, cudaStream_t s);

// The integer-issue probe (probe.cu): lane instructions per second of the
// filter's tap mix (mix 0) or of its ALU operations alone (mix 1).
int probe_int_mix(int device, int mix, int iters, double *lane_instr_per_s, cudaStream_t s);

// Host: the three 2-D tile maps (filter-block boxes with halo) of a frame's
// planes; returns a CDEF status.
int encode_frame_tiles(CUtensorMap maps[3], const cdef_frame *f);

// Device status word values (set by kernels, read by the host).
constexpr int kStatusBadParams = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusMisaligned = 4;  // internal: shared memory not aligned for tile loads
constexpr int kStatusIndex = 8;       // index-checking build (CDEF_DEBUG): an access out of
                                      // its buffer was found and skipped

// Index checks of the CDEF_DEBUG build: CDEF_IN_BOUNDS(i, n, status) is i
// in [0, n); when it is not, the status word gets kStatusIndex, the
// translation unit's fault counter is incremented and the caller skips the
// access.  Without CDEF_DEBUG the check is compiled out (always true).
// CDEF_FAULT_COUNTER(name) defines `unsigned long long name(bool clear)`,
// the host reader of the counter of the translation unit it is placed in
// (always 0 without CDEF_DEBUG).
#ifdef CDEF_DEBUG
static __device__ unsigned long long g_index_faults;   // one per translation unit

__device__ __noinline__ static void note_index_fault(int *status)
{
    atomicOr(status, kStatusIndex);
    atomicAdd(&g_index_faults, 1ull);
}

#define CDEF_IN_BOUNDS(i, n, status) \
    (((long long)(i) >= 0 && (long long)(i) < (long long)(n)) ? true : (note_index_fault(status), false))
#define CDEF_DEBUG_PARAM(decl) , decl
#define CDEF_DEBUG_ARG(name) , name
#define CDEF_FAULT_COUNTER(name)                                                       \
    unsigned long long name(bool clear)                                                 \
    {                                                                                   \
        unsigned long long v = 0, zero = 0;                                             \
        if (cudaMemcpyFromSymbol(&v, g_index_faults, sizeof(v)) != cudaSuccess) return ~0ull; \
        if (clear && v) cudaMemcpyToSymbol(g_index_faults, &zero, sizeof(zero));        \
        return v;                                                                       \
    }
constexpr bool kIndexChecks = true;
#else
#define CDEF_IN_BOUNDS(i, n, status) true
// release build: the status word is not threaded through device helpers,
// so their register allocation is the same as without the checks
#define CDEF_DEBUG_PARAM(decl)
#define CDEF_DEBUG_ARG(name)
#define CDEF_FAULT_COUNTER(name) \
    unsigned long long name(bool) { return 0; }
constexpr bool kIndexChecks = false;
#endif
// the counters of the translation units with checked accesses
unsigned long long index_faults_filter(bool clear);
unsigned long long index_faults_search(bool clear);
unsigned long long index_faults_search_wide(bool clear);

}  // namespace cdefgb
