// C ABI of cdef_gb300: argument validation, the context (device scratch and
// pinned staging), and the launches.  See include/cdef_gb300.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>

#include "cdef_internal.h"

using namespace cdefgb;

struct cdef_ctx {
    int device;
    size_t budget;        // 0 = unlimited
    size_t used;          // bytes of device scratch held
    int *status;          // device status word (kernel-reported errors)
    void *scratch;        // search scratch (distortion tables, greedy state)
    size_t scratch_bytes;
    SearchResultDev *host_results;  // pinned
    SearchResultDev *dev_results;
    unsigned *work;       // kWorkSlots pairs of filter work counters (zeroed)
    unsigned next_slot;   // next pair handed to a launch
    cudaStream_t capture; // records the search's launches into a graph
    cudaGraphExec_t search_exec;  // the last search graph, updated per call
    SearchBatch *search_key;      // what search_exec was recorded for
    void *search_ptrs[7];         // and its tables, ids, scratch and direction-map pointers
    SearchTune search_key_tune;   // and its launch configuration
    SearchTune forced;            // fields > 0 fixed by cdef_ctx_set_tuning
    SearchTune last;              // configuration of the last search
    bool overlap;                 // filter calls on a stream declared independent
    int refine_passes;            // preset re-optimisation passes of the search (0 = greedy)
    int metric;                   // search distortion: 0 squared error, 1 eq. 14
    uint64_t pairs[2];            // allowed (S_p, S_s) pairs of the search (luma, chroma)
    int search_key_refine;        // refine_passes search_exec was recorded with
    bool grid_presets;            // preset selection always in the grid-wide kernel
    bool search_key_grid;         // and what search_exec was recorded with
    bool stage_timing;            // record stage events in the search graph
    bool search_key_timing;       // and whether search_exec holds them
    bool stage_valid;             // the events hold the last search's stages
    cudaEvent_t stage_ev[3];      // before the tables, between, after the presets
    std::unordered_map<uint64_t, SearchTune> *tuned;  // autotuned, per batch shape
    uint8_t *maps_dir;            // direction maps of 4:4:4 filtering
    int32_t *maps_var;
    size_t maps_blocks;
    uint8_t *smaps_dir;           // direction maps of the wide strength search
    int32_t *smaps_var;
    size_t smaps_blocks;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int sample_bytes(int bitdepth) { return bitdepth == 8 ? 1 : 2; }

int check_plane(const cdef_plane &p, int w, int h, int bytes)
{
    if (!p.data) return CDEF_ERR_ARG;
    if (p.width != w || p.height != h) return CDEF_ERR_SIZE;
    if (reinterpret_cast<uintptr_t>(p.data) % 16) return CDEF_ERR_ARG;
    if (p.pitch_bytes <= 0 || p.pitch_bytes % 16 || p.pitch_bytes < (int64_t)w * bytes)
        return CDEF_ERR_ARG;
    return CDEF_OK;
}

// Chroma format from the plane sizes: 420 (W/2 x H/2), 422 (W/2 x H),
// 444 (W x H); 0 for anything else.
int chroma_format(const cdef_frame *f)
{
    const int w = f->y.width, h = f->y.height, cw = f->u.width, ch = f->u.height;
    if (cw == w / 2 && ch == h / 2) return 420;
    if (cw == w / 2 && ch == h) return 422;
    if (cw == w && ch == h) return 444;
    return 0;
}

// `formats`: bit 0 4:2:0, bit 1 4:2:2, bit 2 4:4:4 accepted.
int check_frame(const cdef_frame *f, int formats = 1)
{
    if (!f) return CDEF_ERR_ARG;
    if (f->bitdepth != 8 && f->bitdepth != 10 && f->bitdepth != 12) return CDEF_ERR_BITDEPTH;
    const int w = f->y.width, h = f->y.height;
    if (w <= 0 || h <= 0 || w % 8 || h % 8) return CDEF_ERR_SIZE;
    const int fmt = chroma_format(f);
    if (!((fmt == 420 && (formats & 1)) || (fmt == 422 && (formats & 2)) ||
          (fmt == 444 && (formats & 4))))
        return CDEF_ERR_SIZE;
    const int cw = f->u.width, ch = f->u.height;
    const int b = sample_bytes(f->bitdepth);
    int rc;
    if ((rc = check_plane(f->y, w, h, b))) return rc;
    if ((rc = check_plane(f->u, cw, ch, b))) return rc;
    if ((rc = check_plane(f->v, cw, ch, b))) return rc;
    return CDEF_OK;
}

bool same_geometry(const cdef_frame *a, const cdef_frame *b)
{
    return a->bitdepth == b->bitdepth && a->y.width == b->y.width && a->y.height == b->y.height &&
           a->u.width == b->u.width && a->u.height == b->u.height;
}

bool overlaps(const cdef_plane &a, const cdef_plane &b)
{
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a.data);
    const uintptr_t a1 = a0 + (uintptr_t)a.pitch_bytes * a.height;
    const uintptr_t b0 = reinterpret_cast<uintptr_t>(b.data);
    const uintptr_t b1 = b0 + (uintptr_t)b.pitch_bytes * b.height;
    return a0 < b1 && b0 < a1;
}

bool frames_overlap(const cdef_frame *a, const cdef_frame *b)
{
    const cdef_plane *pa[3] = {&a->y, &a->u, &a->v};
    const cdef_plane *pb[3] = {&b->y, &b->u, &b->v};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (overlaps(*pa[i], *pb[j])) return true;
    return false;
}

int fb_count(const cdef_frame *f) { return ((f->y.width + 63) / 64) * ((f->y.height + 63) / 64); }

}  // namespace

namespace cdefgb {

namespace {
std::mutex g_wait_mutex;
WaitLimits g_waits = {kDefaultWaitCycles, 0, 0};
}  // namespace

WaitLimits wait_limits()
{
    std::lock_guard<std::mutex> lock(g_wait_mutex);
    return g_waits;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// link-time dependency on libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D tile map of one plane with the given box (columns x rows).
int encode_plane(CUtensorMap *m, const cdef_plane &p, int bytes, int box_cols, int box_rows)
{
    const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return CDEF_ERR_CUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)p.width, (cuuint64_t)p.height};
    const cuuint64_t strides[1] = {(cuuint64_t)p.pitch_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(m, bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                          2, p.data, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CDEF_OK : CDEF_ERR_CUDA;
}

int encode_frame_tiles(CUtensorMap maps[3], const cdef_frame *f)
{
    const int b = f->bitdepth == 8 ? 1 : 2;
    int rc;
    if ((rc = encode_plane(&maps[0], f->y, b, luma_box_cols(b), kLumaBoxRows))) return rc;
    if ((rc = encode_plane(&maps[1], f->u, b, chroma_box_cols(b), kChromaBoxRows))) return rc;
    return encode_plane(&maps[2], f->v, b, chroma_box_cols(b), kChromaBoxRows);
}

}  // namespace cdefgb

namespace {

int fill_filter_frame(FilterFrameDev &d, const cdef_frame *in, const cdef_frame *out,
                      const cdef_fb_params *params, const uint8_t *dir, const int32_t *var,
                      int block_start, const uint8_t *coded = nullptr)
{
    d.coded = coded;
    d.mode = 0;
    const cdef_plane *pi[3] = {&in->y, &in->u, &in->v};
    const cdef_plane *po[3] = {&out->y, &out->u, &out->v};
    for (int i = 0; i < 3; i++) {
        d.p[i].in = static_cast<const uint8_t *>(pi[i]->data);
        d.p[i].out = static_cast<uint8_t *>(po[i]->data);
        d.p[i].in_pitch = pi[i]->pitch_bytes;
        d.p[i].out_pitch = po[i]->pitch_bytes;
        d.p[i].w = pi[i]->width;
        d.p[i].h = pi[i]->height;
    }
    d.params = params;
    d.dir = dir;
    d.var = var;
    d.bitdepth = in->bitdepth;
    d.fb_cols = (in->y.width + 63) / 64;
    d.fb_rows = (in->y.height + 63) / 64;
    d.block_start = block_start;
    return encode_frame_tiles(d.tmap, in);
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? CDEF_OK : CDEF_ERR_CUDA; }

int ensure_scratch(cdef_ctx *ctx, size_t bytes)
{
    if (ctx->scratch_bytes >= bytes) return CDEF_OK;
    const size_t grow = bytes - ctx->scratch_bytes;
    if (ctx->budget && ctx->used + grow > ctx->budget) return CDEF_ERR_NOMEM;
    if (ctx->scratch) {
        cudaFree(ctx->scratch);
        ctx->used -= ctx->scratch_bytes;
        ctx->scratch = nullptr;
        ctx->scratch_bytes = 0;
    }
    if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        ctx->scratch = nullptr;
        return CDEF_ERR_NOMEM;
    }
    ctx->scratch_bytes = bytes;
    ctx->used += bytes;
    return CDEF_OK;
}

}  // namespace

extern "C" {

int cdef_ctx_create(cdef_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) return CDEF_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return device < 0 ? CDEF_ERR_ARG : CDEF_ERR_CUDA;
    }
    DeviceGuard g(device);
    if (!g.ok) return CDEF_ERR_CUDA;
    cdef_ctx *ctx = new (std::nothrow) cdef_ctx();
    if (!ctx) return CDEF_ERR_NOMEM;
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    ctx->pairs[0] = ctx->pairs[1] = ~0ull;
    const size_t fixed = sizeof(int) + sizeof(SearchResultDev) * kMaxBatch +
                         sizeof(unsigned) * 2 * kWorkSlots;
    if (ctx->budget && fixed > ctx->budget) {
        delete ctx;
        return CDEF_ERR_NOMEM;
    }
    if (cudaMalloc(&ctx->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->dev_results, sizeof(SearchResultDev) * kMaxBatch) != cudaSuccess ||
        cudaMalloc(&ctx->work, sizeof(unsigned) * 2 * kWorkSlots) != cudaSuccess ||
        cudaMemset(ctx->work, 0, sizeof(unsigned) * 2 * kWorkSlots) != cudaSuccess ||
        cudaMallocHost(&ctx->host_results, sizeof(SearchResultDev) * kMaxBatch) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cdef_ctx_destroy(ctx);
        return CDEF_ERR_CUDA;
    }
    ctx->used = fixed;
    *out = ctx;
    return CDEF_OK;
}

int cdef_ctx_destroy(cdef_ctx *ctx)
{
    if (!ctx) return CDEF_OK;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->status) cudaFree(ctx->status);
    if (ctx->dev_results) cudaFree(ctx->dev_results);
    if (ctx->host_results) cudaFreeHost(ctx->host_results);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->maps_dir) cudaFree(ctx->maps_dir);
    if (ctx->maps_var) cudaFree(ctx->maps_var);
    if (ctx->smaps_dir) cudaFree(ctx->smaps_dir);
    if (ctx->smaps_var) cudaFree(ctx->smaps_var);
    if (ctx->work) cudaFree(ctx->work);
    if (ctx->search_exec) cudaGraphExecDestroy(ctx->search_exec);
    if (ctx->capture) cudaStreamDestroy(ctx->capture);
    for (int k = 0; k < 3; k++)
        if (ctx->stage_ev[k]) cudaEventDestroy(ctx->stage_ev[k]);
    delete ctx->search_key;
    delete ctx->tuned;
    delete ctx;
    return CDEF_OK;
}

int cdef_ctx_set_tuning(cdef_ctx *ctx, const cdef_tuning *t)
{
    if (!ctx) return CDEF_ERR_ARG;
    if (!t) {
        ctx->forced = {0, 0};
        ctx->grid_presets = false;
        return CDEF_OK;
    }
    const int g = t->search_groups, c = t->search_ctas_per_sm;
    if (!(g == 0 || g == 1 || g == 2 || g == 4) || c < 0 || c > 2) return CDEF_ERR_ARG;
    if (t->preset_kernel < 0 || t->preset_kernel > 1 || t->reserved != 0) return CDEF_ERR_ARG;
    ctx->forced = {g, c};
    ctx->grid_presets = t->preset_kernel == 1;
    return CDEF_OK;
}

int cdef_ctx_set_search_metric(cdef_ctx *ctx, int metric)
{
    if (!ctx || (metric != CDEF_METRIC_SSE && metric != CDEF_METRIC_EQ14)) return CDEF_ERR_ARG;
    ctx->metric = metric;
    return CDEF_OK;
}

int cdef_ctx_set_search_subset(cdef_ctx *ctx, uint64_t luma_pairs, uint64_t chroma_pairs)
{
    if (!ctx || !luma_pairs || !chroma_pairs) return CDEF_ERR_ARG;
    ctx->pairs[0] = luma_pairs;
    ctx->pairs[1] = chroma_pairs;
    return CDEF_OK;
}

int cdef_ctx_set_search_refine(cdef_ctx *ctx, int max_passes)
{
    if (!ctx || max_passes < 0 || max_passes > kMaxRefinePasses) return CDEF_ERR_ARG;
    ctx->refine_passes = max_passes;
    return CDEF_OK;
}

int cdef_ctx_set_overlap(cdef_ctx *ctx, int enable)
{
    if (!ctx) return CDEF_ERR_ARG;
    ctx->overlap = enable != 0;
    return CDEF_OK;
}

int cdef_ctx_set_stage_timing(cdef_ctx *ctx, int enable)
{
    if (!ctx) return CDEF_ERR_ARG;
    if (enable && !ctx->stage_ev[0]) {
        DeviceGuard g(ctx->device);
        if (!g.ok) return CDEF_ERR_CUDA;
        for (int k = 0; k < 3; k++) {
            if (cudaEventCreate(&ctx->stage_ev[k]) != cudaSuccess) {
                for (int j = 0; j < k; j++) cudaEventDestroy(ctx->stage_ev[j]);
                for (int j = 0; j < 3; j++) ctx->stage_ev[j] = nullptr;
                cudaGetLastError();
                return CDEF_ERR_CUDA;
            }
        }
    }
    ctx->stage_timing = enable != 0;
    ctx->stage_valid = false;
    return CDEF_OK;
}

int cdef_ctx_get_stage_times(cdef_ctx *ctx, float *distortion_ms, float *presets_ms)
{
    if (!ctx || !distortion_ms || !presets_ms || !ctx->stage_valid) return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok || cudaEventElapsedTime(distortion_ms, ctx->stage_ev[0], ctx->stage_ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(presets_ms, ctx->stage_ev[1], ctx->stage_ev[2]) != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    return CDEF_OK;
}

int cdef_ctx_get_tuning(const cdef_ctx *ctx, cdef_tuning *last)
{
    if (!ctx || !last) return CDEF_ERR_ARG;
    memset(last, 0, sizeof(*last));
    last->search_groups = ctx->last.groups;
    last->search_ctas_per_sm = ctx->last.ctas_per_sm;
    last->preset_kernel = ctx->grid_presets ? 1 : 0;
    return CDEF_OK;
}

int cdef_ctx_status(cdef_ctx *ctx, int clear)
{
    if (!ctx) return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    int v = 0;
    if (cudaMemcpy(&v, ctx->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CDEF_ERR_CUDA;
    if (clear && v && cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess) return CDEF_ERR_CUDA;
    if (v & kStatusTimeout) return CDEF_ERR_TIMEOUT;
    if (v & (kStatusMisaligned | kStatusIndex)) return CDEF_ERR_DEVICE;
    return v ? CDEF_ERR_ARG : CDEF_OK;
}

int cdef_ctx_status_async(cdef_ctx *ctx, int32_t *host_status, void *cuda_stream)
{
    if (!ctx || !host_status) return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    if (cudaMemcpyAsync(host_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost,
                        static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    return CDEF_OK;
}

int cdef_find_dir(cdef_ctx *ctx, const cdef_plane *luma, int32_t bitdepth, uint8_t *dir,
                  int32_t *var, void *cuda_stream)
{
    if (!ctx || !luma || !dir || !var) return CDEF_ERR_ARG;
    if (bitdepth != 8 && bitdepth != 10 && bitdepth != 12) return CDEF_ERR_BITDEPTH;
    const int w = luma->width, h = luma->height;
    if (w <= 0 || h <= 0 || w % 8 || h % 8) return CDEF_ERR_SIZE;
    int rc = check_plane(*luma, w, h, sample_bytes(bitdepth));
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    return cuda_status(launch_find_dir(static_cast<const uint8_t *>(luma->data), luma->pitch_bytes,
                                       w, h, bitdepth, dir, var,
                                       static_cast<cudaStream_t>(cuda_stream)));
}

namespace {

// One launch of the filter over a single plane in the luma slot: mode 1 the
// luma plane, mode 2 a 4:4:4 chroma plane (chroma parameters, maps given).
// One plane of a frame as a filter entry in the luma geometry (mode 1: the
// luma plane, mode 2: a 4:4:4 chroma plane); its blocks start at
// `block_start` of the launch.
int fill_plane_dev(FilterFrameDev &d, const cdef_frame *in, const cdef_plane &pin,
                   const cdef_plane &pout, const cdef_fb_params *params, const uint8_t *dir,
                   const int32_t *var, const uint8_t *coded, int mode, int block_start)
{
    memset(&d, 0, sizeof(d));
    for (int i = 0; i < 3; i++) {
        d.p[i].in = static_cast<const uint8_t *>(pin.data);
        d.p[i].out = static_cast<uint8_t *>(pout.data);
        d.p[i].in_pitch = pin.pitch_bytes;
        d.p[i].out_pitch = pout.pitch_bytes;
        d.p[i].w = pin.width;
        d.p[i].h = pin.height;
    }
    d.params = params;
    d.dir = dir;
    d.var = var;
    d.coded = coded;
    d.mode = mode;
    d.bitdepth = in->bitdepth;
    d.fb_cols = (in->y.width + 63) / 64;
    d.fb_rows = (in->y.height + 63) / 64;
    d.block_start = block_start;
    const int bytes = sample_bytes(in->bitdepth);
    int rc = encode_plane(&d.tmap[0], pin, bytes, luma_box_cols(bytes), kLumaBoxRows);
    if (rc) return rc;
    d.tmap[1] = d.tmap[2] = d.tmap[0];   // not loaded in modes 1 and 2
    return CDEF_OK;
}

// One 8/10-bit 4:4:4 frame as a mode-3 entry: its three planes filtered in
// turn by the CTA that takes a filter block (each plane's map with the luma
// box), the luma directions of the block searched in its first stage (or
// read from dir/var) and kept for the chroma planes.
int fill_444_dev(FilterFrameDev &d, const cdef_frame *in, const cdef_frame *out,
                 const cdef_fb_params *params, const uint8_t *dir, const int32_t *var,
                 const uint8_t *coded)
{
    memset(&d, 0, sizeof(d));
    const cdef_plane *pi[3] = {&in->y, &in->u, &in->v}, *po[3] = {&out->y, &out->u, &out->v};
    const int bytes = sample_bytes(in->bitdepth);
    for (int k = 0; k < 3; k++) {
        d.p[k].in = static_cast<const uint8_t *>(pi[k]->data);
        d.p[k].out = static_cast<uint8_t *>(po[k]->data);
        d.p[k].in_pitch = pi[k]->pitch_bytes;
        d.p[k].out_pitch = po[k]->pitch_bytes;
        d.p[k].w = pi[k]->width;
        d.p[k].h = pi[k]->height;
        const int rc = encode_plane(&d.tmap[k], *pi[k], bytes, luma_box_cols(bytes), kLumaBoxRows);
        if (rc) return rc;
    }
    d.params = params;
    d.dir = dir;
    d.var = var;
    d.coded = coded;
    d.mode = 3;
    d.bitdepth = in->bitdepth;
    d.fb_cols = (in->y.width + 63) / 64;
    d.fb_rows = (in->y.height + 63) / 64;
    d.block_start = 0;
    return CDEF_OK;
}

int plane_pass(cdef_ctx *ctx, const cdef_frame *in, const cdef_plane &pin, const cdef_plane &pout,
               const cdef_fb_params *params, const uint8_t *dir, const int32_t *var,
               const uint8_t *coded, int mode, bool overlap, cudaStream_t s)
{
    FilterBatch<1> b;
    b.n = 1;
    b.total_blocks = fb_count(in);
        b.waits = wait_limits();
    int rc = fill_plane_dev(b.f[0], in, pin, pout, params, dir, var, coded, mode, 0);
    if (rc) return rc;
    unsigned *work = ctx->work + 2 * (1 + ctx->next_slot++ % (kWorkSlots - 1));  // pair 0: search
    return cuda_status(launch_filter_single(b, ctx->status, work, overlap, s));
}

// Direction maps of at least `blocks` 8x8 blocks in (dir, var, have), held
// in the context's scratch budget.  The filter's 4:4:4 path and the wide
// strength search keep separate maps, so that a search never overwrites
// maps a filter launch on another stream still reads.
int ensure_map_set(cdef_ctx *ctx, size_t blocks, uint8_t *&dir, int32_t *&var, size_t &have)
{
    if (have >= blocks) return CDEF_OK;
    const size_t bytes = blocks * (sizeof(uint8_t) + sizeof(int32_t));
    const size_t old = have * (sizeof(uint8_t) + sizeof(int32_t));
    if (ctx->budget && ctx->used - old + bytes > ctx->budget) return CDEF_ERR_NOMEM;
    if (var) cudaFree(var);
    if (dir) cudaFree(dir);
    var = nullptr;
    dir = nullptr;
    ctx->used -= old;
    have = 0;
    if (cudaMalloc(&var, blocks * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&dir, blocks) != cudaSuccess) {
        cudaGetLastError();
        if (var) cudaFree(var);
        var = nullptr;
        dir = nullptr;
        return CDEF_ERR_NOMEM;
    }
    have = blocks;
    ctx->used += bytes;
    return CDEF_OK;
}

int ensure_maps(cdef_ctx *ctx, size_t blocks)
{
    return ensure_map_set(ctx, blocks, ctx->maps_dir, ctx->maps_var, ctx->maps_blocks);
}

int filter_one(cdef_ctx *ctx, const cdef_frame *in, const cdef_fb_params *params,
               const uint8_t *dir, const int32_t *var, const uint8_t *coded,
               const cdef_frame *out, void *cuda_stream)
{
    if (!ctx || !in || !out || !params) return CDEF_ERR_ARG;
    if ((dir == nullptr) != (var == nullptr)) return CDEF_ERR_ARG;
    int rc;
    if ((rc = check_frame(in, 7)) || (rc = check_frame(out, 7))) return rc;
    if (!same_geometry(in, out)) return CDEF_ERR_SIZE;
    if (frames_overlap(in, out)) return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int fmt = chroma_format(in);
    if (fmt == 420) {
        FilterBatch<1> b;
        b.n = 1;
        b.total_blocks = fb_count(in);
        b.waits = wait_limits();
        if ((rc = fill_filter_frame(b.f[0], in, out, params, dir, var, 0, coded))) return rc;
        unsigned *work = ctx->work + 2 * (1 + ctx->next_slot++ % (kWorkSlots - 1));  // pair 0: search
        return cuda_status(launch_filter_single(b, ctx->status, work, ctx->overlap, s));
    }
    if (fmt == 422) {
        // section 4: chroma subsampled differently in the two directions is
        // not filtered; luma as for 4:2:0
        if ((rc = plane_pass(ctx, in, in->y, out->y, params, dir, var, coded, 1, ctx->overlap, s)))
            return rc;
        const size_t row = (size_t)in->u.width * sample_bytes(in->bitdepth);
        const cdef_plane *ci[2] = {&in->u, &in->v}, *co[2] = {&out->u, &out->v};
        for (int k = 0; k < 2; k++)
            if (cudaMemcpy2DAsync(co[k]->data, co[k]->pitch_bytes, ci[k]->data, ci[k]->pitch_bytes,
                                  row, ci[k]->height, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                cudaGetLastError();
                return CDEF_ERR_CUDA;
            }
        return CDEF_OK;
    }
    // 8/10-bit 4:4:4: one launch, a CTA filtering the three planes of a
    // block in turn (consecutive calls on a stream may overlap, as 4:2:0's)
    if (in->bitdepth <= 10) {
        FilterBatch<1> b;
        b.n = 1;
        b.total_blocks = fb_count(in);
        b.waits = wait_limits();
        if ((rc = fill_444_dev(b.f[0], in, out, params, dir, var, coded))) return rc;
        unsigned *work = ctx->work + 2 * (1 + ctx->next_slot++ % (kWorkSlots - 1));  // pair 0: search
        return cuda_status(launch_filter_444(b, ctx->status, work, ctx->overlap, s));
    }
    // 12-bit 4:4:4: the luma directions first (unless given), then the three
    // planes in the luma geometry as one launch, which waits for the maps
    if (!dir) {
        const size_t blocks = (size_t)(in->y.width / 8) * (in->y.height / 8);
        if ((rc = ensure_maps(ctx, blocks))) return rc;
        dir = ctx->maps_dir;
        var = ctx->maps_var;
        if ((rc = cuda_status(launch_find_dir(static_cast<const uint8_t *>(in->y.data),
                                              in->y.pitch_bytes, in->y.width, in->y.height,
                                              in->bitdepth, ctx->maps_dir, ctx->maps_var, s))))
            return rc;
    }
    FilterBatch<3> b;
    b.n = 3;
    const int B = fb_count(in);
    b.total_blocks = 3 * B;
    b.waits = wait_limits();
    if ((rc = fill_plane_dev(b.f[0], in, in->y, out->y, params, dir, var, coded, 1, 0)) ||
        (rc = fill_plane_dev(b.f[1], in, in->u, out->u, params, dir, var, coded, 2, B)) ||
        (rc = fill_plane_dev(b.f[2], in, in->v, out->v, params, dir, var, coded, 2, 2 * B)))
        return rc;
    unsigned *work = ctx->work + 2 * (1 + ctx->next_slot++ % (kWorkSlots - 1));  // pair 0: search
    return cuda_status(launch_filter_planes(b, ctx->status, work, false, s));
}

}  // namespace

int cdef_filter_frame(cdef_ctx *ctx, const cdef_frame *in, const cdef_fb_params *params,
                      const uint8_t *dir, const int32_t *var, const cdef_frame *out,
                      void *cuda_stream)
{
    return filter_one(ctx, in, params, dir, var, nullptr, out, cuda_stream);
}

int cdef_filter_frame_coded(cdef_ctx *ctx, const cdef_frame *in, const cdef_fb_params *params,
                            const uint8_t *coded, const cdef_frame *out, void *cuda_stream)
{
    if (!coded) return CDEF_ERR_ARG;
    return filter_one(ctx, in, params, nullptr, nullptr, coded, out, cuda_stream);
}

int cdef_filter_frames(cdef_ctx *ctx, int32_t n, const cdef_frame *in,
                       const cdef_fb_params *const *params, const cdef_frame *out,
                       void *cuda_stream)
{
    if (!ctx || !in || !out || !params || n <= 0 || n > kMaxFilterBatch) return CDEF_ERR_ARG;
    int start = 0;
    for (int i = 0; i < n; i++) {
        int rc;
        if ((rc = check_frame(&in[i])) || (rc = check_frame(&out[i]))) return rc;
        if (!same_geometry(&in[i], &out[i])) return CDEF_ERR_SIZE;
        if (!params[i]) return CDEF_ERR_ARG;
        for (int j = 0; j < n; j++)
            if (frames_overlap(&in[j], &out[i])) return CDEF_ERR_ARG;
        for (int j = 0; j < i; j++)
            if (frames_overlap(&out[j], &out[i])) return CDEF_ERR_ARG;
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    FilterBatch<kMaxFilterBatch> *bp = new (std::nothrow) FilterBatch<kMaxFilterBatch>();
    if (!bp) return CDEF_ERR_NOMEM;
    bp->n = n;
    for (int i = 0; i < n; i++) {
        const int rc = fill_filter_frame(bp->f[i], &in[i], &out[i], params[i], nullptr, nullptr, start);
        if (rc) {
            delete bp;
            return rc;
        }
        start += fb_count(&in[i]);
    }
    bp->total_blocks = start;
    bp->waits = wait_limits();
    unsigned *work = ctx->work + 2 * (1 + ctx->next_slot++ % (kWorkSlots - 1));  // pair 0: search
    const int rc = cuda_status(launch_filter_batch(*bp, ctx->status, work, ctx->overlap,
                                                   static_cast<cudaStream_t>(cuda_stream)));
    delete bp;
    return rc;
}

namespace {

// Batch shape for the autotuner: frame count, sizes and bit depths.
uint64_t search_shape(const SearchBatch &b)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&h](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix((uint64_t)b.n);
    for (int i = 0; i < b.n; i++) {
        mix((uint64_t)b.f[i].w);
        mix((uint64_t)b.f[i].h);
        mix((uint64_t)b.f[i].bitdepth);
    }
    return h;
}

// The distortion kernel's launch configuration for this call: fixed by the
// caller, known for this batch shape, or found now by timing every
// candidate configuration (a warm-up run and a timed run each) on the call's
// own inputs.  The runs write the call's outputs, which every configuration
// computes identically.
int choose_search_tune(cdef_ctx *ctx, const SearchBatch &b, long long *dl, long long *dc,
                       unsigned long long *cur, unsigned long long *tot, uint8_t *block_ids,
                       uint8_t *skipped, cudaStream_t s, SearchTune *out)
{
    if (ctx->forced.groups > 0 && ctx->forced.ctas_per_sm > 0) {
        *out = ctx->forced;
        return CDEF_OK;
    }
    if (!ctx->tuned) ctx->tuned = new (std::nothrow) std::unordered_map<uint64_t, SearchTune>();
    if (!ctx->tuned) return CDEF_ERR_NOMEM;
    const uint64_t key = search_shape(b) ^ ((uint64_t)ctx->forced.groups << 56) ^
                         ((uint64_t)ctx->forced.ctas_per_sm << 60) ^ (skipped ? 1ull << 52 : 0) ^
                         ((ctx->pairs[0] & ctx->pairs[1]) != ~0ull ? 1ull << 51 : 0);
    auto it = ctx->tuned->find(key);
    if (it != ctx->tuned->end()) {
        *out = it->second;
        return CDEF_OK;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    SearchTune best{0, 0};
    float best_ms = 0.f;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kNumSearchTunes && e == cudaSuccess; k++) {
        const SearchTune t = kSearchTunes[k];
        if ((ctx->forced.groups > 0 && t.groups != ctx->forced.groups) ||
            (ctx->forced.ctas_per_sm > 0 && t.ctas_per_sm != ctx->forced.ctas_per_sm))
            continue;
        e = launch_search(b, dl, dc, cur, tot, ctx->dev_results, block_ids, ctx->status, ctx->work,
                          t, ctx->refine_passes, s, skipped, nullptr, nullptr, nullptr,
                          ctx->grid_presets);
        // the fastest of three timed runs (one run's time varies between
        // processes by more than the configurations of small shapes differ)
        float ms = 0.f;
        for (int r = 0; r < 3 && e == cudaSuccess; r++) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess)
                e = launch_search(b, dl, dc, cur, tot, ctx->dev_results, block_ids, ctx->status,
                                  ctx->work, t, ctx->refine_passes, s, skipped, nullptr, nullptr,
                                  nullptr, ctx->grid_presets);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float one = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&one, e0, e1);
            if (e == cudaSuccess && (r == 0 || one < ms)) ms = one;
        }
        if (e == cudaSuccess && (best.groups == 0 || ms < best_ms)) {
            best = t;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || best.groups == 0) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    (*ctx->tuned)[key] = best;
    *out = best;
    return CDEF_OK;
}

}  // namespace

namespace {

// The search batch of n frames: validation, tile maps, per-frame fields.
// row_begin / row_count (host, per frame; both null = whole frames) select
// a band of filter-block rows of each frame.  *wide is set when a frame is
// not 8/10-bit 4:2:0 (the 32-bit tables); *maps counts the 8x8 blocks of
// the direction maps those need.
int fill_search_batch(cdef_ctx *ctx, int32_t n, const cdef_frame *rec, const cdef_frame *src,
                      const uint8_t *const *coded, const int32_t *damping, const int64_t *lambda,
                      const int32_t *row_begin, const int32_t *row_count, SearchBatch *b,
                      bool *wide_out, size_t *maps_out)
{
    // frames other than 8/10-bit 4:2:0 take the wide tables (64 pairs,
    // squared error)
    bool wide = false;
    for (int i = 0; i < n; i++)
        if (rec[i].bitdepth > 10 || chroma_format(&rec[i]) != 420) wide = true;
    // the 128-combination eq. 14 tables are formed by the 32-bit path
    if (coded && ctx->metric == CDEF_METRIC_EQ14) wide = true;
    // 8/10-bit 4:4:4 frames (squared error over 64 pairs or the 128
    // combinations, eq. 14 over 64 pairs): the packed tables with one plane
    // per work unit (the direction maps formed first, as for the 32-bit
    // path)
    bool planes = n > 0 && !(coded && ctx->metric == CDEF_METRIC_EQ14);
    for (int i = 0; i < n && planes; i++)
        if (rec[i].bitdepth > 10 || chroma_format(&rec[i]) != 444) planes = false;
    int total = 0, rc = CDEF_OK;
    size_t maps = 0;
    for (int i = 0; i < n && rc == CDEF_OK; i++) {
        if ((rc = check_frame(&rec[i], 7)) || (rc = check_frame(&src[i], 7))) break;
        if (!same_geometry(&rec[i], &src[i])) { rc = CDEF_ERR_SIZE; break; }
        if (damping[i] < 3 || damping[i] > 6 || (lambda && lambda[i] < 0)) { rc = CDEF_ERR_ARG; break; }
        if (coded && !coded[i]) { rc = CDEF_ERR_ARG; break; }
        SearchFrameDev &f = b->f[i];
        f.coded = coded ? coded[i] : nullptr;
        f.chroma_format = chroma_format(&rec[i]);
        f.map_start = (int)maps;
        maps += (size_t)(rec[i].y.width / 8) * (rec[i].y.height / 8);
        if (!wide && (rc = encode_frame_tiles(f.tmap, &rec[i]))) break;
        if (planes) {   // every plane with the luma box
            const int bytes = sample_bytes(rec[i].bitdepth);
            const cdef_plane *pl[3] = {&rec[i].y, &rec[i].u, &rec[i].v};
            for (int k = 0; k < 3 && rc == CDEF_OK; k++)
                rc = encode_plane(&f.tmap[k], *pl[k], bytes, luma_box_cols(bytes), kLumaBoxRows);
            if (rc) break;
        }
        const cdef_plane *pr[3] = {&rec[i].y, &rec[i].u, &rec[i].v};
        const cdef_plane *ps[3] = {&src[i].y, &src[i].u, &src[i].v};
        for (int k = 0; k < 3; k++) {
            f.rec[k] = static_cast<const uint8_t *>(pr[k]->data);
            f.src[k] = static_cast<const uint8_t *>(ps[k]->data);
            f.rec_pitch[k] = pr[k]->pitch_bytes;
            f.src_pitch[k] = ps[k]->pitch_bytes;
        }
        f.w = rec[i].y.width;
        f.h = rec[i].y.height;
        f.bitdepth = rec[i].bitdepth;
        f.damping = damping[i];
        f.fb_cols = (f.w + 63) / 64;
        f.fb_rows = (f.h + 63) / 64;
        if (row_begin) {
            const int r0 = row_begin[i], rn = row_count[i];
            if (r0 < 0 || rn < 0 || r0 + rn > f.fb_rows) { rc = CDEF_ERR_ARG; break; }
            f.fb_row0 = r0;
            f.fb_rows = rn;
        }
        f.block_start = total;
        f.lambda = lambda ? lambda[i] : 0;
        f.pairs[0] = ctx->pairs[0];
        f.pairs[1] = ctx->pairs[1];
        total += f.fb_cols * f.fb_rows;
    }
    if (rc != CDEF_OK) return rc;
    b->n = n;
    b->total_blocks = total;
    b->planes = planes ? 1 : 0;
    b->waits = wait_limits();
    *wide_out = wide;
    *maps_out = maps;
    return CDEF_OK;
}

// The strength search; `coded` (host array of n device maps) selects the
// 128-combination variant with section 4's skip semantics.  Exactly one of
// presets / presets_coded is non-null.
int search_impl(cdef_ctx *ctx, int32_t n, const cdef_frame *rec, const cdef_frame *src,
                const uint8_t *const *coded, const int32_t *damping, const int64_t *lambda,
                int64_t *dist_luma, int64_t *dist_chroma, cdef_preset *presets,
                cdef_preset_coded *presets_coded, int32_t *npresets, uint8_t *block_ids,
                int64_t *cost, void *cuda_stream)
{
    if (!ctx || !rec || !src || !damping || !lambda || !(presets || presets_coded) || !npresets ||
        !block_ids || !cost)
        return CDEF_ERR_ARG;
    const int width = coded ? 128 : 64;
    if (n <= 0 || n > kMaxBatch) return CDEF_ERR_ARG;
    if ((dist_luma == nullptr) != (dist_chroma == nullptr)) return CDEF_ERR_ARG;
    SearchBatch *b = new (std::nothrow) SearchBatch();
    if (!b) return CDEF_ERR_NOMEM;
    bool wide = false;
    size_t maps = 0;
    int rc = fill_search_batch(ctx, n, rec, src, coded, damping, lambda, nullptr, nullptr, b,
                               &wide, &maps);
    if (rc != CDEF_OK) { delete b; return rc; }
    const int total = b->total_blocks;

    DeviceGuard g(ctx->device);
    if (!g.ok) { delete b; return CDEF_ERR_CUDA; }
    const size_t greedy = search_scratch_bytes(n, total, width);
    const size_t tables = dist_luma ? 0 : (size_t)total * width * sizeof(long long) * 2;
    if ((rc = ensure_scratch(ctx, greedy + tables))) { delete b; return rc; }
    unsigned long long *cur = static_cast<unsigned long long *>(ctx->scratch);
    unsigned long long *tot = cur + total;
    long long *dl = reinterpret_cast<long long *>(dist_luma);
    long long *dc = reinterpret_cast<long long *>(dist_chroma);
    if (!dl) {
        dl = reinterpret_cast<long long *>(static_cast<char *>(ctx->scratch) + greedy);
        dc = dl + (size_t)total * width;
    }
    uint8_t *skipped = nullptr;   // per-block flags of the 128-combination search
    if (coded)
        skipped = static_cast<uint8_t *>(ctx->scratch) +
                  sizeof(unsigned long long) * ((size_t)total + (size_t)n * width * width) +
                  kPresetCtlBytes;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // Search calls synchronise before returning, so they never overlap: the
    // search owns counter pair 0 (filter launches take pairs 1..).
    unsigned *work = ctx->work;
    SearchTune tune;
    uint8_t *wide_dirs = nullptr;
    int32_t *wide_vars = nullptr;
    if (wide) {
        // direction maps for every frame of the call
        if ((rc = ensure_map_set(ctx, maps, ctx->smaps_dir, ctx->smaps_var, ctx->smaps_blocks))) {
            delete b;
            return rc;
        }
        wide_dirs = ctx->smaps_dir;
        wide_vars = ctx->smaps_var;
        // one CTA per filter block and plane group; groups 8: eq. 14
        tune = {ctx->metric == CDEF_METRIC_EQ14 ? 8 : 1, 1};
    } else if (ctx->metric == CDEF_METRIC_EQ14) {
        tune = {8, 2};   // the eq. 14 tables: 8 candidates per work unit
    } else if ((rc = choose_search_tune(ctx, *b, dl, dc, cur, tot, block_ids, skipped, s, &tune))) {
        delete b;
        return rc;
    }
    ctx->last = tune;
    // The whole search (distortion kernel, 8 greedy steps, final choice) as
    // one graph launch.  A call on the same frames and buffers as the last
    // one relaunches its graph; otherwise the launches are recorded on the
    // capture stream and the cached executable graph updated in place
    // (re-instantiated if the shape changed).
    void *const ptrs[7] = {dl, dc, block_ids, cur, tot, skipped, wide_dirs};
    const bool same = ctx->search_exec && ctx->search_key &&
                      memcmp(ctx->search_key, b, sizeof(SearchBatch)) == 0 &&
                      memcmp(ctx->search_ptrs, ptrs, sizeof(ptrs)) == 0 &&
                      ctx->search_key_tune.groups == tune.groups &&
                      ctx->search_key_tune.ctas_per_sm == tune.ctas_per_sm &&
                      ctx->search_key_refine == ctx->refine_passes &&
                      ctx->search_key_timing == ctx->stage_timing &&
                      ctx->search_key_grid == ctx->grid_presets;
    cudaError_t e = same ? cudaSuccess : cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && !same) {
        const cudaError_t le = launch_search(*b, dl, dc, cur, tot, ctx->dev_results, block_ids,
                                             ctx->status, work, tune, ctx->refine_passes,
                                             ctx->capture, skipped,
                                             ctx->stage_timing ? ctx->stage_ev : nullptr,
                                             wide_dirs, wide_vars, ctx->grid_presets);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(ctx->capture, &graph);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
        if (e == cudaSuccess) {
            cudaGraphExecUpdateResultInfo info;
            if (!ctx->search_exec || cudaGraphExecUpdate(ctx->search_exec, graph, &info) != cudaSuccess) {
                cudaGetLastError();
                if (ctx->search_exec) cudaGraphExecDestroy(ctx->search_exec);
                ctx->search_exec = nullptr;
                e = cudaGraphInstantiate(&ctx->search_exec, graph, 0);
            }
        }
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) {
            if (!ctx->search_key) ctx->search_key = new (std::nothrow) SearchBatch();
            if (ctx->search_key) {
                memcpy(ctx->search_key, b, sizeof(SearchBatch));
                memcpy(ctx->search_ptrs, ptrs, sizeof(ptrs));
                ctx->search_key_tune = tune;
                ctx->search_key_refine = ctx->refine_passes;
                ctx->search_key_grid = ctx->grid_presets;
                ctx->search_key_timing = ctx->stage_timing;
            }
        } else if (ctx->search_key) {
            memset(static_cast<void *>(ctx->search_key), 0, sizeof(SearchBatch));   // no key: re-record
        }
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(ctx->search_exec, s);
    delete b;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->host_results, ctx->dev_results, sizeof(SearchResultDev) * n,
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    ctx->stage_valid = e == cudaSuccess && ctx->stage_timing;
    if (e != cudaSuccess) return CDEF_ERR_CUDA;
    static const uint8_t kSec[4] = {0, 1, 2, 4};
    for (int i = 0; i < n; i++) {
        const SearchResultDev &r = ctx->host_results[i];
        npresets[i] = r.npresets;
        cost[i] = r.cost;
        for (int k = 0; k < 8; k++) {
            const int t = r.presets[k], ql = t / width, qc = t % width;
            if (presets) {
                cdef_preset &p = presets[i * 8 + k];
                p.pri_y = (uint8_t)(ql >> 2);
                p.sec_y = kSec[ql & 3];
                p.pri_uv = (uint8_t)(qc >> 2);
                p.sec_uv = kSec[qc & 3];
            } else {
                // q = skip * 64 + p * 4 + s
                cdef_preset_coded &p = presets_coded[i * 8 + k];
                memset(&p, 0, sizeof(p));
                p.pri_y = (uint8_t)((ql >> 2) & 15);
                p.sec_y = kSec[ql & 3];
                p.pri_uv = (uint8_t)((qc >> 2) & 15);
                p.sec_uv = kSec[qc & 3];
                p.skip = (uint8_t)((ql >> 6) | ((qc >> 6) << 1));
            }
        }
    }
    return CDEF_OK;
}

}  // namespace

int cdef_search_strengths(cdef_ctx *ctx, int32_t n, const cdef_frame *rec, const cdef_frame *src,
                          const int32_t *damping, const int64_t *lambda, int64_t *dist_luma,
                          int64_t *dist_chroma, cdef_preset *presets, int32_t *npresets,
                          uint8_t *block_ids, int64_t *cost, void *cuda_stream)
{
    if (!presets) return CDEF_ERR_ARG;
    return search_impl(ctx, n, rec, src, nullptr, damping, lambda, dist_luma, dist_chroma, presets,
                       nullptr, npresets, block_ids, cost, cuda_stream);
}

int cdef_search_strengths_coded(cdef_ctx *ctx, int32_t n, const cdef_frame *rec,
                                const cdef_frame *src, const uint8_t *const *coded,
                                const int32_t *damping, const int64_t *lambda,
                                int64_t *dist_luma, int64_t *dist_chroma,
                                cdef_preset_coded *presets, int32_t *npresets,
                                uint8_t *block_ids, int64_t *cost, void *cuda_stream)
{
    if (!coded || !presets) return CDEF_ERR_ARG;
    return search_impl(ctx, n, rec, src, coded, damping, lambda, dist_luma, dist_chroma, nullptr,
                       presets, npresets, block_ids, cost, cuda_stream);
}

int cdef_search_tables(cdef_ctx *ctx, int32_t n, const cdef_frame *rec, const cdef_frame *src,
                       const uint8_t *const *coded, const int32_t *damping,
                       const int32_t *row_begin, const int32_t *row_count, int64_t *dist_luma,
                       int64_t *dist_chroma, uint8_t *skipped, void *cuda_stream)
{
    if (!ctx || !rec || !src || !damping || !row_begin || !row_count || !dist_luma ||
        !dist_chroma || n <= 0 || n > kMaxBatch)
        return CDEF_ERR_ARG;
    if ((coded == nullptr) != (skipped == nullptr)) return CDEF_ERR_ARG;
    SearchBatch *b = new (std::nothrow) SearchBatch();
    if (!b) return CDEF_ERR_NOMEM;
    bool wide = false;
    size_t maps = 0;
    int rc = fill_search_batch(ctx, n, rec, src, coded, damping, nullptr, row_begin, row_count, b,
                               &wide, &maps);
    if (rc != CDEF_OK) { delete b; return rc; }
    DeviceGuard g(ctx->device);
    if (!g.ok) { delete b; return CDEF_ERR_CUDA; }
    if (b->total_blocks == 0) { delete b; return CDEF_OK; }
    uint8_t *wide_dirs = nullptr;
    int32_t *wide_vars = nullptr;
    SearchTune tune;
    if (wide) {
        if ((rc = ensure_map_set(ctx, maps, ctx->smaps_dir, ctx->smaps_var, ctx->smaps_blocks))) {
            delete b;
            return rc;
        }
        wide_dirs = ctx->smaps_dir;
        wide_vars = ctx->smaps_var;
        tune = {ctx->metric == CDEF_METRIC_EQ14 ? 8 : 1, 1};
    } else if (ctx->metric == CDEF_METRIC_EQ14) {
        tune = {8, 2};
    } else {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return CDEF_ERR_CUDA;
        }
        tune = default_search_tune(b->total_blocks, sms);
    }
    // the kernels' work counters: a filter-style slot (the call does not
    // synchronise, so it must not share the search's pair)
    unsigned *work = ctx->work + 2 * (1 + ctx->next_slot++ % (kWorkSlots - 1));
    const cudaError_t e = launch_search(*b, reinterpret_cast<long long *>(dist_luma),
                                        reinterpret_cast<long long *>(dist_chroma), nullptr,
                                        nullptr, nullptr, nullptr, ctx->status, work, tune, 0,
                                        static_cast<cudaStream_t>(cuda_stream), skipped, nullptr,
                                        wide_dirs, wide_vars, false, true);
    delete b;
    return cuda_status(e);
}

int cdef_preset_totals(cdef_ctx *ctx, int32_t nblocks, int32_t width, const int64_t *dist_luma,
                       const int64_t *dist_chroma, const uint8_t *skipped, const uint64_t *best,
                       int64_t *totals, void *cuda_stream)
{
    if (!ctx || !totals || nblocks < 0 || (width != 64 && width != 128)) return CDEF_ERR_ARG;
    if (nblocks > 0 && (!dist_luma || !dist_chroma)) return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(totals, 0, sizeof(int64_t) * width * width, s);
    if (e == cudaSuccess)
        e = launch_preset_totals(nblocks, width, reinterpret_cast<const long long *>(dist_luma),
                                 reinterpret_cast<const long long *>(dist_chroma), skipped,
                                 reinterpret_cast<const unsigned long long *>(best),
                                 reinterpret_cast<long long *>(totals), s);
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

int cdef_preset_argmin(cdef_ctx *ctx, int32_t width, const int64_t *totals, uint64_t luma_pairs,
                       uint64_t chroma_pairs, int32_t keep, int64_t *result, void *cuda_stream)
{
    if (!ctx || !totals || !result || (width != 64 && width != 128) || !luma_pairs ||
        !chroma_pairs || keep < -1 || keep >= width * width)
        return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    const cudaError_t e = launch_preset_argmin(width, reinterpret_cast<const long long *>(totals),
                                               luma_pairs, chroma_pairs, keep,
                                               reinterpret_cast<long long *>(result),
                                               static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

int cdef_preset_assign(cdef_ctx *ctx, int32_t nblocks, int32_t width, const int64_t *dist_luma,
                       const int64_t *dist_chroma, const uint8_t *skipped, const int32_t *presets,
                       int32_t npresets, uint64_t *best, uint8_t *block_ids, int64_t *sums,
                       void *cuda_stream)
{
    if (!ctx || nblocks < 0 || (width != 64 && width != 128) || npresets < 0 || npresets > 8 ||
        (npresets > 0 && !presets))
        return CDEF_ERR_ARG;
    if (nblocks > 0 && (!dist_luma || !dist_chroma)) return CDEF_ERR_ARG;
    PresetList set = {};
    set.n = npresets;
    for (int k = 0; k < npresets; k++) {
        if (presets[k] < 0 || presets[k] >= width * width) return CDEF_ERR_ARG;
        set.t[k] = presets[k];
    }
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = sums ? cudaMemsetAsync(sums, 0, 2 * sizeof(int64_t), s) : cudaSuccess;
    if (e == cudaSuccess)
        e = launch_preset_assign(nblocks, width, reinterpret_cast<const long long *>(dist_luma),
                                 reinterpret_cast<const long long *>(dist_chroma), skipped, set,
                                 reinterpret_cast<unsigned long long *>(best), block_ids,
                                 reinterpret_cast<long long *>(sums), s);
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_status(e);
}

const char *cdef_strerror(int status)
{
    switch (status) {
    case CDEF_OK: return "ok";
    case CDEF_ERR_ARG: return "invalid argument";
    case CDEF_ERR_SIZE: return "invalid frame size";
    case CDEF_ERR_BITDEPTH: return "unsupported bit depth";
    case CDEF_ERR_NOMEM: return "out of device memory or over budget";
    case CDEF_ERR_CUDA: return "CUDA error";
    case CDEF_ERR_TIMEOUT: return "bounded device wait timed out";
    case CDEF_ERR_DEVICE: return "device-side consistency error";
    default: return "unknown status";
    }
}

const char *cdef_version(void) { return "cdef_gb300 0.1 sm_103a"; }

int cdef_debug_checks(cdef_ctx *ctx, int64_t *faults, int32_t clear)
{
    if (!ctx || !faults) return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    unsigned long long n = 0;
    for (auto reader : {index_faults_filter, index_faults_search, index_faults_search_wide}) {
        const unsigned long long v = reader(clear != 0);
        if (v == ~0ull) {
            cudaGetLastError();
            return CDEF_ERR_CUDA;
        }
        n += v;
    }
    *faults = (int64_t)n;
    return kIndexChecks ? 1 : 0;
}

int cdef_probe_int_mix(cdef_ctx *ctx, int32_t mix, int32_t iters, double *lane_instr_per_s,
                       void *cuda_stream)
{
    if (!ctx || !lane_instr_per_s || mix < 0 || mix > 6 || iters < 1 || iters > (1 << 20))
        return CDEF_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (!g.ok) return CDEF_ERR_CUDA;
    return probe_int_mix(ctx->device, mix, iters, lane_instr_per_s,
                         static_cast<cudaStream_t>(cuda_stream));
}

int cdef_debug_set_waits(int64_t wait_cycles, int32_t extra_tx_bytes)
{
    if (wait_cycles < 0 || extra_tx_bytes < 0 || extra_tx_bytes > (1 << 16)) return CDEF_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_wait_mutex);
    g_waits.wait_cycles = wait_cycles ? wait_cycles : kDefaultWaitCycles;
    g_waits.extra_tx = extra_tx_bytes;
    return CDEF_OK;
}

}  // extern "C"
