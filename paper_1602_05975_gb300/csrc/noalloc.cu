// cdef_search_strengths_noalloc: the strength search for callers that are
// not allowed to allocate device memory (see include/cdef_gb300.h).
//
// The search needs a little device scratch besides its inputs and outputs:
// the per-block running minimum of the greedy preset search (one int64 per
// filter block) and the per-frame result records.  Here that scratch is a
// file-scope device array of fixed size, shared by every call on a device
// and held by every GPU that loads the library until the process exits.
// No call in this file allocates device or pinned host memory.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "cdef_internal.h"

using namespace cdefgb;

namespace {

constexpr int kMaxDevices = 64;
// greedy state (per-block minima, per-frame preset totals), result records,
// one work-counter pair
constexpr size_t kGreedyBytes = search_scratch_bytes(kMaxBatch, CDEF_NOALLOC_MAX_BLOCKS);
constexpr size_t kResultBytes = sizeof(SearchResultDev) * kMaxBatch;
constexpr size_t kScratchBytes = kGreedyBytes + kResultBytes + 2 * sizeof(unsigned) + sizeof(int);

// The scratch itself.  In host code `g_scratch` names a host-side shadow,
// not device memory: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_dev[kMaxDevices];  // device address of g_scratch per device

// Once per device, with that device current.
int scratch_for_current_device(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CDEF_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return CDEF_OK;
}

int plane_ok(const cdef_plane &p, int w, int h, int bytes)
{
    if (!p.data) return CDEF_ERR_ARG;
    if (p.width != w || p.height != h) return CDEF_ERR_SIZE;
    if (reinterpret_cast<uintptr_t>(p.data) % 16) return CDEF_ERR_ARG;
    if (p.pitch_bytes <= 0 || p.pitch_bytes % 16 || p.pitch_bytes < (int64_t)w * bytes)
        return CDEF_ERR_ARG;
    return CDEF_OK;
}

int frame_ok(const cdef_frame &f)
{
    if (f.bitdepth != 8 && f.bitdepth != 10 && f.bitdepth != 12) return CDEF_ERR_BITDEPTH;
    const int w = f.y.width, h = f.y.height;
    if (w <= 0 || h <= 0 || w % 8 || h % 8) return CDEF_ERR_SIZE;
    const int b = f.bitdepth == 8 ? 1 : 2;
    int rc;
    if ((rc = plane_ok(f.y, w, h, b))) return rc;
    if ((rc = plane_ok(f.u, w / 2, h / 2, b))) return rc;
    return plane_ok(f.v, w / 2, h / 2, b);
}

}  // namespace

extern "C" int cdef_search_strengths_noalloc(int32_t n, const cdef_frame *rec,
                                             const cdef_frame *src, const int32_t *damping,
                                             const int64_t *lambda, int64_t *dist_luma,
                                             int64_t *dist_chroma, cdef_preset *presets,
                                             int32_t *npresets, uint8_t *block_ids,
                                             int64_t *cost, void *cuda_stream)
{
    if (!rec || !src || !damping || !lambda || !dist_luma || !dist_chroma || !presets ||
        !npresets || !block_ids || !cost)
        return CDEF_ERR_ARG;
    if (n <= 0 || n > kMaxBatch) return CDEF_ERR_ARG;
    SearchBatch b;  // on the stack: no heap use either
    int total = 0;
    for (int i = 0; i < n; i++) {
        int rc;
        if ((rc = frame_ok(rec[i])) || (rc = frame_ok(src[i]))) return rc;
        if (rec[i].bitdepth != src[i].bitdepth || rec[i].y.width != src[i].y.width ||
            rec[i].y.height != src[i].y.height)
            return CDEF_ERR_SIZE;
        if (rec[i].bitdepth > 10) return CDEF_ERR_BITDEPTH;
        if (damping[i] < 3 || damping[i] > 6 || lambda[i] < 0) return CDEF_ERR_ARG;
        SearchFrameDev &f = b.f[i];
        int trc;
        if ((trc = encode_frame_tiles(f.tmap, &rec[i]))) return trc;
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
        f.block_start = total;
        f.lambda = lambda[i];
        total += f.fb_cols * f.fb_rows;
        if (total > CDEF_NOALLOC_MAX_BLOCKS) return CDEF_ERR_NOMEM;  // over the fixed scratch
    }
    b.n = n;
    b.total_blocks = total;
    b.waits = wait_limits();

    void *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    unsigned long long *cur = reinterpret_cast<unsigned long long *>(base);
    unsigned long long *tot = cur + CDEF_NOALLOC_MAX_BLOCKS;
    SearchResultDev *results = reinterpret_cast<SearchResultDev *>(base + kGreedyBytes);
    unsigned *work = reinterpret_cast<unsigned *>(base + kGreedyBytes + kResultBytes);
    int *status = reinterpret_cast<int *>(work + 2);
    // Every scratch word the kernels read is written by them first in this
    // call (the greedy minima and preset totals are reset at its start, the
    // result records written whole); the work counters start at zero (static
    // storage) and every launch leaves them at zero again.  The status word
    // collects the kernels' error bits: cleared here, read back with the
    // results.
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = launch_search(b, reinterpret_cast<long long *>(dist_luma),
                          reinterpret_cast<long long *>(dist_chroma), cur, tot, results, block_ids,
                          status, work, default_search_tune(total, sms), 0, s);
    SearchResultDev host[kMaxBatch];  // pageable stack copies: no pinned allocation
    int host_status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host, results, sizeof(SearchResultDev) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CDEF_ERR_CUDA;
    }
    // a kernel that gave up leaves the tables and presets unspecified
    if (host_status & kStatusTimeout) return CDEF_ERR_TIMEOUT;
    if (host_status) return CDEF_ERR_DEVICE;
    static const uint8_t kSec[4] = {0, 1, 2, 4};
    for (int i = 0; i < n; i++) {
        npresets[i] = host[i].npresets;
        cost[i] = host[i].cost;
        for (int k = 0; k < 8; k++) {
            const int t = host[i].presets[k], ql = t >> 6, qc = t & 63;
            cdef_preset &p = presets[i * 8 + k];
            p.pri_y = (uint8_t)(ql >> 2);
            p.sec_y = kSec[ql & 3];
            p.pri_uv = (uint8_t)(qc >> 2);
            p.sec_uv = kSec[qc & 3];
        }
    }
    return CDEF_OK;
}
