// Standalone direction search (section 2, Algorithm 1): one thread per 8x8
// luma block, reading its 8 rows straight from HBM with one vector load per
// row (8 bytes at 8 bits, 16 bytes at 10/12 bits).  Adjacent threads own
// adjacent blocks, so each row load of a warp is one contiguous segment.
#include "cdef_device.cuh"
#include "cdef_internal.h"

namespace cdefgb {

template <typename T>
__global__ void __launch_bounds__(128)
find_dir_kernel(const uint8_t *__restrict__ luma, int64_t pitch, int bw, int bh,
                int sh8, uint8_t *__restrict__ dir, int32_t *__restrict__ var)
{
    const int bx = blockIdx.x * blockDim.x + threadIdx.x;
    const int by = blockIdx.y;
    if (bx >= bw || by >= bh) return;
    const uint8_t *base = luma + (int64_t)by * 8 * pitch + (int64_t)bx * 8 * sizeof(T);
    int px[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        if (sizeof(T) == 1) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(base + i * pitch));
#pragma unroll
            for (int j = 0; j < 4; j++) {
                px[i][j] = (v.x >> (8 * j)) & 0xff;
                px[i][j + 4] = (v.y >> (8 * j)) & 0xff;
            }
        } else {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(base + i * pitch));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                px[i][2 * j] = w[j] & 0xffff;
                px[i][2 * j + 1] = w[j] >> 16;
            }
        }
    }
    int v = 0;
    const int d = find_dir_8x8([&](int i, int j) { return px[i][j]; }, sh8, &v);
    dir[by * bw + bx] = (uint8_t)d;
    var[by * bw + bx] = v;
}

cudaError_t launch_find_dir(const uint8_t *luma, int64_t pitch, int w, int h,
                            int bitdepth, uint8_t *dir, int32_t *var,
                            cudaStream_t s)
{
    const int bw = w / 8, bh = h / 8;
    const dim3 grid((bw + 127) / 128, bh);
    if (bitdepth == 8)
        find_dir_kernel<uint8_t><<<grid, 128, 0, s>>>(luma, pitch, bw, bh, 0, dir, var);
    else
        find_dir_kernel<uint16_t><<<grid, 128, 0, s>>>(luma, pitch, bw, bh, bitdepth - 8, dir, var);
    return cudaGetLastError();
}

}  // namespace cdefgb
