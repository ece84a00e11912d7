// Hull diagnostics: extra and missing voxels of a hull against the true
// object, per slice (the counts of Tables 1-2, Sec. 4), and the part of a
// mask that it encloses within each slice (applied to the literal MSC hull
// H_2 of Eq. 3.6, whose excluded voxels form a shell around the object, it
// keeps the region the shell encloses).
//
//   compare_kernel  one block per slice: block sums of the two counts
//   fill_kernel     one block per slice: the mask and the exterior (mask
//                   voxels joined to the slice border) as bitmaps in shared
//                   memory, one row of words per voxel row; the exterior
//                   grows by one voxel across words and rows and by whole
//                   runs inside a word per sweep, until a sweep adds nothing
#include <cuda_runtime.h>

#include "hd_internal.cuh"

namespace {

constexpr int kDiagThreads = 1024;
constexpr int kFillMaxWords = 24 * 1024;  // two bitmaps of 96 KB

__device__ __forceinline__ long long block_sum(long long v, long long *s_warp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t += s_warp[k];
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kDiagThreads) compare_kernel(const uint8_t *hull,
                                                               const uint8_t *object, int64_t plane,
                                                               int nz, long long *counts)
{
    __shared__ long long s_warp[32];
    const int z = blockIdx.x;
    const uint8_t *h = hull + static_cast<int64_t>(z) * plane;
    const uint8_t *o = object + static_cast<int64_t>(z) * plane;
    long long extra = 0, missing = 0;
    for (int64_t j = threadIdx.x; j < plane; j += blockDim.x) {
        const bool hv = h[j] != 0, ov = o[j] != 0;
        extra += hv && !ov ? 1 : 0;
        missing += ov && !hv ? 1 : 0;
    }
    const long long e = block_sum(extra, s_warp);
    const long long m = block_sum(missing, s_warp);
    if (threadIdx.x == 0) {
        counts[z] = e;
        counts[nz + z] = m;
        atomicAdd(reinterpret_cast<unsigned long long *>(counts + 2 * nz),
                  static_cast<unsigned long long>(e));
        atomicAdd(reinterpret_cast<unsigned long long *>(counts + 2 * nz + 1),
                  static_cast<unsigned long long>(m));
    }
}

// Bits of g reachable from g through set bits of p, moving toward higher
// bits (left) and toward lower bits (right) inside one word (Kogge-Stone).
__device__ __forceinline__ uint32_t fill_word(uint32_t g, uint32_t p)
{
    uint32_t l = g, pl = p;
    l |= pl & (l << 1);
    pl &= pl << 1;
    l |= pl & (l << 2);
    pl &= pl << 2;
    l |= pl & (l << 4);
    pl &= pl << 4;
    l |= pl & (l << 8);
    pl &= pl << 8;
    l |= pl & (l << 16);
    uint32_t r = g, pr = p;
    r |= pr & (r >> 1);
    pr &= pr >> 1;
    r |= pr & (r >> 2);
    pr &= pr >> 2;
    r |= pr & (r >> 4);
    pr &= pr >> 4;
    r |= pr & (r >> 8);
    pr &= pr >> 8;
    r |= pr & (r >> 16);
    return l | r;
}

// Bitmaps: word (y, w) = y * rw + w holds voxels x = 32 w .. 32 w + 31 of
// row y (bit x & 31); bits past nx are 0 in the mask, so nothing grows there.
__global__ void __launch_bounds__(kDiagThreads) fill_kernel(const uint8_t *mask, int nx, int ny,
                                                            int rw, uint8_t *out)
{
    extern __shared__ uint32_t s_bits[];
    uint32_t *M = s_bits;
    uint32_t *E = s_bits + ny * rw;
    const int z = blockIdx.x;
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    const uint8_t *m = mask + static_cast<int64_t>(z) * plane;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int words = ny * rw;
    // mask bits, a warp per word (coalesced bytes, one ballot)
    for (int k = warp; k < words; k += nwarps) {
        const int y = k / rw, x = (k - y * rw) * 32 + lane;
        const bool bit = x < nx && m[static_cast<int64_t>(y) * nx + x] != 0;
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) M[k] = word;
    }
    __syncthreads();
    // seeds: the mask voxels on the slice border
    for (int k = threadIdx.x; k < words; k += blockDim.x) {
        const int y = k / rw, w = k - y * rw;
        uint32_t seed = 0;
        if (y == 0 || y == ny - 1) {
            seed = 0xffffffffu;
        } else {
            if (w == 0) seed |= 1u;
            if (w == (nx - 1) >> 5) seed |= 1u << ((nx - 1) & 31);
        }
        E[k] = seed & M[k];
    }
    __syncthreads();
    // sweeps until nothing changes; each sweep that changes adds a voxel, so
    // at most nx ny + 1 sweeps run
    const long long max_sweeps = plane + 1;
    for (long long it = 0; it < max_sweeps; ++it) {
        int changed = 0;
        for (int k = threadIdx.x; k < words; k += blockDim.x) {
            const int y = k / rw, w = k - y * rw;
            const uint32_t e = E[k], mk = M[k];
            uint32_t g = e | (e << 1) | (e >> 1);
            if (w > 0) g |= E[k - 1] >> 31;
            if (w + 1 < rw) g |= E[k + 1] << 31;
            if (y > 0) g |= E[k - rw];
            if (y + 1 < ny) g |= E[k + rw];
            const uint32_t ne = fill_word(g & mk, mk);
            if (ne != e) {
                E[k] = ne;  // only this thread writes word k; neighbours may
                changed = 1;  // read it old or new, both inside the exterior
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    // enclosed = mask, not exterior
    uint8_t *o = out + static_cast<int64_t>(z) * plane;
    for (int64_t j = threadIdx.x; j < plane; j += blockDim.x) {
        const int y = static_cast<int>(j / nx), x = static_cast<int>(j - static_cast<int64_t>(y) * nx);
        const int k = y * rw + (x >> 5);
        o[j] = static_cast<uint8_t>(((M[k] & ~E[k]) >> (x & 31)) & 1u);
    }
}

}  // namespace

extern "C" {

hd_status hd_hull_compare(const uint8_t *hull, const uint8_t *object, int32_t nx, int32_t ny,
                          int32_t nz, int64_t *counts, void *stream)
{
    if (!hull || !object || !counts || nx < 1 || ny < 1 || nz < 1) return HD_ERR_ARG;
    if (nz > 65535) return HD_ERR_RANGE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counts + 2 * static_cast<int64_t>(nz), 0,
                                    2 * sizeof(int64_t), st);
    if (e == cudaSuccess) {
        compare_kernel<<<nz, kDiagThreads, 0, st>>>(hull, object, static_cast<int64_t>(nx) * ny,
                                                    nz, reinterpret_cast<long long *>(counts));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        hd::note_cuda_error(e, "hd_hull_compare");
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

hd_status hd_fill_enclosed(const uint8_t *mask, int32_t nx, int32_t ny, int32_t nz, uint8_t *out,
                           void *stream)
{
    if (!mask || !out || nx < 1 || ny < 1 || nz < 1) return HD_ERR_ARG;
    if (nz > 65535) return HD_ERR_RANGE;
    const int rw = (nx + 31) / 32;
    const int64_t words = static_cast<int64_t>(rw) * ny;
    if (words > kFillMaxWords) return HD_ERR_RANGE;
    const size_t smem = 2 * sizeof(uint32_t) * static_cast<size_t>(words);
    cudaError_t e = cudaFuncSetAttribute(fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(2 * sizeof(uint32_t) * kFillMaxWords));
    if (e == cudaSuccess) {
        fill_kernel<<<nz, kDiagThreads, smem, static_cast<cudaStream_t>(stream)>>>(mask, nx, ny,
                                                                                   rw, out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        hd::note_cuda_error(e, "hd_fill_enclosed");
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // extern "C"
