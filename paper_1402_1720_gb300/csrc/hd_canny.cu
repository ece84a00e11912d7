// SM threshold by edge detection: a documented form of the "modified Canny"
// picker the paper used for M_t (Sec. 4, which names the method but not its
// modification).  Per slice of M: binomial smoothing, Sobel derivatives, L1
// magnitude, non-maximum suppression (ties kept on the side of larger M),
// hysteresis at 1/2 and 1/5 of the slice's largest suppressed magnitude
// (8-connected), M_t = a quantile of M over the edge voxels, H_3 = [M >= M_t].
// All integer arithmetic.
//
//   canny_smooth_kernel    thread per voxel: S = [1 2 1]^T [1 2 1] * M
//   canny_gradient_kernel  thread per voxel: Sobel of S, magnitude, direction
//   canny_nms_kernel       thread per voxel: local maximum test
//   canny_slice_kernel     block per slice: the slice maximum, hysteresis on bitmaps in shared
//                          memory, the edge voxels' M listed in shared memory,
//                          the quantile by a 32-step radix select, the hull
#include <cuda_runtime.h>

#include "hd_internal.cuh"

namespace {

constexpr int kVoxThreads = 256;
constexpr int kSliceThreads = 1024;
constexpr int kMaxWords = 24 * 1024;  // two slice bitmaps of 96 KB
constexpr int kListCap = 4096;        // edge values listed in shared memory

struct CannyWs {
    long long *S, *mag;
    uint8_t *dir;  // (dx + 1) | (dy + 1) << 2 of the gradient direction
    uint8_t *nms;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void __launch_bounds__(kVoxThreads) canny_smooth_kernel(const uint32_t *M, int nx,
                                                                   int ny, int64_t V,
                                                                   long long *S)
{
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    const int64_t z = v / plane;
    const int j = static_cast<int>(v - z * plane);
    const int y = j / nx, x = j - y * nx;
    const uint32_t *m = M + z * plane;
    const int w[3] = {1, 2, 1};
    long long acc = 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int Y = clampi(y + dy, 0, ny - 1);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int X = clampi(x + dx, 0, nx - 1);
            acc += static_cast<long long>(w[dx + 1] * w[dy + 1]) * m[X + nx * Y];
        }
    }
    S[v] = acc;
}

__global__ void __launch_bounds__(kVoxThreads) canny_gradient_kernel(const long long *S, int nx,
                                                                     int ny, int64_t V,
                                                                     long long *mag, uint8_t *dir)
{
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    const int64_t z = v / plane;
    const int j = static_cast<int>(v - z * plane);
    const int y = j / nx, x = j - y * nx;
    const long long *s = S + z * plane;
    const int xm = clampi(x - 1, 0, nx - 1), xp = clampi(x + 1, 0, nx - 1);
    const int ym = clampi(y - 1, 0, ny - 1), yp = clampi(y + 1, 0, ny - 1);
    const int w[3] = {1, 2, 1};
    long long gx = 0, gy = 0;
#pragma unroll
    for (int k = -1; k <= 1; ++k) {
        const int Yk = clampi(y + k, 0, ny - 1), Xk = clampi(x + k, 0, nx - 1);
        gx += w[k + 1] * (s[xp + nx * Yk] - s[xm + nx * Yk]);
        gy += w[k + 1] * (s[Xk + nx * yp] - s[Xk + nx * ym]);
    }
    const long long ax = gx < 0 ? -gx : gx, ay = gy < 0 ? -gy : gy;
    int dx, dy;
    if (5 * ay < 2 * ax) {
        dx = gx > 0 ? 1 : -1;
        dy = 0;
    } else if (5 * ax < 2 * ay) {
        dx = 0;
        dy = gy > 0 ? 1 : -1;
    } else {
        dx = gx > 0 ? 1 : -1;
        dy = gy > 0 ? 1 : -1;
    }
    mag[v] = ax + ay;
    dir[v] = static_cast<uint8_t>((dx + 1) | ((dy + 1) << 2));
}

__global__ void __launch_bounds__(kVoxThreads) canny_nms_kernel(const long long *mag,
                                                                const uint8_t *dir, int nx, int ny,
                                                                int64_t V, uint8_t *nms)
{
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    const int64_t z = v / plane;
    const int j = static_cast<int>(v - z * plane);
    const int y = j / nx, x = j - y * nx;
    const long long *mg = mag + z * plane;
    const int d = dir[v];
    const int dx = (d & 3) - 1, dy = (d >> 2) - 1;
    long long fwd = 0, bwd = 0;  // along and against the gradient
    if (x + dx >= 0 && x + dx < nx && y + dy >= 0 && y + dy < ny) fwd = mg[(x + dx) + nx * (y + dy)];
    if (x - dx >= 0 && x - dx < nx && y - dy >= 0 && y - dy < ny) bwd = mg[(x - dx) + nx * (y - dy)];
    const long long m = mg[j];
    nms[v] = (m > 0 && m >= bwd && m > fwd) ? 1 : 0;
}

// Horizontal dilation of row word k by one voxel, across word boundaries.
__device__ __forceinline__ uint32_t hdilate(const uint32_t *E, int k, int w, int rw)
{
    const uint32_t e = E[k];
    uint32_t g = e | (e << 1) | (e >> 1);
    if (w > 0) g |= E[k - 1] >> 31;
    if (w + 1 < rw) g |= E[k + 1] << 31;
    return g;
}

__device__ __forceinline__ uint32_t fill_runs(uint32_t g, uint32_t p)
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

__device__ __forceinline__ long long block_sum(long long v, long long *s_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    long long t = 0;
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t += s_red[k];
    __syncthreads();
    return t;  // in every thread
}

__device__ __forceinline__ long long block_max(long long v, long long *s_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    long long t = 0;
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t = max(t, s_red[k]);
    __syncthreads();
    return t;  // in every thread
}

__global__ void __launch_bounds__(kSliceThreads) canny_slice_kernel(
    const uint32_t *M, const long long *mag, const uint8_t *nms, int nx, int ny, int rw, int q_pct,
    uint32_t *mt, uint8_t *has_edge, uint8_t *H3)
{
    extern __shared__ uint32_t s_bits[];
    __shared__ long long s_red[32];
    uint32_t *W = s_bits;           // weak voxels
    uint32_t *E = s_bits + ny * rw;  // edge voxels found so far
    const int z = blockIdx.x;
    const int64_t plane = static_cast<int64_t>(nx) * ny;
    const uint32_t *m = M + z * plane;
    const long long *mg = mag + z * plane;
    const uint8_t *nm = nms + z * plane;
    // the slice's largest suppressed magnitude
    long long mloc = 0;
    for (int64_t j = threadIdx.x; j < plane; j += blockDim.x)
        if (nm[j]) mloc = max(mloc, mg[j]);
    const long long mmax = block_max(mloc, s_red);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int words = ny * rw;
    for (int k = warp; k < words; k += nwarps) {  // a warp per word: one ballot each
        const int y = k / rw, x = (k - y * rw) * 32 + lane;
        bool weak = false, strong = false;
        if (x < nx && mmax > 0) {
            const int64_t j = static_cast<int64_t>(y) * nx + x;
            if (nm[j]) {
                const long long a = mg[j];
                weak = 5 * a >= mmax;
                strong = 2 * a >= mmax;
            }
        }
        const uint32_t wb = __ballot_sync(0xffffffffu, weak);
        const uint32_t sb = __ballot_sync(0xffffffffu, strong);
        if (lane == 0) {
            W[k] = wb;
            E[k] = sb;
        }
    }
    __syncthreads();
    // hysteresis: grow the strong voxels through weak ones, 8-connected;
    // each sweep that changes adds a voxel, so at most nx ny + 1 run
    for (long long it = 0; it < plane + 1; ++it) {
        int changed = 0;
        for (int k = threadIdx.x; k < words; k += blockDim.x) {
            const int y = k / rw, w = k - y * rw;
            uint32_t g = hdilate(E, k, w, rw);
            if (y > 0) g |= hdilate(E, k - rw, w, rw);
            if (y + 1 < ny) g |= hdilate(E, k + rw, w, rw);
            const uint32_t e = E[k];
            const uint32_t ne = fill_runs(g & W[k], W[k]) | e;
            if (ne != e) {
                E[k] = ne;
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
    }
    // the edge voxels' M values, listed in shared memory when they fit
    __shared__ int s_n;
    uint32_t *L = s_bits + 2 * words;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < words; k += blockDim.x) {
        const int y = k / rw, x0 = (k - y * rw) * 32;
        for (uint32_t bits = E[k]; bits != 0; bits &= bits - 1u) {
            const int slot = atomicAdd(&s_n, 1);
            if (slot < kListCap) L[slot] = m[static_cast<int64_t>(y) * nx + x0 + __ffs(bits) - 1];
        }
    }
    __syncthreads();
    const long long kedge = s_n;
    uint8_t *h = H3 + static_cast<int64_t>(z) * plane;
    if (kedge == 0) {
        for (int64_t j = threadIdx.x; j < plane; j += blockDim.x) h[j] = 0;
        if (threadIdx.x == 0) {
            mt[z] = 0;
            has_edge[z] = 0;
        }
        return;
    }
    // the element of rank t among the edge voxels' M: radix select, MSB first
    // (over the list, or over the edge bitmap when the list overflowed)
    const bool listed = kedge <= kListCap;
    long long t = (static_cast<long long>(q_pct) * (kedge - 1)) / 100;
    uint32_t prefix = 0;
    for (int b = 31; b >= 0; --b) {
        const uint32_t hi_mask = b == 31 ? 0u : ~((2u << b) - 1u);  // bits above b
        long long c = 0;
        if (listed) {
            for (int i = threadIdx.x; i < kedge; i += blockDim.x) {
                const uint32_t v = L[i];
                c += ((v & hi_mask) == prefix && !((v >> b) & 1u)) ? 1 : 0;
            }
        } else {
            for (int k = threadIdx.x; k < words; k += blockDim.x) {
                const int y = k / rw, x0 = (k - y * rw) * 32;
                for (uint32_t bits = E[k]; bits != 0; bits &= bits - 1u) {
                    const uint32_t v = m[static_cast<int64_t>(y) * nx + x0 + __ffs(bits) - 1];
                    c += ((v & hi_mask) == prefix && !((v >> b) & 1u)) ? 1 : 0;
                }
            }
        }
        const long long zeros = block_sum(c, s_red);
        if (t >= zeros) {
            t -= zeros;
            prefix |= 1u << b;
        }
    }
    for (int64_t j = threadIdx.x; j < plane; j += blockDim.x) h[j] = m[j] >= prefix ? 1 : 0;
    if (threadIdx.x == 0) {
        mt[z] = prefix;
        has_edge[z] = 1;
    }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

bool layout(int32_t nx, int32_t ny, int32_t nz, void *base, CannyWs *ws, size_t *bytes)
{
    const size_t V = static_cast<size_t>(nx) * ny * nz;
    size_t off = 0;
    const size_t oS = off;
    off += align256(8 * V);
    const size_t oM = off;
    off += align256(8 * V);
    const size_t oD = off;
    off += align256(V);
    const size_t oN = off;
    off += align256(V);
    if (bytes) *bytes = off;
    if (ws && base) {
        char *p = static_cast<char *>(base);
        ws->S = reinterpret_cast<long long *>(p + oS);
        ws->mag = reinterpret_cast<long long *>(p + oM);
        ws->dir = reinterpret_cast<uint8_t *>(p + oD);
        ws->nms = reinterpret_cast<uint8_t *>(p + oN);
    }
    return true;
}

hd_status check_dims(int32_t nx, int32_t ny, int32_t nz)
{
    if (nx < 1 || ny < 1 || nz < 1) return HD_ERR_ARG;
    if (static_cast<int64_t>(nx) * ny * nz > (int64_t(1) << 31)) return HD_ERR_RANGE;
    if (static_cast<int64_t>((nx + 31) / 32) * ny > kMaxWords) return HD_ERR_RANGE;
    return HD_OK;
}

}  // namespace

extern "C" {

hd_status hd_sm_canny_workspace(int32_t nx, int32_t ny, int32_t nz, size_t *bytes)
{
    if (!bytes) return HD_ERR_ARG;
    const hd_status s = check_dims(nx, ny, nz);
    if (s != HD_OK) return s;
    layout(nx, ny, nz, nullptr, nullptr, bytes);
    return HD_OK;
}

hd_status hd_sm_canny(const uint32_t *M, int32_t nx, int32_t ny, int32_t nz, int32_t q_pct,
                      void *workspace, size_t workspace_bytes, uint32_t *mt, uint8_t *has_edge,
                      uint8_t *H3, void *stream)
{
    if (!M || !workspace || !mt || !has_edge || !H3) return HD_ERR_ARG;
    if (q_pct < 0 || q_pct > 100) return HD_ERR_ARG;
    const hd_status s = check_dims(nx, ny, nz);
    if (s != HD_OK) return s;
    size_t need = 0;
    CannyWs ws{};
    layout(nx, ny, nz, workspace, &ws, &need);
    if (workspace_bytes < need) return HD_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return HD_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t V = static_cast<int64_t>(nx) * ny * nz;
    const unsigned blocks = static_cast<unsigned>((V + kVoxThreads - 1) / kVoxThreads);
    const int rw = (nx + 31) / 32;
    cudaError_t e = cudaSuccess;
    {
        canny_smooth_kernel<<<blocks, kVoxThreads, 0, st>>>(M, nx, ny, V, ws.S);
        canny_gradient_kernel<<<blocks, kVoxThreads, 0, st>>>(ws.S, nx, ny, V, ws.mag, ws.dir);
        canny_nms_kernel<<<blocks, kVoxThreads, 0, st>>>(ws.mag, ws.dir, nx, ny, V, ws.nms);
        e = cudaFuncSetAttribute(canny_slice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(sizeof(uint32_t) * (2 * kMaxWords + kListCap)));
    }
    if (e == cudaSuccess) {
        canny_slice_kernel<<<nz, kSliceThreads, sizeof(uint32_t) * (2 * rw * ny + kListCap), st>>>(
            M, ws.mag, ws.nms, nx, ny, rw, q_pct, mt, has_edge, H3);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        hd::note_cuda_error(e, "hd_sm_canny");
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // extern "C"
