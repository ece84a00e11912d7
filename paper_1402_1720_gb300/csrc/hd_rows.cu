// Rows of the hull-restricted system matrix: for each history, the voxels of
// its path A_i that lie inside a hull, in the order the path meets them.
// The hull's bitmap sits in each block's shared memory when it fits, so the
// per-voxel hull test is a shared-memory read.  The
// hull exists to shrink the unknowns of the reconstruction to these voxels
// (Sec. 1); the rows are what an iterative solver reads.  Two passes over
// the histories (count, then emit into CSR offsets from an exclusive scan),
// each walking the path with the exact run walk over the whole grid.
#include "hd_geom.cuh"
#include "hd_rows.cuh"

namespace hd {

namespace {

constexpr int kRowsThreads = 1024;  // one block per SM when the hull sits in shared memory
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

// Grid endpoints of history i (false when rejected), with the gantry
// cos/sin of the last angle this thread saw kept for reuse.
struct RowsTrig {
    bool valid = false;
    float ang = 0.0f;
    long long c = 0, s = 0;
};

__device__ __forceinline__ bool row_endpoints(const Inputs &in, int64_t i, const GeomQ &g,
                                              const Cordic &cd, RowsTrig &tc, int32_t r[6])
{
    const float ang = in.angle[i];
    if (!(fabsf(ang) < 1048576.0f)) return false;
    if (!tc.valid || ang != tc.ang) {
        cordic_cs(q16_of(ang), cd, tc.c, tc.s);
        tc.ang = ang;
        tc.valid = true;
    }
    return endpoints_cs(g, tc.c, tc.s, in.u_in[i], in.v_in[i], in.u_out[i], in.v_out[i], r);
}

// The hull as a bitmap (voxel v at bit v & 31 of word v >> 5), in shared
// memory when it fits there, else read as bytes from global memory.
template <bool kBits>
struct HullTest {
    const uint8_t *bytes;
    const uint32_t *bits;
    __device__ __forceinline__ bool operator()(uint32_t v) const
    {
        if (kBits) return (bits[v >> 5] >> (v & 31u)) & 1u;
        return bytes[v] != 0;
    }
};

template <bool kBits>
struct CountInHull {
    HullTest<kBits> in;
    int64_t count;
    __device__ __forceinline__ void operator()(uint32_t v) { count += in(v) ? 1 : 0; }
};

template <bool kBits>
struct EmitInHull {
    HullTest<kBits> in;
    int32_t *out;
    __device__ __forceinline__ void operator()(uint32_t v)
    {
        if (in(v)) *out++ = static_cast<int32_t>(v);
    }
};

// Copies the packed hull (words 32-bit words) into shared memory.
__device__ __forceinline__ void stage_hull(uint32_t *s_bits, const uint32_t *bits, int64_t words)
{
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) s_bits[w] = __ldg(bits + w);
    __syncthreads();
}

template <bool kBits>
__global__ void __launch_bounds__(kRowsThreads) rows_count_kernel(Inputs in, int64_t n, GeomQ g,
                                                                  Cordic cd, const uint8_t *hull,
                                                                  const uint32_t *hull_bits,
                                                                  int64_t words, int64_t *row_ptr)
{
    extern __shared__ uint32_t s_bits[];
    if (kBits) stage_hull(s_bits, hull_bits, words);
    RowsTrig tc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        int32_t r[6];
        CountInHull<kBits> c{{hull, s_bits}, 0};
        if (row_endpoints(in, i, g, cd, tc, r)) walk_path(r, g.nx, g.ny, g.nz, c);
        row_ptr[i + 1] = c.count;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[0] = 0;
}

template <bool kBits>
__global__ void __launch_bounds__(kRowsThreads) rows_emit_kernel(Inputs in, int64_t n, GeomQ g,
                                                                 Cordic cd, const uint8_t *hull,
                                                                 const uint32_t *hull_bits,
                                                                 int64_t words,
                                                                 const int64_t *row_ptr,
                                                                 int32_t *cols)
{
    extern __shared__ uint32_t s_bits[];
    if (kBits) stage_hull(s_bits, hull_bits, words);
    RowsTrig tc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        int32_t r[6];
        EmitInHull<kBits> e{{hull, s_bits}, cols + row_ptr[i]};
        if (row_endpoints(in, i, g, cd, tc, r)) walk_path(r, g.nx, g.ny, g.nz, e);
    }
}

// Inclusive block scan of int64 values: `v` is this thread's value; returns
// its inclusive prefix, *total the block's sum.
__device__ __forceinline__ long long block_incl_scan64(long long v, long long *s_warp,
                                                       long long &total)
{
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<unsigned>(o)) x += t;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        long long y = lane < static_cast<unsigned>(nw) ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= static_cast<unsigned>(o)) y += t;
        }
        if (lane < static_cast<unsigned>(nw)) s_warp[lane] = y;
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    const long long before = warp > 0 ? s_warp[warp - 1] : 0;
    __syncthreads();
    return before + x;
}

// Tile b of kScanTile values: inclusive scan in place, its sum to sums[b].
__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(int64_t *a, int64_t n,
                                                                  int64_t *sums)
{
    __shared__ long long s_warp[32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile +
                         static_cast<int64_t>(threadIdx.x) * kScanPerThread;
    long long v[kScanPerThread];
    long long acc = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        v[k] = base + k < n ? a[base + k] : 0;
        acc += v[k];
        v[k] = acc;
    }
    long long total;
    const long long before = block_incl_scan64(acc, s_warp, total) - acc;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k)
        if (base + k < n) a[base + k] = before + v[k];
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums, kScanThreads at a time.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int64_t *sums, int64_t nb)
{
    __shared__ long long s_warp[32];
    long long carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const long long v = i < nb ? sums[i] : 0;
        long long total;
        const long long incl = block_incl_scan64(v, s_warp, total);
        if (i < nb) sums[i] = carry + incl - v;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_add_kernel(int64_t *a, int64_t n,
                                                                const int64_t *offsets)
{
    const long long off = offsets[blockIdx.x];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
    for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
        const int64_t i = base + k;
        if (i < n) a[i] += off;
    }
}

int64_t grid_for(int64_t n, int sm_count, bool bits)
{
    int64_t blocks = (n + kRowsThreads - 1) / kRowsThreads;
    const int64_t cap = static_cast<int64_t>(sm_count > 0 ? sm_count : 1) * (bits ? 1 : 2);
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : blocks;
}

constexpr int64_t kMaxHullWords = 48 * 1024;  // 192 KB of shared memory

template <class K>
cudaError_t allow_smem(K kernel)
{
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(sizeof(uint32_t) * kMaxHullWords));
}

}  // namespace

int64_t rows_scan_scratch(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

int64_t rows_hull_words(int64_t V) { return (V + 31) / 32; }

// hull_bits: the packed hull (rows_hull_words(V) words) or null; with it,
// when it fits, each block holds the hull in shared memory.
cudaError_t launch_rows_count(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cd,
                              const uint8_t *hull, const uint32_t *hull_bits, int64_t *row_ptr,
                              int sm_count, cudaStream_t s)
{
    const int64_t words = rows_hull_words(int64_t(g.nx) * g.ny * g.nz);
    if (hull_bits && words <= kMaxHullWords) {
        const cudaError_t e = allow_smem(rows_count_kernel<true>);
        if (e != cudaSuccess) return e;
        rows_count_kernel<true><<<static_cast<unsigned>(grid_for(n, sm_count, true)), kRowsThreads,
                                  sizeof(uint32_t) * words, s>>>(in, n, g, cd, hull, hull_bits,
                                                                 words, row_ptr);
    } else {
        rows_count_kernel<false><<<static_cast<unsigned>(grid_for(n, sm_count, false)),
                                   kRowsThreads, 0, s>>>(in, n, g, cd, hull, nullptr, 0, row_ptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_scan(int64_t *a, int64_t n, int64_t *scratch, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = rows_scan_scratch(n);
    scan_tiles_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(a, n, scratch);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(scratch, nb);
    scan_add_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, s>>>(a, n, scratch);
    return cudaGetLastError();
}

cudaError_t launch_rows_emit(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cd,
                             const uint8_t *hull, const uint32_t *hull_bits,
                             const int64_t *row_ptr, int32_t *cols, int sm_count, cudaStream_t s)
{
    const int64_t words = rows_hull_words(int64_t(g.nx) * g.ny * g.nz);
    if (hull_bits && words <= kMaxHullWords) {
        const cudaError_t e = allow_smem(rows_emit_kernel<true>);
        if (e != cudaSuccess) return e;
        rows_emit_kernel<true><<<static_cast<unsigned>(grid_for(n, sm_count, true)), kRowsThreads,
                                 sizeof(uint32_t) * words, s>>>(in, n, g, cd, hull, hull_bits,
                                                                words, row_ptr, cols);
    } else {
        rows_emit_kernel<false><<<static_cast<unsigned>(grid_for(n, sm_count, false)),
                                  kRowsThreads, 0, s>>>(in, n, g, cd, hull, nullptr, 0, row_ptr,
                                                        cols);
    }
    return cudaGetLastError();
}

}  // namespace hd
