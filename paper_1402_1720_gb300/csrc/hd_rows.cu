// Rows of the hull-restricted system matrix: for each history, the voxels of
// its path A_i that lie inside a hull, in the order the path meets them.  The
// hull exists to shrink the unknowns of the reconstruction to these voxels
// (Sec. 1); the rows are what an iterative solver reads.  Two passes over
// the histories (count, then emit into CSR offsets from an exclusive scan),
// each walking the path with the exact run walk over the whole grid.
#include "hd_geom.cuh"

namespace hd {

namespace {

constexpr int kRowsThreads = 256;
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

struct CountInHull {
    const uint8_t *hull;
    int64_t count;
    __device__ __forceinline__ void operator()(uint32_t v) { count += hull[v] != 0 ? 1 : 0; }
};

struct EmitInHull {
    const uint8_t *hull;
    int32_t *out;
    __device__ __forceinline__ void operator()(uint32_t v)
    {
        if (hull[v] != 0) *out++ = static_cast<int32_t>(v);
    }
};

__global__ void __launch_bounds__(kRowsThreads) rows_count_kernel(Inputs in, int64_t n, GeomQ g,
                                                                  Cordic cd, const uint8_t *hull,
                                                                  int64_t *row_ptr)
{
    RowsTrig tc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        int32_t r[6];
        CountInHull c{hull, 0};
        if (row_endpoints(in, i, g, cd, tc, r)) walk_path(r, g.nx, g.ny, g.nz, c);
        row_ptr[i + 1] = c.count;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[0] = 0;
}

__global__ void __launch_bounds__(kRowsThreads) rows_emit_kernel(Inputs in, int64_t n, GeomQ g,
                                                                 Cordic cd, const uint8_t *hull,
                                                                 const int64_t *row_ptr,
                                                                 int32_t *cols)
{
    RowsTrig tc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        int32_t r[6];
        EmitInHull e{hull, cols + row_ptr[i]};
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

int64_t grid_for(int64_t n, int sm_count)
{
    int64_t blocks = (n + kRowsThreads - 1) / kRowsThreads;
    const int64_t cap = static_cast<int64_t>(sm_count > 0 ? sm_count : 1) * 8;
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : blocks;
}

}  // namespace

int64_t rows_scan_scratch(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t launch_rows_count(const Inputs &in, int64_t n, const GeomQ &g, const Cordic &cd,
                              const uint8_t *hull, int64_t *row_ptr, int sm_count, cudaStream_t s)
{
    rows_count_kernel<<<static_cast<unsigned>(grid_for(n, sm_count)), kRowsThreads, 0, s>>>(
        in, n, g, cd, hull, row_ptr);
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
                             const uint8_t *hull, const int64_t *row_ptr, int32_t *cols,
                             int sm_count, cudaStream_t s)
{
    rows_emit_kernel<<<static_cast<unsigned>(grid_for(n, sm_count)), kRowsThreads, 0, s>>>(
        in, n, g, cd, hull, row_ptr, cols);
    return cudaGetLastError();
}

}  // namespace hd
