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
// memory when it fits there, else read as bytes from global memory; and the
// hull voxels of one run of a path.  A run along x covers consecutive bits
// (v = nx row + m): with the bitmap they are counted by population counts
// of its words and listed from its set bits; a run along y has stride nx.
template <bool kBits>
struct HullRuns {
    const uint8_t *bytes;
    const uint32_t *bits;
    int nx, ny;

    __device__ __forceinline__ bool test(uint32_t v) const
    {
        if (kBits) return (bits[v >> 5] >> (v & 31u)) & 1u;
        return bytes[v] != 0;
    }

    // first voxel and stride of run row (the major axis' layout: y + ny z
    // along x, x + nx z along y)
    __device__ __forceinline__ void frame(bool ymaj, int row, uint32_t &base,
                                          uint32_t &stride) const
    {
        if (!ymaj) {
            base = static_cast<uint32_t>(nx) * static_cast<uint32_t>(row);
            stride = 1;
        } else {
            const int z = static_cast<int>(fdiv_small(row, nx));
            base = static_cast<uint32_t>(row - z * nx) +
                   static_cast<uint32_t>(nx) * static_cast<uint32_t>(ny) * static_cast<uint32_t>(z);
            stride = static_cast<uint32_t>(nx);
        }
    }

    // number of hull voxels of the run
    __device__ __forceinline__ int count(bool ymaj, int row, int lo, int hi) const
    {
        uint32_t base, stride;
        frame(ymaj, row, base, stride);
        if (kBits && !ymaj) {
            const uint32_t s = base + lo, e = base + hi;
            const uint32_t ws = s >> 5, we = e >> 5;
            const uint32_t ml = ~0u << (s & 31u), mh = ~0u >> (31u - (e & 31u));
            if (ws == we) return __popc(bits[ws] & ml & mh);
            int c = __popc(bits[ws] & ml) + __popc(bits[we] & mh);
            for (uint32_t w = ws + 1; w < we; ++w) c += __popc(bits[w]);
            return c;
        }
        int c = 0;
        for (int m = lo; m <= hi; ++m) c += test(base + stride * static_cast<uint32_t>(m)) ? 1 : 0;
        return c;
    }

    // writes the run's hull voxels to out in path order (m rising when up)
    __device__ __forceinline__ int32_t *emit(bool ymaj, bool up, int row, int lo, int hi,
                                             int32_t *out) const
    {
        uint32_t base, stride;
        frame(ymaj, row, base, stride);
        if (kBits && !ymaj) {
            const uint32_t s = base + lo, e = base + hi;
            const int ws = static_cast<int>(s >> 5), we = static_cast<int>(e >> 5);
            const uint32_t ml = ~0u << (s & 31u), mh = ~0u >> (31u - (e & 31u));
            if (up) {
                for (int w = ws; w <= we; ++w) {
                    uint32_t b = bits[w] & (w == ws ? ml : ~0u) & (w == we ? mh : ~0u);
                    while (b) {
                        *out++ = static_cast<int32_t>((static_cast<uint32_t>(w) << 5) +
                                                      static_cast<uint32_t>(__ffs(b) - 1));
                        b &= b - 1u;
                    }
                }
            } else {
                for (int w = we; w >= ws; --w) {
                    uint32_t b = bits[w] & (w == ws ? ml : ~0u) & (w == we ? mh : ~0u);
                    while (b) {
                        const int j = 31 - __clz(b);
                        *out++ = static_cast<int32_t>((static_cast<uint32_t>(w) << 5) +
                                                      static_cast<uint32_t>(j));
                        b ^= 1u << j;
                    }
                }
            }
            return out;
        }
        for (int k = 0; k <= hi - lo; ++k) {
            const uint32_t v = base + stride * static_cast<uint32_t>(up ? lo + k : hi - k);
            if (test(v)) *out++ = static_cast<int32_t>(v);
        }
        return out;
    }
};

// Copies the packed hull (words 32-bit words) into shared memory.
__device__ __forceinline__ void stage_hull(uint32_t *s_bits, const uint32_t *bits, int64_t words)
{
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) s_bits[w] = __ldg(bits + w);
    __syncthreads();
}

// Every lane walks its history's path as runs of the whole-grid run walk
// (one loop for all lanes; the runs come in path order, each expanded in
// the direction the major axis moves).
template <bool kBits>
__global__ void __launch_bounds__(kRowsThreads) rows_count_kernel(Inputs in, int64_t n, GeomQ g,
                                                                  Cordic cd, const uint8_t *hull,
                                                                  const uint32_t *hull_bits,
                                                                  int64_t words, int64_t *row_ptr)
{
    extern __shared__ uint32_t s_bits[];
    if (kBits) stage_hull(s_bits, hull_bits, words);
    const HullRuns<kBits> h{hull, s_bits, g.nx, g.ny};
    RowsTrig tc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        int32_t r[6];
        int64_t count = 0;
        RunWalk w;
        if (row_endpoints(in, i, g, cd, tc, r) && run_begin(w, r, r + 3, g.nx, g.ny, g.nz)) {
            const bool ymaj = (w.flags >> 5) & 1;
            int row, lo, hi;
            while (run_next(w, row, lo, hi)) count += h.count(ymaj, row, lo, hi);
        }
        row_ptr[i + 1] = count;
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
    const HullRuns<kBits> h{hull, s_bits, g.nx, g.ny};
    RowsTrig tc;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        int32_t r[6];
        RunWalk w;
        if (row_endpoints(in, i, g, cd, tc, r) && run_begin(w, r, r + 3, g.nx, g.ny, g.nz)) {
            const bool ymaj = (w.flags >> 5) & 1, up = w.flags & 1;
            int32_t *out = cols + row_ptr[i];
            int row, lo, hi;
            while (run_next(w, row, lo, hi)) out = h.emit(ymaj, up, row, lo, hi, out);
        }
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
